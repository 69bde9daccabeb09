"""Continuous-batching server: each result is the same alone and in a mix of
concurrent requests (images 1e-4, gradients 1e-3 relative); batches overlap
on the device; admission respects the HBM budget."""

import numpy as np
import pytest
import torch

import synth
from paper_2406_01579_b300 import Params
from paper_2406_01579_b300.camera import on_sphere, orbit
from paper_2406_01579_b300.serve import Request, Server, poisson_requests
from parity import to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def server():
    rng = np.random.default_rng(7)
    scenes = [to_dev(synth.scene_sphere16())]
    for n, kind in ((12, "torus"), (20, "sphere")):
        V, T, f, rgb = synth.random_scene(rng, n, kind)
        scenes.append(to_dev((V, T, f, rgb)))
    return Server(scenes, Params(s=120.0, tile=16), hbm_budget=4e9, max_views=8, streams=3,
                  ref_res=256)


def _upstream(rng, res):
    return (rng.normal(size=(3, res, res)).astype(np.float32),
            rng.normal(size=(res, res)).astype(np.float32),
            rng.normal(size=(res, res)).astype(np.float32))


def test_result_alone_equals_result_in_mix(server):
    rng = np.random.default_rng(11)
    x_fwd = Request(0, 1, orbit(40.0, 10.0, 192, 192), False, 0.0)
    x_grad = Request(1, 2, orbit(-20.0, 30.0, 160, 160), True, 0.0, _upstream(rng, 160))
    alone_f, _ = server.run([x_fwd])
    alone_g, _ = server.run([x_grad])
    mix = poisson_requests(np.random.default_rng(3), 40, 4000.0, 3, sizes=(128, 192, 256),
                           grad_fraction=0.4, start=0.0)
    for i, q in enumerate(mix):
        q.rid = 100 + i
    x_fwd.arrival = x_grad.arrival = mix[5].arrival
    res, stats = server.run(mix + [x_fwd, x_grad])
    assert stats["batches"] < len(mix) + 2          # requests were batched
    assert res[0].batch_views > 1 or res[1].batch_views > 1
    for a, b in ((alone_f[0], res[0]), (alone_g[1], res[1])):
        for u, v in ((a.image, b.image), (a.alpha, b.alpha), (a.depth, b.depth)):
            assert (u - v).abs().max().item() <= 1e-4
    ga, gb = alone_g[1].grads, res[1].grads
    for u, v in zip(ga, gb):
        u, v = u.cpu().numpy(), v.cpu().numpy()
        assert np.abs(u - v).max() <= 1e-3 * max(np.abs(u).max(), 1e-30)
    assert len(res) == len(mix) + 2


def test_batches_overlap_and_budget(server):
    reqs = poisson_requests(np.random.default_rng(5), 60, 20000.0, 3, sizes=(256,),
                            grad_fraction=0.3)
    res, stats = server.run(reqs)
    assert len(res) == 60
    assert stats["max_inflight"] >= 2                # several batches on the device at once
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    small = Server(server.scenes, Params(s=120.0, tile=16), hbm_budget=1.0, max_views=8,
                   streams=3, ref_res=256)
    res2, stats2 = small.run(reqs[:10])
    assert len(res2) == 10 and stats2["max_inflight"] == 1   # budget admits one batch at a time
