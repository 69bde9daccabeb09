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


def test_cancelled_requests_neither_return_nor_block(server):
    """Requests cancelled before the run (cancel), by a deadline before
    their arrival, or from another thread while the loop runs: none returns
    a result, the others all complete, and a request's result is the same
    as without the cancellations."""
    import threading

    reqs = poisson_requests(np.random.default_rng(21), 40, 2000.0, 3, sizes=(128, 192),
                            grad_fraction=0.3)
    probe = reqs[7]
    alone, _ = server.run([Request(probe.rid, probe.scene, probe.camera, probe.want_grad, 0.0,
                                   probe.upstream)])
    gone = {3, 11, 25}
    for rid in gone:
        server.cancel(rid)
    reqs[30].deadline = reqs[30].arrival - 1e-3        # expired when it arrives
    late = max(reqs, key=lambda q: q.arrival)
    late.arrival += 0.2                                 # cancelled by a thread before it arrives
    t = threading.Timer(0.05, server.cancel, args=(late.rid,))
    t.start()
    res, stats = server.run(reqs)
    t.join()
    dropped = gone | {reqs[30].rid, late.rid}
    assert set(res) == {q.rid for q in reqs} - dropped
    assert stats["cancelled"] == len(dropped)
    a, b = alone[probe.rid], res[probe.rid]
    for u, v in ((a.image, b.image), (a.alpha, b.alpha), (a.depth, b.depth)):
        assert (u - v).abs().max().item() <= 1e-4


def test_bad_scene_fails_alone():
    """A resident scene with a tet index outside [0, N): batches holding its
    requests are split per scene, its requests fail with an error once they
    fail alone, and the other scenes' requests batched with them complete
    normally."""
    good = synth.scene_sphere16()
    bad = to_dev(good)
    srv = Server([to_dev(good), bad], Params(s=120.0, tile=16), hbm_budget=4e9, max_views=8,
                 streams=2, ref_res=128)
    bad.T[5, 2] = good.N + 7        # goes bad after registration: found in its batches
    reqs = poisson_requests(np.random.default_rng(4), 24, 5000.0, 2, sizes=(128,),
                            grad_fraction=0.3)
    res, stats = srv.run(reqs)
    assert set(res) == {q.rid for q in reqs}
    for q in reqs:
        r = res[q.rid]
        if q.scene == 1:
            assert r.error is not None and r.image is None
        else:
            assert r.error is None and r.alpha.max().item() > 0.5
    assert stats["failed"] == sum(q.scene == 1 for q in reqs) and 1 in srv.bad_scenes


def test_layout_reuse_matches_fresh_rasterizer(server):
    """Batches whose workspace layout repeats reuse the slot's rasterizer
    (rebound to other scenes of the same size and other cameras): the result
    equals a fresh render of the same request."""
    rng = np.random.default_rng(31)
    q0 = Request(0, 0, on_sphere(rng, 160, 160), False, 0.0)
    q1 = Request(1, 0, on_sphere(rng, 160, 160), False, 0.0)   # same layout, other camera
    r0, _ = server.run([q0])
    r1, _ = server.run([q1])
    fresh = Server(server.scenes, Params(s=120.0, tile=16), hbm_budget=4e9, max_views=8,
                   streams=1, ref_res=256)
    f1, _ = fresh.run([Request(1, 0, q1.camera, False, 0.0)])
    assert (r1[1].image - f1[1].image).abs().max().item() <= 1e-6
    assert (r0[0].alpha - r1[1].alpha).abs().max().item() > 0.0   # different cameras


def test_reserve_sizes_every_slot_and_keeps_results(server):
    """After reserve() every slot holds the largest workspace and buffer any
    slot had, and a request served afterwards equals one served by a fresh
    server."""
    rng = np.random.default_rng(41)
    reqs = [Request(i, i % len(server.scenes), on_sphere(rng, 128, 128), i % 2 == 0, 0.0,
                    upstream=_upstream(rng, 128) if i % 2 == 0 else None) for i in range(6)]
    server.run(reqs)
    server.reserve()
    ws = {sl.ws.numel() for sl in server.slots if sl.ws is not None}
    nf = {sl.dev.numel() for sl in server.slots if sl.dev is not None}
    assert len(ws) == 1 and len(nf) == 1 and len(server.slots) == 3
    assert all(sl.ws is not None and sl.dev is not None for sl in server.slots)
    q = Request(99, 1, on_sphere(rng, 160, 160), False, 0.0)
    r, _ = server.run([q])
    fresh = Server(server.scenes, Params(s=120.0, tile=16), hbm_budget=4e9, max_views=8,
                   streams=1, ref_res=256)
    f, _ = fresh.run([Request(99, 1, q.camera, False, 0.0)])
    assert (r[99].image - f[99].image).abs().max().item() <= 1e-6


def test_pinned_result_pool_reuses_freed_buffers():
    """Result buffers are pinned, of the requested size, and their storage is
    reused once every tensor on it is gone (not before)."""
    from paper_2406_01579_b300.serve import _PinnedPool
    pool = _PinnedPool()
    a = pool.get(1000)
    assert a.is_pinned() and a.numel() == 1000 and a.dtype == torch.float32
    view = a[10:20].view(2, 5)
    pa = a.data_ptr()
    del a
    b = pool.get(900)                 # the first buffer is still held by its view
    assert b.data_ptr() != pa
    del view
    c = pool.get(800)                 # now free: the same storage again
    assert c.data_ptr() == pa and c.numel() == 800 and c.is_pinned()
    d = torch.arange(800, dtype=torch.float32, device="cuda")
    c.copy_(d, non_blocking=True)
    torch.cuda.synchronize()
    assert torch.equal(c, d.cpu())
    big = pool.get(1 << 20)
    assert big.numel() == 1 << 20 and big.data_ptr() not in (pa, b.data_ptr())


def test_pinned_pool_top_up_allocates_ahead():
    from paper_2406_01579_b300.serve import _PinnedPool
    pool = _PinnedPool()
    held = [pool.get(3000) for _ in range(3)]          # three out at once
    del held
    pool.top_up(2.0, 100)
    cls = 1 << 16
    assert pool.out[cls] == 0 and len(pool.free[cls]) == 6
    pool.top_up(2.0, 4)                                 # the cap never shrinks the pool
    assert len(pool.free[cls]) == 6
    ptrs = {pool.get(100).data_ptr() for _ in range(1)}
    assert ptrs and all(p != 0 for p in ptrs)
