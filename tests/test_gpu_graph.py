"""A whole step (pre-filter, forward, backward) captured in a CUDA graph
replays to the same results as the eager calls."""

import numpy as np
import pytest
import torch

import synth
from paper_2406_01579_b300 import Params, Rasterizer
from parity import to_dev

pytestmark = pytest.mark.gpu


def test_graph_replay_matches_eager():
    sc = synth.scene_sphere16()
    rng = np.random.default_rng(4)
    cams = [sc.cams[0], synth.random_camera(rng, 96, 80)]
    st = to_dev(sc)
    r = Rasterizer([st], [(c, 0) for c in cams], Params(s=60.0, tile=16))
    r.forward()
    r.shrink_to_fit(1.5)
    ups = synth.upstream_grads(3, cams)
    up = tuple(torch.from_numpy(np.concatenate([u[i].ravel() for u in ups])).cuda() for i in range(3))
    out = r._outputs()
    grads = [(torch.empty_like(st.V), torch.empty_like(st.f), torch.empty_like(st.rgb))]
    r.step(out, up, grads)
    torch.cuda.synchronize()
    ref = [x.clone() for x in out] + [g.clone() for g in grads[0]]
    g = r.capture_step(out, up, grads)
    for x in list(out) + list(grads[0]):
        x.zero_()
    g.replay()
    torch.cuda.synchronize()
    got = list(out) + list(grads[0])
    for a, b in zip(ref[:3], got[:3]):
        assert torch.equal(a, b)
    # float atomics: the summation order differs from run to run.  Two eager
    # steps differ by up to ~7e-7 of the largest entry where terms cancel
    # (with or without the per-pixel fragment lists), so the floor is 1e-5 of
    # it; a wrong replay would be off by O(1).
    for a, b in zip(ref[3:], got[3:]):
        assert torch.allclose(a, b, rtol=1e-5, atol=1e-5 * float(a.abs().max()))
    # inputs updated in place are picked up by the next replay
    st.f.add_(0.01)
    g.replay()
    torch.cuda.synchronize()
    r2 = Rasterizer([st], [(c, 0) for c in cams], Params(s=60.0, tile=16))
    img2, _, _ = r2.forward()
    assert torch.equal(out[0], img2)
    assert r.info().status == 0
