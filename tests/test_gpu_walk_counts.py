"""TTS_FLAG_COUNT: the blend kernels' walk statistics change nothing in the
result, are zero without the flag, and are consistent with each other."""

import numpy as np
import pytest
import torch

import synth
from paper_2406_01579_b300 import Params, Rasterizer
from parity import to_dev

pytestmark = pytest.mark.gpu


def _step(sc, cams, p, up):
    st = to_dev(sc)
    r = Rasterizer([st], [(c, 0) for c in cams], p)
    out = r.forward()
    r.debug_walk_counts(reset=True)
    gi, ga, gd = (torch.from_numpy(np.concatenate([u[i].ravel() for u in up])).cuda()
                  for i in range(3))
    out = r.forward()
    g = r.backward(gi, ga, gd)
    torch.cuda.synchronize()
    return r, [x.clone() for x in out], [x.clone() for x in g[0]]


@pytest.mark.parametrize("frag_cap", [0, 2])
def test_counting_changes_nothing(frag_cap):
    sc = synth.scene_sphere16()
    cams = [sc.cams[0], synth.orbit_camera(-40.0, 25.0, 96, 80)]
    up = synth.upstream_grads(9, cams)
    p = Params(s=175.0, tile=8, blend_segment=64, frag_cap=frag_cap)
    r0, out0, g0 = _step(sc, cams, p, up)
    assert all(v == 0 for v in r0.debug_walk_counts().values())   # no flag: nothing counted
    r1, out1, g1 = _step(sc, cams, Params(s=175.0, tile=8, blend_segment=64, frag_cap=frag_cap,
                                          count_walk=True), up)
    for a, b in zip(out0, out1):
        assert torch.equal(a, b)
    for a, b in zip(g0, g1):   # float atomics: summation order only
        assert torch.allclose(a, b, rtol=1e-5, atol=1e-5 * float(a.abs().max()))
    w = r1.debug_walk_counts()
    assert w["fwd_groups"] > 0 and 0 < w["fwd_candidates"] <= 32 * w["fwd_groups"]
    assert w["fwd_blocks"] > 0
    assert w["bwd_candidates"] <= 32 * w["bwd_groups"]
    lists = r1.debug_frag_lists()
    over = int((lists[1] > lists[3]).sum().item())
    if frag_cap == 0:
        assert over == 0 and w["bwd_groups"] == 0      # every pixel from its list
    else:
        assert over > 0 and w["bwd_groups"] > 0        # the list walk takes the rest
    assert all(v == 0 for v in r1.debug_walk_counts().values())   # reset by the last read
