"""Host-fed training steps with overlapped copies (HostStepPipeline): every
step's gradients, read back to host memory, equal those of the same step run
alone on device copies of its own inputs, even with the inputs changing from
step to step (the two device buffer sets must never mix steps)."""

import numpy as np
import pytest
import torch

import synth
from paper_2406_01579_b300 import Params, Rasterizer, SceneTensors
from paper_2406_01579_b300.pipeline import HostStepPipeline
from parity import to_dev

pytestmark = pytest.mark.gpu


def _host_inputs(sc, cams, k):
    """Step k's inputs: the SDF shifted by 0.01 k, colours scaled, fresh
    upstream gradients."""
    f = (sc.f + np.float32(0.01 * k)).astype(np.float32)
    rgb = (sc.rgb * np.float32(1.0 - 0.05 * k)).astype(np.float32)
    ups = synth.upstream_grads(10 + k, cams)
    up = [np.concatenate([u[i].ravel() for u in ups]).astype(np.float32) for i in range(3)]
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    return (pin(sc.V), pin(f), pin(rgb)), [pin(x) for x in up]


def test_pipelined_steps_match_single_steps():
    sc = synth.scene_torus64(res=160)
    rng = np.random.default_rng(6)
    cams = [sc.cams[0], synth.random_camera(rng, 128, 96)]
    p = Params(s=60.0, tile=16)
    st = to_dev(sc)
    r = Rasterizer([st], [(c, 0) for c in cams], p)
    r.forward()
    r.shrink_to_fit(1.5)
    steps = 5
    inputs = [_host_inputs(sc, cams, k) for k in range(steps)]
    # reference: each step alone, synchronously
    ref = []
    for (hs, hu) in inputs:
        s_k = SceneTensors(hs[0].cuda(), st.T, hs[1].cuda(), hs[2].cuda())
        rk = Rasterizer([s_k], [(c, 0) for c in cams], p, key_capacity=r.key_capacity,
                        surv_capacity=r.surv_capacity)
        out = rk._outputs()
        g = [(torch.empty_like(s_k.V), torch.empty_like(s_k.f), torch.empty_like(s_k.rgb))]
        rk.step(out, [x.cuda() for x in hu], g)
        torch.cuda.synchronize()
        assert rk.info().status == 0
        ref.append([x.cpu() for x in g[0]])
    # pipelined: all steps enqueued back to back
    pipe = HostStepPipeline(r)
    outs = [[torch.empty_like(x).pin_memory() for x in ref[0]] for _ in range(steps)]
    pipe.begin()
    for k, (hs, hu) in enumerate(inputs):
        pipe.step([hs], hu, [outs[k]])
    pipe.end()
    torch.cuda.synchronize()
    assert r.info().status == 0
    for k in range(steps):
        for a, b in zip(ref[k], outs[k]):
            # float atomics sum in a different order from run to run: two lone
            # runs of one step differ by up to ~1e-6 of the tensor's maximum;
            # steps mixed up would differ at order 1
            err = float((a - b).abs().max()) / float(a.abs().max())
            assert err < 1e-5, (k, err)
    # the steps differ from one another (the inputs changed)
    assert not torch.allclose(ref[0][1], ref[1][1])
