"""The two ways to run the backward give the same vertex gradients: the
render backward (the blend backward's warps clear the gradient arrays when
their queue is empty, then the record -> vertex scatter) and the split calls
(blend backward, then the scatter with its own clearing).  Gradients are
overwritten in full unless TTS_FLAG_ACCUM_GRAD is set, which adds to them."""

import ctypes
import dataclasses

import numpy as np
import pytest
import torch

import synth
from paper_2406_01579_b300 import Params, Rasterizer, _lib
from parity import to_dev

pytestmark = pytest.mark.gpu


def _setup(params, n_scenes=2):
    rng = np.random.default_rng(11)
    scenes = [synth.scene_sphere16(), synth.scene_torus64(res=96)][:n_scenes]
    views = [(scenes[0].cams[0], 0), (synth.random_camera(rng, 80, 64), 0)]
    if n_scenes > 1:
        views.append((scenes[1].cams[0], 1))
    st = [to_dev(s) for s in scenes]
    r = Rasterizer(st, views, params)
    r.forward()
    ups = synth.upstream_grads(5, [c for c, _ in views])
    up = [torch.from_numpy(np.concatenate([u[i].ravel() for u in ups])).cuda() for i in range(3)]
    return r, st, up


def _grads(st, fill):
    return [(torch.full_like(s.V, fill), torch.full_like(s.f, fill), torch.full_like(s.rgb, fill))
            for s in st]


def _rel(a, b):
    return float((a - b).abs().max()) / max(float(a.abs().max()), 1e-30)


def _split_backward(r, up, grads):
    L = r.lib
    b = r.batch()
    u = r._c_upstream(up)
    n = len(r.scenes)
    dV = (ctypes.c_void_p * n)(*[g[0].data_ptr() for g in grads])
    df = (ctypes.c_void_p * n)(*[g[1].data_ptr() for g in grads])
    dc = (ctypes.c_void_p * n)(*[g[2].data_ptr() for g in grads])
    sp = torch.cuda.current_stream().cuda_stream
    _lib.check(L.tts_blend_bwd_ex(ctypes.byref(b), ctypes.byref(u), sp))
    _lib.check(L.tts_scatter_bwd(ctypes.byref(b), dV, df, dc, sp))


def test_render_backward_matches_split_calls_and_overwrites():
    r, st, up = _setup(Params(s=60.0, tile=8))
    fused = r.backward(*up, grads=_grads(st, float("nan")))   # stale NaNs must all go
    split = _grads(st, float("nan"))
    _split_backward(r, up, split)
    torch.cuda.synchronize()
    assert r.info().status == 0
    for gf, gs in zip(fused, split):
        for a, b in zip(gf, gs):
            assert torch.isfinite(a).all() and torch.isfinite(b).all()
            assert float(a.abs().max()) > 0
            assert _rel(a, b) < 1e-5


def test_accum_grad_adds_to_the_buffers():
    p = Params(s=60.0, tile=8)
    r, st, up = _setup(p)
    ref = r.backward(*up, grads=_grads(st, 0.0))
    ra = Rasterizer(st, r.views, dataclasses.replace(p, accum_grad=True))
    ra.forward()
    acc = _grads(st, 1.5)
    ra.backward(*up, grads=acc)
    ra.backward(*up, grads=acc)
    torch.cuda.synchronize()
    for gr, ga in zip(ref, acc):
        for a, b in zip(gr, ga):
            assert _rel(2.0 * a + 1.5, b) < 1e-5
