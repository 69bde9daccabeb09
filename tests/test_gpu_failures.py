"""Failure handling on the device, without faulting the GPU: the tile scan's
bounded look-back wait is made to run out (one scan block polls a word that
no block publishes, with a short poll limit), and the library must report
TTS_STATUS_TIMEOUT, keep every kernel in bounds (the forward uses no key), and
recover on the next forward once the hook is off."""

import numpy as np
import pytest
import torch

import synth
from paper_2406_01579_b300 import Params, Rasterizer, TetsError, _lib
from parity import to_dev

pytestmark = pytest.mark.gpu


def test_scan_wait_timeout_is_reported_and_recovers():
    L = _lib.load()
    sc = synth.scene_sphere16()
    rng = np.random.default_rng(8)
    cams = [synth.random_camera(rng, 512, 512) for _ in range(4)]
    p = Params(s=175.0, tile=8)      # 4 x 4,096 tiles: eight scan blocks of 2,048
    r = Rasterizer([to_dev(sc)], [(c, 0) for c in cams], p)
    ref = [x.clone() for x in r.forward()]
    assert float(ref[1].max()) > 0.5
    try:
        assert L.tts_debug_scan_wait(256, 3) == _lib.TTS_OK
        with pytest.raises(TetsError, match="gave up"):
            r.forward()
        assert r.info().status & _lib.TTS_STATUS_TIMEOUT
        img, alpha, depth = r.forward(check_status=False)
        torch.cuda.synchronize()
        assert r.info().status & _lib.TTS_STATUS_TIMEOUT
        # the forward used no key: the outputs are those of an empty scene
        assert float(alpha.abs().max()) == 0.0 and float(img.abs().max()) == 0.0
        # a backward after it reads no list either
        gi, ga, gd = (torch.ones_like(x) for x in (img, alpha, depth))
        (dV, df, drgb), = r.backward(gi, ga, gd)
        torch.cuda.synchronize()
        assert float(dV.abs().max()) == 0.0 and float(drgb.abs().max()) == 0.0
    finally:
        assert L.tts_debug_scan_wait(0, -1) == _lib.TTS_OK
    out = r.forward()
    assert r.info().status == 0
    for a, b in zip(out, ref):
        assert torch.equal(a, b)
