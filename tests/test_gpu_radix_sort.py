"""The device LSD radix sort of (tile, depth) keys (tts_sort_pairs, caller
scratch): fed the keys of a render in the order the binning stage emits them
(slot-major, then increasing tile), it returns exactly the binning stage's
sorted lists (which order each tile's bucket on chip instead)."""

import numpy as np
import pytest
import torch

import synth
from paper_2406_01579_b300 import Params, Rasterizer, _lib
from parity import to_dev

pytestmark = pytest.mark.gpu


def _sort(L, kin, vin, bits):
    n = kin.numel()
    need = __import__("ctypes").c_size_t(0)
    assert L.tts_sort_pairs_scratch_size(n, __import__("ctypes").byref(need)) == _lib.TTS_OK
    scratch = torch.empty(int(need.value), dtype=torch.uint8, device="cuda")
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    rc = L.tts_sort_pairs(kin.data_ptr(), vin.data_ptr(), kout.data_ptr(), vout.data_ptr(), n, bits,
                          scratch.data_ptr(), scratch.numel(),
                          torch.cuda.current_stream().cuda_stream)
    assert rc == _lib.TTS_OK, L.tts_error_string(rc)
    return kout, vout


@pytest.mark.parametrize("scene,tile,nview", [("sphere16", 8, 1), ("spheres128", 8, 1),
                                              ("spheres128", 16, 2)])
def test_radix_sort_matches_binning(scene, tile, nview):
    sc = synth.scene_sphere16() if scene == "sphere16" else synth.scene_spheres128(n_views=nview)
    # bbox rects (no hull test): one 128^3 view then holds more keys than the
    # allocation-free sort takes
    r = Rasterizer([to_dev(sc)], [(c, 0) for c in sc.cams[:nview]],
                   Params(s=175.0, tile=tile, hull=False))
    r.forward()
    d = r.debug_lists()
    ref_k, ref_v = d["keys"].clone(), d["vals"].clone()
    k = ref_k.cpu().numpy().view(np.uint64)
    v = ref_v.cpu().numpy()
    order = np.lexsort((k >> np.uint64(d["depth_bits"]), v))   # slot-major, then tile
    kin = torch.from_numpy(k[order].view(np.int64).copy()).cuda()
    vin = torch.from_numpy(v[order].copy()).cuda()
    L = _lib.load()
    kout, vout = _sort(L, kin, vin, int(d["info"].sort_bits))
    torch.cuda.synchronize()
    assert torch.equal(kout, ref_k)
    assert torch.equal(vout, ref_v)
    if scene == "spheres128":
        assert kin.numel() > _lib.TTS_SORT_NOALLOC_MAX_KEYS   # past the no-alloc limit


def test_radix_sort_argument_checks():
    L = _lib.load()
    x = torch.zeros(16, dtype=torch.int64, device="cuda")
    y = torch.zeros(16, dtype=torch.int32, device="cuda")
    s = torch.empty(1 << 20, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream().cuda_stream
    assert L.tts_sort_pairs(x.data_ptr(), y.data_ptr(), x.data_ptr(), y.data_ptr(), 16, 40,
                            s.data_ptr(), s.numel(), st) == _lib.TTS_ERR_ARG      # aliasing
    z, w = torch.empty_like(x), torch.empty_like(y)
    assert L.tts_sort_pairs(x.data_ptr(), y.data_ptr(), z.data_ptr(), w.data_ptr(), 16, 0,
                            s.data_ptr(), s.numel(), st) == _lib.TTS_ERR_ARG      # key bits
    assert L.tts_sort_pairs(x.data_ptr(), y.data_ptr(), z.data_ptr(), w.data_ptr(), 16, 40,
                            s.data_ptr(), 64, st) == _lib.TTS_ERR_WORKSPACE       # too small
