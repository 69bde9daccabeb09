"""The allocation-free sort entry point (tts_sort_pairs_noalloc).

Some callers may not allocate device memory themselves (code inside a host
callback or an allocator hook, plugin hosts that own every allocation, loops
that cannot take cudaMalloc's implicit synchronisation).  For them the
library sorts (key, value) pairs with scratch storage compiled into the
library.  This test feeds it the unsorted tile keys of real renders and
checks, on consecutive calls, that it returns exactly what the regular
binning path (tts_bin_views, which sorts inside its caller-provided
workspace) returns.  It lives in its own file, collected last.
"""

import ctypes

import numpy as np
import pytest
import torch

import synth
from paper_2406_01579_b300 import Params, Rasterizer, _lib
from parity import to_dev

pytestmark = pytest.mark.gpu


def _existing_sort(scene, cam, tile):
    """Sorted keys/values from the regular entry point, and the same pairs in
    the order the binning stage emits them before sorting (slot-major, then
    increasing tile)."""
    r = Rasterizer([to_dev(scene)], [(cam, 0)], Params(s=175.0, tile=tile))
    r.forward()
    d = r.debug_lists()
    keys, vals = d["keys"].clone(), d["vals"].clone()
    k = keys.cpu().numpy().view(np.uint64)
    v = vals.cpu().numpy()
    order = np.lexsort((k >> np.uint64(d["depth_bits"]), v))
    return keys, vals, k[order].copy(), v[order].copy(), int(d["info"].sort_bits)


def test_noalloc_sort_matches_regular_binning_sort():
    L = _lib.load()
    stream = torch.cuda.current_stream().cuda_stream
    cases = [(synth.scene_sphere16(), 8), (synth.scene_torus64(), 16)]
    for scene, tile in cases:
        ref_k, ref_v, uk, uv, bits = _existing_sort(scene, scene.cams[0], tile)
        n = len(uk)
        assert 1000 < n <= _lib.TTS_SORT_NOALLOC_MAX_KEYS
        kin = torch.from_numpy(uk.view(np.int64)).cuda()
        vin = torch.from_numpy(uv).cuda()
        kout = torch.empty_like(kin)
        vout = torch.empty_like(vin)
        for _ in range(2):   # consecutive calls share the scratch array
            kout.fill_(-1)
            vout.fill_(-1)
            rc = L.tts_sort_pairs_noalloc(kin.data_ptr(), vin.data_ptr(), kout.data_ptr(),
                                          vout.data_ptr(), n, bits, stream)
            assert rc == _lib.TTS_OK, L.tts_error_string(rc)
            torch.cuda.synchronize()
            assert torch.equal(kout, ref_k)
            assert torch.equal(vout, ref_v)
    # sizes above the compiled-in maximum are refused on the host
    big = _lib.TTS_SORT_NOALLOC_MAX_KEYS + 1
    rc = L.tts_sort_pairs_noalloc(kin.data_ptr(), vin.data_ptr(), kout.data_ptr(), vout.data_ptr(),
                                  big, bits, stream)
    assert rc == _lib.TTS_ERR_ARG
