"""The allocation-free sort entry point (tts_sort_pairs_noalloc).

Some callers may not allocate device memory themselves: a custom allocator
hook cannot call back into cudaMalloc, a plugin host may own every device
allocation, and a tight loop may not afford cudaMalloc's implicit
synchronisation.  For them the library sorts (key, value) pairs with scratch
storage compiled into the library.  These tests check, on consecutive calls,
that it returns exactly what the regular entry points return: the binning
path (tts_bin_views, which orders the tile keys inside its caller-provided
workspace) on the unsorted keys of real renders, and tts_sort_pairs (caller
scratch) and a numpy stable sort on random 64-bit keys whose bits above
key_bits must not take part in the order.  The file is collected last.
"""

import ctypes

import numpy as np
import pytest
import torch

import synth
from paper_2406_01579_b300 import Params, Rasterizer, _lib
from parity import to_dev

pytestmark = pytest.mark.gpu

MAX = _lib.TTS_SORT_NOALLOC_MAX_KEYS


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


def _noalloc(L, kin, vin, kout, vout, n, bits):
    stream = torch.cuda.current_stream().cuda_stream
    return L.tts_sort_pairs_noalloc(kin.data_ptr(), vin.data_ptr(), kout.data_ptr(),
                                    vout.data_ptr(), n, bits, stream)


def test_noalloc_sort_matches_regular_binning_sort():
    L = _lib.load()
    cases = [(synth.scene_sphere16(), 8), (synth.scene_torus64(), 16)]
    for scene, tile in cases:
        ref_k, ref_v, uk, uv, bits = _existing_sort(scene, scene.cams[0], tile)
        n = len(uk)
        assert 1000 < n <= MAX
        kin = torch.from_numpy(uk.view(np.int64)).cuda()
        vin = torch.from_numpy(uv).cuda()
        kout = torch.empty_like(kin)
        vout = torch.empty_like(vin)
        for _ in range(2):   # consecutive calls share the scratch array
            kout.fill_(-1)
            vout.fill_(-1)
            rc = _noalloc(L, kin, vin, kout, vout, n, bits)
            assert rc == _lib.TTS_OK, L.tts_error_string(rc)
            torch.cuda.synchronize()
            assert torch.equal(kout, ref_k)
            assert torch.equal(vout, ref_v)


@pytest.mark.parametrize("n", [1, 2047, 2049, MAX])
@pytest.mark.parametrize("key_bits", [1, 12, 33, 64])
def test_noalloc_sort_random_keys(n, key_bits):
    """Random 64-bit keys (few distinct values in the sorted bits, so stability
    matters; payload bits above key_bits): the allocation-free sort, the
    caller-scratch sort and numpy's stable sort of the masked keys agree."""
    L = _lib.load()
    rng = np.random.default_rng(n * 131 + key_bits)
    k = rng.integers(0, 2**63, size=n, dtype=np.uint64) * np.uint64(2) + \
        rng.integers(0, 2, size=n, dtype=np.uint64)
    if key_bits < 64:
        # draw the sorted bits from a small set: many equal sort keys
        low = rng.integers(0, min(1 << key_bits, 97), size=n, dtype=np.uint64)
        low = (low * np.uint64(0x9E3779B97F4A7C15)) & np.uint64((1 << key_bits) - 1)
        k = (k & ~np.uint64((1 << key_bits) - 1)) | low
    v = np.arange(n, dtype=np.uint32)
    mask = np.uint64((1 << key_bits) - 1) if key_bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    order = np.argsort(k & mask, kind="stable")
    want_k = torch.from_numpy(k[order].view(np.int64).copy())
    want_v = torch.from_numpy(v[order].copy())
    kin = torch.from_numpy(k.view(np.int64)).cuda()
    vin = torch.from_numpy(v).cuda()
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    for _ in range(2):
        kout.fill_(-1)
        vout.fill_(-1)
        rc = _noalloc(L, kin, vin, kout, vout, n, key_bits)
        assert rc == _lib.TTS_OK, L.tts_error_string(rc)
        torch.cuda.synchronize()
        assert torch.equal(kout.cpu(), want_k)
        assert torch.equal(vout.cpu(), want_v)
    # the caller-scratch entry point gives the same pairs
    need = ctypes.c_size_t(0)
    assert L.tts_sort_pairs_scratch_size(n, ctypes.byref(need)) == _lib.TTS_OK
    scratch = torch.empty(int(need.value), dtype=torch.uint8, device="cuda")
    k2, v2 = torch.empty_like(kin), torch.empty_like(vin)
    rc = L.tts_sort_pairs(kin.data_ptr(), vin.data_ptr(), k2.data_ptr(), v2.data_ptr(), n,
                          key_bits, scratch.data_ptr(), scratch.numel(),
                          torch.cuda.current_stream().cuda_stream)
    assert rc == _lib.TTS_OK, L.tts_error_string(rc)
    torch.cuda.synchronize()
    assert torch.equal(k2, kout) and torch.equal(v2, vout)


def test_noalloc_sort_refusals():
    """Arguments the entry point refuses on the host, before anything is
    enqueued: more pairs than the compiled-in scratch holds, key_bits outside
    [1, 64], outputs aliasing inputs, missing pointers."""
    L = _lib.load()
    kin = torch.zeros(16, dtype=torch.int64, device="cuda")
    vin = torch.zeros(16, dtype=torch.int32, device="cuda")
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)
    st = torch.cuda.current_stream().cuda_stream
    args = (kin.data_ptr(), vin.data_ptr(), kout.data_ptr(), vout.data_ptr())
    assert L.tts_sort_pairs_noalloc(*args, MAX + 1, 40, st) == _lib.TTS_ERR_ARG
    assert L.tts_sort_pairs_noalloc(*args, -1, 40, st) == _lib.TTS_ERR_ARG
    assert L.tts_sort_pairs_noalloc(*args, 16, 0, st) == _lib.TTS_ERR_ARG
    assert L.tts_sort_pairs_noalloc(*args, 16, 65, st) == _lib.TTS_ERR_ARG
    assert L.tts_sort_pairs_noalloc(kin.data_ptr(), vin.data_ptr(), kin.data_ptr(),
                                    vout.data_ptr(), 16, 40, st) == _lib.TTS_ERR_ARG
    assert L.tts_sort_pairs_noalloc(kin.data_ptr(), vin.data_ptr(), kout.data_ptr(),
                                    vin.data_ptr(), 16, 40, st) == _lib.TTS_ERR_ARG
    assert L.tts_sort_pairs_noalloc(None, vin.data_ptr(), kout.data_ptr(), vout.data_ptr(), 16,
                                    40, st) == _lib.TTS_ERR_ARG
    assert L.tts_sort_pairs_noalloc(*args, 0, 40, st) == _lib.TTS_OK   # nothing to sort
