"""Host-side checks of the C ABI: the library loads and exports every entry
point declared in include/tets.h; argument errors are caught on the host
before anything is enqueued (these calls never reach the GPU)."""

import ctypes
import os
import re

import pytest

from paper_2406_01579_b300 import _lib, build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    hdr = open(os.path.join(ROOT, "include", "tets.h")).read()
    hdr = re.sub(r"/\*.*?\*/", "", hdr, flags=re.S)
    return sorted(set(re.findall(r"\b(tts_[a-z_]+)\s*\(", hdr)))


def test_library_builds_and_exports_every_declared_symbol():
    build.build()
    L = _lib.load()
    names = declared_symbols()
    assert len(names) >= 10
    for n in names:
        assert hasattr(L, n), n
    assert set(names) == set(_lib.ENTRY_POINTS)
    assert b"sm_103a" in L.tts_version()


def _batch(n_scenes=1, n_views=1, tile=16, W=64, H=48, K=100, N=50, key_cap=1000):
    scenes = (_lib.tts_scene * max(n_scenes, 1))()
    for s in scenes:
        s.V = s.T = s.f = s.rgb = 0x100000  # never dereferenced by host checks
        s.N, s.K, s.surv_capacity = N, K, 0
    views = (_lib.tts_view * max(n_views, 1))()
    for v in views:
        for i in range(9):
            v.cam.R[i] = 1.0 if i in (0, 4, 8) else 0.0
        v.cam.fx = v.cam.fy = 100.0
        v.cam.cx, v.cam.cy, v.cam.znear = W / 2, H / 2, 0.1
        v.cam.width, v.cam.height = W, H
        v.scene = 0
    b = _lib.tts_batch()
    b.scenes = ctypes.cast(scenes, ctypes.POINTER(_lib.tts_scene))
    b.n_scenes = n_scenes
    b.views = ctypes.cast(views, ctypes.POINTER(_lib.tts_view))
    b.n_views = n_views
    b.params.s, b.params.prefilter_thresh, b.params.alpha_skip = 175.0, 1 / 255, 1 / 255
    b.params.alpha_cap, b.params.t_eps, b.params.tile = 0.99, 1e-4, tile
    b.key_capacity = key_cap
    return b, (scenes, views)


def test_workspace_size_and_argument_checks():
    L = _lib.load()
    b, keep = _batch()
    n = ctypes.c_size_t()
    assert L.tts_workspace_size(ctypes.byref(b), ctypes.byref(n)) == _lib.TTS_OK
    assert n.value > 0 and n.value % 256 == 0
    # workspace grows with capacity and views
    b2, keep2 = _batch(n_views=3, key_cap=100000)
    n2 = ctypes.c_size_t()
    assert L.tts_workspace_size(ctypes.byref(b2), ctypes.byref(n2)) == _lib.TTS_OK
    assert n2.value > n.value
    for field, bad in (("tile", 12), ("s", -1.0), ("s", float("nan"))):
        b3, k3 = _batch()
        setattr(b3.params, field, bad)
        assert L.tts_workspace_size(ctypes.byref(b3), ctypes.byref(n)) == _lib.TTS_ERR_ARG
    b4, k4 = _batch(n_views=0)
    assert L.tts_workspace_size(ctypes.byref(b4), ctypes.byref(n)) == _lib.TTS_ERR_ARG
    b5, k5 = _batch(key_cap=0)
    assert L.tts_workspace_size(ctypes.byref(b5), ctypes.byref(n)) == _lib.TTS_ERR_ARG
    # missing workspace is rejected before any launch
    b6, k6 = _batch()
    assert L.tts_prepare_scene(ctypes.byref(b6), None) == _lib.TTS_ERR_WORKSPACE
    assert L.tts_error_string(3) == b"key or survivor capacity exceeded"


def test_scan_wait_hook_arguments():
    """The tile-scan wait hook checks its arguments on the host and leaves the
    defaults in place afterwards (no device call)."""
    L = _lib.load()
    assert L.tts_debug_scan_wait(-1, -1) == _lib.TTS_ERR_ARG
    assert L.tts_debug_scan_wait(100, -2) == _lib.TTS_ERR_ARG
    assert L.tts_debug_scan_wait(100, 1) == _lib.TTS_OK
    assert L.tts_debug_scan_wait(0, -1) == _lib.TTS_OK
