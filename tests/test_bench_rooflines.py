"""bench.py's per-kernel roofline model: the algorithmic bytes and flop each
kernel is credited with follow the stated per-unit figures, the record ->
vertex adjoint is credited only with the touched slots when their count is
known, and the backward's work goes to the pixel-list kernel unless pixels
overflowed the fragment lists."""

import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402

COUNTS = {"K": 1000, "N": 300, "surv": 100, "views": 2, "keys": 500, "tiles": 64,
          "fragments": 4000, "surv_vertices": 90, "visible_slots": 150}
PEAKS = {"fma_tflops": 10.0, "mufu_gops": 1000.0}


def _by_kernel(recs):
    return {r["kernel"]: r for r in recs}


def test_hbm_kernels_bytes_and_fractions():
    kt = {"k_prefilter_flags": 0.01, "k_place": 0.02, "k_tile_sort": 0.03, "k_tet_bwd": 0.04}
    r = _by_kernel(bench.kernel_rooflines(kt, COUNTS, PEAKS, 1000.0))
    assert r["k_prefilter_flags"]["bytes"] == 16 * 1000 + 4 * 300 + 1000
    assert r["k_place"]["bytes"] == 20 * 200 + 8 * 500
    assert r["k_tile_sort"]["bytes"] == 12 * 500
    # no touched-slot count: every visible slot's gradient row
    assert r["k_tet_bwd"]["bytes"] == 200 + 225 * 150 + 56 * 90
    x = r["k_place"]
    assert x["achieved"] == pytest.approx(x["bytes"] / 0.02e-3 / 1e9)
    assert x["frac"] == pytest.approx(x["achieved"] / 1000.0)
    # ordered by duration, longest first
    assert [y["kernel"] for y in bench.kernel_rooflines(kt, COUNTS, PEAKS, 1000.0)][0] == "k_tet_bwd"


def test_scatter_credits_touched_slots_only():
    c = dict(COUNTS, touched_slots=40)
    r = _by_kernel(bench.kernel_rooflines({"k_tet_bwd": 0.04}, c, PEAKS, 1000.0))
    assert r["k_tet_bwd"]["bytes"] == 200 + 225 * 40 + 56 * 90


def test_backward_work_split_between_list_kernels():
    kt = {"k_blend_fwd": 0.1, "k_blend_bwd_px": 0.05, "k_blend_bwd": 0.01}
    flop = bench.BWD_FLOP_PER_FRAG - bench.BWD_MUFU_PER_FRAG
    r = _by_kernel(bench.kernel_rooflines(kt, dict(COUNTS, listed_pixels=90, overflow_pixels=0),
                                          PEAKS, 1000.0))
    assert r["k_blend_bwd_px"]["fma_flop"] == 4000 * flop
    assert "fma_flop" not in r["k_blend_bwd"]          # only its empty pass ran
    r = _by_kernel(bench.kernel_rooflines(kt, dict(COUNTS, listed_pixels=90, overflow_pixels=10),
                                          PEAKS, 1000.0))
    assert abs(r["k_blend_bwd_px"]["fma_flop"] - 4000 * flop * 0.9) <= 1
    assert abs(r["k_blend_bwd"]["fma_flop"] - 4000 * flop * 0.1) <= 1
    f = r["k_blend_fwd"]
    assert f["mufu_ops"] == 4000 * bench.FWD_MUFU_PER_FRAG
    assert f["frac"] == pytest.approx(max(f["fma_frac"], f["mufu_frac"]))
