"""Parity of the GPU coarse-to-fine pre-filter (App. B.1) with the oracle:
survivor bounds bit for bit, the grid refit within FP32 rounding, and a
second-round render of the refitted grid."""

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2406_01579_b300 import Params, Rasterizer, fit_grid
from parity import compare_images, oracle_run, to_dev

pytestmark = pytest.mark.gpu


def _sphere(V, r):
    return (np.linalg.norm(V.astype(np.float64), axis=1) - r).astype(np.float32)


@pytest.mark.parametrize("s", [60.0, 175.0])
def test_bounds_and_refit_match_oracle(s):
    n, r = 32, 0.4
    V = synth.grid_vertices(n)
    T = synth.grid_tets(n)
    f = _sphere(V, r) + np.float32(0.003) * np.random.default_rng(2).normal(size=len(V)).astype(np.float32)
    rgb = np.full((len(V), 3), 0.5, np.float32)
    p = Params(s=s)
    surv_o, band, _ = oracle.prefilter(T, f, oracle.make_params(s=float(np.float32(s))))
    assert band.sum() == 0          # no decision near T_f: identical survivor sets
    sc = to_dev((V, T, f, rgb))
    cam = synth.orbit_camera(30.0, 20.0, 64, 64)
    r_ = Rasterizer([sc], [(cam, 0)], p)
    r_.prepare()
    b = r_.survivor_bounds()
    b_o = oracle.survivor_bounds(V, T, surv_o)
    np.testing.assert_array_equal(b[0].cpu().numpy(), b_o)
    V2 = fit_grid(sc.V, [-1.0] * 3, [1.0] * 3, b[0], 0.05)
    V2_o = oracle.fit_grid(V, [-1.0] * 3, [1.0] * 3, b_o, 0.05)
    assert np.abs(V2.cpu().numpy() - V2_o).max() < 1e-6


def test_two_round_render_matches_oracle():
    """Round 1 on the 32^3 grid, refit into the survivor bounds, SDF
    re-evaluated at the new vertices, round 2 rendered: image, alpha and
    depth against the oracle's own two-round pipeline."""
    n, r, s = 32, 0.45, 175.0
    V = synth.grid_vertices(n)
    T = synth.grid_tets(n)
    rgb = np.random.default_rng(3).uniform(size=(len(V), 3)).astype(np.float32)
    cam = synth.orbit_camera(30.0, 20.0, 128, 128)
    p = Params(s=s, tile=16)
    # GPU: both rounds on the device; the SDF evaluation is the caller's
    sc = to_dev((V, T, _sphere(V, r), rgb))
    rast = Rasterizer([sc], [(cam, 0)], p)
    rast.prepare()
    b = rast.survivor_bounds()[0]
    V2 = fit_grid(sc.V, [-1.0] * 3, [1.0] * 3, b, 0.05)
    f2 = (torch.linalg.norm(V2.double(), dim=1) - r).float()
    sc2 = to_dev((V2.cpu().numpy(), T, f2.cpu().numpy(), rgb))
    rast2 = Rasterizer([sc2], [(cam, 0)], p)
    gv = [x.cpu().numpy() for x in rast2.view_outputs(*rast2.forward())[0]]
    # oracle: the same two rounds from its own survivors
    surv1, _, _ = oracle.prefilter(T, _sphere(V, r), oracle.make_params(s=s))
    bo = oracle.survivor_bounds(V, T, surv1)
    V2o = oracle.fit_grid(V, [-1.0] * 3, [1.0] * 3, bo, 0.05).astype(np.float32)
    orc = oracle_run((V2o, T, _sphere(V2o, r), rgb), cam, p)
    bad, namb, emax, multi = compare_images(gv, orc)
    npx = cam.width * cam.height
    assert bad <= 1e-3 * npx, (bad, emax)
    assert (orc["alpha"] > 0.5).sum() > 1000
