"""The chord's kink (the reading of a ray through a tet edge): the entry and
exit points are a minimum and a maximum over the faces, so where a pixel's
ray passes through an edge two faces give the same point with different
derivatives.  Look-at cameras put the world z axis on the image's centre
column, which holds pixel centres only when the width is odd; grid tets have
edges on that axis.  There the oracle's dual-number derivative (one face's)
differs from central finite differences (their mean); with an even width it
agrees.  The parity tests therefore use even image sizes."""

import numpy as np
import pytest

import oracle
import synth
from paper_2406_01579_b300 import Params
from parity import oracle_params

TET = 5324          # sphere16 tet (993, 1010, 1011, 1300): edge 1011-1300 on the z axis
VERT = 1300         # (0, 0, -0.5)


def _dual_vs_fd(width):
    sph = synth.scene_sphere16()
    p = Params(s=60.0, tile=8)
    op = oracle_params(p)
    V0 = sph.V.astype(np.float64)
    T = sph.T[[TET]]
    surv, _, _ = oracle.prefilter(T, sph.f, op)
    rng = np.random.default_rng(11)
    synth.random_camera(rng, 40, 36)
    cam = synth.random_camera(rng, width, 38)
    H, W = 38, width
    bins = oracle.bin_view(surv, T, V0, cam, p.tile)
    r0 = oracle.render(V0, T, sph.f, sph.rgb, cam, op, surv=surv, bins=bins)
    h = 1e-6            # V[VERT, 0] = 0, so the perturbation is exact in FP32
    Vp, Vm = V0.copy(), V0.copy()
    Vp[VERT, 0] += h
    Vm[VERT, 0] -= h
    rp = oracle.render(Vp, T, sph.f, sph.rgb, cam, op, surv=surv,
                       bins=oracle.bin_view(surv, T, Vp, cam, p.tile))
    rm = oracle.render(Vm, T, sph.f, sph.rgb, cam, op, surv=surv,
                       bins=oracle.bin_view(surv, T, Vm, cam, p.tile))
    tV = np.zeros_like(V0)
    tV[VERT, 0] = 1.0
    out = []
    for y, x in zip(*np.nonzero(r0["alpha"] > 0)):
        ga = np.zeros((H, W), np.float32)
        ga[y, x] = 1
        u = (np.zeros((3, H, W), np.float32), ga, np.zeros((H, W), np.float32))
        _, dual = oracle.dirderiv(V0, T, sph.f, sph.rgb, cam, op, surv, bins, u, tV,
                                  np.zeros(sph.N), np.zeros((sph.N, 3)), V64=V0)
        fd = (rp["alpha"][y, x] - rm["alpha"][y, x]) / (2 * h)
        out.append((x + 0.5 == cam.cx, abs(fd - dual) / max(1.0, abs(fd))))
    return out


@pytest.mark.parametrize("width", [43, 45])
def test_odd_width_puts_a_pixel_column_on_the_kink(width):
    res = _dual_vs_fd(width)
    assert res and all(on_axis for on_axis, _ in res)
    assert max(err for _, err in res) > 0.1


@pytest.mark.parametrize("width", [42, 44])
def test_even_width_derivatives_agree(width):
    res = _dual_vs_fd(width)
    assert res and not any(on_axis for on_axis, _ in res)
    assert max(err for _, err in res) < 1e-4


def _kink_allowance(width):
    """(adjoint dL/dV[VERT, 0], its kink allowance, central FD) per covered
    pixel, L = alpha at that pixel."""
    sph = synth.scene_sphere16()
    p = Params(s=60.0, tile=8)
    op = oracle_params(p)
    V0 = sph.V.astype(np.float64)
    T = sph.T[[TET]]
    surv, _, _ = oracle.prefilter(T, sph.f, op)
    rng = np.random.default_rng(11)
    synth.random_camera(rng, 40, 36)
    cam = synth.random_camera(rng, width, 38)
    H, W = 38, width
    bins = oracle.bin_view(surv, T, V0, cam, p.tile)
    r0 = oracle.render(V0, T, sph.f, sph.rgb, cam, op, surv=surv, bins=bins)
    h = 1e-6
    Vp, Vm = V0.copy(), V0.copy()
    Vp[VERT, 0] += h
    Vm[VERT, 0] -= h
    rp = oracle.render(Vp, T, sph.f, sph.rgb, cam, op, surv=surv,
                       bins=oracle.bin_view(surv, T, Vp, cam, p.tile))
    rm = oracle.render(Vm, T, sph.f, sph.rgb, cam, op, surv=surv,
                       bins=oracle.bin_view(surv, T, Vm, cam, p.tile))
    out = []
    for y, x in zip(*np.nonzero(r0["alpha"] > 0)):
        ga = np.zeros((H, W), np.float32)
        ga[y, x] = 1
        u = (np.zeros((3, H, W), np.float32), ga, np.zeros((H, W), np.float32))
        r = oracle.render(V0, T, sph.f, sph.rgb, cam, op, surv=surv, bins=bins, upstream=u,
                          abs_terms=True)
        fd = (rp["alpha"][y, x] - rm["alpha"][y, x]) / (2 * h)
        out.append((r["dV"][VERT, 0], r["dV_kink"][VERT, 0], fd))
    return out


@pytest.mark.parametrize("width", [43, 45])
def test_kink_allowance_covers_the_other_one_sided_derivative(width):
    """On the kink the adjoint takes one face's derivative and finite
    differences their mean: the oracle's kink allowance (the change under
    the other face) is nonzero there and the gap is half of it."""
    res = _kink_allowance(width)
    assert res
    for adj, kink, fd in res:
        assert kink > 0
        assert 0.49 * kink <= abs(adj - fd) <= 0.51 * kink


@pytest.mark.parametrize("width", [42, 44])
def test_no_kink_allowance_away_from_edges(width):
    res = _kink_allowance(width)
    assert res and all(kink == 0.0 for _, kink, _ in res)
