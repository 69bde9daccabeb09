"""Pins of the oracle's geometry-stage terms (Sec. 4.2 eikonal and normal
consistency losses, App. A.3 per-tet gradient) against closed forms,
invariances, dual numbers and finite differences."""

import numpy as np
import pytest

import oracle
import synth


def _kuhn_edge_count(n):
    # axis edges, one diagonal per cube face, one body diagonal per cube
    return 3 * n * (n + 1) ** 2 + 3 * n * n * (n + 1) + n ** 3


@pytest.mark.parametrize("n", [1, 2, 3, 5])
def test_edges_of_kuhn_grid(n):
    T = synth.grid_tets(n)
    E = oracle.tet_edges(T)
    assert len(E) == _kuhn_edge_count(n)
    assert (E[:, 0] < E[:, 1]).all()
    keys = E[:, 0].astype(np.int64) * (1 << 32) + E[:, 1]
    assert (np.diff(keys) > 0).all()
    # every tet edge is listed
    allk = set(keys.tolist())
    for t in T[:: max(1, len(T) // 50)]:
        for i in range(4):
            for j in range(i + 1, 4):
                a, b = sorted((int(t[i]), int(t[j])))
                assert a * (1 << 32) + b in allk


def test_single_tet_gradient_is_the_affine_slope():
    """App. A.3: the 4 x 4 system recovers the slope of an affine field, so
    L_eik = (|a| - 1)^2 and every vertex normal is a / |a| (L_nc = 0)."""
    rng = np.random.default_rng(3)
    V = rng.normal(size=(4, 3))
    T = np.array([[0, 1, 2, 3]], np.int32)
    a = rng.normal(size=3)
    f = V @ a + 0.7
    r = oracle.regularizers(V, T, f, oracle.tet_edges(T))
    assert r["L_eik"] == pytest.approx((np.linalg.norm(a) - 1.0) ** 2, rel=1e-12)
    assert abs(r["L_nc"]) < 1e-14


def test_affine_field_on_a_grid():
    V = synth.grid_vertices(3).astype(np.float64)
    T = synth.grid_tets(3)
    a = np.array([1.2, -0.9, 1.5])
    a = 2.0 * a / np.linalg.norm(a)          # |g| = 2 everywhere
    f = V @ a - 0.1
    E = oracle.tet_edges(T)
    r = oracle.regularizers(V, T, f, E)
    assert r["L_eik"] == pytest.approx(len(T) * 1.0, rel=1e-12)
    assert abs(r["L_nc"]) < 1e-11
    # |g| = 1: both losses and the eikonal gradient vanish
    r1 = oracle.regularizers(V, T, f / 2.0, E, w_eik=1.0, w_nc=0.0)
    assert abs(r1["L_eik"]) < 1e-20
    assert np.abs(r1["dV"]).max() < 1e-10 and np.abs(r1["df"]).max() < 1e-10


def test_two_tets_closed_form():
    """Two tets sharing face (1, 2, 3) with apexes 0 and 4: the shared vertices
    carry n1 + n2, the apexes n1 and n2, so the three shared-face edges give
    cos = 1 and the six apex edges give cos = sqrt((1 + c) / 2), c = n1 . n2."""
    rng = np.random.default_rng(5)
    V = np.array([[0.0, 0.0, -1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [-0.7, -0.6, 0.1],
                  [0.1, 0.2, 1.1]])
    T = np.array([[0, 1, 2, 3], [4, 1, 2, 3]], np.int32)
    f = rng.normal(size=5)
    E = oracle.tet_edges(T)
    assert len(E) == 9
    r = oracle.regularizers(V, T, f, E)
    n = []
    for t in T:
        A = np.c_[V[t], np.ones(4)]
        g = np.linalg.solve(A, f[t])[:3]
        n.append(g / np.linalg.norm(g))
    c = float(n[0] @ n[1])
    assert r["L_nc"] == pytest.approx(6.0 * (1.0 - np.sqrt((1.0 + c) / 2.0)), rel=1e-12, abs=1e-14)


def _noisy_sphere(n, seed):
    V = synth.grid_vertices(n).astype(np.float64)
    T = synth.grid_tets(n)
    rng = np.random.default_rng(seed)
    V = V + rng.uniform(-0.05, 0.05, size=V.shape) / n
    f = np.linalg.norm(V, axis=1) - 0.55 + 0.05 * rng.normal(size=len(V))
    return V, T, f


def test_invariances():
    V, T, f = _noisy_sphere(3, 7)
    E = oracle.tet_edges(T)
    r = oracle.regularizers(V, T, f, E)
    q, _ = np.linalg.qr(np.random.default_rng(8).normal(size=(3, 3)))
    rr = oracle.regularizers(V @ q.T + np.array([0.3, -0.2, 0.1]), T, f, E)
    assert rr["L_eik"] == pytest.approx(r["L_eik"], rel=1e-11)
    assert rr["L_nc"] == pytest.approx(r["L_nc"], rel=1e-11)
    rs = oracle.regularizers(V, T, 3.0 * f, E)
    assert rs["L_nc"] == pytest.approx(r["L_nc"], rel=1e-11)


def test_adjoint_matches_dual_numbers():
    V, T, f = _noisy_sphere(3, 9)
    E = oracle.tet_edges(T)
    w_eik, w_nc = 0.7, 1.3
    r = oracle.regularizers(V, T, f, E, w_eik, w_nc)
    rng = np.random.default_rng(10)
    tV, tf = rng.normal(size=V.shape), rng.normal(size=f.shape)
    L, dL = oracle.regularizers_dirderiv(V, T, f, E, w_eik, w_nc, tV, tf)
    assert L == pytest.approx(w_eik * r["L_eik"] + w_nc * r["L_nc"], rel=1e-13)
    assert (r["dV"] * tV).sum() + (r["df"] * tf).sum() == pytest.approx(dL, rel=1e-10)


def test_adjoint_matches_finite_differences():
    V, T, f = _noisy_sphere(2, 11)
    E = oracle.tet_edges(T)
    r = oracle.regularizers(V, T, f, E, 1.0, 1.0)
    h = 1e-6
    rng = np.random.default_rng(12)

    def L(V_, f_):
        q = oracle.regularizers(V_, T, f_, E, grad=False)
        return q["L_eik"] + q["L_nc"]

    for i in rng.choice(len(f), 6, replace=False):
        fp, fm = f.copy(), f.copy()
        fp[i] += h
        fm[i] -= h
        assert r["df"][i] == pytest.approx((L(V, fp) - L(V, fm)) / (2 * h), rel=1e-5, abs=1e-7)
        for c in range(3):
            Vp, Vm = V.copy(), V.copy()
            Vp[i, c] += h
            Vm[i, c] -= h
            assert r["dV"][i, c] == pytest.approx((L(Vp, f) - L(Vm, f)) / (2 * h), rel=1e-5,
                                                  abs=1e-7)
