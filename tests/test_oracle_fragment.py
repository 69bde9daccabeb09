"""Pins for the oracle's single-ray/single-tet chord and Eq. 1 opacity.

The oracle intersects a ray with a tet through the four projected triangles
(App. A.1 2D barycentrics + App. A.2 perspective correction).  These tests
check it against two routes written here from textbook geometry:

* plane clipping: the tet is the intersection of four half-spaces; the ray
  enters at the last entering plane and leaves at the first exiting plane;
* 3D barycentrics (App. A.3): the SDF is affine inside the tet, with gradient
  and offset from the 4x4 system [v^T 1] [g; c0] = f.

and Eq. 1 against its definition with Phi_s(x) = 1 / (1 + exp(-s x)).
"""

import math

import numpy as np
import pytest

import oracle

FX = FY = 300.0
CX = CY = 128.0


def phi(x, s):
    return 1.0 / (1.0 + math.exp(-s * x))


def eq1_definition(fp, fn, s):
    return max((phi(fp, s) - phi(fn, s)) / phi(fp, s), 0.0)


def random_tet(rng, depth=3.0, size=0.3):
    c = np.array([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), depth])
    while True:
        X = c + rng.uniform(-size, size, size=(4, 3))
        vol = np.dot(np.cross(X[1] - X[0], X[2] - X[0]), X[3] - X[0])
        if abs(vol) > 0.2 * size ** 3:
            return X


def clip_route(X, F, px, py):
    """Plane clipping: returns (z_in, z_out, f_in, f_out) or None."""
    d = np.array([(px - CX) / FX, (py - CY) / FY, 1.0])
    t_in, t_out = 0.0, np.inf
    for k in range(4):
        idx = [j for j in range(4) if j != k]
        a, b, c = X[idx]
        n = np.cross(b - a, c - a)
        if np.dot(n, X[k] - a) > 0:   # outward = away from the opposite vertex
            n = -n
        e = np.dot(n, a)              # inside: n . x <= e
        den = np.dot(n, d)
        if abs(den) < 1e-300:
            if e < 0:
                return None
            continue
        t = e / den
        if den < 0:
            t_in = max(t_in, t)
        else:
            t_out = min(t_out, t)
    if not t_in < t_out:
        return None
    # App. A.3: [v^T 1] [g; c0] = f
    M = np.hstack([X, np.ones((4, 1))])
    gc = np.linalg.solve(M, F)
    g, c0 = gc[:3], gc[3]
    fi = np.dot(g, t_in * d) + c0
    fo = np.dot(g, t_out * d) + c0
    return t_in, t_out, fi, fo   # d_z = 1, so the ray parameter is the depth


def project(X):
    return FX * X[:, 0] / X[:, 2] + CX, FY * X[:, 1] / X[:, 2] + CY


def test_eq1_worked_value():
    # s = 1, f_prev = 0, f_next = -1: (Phi(0) - Phi(-1)) / Phi(0) = 0.46211715...
    X = np.array([[0.0, 0.0, 2.0], [1.0, 0.0, 2.0], [0.0, 1.0, 2.0], [0.0, 0.0, 3.0]])
    # build F so that along the optical-axis ray f goes from 0 (z=2) to -1 (z=3)
    F = np.array([0.0, 0.0, 0.0, -1.0])
    r = oracle.fragment(X, F, CX + 1e-3, CY + 1e-3, FX, FY, CX, CY, 1.0)
    assert r is not None
    fp, fn, zi, zo, a = r
    assert a == pytest.approx(eq1_definition(fp, fn, 1.0), abs=1e-14)
    assert eq1_definition(0.0, -1.0, 1.0) == pytest.approx(0.4621171572600098, abs=1e-15)


def test_eq1_stable_form_matches_definition():
    rng = np.random.default_rng(0)
    n = 0
    while n < 300:
        X = random_tet(rng)
        F = rng.normal(0, 0.2, size=4)
        u, v = project(X)
        w = rng.dirichlet(np.ones(4))
        px, py = float(w @ u), float(w @ v)
        s = float(rng.choice([1.0, 20.0, 175.0]))
        r = oracle.fragment(X, F, px, py, FX, FY, CX, CY, s)
        if r is None:
            continue
        fp, fn, zi, zo, a = r
        if abs(s * fn) > 30:      # the definition loses all digits there; the rewrite does not
            continue
        assert a == pytest.approx(eq1_definition(fp, fn, s), rel=1e-9, abs=1e-13)
        assert 0.0 <= a <= 1.0
        n += 1


def test_chord_three_routes_agree():
    """2D barycentric + perspective route (oracle) == plane clipping == 3D
    barycentric SDF, to 1e-10."""
    rng = np.random.default_rng(1)
    n = 0
    while n < 500:
        X = random_tet(rng)
        F = rng.normal(0, 0.3, size=4)
        u, v = project(X)
        w = rng.dirichlet(np.ones(4) * 0.7)
        px, py = float(w @ u), float(w @ v)
        ref = clip_route(X, F, px, py)
        got = oracle.fragment(X, F, px, py, FX, FY, CX, CY, 20.0)
        if ref is None:
            assert got is None or abs(got[3] - got[2]) < 1e-9
            continue
        assert got is not None
        zi, zo, fi, fo = ref
        assert got[2] == pytest.approx(zi, rel=1e-10)
        assert got[3] == pytest.approx(zo, rel=1e-10)
        assert got[0] == pytest.approx(fi, abs=1e-10)
        assert got[1] == pytest.approx(fo, abs=1e-10)
        n += 1


def test_miss_outside_projection():
    rng = np.random.default_rng(2)
    for _ in range(100):
        X = random_tet(rng)
        u, v = project(X)
        px, py = u.max() + 1.0, v.max() + 1.0
        assert oracle.fragment(X, rng.normal(size=4), px, py, FX, FY, CX, CY, 20.0) is None


def test_constant_and_increasing_sdf_give_zero_alpha():
    rng = np.random.default_rng(3)
    for _ in range(100):
        X = random_tet(rng)
        u, v = project(X)
        w = rng.dirichlet(np.ones(4))
        px, py = float(w @ u), float(w @ v)
        c = rng.normal()
        r = oracle.fragment(X, np.full(4, c), px, py, FX, FY, CX, CY, 100.0)
        # exactly 0 in exact arithmetic; FP64 interpolation of a constant leaves ~1 ulp
        assert r is None or r[4] < 1e-12
        # SDF increasing with depth (f = z): the ray leaves the surface, alpha = 0
        r = oracle.fragment(X, X[:, 2].copy(), px, py, FX, FY, CX, CY, 100.0)
        assert r is None or r[4] == 0.0


def test_fragment_gradient_matches_central_differences():
    rng = np.random.default_rng(4)
    n = 0
    h = 1e-6
    while n < 60:
        X = random_tet(rng)
        F = rng.normal(0, 0.1, size=4)
        u, v = project(X)
        w = rng.dirichlet(np.ones(4) * 2.0)
        px, py = float(w @ u), float(w @ v)
        got = oracle.fragment_grad(X, F, px, py, FX, FY, CX, CY, 20.0)
        if got is None or got[0] < 1e-3:
            continue
        a, g = got
        x0 = np.concatenate([X.ravel(), F])
        fd = np.zeros(16)
        ok = True
        for i in range(16):
            xp, xm = x0.copy(), x0.copy()
            xp[i] += h
            xm[i] -= h
            rp = oracle.fragment(xp[:12].reshape(4, 3), xp[12:], px, py, FX, FY, CX, CY, 20.0)
            rm = oracle.fragment(xm[:12].reshape(4, 3), xm[12:], px, py, FX, FY, CX, CY, 20.0)
            if rp is None or rm is None:
                ok = False
                break
            fd[i] = (rp[4] - rm[4]) / (2 * h)
        if not ok:
            continue
        # a kink (face switch) inside [-h, h] shows up as a large mismatch: skip those
        err = np.abs(fd - g).max() / max(np.abs(g).max(), 1e-12)
        if err > 1e-2:
            continue
        assert err < 1e-5
        n += 1
