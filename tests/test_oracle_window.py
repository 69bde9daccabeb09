"""Pins for the resort window (Sec. 3.3): per pixel, fragments pass through
a window of N_w kept sorted by their entry depth before blending."""

import numpy as np
import pytest

import oracle
import synth


def _scene(n=6):
    V = synth.grid_vertices(n)
    T = synth.grid_tets(n)
    f = (np.linalg.norm(V.astype(np.float64), axis=1) - 0.7).astype(np.float32)
    rgb = np.random.default_rng(1).uniform(size=(len(V), 3)).astype(np.float32)
    return V, T, f, rgb


def test_full_sort_equals_bruteforce_depth_order():
    """N_w < 0 blends each pixel's fragments in increasing entry depth: the
    same as collecting every fragment (App. A.1/A.2 chord) and sorting."""
    V, T, f, rgb = _scene(3)
    cam = synth.orbit_camera(25.0, 15.0, 28, 28)
    s = 30.0
    p = oracle.make_params(s=s, tile=8, window=-1)
    r = oracle.render(V, T, f, rgb, cam, p, surv=np.arange(len(T), dtype=np.int32))
    R, t = cam.R.astype(np.float64), cam.t.astype(np.float64)
    X = np.einsum("ij,kmj->kmi", R, V[T].astype(np.float64)) + t
    for j in range(0, 28, 2):
        for i in range(0, 28, 2):
            frs = []
            for k in range(len(T)):
                res = oracle.fragment(X[k], f[T[k]].astype(np.float64), i + 0.5, j + 0.5,
                                      cam.fx, cam.fy, cam.cx, cam.cy, s)
                if res is None:
                    continue
                a = min(res[4], 0.99)
                if a < 1 / 255:
                    continue
                frs.append((res[2], k, a))
            frs.sort(key=lambda x: x[0])
            Tr, C = 1.0, np.zeros(3)
            for _, k, a in frs:
                if Tr * (1 - a) < 1e-4:
                    break
                C += Tr * a * rgb[T[k]].astype(np.float64).mean(0)
                Tr *= 1 - a
            if r["amb"][j, i] == 0:
                assert r["image"][:, j, i] == pytest.approx(C, abs=1e-12)


def test_window_limits():
    """N_w = 0 is the tile order; a window larger than any pixel list is the
    full sort."""
    V, T, f, rgb = _scene(6)
    cam = synth.orbit_camera(40.0, 25.0, 48, 48)
    base = dict(s=60.0, tile=16)
    r0 = oracle.render(V, T, f, rgb, cam, oracle.make_params(**base))
    rw0 = oracle.render(V, T, f, rgb, cam, oracle.make_params(**base, window=0))
    np.testing.assert_array_equal(r0["image"], rw0["image"])
    rfull = oracle.render(V, T, f, rgb, cam, oracle.make_params(**base, window=-1))
    rbig = oracle.render(V, T, f, rgb, cam, oracle.make_params(**base, window=100000))
    np.testing.assert_array_equal(rfull["image"], rbig["image"])


def test_window_reduces_sorting_error():
    """The paper's claim (Sec. 3.3): a short window nearly removes the error of
    per-tile sorting.  Error = image difference to the full per-pixel sort."""
    sc = synth.scene_sphere16()
    cam = sc.cams[0]
    err = {}
    full = oracle.render(sc.V, sc.T, sc.f, sc.rgb, cam, oracle.make_params(s=20.0, window=-1))
    for w in (0, 1, 2, 5):
        r = oracle.render(sc.V, sc.T, sc.f, sc.rgb, cam, oracle.make_params(s=20.0, window=w))
        err[w] = np.abs(r["image"] - full["image"]).mean()
    assert err[0] > 0
    assert err[5] <= err[2] <= err[1] <= err[0]
    assert err[5] < 0.2 * err[0]


def test_window_adjoint_matches_dual_numbers():
    sc = synth.scene_sphere16()
    cam = sc.cams[0]
    p = oracle.make_params(s=60.0, window=5)
    up = synth.upstream_grads(5, [cam])[0]
    r = oracle.render(sc.V, sc.T, sc.f, sc.rgb, cam, p, upstream=up)
    rng = np.random.default_rng(3)
    tV, tf, tr = rng.normal(size=sc.V.shape), rng.normal(size=sc.N), rng.normal(size=sc.rgb.shape)
    L, dL = oracle.dirderiv(sc.V, sc.T, sc.f, sc.rgb, cam, p, r["surv"], r["bins"], up, tV, tf, tr)
    pred = (r["dV"] * tV).sum() + (r["df"] * tf).sum() + (r["drgb"] * tr).sum()
    assert pred == pytest.approx(dL, rel=1e-9)


# ---------------------------------------------------------------------------
# normal channel of Eq. 2 (Sec. 3.2 per-tet normal, App. A.3)
# ---------------------------------------------------------------------------

def test_normal_map_of_affine_sdf_is_its_unit_gradient():
    """An affine SDF has one normal everywhere: N = O * n with n = grad/|grad|."""
    rng = np.random.default_rng(21)
    nvec = rng.normal(size=3)
    nvec /= np.linalg.norm(nvec)
    V = synth.grid_vertices(3)
    T = synth.grid_tets(3)
    f = (2.0 * (V.astype(np.float64) @ nvec) - 0.1).astype(np.float32)
    rgb = np.ones((len(V), 3), np.float32)
    cam = synth.orbit_camera(35.0, 25.0, 40, 40)
    p = oracle.make_params(s=5.0, tile=8, pure=True)
    r = oracle.render(V, T, f, rgb, cam, p, surv=np.arange(len(T), dtype=np.int32), normals=True)
    expect = r["alpha"][None] * nvec[:, None, None]
    assert np.abs(r["normal"] - expect).max() < 1e-6
    assert (r["alpha"] > 0.05).sum() > 100


def test_normal_adjoint_matches_dual_numbers():
    sc = synth.scene_sphere16()
    cam = sc.cams[0]
    p = oracle.make_params(s=60.0)
    up = list(synth.upstream_grads(8, [cam])[0])
    up.append(np.random.default_rng(9).normal(size=(3, cam.height, cam.width)).astype(np.float32))
    r = oracle.render(sc.V, sc.T, sc.f, sc.rgb, cam, p, upstream=up, normals=True)
    rng = np.random.default_rng(10)
    tV, tf, tr = rng.normal(size=sc.V.shape), rng.normal(size=sc.N), rng.normal(size=sc.rgb.shape)
    L, dL = oracle.dirderiv(sc.V, sc.T, sc.f, sc.rgb, cam, p, r["surv"], r["bins"], up, tV, tf, tr)
    pred = (r["dV"] * tV).sum() + (r["df"] * tf).sum() + (r["drgb"] * tr).sum()
    assert pred == pytest.approx(dL, rel=1e-9)
    Lr = sum((u * x).sum() for u, x in zip(up, (r["image"], r["alpha"], r["depth"], r["normal"])))
    assert L == pytest.approx(Lr, rel=1e-12)
