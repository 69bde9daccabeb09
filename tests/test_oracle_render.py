"""Pins for the oracle's full render (binning + Eq. 1 + Eq. 2) and its adjoint.

Each test checks the oracle against something it does not compute itself:
closed forms that follow from Eq. 1/Eq. 2, invariances of the method,
brute-force enumeration, forward-mode dual numbers and central finite
differences.
"""

import math

import numpy as np
import pytest

import oracle
import synth


def eq1(fp, fn, s):
    """Eq. 1 from its definition (stable for the moderate s*f used here)."""
    if not fp > fn:
        return 0.0
    phi = lambda x: 1.0 / (1.0 + math.exp(-s * x))
    return (phi(fp) - phi(fn)) / phi(fp)


def ray_dir(cam, i, j):
    return np.array([(i + 0.5 - cam.cx) / cam.fx, (j + 0.5 - cam.cy) / cam.fy, 1.0])


def cam_world(cam):
    """(R, t, camera centre, R^-1); the FP32 rotation is not exactly
    orthonormal, so world-space rays use its true inverse."""
    R = cam.R.astype(np.float64)
    t = cam.t.astype(np.float64)
    Ri = np.linalg.inv(R)
    return R, t, -Ri @ t, Ri


def small_grid(n, f, rgb=None):
    V = synth.grid_vertices(n)
    T = synth.grid_tets(n)
    fv = f(V.astype(np.float64)).astype(np.float32)
    if rgb is None:
        rgb = np.random.default_rng(0).uniform(0, 1, size=(len(V), 3))
    return V, T, fv, rgb.astype(np.float32)


# ---------------------------------------------------------------------------
# closed forms
# ---------------------------------------------------------------------------

def test_telescoping_linear_sdf_pure_mode():
    """For an affine SDF f = n.x - d, the tet-wise interpolation is exact and
    every fragment has 1 - alpha = Phi(f_next)/Phi(f_prev), so in PURE mode
    T_final = Phi(f_out)/Phi(f_in) whatever the tessellation and the order:
    O = Eq.1(f_in, f_out) with f at the ray's entry/exit of [-1,1]^3, and with a
    constant colour c, C = O c."""
    rng = np.random.default_rng(7)
    nvec = rng.normal(size=3)
    nvec /= np.linalg.norm(nvec)
    d0 = 0.1
    V, T, f, _ = small_grid(3, lambda X: X @ nvec - d0)
    # the FP32-rounded vertex values define (to ~3e-8) the affine field used below
    A = np.hstack([V.astype(np.float64), np.ones((len(V), 1))])
    coef = np.linalg.lstsq(A, f.astype(np.float64), rcond=None)[0]
    assert np.abs(A @ coef - f).max() < 1e-7
    col = np.array([0.25, 0.5, 0.75])
    rgb = np.tile(col, (len(V), 1)).astype(np.float32)
    cam = synth.orbit_camera(40.0, 25.0, 48, 48)
    s = 6.0
    p = oracle.make_params(s=s, tile=8, pure=True)
    r = oracle.render(V, T, f, rgb, cam, p, surv=np.arange(len(T), dtype=np.int32))
    R, t, C0, Ri = cam_world(cam)
    checked = 0
    for j in range(cam.height):
        for i in range(cam.width):
            dw = Ri @ ray_dir(cam, i, j)     # world-space ray C0 + tau dw
            lo, hi = -np.inf, np.inf
            for a in range(3):
                t1 = (-1.0 - C0[a]) / dw[a]
                t2 = (1.0 - C0[a]) / dw[a]
                lo, hi = max(lo, min(t1, t2)), min(hi, max(t1, t2))
            O = r["alpha"][j, i]
            if not lo < hi - 1e-3:       # misses or grazes the cube
                if lo > hi + 1e-3:
                    assert O == 0.0
                continue
            fin = (C0 + lo * dw) @ coef[:3] + coef[3]
            fout = (C0 + hi * dw) @ coef[:3] + coef[3]
            expect = eq1(fin, fout, s)
            assert O == pytest.approx(expect, abs=2e-7)
            assert r["image"][:, j, i] == pytest.approx(expect * col, abs=2e-7)
            checked += 1
    assert checked > 300


def test_single_tet_closed_forms_pure():
    """One tet, PURE mode: O = alpha, C = alpha * mean(rgb), D = alpha * zbar,
    with alpha from the plane-clipping chord and Eq. 1 from its definition."""
    V = np.array([[-0.3, -0.2, -0.1], [0.35, -0.25, 0.05], [0.0, 0.4, -0.2], [0.05, 0.0, 0.45]],
                 np.float32)
    T = np.array([[0, 1, 2, 3]], np.int32)
    f = np.array([-0.2, 0.1, -0.05, 0.3], np.float32)   # decreasing away from this camera
    rgb = np.array([[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 1]], np.float32)
    cam = synth.orbit_camera(10.0, 15.0, 40, 40)
    s = 8.0
    p = oracle.make_params(s=s, tile=8, pure=True)
    r = oracle.render(V, T, f, rgb, cam, p, surv=np.array([0], np.int32))
    R, t, _, _ = cam_world(cam)
    X = (R @ V.astype(np.float64).T).T + t
    M = np.hstack([X, np.ones((4, 1))])
    gc = np.linalg.solve(M, f.astype(np.float64))
    zbar = X[:, 2].mean()
    cbar = rgb.astype(np.float64).mean(0)
    hits = 0
    for j in range(40):
        for i in range(40):
            d = ray_dir(cam, i, j)
            t_in, t_out = 0.0, np.inf
            miss = False
            for k in range(4):
                idx = [q for q in range(4) if q != k]
                a, b, c = X[idx]
                nrm = np.cross(b - a, c - a)
                if np.dot(nrm, X[k] - a) > 0:
                    nrm = -nrm
                e, den = nrm @ a, nrm @ d
                if den < 0:
                    t_in = max(t_in, e / den)
                elif den > 0:
                    t_out = min(t_out, e / den)
                elif e < 0:
                    miss = True
            if miss or not t_in < t_out:
                assert r["alpha"][j, i] < 1e-9
                continue
            fp = gc[:3] @ (t_in * d) + gc[3]
            fn = gc[:3] @ (t_out * d) + gc[3]
            a = eq1(fp, fn, s)
            assert r["alpha"][j, i] == pytest.approx(a, abs=1e-9)
            assert r["depth"][j, i] == pytest.approx(a * zbar, abs=1e-9)
            assert r["image"][:, j, i] == pytest.approx(a * cbar, abs=1e-9)
            hits += a > 0
    assert hits > 20


def test_all_positive_sdf_is_prefiltered_to_transparent():
    V, T, f, rgb = small_grid(4, lambda X: 1.0 + 0.1 * X[:, 0])
    p = oracle.make_params(s=20.0, tile=8)
    surv, amb, amax = oracle.prefilter(T, f, p)
    assert amax.max() < 1.0 / 255.0 and len(surv) == 0
    cam = synth.orbit_camera(30.0, 20.0, 32, 32)
    r = oracle.render(V, T, f, rgb, cam, p)
    assert np.all(r["alpha"] == 0.0) and np.all(r["image"] == 0.0)


def test_large_s_limit_matches_level_set():
    """s -> infinity: rays crossing the zero level set become opaque, the
    others transparent (Sec. 3.2, relation to DMTet)."""
    V, T, f, rgb = small_grid(16, lambda X: np.linalg.norm(X, axis=1) - 0.5)
    cam = synth.orbit_camera(30.0, 20.0, 64, 64)
    p = oracle.make_params(s=3000.0, tile=16)
    r = oracle.render(V, T, f, rgb, cam, p)
    R, t, C0, Ri = cam_world(cam)
    n_in = n_out = 0
    for j in range(64):
        for i in range(64):
            dw = Ri @ ray_dir(cam, i, j)
            dw /= np.linalg.norm(dw)
            dist = np.linalg.norm(C0 - (C0 @ dw) * dw)   # ray-to-origin distance
            if dist < 0.42:
                assert r["alpha"][j, i] > 0.99
                n_in += 1
            elif dist > 0.6:
                assert r["alpha"][j, i] < 0.01
                n_out += 1
    assert n_in > 100 and n_out > 100


def test_capped_stop_tie_is_decided_in_fp32():
    """With the 3DGS constants two fragments at the cap leave T = (1 - 0.99)^2,
    which equals t_eps = 1e-4 in real arithmetic.  With the FP32 thresholds a
    kernel receives, the oracle takes that stop decision exactly as FP32 does:
    1 - 0.99f = 0.0099999905 (exact), its square rounds to 9.99998e-5 <
    1e-4f, so a ray whose first two fragments are capped stops before the
    second (alpha = 0.99f exactly) and the decision is not ambiguous.  With
    the FP64 constants 0.99 and 1e-4 the square is 1.0000000000000018e-4 >=
    1e-4: the FP64 decision blends the second fragment and stays a band
    decision."""
    cap32, eps32 = float(np.float32(0.99)), float(np.float32(1e-4))
    x = np.float32(1.0) - np.float32(cap32)
    assert float(x) == 1.0 - cap32                       # Sterbenz: exact
    assert np.float32(x * x) < np.float32(eps32)         # FP32: stop
    assert (1.0 - 0.99) ** 2 >= 1e-4                     # FP64 constants: blend
    V, T, f, rgb = small_grid(16, lambda X: np.linalg.norm(X, axis=1) - 0.5)
    cam = synth.orbit_camera(30.0, 20.0, 64, 64)
    R, t, C0, Ri = cam_world(cam)
    p32 = oracle.make_params(s=3000.0, tile=16, alpha_cap=cap32, t_eps=eps32,
                             alpha_skip=float(np.float32(1 / 255)),
                             prefilter_thresh=float(np.float32(1 / 255)))
    p64 = oracle.make_params(s=3000.0, tile=16)
    r32 = oracle.render(V, T, f, rgb, cam, p32)
    r64 = oracle.render(V, T, f, rgb, cam, p64)
    # rays stopped before their second fragment, the first one at the cap
    stopped = r32["alpha"] == cap32
    assert stopped.sum() > 100
    assert np.all(r32["amb"][stopped] == 0)
    # with the FP64 constants nearly all of them blend that second fragment,
    # as a band decision
    blended = (r64["alpha"][stopped] > 0.99) & (r64["amb"][stopped] > 0)
    assert blended.mean() > 0.95
    # they are the rays through the sphere's interior
    for j, i in zip(*np.nonzero(stopped)):
        dw = Ri @ ray_dir(cam, i, j)
        dw /= np.linalg.norm(dw)
        assert np.linalg.norm(C0 - (C0 @ dw) * dw) < 0.52


# ---------------------------------------------------------------------------
# invariants
# ---------------------------------------------------------------------------

@pytest.fixture(scope="module")
def sphere16():
    s = synth.scene_sphere16()
    p = oracle.make_params(s=175.0, tile=16)
    up = synth.upstream_grads(0, s.cams)[0]
    r = oracle.render(s.V, s.T, s.f, s.rgb, s.cams[0], p, upstream=up)
    return s, p, up, r


def test_ranges_and_bounds(sphere16):
    s, p, up, r = sphere16
    assert r["alpha"].min() >= 0.0 and r["alpha"].max() <= 1.0
    img = r["image"]
    assert img.min() >= 0.0 and np.all(img <= r["alpha"][None] + 1e-12)   # rgb in [0,1]
    assert r["depth"].min() >= 0.0
    # fewer than 1% of pixels sit on a decision band
    assert (r["amb"] > 0).mean() < 0.01


def test_permuting_tets_leaves_image_unchanged(sphere16):
    s, p, up, r = sphere16
    bins = r["bins"]
    kt, kz = bins["key_tile"], bins["key_z"]
    assert not np.any((kt[1:] == kt[:-1]) & (kz[1:] == kz[:-1])), "exact key ties present"
    perm = np.random.default_rng(3).permutation(len(s.T))
    r2 = oracle.render(s.V, s.T[perm], s.f, s.rgb, s.cams[0], p)
    np.testing.assert_array_equal(r2["image"], r["image"])
    np.testing.assert_array_equal(r2["alpha"], r["alpha"])


def test_reordering_tet_vertices_leaves_image_unchanged(sphere16):
    s, p, up, r = sphere16
    rng = np.random.default_rng(4)
    T2 = np.array([t[rng.permutation(4)] for t in s.T])
    r2 = oracle.render(s.V, T2, s.f, s.rgb, s.cams[0], p)
    ok = (r["amb"] == 0) & (r2["amb"] == 0)
    # the FP32 mean depth may move by one ulp (summation order), which can only
    # swap near-coincident tets; everything else is identical up to FP64 rounding
    d = np.abs(r2["image"] - r["image"]).max(0)
    assert np.mean(d[ok] < 1e-12) > 0.999
    assert d[ok].max() < 1e-3


def test_relabelling_vertices_leaves_image_unchanged(sphere16):
    s, p, up, r = sphere16
    perm = np.random.default_rng(5).permutation(len(s.V))
    inv = np.empty_like(perm)
    inv[perm] = np.arange(len(perm))
    V2, f2, rgb2 = s.V[perm], s.f[perm], s.rgb[perm]
    T2 = inv[s.T].astype(np.int32)
    r2 = oracle.render(V2, T2, f2, rgb2, s.cams[0], p, upstream=up)
    np.testing.assert_array_equal(r2["image"], r["image"])
    np.testing.assert_allclose(r2["dV"], r["dV"][perm], rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r2["df"], r["df"][perm], rtol=1e-12, atol=1e-12)


def test_scale_invariance_of_image_and_gradients(sphere16):
    """Eq. 1 depends on s*f only: (2f, s/2) renders the same image; the SDF
    gradient halves, position and colour gradients are unchanged."""
    s, p, up, r = sphere16
    p2 = oracle.make_params(s=175.0 / 2, tile=16)
    r2 = oracle.render(s.V, s.T, 2 * s.f, s.rgb, s.cams[0], p2, upstream=up)
    np.testing.assert_array_equal(r2["image"], r["image"])
    np.testing.assert_allclose(r2["df"], r["df"] / 2, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(r2["dV"], r["dV"], rtol=1e-12, atol=1e-12)


def test_rigid_motion_of_scene_and_camera(sphere16):
    s, p, up, r = sphere16
    rng = np.random.default_rng(6)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    if np.linalg.det(Q) < 0:
        Q[:, 0] = -Q[:, 0]
    q = rng.uniform(-0.2, 0.2, size=3)
    V2 = (s.V.astype(np.float64) @ Q.T + q).astype(np.float32)
    c = s.cams[0]
    R2 = c.R.astype(np.float64) @ Q.T
    t2 = c.t.astype(np.float64) - R2 @ q
    cam2 = synth.Camera(R2.astype(np.float32), t2.astype(np.float32), c.fx, c.fy, c.cx, c.cy,
                        c.znear, c.width, c.height)
    r2 = oracle.render(V2, s.T, s.f, s.rgb, cam2, p)
    ok = (r["amb"] == 0) & (r2["amb"] == 0)
    d = np.abs(r2["image"] - r["image"]).max(0)
    # inputs are re-rounded to FP32, so bbox borders / near ties may move
    assert np.mean(d[ok] < 1e-4) > 0.999


def test_prefilter_does_not_change_the_image(sphere16):
    """alpha <= alpha_max, so with the 1/255 skip on, pre-filtering at 1/255
    removes only fragments that would have been skipped."""
    s, p, up, r = sphere16
    r2 = oracle.render(s.V, s.T, s.f, s.rgb, s.cams[0], p,
                       surv=np.arange(len(s.T), dtype=np.int32))
    ok = (r["amb"] == 0) & (r2["amb"] == 0)
    d = np.abs(r2["image"] - r["image"]).max(0)
    assert d[ok].max() < 1e-12


def test_alpha_never_exceeds_alpha_max():
    rng = np.random.default_rng(8)
    s = synth.scene_sphere16()
    p = oracle.make_params(s=20.0)
    _, _, amax = oracle.prefilter(s.T, s.f, p)
    c = s.cams[0]
    R, t, _, _ = cam_world(c)
    n = 0
    for k in rng.choice(len(s.T), 3000, replace=False):
        X = (R @ s.V[s.T[k]].astype(np.float64).T).T + t
        u = c.fx * X[:, 0] / X[:, 2] + c.cx
        v = c.fy * X[:, 1] / X[:, 2] + c.cy
        w = rng.dirichlet(np.ones(4))
        res = oracle.fragment(X, s.f[s.T[k]].astype(np.float64), w @ u, w @ v, c.fx, c.fy,
                              c.cx, c.cy, 20.0)
        if res is not None:
            assert res[4] <= amax[k] * (1 + 1e-12) + 1e-300
            n += 1
    assert n > 1000


# ---------------------------------------------------------------------------
# binning: brute-force tile enumeration and sort order
# ---------------------------------------------------------------------------

def test_binning_matches_bruteforce_enumeration():
    rng = np.random.default_rng(9)
    V, T, f, rgb = small_grid(3, lambda X: np.linalg.norm(X, axis=1) - 0.6)
    for trial in range(3):
        cam = synth.random_camera(rng, 40 + 8 * trial, 36)
        tile = [4, 8, 16][trial]
        surv = np.arange(len(T), dtype=np.int32)
        b = oracle.bin_view(surv, T, V, cam, tile)
        R, t, _, _ = cam_world(cam)
        tx = (cam.width + tile - 1) // tile
        expect = []
        border = 0
        for k in range(len(T)):
            X = (R @ V[T[k]].astype(np.float64).T).T + t
            u = cam.fx * X[:, 0] / X[:, 2] + cam.cx
            v = cam.fy * X[:, 1] / X[:, 2] + cam.cy
            tiles = set()
            for j in range(cam.height):
                for i in range(cam.width):
                    if u.min() <= i + 0.5 <= u.max() and v.min() <= j + 0.5 <= v.max():
                        tiles.add((j // tile) * tx + i // tile)
            near = (np.min(np.abs(np.concatenate([u, v])[:, None] - (np.arange(64) + 0.5))) < 1e-4)
            got = set(b["key_tile"][b["key_val"] == k].tolist())
            if got != tiles:
                assert near
                border += 1
            for tt in tiles:
                expect.append((tt, k))
        assert border <= 2
        # sorted by (tile, zbits); equal keys keep survivor order
        kt, kz, kv = b["key_tile"], b["key_z"], b["key_val"]
        order = np.lexsort((kv, kz, kt))
        np.testing.assert_array_equal(order, np.arange(len(kt)))
        # ranges delimit each tile's run
        for tt in range(len(b["ranges"])):
            s0, s1 = b["ranges"][tt]
            assert np.all(kt[s0:s1] == tt)
            assert np.sum(kt == tt) == s1 - s0
        # depth bits are the FP32 mean of the camera-space vertex depths
        zb = b["zbits"].view(np.float32)
        X = np.einsum("ij,kmj->kmi", R, V[T].astype(np.float64)) + t
        np.testing.assert_allclose(zb, X[:, :, 2].mean(1), rtol=1e-6)


def test_bbox_restriction_equals_every_tet_every_pixel():
    """The bbox-restricted walk equals compositing every tet that the pixel
    ray meets, ordered by (mean depth bits, index)."""
    V, T, f, rgb = small_grid(2, lambda X: np.linalg.norm(X, axis=1) - 0.7)
    cam = synth.orbit_camera(35.0, 25.0, 24, 24)
    s = 20.0
    p = oracle.make_params(s=s, tile=8)
    surv = np.arange(len(T), dtype=np.int32)
    r = oracle.render(V, T, f, rgb, cam, p, surv=surv)
    R, t, _, _ = cam_world(cam)
    X = np.einsum("ij,kmj->kmi", R, V[T].astype(np.float64)) + t
    zbits = r["bins"]["zbits"]
    order = np.lexsort((np.arange(len(T)), zbits))
    for j in range(cam.height):
        for i in range(cam.width):
            Tr, C = 1.0, np.zeros(3)
            for k in order:
                res = oracle.fragment(X[k], f[T[k]].astype(np.float64), i + 0.5, j + 0.5,
                                      cam.fx, cam.fy, cam.cx, cam.cy, s)
                if res is None:
                    continue
                a = min(res[4], 0.99)
                if a < 1 / 255:
                    continue
                if Tr * (1 - a) < 1e-4:
                    break
                C += Tr * a * rgb[T[k]].astype(np.float64).mean(0)
                Tr *= 1 - a
            if r["amb"][j, i] == 0:
                assert r["image"][:, j, i] == pytest.approx(C, abs=1e-12)
                assert r["alpha"][j, i] == pytest.approx(1 - Tr, abs=1e-12)


# ---------------------------------------------------------------------------
# gradients
# ---------------------------------------------------------------------------

def _rand_dir(rng, N):
    return rng.normal(size=(N, 3)), rng.normal(size=N), rng.normal(size=(N, 3))


def test_adjoint_equals_forward_mode_dual(sphere16):
    s, p, up, r = sphere16
    rng = np.random.default_rng(10)
    for _ in range(3):
        tV, tf, tr = _rand_dir(rng, s.N)
        L, dL = oracle.dirderiv(s.V, s.T, s.f, s.rgb, s.cams[0], p, r["surv"], r["bins"], up,
                                tV, tf, tr)
        pred = (r["dV"] * tV).sum() + (r["df"] * tf).sum() + (r["drgb"] * tr).sum()
        assert pred == pytest.approx(dL, rel=1e-10)
    Lr = ((up[0] * r["image"]).sum() + (up[1] * r["alpha"]).sum() + (up[2] * r["depth"]).sum())
    assert L == pytest.approx(Lr, rel=1e-12)


def _fd_check(V, T, f, rgb, cam, p, up, n_dirs, seed, h=1e-6, rtol=1e-4):
    r = oracle.render(V, T, f, rgb, cam, p, upstream=up)
    surv, bins = r["surv"], r["bins"]
    rng = np.random.default_rng(seed)
    V64, f64, c64 = V.astype(np.float64), f.astype(np.float64), rgb.astype(np.float64)

    def loss(Vd, fd, cd):
        rr = oracle.render(V, T, f, rgb, cam, p, surv=surv, bins=bins, V64=Vd, f64=fd, rgb64=cd)
        return ((up[0] * rr["image"]).sum() + (up[1] * rr["alpha"]).sum() +
                (up[2] * rr["depth"]).sum())

    for _ in range(n_dirs):
        tV, tf, tr = _rand_dir(rng, len(V))
        Lp = loss(V64 + h * tV, f64 + h * tf, c64 + h * tr)
        Lm = loss(V64 - h * tV, f64 - h * tf, c64 - h * tr)
        fd = (Lp - Lm) / (2 * h)
        pred = (r["dV"] * tV).sum() + (r["df"] * tf).sum() + (r["drgb"] * tr).sum()
        assert pred == pytest.approx(fd, rel=rtol, abs=1e-6)


def test_gradient_fd_single_tet_pure():
    V = np.array([[-0.3, -0.2, -0.1], [0.35, -0.25, 0.05], [0.0, 0.4, -0.2], [0.05, 0.0, 0.45]],
                 np.float32)
    T = np.array([[0, 1, 2, 3]], np.int32)
    f = np.array([-0.2, 0.1, -0.05, 0.3], np.float32)
    rgb = np.random.default_rng(0).uniform(size=(4, 3)).astype(np.float32)
    cam = synth.orbit_camera(10.0, 15.0, 32, 32)
    p = oracle.make_params(s=6.0, tile=8, pure=True)
    up = synth.upstream_grads(11, [cam])[0]
    _fd_check(V, T, f, rgb, cam, p, up, 4, 1)


@pytest.mark.parametrize("n", [1, 2, 4])
def test_gradient_fd_small_grids_pure(n):
    rng = np.random.default_rng(n)
    V, T, f, rgb = small_grid(n, lambda X: np.linalg.norm(X, axis=1) - 0.6 + 0.05 * X[:, 0])
    cam = synth.orbit_camera(33.0, 21.0, 32, 32)
    p = oracle.make_params(s=3.0, tile=8, pure=True)
    up = synth.upstream_grads(20 + n, [cam])[0]
    _fd_check(V, T, f, rgb, cam, p, up, 3, 100 + n)


def test_gradient_fd_subgrid_of_spheres128_default_mode():
    """Cubes [62,66)^3 of the 128^3 three-sphere scene as a standalone grid,
    seen by the first of its 512x512 cameras; default mode, pixels that sit on
    a decision band get a zero upstream gradient."""
    scene = synth.scene_spheres128(tets=False)
    sub = synth.subgrid(scene, 62, 66)
    p = oracle.make_params(s=20.0, tile=16)
    cam = sub.cams[0]
    up = list(synth.upstream_grads(2, [cam])[0])
    r = oracle.render(sub.V, sub.T, sub.f, sub.rgb, cam, p)
    mask = r["amb"] > 0
    up = [up[0] * ~mask[None], up[1] * ~mask, up[2] * ~mask]
    assert (r["alpha"] > 0).sum() > 50
    _fd_check(sub.V, sub.T, sub.f, sub.rgb, cam, p, up, 3, 7, h=1e-7, rtol=1e-4)


def test_colour_gradient_is_independent_of_colours(sphere16):
    """The image is linear in the vertex colours: d/drgb does not depend on
    rgb (equal up to the order of the per-thread FP64 sums)."""
    s, p, up, r = sphere16
    rgb2 = np.random.default_rng(12).uniform(size=s.rgb.shape).astype(np.float32)
    r2 = oracle.render(s.V, s.T, s.f, rgb2, s.cams[0], p, upstream=up)
    np.testing.assert_allclose(r2["drgb"], r["drgb"], rtol=1e-12, atol=1e-14)


def _check_blend_lists(s, p, r, cap):
    """Blended lists of every pixel: at most the hits, distinct slots whose
    bbox rect covers the pixel, in the order of the tile's sorted list, -1
    past the end."""
    bins = r["bins"]
    nb, sl = r["nblend"], r["blend_slots"]
    assert np.all(nb <= r["nfrag"])
    tx = bins["tiles_x"]
    pos_in_list = {}
    H, W = nb.shape
    for j in range(H):
        for i in range(W):
            n = int(nb[j, i])
            row = sl[j, i]
            k = min(n, cap)
            assert np.all(row[k:] == -1)
            if k == 0:
                continue
            t = (j // p.tile) * tx + i // p.tile
            a, b = bins["ranges"][t]
            if t not in pos_in_list:
                pos_in_list[t] = {int(v): q for q, v in enumerate(bins["key_val"][a:b])}
            pos = [pos_in_list[t][int(x)] for x in row[:k]]
            assert pos == sorted(pos) and len(set(pos)) == k
            for x in row[:k]:
                x0, x1, y0, y1 = (int(v) for v in bins["rect"][x])   # pixel bbox of the slot
                assert x0 <= i <= x1 and y0 <= j <= y1


def test_blend_lists_soft_surface(sphere16):
    """sphere16 at s = 175: blended counts below the hits where the pixel
    stops, and the recorded slots obey the list order (checked on the full
    128x128 view)."""
    s, p, up, r0 = sphere16
    r = oracle.render(s.V, s.T, s.f, s.rgb, s.cams[0], p, blend_cap=8)
    assert np.array_equal(r["image"], r0["image"])    # recording changes nothing
    nb = r["nblend"]
    assert nb.max() > 8 and (nb > 0).mean() > 0.1
    assert np.any(nb < r["nfrag"])                      # some pixels stop early
    _check_blend_lists(s, p, r, 8)


def test_blend_lists_pure_mode_blend_every_hit():
    """PURE mode (no stop, no skip) on a linear field that decreases along
    every camera ray (f = 0.6 c.x, c the unit vector to the camera), so every
    chord has f_prev > f_next and a positive alpha: every hit is blended and
    the blended count equals the hit count."""
    a, e = math.radians(-20.0), math.radians(15.0)
    c = np.array([math.cos(e) * math.cos(a), math.cos(e) * math.sin(a), math.sin(e)])
    V, T, f, rgb = small_grid(3, lambda X: 0.6 * X @ c)
    cam = synth.orbit_camera(-20.0, 15.0, 40, 40)
    p = oracle.make_params(s=6.0, tile=8, pure=True)
    r = oracle.render(V, T, f, rgb, cam, p, blend_cap=64)
    assert np.array_equal(r["nblend"], r["nfrag"]) and r["nblend"].max() > 2
    _check_blend_lists(None, p, r, 64)
