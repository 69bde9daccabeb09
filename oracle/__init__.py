"""CPU oracle for the tetrahedron splatting rasterizer — TEST INFRASTRUCTURE.

Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline leg may import this package.  The product path never does, and the
oracle shares no code with the CUDA path (it is a separate C++ library,
``oracle.cpp``, loaded here through ctypes).

What each function restates (paper sections):
  prefilter   Sec. 3.2 "Pre-filtering" with Eq. 1 at the max/min vertex SDF
  bin         Sec. 3.3 tile binning: near-plane/image culling, pixel bbox,
              (tile, mean vertex depth) keys, stable sort, per-tile ranges.
              The key path is an exact FP32 op sequence (see oracle.cpp).
  render      Sec. 3.2 + App. A.1/A.2 chord through the projected triangles,
              Eq. 1 opacity, Eq. 2 front-to-back blending (3DGS conventions),
              and the exact adjoint (compositing adjoint + dual numbers).
  fragment    one ray against one tet (App. A.1/A.2), for closed-form tests.
  tet_edges, regularizers
              Sec. 4.2 eikonal and normal-consistency losses of the grid's SDF
              with their gradients (``geometry_terms.cpp``).
  marching_tets
              Marching Tetrahedra mesh extraction (Sec. 3.1).
  survivor_bounds, fit_grid
              the coarse-to-fine pre-filter of App. B.1.

Parity status: pinned by the tests under ``tests/test_oracle_*.py``.
"""

from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, n) for n in ("oracle.cpp", "geometry_terms.cpp")]
_DEPS = _SRCS + [os.path.join(_HERE, "dual.h")]
_LIB = os.path.join(_HERE, "liboracle.so")

PURE = 1


class OrcCam(ctypes.Structure):
    _fields_ = [("R", ctypes.c_float * 9), ("t", ctypes.c_float * 3), ("fx", ctypes.c_float),
                ("fy", ctypes.c_float), ("cx", ctypes.c_float), ("cy", ctypes.c_float),
                ("znear", ctypes.c_float), ("width", ctypes.c_int32), ("height", ctypes.c_int32)]


class OrcParams(ctypes.Structure):
    _fields_ = [("s", ctypes.c_double), ("prefilter_thresh", ctypes.c_double),
                ("alpha_skip", ctypes.c_double), ("alpha_cap", ctypes.c_double),
                ("t_eps", ctypes.c_double), ("band", ctypes.c_double),
                ("tile", ctypes.c_int32), ("flags", ctypes.c_int32),
                ("window", ctypes.c_int32), ("pad", ctypes.c_int32)]


def build(force: bool = False) -> str:
    """Compile the oracle sources into liboracle.so (FP contraction off: the
    key path is an exact FP32 op sequence)."""
    if (not force and os.path.exists(_LIB)
            and all(os.path.getmtime(_LIB) >= os.path.getmtime(d) for d in _DEPS)):
        return _LIB
    cmd = ["g++", "-O2", "-std=c++17", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", *_SRCS, "-o", _LIB + ".tmp"]
    subprocess.check_call(cmd)
    os.replace(_LIB + ".tmp", _LIB)
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64, i32, f64 = ctypes.c_int64, ctypes.c_int32, ctypes.c_double
        L.orc_prefilter.argtypes = [i64, P, i64, P, P, P, P, P]
        L.orc_prefilter.restype = i64
        L.orc_bin_prepare.argtypes = [i64, P, P, P, P, i32, P, P, P, i32, P]
        L.orc_bin_prepare.restype = i64
        L.orc_bin_sort.argtypes = [i64, P, P, P, i32, P, P, P, P, P]
        L.orc_bin_sort.restype = i64
        L.orc_fragment.argtypes = [P, P, f64, f64, f64, f64, f64, f64, f64, P]
        L.orc_fragment.restype = ctypes.c_int
        L.orc_fragment_grad.argtypes = [P, P, f64, f64, f64, f64, f64, f64, f64, P, P]
        L.orc_fragment_grad.restype = ctypes.c_int
        L.orc_render.argtypes = [i64, P, P, P, P, i64, P, P, P, P, P, P,
                                 P, P, P, P, P, P, P, P, P, P, P, P, P, P, ctypes.c_int,
                                 P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, ctypes.c_int]
        L.orc_render.restype = ctypes.c_int
        L.orc_render_dirderiv.argtypes = [i64, P, P, P, P, i64, P, P, P, P, P, P, P, P, P,
                                          P, P, P, P, P, P, P, P]
        L.orc_render_dirderiv.restype = ctypes.c_int
        L.orc_tet_edges.argtypes = [i64, i64, P, P]
        L.orc_tet_edges.restype = i64
        L.orc_regularizers.argtypes = [i64, P, i64, P, P, i64, P, f64, f64, P, P, P]
        L.orc_regularizers.restype = None
        L.orc_regularizers_dirderiv.argtypes = [i64, P, i64, P, P, i64, P, f64, f64, P, P, P]
        L.orc_regularizers_dirderiv.restype = None
        L.orc_marching_tets.argtypes = [i64, P, i64, P, P, i64, P, P, P, i64, P, i64, P]
        L.orc_marching_tets.restype = ctypes.c_int
        L.orc_survivor_bounds.argtypes = [P, P, P, i64, P]
        L.orc_survivor_bounds.restype = None
        L.orc_fit_grid.argtypes = [i64, P, P, P, P, f64, P]
        L.orc_fit_grid.restype = None
        _lib = L
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def make_cam(cam) -> OrcCam:
    c = OrcCam()
    R = np.asarray(cam.R, dtype=np.float32).ravel()
    t = np.asarray(cam.t, dtype=np.float32).ravel()
    for i in range(9):
        c.R[i] = float(R[i])
    for i in range(3):
        c.t[i] = float(t[i])
    c.fx, c.fy, c.cx, c.cy, c.znear = cam.fx, cam.fy, cam.cx, cam.cy, cam.znear
    c.width, c.height = cam.width, cam.height
    return c


def make_params(s=175.0, tile=16, pure=False, prefilter_thresh=1.0 / 255.0,
                alpha_skip=1.0 / 255.0, alpha_cap=0.99, t_eps=1e-4, band=1e-4,
                window=0) -> OrcParams:
    """``window``: resort window N_w (0: tile order, < 0: full per-pixel sort)."""
    p = OrcParams()
    p.s = s
    p.prefilter_thresh = prefilter_thresh
    p.alpha_skip = alpha_skip
    p.alpha_cap = alpha_cap
    p.t_eps = t_eps
    p.band = band
    p.tile = tile
    p.flags = PURE if pure else 0
    p.window = window
    p.pad = 0
    return p


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def prefilter(T, f, params: OrcParams):
    T = _c(T, np.int32)
    f = _c(f, np.float32)
    K = len(T)
    keep = np.zeros(K, np.int8)
    amb = np.zeros(K, np.int8)
    amax = np.zeros(K, np.float64)
    n = lib().orc_prefilter(K, _p(T), len(f), _p(f), ctypes.byref(params), _p(keep), _p(amb),
                            _p(amax))
    if n < 0:
        raise ValueError("tet index outside [0, N)")
    surv = np.nonzero(keep)[0].astype(np.int32)
    return surv, amb.astype(bool), amax


def bin_view(surv, T, V, cam, tile: int, hull: bool = False):
    """Sec. 3.3 binning of one view; ``hull``: the tile test against the
    projected tet (only tiles whose (tile x bbox) corner pixel centres are not
    all outside one hull edge keep their key)."""
    surv = _c(surv, np.int32)
    T = _c(T, np.int32)
    V = _c(V, np.float32)
    c = make_cam(cam)
    ns = len(surv)
    rect = np.zeros((ns, 4), np.int32)
    zbits = np.zeros(ns, np.uint32)
    ntl = np.zeros(ns, np.int32)
    keep = np.zeros(ns, np.uint32)
    total = lib().orc_bin_prepare(ns, _p(surv), _p(T), _p(V), ctypes.byref(c), tile, _p(rect),
                                  _p(zbits), _p(ntl), 1 if hull else 0, _p(keep))
    tx = (cam.width + tile - 1) // tile
    ty = (cam.height + tile - 1) // tile
    ktile = np.zeros(total, np.int32)
    kz = np.zeros(total, np.uint32)
    kval = np.zeros(total, np.int32)
    ranges = np.zeros((tx * ty, 2), np.int32)
    n = lib().orc_bin_sort(ns, _p(rect), _p(zbits), ctypes.byref(c), tile, _p(ktile), _p(kz),
                           _p(kval), _p(ranges), _p(keep) if hull else None)
    assert n == total
    return dict(rect=rect, zbits=zbits, ntiles=ntl, key_tile=ktile, key_z=kz, key_val=kval,
                ranges=ranges, tiles_x=tx, tiles_y=ty)


def render(V, T, f, rgb, cam, params: OrcParams, surv=None, bins=None, upstream=None,
           nthreads: int = 0, V64=None, f64=None, rgb64=None, normals: bool = False,
           branch=None, abs_terms: bool = False, blend_cap: int = 0):
    """Render one view; returns a dict with image (3,H,W), alpha, depth, amb,
    alt_*, nfrag, the binning lists and (if ``upstream`` = (dimg, dalpha,
    ddepth) is given) the FP64 gradients dV, df, drgb.  ``V64``/``f64``/``rgb64``
    override the FP64 values used after binning (the lists come from the FP32
    inputs).  ``branch`` (H,W int8, optional): where 1, the gradient is that of
    the pixel's alternative branch (first ambiguous decision inverted).
    ``abs_terms``: also return dV_abs, df_abs, drgb_abs, the sums of the
    absolute values of the per-fragment terms of each gradient entry, and
    dV_kink, df_kink, drgb_kink (zero): per entry the sum over fragments whose
    ray passes within rounding of an edge of its entry or exit face of the
    change of the fragment's term under the other one-sided derivative, and
    dV_graze (df_graze, drgb_graze zero): per entry the sum over fragments of
    |the term through the opacity| / c^2, c the smaller |cos| between the
    pixel ray and the chord's entry and exit face normals.  ``blend_cap`` > 0:
    also return nblend (H,W int32: the pixel's blended fragments, primary
    branch) and blend_slots (H,W,blend_cap int32: the view slots of its first
    blend_cap blended fragments in blend order, -1 past the end)."""
    V = _c(V, np.float32)
    T = _c(T, np.int32)
    f = _c(f, np.float32)
    rgb = _c(rgb, np.float32)
    V64, f64, rgb64 = (None if a is None else _c(a, np.float64) for a in (V64, f64, rgb64))
    if surv is None:
        surv, _, _ = prefilter(T, f, params)
    if bins is None:
        bins = bin_view(surv, T, V, cam, params.tile)
    H, W = cam.height, cam.width
    c = make_cam(cam)
    img = np.zeros((3, H, W))
    alpha = np.zeros((H, W))
    depth = np.zeros((H, W))
    amb = np.zeros((H, W), np.int32)
    aimg = np.zeros((3, H, W))
    aalpha = np.zeros((H, W))
    adepth = np.zeros((H, W))
    nfrag = np.zeros((H, W), np.int32)
    N = len(V)
    dV = df = drgb = None
    gi = ga = gd = gn = None
    nrm = np.zeros((3, H, W)) if normals else None
    anrm = np.zeros((3, H, W)) if normals else None
    if upstream is not None:
        gi, ga, gd = (_c(u, np.float32) for u in upstream[:3])
        if len(upstream) > 3 and upstream[3] is not None:
            gn = _c(upstream[3], np.float32)
        dV = np.zeros((N, 3))
        df = np.zeros(N)
        drgb = np.zeros((N, 3))
    aV = af = argb = kV = kf = gzV = None
    if upstream is not None and abs_terms:
        aV, af, argb = np.zeros((N, 3)), np.zeros(N), np.zeros((N, 3))
        kV, kf, gzV = np.zeros((N, 3)), np.zeros(N), np.zeros((N, 3))
    br = None if branch is None else _c(branch, np.int8)
    if br is not None:
        assert br.shape == (H, W)
    surv = _c(surv, np.int32)
    nbl = bsl = None
    if blend_cap > 0:
        nbl = np.zeros((H, W), np.int32)
        bsl = np.full((H, W, blend_cap), -1, np.int32)
    rc = lib().orc_render(N, _p(V), _p(f), _p(rgb), _p(T), len(surv), _p(surv),
                          _p(bins["rect"]), ctypes.byref(c), ctypes.byref(params),
                          _p(bins["key_val"]), _p(bins["ranges"]), _p(img), _p(alpha), _p(depth),
                          _p(amb), _p(aimg), _p(aalpha), _p(adepth), _p(nfrag), _p(gi), _p(ga),
                          _p(gd), _p(dV), _p(df), _p(drgb), nthreads, _p(V64), _p(f64),
                          _p(rgb64), _p(nrm), _p(anrm), _p(gn), _p(br), _p(aV), _p(af),
                          _p(argb), _p(kV), _p(kf), _p(gzV), _p(nbl), _p(bsl), int(blend_cap))
    assert rc == 0
    out = dict(image=img, alpha=alpha, depth=depth, amb=amb, alt_image=aimg, alt_alpha=aalpha,
               alt_depth=adepth, nfrag=nfrag, surv=surv, bins=bins, normal=nrm, alt_normal=anrm)
    if blend_cap > 0:
        out.update(nblend=nbl, blend_slots=bsl)
    if upstream is not None:
        out.update(dV=dV, df=df, drgb=drgb)
        if abs_terms:
            out.update(dV_abs=aV, df_abs=af, drgb_abs=argb, dV_kink=kV, df_kink=kf,
                       drgb_kink=np.zeros_like(argb), dV_graze=gzV, df_graze=np.zeros_like(af),
                       drgb_graze=np.zeros_like(argb))
    return out


def dirderiv(V, T, f, rgb, cam, params: OrcParams, surv, bins, upstream, tV, tf, trgb,
             V64=None, f64=None, rgb64=None):
    """(L, dL) along the tangent (tV, tf, trgb) by one dual pass."""
    V = _c(V, np.float32)
    T = _c(T, np.int32)
    f = _c(f, np.float32)
    rgb = _c(rgb, np.float32)
    V64, f64, rgb64 = (None if a is None else _c(a, np.float64) for a in (V64, f64, rgb64))
    tV, tf, trgb = (_c(a, np.float64) for a in (tV, tf, trgb))
    surv = _c(surv, np.int32)
    gi, ga, gd = (_c(u, np.float32) for u in upstream[:3])
    gn = _c(upstream[3], np.float32) if len(upstream) > 3 and upstream[3] is not None else None
    c = make_cam(cam)
    out = np.zeros(2)
    lib().orc_render_dirderiv(len(V), _p(V), _p(f), _p(rgb), _p(T), len(surv),
                              _p(surv), _p(bins["rect"]), ctypes.byref(c),
                              ctypes.byref(params), _p(bins["key_val"]), _p(bins["ranges"]),
                              _p(gi), _p(ga), _p(gd), _p(tV), _p(tf), _p(trgb), _p(out),
                              _p(V64), _p(f64), _p(rgb64), _p(gn))
    return float(out[0]), float(out[1])


def fragment(X, F, px, py, fx, fy, cx, cy, s):
    """One ray through pixel centre (px, py) against one tet given by its
    camera-space vertices X (4x3) and SDF F (4).  Returns None on a miss, else
    (f_prev, f_next, z_in, z_out, alpha)."""
    X = _c(X, np.float64).ravel()
    F = _c(F, np.float64).ravel()
    out = np.zeros(5)
    hit = lib().orc_fragment(_p(X), _p(F), px, py, fx, fy, cx, cy, s, _p(out))
    return tuple(out) if hit else None


def fragment_grad(X, F, px, py, fx, fy, cx, cy, s):
    X = _c(X, np.float64).ravel()
    F = _c(F, np.float64).ravel()
    a = np.zeros(1)
    g = np.zeros(16)
    hit = lib().orc_fragment_grad(_p(X), _p(F), px, py, fx, fy, cx, cy, s, _p(a), _p(g))
    return (float(a[0]), g) if hit else None


def tet_edges(T, N=None):
    """Unique edges of a tet grid as an (E, 2) int32 array of (lo, hi) pairs
    sorted lexicographically."""
    T = _c(T, np.int32)
    N = int(T.max()) + 1 if N is None else int(N)
    out = np.zeros((6 * len(T), 2), np.int32)
    n = lib().orc_tet_edges(N, len(T), _p(T), _p(out))
    if n < 0:
        raise ValueError("tet index outside [0, N)")
    return out[:n].copy()


def regularizers(V, T, f, edges, w_eik=1.0, w_nc=1.0, grad=True):
    """Sec. 4.2 eikonal and normal-consistency losses (FP64) and the gradients
    of w_eik L_eik + w_nc L_nc with respect to V and f."""
    V = _c(V, np.float64)
    f = _c(f, np.float64)
    T = _c(T, np.int32)
    edges = _c(edges, np.int32)
    out = np.zeros(2)
    dV = np.zeros_like(V) if grad else None
    df = np.zeros_like(f) if grad else None
    lib().orc_regularizers(len(V), _p(V), len(T), _p(T), _p(f), len(edges), _p(edges),
                           float(w_eik), float(w_nc), _p(out), _p(dV), _p(df))
    return dict(L_eik=float(out[0]), L_nc=float(out[1]), dV=dV, df=df)


def regularizers_dirderiv(V, T, f, edges, w_eik, w_nc, tV, tf):
    """(value, directional derivative along (tV, tf)) of w_eik L_eik + w_nc
    L_nc by dual numbers."""
    V, f, tV, tf = (_c(x, np.float64) for x in (V, f, tV, tf))
    T = _c(T, np.int32)
    edges = _c(edges, np.int32)
    out = np.zeros(2)
    lib().orc_regularizers_dirderiv(len(V), _p(V), len(T), _p(T), _p(f), len(edges), _p(edges),
                                    float(w_eik), float(w_nc), _p(tV), _p(tf), _p(out))
    return float(out[0]), float(out[1])


def marching_tets(V, T, f, edges=None):
    """Marching Tetrahedra: returns dict(verts (nv, 3) float64, vert_edge
    (nv,) int32 index into ``edges``, tris (nt, 3) int32, edges)."""
    V = _c(V, np.float64)
    f = _c(f, np.float64)
    T = _c(T, np.int32)
    edges = tet_edges(T, len(V)) if edges is None else _c(edges, np.int32)
    E = len(edges)
    verts = np.zeros((E, 3))
    vedge = np.zeros(E, np.int32)
    tris = np.zeros((2 * len(T), 3), np.int32)
    counts = np.zeros(2, np.int64)
    rc = lib().orc_marching_tets(len(V), _p(V), len(T), _p(T), _p(f), E, _p(edges), _p(verts),
                                 _p(vedge), E, _p(tris), 2 * len(T), _p(counts))
    if rc != 0:
        raise ValueError("a tet edge is missing from the edge list")
    nv, nt = int(counts[0]), int(counts[1])
    return dict(verts=verts[:nv].copy(), vert_edge=vedge[:nv].copy(), tris=tris[:nt].copy(),
                edges=edges)


def survivor_bounds(V, T, surv):
    """(xmin, ymin, zmin, xmax, ymax, zmax) of the survivors' vertices."""
    V = _c(V, np.float32)
    T = _c(T, np.int32)
    surv = _c(surv, np.int32)
    out = np.zeros(6, np.float32)
    lib().orc_survivor_bounds(_p(V), _p(T), _p(surv), len(surv), _p(out))
    return out


def fit_grid(V, grid_lo, grid_hi, aabb, pad=0.05):
    """Grid vertices mapped per axis from [grid_lo, grid_hi] onto the bounds
    widened by pad * extent (FP64)."""
    V = _c(V, np.float32)
    lo = _c(grid_lo, np.float64)
    hi = _c(grid_hi, np.float64)
    aabb = _c(aabb, np.float32)
    out = np.zeros(V.shape, np.float64)
    lib().orc_fit_grid(len(V), _p(V), _p(lo), _p(hi), _p(aabb), float(pad), _p(out))
    return out
