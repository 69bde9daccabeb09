"""The differentiable entry points: ``render()`` and the ``TetRender`` /
``TetRenderBatch`` autograd Functions (the hand-written adjoint kernels behind
torch.autograd).

* gradients through ``torch.autograd.grad`` of ``render()`` against the FP64
  oracle, per element (sphere16 and the 4^3 sub-grid of the benchmark scene);
* central finite differences of the GPU forward against the autograd
  directional derivative in PURE mode on a 2^3 grid;
* two renders followed by two backwards: each backward gets its own
  forward's gradient (``render()``), or raises (one shared ``Rasterizer``).
"""

import numpy as np
import pytest
import torch

import synth
from paper_2406_01579_b300 import (Params, Rasterizer, SceneTensors, TetRender, TetRenderBatch,
                                   TetsError, render)
from parity import cat_upstream, compare_with_oracle, elementwise, prepare_upstream, to_dev

pytestmark = pytest.mark.gpu


def _leaves(scene):
    st = to_dev(scene)
    return (st.V.clone().requires_grad_(True), st.T, st.f.clone().requires_grad_(True),
            st.rgb.clone().requires_grad_(True))


def _loss(views_out, ups):
    """sum over views of <upstream, outputs> (the loss whose gradient the
    oracle computes)."""
    L = 0.0
    for out, up in zip(views_out, ups):
        for x, u in zip(out, up):
            L = L + (x * torch.as_tensor(u, device=x.device).reshape(x.shape)).sum()
    return L


def _render_vs_oracle(scene, cams, p, seed, name):
    views = [(c, 0) for c in cams]
    ups0 = synth.upstream_grads(seed, cams)
    _, ups, brs, orcs0, report = prepare_upstream([scene], views, p, ups0, name)
    V, T, f, rgb = _leaves(scene)
    out = render(V, T, f, rgb, cams, p)
    g = torch.autograd.grad(_loss(out, ups), (V, f, rgb))
    torch.cuda.synchronize()
    return compare_with_oracle([scene], views, p, ups, brs, orcs0, [g], report, name)


def test_render_grad_sphere16():
    sc = synth.scene_sphere16()
    _render_vs_oracle(sc, sc.cams, Params(s=175.0, tile=16), 0, "render sphere16")


def test_render_grad_subgrid():
    """The 4^3 sub-grid (cubes [62,66)^3) of the benchmark's 128^3 scene, two
    of its cameras in one render call (views of uneven content)."""
    sub = synth.subgrid(synth.scene_spheres128(), 62, 66)
    cams = [c for c in sub.cams]
    _render_vs_oracle(sub, cams, Params(s=175.0, tile=8), 2, "render subgrid")


def test_render_batch_function():
    """TetRenderBatch over two scenes and three views equals the per-element
    oracle gradient of both scenes."""
    rng = np.random.default_rng(5)
    s0 = synth.scene_sphere16()
    s1 = synth.Scene(8, *synth.random_scene(rng, 8, "torus")[:4], [], "torus8")
    cams = [synth.orbit_camera(30.0, 20.0, 96, 96), synth.random_camera(rng, 64, 48),
            synth.random_camera(rng, 80, 80)]
    views = [(cams[0], 0), (cams[1], 1), (cams[2], 0)]
    p = Params(s=60.0, tile=16)
    _, ups, brs, orcs0, report = prepare_upstream([s0, s1], views, p,
                                                  synth.upstream_grads(17, cams), "batch fn")
    leaves = [_leaves(s0), _leaves(s1)]
    r = Rasterizer([SceneTensors(V.detach(), T, f.detach(), c.detach())
                    for V, T, f, c in leaves], views, p)
    flat = [x for V, T, f, c in leaves for x in (V, f, c)]
    out = TetRenderBatch.apply(r, True, *flat)
    u = cat_upstream(ups)
    L = sum((o * w).sum() for o, w in zip(out, u))
    g = torch.autograd.grad(L, flat)
    torch.cuda.synchronize()
    compare_with_oracle([s0, s1], views, p, ups, brs, orcs0, [g[0:3], g[3:6]], report,
                        "batch fn")


def test_render_finite_differences_pure():
    """PURE mode (no thresholds) on a 2^3 grid: the autograd directional
    derivative equals central finite differences of the GPU forward along
    random directions in rgb (the image is linear in it), in f and in V.  The
    field decreases along every camera ray (f = 0.6 c.x + 0.1 |x|^2 - 0.1, c
    the unit vector to the camera), so no chord has f_prev = f_next, where
    Eq. 1's max(., 0) has a kink.  In V every tet's silhouette and every face
    switch of a chord is a kink that a finite step can cross: the FP64
    oracle's central difference at the same step, against its exact
    dual-number derivative, measures that part of the gap, which the GPU's
    gap may use besides its rounding."""
    import oracle
    from parity import oracle_params
    n, s = 2, 2.0
    V0 = synth.grid_vertices(n)
    T = synth.grid_tets(n)
    cam = synth.orbit_camera(33.0, 21.0, 48, 48)
    a, e = np.radians(33.0), np.radians(21.0)
    c = np.array([np.cos(e) * np.cos(a), np.cos(e) * np.sin(a), np.sin(e)])
    X = V0.astype(np.float64)
    f0 = (0.6 * X @ c + 0.1 * (X ** 2).sum(1) - 0.1).astype(np.float32)
    rgb0 = np.random.default_rng(n).uniform(size=(len(V0), 3)).astype(np.float32)
    p = Params(s=s, tile=8, pure=True)
    op = oracle_params(p)
    up = synth.upstream_grads(41, [cam])[0]
    surv, _, _ = oracle.prefilter(T, f0, op)
    bins = oracle.bin_view(surv, T, V0, cam, p.tile)
    dev = "cuda"
    Tt = torch.from_numpy(T).to(dev)
    w = [torch.from_numpy(u).to(dev).double() for u in up]

    def loss(V, f, rgb):
        out = render(V, Tt, f, rgb, [cam], p)[0]
        return sum((x.double() * u).sum() for x, u in zip(out, w))

    def oracle_loss(Vd, fd_, cd):
        r = oracle.render(V0, T, f0, rgb0, cam, op, surv=surv, bins=bins, V64=Vd, f64=fd_,
                          rgb64=cd)
        return float((up[0] * r["image"]).sum() + (up[1] * r["alpha"]).sum() +
                     (up[2] * r["depth"]).sum())

    V = torch.from_numpy(V0).to(dev).requires_grad_(True)
    f = torch.from_numpy(f0).to(dev).requires_grad_(True)
    rgb = torch.from_numpy(rgb0).to(dev).requires_grad_(True)
    gV, gf, gc = torch.autograd.grad(loss(V, f, rgb), (V, f, rgb))
    with torch.no_grad():
        out0 = render(V, Tt, f, rgb, [cam], p)[0]
        mag = float(sum((x.double().abs() * u.abs()).sum() for x, u in zip(out0, w)))
    rng = np.random.default_rng(3)
    for which, h, tol in (("rgb", 1e-2, 1e-3), ("f", 1e-4, 5e-3), ("V", 1e-4, 5e-3)):
        for _ in range(3):
            tV = np.zeros_like(V0) if which != "V" else rng.normal(size=V0.shape).astype(np.float32)
            tf = np.zeros_like(f0) if which != "f" else rng.normal(size=f0.shape).astype(np.float32)
            tc = np.zeros_like(rgb0) if which != "rgb" else rng.normal(size=rgb0.shape).astype(np.float32)
            tVt, tft, tct = (torch.from_numpy(x).to(dev) for x in (tV, tf, tc))
            ad = float((gV.double() * tVt).sum() + (gf.double() * tft).sum() +
                       (gc.double() * tct).sum())
            with torch.no_grad():
                lp = float(loss(V + h * tVt, f + h * tft, rgb + h * tct))
                lm = float(loss(V - h * tVt, f - h * tft, rgb - h * tct))
            fd = (lp - lm) / (2 * h)
            # the oracle at the same step and its exact derivative
            X64, f64, c64 = (x.astype(np.float64) for x in (V0, f0, rgb0))
            t64 = [x.astype(np.float64) for x in (tV, tf, tc)]
            fd_o = (oracle_loss(X64 + h * t64[0], f64 + h * t64[1], c64 + h * t64[2]) -
                    oracle_loss(X64 - h * t64[0], f64 - h * t64[1], c64 - h * t64[2])) / (2 * h)
            _, d_o = oracle.dirderiv(V0, T, f0, rgb0, cam, op, surv, bins, up, *t64, V64=X64)
            kink = abs(fd_o - d_o)
            print(f"[fd] {which}: autograd {ad:.6g} fd {fd:.6g} | oracle exact {d_o:.6g} "
                  f"fd {fd_o:.6g} kink {kink:.3g}")
            assert abs(ad - d_o) <= 1e-3 * abs(d_o) + 1e-6 * mag, (which, ad, d_o)
            assert abs(ad - fd) <= tol * abs(ad) + 2 * kink, (which, ad, fd, kink)


def test_two_renders_two_backwards():
    """Two render() calls before either backward (e.g. a second batch of views
    of the same shape): each backward gets the gradient of its own forward,
    equal to that forward rendered and differentiated alone."""
    sc = synth.scene_sphere16()
    p = Params(s=120.0, tile=16)
    cams = [synth.orbit_camera(30.0, 20.0, 96, 96), synth.orbit_camera(-60.0, 35.0, 96, 96)]
    ups = [synth.upstream_grads(50 + i, [c])[0] for i, c in enumerate(cams)]
    alone = []
    for c, u in zip(cams, ups):
        V, T, f, rgb = _leaves(sc)
        out = render(V, T, f, rgb, [c], p)
        alone.append(torch.autograd.grad(_loss(out, [u]), (V, f, rgb)))
    V, T, f, rgb = _leaves(sc)
    outs = [render(V, T, f, rgb, [c], p) for c in cams]       # both forwards first
    L = [_loss(o, [u]) for o, u in zip(outs, ups)]
    g1 = torch.autograd.grad(L[1], (V, f, rgb), retain_graph=True)
    g0 = torch.autograd.grad(L[0], (V, f, rgb))
    for got, ref in ((g0, alone[0]), (g1, alone[1])):
        for a, b in zip(got, ref):
            a, b = a.cpu().numpy(), b.cpu().numpy()
            frac, ratio, _ = elementwise(a, b, np.abs(b))
            assert frac == 1.0, ratio


def test_stale_backward_raises():
    """One shared Rasterizer, two forwards, then the first forward's backward:
    the workspace holds the second forward's lists, so it raises instead of
    returning the wrong gradient."""
    sc = synth.scene_sphere16()
    V, T, f, rgb = _leaves(sc)
    r = Rasterizer([SceneTensors(V.detach(), T, f.detach(), rgb.detach())],
                   [(synth.orbit_camera(30.0, 20.0, 64, 64), 0)], Params(s=120.0, tile=16))
    out0 = TetRender.apply(V, f, rgb, r, True)
    out1 = TetRender.apply(V, f, rgb, r, True)
    g = torch.autograd.grad(out1[0].sum(), (V, f, rgb), retain_graph=True)   # latest: fine
    assert all(torch.isfinite(x).all() for x in g)
    with pytest.raises(TetsError):
        torch.autograd.grad(out0[0].sum(), (V, f, rgb))


def test_autograd_rejects_accumulating_rasterizer():
    sc = synth.scene_sphere16()
    V, T, f, rgb = _leaves(sc)
    r = Rasterizer([SceneTensors(V.detach(), T, f.detach(), rgb.detach())],
                   [(synth.orbit_camera(30.0, 20.0, 32, 32), 0)],
                   Params(s=120.0, tile=16, accum_grad=True))
    with pytest.raises(TetsError):
        TetRender.apply(V, f, rgb, r, True)
