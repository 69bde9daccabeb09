"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs, and compare them.

Comparison rules
* keys, ranges, survivors: bit for bit, after removing tets whose alpha_max
  lies in the oracle's decision band around T_f (FP32 vs FP64 may legitimately
  disagree on those; they never contribute since alpha <= alpha_max).
* image/alpha/depth: max abs error <= 1e-4 per pixel against the oracle's
  primary branch, or against its alternative branch when the pixel met a
  decision (cap, skip, stop) within the band of its threshold.
* gradients, per element: |gpu - oracle| <= GRAD_TOL |oracle| + KAPPA S
  + K + C_GRAZE u G + FLOOR max|oracle|, where S is the oracle's sum of the
  absolute values of the per-fragment terms of that entry (the scale of the
  rounding that the GPU's FP32 evaluation of those terms and their atomic
  sums in another order can show), K its kink allowance (fragments whose ray
  passes within rounding of a tet edge, where either one-sided derivative is
  correct) and G the sum of its opacity terms weighted by 1/c^2, c the
  grazing cosine of the chord's entry or exit face (dV only).  At band pixels the oracle differentiates
  the branch the GPU took, read off the GPU's own final transmittance; only
  pixels whose two branches cannot be told apart get a zero upstream
  gradient on both sides, and their count is reported.  The max-normalised
  error max |gpu - oracle| / max |oracle| is reported beside it.
"""

from __future__ import annotations

import numpy as np
import torch

import oracle
import synth
from paper_2406_01579_b300 import Params, Rasterizer, SceneTensors

IMG_TOL = 1e-4
GRAD_TOL = 1e-3
# per-element gradient check (see the module docstring)
KAPPA = 1e-4
FLOOR = 1e-6
# grazing incidence: a fragment whose chord enters or leaves through a face
# seen at a small angle c between the face normal and the ray has an
# ill-conditioned entry or exit point; its terms through the opacity carry an
# FP32 rounding error of about u / c^2 times the largest of them (the
# record's face coefficients scale with 1 / e, e the face plane's distance
# from the camera centre, which is proportional to c, the derivative takes
# two of them, and the record-field gradients are shared by the tet's four
# vertices).  The bound adds C_GRAZE u sum(max |term| / c^2) per dV entry.
C_GRAZE = 32.0
U32 = 2.0 ** -24
# band pixels whose branches' final transmittances differ by less than this
# (relative) cannot be told apart by the GPU's FP32 transmittance
T_SEP = 3e-4
# band pixels (a decision within the band of its threshold) allowed per view;
# measured on sphere16 at s = 20 / 175 / 620: 0.02% / 0.12% / 0.09%, all of
# them cap decisions (alpha within 1e-4 of 0.99)
BAND_MAX = 0.005


def to_dev(scene_or_arrays, device="cuda"):
    if isinstance(scene_or_arrays, synth.Scene):
        V, T, f, rgb = scene_or_arrays.V, scene_or_arrays.T, scene_or_arrays.f, scene_or_arrays.rgb
    else:
        V, T, f, rgb = scene_or_arrays
    return SceneTensors(torch.from_numpy(np.ascontiguousarray(V, np.float32)).to(device),
                        torch.from_numpy(np.ascontiguousarray(T, np.int32)).to(device),
                        torch.from_numpy(np.ascontiguousarray(f, np.float32)).to(device),
                        torch.from_numpy(np.ascontiguousarray(rgb, np.float32)).to(device))


def oracle_params(p: Params, band=1e-4):
    """The oracle gets the FP32 values the C ABI receives (as FP64)."""
    f = lambda x: float(np.float32(x))
    return oracle.make_params(s=f(p.s), tile=p.tile, pure=p.pure,
                              prefilter_thresh=f(p.prefilter_thresh), alpha_skip=f(p.alpha_skip),
                              alpha_cap=f(p.alpha_cap), t_eps=f(p.t_eps), band=band,
                              window=int(p.resort_window))


def gpu_run(scenes, views, params: Params, upstream=None, lists=False):
    """scenes: list of synth.Scene or (V,T,f,rgb); views: list of (cam, scene_idx).
    Returns per-view outputs (numpy), optional gradients per scene, lists."""
    st = [to_dev(s) for s in scenes]
    r = Rasterizer(st, views, params)
    res = r.forward()
    out = dict(raster=r, views=[tuple(x.cpu().numpy() for x in v)
                                for v in r.view_outputs(*res)])
    if lists:
        out["lists"] = {k: (v.cpu().numpy() if torch.is_tensor(v) else v)
                        for k, v in r.debug_lists().items() if k not in ("surv", "info")}
        out["surv"] = r.debug_lists()["surv"][0].cpu().numpy()
        out["info"] = r.info()
    if upstream is not None:
        gi = torch.from_numpy(np.concatenate([u[0].reshape(-1) for u in upstream])).cuda()
        ga = torch.from_numpy(np.concatenate([u[1].reshape(-1) for u in upstream])).cuda()
        gd = torch.from_numpy(np.concatenate([u[2].reshape(-1) for u in upstream])).cuda()
        gn = None
        if len(upstream[0]) > 3:
            gn = torch.from_numpy(np.concatenate([u[3].reshape(-1) for u in upstream])).cuda()
        grads = r.backward(gi, ga, gd, dnormal=gn)
        out["grads"] = [tuple(g.cpu().numpy().astype(np.float64) for g in gs) for gs in grads]
    torch.cuda.synchronize()
    return out


def oracle_run(scene, cam, params: Params, upstream=None, branch=None, abs_terms=False,
               pre=None, fp64=None):
    """``pre``: (surv, amb_tets, bins) of an earlier call on the same scene and
    camera, to skip the pre-filter and binning.  ``fp64``: (V64, f64, rgb64)
    values used after binning instead of the FP32 inputs (the oracle at
    perturbed inputs with the same lists)."""
    if isinstance(scene, synth.Scene):
        V, T, f, rgb = scene.V, scene.T, scene.f, scene.rgb
    else:
        V, T, f, rgb = scene
    op = oracle_params(params)
    if pre is None:
        surv, amb_t, _ = oracle.prefilter(T, f, op)
        bins = oracle.bin_view(surv, T, V, cam, params.tile, hull=params.hull)
    else:
        surv, amb_t, bins = pre
    V64, f64, rgb64 = fp64 if fp64 is not None else (None, None, None)
    r = oracle.render(V, T, f, rgb, cam, op, surv=surv, bins=bins, upstream=upstream,
                      normals=params.normals, branch=branch, abs_terms=abs_terms, V64=V64,
                      f64=f64, rgb64=rgb64)
    r["amb_tets"] = amb_t
    r["pre"] = (surv, amb_t, bins)
    return r


def masked_upstream(up, amb):
    """Zero the upstream gradient at band pixels."""
    m = amb > 0
    out = (up[0] * ~m[None], up[1] * ~m, up[2] * ~m)
    if len(up) > 3:
        out = out + (up[3] * ~m[None],)
    return out


def compare_images(gpu_view, orc, tol=IMG_TOL):
    """Returns (n_bad, n_amb_pixels, max_err_on_unambiguous)."""
    gi, ga, gd = gpu_view[:3]
    prim = [orc["image"], orc["alpha"][None], orc["depth"][None]]
    alt = [orc["alt_image"], orc["alt_alpha"][None], orc["alt_depth"][None]]
    got = [gi, ga[None], gd[None]]
    if len(gpu_view) > 3:           # normal map channel
        prim.append(orc["normal"])
        alt.append(orc["alt_normal"])
        got.append(gpu_view[3])
    prim, alt = np.concatenate(prim, 0), np.concatenate(alt, 0)
    got = np.concatenate(got, 0).astype(np.float64)
    e1 = np.abs(got - prim).max(0)
    e2 = np.abs(got - alt).max(0)
    amb = orc["amb"] > 0
    ok = (e1 <= tol) | (amb & (e2 <= tol))
    multi = orc["amb"] >= 2
    bad = ~ok & ~multi
    return int(bad.sum()), int(amb.sum()), float(e1[~amb].max() if (~amb).any() else 0.0), \
        int((~ok & multi).sum())


def gpu_key_triples(lists, surv_gpu, view_tile_base=0, rec_base=0):
    keys = lists["keys"].view(np.uint64) if lists["keys"].dtype == np.int64 else lists["keys"]
    db, zmin = lists["depth_bits"], lists["zmin_bits"]
    tile = (keys >> np.uint64(db)).astype(np.int64) - view_tile_base
    z = (keys & np.uint64((1 << db) - 1)).astype(np.int64) + zmin
    slot = lists["vals"].astype(np.int64) - rec_base
    orig = surv_gpu[slot]
    return tile, z.astype(np.uint32), orig


def compare_keys(gpu, orc):
    """Bit-exact comparison of the sorted (tile, zbits, tet) lists and ranges."""
    lists = gpu["lists"]
    surv_g = gpu["surv"]
    surv_o = orc["surv"]
    band = orc["amb_tets"]
    band_ids = np.nonzero(band)[0]
    # survivor sets agree outside the band
    sg = np.setdiff1d(surv_g, band_ids)
    so = np.setdiff1d(surv_o, band_ids)
    np.testing.assert_array_equal(sg, so)
    assert np.all(np.diff(surv_g) > 0), "survivors not in original order"
    t_g, z_g, id_g = gpu_key_triples(lists, surv_g)
    b = orc["bins"]
    t_o, z_o, id_o = b["key_tile"].astype(np.int64), b["key_z"], surv_o[b["key_val"]]
    keep_g = ~np.isin(id_g, band_ids)
    keep_o = ~np.isin(id_o, band_ids)
    np.testing.assert_array_equal(t_g[keep_g], t_o[keep_o])
    np.testing.assert_array_equal(z_g[keep_g], z_o[keep_o])
    np.testing.assert_array_equal(id_g[keep_g], id_o[keep_o])
    if len(band_ids) == 0 or (keep_g.all() and keep_o.all()):
        ntiles = len(b["ranges"])
        np.testing.assert_array_equal(lists["ranges"][:ntiles], b["ranges"])
    return len(t_g)


def grad_rel_err(g, o):
    den = np.abs(o).max()
    return float(np.abs(g - o).max() / den) if den > 0 else float(np.abs(g).max())


# ---------------------------------------------------------------------------
# strict gradient parity
# ---------------------------------------------------------------------------
def select_branches(gpu_view, gpu_T, orc, tol=IMG_TOL, t_sep=T_SEP):
    """Which of the oracle's branches each pixel of the GPU took: 0 primary, 1
    alternative (first ambiguous decision inverted), -1 undecidable.  Pixels
    without an ambiguous decision are 0.  A band pixel takes the branch whose
    final transmittance is nearer (in ratio) to the GPU's; it is undecidable
    when the two branches' transmittances differ by less than t_sep
    (relative) or when the chosen branch's image does not match within tol
    (a later ambiguous decision flipped instead)."""
    amb = orc["amb"] > 0
    br = np.zeros(amb.shape, np.int8)
    if not amb.any():
        return br
    lg = lambda x: np.log(np.clip(x, 1e-300, None))
    Tg = lg(np.asarray(gpu_T, np.float64))
    Tp, Ta = lg(1.0 - orc["alpha"]), lg(1.0 - orc["alt_alpha"])
    dp, da, sep = np.abs(Tg - Tp), np.abs(Tg - Ta), np.abs(Tp - Ta)
    gi, ga, gd = gpu_view[:3]
    got = [gi, ga[None], gd[None]]
    prim = [orc["image"], orc["alpha"][None], orc["depth"][None]]
    alt = [orc["alt_image"], orc["alt_alpha"][None], orc["alt_depth"][None]]
    if len(gpu_view) > 3:
        got.append(gpu_view[3])
        prim.append(orc["normal"])
        alt.append(orc["alt_normal"])
    got = np.concatenate(got, 0).astype(np.float64)
    e1 = np.abs(got - np.concatenate(prim, 0)).max(0)
    e2 = np.abs(got - np.concatenate(alt, 0)).max(0)
    # a band pixel without a decision to invert (a near tie of two entry
    # depths in the resort window) has alt == primary: primary if it matches
    same = np.all(np.concatenate(prim, 0) == np.concatenate(alt, 0), axis=0)
    take_alt = amb & ~same & (da < dp)
    br[take_alt] = 1
    err = np.where(take_alt, e2, e1)
    br[amb & ((~same & (sep < t_sep)) | (err > tol))] = -1
    return br


def elementwise(g, o, oabs, kink=None, rtol=GRAD_TOL, kappa=KAPPA, floor=FLOOR):
    """(fraction of entries within |g-o| <= rtol|o| + kappa oabs + kink +
    floor max|o|, worst ratio of error to that bound, max-normalised error)."""
    g, o, oabs = (np.asarray(x, np.float64).ravel() for x in (g, o, oabs))
    kink = np.zeros_like(o) if kink is None else np.asarray(kink, np.float64).ravel()
    scale = np.abs(o).max() if o.size else 0.0
    err = np.abs(g - o)
    bound = rtol * np.abs(o) + kappa * oabs + kink + floor * scale
    ok = err <= bound
    ratio = float((err / np.where(bound > 0, bound, 1e-300)).max()) if o.size else 0.0
    maxnorm = float(err.max() / scale) if scale > 0 else float(err.max() if err.size else 0.0)
    return float(ok.mean()) if o.size else 1.0, ratio, maxnorm


def prepare_upstream(scenes, views, params: Params, upstream, name="", max_undecided=None):
    """A forward of the CUDA path (through the C ABI) and of the oracle: checks
    the images, picks per band pixel the branch the GPU took and zeroes the
    upstream gradient at undecidable pixels.  Returns (raster, upstream per
    view, branch per view (int8, 1 = alternative), oracle forwards, report)."""
    st = [to_dev(s) for s in scenes]
    r = Rasterizer(st, views, params)
    res = r.forward()
    outs = [tuple(x.cpu().numpy() for x in v) for v in r.view_outputs(*res)]
    Tg = r.debug_pixels()[0].cpu().numpy()
    report = {"views": [], "tensors": {}}
    ups, brs, orcs0 = [], [], []
    for i, ((cam, si), up) in enumerate(zip(views, upstream)):
        H, W = int(cam.height), int(cam.width)
        o0 = oracle_run(scenes[si], cam, params)
        T_v = Tg[r.pix_off[i]:r.pix_off[i] + H * W].reshape(H, W)
        br = select_branches(outs[i], T_v, o0)
        bad, namb, emax, multi = compare_images(outs[i], o0)
        assert bad == 0, f"{name} view{i}: {bad} pixels off by > {IMG_TOL}"
        assert namb <= BAND_MAX * H * W, f"{name} view{i}: {namb} band pixels"
        und = int((br < 0).sum())
        lim = max(2, int(1e-4 * H * W)) if max_undecided is None else max_undecided
        assert und <= lim, f"{name} view{i}: {und} undecidable band pixels"
        keep = br >= 0
        up = tuple(np.asarray(u, np.float32) * (keep[None] if np.ndim(u) == 3 else keep)
                   for u in up)
        ups.append(up)
        brs.append((br == 1).astype(np.int8))
        orcs0.append(o0)
        report["views"].append({"band": namb, "alt": int((br == 1).sum()), "undecided": und,
                                "pixels": H * W, "max_img_err": emax})
    return r, ups, brs, orcs0, report


def compare_with_oracle(scenes, views, params: Params, ups, brs, orcs0, grads, report, name="",
                        min_pass=1.0):
    """Per-element comparison of the GPU gradients ``grads`` (per scene (dV,
    df, drgb) tensors) with the oracle's for the upstream ``ups`` and the
    branches ``brs`` (from prepare_upstream)."""
    for si, sc in enumerate(scenes):
        N = len(sc.V) if isinstance(sc, synth.Scene) else len(sc[0])
        acc = {k: np.zeros(shp) for k, shp in (("dV", (N, 3)), ("df", (N,)), ("drgb", (N, 3)))}
        absacc = {k: np.zeros_like(v) for k, v in acc.items()}
        kinkacc = {k: np.zeros_like(v) for k, v in acc.items()}
        graze = {k: np.zeros_like(v) for k, v in acc.items()}
        for i, (cam, sj) in enumerate(views):
            if sj != si:
                continue
            o = oracle_run(sc, cam, params, upstream=ups[i], branch=brs[i], abs_terms=True,
                           pre=orcs0[i]["pre"])
            for k in acc:
                acc[k] += o[k]
                absacc[k] += o[k + "_abs"]
                kinkacc[k] += o[k + "_kink"]
                graze[k] += o[k + "_graze"]
        fails = []
        for k, g in zip(("dV", "df", "drgb"), grads[si]):
            g = g.detach().cpu().numpy() if torch.is_tensor(g) else np.asarray(g)
            extra = kinkacc[k] + C_GRAZE * U32 * graze[k]
            frac, ratio, maxnorm = elementwise(g, acc[k], absacc[k], extra)
            report["tensors"][f"s{si}.{k}"] = {
                "pass": frac, "worst": ratio, "maxnorm": maxnorm,
                "kink_entries": int((kinkacc[k] > 0).sum()),
                "graze_entries": int((~_within(g, acc[k], absacc[k], kinkacc[k])).sum())}
            if frac < min_pass:
                fails.append(f"{name} scene{si} {k}: {frac:.6f} of entries within the bound "
                             f"(worst error/bound {ratio:.3g}, max-normalised {maxnorm:.3e})")
                _dump(name, si, k, g, acc[k], absacc[k], kinkacc[k], C_GRAZE * U32 * graze[k])
        assert not fails, "; ".join(fails)
    print(f"[grad parity] {name}: {report}")
    return report


def _within(g, o, oabs, kink):
    g, o, oabs, kink = (np.asarray(x, np.float64).ravel() for x in (g, o, oabs, kink))
    return np.abs(g - o) <= (GRAD_TOL * np.abs(o) + KAPPA * oabs + kink +
                             FLOOR * np.abs(o).max())


def _dump(name, si, k, g, o, oabs, kink, cond=None):
    """With TTS_PARITY_DUMP=<dir>: the entries outside the bound without the
    grazing term (index, GPU value, oracle value, sum of absolute terms, kink
    allowance, grazing allowance) as .npy."""
    import os
    d = os.environ.get("TTS_PARITY_DUMP")
    if not d:
        return
    os.makedirs(d, exist_ok=True)
    g, o, oabs, kink = (np.asarray(x, np.float64).ravel() for x in (g, o, oabs, kink))
    cond = np.zeros_like(o) if cond is None else np.asarray(cond, np.float64).ravel()
    idx = np.nonzero(~_within(g, o, oabs, kink))[0]
    tag = "".join(ch if ch.isalnum() else "_" for ch in name)
    np.save(os.path.join(d, f"fail_{tag}_s{si}_{k}.npy"),
            np.stack([idx, g[idx], o[idx], oabs[idx], kink[idx], cond[idx]], 1))


def cat_upstream(ups, device="cuda"):
    """Per-view upstream tuples -> flat (dimage, dalpha, ddepth[, dnormal])."""
    n = len(ups[0])
    return tuple(torch.from_numpy(np.concatenate([u[k].reshape(-1) for u in ups])).to(device)
                 for k in range(n))


def check_gradients(scenes, views, params: Params, upstream, name="", min_pass=1.0,
                    max_undecided=None):
    """Forward + backward of the CUDA path through the C ABI against the
    oracle's gradient of the same loss, per element.

    scenes: list of synth.Scene or (V, T, f, rgb); views: (camera, scene index)
    pairs; upstream: per view (dimage, dalpha, ddepth[, dnormal]).  Returns a
    report: per scene and tensor the pass fraction, the worst error/bound and
    the max-normalised error, plus per view the band, alternative-branch and
    undecidable pixel counts.  Asserts the pass fraction >= min_pass and at
    most max_undecided (default max(2, 1e-4 of the pixels)) undecidable
    pixels per view."""
    r, ups, brs, orcs0, report = prepare_upstream(scenes, views, params, upstream, name,
                                                  max_undecided)
    u = cat_upstream(ups)
    grads = r.backward(u[0], u[1], u[2], dnormal=u[3] if len(u) > 3 else None)
    torch.cuda.synchronize()
    return compare_with_oracle(scenes, views, params, ups, brs, orcs0, grads, report, name,
                               min_pass)
