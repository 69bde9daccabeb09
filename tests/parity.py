"""Helpers shared by the GPU parity tests: run the CUDA path through the C ABI
and the oracle on the same seeded inputs, and compare them.

Comparison rules
* keys, ranges, survivors: bit for bit, after removing tets whose alpha_max
  lies in the oracle's decision band around T_f (FP32 vs FP64 may legitimately
  disagree on those; they never contribute since alpha <= alpha_max).
* image/alpha/depth: max abs error <= 1e-4 per pixel against the oracle's
  primary branch, or against its alternative branch when the pixel met a
  decision (cap, skip, stop) within the band of its threshold.
* gradients: max |gpu - oracle| / max |oracle| <= 1e-3 per tensor, with the
  upstream gradient set to zero at band pixels on both sides.
"""

from __future__ import annotations

import numpy as np
import torch

import oracle
import synth
from paper_2406_01579_b300 import Params, Rasterizer, SceneTensors

IMG_TOL = 1e-4
GRAD_TOL = 1e-3


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


def oracle_run(scene, cam, params: Params, upstream=None):
    if isinstance(scene, synth.Scene):
        V, T, f, rgb = scene.V, scene.T, scene.f, scene.rgb
    else:
        V, T, f, rgb = scene
    op = oracle_params(params)
    surv, amb_t, amax = oracle.prefilter(T, f, op)
    bins = oracle.bin_view(surv, T, V, cam, params.tile)
    r = oracle.render(V, T, f, rgb, cam, op, surv=surv, bins=bins, upstream=upstream,
                      normals=params.normals)
    r["amb_tets"] = amb_t
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
