"""Parity of the CUDA path (called through the C ABI) with the oracle.

Sizes: the 16^3 sphere at 128^2 (several tiles, ragged tail views), the 64^3
torus at 512^2 and the 128^3 three-sphere scene at 4 x 512^2 (the benchmark's
workload, in the launch configuration the benchmark times).
"""

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2406_01579_b300 import Params, Rasterizer, SceneTensors
from parity import (BAND_MAX, IMG_TOL, check_gradients, compare_images, compare_keys, gpu_run,
                    oracle_params, oracle_run, to_dev)

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sphere16():
    return synth.scene_sphere16()


def _check_view(gpu, orc, name=""):
    bad, namb, emax, multi = compare_images(gpu, orc)
    npx = orc["alpha"].size
    assert bad == 0, f"{name}: {bad} pixels off by > {IMG_TOL} (max unambiguous err {emax})"
    assert multi <= max(2, 1e-4 * npx), f"{name}: {multi} multi-band pixels unmatched"
    assert namb <= BAND_MAX * npx, f"{name}: {namb} band pixels"
    return emax


@pytest.mark.parametrize("hull", [True, False])
@pytest.mark.parametrize("tile", [8, 16, 32])
@pytest.mark.parametrize("s", [20.0, 175.0, 620.0])
def test_sphere16_keys_and_image(sphere16, tile, s, hull):
    """Keys bit for bit and images, with the tile test against the projected
    tet (hull) and with bbox rects only."""
    p = Params(s=s, tile=tile, hull=hull)
    cam = sphere16.cams[0]
    gpu = gpu_run([sphere16], [(cam, 0)], p, lists=True)
    orc = oracle_run(sphere16, cam, p)
    n = compare_keys(gpu, orc)
    assert n > 1000
    _check_view(gpu["views"][0], orc, f"tile{tile} s{s}")


def test_sphere16_pure_mode(sphere16):
    p = Params(s=20.0, tile=16, pure=True)
    cam = sphere16.cams[0]
    gpu = gpu_run([sphere16], [(cam, 0)], p, lists=True)
    orc = oracle_run(sphere16, cam, p)
    compare_keys(gpu, orc)
    assert orc["amb"].sum() == 0
    _check_view(gpu["views"][0], orc, "pure")


@pytest.mark.parametrize("s", [20.0, 175.0, 620.0])
def test_sphere16_gradients(sphere16, s):
    """Per-element gradient parity; band pixels are differentiated on the
    branch the GPU took (at s = 620 most covered pixels stop after two
    fragments at the cap, a decision both sides take exactly in FP32)."""
    p = Params(s=s, tile=16)
    cam = sphere16.cams[0]
    check_gradients([sphere16], [(cam, 0)], p, [synth.upstream_grads(0, [cam])[0]],
                    name=f"sphere16 s{s}")


@pytest.mark.parametrize("nw", [1, 5])
def test_resort_window_parity(sphere16, nw):
    """Sec. 3.3 resort window: images and gradients against the oracle's
    window of the same size."""
    p = Params(s=60.0, tile=16, resort_window=nw)
    cam = sphere16.cams[0]
    check_gradients([sphere16], [(cam, 0)], p, [synth.upstream_grads(6, [cam])[0]],
                    name=f"window{nw}")


def _with_normal_upstream(seed_up, seed_n, cam):
    up = tuple(synth.upstream_grads(seed_up, [cam])[0])
    return up + (np.random.default_rng(seed_n).normal(size=(3, cam.height, cam.width))
                 .astype(np.float32),)


@pytest.mark.parametrize("tile,nw,pure", [(8, 0, False), (16, 0, False), (16, 0, True),
                                          (32, 5, False)])
def test_normal_map_and_gradients(sphere16, tile, nw, pure):
    """Eq. 2 normal channel (per-tet normal of Sec. 3.2 / App. A.3): the
    normal map and the gradients of all four upstream channels."""
    p = Params(s=60.0, tile=tile, resort_window=nw, pure=pure, normals=True)
    cam = sphere16.cams[0]
    orc0 = oracle_run(sphere16, cam, p)
    assert np.abs(orc0["normal"]).max() > 0.5
    check_gradients([sphere16], [(cam, 0)], p, [_with_normal_upstream(11, 12, cam)],
                    name=f"normals tile{tile} nw{nw} pure{pure}")


def test_normal_gradient_alone(sphere16):
    """Only dL/dnormal nonzero: the gradient reaches V and f through the
    per-tet normals and through the opacities."""
    p = Params(s=60.0, tile=16, normals=True)
    cam = sphere16.cams[0]
    H, W = cam.height, cam.width
    rng = np.random.default_rng(13)
    up = (np.zeros((3, H, W), np.float32), np.zeros((H, W), np.float32),
          np.zeros((H, W), np.float32), rng.normal(size=(3, H, W)).astype(np.float32))
    rep = check_gradients([sphere16], [(cam, 0)], p, [up], name="normal-only")
    assert rep["tensors"]["s0.drgb"]["maxnorm"] == 0.0


@pytest.mark.parametrize("seg", [32, 96])
@pytest.mark.parametrize("s,pure", [(20.0, False), (175.0, False), (20.0, True)])
def test_split_tile_lists(sphere16, seg, s, pure):
    """Tile lists split into segments of `seg` entries (the forward records
    its state at every segment end, the backward walks the segments in
    parallel from those states): image, normal map and gradients against the
    oracle."""
    p = Params(s=s, tile=16, pure=pure, normals=True, blend_segment=seg)
    cam = sphere16.cams[0]
    gpu = gpu_run([sphere16], [(cam, 0)], p, lists=True)
    assert int(np.diff(gpu["lists"]["ranges"], axis=1).max()) > 4 * seg
    check_gradients([sphere16], [(cam, 0)], p, [_with_normal_upstream(21, 22, cam)],
                    name=f"split{seg} s{s} pure{pure}")


def test_resort_window_torus64(torus64):
    p = Params(s=175.0, tile=16, resort_window=5)
    cam = torus64.cams[0]
    gpu = gpu_run([torus64], [(cam, 0)], p)
    orc = oracle_run(torus64, cam, p)
    _check_view(gpu["views"][0], orc, "torus64 window5")


def test_gradients_pure_small_grids():
    for n, s in ((2, 3.0), (4, 6.0)):
        V = synth.grid_vertices(n)
        T = synth.grid_tets(n)
        f = (np.linalg.norm(V, axis=1) - 0.6 + 0.05 * V[:, 0]).astype(np.float32)
        rgb = np.random.default_rng(n).uniform(size=(len(V), 3)).astype(np.float32)
        cam = synth.orbit_camera(33.0, 21.0, 40, 40)
        p = Params(s=s, tile=8, pure=True)
        rep = check_gradients([(V, T, f, rgb)], [(cam, 0)], p,
                              [synth.upstream_grads(30 + n, [cam])[0]], name=f"pure{n}")
        assert rep["views"][0]["band"] == 0


def test_batch_of_views_and_scenes_matches_single_views(sphere16):
    """Several scenes and views of uneven sizes (ragged tiles) in one call;
    each scene's gradient sums over its views."""
    rng = np.random.default_rng(5)
    sc2 = synth.Scene(8, *synth.random_scene(rng, 8, "torus")[:4], [], "torus8")
    cams = [synth.orbit_camera(30.0, 20.0, 128, 128), synth.random_camera(rng, 77, 53),
            synth.random_camera(rng, 200, 96), synth.random_camera(rng, 33, 130)]
    views = [(cams[0], 0), (cams[1], 1), (cams[2], 0), (cams[3], 1)]
    check_gradients([sphere16, sc2], views, Params(s=60.0, tile=16),
                    synth.upstream_grads(9, cams), name="ragged batch")


@pytest.mark.parametrize("nv", [14, 18])
def test_many_views_of_one_scene(sphere16, nv):
    """Up to and more views of one scene than the preprocess stages in shared
    memory (16): past that it reads the view constants from the descriptor.
    Image sizes are even: with an odd width the look-at cameras put a column of
    pixel centres exactly on the image of the world z axis, where grid tets have
    edges, and a ray through an edge meets two faces at one point (a kink of the
    chord where adjoint, dual-number and finite-difference derivatives differ)."""
    rng = np.random.default_rng(11)
    cams = [synth.random_camera(rng, 40 + 4 * i, 36 + 2 * (i % 5)) for i in range(nv)]
    check_gradients([sphere16], [(c, 0) for c in cams], Params(s=60.0, tile=8),
                    synth.upstream_grads(13, cams), name=f"{nv} views")


def test_empty_and_degenerate_inputs(sphere16):
    p = Params(s=175.0, tile=16)
    # all tets pre-filtered away: transparent image
    f = np.full(sphere16.N, 2.0, np.float32)
    sc = (sphere16.V, sphere16.T, f, sphere16.rgb)
    gpu = gpu_run([sc], [(sphere16.cams[0], 0)], p, lists=True)
    assert gpu["info"].n_surv[0] == 0 and gpu["info"].n_keys == 0
    for x in gpu["views"][0]:
        assert np.all(x == 0.0)
    # camera looking away: everything culled
    cam = synth.look_at_camera((0.0, 0.0, 2.5), 64, 64, target=(0.0, 0.0, 5.0))
    gpu = gpu_run([sphere16], [(cam, 0)], p, lists=True)
    assert gpu["info"].n_keys == 0
    assert np.all(gpu["views"][0][1] == 0.0)
    # one-pixel image
    cam = synth.orbit_camera(30.0, 20.0, 1, 1)
    gpu = gpu_run([sphere16], [(cam, 0)], p)
    orc = oracle_run(sphere16, cam, p)
    _check_view(gpu["views"][0], orc, "1px")


def test_bad_index_sets_status(sphere16):
    T = sphere16.T.copy()
    T[5, 2] = sphere16.N + 7
    st = to_dev((sphere16.V, T, sphere16.f, sphere16.rgb))
    r = Rasterizer([st], [(sphere16.cams[0], 0)], Params())
    r.prepare()
    r.forward_raw()
    info = r.info()
    assert info.status & 1


def test_key_capacity_overflow_grows_and_matches(sphere16):
    st = to_dev(sphere16)
    p = Params(s=175.0, tile=8)
    r = Rasterizer([st], [(sphere16.cams[0], 0)], p, key_capacity=16)
    img, alpha, depth = r.forward()
    assert r.key_capacity > 16
    orc = oracle_run(sphere16, sphere16.cams[0], p)
    gv = [x.cpu().numpy() for x in r.view_outputs(img, alpha, depth)[0]]
    _check_view(gv, orc, "regrown")


def test_repeat_calls_are_deterministic(sphere16):
    st = to_dev(sphere16)
    r = Rasterizer([st], [(sphere16.cams[0], 0)], Params())
    a = [x.clone() for x in r.forward()]
    b = r.forward()
    for x, y in zip(a, b):
        assert torch.equal(x, y)


@pytest.fixture(scope="module")
def torus64():
    return synth.scene_torus64()


def test_torus64_full_size(torus64):
    p = Params(s=175.0, tile=16)
    cam = torus64.cams[0]
    gpu = gpu_run([torus64], [(cam, 0)], p, lists=True)
    orc = oracle_run(torus64, cam, p)
    n = compare_keys(gpu, orc)
    assert n > 100000
    _check_view(gpu["views"][0], orc, "torus64")


def test_torus64_gradients(torus64):
    p = Params(s=175.0, tile=16)
    cam = torus64.cams[0]
    check_gradients([torus64], [(cam, 0)], p, [synth.upstream_grads(1, [cam])[0]],
                    name="torus64")


@pytest.mark.parametrize("res,tile,lo,hi", [(64, 32, 16385, None), (256, 32, 2049, 16384),
                                            (96, 8, 1, 2048)])
def test_long_tile_lists(res, tile, lo, hi):
    """Tile lists of every length class of the per-tile depth sort: up to 256
    keys (a warp), 2,048 (half a block), 4,096 (a block) and longer (sorted
    runs of 4,096 merged in global memory).  The 64^3 torus seen at a low
    resolution piles many tets into each tile.  Keys, values and ranges bit
    for bit against the oracle's sort."""
    sc = synth.scene_torus64(res=res)
    p = Params(s=60.0, tile=tile)
    cam = sc.cams[0]
    gpu = gpu_run([sc], [(cam, 0)], p, lists=True)
    surv, amb_t, _ = oracle.prefilter(sc.T, sc.f, oracle_params(p))
    orc = {"surv": surv, "amb_tets": amb_t,
           "bins": oracle.bin_view(surv, sc.T, sc.V, cam, tile, hull=p.hull)}
    compare_keys(gpu, orc)
    r = gpu["lists"]["ranges"]
    lens = r[:, 1] - r[:, 0]
    assert ((lens >= lo) & (lens <= (hi or lens.max()))).sum() >= 1, lens.max()
    assert gpu["info"].long_lists == (lens > 4096).sum()


@pytest.fixture(scope="module")
def spheres128():
    return synth.scene_spheres128()


@pytest.mark.parametrize("tile,hull", [(8, True), (8, False), (16, True)])
def test_spheres128_bench_workload(spheres128, tile, hull):
    """The benchmark's configuration: 128^3 grid, 4 views at 512^2, s = 175,
    one batched call (tile 8 is the size the benchmark's autotuner picks).
    Keys are compared bit for bit per view; images pixel by pixel."""
    p = Params(s=175.0, tile=tile, hull=hull)
    sc = spheres128
    views = [(c, 0) for c in sc.cams]
    gpu = gpu_run([sc], views, p, lists=True)
    r = gpu["raster"]
    lists = gpu["lists"]
    keys = lists["keys"].view(np.uint64)
    db = lists["depth_bits"]
    gtile = (keys >> np.uint64(db)).astype(np.int64)
    tiles_per_view = (512 // tile) ** 2
    for vi, cam in enumerate(sc.cams):
        orc = oracle_run(sc, cam, p)
        sel = (gtile >= vi * tiles_per_view) & (gtile < (vi + 1) * tiles_per_view)
        sub = dict(lists)
        sub["keys"] = lists["keys"][sel]
        sub["vals"] = lists["vals"][sel]
        rec_base = vi * int(r.surv_capacity[0])
        t_g = gtile[sel] - vi * tiles_per_view
        z_g = ((keys[sel] & np.uint64((1 << db) - 1)).astype(np.int64) + lists["zmin_bits"]).astype(np.uint32)
        id_g = gpu["surv"][lists["vals"][sel].astype(np.int64) - rec_base]
        b = orc["bins"]
        band = np.nonzero(orc["amb_tets"])[0]
        kg = ~np.isin(id_g, band)
        ko = ~np.isin(orc["surv"][b["key_val"]], band)
        np.testing.assert_array_equal(t_g[kg], b["key_tile"][ko])
        np.testing.assert_array_equal(z_g[kg], b["key_z"][ko])
        np.testing.assert_array_equal(id_g[kg], orc["surv"][b["key_val"]][ko])
        _check_view(gpu["views"][vi], orc, f"spheres128 view{vi}")


def test_spheres128_subgrid_gradients(spheres128):
    """Gradients on the 4^3 sub-grid (cubes [62,66)^3) against the oracle."""
    sub = synth.subgrid(spheres128, 62, 66)
    p = Params(s=175.0, tile=16)
    for k, cam in enumerate(sub.cams):
        if oracle_run(sub, cam, p)["alpha"].max() == 0:
            continue
        check_gradients([sub], [(cam, 0)], p, [synth.upstream_grads(2, [cam])[0]],
                        name=f"sub view{k}")


def test_spheres128_full_gradients(spheres128):
    """The benchmark's own step at full size: 128^3 grid (12.6 M tets), 4
    views at 512^2, s = 175, tile 8, the default backward segment (split
    lists walked by four lanes per pixel in the forward and in parallel
    segments in the backward): every entry of dV, df and drgb against the
    oracle, per element."""
    sc = spheres128
    p = Params(s=175.0, tile=8)
    rep = check_gradients([sc], [(c, 0) for c in sc.cams], p, synth.upstream_grads(2, sc.cams),
                          name="spheres128 4x512 tile8")
    assert sum(v["band"] for v in rep["views"]) <= BAND_MAX * 4 * 512 * 512


@pytest.mark.parametrize("s,tile,cap", [(175.0, 8, 4), (620.0, 16, 16), (20.0, 8, 8)])
def test_fragment_lists_match_oracle(sphere16, s, tile, cap):
    """The forward's per-pixel fragment lists, bit for bit: off the decision
    band every pixel's blended count and the record slots of its first
    frag_cap blended fragments (in blend order) equal the oracle's, and the
    overflow flags mark exactly the tiles holding a pixel past the cap."""
    cam = sphere16.cams[0]
    p = Params(s=s, tile=tile, frag_cap=cap)
    r = gpu_run([sphere16], [(cam, 0)], p)["raster"]
    lists, nb, ov, c = r.debug_frag_lists()
    assert c == cap
    H, W = cam.height, cam.width
    lists = lists.cpu().numpy().reshape(H, W, cap)
    nb = nb.cpu().numpy().reshape(H, W)
    ov = ov.cpu().numpy()
    orc = oracle.render(sphere16.V, sphere16.T, sphere16.f, sphere16.rgb, cam, oracle_params(p),
                        blend_cap=cap)
    off = orc["amb"] == 0
    assert (~off).sum() <= BAND_MAX * H * W
    assert np.array_equal(nb[off], orc["nblend"][off])
    k = np.minimum(nb, cap)
    for q in range(cap):
        sel = off & (k > q)
        assert np.array_equal(lists[..., q][sel], orc["blend_slots"][..., q][sel]), q
    tx = (W + tile - 1) // tile
    over = np.zeros_like(ov)
    jj, ii = np.nonzero(nb > cap)
    np.maximum.at(over, (jj // tile) * tx + ii // tile, 1)
    assert np.array_equal(ov, over)
    if s < 600:
        assert over.any()   # some pixels past the cap: the list walk takes their tiles


@pytest.mark.parametrize("frag_cap,normals", [(1, False), (6, False), (-1, False), (3, True)])
def test_fragment_list_caps(sphere16, frag_cap, normals):
    """The backward from the forward's per-pixel fragment lists and its
    list-walk fallback: with a cap of 1 almost every covered pixel is past
    the cap and its tile is re-walked, with 3 or 6 the two paths share most
    tiles (each pixel taken by exactly one), with -1 no lists are kept.
    Per-element gradients against the oracle, split lists included
    (segments of 64 entries), with the normal channel in one case."""
    p = Params(s=60.0 if normals else 175.0, tile=8, frag_cap=frag_cap, blend_segment=64,
               normals=normals)
    cam = sphere16.cams[0]
    up = _with_normal_upstream(14, 15, cam) if normals else synth.upstream_grads(4, [cam])[0]
    check_gradients([sphere16], [(cam, 0)], p, [up], name=f"frag_cap {frag_cap} normals {normals}")


def test_fragment_lists_match_list_walk(sphere16):
    """Gradients from the per-pixel fragment lists equal those of the list
    walk alone (-1) up to the order of the float atomics, on the benchmark's
    tile size with split lists; images are identical."""
    cam = sphere16.cams[0]
    up = synth.upstream_grads(5, [cam])[0]
    out = {}
    for fc in (0, -1):
        p = Params(s=175.0, tile=8, frag_cap=fc, blend_segment=64)
        out[fc] = gpu_run([sphere16], [(cam, 0)], p, upstream=[up])
    for a, b in zip(out[0]["views"][0][:3], out[-1]["views"][0][:3]):
        assert np.array_equal(np.asarray(a), np.asarray(b))
    for a, b in zip(out[0]["grads"][0], out[-1]["grads"][0]):
        a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
        assert np.abs(a - b).max() <= 2e-4 * max(np.abs(b).max(), 1e-30)


@pytest.mark.parametrize("warps", [2, 8])
def test_blend_warps_per_block(sphere16, warps):
    """The blend kernels at 2 and 8 warps per block (the autotuner's other
    candidates): keys, images and per-element gradients against the oracle,
    split lists included (segments of 64 entries)."""
    p = Params(s=175.0, tile=8, blend_warps=warps, blend_segment=64)
    cam = sphere16.cams[0]
    gpu = gpu_run([sphere16], [(cam, 0)], p, lists=True)
    orc = oracle_run(sphere16, cam, p)
    compare_keys(gpu, orc)
    assert int(np.diff(gpu["lists"]["ranges"], axis=1).max()) > 64
    check_gradients([sphere16], [(cam, 0)], p, [synth.upstream_grads(3, [cam])[0]],
                    name=f"warps{warps}")
