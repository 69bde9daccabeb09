"""The tile test against the projected tet (Sec. 3.3 culling, the HULL
reading): a tile of a tet's bbox rect loses its key only when no pixel centre
of (tile x bbox) can lie inside the tet's projection, the convex hull of its
four projected vertices.  Pinned by brute force over the pixel centres and by
rendering: the oracle's image from the culled lists equals the one from the
bbox lists (a pixel centre outside the projection meets no chord)."""

import numpy as np
import pytest

import oracle
import synth
from paper_2406_01579_b300 import Params
from parity import oracle_params


def _inside_hull(P, x, y, eps=1e-9):
    """Pixel centre (x, y) inside the convex hull of the 4 points P (FP64),
    by the triangles of the hull's fan over all point triples."""
    for a, b, c in ((0, 1, 2), (0, 1, 3), (0, 2, 3), (1, 2, 3)):
        A, B, C = P[a], P[b], P[c]
        d = (B[0] - A[0]) * (C[1] - A[1]) - (C[0] - A[0]) * (B[1] - A[1])
        if abs(d) < 1e-14:
            continue
        l1 = ((x - A[0]) * (C[1] - A[1]) - (C[0] - A[0]) * (y - A[1])) / d
        l2 = ((B[0] - A[0]) * (y - A[1]) - (x - A[0]) * (B[1] - A[1])) / d
        if l1 >= -eps and l2 >= -eps and l1 + l2 <= 1 + eps:
            return True
    return False


@pytest.mark.parametrize("tile", [8, 16])
def test_culled_tiles_hold_no_pixel_centre_of_the_hull(tile):
    sc = synth.scene_sphere16()
    cam = sc.cams[0]
    p = Params(s=60.0, tile=tile)
    surv, _, _ = oracle.prefilter(sc.T, sc.f, oracle_params(p))
    full = oracle.bin_view(surv, sc.T, sc.V, cam, tile)
    hull = oracle.bin_view(surv, sc.T, sc.V, cam, tile, hull=True)
    assert len(hull["key_val"]) < len(full["key_val"])
    kept = set(zip(hull["key_tile"].tolist(), hull["key_val"].tolist()))
    R, t = cam.R.astype(np.float64), cam.t.astype(np.float64)
    tx = (cam.width + tile - 1) // tile
    culled = 0
    for tl, s in zip(full["key_tile"].tolist(), full["key_val"].tolist()):
        if (tl, s) in kept:
            continue
        culled += 1
        X = (R @ sc.V[sc.T[surv[s]]].astype(np.float64).T).T + t
        P = np.stack([cam.fx * X[:, 0] / X[:, 2] + cam.cx, cam.fy * X[:, 1] / X[:, 2] + cam.cy], 1)
        i0, i1, j0, j1 = full["rect"][s]
        cx, cy = tl % tx, tl // tx
        for j in range(max(cy * tile, j0), min(cy * tile + tile - 1, j1) + 1):
            for i in range(max(cx * tile, i0), min(cx * tile + tile - 1, i1) + 1):
                assert not _inside_hull(P, i + 0.5, j + 0.5), (tl, s, i, j)
    assert culled > 0


@pytest.mark.parametrize("s,pure", [(60.0, False), (175.0, False), (20.0, True)])
def test_hull_lists_render_the_same_image(s, pure):
    sc = synth.scene_sphere16()
    cam = sc.cams[0]
    p = Params(s=s, tile=8, pure=pure)
    op = oracle_params(p)
    surv, _, _ = oracle.prefilter(sc.T, sc.f, op)
    a = oracle.render(sc.V, sc.T, sc.f, sc.rgb, cam, op, surv=surv,
                      bins=oracle.bin_view(surv, sc.T, sc.V, cam, 8))
    b = oracle.render(sc.V, sc.T, sc.f, sc.rgb, cam, op, surv=surv,
                      bins=oracle.bin_view(surv, sc.T, sc.V, cam, 8, hull=True))
    for k in ("image", "alpha", "depth"):
        assert np.abs(a[k] - b[k]).max() <= 1e-12, k
