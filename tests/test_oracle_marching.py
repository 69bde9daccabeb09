"""Pins of the oracle's Marching Tetrahedra (Sec. 3.1): a hand-cut tet,
affine fields (vertices exactly on the plane, normals along the gradient),
and for closed surfaces watertightness, orientation, Euler characteristic
and enclosed volume."""

import numpy as np
import pytest

import oracle
import synth


def _edge_use(tris):
    """Directed edge -> count; an oriented closed 2-manifold uses every
    undirected edge once in each direction."""
    d = {}
    for t in tris:
        for a, b in ((t[0], t[1]), (t[1], t[2]), (t[2], t[0])):
            d[(int(a), int(b))] = d.get((int(a), int(b)), 0) + 1
    return d


def _signed_volume(verts, tris):
    p0, p1, p2 = verts[tris[:, 0]], verts[tris[:, 1]], verts[tris[:, 2]]
    return float(np.einsum("ij,ij->i", p0, np.cross(p1, p2)).sum() / 6.0)


def test_single_tet_by_hand():
    V = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    T = np.array([[0, 1, 2, 3]], np.int32)
    # 1-3 split: the cut is at the edge midpoints around vertex 0
    r = oracle.marching_tets(V, T, np.array([-1.0, 1.0, 1.0, 1.0]))
    np.testing.assert_allclose(np.sort(r["verts"], axis=0),
                               np.sort(0.5 * np.eye(3), axis=0), atol=1e-15)
    (t,) = r["tris"]
    p = r["verts"][t]
    n = np.cross(p[1] - p[0], p[2] - p[0])
    assert n @ np.array([1.0, 1.0, 1.0]) > 0           # towards increasing f
    # 2-2 split (positive 0, 1): a quad through the four cut edges
    f = np.array([1.0, 3.0, -1.0, -3.0])
    r = oracle.marching_tets(V, T, f)
    assert len(r["verts"]) == 4 and len(r["tris"]) == 2
    A = np.c_[V, np.ones(4)]
    g = np.linalg.solve(A, f)[:3]
    for t in r["tris"]:
        p = r["verts"][t]
        assert np.cross(p[1] - p[0], p[2] - p[0]) @ g > 0
    # a non-degenerate quad whose corners lie on the zero plane of the field
    area = sum(0.5 * np.linalg.norm(np.cross(*(r["verts"][t[1:]] - r["verts"][t[0]])))
               for t in r["tris"])
    pts = r["verts"]
    assert np.abs(pts @ g + np.linalg.solve(A, f)[3]).max() < 1e-14
    assert area > 0.1


@pytest.mark.parametrize("seed", [0, 1])
def test_affine_field_vertices_on_the_plane(seed):
    rng = np.random.default_rng(seed)
    V = synth.grid_vertices(6).astype(np.float64)
    T = synth.grid_tets(6)
    a = rng.normal(size=3)
    b = 0.1 * rng.normal()
    f = V @ a + b
    r = oracle.marching_tets(V, T, f)
    assert len(r["tris"]) > 20
    assert np.abs(r["verts"] @ a + b).max() < 1e-12
    p = r["verts"][r["tris"]]
    n = np.cross(p[:, 1] - p[:, 0], p[:, 2] - p[:, 0])
    assert (n @ a > 0).all()
    # every vertex lies on its source edge, between the end points
    e = r["edges"][r["vert_edge"]]
    t = np.einsum("ij,ij->i", r["verts"] - V[e[:, 0]], V[e[:, 1]] - V[e[:, 0]]) / \
        np.einsum("ij,ij->i", V[e[:, 1]] - V[e[:, 0]], V[e[:, 1]] - V[e[:, 0]])
    assert (t >= -1e-12).all() and (t <= 1 + 1e-12).all()


@pytest.mark.parametrize("kind,n,euler", [("sphere", 12, 2), ("torus", 24, 0)])
def test_closed_surface_is_watertight_and_outward(kind, n, euler):
    V = synth.grid_vertices(n).astype(np.float64)
    T = synth.grid_tets(n)
    if kind == "sphere":
        f = np.linalg.norm(V, axis=1) - 0.61
    else:
        f = np.sqrt((np.sqrt(V[:, 0] ** 2 + V[:, 1] ** 2) - 0.5) ** 2 + V[:, 2] ** 2) - 0.23
    r = oracle.marching_tets(V, T, f)
    tris = r["tris"]
    use = _edge_use(tris)
    assert all(c == 1 for c in use.values())                  # no repeated directed edge
    assert all(use.get((b, a), 0) == 1 for (a, b) in use)     # each edge used both ways
    nV, nE, nF = len(r["verts"]), len(use) // 2, len(tris)
    assert nV - nE + nF == euler
    vol = _signed_volume(r["verts"], tris)
    exact = 4.0 / 3.0 * np.pi * 0.61 ** 3 if kind == "sphere" else 2 * np.pi ** 2 * 0.5 * 0.23 ** 2
    assert vol > 0                                            # outward normals
    assert vol == pytest.approx(exact, rel=0.05)


def test_enclosed_volume_converges_quadratically():
    """The piecewise-linear level set approaches the sphere at O(h^2)."""
    errs = []
    for n in (12, 24, 48):
        V = synth.grid_vertices(n).astype(np.float64)
        T = synth.grid_tets(n)
        r = oracle.marching_tets(V, T, np.linalg.norm(V, axis=1) - 0.61)
        errs.append(abs(_signed_volume(r["verts"], r["tris"]) / (4.0 / 3.0 * np.pi * 0.61 ** 3) - 1))
    assert errs[1] < 0.35 * errs[0] and errs[2] < 0.35 * errs[1]


def test_zero_values_count_as_inside():
    """f = 0 is on the non-positive side: a vertex exactly on the level set
    gives a cut vertex at its own position."""
    V = np.array([[0.0, 0, 0], [1, 0, 0], [0, 1, 0], [0, 0, 1]])
    T = np.array([[0, 1, 2, 3]], np.int32)
    r = oracle.marching_tets(V, T, np.array([0.0, 1.0, 1.0, 1.0]))
    np.testing.assert_allclose(r["verts"], np.zeros((3, 3)), atol=0)
    r = oracle.marching_tets(V, T, np.array([0.0, -1.0, -1.0, -1.0]))
    assert len(r["tris"]) == 0
