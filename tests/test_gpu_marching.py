"""Parity of the GPU Marching Tetrahedra (Sec. 3.1) with the oracle, through
the C ABI: vertex indices, triangle indices and windings bit for bit,
positions within FP32 rounding; at the benchmark's 128^3 grid the mesh is
checked for being a closed, consistently oriented surface."""

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2406_01579_b300.geometry import marching_tets, tet_edges
from paper_2406_01579_b300._lib import TetsError

pytestmark = pytest.mark.gpu

POS_TOL = 2e-6


def _dev(*xs):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in xs]


def _run(V, T, f):
    Vd, Td, fd = _dev(V.astype(np.float32), T, f.astype(np.float32))
    E = tet_edges(Td, len(V))
    verts, tris, vedge = marching_tets(Vd, Td, fd, E)
    return verts.cpu().numpy(), tris.cpu().numpy(), vedge.cpu().numpy(), E.cpu().numpy()


def _compare(V, T, f):
    verts, tris, vedge, E = _run(V, T, f)
    ref = oracle.marching_tets(V.astype(np.float32), T, f.astype(np.float32))
    np.testing.assert_array_equal(E, ref["edges"])
    np.testing.assert_array_equal(vedge, ref["vert_edge"])
    np.testing.assert_array_equal(tris, ref["tris"])
    assert np.abs(verts - ref["verts"]).max() < POS_TOL
    return len(tris)


def test_sphere16_jittered():
    V = synth.grid_vertices(16).astype(np.float64)
    T = synth.grid_tets(16)
    rng = np.random.default_rng(1)
    V = V + rng.uniform(-0.1, 0.1, size=V.shape) / 16
    f = np.linalg.norm(V, axis=1) - 0.5 + 0.01 * rng.normal(size=len(V))
    assert _compare(V, T, f) > 1000


def test_torus64_scene():
    sc = synth.scene_torus64()
    assert _compare(sc.V, sc.T, sc.f) > 10000


def test_affine_and_empty_cases():
    V = synth.grid_vertices(5).astype(np.float64)
    T = synth.grid_tets(5)
    _compare(V, T, V @ np.array([0.3, -1.1, 0.7]) + 0.05)
    verts, tris, _, _ = _run(V, T, np.ones(len(V)))          # no crossing at all
    assert len(verts) == 0 and len(tris) == 0


def test_missing_edge_is_reported():
    V = synth.grid_vertices(3).astype(np.float32)
    T = synth.grid_tets(3)
    f = (np.linalg.norm(V, axis=1) - 0.7).astype(np.float32)   # the 8 inner vertices inside
    assert (f < 0).sum() == 8
    Vd, Td, fd = _dev(V, T, f)
    E = tet_edges(Td, len(V))
    with pytest.raises(TetsError):
        marching_tets(Vd, Td, fd, E[::2].contiguous())


def test_spheres128_mesh_is_closed_and_oriented():
    sc = synth.scene_spheres128(n_views=1)
    verts, tris, _, _ = _run(sc.V, sc.T, sc.f)
    assert len(tris) > 100000
    # every directed edge once, and its reverse once
    d = np.concatenate([tris[:, [0, 1]], tris[:, [1, 2]], tris[:, [2, 0]]])
    key = d[:, 0].astype(np.int64) * (1 << 32) + d[:, 1]
    rev = d[:, 1].astype(np.int64) * (1 << 32) + d[:, 0]
    assert len(np.unique(key)) == len(key)
    np.testing.assert_array_equal(np.sort(key), np.sort(rev))
    # outward normals enclose a positive volume; vertices stay in the grid
    p0, p1, p2 = (verts[tris[:, i]].astype(np.float64) for i in range(3))
    vol = np.einsum("ij,ij->i", p0, np.cross(p1, p2)).sum() / 6.0
    assert vol > 0
    assert np.abs(verts).max() <= 1.0
