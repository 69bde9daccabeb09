"""Parity of the GPU geometry-stage terms (Sec. 4.2 eikonal and normal
consistency, unique grid edges) with the oracle, through the C ABI."""

import numpy as np
import pytest
import torch

import oracle
import synth
from paper_2406_01579_b300.geometry import Regularizers, regularizer_loss, tet_edges
from paper_2406_01579_b300._lib import TTS_STATUS_BAD_INDEX, TetsError

pytestmark = pytest.mark.gpu


def _grid(n, seed, jitter=0.2):
    V = synth.grid_vertices(n).astype(np.float64)
    T = synth.grid_tets(n)
    rng = np.random.default_rng(seed)
    V = V + rng.uniform(-jitter, jitter, size=V.shape) / n
    f = np.linalg.norm(V, axis=1) - 0.55 + 0.05 * rng.normal(size=len(V))
    return V.astype(np.float32), T, f.astype(np.float32)


def _dev(*xs):
    return [torch.from_numpy(np.ascontiguousarray(x)).cuda() for x in xs]


@pytest.mark.parametrize("n", [1, 4, 16, 33])
def test_edges_match_oracle(n):
    T = synth.grid_tets(n)
    N = (n + 1) ** 3
    (Td,) = _dev(T)
    got = tet_edges(Td, N).cpu().numpy()
    np.testing.assert_array_equal(got, oracle.tet_edges(T, N))


def test_edges_unstructured_with_repeats():
    rng = np.random.default_rng(4)
    N = 500
    T = rng.integers(0, N, size=(3000, 4)).astype(np.int32)
    T[::7, 1] = T[::7, 0]          # degenerate tets with a repeated vertex
    (Td,) = _dev(T)
    np.testing.assert_array_equal(tet_edges(Td, N).cpu().numpy(), oracle.tet_edges(T, N))


def test_edges_bad_index_is_reported():
    T = synth.grid_tets(2).copy()
    T[5, 2] = 10_000
    (Td,) = _dev(T)
    with pytest.raises(TetsError):
        tet_edges(Td, 27)


@pytest.mark.parametrize("n,seed", [(3, 1), (16, 2), (32, 3)])
def test_regularizers_match_oracle(n, seed):
    V, T, f = _grid(n, seed)
    E = oracle.tet_edges(T)
    w_eik, w_nc = 0.3, 1.7
    ref = oracle.regularizers(V, T, f, E, w_eik, w_nc)
    Vd, Td, fd, Ed = _dev(V, T, f, E)
    reg = Regularizers(len(V), "cuda")
    dV, df = torch.empty_like(Vd), torch.empty_like(fd)
    losses = reg(Vd, Td, fd, Ed, w_eik, w_nc, grads=(dV, df)).cpu().numpy()
    assert reg.status() == 0
    assert losses[0] == pytest.approx(ref["L_eik"], rel=1e-5)
    assert losses[1] == pytest.approx(ref["L_nc"], rel=1e-4)
    for name, g, o in (("dV", dV, ref["dV"]), ("df", df, ref["df"])):
        g = g.cpu().numpy().astype(np.float64)
        err = np.abs(g - o).max() / np.abs(o).max()
        assert err < 1e-3, f"{name}: {err:.2e}"


def test_regularizers_accumulate_losses_only_and_no_edges():
    V, T, f = _grid(4, 5)
    E = oracle.tet_edges(T)
    Vd, Td, fd, Ed = _dev(V, T, f, E)
    reg = Regularizers(len(V), "cuda")
    dV, df = torch.empty_like(Vd), torch.empty_like(fd)
    reg(Vd, Td, fd, Ed, 1.0, 1.0, grads=(dV, df))
    once = (dV.clone(), df.clone())
    reg(Vd, Td, fd, Ed, 1.0, 1.0, grads=(dV, df), accumulate=True)
    torch.testing.assert_close(dV, 2 * once[0], rtol=1e-5, atol=1e-6)
    torch.testing.assert_close(df, 2 * once[1], rtol=1e-5, atol=1e-6)
    lo = reg(Vd, Td, fd, Ed, 1.0, 1.0).cpu().numpy()
    ref = oracle.regularizers(V, T, f, E, grad=False)
    assert lo[0] == pytest.approx(ref["L_eik"], rel=1e-5)
    none = reg(Vd, Td, fd, Ed[:0], 1.0, 1.0).cpu().numpy()
    assert none[1] == 0.0 and none[0] == pytest.approx(ref["L_eik"], rel=1e-5)


def test_regularizers_bad_index_sets_status():
    V, T, f = _grid(2, 6)
    T = T.copy()
    T[3, 0] = -1
    E = oracle.tet_edges(synth.grid_tets(2))
    Vd, Td, fd, Ed = _dev(V, T, f, E)
    reg = Regularizers(len(V), "cuda")
    reg(Vd, Td, fd, Ed, 1.0, 1.0)
    assert reg.status() & TTS_STATUS_BAD_INDEX


def test_regularizer_autograd_function():
    V, T, f = _grid(4, 7)
    E = oracle.tet_edges(T)
    Vd, Td, fd, Ed = _dev(V, T, f, E)
    Vd.requires_grad_(True)
    fd.requires_grad_(True)
    loss = regularizer_loss(Vd, fd, Td, Ed, 0.5, 2.0)
    (3.0 * loss).backward()
    ref = oracle.regularizers(V, T, f, E, 0.5, 2.0)
    assert float(loss.detach()) == pytest.approx(0.5 * ref["L_eik"] + 2.0 * ref["L_nc"], rel=1e-5)
    g = fd.grad.cpu().numpy()
    assert np.abs(g - 3.0 * ref["df"]).max() / np.abs(3.0 * ref["df"]).max() < 1e-3
