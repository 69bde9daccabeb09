"""Geometry terms over the C ABI: the unique edges of a tet grid, the
eikonal / normal-consistency regularizers of its SDF (Sec. 4.2) and Marching
Tetrahedra mesh extraction (Sec. 3.1).  Device memory comes from PyTorch; the
work runs in libtets' kernels."""

from __future__ import annotations

import ctypes

import torch

from . import _lib
from ._lib import TTS_FLAG_ACCUM_GRAD, TTS_STATUS_BAD_INDEX, TetsError, check


def _stream_ptr():
    return torch.cuda.current_stream().cuda_stream


def _ws(nbytes: int, device) -> torch.Tensor:
    # torch's caching allocator hands out 512-byte aligned blocks
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def tet_edges(T: torch.Tensor, N: int) -> torch.Tensor:
    """(E, 2) int32 tensor of the grid's unique edges (lo < hi), sorted."""
    L = _lib.load()
    if T.dtype != torch.int32 or not T.is_contiguous() or T.dim() != 2 or T.shape[1] != 4:
        raise TetsError("T must be a contiguous K x 4 int32 CUDA tensor")
    K = int(T.shape[0])
    nb = ctypes.c_size_t(0)
    check(L.tts_tet_edges_workspace_size(int(N), K, ctypes.byref(nb)), "tts_tet_edges_workspace_size")
    ws = _ws(nb.value, T.device)
    edges = torch.empty((6 * K, 2), dtype=torch.int32, device=T.device)
    n = torch.empty(1, dtype=torch.int64, device=T.device)
    check(L.tts_tet_edges(T.data_ptr(), K, int(N), edges.data_ptr(), 6 * K, n.data_ptr(),
                          ws.data_ptr(), ws.numel(), _stream_ptr()), "tts_tet_edges")
    count = int(n.item())
    if count < 0:
        raise TetsError("a tet index is outside [0, N)")
    return edges[:count].clone()


class Regularizers:
    """Workspace + call for the Sec. 4.2 regularizers of one grid size."""

    def __init__(self, N: int, device):
        self.lib = _lib.load()
        self.N = int(N)
        nb = ctypes.c_size_t(0)
        check(self.lib.tts_regularizers_workspace_size(self.N, ctypes.byref(nb)),
              "tts_regularizers_workspace_size")
        self.ws = _ws(nb.value, device)
        self.losses = torch.zeros(2, dtype=torch.float64, device=device)

    def __call__(self, V, T, f, edges, w_eik=1.0, w_nc=1.0, grads=None, accumulate=False):
        """Enqueues the call.  Returns the device (L_eik, L_nc) float64 tensor
        (a view of a buffer reused by the next call) and, when ``grads`` =
        (dV, df) is given, fills it with the gradients of w_eik L_eik +
        w_nc L_nc."""
        dV, df = grads if grads is not None else (None, None)
        E = int(edges.shape[0]) if edges is not None else 0
        check(self.lib.tts_regularizers(
            V.data_ptr(), T.data_ptr(), f.data_ptr(), self.N, int(T.shape[0]),
            edges.data_ptr() if E else None, E, float(w_eik), float(w_nc), self.losses.data_ptr(),
            dV.data_ptr() if dV is not None else None, df.data_ptr() if df is not None else None,
            TTS_FLAG_ACCUM_GRAD if accumulate else 0, self.ws.data_ptr(), self.ws.numel(),
            _stream_ptr()), "tts_regularizers")
        return self.losses

    def status(self) -> int:
        st = ctypes.c_uint32(0)
        check(self.lib.tts_geometry_status(self.ws.data_ptr(), ctypes.byref(st), _stream_ptr()),
              "tts_geometry_status")
        return int(st.value)


class RegularizerLoss(torch.autograd.Function):
    """(V, f) -> w_eik L_eik + w_nc L_nc (float64 scalar) with gradients."""

    @staticmethod
    def forward(ctx, V, f, T, edges, w_eik, w_nc, reg: Regularizers):
        dV = torch.empty_like(V)
        df = torch.empty_like(f)
        losses = reg(V.detach(), T, f.detach(), edges, w_eik, w_nc, grads=(dV, df))
        ctx.save_for_backward(dV, df)
        return w_eik * losses[0] + w_nc * losses[1]

    @staticmethod
    def backward(ctx, g):
        dV, df = ctx.saved_tensors
        gf = g.to(torch.float32)
        return dV * gf, df * gf, None, None, None, None, None


def regularizer_loss(V, f, T, edges, w_eik=1.0, w_nc=1.0, reg: Regularizers | None = None):
    reg = reg or Regularizers(V.shape[0], V.device)
    return RegularizerLoss.apply(V, f, T, edges, w_eik, w_nc, reg)


def marching_tets(V, T, f, edges):
    """Marching Tetrahedra: (verts (nv, 3) float32, tris (nt, 3) int32,
    vert_edge (nv,) int32) for the zero level set of f.  Two calls: the first
    sizes the outputs (one stream synchronisation), the second fills them."""
    L = _lib.load()
    N, K, E = int(V.shape[0]), int(T.shape[0]), int(edges.shape[0])
    nb = ctypes.c_size_t(0)
    check(L.tts_marching_tets_workspace_size(K, E, ctypes.byref(nb)),
          "tts_marching_tets_workspace_size")
    ws = _ws(nb.value, V.device)
    counts = torch.zeros(2, dtype=torch.int64, device=V.device)
    dummy_v = torch.empty(3, dtype=torch.float32, device=V.device)
    dummy_t = torch.empty(3, dtype=torch.int32, device=V.device)
    args = (V.data_ptr(), T.data_ptr(), f.data_ptr(), N, K, edges.data_ptr(), E)
    check(L.tts_marching_tets(*args, dummy_v.data_ptr(), None, 0, dummy_t.data_ptr(), 0,
                              counts.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr()),
          "tts_marching_tets")
    nv, nt = (int(x) for x in counts.cpu())
    verts = torch.empty((max(nv, 1), 3), dtype=torch.float32, device=V.device)
    vedge = torch.empty(max(nv, 1), dtype=torch.int32, device=V.device)
    tris = torch.empty((max(nt, 1), 3), dtype=torch.int32, device=V.device)
    check(L.tts_marching_tets(*args, verts.data_ptr(), vedge.data_ptr(), nv, tris.data_ptr(), nt,
                              counts.data_ptr(), ws.data_ptr(), ws.numel(), _stream_ptr()),
          "tts_marching_tets")
    st = ctypes.c_uint32(0)
    check(L.tts_geometry_status(ws.data_ptr(), ctypes.byref(st), _stream_ptr()),
          "tts_geometry_status")
    if st.value & TTS_STATUS_BAD_INDEX:
        raise TetsError("an index is out of range or a tet edge is missing from the edge list")
    return verts[:nv], tris[:nt], vedge[:nv]


__all__ = ["tet_edges", "Regularizers", "RegularizerLoss", "regularizer_loss", "marching_tets",
           "TTS_STATUS_BAD_INDEX"]
