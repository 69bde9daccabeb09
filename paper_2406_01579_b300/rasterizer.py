"""Python front end of libtets: device memory and streams come from PyTorch,
every step of the rasterizer runs in the CUDA kernels behind the C ABI.

``Rasterizer`` owns the workspace for one batch shape (scenes x views) and
exposes prepare / forward / backward.  ``TetRender`` is the autograd
Function over it, and ``render`` the one-call convenience for a single
scene.
"""

from __future__ import annotations

import ctypes
import dataclasses
import math
import weakref
from typing import Sequence

import torch

from . import _lib
from ._lib import (TTS_FLAG_ACCUM_GRAD, TTS_FLAG_FORWARD_ONLY, TTS_FLAG_NORMALS, TTS_FLAG_PURE,
                   TTS_STATUS_BAD_INDEX, TTS_STATUS_KEY_OVERFLOW, TTS_STATUS_SURV_OVERFLOW,
                   TetsError, check)


@dataclasses.dataclass
class Params:
    """Rasterizer parameters.  ``s`` is the Eq. 1 steepness; the thresholds
    are the 3DGS blending constants and the Sec. 3.2 pre-filter T_f."""
    s: float = 175.0
    tile: int = 16
    pure: bool = False
    prefilter_thresh: float = 1.0 / 255.0
    alpha_skip: float = 1.0 / 255.0
    alpha_cap: float = 0.99
    t_eps: float = 1e-4
    accum_grad: bool = False
    forward_only: bool = False
    resort_window: int = 0      # N_w of Sec. 3.3 (0..7)
    normals: bool = False       # also render the Eq. 2 normal map
    blend_segment: int = 0      # list entries per backward work unit (0: library default)
    hull: bool = False          # tile test against the projected tet (fewer keys, same image)
    blend_warps: int = 0        # warps per block of the blend kernels (0: library default, 4)
    frag_cap: int = 0           # per-pixel fragment lists for the backward (0: default 128, -1: none)
    count_walk: bool = False    # the blend kernels count their walk (debug_walk_counts)

    def to_c(self) -> _lib.tts_params:
        p = _lib.tts_params()
        p.s = self.s
        p.prefilter_thresh = self.prefilter_thresh
        p.alpha_skip = self.alpha_skip
        p.alpha_cap = self.alpha_cap
        p.t_eps = self.t_eps
        p.tile = self.tile
        p.flags = ((TTS_FLAG_PURE if self.pure else 0) | (TTS_FLAG_ACCUM_GRAD if self.accum_grad else 0)
                   | (TTS_FLAG_FORWARD_ONLY if self.forward_only else 0)
                   | (TTS_FLAG_NORMALS if self.normals else 0)
                   | (_lib.TTS_FLAG_HULL if self.hull else 0)
                   | (_lib.TTS_FLAG_COUNT if self.count_walk else 0))
        p.resort_window = int(self.resort_window)
        p.blend_segment = int(self.blend_segment)
        p.blend_warps = int(self.blend_warps)
        p.frag_cap = int(self.frag_cap)
        return p


def make_camera(cam) -> _lib.tts_camera:
    """From any object with R (3x3), t (3), fx, fy, cx, cy, znear, width, height."""
    c = _lib.tts_camera()
    R = [float(x) for x in _flat(cam.R)]
    t = [float(x) for x in _flat(cam.t)]
    for i in range(9):
        c.R[i] = R[i]
    for i in range(3):
        c.t[i] = t[i]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.znear = float(cam.znear)
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def _flat(a):
    if hasattr(a, "reshape"):
        return a.reshape(-1).tolist()
    out = []
    for x in a:
        out.extend(_flat(x) if hasattr(x, "__len__") else [x])
    return out


def _stream_ptr(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return s.cuda_stream


@dataclasses.dataclass
class SceneTensors:
    V: torch.Tensor      # N x 3 float32
    T: torch.Tensor      # K x 4 int32
    f: torch.Tensor      # N float32
    rgb: torch.Tensor    # N x 3 float32

    def check(self):
        for name, x, dt in (("V", self.V, torch.float32), ("T", self.T, torch.int32),
                            ("f", self.f, torch.float32), ("rgb", self.rgb, torch.float32)):
            if not x.is_cuda:
                raise TetsError(f"{name} must be a CUDA tensor")
            if x.dtype != dt or not x.is_contiguous():
                raise TetsError(f"{name} must be contiguous {dt}")
        N = self.V.shape[0]
        if self.V.shape != (N, 3) or self.f.shape != (N,) or self.rgb.shape != (N, 3):
            raise TetsError("V, f, rgb must be N x 3, N, N x 3")
        if self.T.dim() != 2 or self.T.shape[1] != 4:
            raise TetsError("T must be K x 4")


class Rasterizer:
    """Workspace + calls for one batch: ``scenes`` (SceneTensors) and
    ``views`` as (camera, scene index) pairs."""

    def __init__(self, scenes: Sequence[SceneTensors], views: Sequence, params: Params,
                 key_capacity: int | None = None, surv_capacity: Sequence[int] | None = None,
                 device=None, workspace: torch.Tensor | None = None):
        """``workspace``: an optional uint8 device buffer to use (its leading
        bytes) when it is large enough, or a callable that returns one for a
        byte count, instead of allocating one."""
        self.lib = _lib.load()
        self._ext_ws = workspace
        # forwards enqueued on this workspace so far: a backward uses the
        # state of the latest one (TetRender checks it has not moved on)
        self.generation = 0
        # a TetRender output of this rasterizer still awaits its backward
        self.awaiting_backward = False
        self.params = params
        self.device = torch.device(device) if device is not None else scenes[0].V.device
        self.views = [(c, int(s)) for c, s in views]
        self.set_scenes(scenes)
        K = [int(s.T.shape[0]) for s in self.scenes]
        self.surv_capacity = list(surv_capacity) if surv_capacity is not None else K
        if key_capacity is None:
            key_capacity = sum(max(65536, K[s] // 3) for _, s in self.views)
        self.key_capacity = int(key_capacity)
        self.ws = None
        self.ws_bytes = 0
        self._c_views = (_lib.tts_view * len(self.views))()
        for i, (cam, s) in enumerate(self.views):
            self._c_views[i].cam = make_camera(cam)
            self._c_views[i].scene = s
            self._c_views[i].reserved = 0
        self.pix_off = []
        off = 0
        for cam, _ in self.views:
            self.pix_off.append(off)
            off += int(cam.width) * int(cam.height)
        self.total_pixels = off
        self._alloc()

    # -- batch / workspace -------------------------------------------------
    def set_scenes(self, scenes: Sequence[SceneTensors]):
        for s in scenes:
            s.check()
        self.scenes = list(scenes)
        self._c_scenes = (_lib.tts_scene * len(self.scenes))()
        caps = getattr(self, "surv_capacity", None)
        for i, s in enumerate(self.scenes):
            c = self._c_scenes[i]
            c.V, c.T, c.f, c.rgb = (s.V.data_ptr(), s.T.data_ptr(), s.f.data_ptr(),
                                    s.rgb.data_ptr())
            c.N, c.K = s.V.shape[0], s.T.shape[0]
            c.surv_capacity = caps[i] if caps is not None else 0

    def batch(self) -> _lib.tts_batch:
        b = _lib.tts_batch()
        for i, cap in enumerate(self.surv_capacity):
            self._c_scenes[i].surv_capacity = int(cap)
        b.scenes = ctypes.cast(self._c_scenes, ctypes.POINTER(_lib.tts_scene))
        b.n_scenes = len(self.scenes)
        b.views = ctypes.cast(self._c_views, ctypes.POINTER(_lib.tts_view))
        b.n_views = len(self.views)
        b.params = self.params.to_c()
        b.key_capacity = self.key_capacity
        b.workspace = self.ws.data_ptr() if self.ws is not None else None
        b.workspace_bytes = self.ws_bytes
        return b

    def workspace_bytes(self) -> int:
        n = ctypes.c_size_t(0)
        b = self.batch()
        check(self.lib.tts_workspace_size(ctypes.byref(b), ctypes.byref(n)), "tts_workspace_size")
        return int(n.value)

    def _alloc(self):
        self.ws = None
        nbytes = self.workspace_bytes()
        ext = self._ext_ws(nbytes) if callable(self._ext_ws) else self._ext_ws
        if ext is not None and ext.numel() >= nbytes and ext.data_ptr() % 256 == 0:
            self.ws = ext[:nbytes]
        else:
            self.ws = torch.empty(nbytes, dtype=torch.uint8, device=self.device)
        self.ws_bytes = nbytes
        b = self.batch()
        check(self.lib.tts_workspace_init(ctypes.byref(b), _stream_ptr()), "tts_workspace_init")

    def rebind(self, scenes: Sequence[SceneTensors] | None = None, cams: Sequence | None = None):
        """Points the batch at other scenes (each with the N and K of the one
        it replaces) and other cameras (the same image sizes): the workspace
        layout is unchanged, so nothing is reallocated."""
        if scenes is not None:
            old = [(int(s.V.shape[0]), int(s.T.shape[0])) for s in self.scenes]
            new = [(int(s.V.shape[0]), int(s.T.shape[0])) for s in scenes]
            if old != new:
                raise TetsError("rebind: the scenes must keep their vertex and tet counts")
            self.set_scenes(scenes)
        if cams is not None:
            if len(cams) != len(self.views):
                raise TetsError("rebind: one camera per view")
            for i, c in enumerate(cams):
                w, h = int(c.width), int(c.height)
                if (w, h) != (int(self.views[i][0].width), int(self.views[i][0].height)):
                    raise TetsError("rebind: the views must keep their image sizes")
                self._c_views[i].cam = make_camera(c)
            self.views = [(c, s) for c, (_, s) in zip(cams, self.views)]

    def reinit(self):
        """Clears the workspace's persistent state (status word, gradient
        accumulators), as after allocation."""
        b = self.batch()
        check(self.lib.tts_workspace_init(ctypes.byref(b), _stream_ptr()), "tts_workspace_init")

    # -- calls ------------------------------------------------------------
    def prepare(self):
        b = self.batch()
        check(self.lib.tts_prepare_scene(ctypes.byref(b), _stream_ptr()), "tts_prepare_scene")

    def survivor_bounds(self, out=None) -> torch.Tensor:
        """(n_scenes, 6) device tensor of the survivors' axis-aligned bounds
        after the last ``prepare`` (App. B.1 coarse-to-fine pre-filter)."""
        out = out if out is not None else torch.empty((len(self.scenes), 6), dtype=torch.float32,
                                                      device=self.device)
        b = self.batch()
        check(self.lib.tts_survivor_bounds(ctypes.byref(b), out.data_ptr(), _stream_ptr()),
              "tts_survivor_bounds")
        return out

    def _outputs(self):
        """Flat output tensors: (image, alpha, depth) and, with
        ``params.normals``, the normal map (3 planes per view, like image)."""
        dev = self.device
        img = torch.empty(3 * self.total_pixels, dtype=torch.float32, device=dev)
        alpha = torch.empty(self.total_pixels, dtype=torch.float32, device=dev)
        depth = torch.empty(self.total_pixels, dtype=torch.float32, device=dev)
        if self.params.normals:
            return img, alpha, depth, torch.empty(3 * self.total_pixels, dtype=torch.float32,
                                                  device=dev)
        return img, alpha, depth

    @staticmethod
    def _c_outputs(out) -> _lib.tts_outputs:
        o = _lib.tts_outputs()
        o.image, o.alpha, o.depth = out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr()
        o.normal = out[3].data_ptr() if len(out) > 3 else None
        return o

    @staticmethod
    def _c_upstream(upstream) -> _lib.tts_upstream:
        ptr = [(x.data_ptr() if x is not None else None) for x in upstream]
        ptr += [None] * (4 - len(ptr))
        u = _lib.tts_upstream()
        u.dimage, u.dalpha, u.ddepth, u.dnormal = ptr
        return u

    def forward_raw(self, out=None):
        """Enqueue the forward (no synchronisation, no capacity check)."""
        out = tuple(out) if out is not None else self._outputs()
        b = self.batch()
        o = self._c_outputs(out)
        self.generation += 1
        check(self.lib.tts_render_fwd_ex(ctypes.byref(b), ctypes.byref(o), _stream_ptr()),
              "tts_render_fwd_ex")
        return out

    def forward(self, prepare: bool = True, check_status: bool = True, out=None):
        """prepare (optional) + forward; with ``check_status`` the status word
        is read (one stream sync) and capacities grow and the call is re-run
        when a capacity was exceeded."""
        for _ in range(4):
            if prepare:
                self.prepare()
            res = self.forward_raw(out)
            if not check_status:
                return res
            info = self.info()
            if info.status & TTS_STATUS_BAD_INDEX:
                raise TetsError("a tet index is outside [0, N)")
            if info.status & _lib.TTS_STATUS_TIMEOUT:
                raise TetsError("a bounded device wait gave up (the outputs are undefined)")
            grow = False
            if info.status & TTS_STATUS_SURV_OVERFLOW:
                self.surv_capacity = [int(s.T.shape[0]) for s in self.scenes]
                grow = True
            if info.status & TTS_STATUS_KEY_OVERFLOW:
                self.key_capacity = int(math.ceil(info.n_keys * 1.25)) + 1024
                grow = True
            if not grow:
                return res
            self._alloc()
            prepare = True
        raise TetsError("capacity growth did not converge")

    def shrink_to_fit(self, slack: float = 1.25):
        """Resize survivor and key capacities to the last forward's counts
        (times ``slack``).  Re-run prepare + forward afterwards."""
        info = self.info()
        self.surv_capacity = [min(int(s.T.shape[0]), int(math.ceil(info.n_surv[i] * slack)) + 1024)
                              for i, s in enumerate(self.scenes)]
        self.key_capacity = int(math.ceil(max(info.n_keys, 1) * slack)) + 4096
        self._alloc()

    def backward(self, dimage, dalpha=None, ddepth=None, grads=None, dnormal=None):
        """Gradients of the last forward; returns [(dV, df, drgb)] per scene."""
        if grads is None:
            grads = [(torch.empty_like(s.V), torch.empty_like(s.f), torch.empty_like(s.rgb))
                     for s in self.scenes]
        n = len(self.scenes)
        dV = (ctypes.c_void_p * n)(*[g[0].data_ptr() for g in grads])
        df = (ctypes.c_void_p * n)(*[g[1].data_ptr() for g in grads])
        dc = (ctypes.c_void_p * n)(*[g[2].data_ptr() for g in grads])
        up = tuple(x.contiguous() if x is not None else None
                   for x in (dimage, dalpha, ddepth, dnormal))
        b = self.batch()
        u = self._c_upstream(up)
        check(self.lib.tts_render_bwd_ex(ctypes.byref(b), ctypes.byref(u), dV, df, dc,
                                         _stream_ptr()), "tts_render_bwd_ex")
        return grads

    # -- whole training step (pre-filter + forward + backward) -----------------
    def step(self, out, upstream, grads):
        """Enqueue one step: pre-filter, forward of every view, backward into
        ``grads`` with the upstream gradients ``upstream`` = (dimage, dalpha,
        ddepth[, dnormal]) for the outputs ``out`` (as from ``_outputs``).  No
        synchronisation, no capacity check (size the workspace
        first, e.g. with ``forward()`` + ``shrink_to_fit``)."""
        L = self.lib
        b = self.batch()
        sp = _stream_ptr()
        n = len(self.scenes)
        dV = (ctypes.c_void_p * n)(*[g[0].data_ptr() for g in grads])
        df = (ctypes.c_void_p * n)(*[g[1].data_ptr() for g in grads])
        dc = (ctypes.c_void_p * n)(*[g[2].data_ptr() for g in grads])
        o = self._c_outputs(out)
        u = self._c_upstream(upstream)
        check(L.tts_prepare_scene(ctypes.byref(b), sp), "tts_prepare_scene")
        self.generation += 1
        check(L.tts_render_fwd_ex(ctypes.byref(b), ctypes.byref(o), sp), "tts_render_fwd_ex")
        check(L.tts_render_bwd_ex(ctypes.byref(b), ctypes.byref(u), dV, df, dc, sp),
              "tts_render_bwd_ex")

    def capture_step(self, out, upstream, grads, warmup: int = 2):
        """A CUDA graph of ``step`` on these exact buffers.  Replays read the
        current contents of the scene tensors, the upstream gradients and the
        workspace; the scene tensors must be updated in place."""
        side = torch.cuda.Stream(device=self.device)
        side.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(side):
            for _ in range(warmup):
                self.step(out, upstream, grads)
        torch.cuda.current_stream(self.device).wait_stream(side)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.step(out, upstream, grads)
        return g

    def info(self) -> _lib.tts_info:
        info = _lib.tts_info()
        b = self.batch()
        check(self.lib.tts_get_info(ctypes.byref(b), ctypes.byref(info), _stream_ptr()),
              "tts_get_info")
        return info

    # -- inspection -------------------------------------------------------
    def _ws_slice(self, ptr: int, nbytes: int, dtype) -> torch.Tensor:
        off = ptr - self.ws.data_ptr()
        assert 0 <= off and off + nbytes <= self.ws_bytes
        return self.ws[off:off + nbytes].view(dtype)

    def debug_lists(self):
        """Sorted keys (int64 view of the uint64 keys), values (int32 slot),
        ranges (total_tiles x 2), survivors (scene 0), zmin_bits, depth_bits."""
        P = ctypes.c_void_p
        k, v, r, s = P(), P(), P(), P()
        zmin = ctypes.c_uint32()
        db = ctypes.c_int32()
        b = self.batch()
        check(self.lib.tts_debug_lists(ctypes.byref(b), ctypes.byref(k), ctypes.byref(v),
                                       ctypes.byref(r), ctypes.byref(s), ctypes.byref(zmin),
                                       ctypes.byref(db), _stream_ptr()), "tts_debug_lists")
        info = self.info()
        n = int(info.n_keys)
        tiles = sum(((int(c.width) + self.params.tile - 1) // self.params.tile) *
                    ((int(c.height) + self.params.tile - 1) // self.params.tile)
                    for c, _ in self.views)
        keys = self._ws_slice(k.value, 8 * n, torch.int64) if n else torch.zeros(0, dtype=torch.int64)
        vals = self._ws_slice(v.value, 4 * n, torch.int32) if n else torch.zeros(0, dtype=torch.int32)
        ranges = self._ws_slice(r.value, 8 * tiles, torch.int32).view(tiles, 2)
        surv = [self._ws_slice(s.value, 4 * int(self.surv_capacity[0]), torch.int32)[:int(info.n_surv[0])]]
        return dict(keys=keys, vals=vals, ranges=ranges, surv=surv, zmin_bits=int(zmin.value),
                    depth_bits=int(db.value), n_keys=n, info=info)

    def debug_pixels(self):
        """Per-pixel state of the last forward (flat, view-major like alpha):
        final transmittance (float32), list entries walked up to the last
        blended one and fragments met (int32)."""
        P = ctypes.c_void_p
        t, last, nf = P(), P(), P()
        b = self.batch()
        check(self.lib.tts_debug_pixels(ctypes.byref(b), ctypes.byref(t), ctypes.byref(last),
                                        ctypes.byref(nf), _stream_ptr()), "tts_debug_pixels")
        n = 4 * self.total_pixels
        return (self._ws_slice(t.value, n, torch.float32), self._ws_slice(last.value, n, torch.int32),
                self._ws_slice(nf.value, n, torch.int32))

    def debug_walk_counts(self, reset: bool = True) -> dict:
        """Walk statistics of the blend kernels accumulated by the calls made
        with ``params.count_walk`` (see tts_debug_walk_counts)."""
        c = (ctypes.c_uint64 * 5)()
        b = self.batch()
        check(self.lib.tts_debug_walk_counts(ctypes.byref(b), c, 1 if reset else 0, _stream_ptr()),
              "tts_debug_walk_counts")
        return dict(zip(("fwd_groups", "fwd_candidates", "fwd_blocks", "bwd_groups",
                         "bwd_candidates"), (int(x) for x in c)))

    def debug_frag_lists(self):
        """Per-pixel fragment lists of the last forward: (lists (pixels, cap)
        int32 record slots in blend order, blended count per pixel (int32),
        per-tile overflow flags (int32), cap); None when the batch keeps no
        lists."""
        P = ctypes.c_void_p
        fr, nb, ov = P(), P(), P()
        cap = ctypes.c_int32(0)
        b = self.batch()
        check(self.lib.tts_debug_frag_lists(ctypes.byref(b), ctypes.byref(fr), ctypes.byref(nb),
                                            ctypes.byref(ov), ctypes.byref(cap), _stream_ptr()),
              "tts_debug_frag_lists")
        if cap.value == 0:
            return None
        n, c = self.total_pixels, cap.value
        tiles = sum(((int(cam.width) + self.params.tile - 1) // self.params.tile) *
                    ((int(cam.height) + self.params.tile - 1) // self.params.tile)
                    for cam, _ in self.views)
        lists = self._ws_slice(fr.value, 4 * n * c, torch.int32).view(n, c)
        return (lists, self._ws_slice(nb.value, 4 * n, torch.int32),
                self._ws_slice(ov.value, 4 * tiles, torch.int32), c)

    def view_outputs(self, img, alpha, depth, normal=None):
        """Split flat outputs into per-view (3,H,W), (H,W), (H,W) tensors
        (and a (3,H,W) normal map when given)."""
        out = []
        for (cam, _), off in zip(self.views, self.pix_off):
            H, W = int(cam.height), int(cam.width)
            v = (img[3 * off:3 * off + 3 * H * W].view(3, H, W),
                 alpha[off:off + H * W].view(H, W), depth[off:off + H * W].view(H, W))
            if normal is not None:
                v = v + (normal[3 * off:3 * off + 3 * H * W].view(3, H, W),)
            out.append(v)
        return out


def fit_grid(V: torch.Tensor, grid_lo, grid_hi, aabb: torch.Tensor, pad: float = 0.05,
             out: torch.Tensor | None = None) -> torch.Tensor:
    """Second round of the coarse-to-fine pre-filter (App. B.1): the grid's
    vertices V (inside the box [grid_lo, grid_hi]) mapped per axis onto the
    survivor bounds ``aabb`` (6 floats, device) widened by ``pad`` times
    their extent on each side.  Runs on the device without synchronising."""
    lib = _lib.load()
    out = out if out is not None else torch.empty_like(V)
    lo = (ctypes.c_float * 3)(*[float(x) for x in grid_lo])
    hi = (ctypes.c_float * 3)(*[float(x) for x in grid_hi])
    check(lib.tts_fit_grid(V.data_ptr(), int(V.shape[0]), lo, hi, aabb.data_ptr(), float(pad),
                           out.data_ptr(), _stream_ptr()), "tts_fit_grid")
    return out


def _check_autograd_params(raster: Rasterizer):
    if raster.params.accum_grad or raster.params.forward_only:
        raise TetsError("TetRender needs a rasterizer without accum_grad and forward_only")


def _mark_pending(raster: Rasterizer, outputs, ctx) -> None:
    """Records that a backward through these outputs may follow; the mark is
    dropped by that backward or once the outputs are freed."""
    if not any(ctx.needs_input_grad):
        return
    raster.awaiting_backward = True
    gen = raster.generation

    def release(r=raster, g=gen):
        if r.generation == g:
            r.awaiting_backward = False
    weakref.finalize(outputs[0], release)


def _stale(raster: Rasterizer, gen: int):
    if raster.generation != gen:
        raise TetsError(
            "backward of a TetRender output after another forward ran on the same rasterizer: "
            "the workspace holds the later forward's lists and per-pixel state.  Call backward "
            "before the next forward on that rasterizer, or render with separate rasterizers "
            "(render() keeps one per output that awaits its backward).")


class TetRender(torch.autograd.Function):
    """(V, f, rgb) -> (image, alpha, depth[, normal]) for the views of a
    single-scene ``Rasterizer``; outputs are flat view-major planar tensors
    (the normal map when the rasterizer's params ask for it).

    The backward re-walks the tile lists of the forward, which live in the
    rasterizer's workspace: it raises if another forward ran on that
    rasterizer in between (per-pixel transmittance is recomputed in the
    backward, never stored per fragment)."""

    @staticmethod
    def forward(ctx, V, f, rgb, raster: Rasterizer, check_status: bool = True):
        _check_autograd_params(raster)
        sc = raster.scenes[0]
        if V.data_ptr() != sc.V.data_ptr() or f.data_ptr() != sc.f.data_ptr() or \
                rgb.data_ptr() != sc.rgb.data_ptr():
            raster.set_scenes([SceneTensors(V.detach(), sc.T, f.detach(), rgb.detach())])
        out = raster.forward(prepare=True, check_status=check_status)
        ctx.raster = raster
        ctx.gen = raster.generation
        _mark_pending(raster, out, ctx)
        return tuple(out)

    @staticmethod
    def backward(ctx, gimg, galpha, gdepth, gnormal=None):
        raster = ctx.raster
        _stale(raster, ctx.gen)
        gimg = gimg if gimg is not None else torch.zeros(3 * raster.total_pixels, device=raster.device)
        (dV, df, drgb), = raster.backward(gimg, galpha, gdepth, dnormal=gnormal)
        raster.awaiting_backward = False
        return dV, df, drgb, None, None


class TetRenderBatch(torch.autograd.Function):
    """The batched form: ``raster`` over any number of scenes (and views of
    them), inputs ``V_0, f_0, rgb_0, V_1, f_1, rgb_1, ...`` in scene order;
    outputs as ``TetRender`` (flat over all views of the batch)."""

    @staticmethod
    def forward(ctx, raster: Rasterizer, check_status: bool, *vfr):
        _check_autograd_params(raster)
        n = len(raster.scenes)
        if len(vfr) != 3 * n:
            raise TetsError(f"expected 3 tensors per scene ({3 * n}), got {len(vfr)}")
        scenes = []
        for i, sc in enumerate(raster.scenes):
            V, f, rgb = vfr[3 * i:3 * i + 3]
            scenes.append(SceneTensors(V.detach(), sc.T, f.detach(), rgb.detach()))
        raster.set_scenes(scenes)
        out = raster.forward(prepare=True, check_status=check_status)
        ctx.raster = raster
        ctx.gen = raster.generation
        _mark_pending(raster, out, ctx)
        return tuple(out)

    @staticmethod
    def backward(ctx, gimg, galpha, gdepth, gnormal=None):
        raster = ctx.raster
        _stale(raster, ctx.gen)
        gimg = gimg if gimg is not None else torch.zeros(3 * raster.total_pixels, device=raster.device)
        grads = raster.backward(gimg, galpha, gdepth, dnormal=gnormal)
        raster.awaiting_backward = False
        flat = [g for trio in grads for g in trio]
        return (None, None, *flat)


# render(): rasterizers per batch shape, at most _POOL_MAX per shape; one
# whose output still awaits its backward is not handed out again while
# another can be (a reused one makes that pending backward raise).
_POOL_MAX = 4
_pools: dict = {}


def _pooled(key, make):
    pool = _pools.setdefault(key, [])
    for r in pool:
        if not r.awaiting_backward:
            pool.remove(r)
            pool.append(r)      # most recently used last
            return r
    if len(pool) < _POOL_MAX:
        r = make()
        pool.append(r)
        return r
    r = pool.pop(0)             # all busy: the least recently used
    pool.append(r)
    return r


def render(V, T, f, rgb, cams, params: Params | None = None, check_status: bool = True):
    """Renders the views ``cams`` of one scene and returns a list of
    (image (3,H,W), alpha (H,W), depth (H,W)[, normal (3,H,W)]) per view;
    differentiable with respect to V, f and rgb.  Each call's backward gets
    its own forward's gradient: outputs that still await their backward keep
    their rasterizer (up to four per batch shape; past that the oldest one is
    reused and its backward raises)."""
    params = params or Params()
    key = (tuple(V.shape), tuple(T.shape), T.data_ptr(), V.device.index, len(cams),
           tuple((int(c.width), int(c.height)) for c in cams), dataclasses.astuple(params))
    raster = _pooled(key, lambda: Rasterizer([SceneTensors(V.detach(), T, f.detach(),
                                                           rgb.detach())],
                                             [(c, 0) for c in cams], params))
    for i, c in enumerate(cams):
        raster._c_views[i].cam = make_camera(c)
    raster.views = [(c, 0) for c in cams]
    out = TetRender.apply(V, f, rgb, raster, check_status)
    return raster.view_outputs(*out)
