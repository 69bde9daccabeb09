"""Continuous-batching render server over resident tetrahedral scenes.

Requests ask for one view of one resident scene, forward only or forward +
backward (with an upstream gradient).  The loop admits requests as they
arrive: whenever a stream slot is free and the HBM budget allows, the oldest
waiting requests of one kind are batched into a single library call (one
pre-filter per scene entry, one sort, one blend queue for all the views) and
launched asynchronously on that slot's stream, so batches overlap on the
device.  Gradient requests get their own scene entry, hence their own
gradient buffers; forward-only requests of the same scene share one entry.

Memory and host work per batch:
* each stream slot keeps its workspace and device buffers across batches
  (grown when a batch needs more), and a rasterizer per workspace layout:
  batches whose layout repeats (same scene sizes, view sizes, capacities,
  kind) reuse it, and skip even the workspace clearing when the slot's
  previous batch had that layout and finished clean;
* upstream gradients given as pinned host (or device) tensors are copied
  asynchronously on the slot's stream; numpy arrays are accepted too;
* each result's image, alpha and depth are copied from the device directly
  into pinned host tensors of its own (torch's caching host allocator), with
  no host-side copy; gradients stay on the device.

Failures: a batch that exceeds its key or survivor capacity is re-run with
larger estimates; one whose bounded device wait gave up is re-run (a request
that meets it twice fails); one with a tet index outside [0, N) is split into
one batch per scene, and a scene that fails alone is marked bad (its
requests fail without a launch).  A failed request gets a Result whose
``error`` says why and whose tensors are None.

Cancellation: ``cancel(rid)`` (from any thread) or a request's ``deadline``
(seconds from the start of the run): a request cancelled before its batch is
launched is never launched; one cancelled while its batch runs gets no
result.  Neither holds up other requests.
"""

from __future__ import annotations

import collections
import dataclasses
import gc
import math
import threading
import time
import weakref
from typing import Any, Callable, Sequence

import numpy as np
import torch

from . import camera as _camera
from ._lib import (TTS_STATUS_BAD_INDEX, TTS_STATUS_KEY_OVERFLOW, TTS_STATUS_SURV_OVERFLOW,
                   TTS_STATUS_TIMEOUT)
from .rasterizer import Params, Rasterizer, SceneTensors

SLOT_BYTES = 4 + 4 + 16 + 96      # per (view, survivor) workspace bytes, forward only
GRAD_SLOT_BYTES = 96               # extra per slot with a backward
KEY_BYTES = 24                     # keys and values, double buffered
PIXEL_BYTES = 12 + 20              # per-pixel state + outputs
LIST_PIXEL_BYTES = 4 + 8           # per pixel with a backward: blended count, task entry
DEFAULT_FRAG_CAP = 128             # tts_params.frag_cap 0
MAX_TIMEOUTS = 2                   # device-wait timeouts a request may meet before it fails


@dataclasses.dataclass
class Request:
    rid: int
    scene: int
    camera: Any
    want_grad: bool = False
    arrival: float = 0.0            # seconds since the start of the run
    upstream: tuple | None = None   # (dimage (3,H,W), dalpha (H,W), ddepth (H,W)) float32:
                                    # numpy, or torch tensors (pinned host or device)
    deadline: float | None = None   # cancelled once the run's clock passes it


@dataclasses.dataclass
class Result:
    rid: int
    image: torch.Tensor | None      # (3, H, W) pinned host
    alpha: torch.Tensor | None      # (H, W)
    depth: torch.Tensor | None      # (H, W)
    grads: tuple | None             # (dV, df, drgb) on the device
    done: float
    latency: float
    batch_views: int
    error: str | None = None


def _bucket(x: int, step: float = 1.25) -> int:
    """x rounded up to the next of 1024 * step^k (capacities that repeat)."""
    if x <= 1024:
        return 1024
    return int(math.ceil(1024 * step ** math.ceil(math.log(x / 1024.0, step))))


class _PinnedPool:
    """Pinned host buffers for results, by size class (a power of two of
    floats), reused once the tensors handed out on them are freed.  A fresh
    pinned allocation costs a few hundred microseconds, which bounded the
    loop at high request rates."""

    def __init__(self):
        self.free = collections.defaultdict(list)
        self.out = collections.Counter()    # buffers handed out and not yet back
        self.peak = collections.Counter()   # the most of them at once

    @staticmethod
    def _new(cls: int):
        return torch.empty(cls, dtype=torch.float32, pin_memory=True).untyped_storage()

    def _back(self, cls: int, store):
        self.out[cls] -= 1
        self.free[cls].append(store)

    def get(self, n: int) -> torch.Tensor:
        cls = 1 << max(16, (n - 1).bit_length())
        pool = self.free[cls]
        store = pool.pop() if pool else self._new(cls)
        t = torch.empty(0, dtype=torch.float32).set_(store, 0, (n,), (1,))
        self.out[cls] += 1
        self.peak[cls] = max(self.peak[cls], self.out[cls])
        # the storage goes back to the pool when the tensor (and every view of
        # it) is gone: a result is freed only after its copy has completed
        weakref.finalize(t, self._back, cls, store)
        return t

    def top_up(self, factor: float, cap: int):
        """Allocates ahead, per size class used so far, up to factor x the
        most buffers of it ever out at once (at most cap)."""
        for cls, pk in list(self.peak.items()):
            want = min(cap, int(math.ceil(factor * pk)))
            while len(self.free[cls]) + self.out[cls] < want:
                self.free[cls].append(self._new(cls))


class _Slot:
    """A stream with buffers that persist across the batches it runs."""

    def __init__(self, device):
        self.stream = torch.cuda.Stream(device=device)
        self.device = device
        self.ws = None          # uint8 device workspace
        self.dev = None         # float32 device outputs / upstream gradients
        self.rasters: collections.OrderedDict = collections.OrderedDict()   # layout -> Rasterizer
        self.last_layout = None  # layout of the last batch, while its workspace state is clean

    def workspace(self, ws_bytes: int):
        """The slot's workspace, grown (x1.5) when too small (the rasterizers
        built on the old one are dropped)."""
        if self.ws is None or self.ws.numel() < ws_bytes:
            self.ws = None
            self.rasters.clear()
            self.last_layout = None
            self.ws = torch.empty(int(ws_bytes * 1.5) + 4096, dtype=torch.uint8, device=self.device)
        return self.ws

    def buffer(self, n_float: int):
        """Device float buffer of at least n_float, grown (x1.5) when too small."""
        if self.dev is None or self.dev.numel() < n_float:
            self.dev = torch.empty(int(n_float * 1.5) + 4096, dtype=torch.float32,
                                   device=self.device)
        return self.dev


class _Inflight:
    def __init__(self, reqs, raster, slot, layout, outs, grads, event, nbytes):
        self.reqs = reqs
        self.raster = raster
        self.slot = slot
        self.layout = layout
        self.outs = outs        # per request (image, alpha, depth) pinned host tensors
        self.grads = grads
        self.event = event
        self.nbytes = nbytes


class Server:
    def __init__(self, scenes: Sequence[SceneTensors], params: Params | None = None,
                 hbm_budget: float = 120e9, max_views: int = 16, streams: int = 3,
                 device=None, ref_res: int = 512, max_layouts: int = 16):
        self.params = params or Params()
        self.scenes = list(scenes)
        self.device = torch.device(device) if device is not None else self.scenes[0].V.device
        self.budget = float(hbm_budget)
        self.max_views = int(max_views)
        self.max_layouts = int(max_layouts)
        self.slots = [_Slot(self.device) for _ in range(streams)]
        self._pinned = _PinnedPool()
        self.surv = []
        self.key_scale = []     # per scene: c in keys ~ surv (1 + c res / tile)^2
        self.key_margin = []    # per scene: safety factor, doubled after an overflow
        self.bad_scenes: set = set()
        self._cancel_lock = threading.Lock()
        self._cancelled: set = set()
        self._register(ref_res)

    def _register(self, res: int):
        """Survivors of each resident scene and its keys at a reference view
        (capacity estimates).  A tet whose bbox spans w pixels overlaps about
        (1 + w / tile)^2 tiles and w grows with the image size, so the keys of
        a view of size res are modelled as surv (1 + c res / tile)^2 with c
        fitted at the reference view."""
        cam = _camera.orbit(30.0, 20.0, res, res)
        T = float(self.params.tile)
        for i, sc in enumerate(self.scenes):
            r = Rasterizer([sc], [(cam, 0)], dataclasses.replace(self.params, forward_only=True))
            r.forward(check_status=False)
            info = r.info()
            if info.status & TTS_STATUS_BAD_INDEX:
                self.bad_scenes.add(i)
            surv = max(1, int(info.n_surv[0]))
            self.surv.append(surv)
            ratio = max(1.0, info.n_keys / float(surv))
            self.key_scale.append((ratio ** 0.5 - 1.0) * T / res)
            self.key_margin.append(1.5)
            del r

    # -- cancellation ----------------------------------------------------------
    def cancel(self, rid: int) -> None:
        """Cancels request ``rid`` (any thread, before or during ``run``; the
        cancellations are used up when ``run`` returns)."""
        with self._cancel_lock:
            self._cancelled.add(int(rid))

    def _is_cancelled(self, q: Request, now: float) -> bool:
        if q.deadline is not None and now >= q.deadline:
            return True
        with self._cancel_lock:
            return q.rid in self._cancelled

    # -- batching ------------------------------------------------------------
    def _estimate(self, reqs, want_grad: bool):
        scenes, views, ent = [], [], {}
        for q in reqs:
            if want_grad or q.scene not in ent:
                ent[q.scene] = len(scenes)
                scenes.append(q.scene)
            views.append((q.camera, ent[q.scene] if not want_grad else len(scenes) - 1))
        surv_cap = [min(int(self.scenes[s].T.shape[0]), _bucket(int(self.surv[s] * 1.02) + 1024))
                    for s in scenes]
        keys = 0.0
        slots = 0
        px = 0
        for (cam, e), q in zip(views, reqs):
            npx = int(cam.width) * int(cam.height)
            res = max(int(cam.width), int(cam.height))
            grow = (1.0 + self.key_scale[q.scene] * res / float(self.params.tile)) ** 2
            keys += self.key_margin[q.scene] * self.surv[q.scene] * grow
            slots += surv_cap[e]
            px += npx
        key_cap = _bucket(int(keys) + 65536)
        nbytes = slots * (SLOT_BYTES + (GRAD_SLOT_BYTES if want_grad else 0)) + \
            key_cap * KEY_BYTES + px * PIXEL_BYTES
        if want_grad and self.params.frag_cap >= 0 and self.params.resort_window == 0:
            # the backward's per-pixel fragment lists
            cap = self.params.frag_cap or DEFAULT_FRAG_CAP
            nbytes += px * (4 * cap + LIST_PIXEL_BYTES)
        return scenes, views, surv_cap, key_cap, nbytes

    def _rasterizer(self, slot: _Slot, scenes, views, p, surv_cap, key_cap):
        """(rasterizer, layout) for the batch: the slot's rasterizer of this
        workspace layout rebound to the batch's scenes and cameras, or a new
        one.  Its workspace is cleared unless the slot's last batch had the
        same layout and finished clean."""
        layout = (tuple((int(self.scenes[s].V.shape[0]), int(self.scenes[s].T.shape[0]), c)
                        for s, c in zip(scenes, surv_cap)),
                  tuple((int(c.width), int(c.height), e) for c, e in views),
                  key_cap, p.forward_only)
        sts = [self.scenes[s] for s in scenes]
        r = slot.rasters.get(layout)
        if (r is not None and slot.ws is not None and r.ws is not None
                and r.ws.data_ptr() == slot.ws.data_ptr()):
            slot.rasters.move_to_end(layout)
            r.rebind(sts, [c for c, _ in views])
            if slot.last_layout != layout:
                r.reinit()
            return r, layout
        r = Rasterizer(sts, views, p, key_capacity=key_cap, surv_capacity=surv_cap,
                       device=self.device, workspace=slot.workspace)
        slot.rasters[layout] = r
        while len(slot.rasters) > self.max_layouts:
            slot.rasters.popitem(last=False)
        return r, layout

    def _launch(self, reqs, want_grad, slot: _Slot) -> _Inflight:
        scenes, views, surv_cap, key_cap, nbytes = self._estimate(reqs, want_grad)
        p = dataclasses.replace(self.params, forward_only=not want_grad)
        stream = slot.stream
        with torch.cuda.stream(stream):
            r, layout = self._rasterizer(slot, scenes, views, p, surv_cap, key_cap)
            slot.last_layout = None          # clean again only once this batch checks out
            P = r.total_pixels
            n_out = 5 * P
            dev = slot.buffer(2 * n_out if want_grad else n_out)
            out = (dev[:3 * P], dev[3 * P:4 * P], dev[4 * P:5 * P])
            grads = None
            if want_grad:
                du = dev[n_out:2 * n_out]
                for q, off in zip(reqs, r.pix_off):
                    H, W = int(q.camera.height), int(q.camera.width)
                    for src, (a, n) in zip(q.upstream, ((3 * off, 3 * H * W),
                                                        (3 * P + off, H * W),
                                                        (4 * P + off, H * W))):
                        t = src if torch.is_tensor(src) else torch.from_numpy(
                            np.ascontiguousarray(src, np.float32))
                        du[a:a + n].copy_(t.reshape(-1), non_blocking=True)
                grads = [(torch.empty_like(self.scenes[s].V), torch.empty_like(self.scenes[s].f),
                          torch.empty_like(self.scenes[s].rgb)) for s in scenes]
                r.step(out, (du[:3 * P], du[3 * P:4 * P], du[4 * P:5 * P]), grads)
            else:
                r.prepare()
                r.forward_raw(out)
            outs = []
            for q, off in zip(reqs, r.pix_off):
                H, W = int(q.camera.height), int(q.camera.width)
                h = self._pinned.get(5 * H * W)
                h[:3 * H * W].copy_(dev[3 * off:3 * off + 3 * H * W], non_blocking=True)
                h[3 * H * W:4 * H * W].copy_(dev[3 * P + off:3 * P + off + H * W], non_blocking=True)
                h[4 * H * W:].copy_(dev[4 * P + off:4 * P + off + H * W], non_blocking=True)
                outs.append(h)
            ev = torch.cuda.Event()
            ev.record(stream)
        return _Inflight(reqs, r, slot, layout, outs, grads, ev, nbytes)

    def _finish(self, b: _Inflight, now: float, results: dict, deliver, stats) -> str:
        """Checks a completed batch: 'ok' (results delivered), 'capacity',
        'timeout' or 'bad_index' (the caller re-queues or splits it)."""
        with torch.cuda.stream(b.slot.stream):
            info = b.raster.info()   # the batch is complete: this does not wait
        st = int(info.status)
        if st & TTS_STATUS_BAD_INDEX:
            return "bad_index"
        if st & TTS_STATUS_TIMEOUT:
            return "timeout"
        if st & (TTS_STATUS_KEY_OVERFLOW | TTS_STATUS_SURV_OVERFLOW):
            return "capacity"
        b.slot.last_layout = b.layout
        for i, (q, h) in enumerate(zip(b.reqs, b.outs)):
            if self._is_cancelled(q, now):
                stats["cancelled"] += 1
                continue
            H, W = int(q.camera.height), int(q.camera.width)
            g = b.grads[i] if b.grads is not None else None
            deliver(results, Result(q.rid, h[:3 * H * W].view(3, H, W),
                                    h[3 * H * W:4 * H * W].view(H, W),
                                    h[4 * H * W:].view(H, W), g, now, now - q.arrival,
                                    len(b.reqs)))
        return "ok"

    def reserve(self):
        """Grows every slot's workspace and device buffer to the largest any
        slot holds (e.g. after a warm-up run), so that no batch of a later run
        allocates device memory: a large allocation in the middle of a run
        stalls every batch in flight.  The pinned result buffers are topped up
        to twice the most of each size that the runs so far held at once (at
        most one per view the slots can run together)."""
        self._pinned.top_up(2.0, len(self.slots) * self.max_views)
        torch.cuda.synchronize(self.device)
        ws = max((sl.ws.numel() for sl in self.slots if sl.ws is not None), default=0)
        nf = max((sl.dev.numel() for sl in self.slots if sl.dev is not None), default=0)
        for sl in self.slots:
            if ws and (sl.ws is None or sl.ws.numel() < ws):
                sl.ws = None
                sl.rasters.clear()
                sl.last_layout = None
                sl.ws = torch.empty(ws, dtype=torch.uint8, device=self.device)
            if nf and (sl.dev is None or sl.dev.numel() < nf):
                sl.dev = torch.empty(nf, dtype=torch.float32, device=self.device)

    # -- the loop --------------------------------------------------------------
    def run(self, requests: Sequence[Request], realtime: bool = True,
            on_result: Callable[[Result], None] | None = None):
        """Serves ``requests`` (arrival times in seconds from the start) and
        returns ({rid: Result}, stats).  With ``on_result``, each result is
        handed to it as it completes instead of being kept in the dict.
        Python's cyclic garbage collector is paused while the loop runs (its
        full collections over the run's request and result objects stall the
        loop for tens of milliseconds); it is restored afterwards."""
        paused = gc.isenabled()
        gc.disable()
        try:
            return self._run(requests, realtime, on_result)
        finally:
            if paused:
                gc.enable()

    def _run(self, requests, realtime, on_result):
        pending = collections.deque(sorted(requests, key=lambda q: q.arrival))
        ready = collections.deque()
        inflight: list[_Inflight] = []
        results: dict = {}
        lat: list = []
        done_px = [0]
        free = list(range(len(self.slots)))
        busy_bytes = 0.0
        stats = {"cancelled": 0, "failed": 0}
        timeouts = collections.Counter()
        isolate = set()          # rids to be batched per scene (after a bad index)
        n_batches = 0
        retries = 0
        max_inflight = 0
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if realtime else (lambda: float("inf"))

        def deliver(res, r: Result):
            lat.append(r.latency)
            if r.error is None and r.image is not None:
                done_px[0] += int(r.image.shape[1]) * int(r.image.shape[2])
            if on_result is not None:
                on_result(r)
            else:
                res[r.rid] = r

        def fail(q: Request, why: str, t: float):
            stats["failed"] += 1
            r = Result(q.rid, None, None, None, None, t, t - q.arrival, 0, error=why)
            if on_result is not None:
                on_result(r)
            else:
                results[q.rid] = r

        while pending or ready or inflight:
            now = clock()
            while pending and pending[0].arrival <= now:
                ready.append(pending.popleft())
            progressed = False
            for b in list(inflight):
                if b.event.query():
                    t = time.perf_counter() - t0
                    inflight.remove(b)
                    busy_bytes -= b.nbytes
                    free.append(self.slots.index(b.slot))
                    verdict = self._finish(b, t, results, deliver, stats)
                    if verdict == "capacity":
                        # an estimate was too small: grow this batch's scenes'
                        # estimates and run it again
                        for q in reversed(b.reqs):
                            ready.appendleft(q)
                        for sc in {q.scene for q in b.reqs}:
                            self.key_margin[sc] *= 2.0
                        retries += 1
                    elif verdict == "timeout":
                        for q in reversed(b.reqs):
                            timeouts[q.rid] += 1
                            if timeouts[q.rid] >= MAX_TIMEOUTS:
                                fail(q, "a bounded device wait gave up", t)
                            else:
                                ready.appendleft(q)
                        retries += 1
                    elif verdict == "bad_index":
                        if len({q.scene for q in b.reqs}) == 1 and b.reqs[0].rid in isolate:
                            self.bad_scenes.add(b.reqs[0].scene)
                            for q in b.reqs:
                                fail(q, "a tet index of the scene is outside [0, N)", t)
                        else:
                            for q in reversed(b.reqs):
                                isolate.add(q.rid)
                                ready.appendleft(q)
                            retries += 1
                    progressed = True
            # drop cancelled requests and requests of bad scenes before launch
            if ready:
                keep = collections.deque()
                for q in ready:
                    if self._is_cancelled(q, now):
                        stats["cancelled"] += 1
                    elif q.scene in self.bad_scenes:
                        fail(q, "a tet index of the scene is outside [0, N)", now)
                    else:
                        keep.append(q)
                ready = keep
            while ready and free:
                kind = ready[0].want_grad
                alone = ready[0].rid in isolate
                scene0 = ready[0].scene
                batch = []
                rest = collections.deque()
                while ready and len(batch) < self.max_views:
                    q = ready.popleft()
                    same = q.want_grad == kind and (not alone or q.scene == scene0)
                    (batch if same else rest).append(q)
                ready.extendleft(reversed(rest))
                nbytes = self._estimate(batch, kind)[4]
                while len(batch) > 1 and busy_bytes + nbytes > self.budget:
                    ready.appendleft(batch.pop())
                    nbytes = self._estimate(batch, kind)[4]
                if busy_bytes + nbytes > self.budget and inflight:
                    for q in reversed(batch):
                        ready.appendleft(q)
                    break
                si = free.pop(0)
                b = self._launch(batch, kind, self.slots[si])
                busy_bytes += b.nbytes
                inflight.append(b)
                n_batches += 1
                max_inflight = max(max_inflight, len(inflight))
                progressed = True
            if not progressed:
                if inflight:
                    time.sleep(0.0002)
                elif pending and realtime:
                    time.sleep(max(0.0, min(0.001, pending[0].arrival - clock())))
        t_end = time.perf_counter() - t0
        with self._cancel_lock:
            self._cancelled.clear()
        lat_ms = np.array(lat) * 1e3
        first = min(q.arrival for q in requests) if requests else 0.0
        stats.update({"requests": len(requests), "completed": len(lat),
                      "batches": n_batches, "retries": retries, "max_inflight": max_inflight,
                      "p50_ms": float(np.percentile(lat_ms, 50)) if len(lat_ms) else None,
                      "p99_ms": float(np.percentile(lat_ms, 99)) if len(lat_ms) else None,
                      "mpix_s": done_px[0] / max(t_end - first, 1e-9) / 1e6, "wall_s": t_end})
        return results, stats


def poisson_requests(rng: np.random.Generator, n: int, rate: float, n_scenes: int,
                     sizes=(256, 512, 768, 1024), grad_fraction: float = 0.3, start: float = 0.0,
                     pinned: bool = False):
    """Synthetic request stream: Poisson arrivals at ``rate`` per second,
    random scene, random view on the radius-2.5 sphere at a size from
    ``sizes``, ``grad_fraction`` of them forward + backward with N(0,1)
    upstream gradients: numpy arrays drawn per request, or with ``pinned``
    pinned host tensors drawn once per image size and shared by the requests
    of that size (a load generator that does not spend seconds drawing and
    pinning gigabytes)."""
    t = start
    out = []
    shared = {}
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        res = int(rng.choice(sizes))
        cam = _camera.on_sphere(rng, res, res)
        want = bool(rng.uniform() < grad_fraction)
        up = None
        if want:
            if pinned:
                if res not in shared:
                    g = np.random.default_rng(res)
                    shared[res] = tuple(torch.from_numpy(
                        g.normal(size=shp).astype(np.float32)).pin_memory()
                        for shp in ((3, res, res), (res, res), (res, res)))
                up = shared[res]
            else:
                up = (rng.normal(size=(3, res, res)).astype(np.float32),
                      rng.normal(size=(res, res)).astype(np.float32),
                      rng.normal(size=(res, res)).astype(np.float32))
        out.append(Request(i, int(rng.integers(n_scenes)), cam, want, t, up))
    return out


def latency_of(results: dict) -> tuple:
    lat = np.array([r.latency for r in results.values() if r.error is None]) * 1e3
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99))


__all__ = ["Server", "Request", "Result", "poisson_requests", "latency_of"]
