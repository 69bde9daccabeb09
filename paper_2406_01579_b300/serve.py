"""Continuous-batching render server over resident tetrahedral scenes.

Requests ask for one view of one resident scene, forward only or forward +
backward (with an upstream gradient).  The loop admits requests as they
arrive: whenever a stream slot is free and the HBM budget allows, the oldest
waiting requests of one kind are batched into a single library call (one
pre-filter per scene entry, one sort, one blend queue for all the views) and
launched asynchronously on that slot's stream, so batches overlap on the
device.  Gradient requests get their own scene entry, hence their own
gradient buffers; forward-only requests of the same scene share one entry.
Each stream slot keeps its workspace, output and pinned host staging buffers
across batches (grown when a batch needs more), so the steady state
allocates no device or pinned memory per batch.  Images come back through
the slot's pinned buffer into host tensors of their own; gradients stay on
the device.
"""

from __future__ import annotations

import collections
import dataclasses
import time
from typing import Any, Sequence

import numpy as np
import torch

from . import camera as _camera
from ._lib import TTS_STATUS_KEY_OVERFLOW, TTS_STATUS_SURV_OVERFLOW
from .rasterizer import Params, Rasterizer, SceneTensors

SLOT_BYTES = 4 + 4 + 16 + 96      # per (view, survivor) workspace bytes, forward only
GRAD_SLOT_BYTES = 96               # extra per slot with a backward
KEY_BYTES = 24                     # keys and values, double buffered
PIXEL_BYTES = 12 + 20              # per-pixel state + outputs


@dataclasses.dataclass
class Request:
    rid: int
    scene: int
    camera: Any
    want_grad: bool = False
    arrival: float = 0.0            # seconds since the start of the run
    upstream: tuple | None = None   # (dimage (3,H,W), dalpha (H,W), ddepth (H,W)) float32


@dataclasses.dataclass
class Result:
    rid: int
    image: torch.Tensor      # (3, H, W) host
    alpha: torch.Tensor      # (H, W)
    depth: torch.Tensor      # (H, W)
    grads: tuple | None
    done: float
    latency: float
    batch_views: int


class _Slot:
    """A stream with buffers that persist across the batches it runs."""

    def __init__(self, device):
        self.stream = torch.cuda.Stream(device=device)
        self.device = device
        self.ws = None          # uint8 device workspace
        self.dev = None         # float32 device outputs / upstream gradients
        self.host = None        # float32 pinned host staging

    def workspace(self, ws_bytes: int):
        """The slot's workspace, grown (x1.5) when too small."""
        if self.ws is None or self.ws.numel() < ws_bytes:
            self.ws = None
            self.ws = torch.empty(int(ws_bytes * 1.5) + 4096, dtype=torch.uint8, device=self.device)
        return self.ws

    def buffers(self, n_float: int):
        """Device and pinned host float buffers of at least n_float, grown
        (x1.5) when too small."""
        if self.dev is None or self.dev.numel() < n_float:
            self.dev = torch.empty(int(n_float * 1.5) + 4096, dtype=torch.float32,
                                   device=self.device)
            self.host = torch.empty(self.dev.numel(), dtype=torch.float32, pin_memory=True)
        return self.dev, self.host


class _Inflight:
    def __init__(self, reqs, raster, slot, n_out, grads, event, nbytes):
        self.reqs = reqs
        self.raster = raster
        self.slot = slot
        self.n_out = n_out      # floats of image + alpha + depth at the slot's buffers' start
        self.grads = grads
        self.event = event
        self.nbytes = nbytes


class Server:
    def __init__(self, scenes: Sequence[SceneTensors], params: Params | None = None,
                 hbm_budget: float = 120e9, max_views: int = 16, streams: int = 3,
                 device=None, ref_res: int = 512):
        self.params = params or Params()
        self.scenes = list(scenes)
        self.device = torch.device(device) if device is not None else self.scenes[0].V.device
        self.budget = float(hbm_budget)
        self.max_views = int(max_views)
        self.slots = [_Slot(self.device) for _ in range(streams)]
        self.surv = []
        self.key_scale = []     # per scene: c in keys ~ surv (1 + c res / tile)^2
        self.key_margin = []    # per scene: safety factor, doubled after an overflow
        self._register(ref_res)

    def _register(self, res: int):
        """Survivors of each resident scene and its keys at a reference view
        (capacity estimates).  A tet whose bbox spans w pixels overlaps about
        (1 + w / tile)^2 tiles and w grows with the image size, so the keys of
        a view of size res are modelled as surv (1 + c res / tile)^2 with c
        fitted at the reference view."""
        cam = _camera.orbit(30.0, 20.0, res, res)
        T = float(self.params.tile)
        for sc in self.scenes:
            r = Rasterizer([sc], [(cam, 0)], dataclasses.replace(self.params, forward_only=True))
            r.forward()
            info = r.info()
            surv = max(1, int(info.n_surv[0]))
            self.surv.append(surv)
            ratio = max(1.0, info.n_keys / float(surv))
            self.key_scale.append((ratio ** 0.5 - 1.0) * T / res)
            self.key_margin.append(1.5)
            del r

    # -- batching ------------------------------------------------------------
    def _estimate(self, reqs, want_grad: bool):
        scenes, views, ent = [], [], {}
        for q in reqs:
            if want_grad or q.scene not in ent:
                ent[q.scene] = len(scenes)
                scenes.append(q.scene)
            views.append((q.camera, ent[q.scene] if not want_grad else len(scenes) - 1))
        surv_cap = [int(self.surv[s] * 1.02) + 1024 for s in scenes]
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
        key_cap = int(keys) + 65536
        nbytes = slots * (SLOT_BYTES + (GRAD_SLOT_BYTES if want_grad else 0)) + \
            key_cap * KEY_BYTES + px * PIXEL_BYTES
        return scenes, views, surv_cap, key_cap, nbytes

    def _launch(self, reqs, want_grad, slot: _Slot) -> _Inflight:
        scenes, views, surv_cap, key_cap, nbytes = self._estimate(reqs, want_grad)
        p = dataclasses.replace(self.params, forward_only=not want_grad)
        stream = slot.stream
        with torch.cuda.stream(stream):
            r = Rasterizer([self.scenes[s] for s in scenes], views, p, key_capacity=key_cap,
                           surv_capacity=surv_cap, device=self.device, workspace=slot.workspace)
            P = r.total_pixels
            n_out = 5 * P
            dev, host = slot.buffers(2 * n_out if want_grad else n_out)
            out = (dev[:3 * P], dev[3 * P:4 * P], dev[4 * P:5 * P])
            grads = None
            if want_grad:
                # upstream gradients staged through the slot's pinned buffer
                hu = host[n_out:2 * n_out]
                for q, off in zip(reqs, r.pix_off):
                    H, W = int(q.camera.height), int(q.camera.width)
                    ui, ua, ud = (torch.from_numpy(np.ascontiguousarray(x, np.float32)).view(-1)
                                  for x in q.upstream)
                    hu[3 * off:3 * off + 3 * H * W].copy_(ui)
                    hu[3 * P + off:3 * P + off + H * W].copy_(ua)
                    hu[4 * P + off:4 * P + off + H * W].copy_(ud)
                du = dev[n_out:2 * n_out]
                du.copy_(hu, non_blocking=True)
                grads = [(torch.empty_like(self.scenes[s].V), torch.empty_like(self.scenes[s].f),
                          torch.empty_like(self.scenes[s].rgb)) for s in scenes]
                r.step(out, (du[:3 * P], du[3 * P:4 * P], du[4 * P:5 * P]), grads)
            else:
                r.prepare()
                r.forward_raw(out)
            host[:n_out].copy_(dev[:n_out], non_blocking=True)
            ev = torch.cuda.Event()
            ev.record(stream)
        return _Inflight(reqs, r, slot, n_out, grads, ev, nbytes)

    def _finish(self, b: _Inflight, now: float, results: dict):
        with torch.cuda.stream(b.slot.stream):
            info = b.raster.info()   # the batch is complete: this does not wait
        if info.status & (TTS_STATUS_KEY_OVERFLOW | TTS_STATUS_SURV_OVERFLOW):
            return False         # capacity estimate too small: caller re-runs the batch
        P = b.raster.total_pixels
        host = b.slot.host
        for i, (q, off) in enumerate(zip(b.reqs, b.raster.pix_off)):
            H, W = int(q.camera.height), int(q.camera.width)
            g = b.grads[i] if b.grads is not None else None
            results[q.rid] = Result(
                q.rid, host[3 * off:3 * off + 3 * H * W].clone().view(3, H, W),
                host[3 * P + off:3 * P + off + H * W].clone().view(H, W),
                host[4 * P + off:4 * P + off + H * W].clone().view(H, W), g, now,
                now - q.arrival, len(b.reqs))
        return True

    # -- the loop --------------------------------------------------------------
    def run(self, requests: Sequence[Request], realtime: bool = True):
        """Serves ``requests`` (arrival times in seconds from the start) and
        returns ({rid: Result}, stats)."""
        pending = collections.deque(sorted(requests, key=lambda q: q.arrival))
        ready = collections.deque()
        inflight: list[_Inflight] = []
        results: dict = {}
        free = list(range(len(self.slots)))
        busy_bytes = 0.0
        n_batches = 0
        retries = 0
        max_inflight = 0
        t0 = time.perf_counter()
        clock = (lambda: time.perf_counter() - t0) if realtime else (lambda: float("inf"))
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
                    if not self._finish(b, t, results):
                        # a capacity estimate was too small: grow the
                        # estimates of this batch's scenes and run it again
                        for q in reversed(b.reqs):
                            ready.appendleft(q)
                        for sc in {q.scene for q in b.reqs}:
                            self.key_margin[sc] *= 2.0
                        retries += 1
                    progressed = True
            while ready and free:
                kind = ready[0].want_grad
                batch = []
                rest = collections.deque()
                while ready and len(batch) < self.max_views:
                    q = ready.popleft()
                    (batch if q.want_grad == kind else rest).append(q)
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
        lat = np.array([r.latency for r in results.values()]) * 1e3
        px = sum(int(q.camera.width) * int(q.camera.height) for q in requests)
        first = min(q.arrival for q in requests) if requests else 0.0
        stats = {"requests": len(requests), "batches": n_batches, "retries": retries,
                 "max_inflight": max_inflight,
                 "p50_ms": float(np.percentile(lat, 50)) if len(lat) else None,
                 "p99_ms": float(np.percentile(lat, 99)) if len(lat) else None,
                 "mpix_s": px / max(t_end - first, 1e-9) / 1e6, "wall_s": t_end}
        return results, stats


def poisson_requests(rng: np.random.Generator, n: int, rate: float, n_scenes: int,
                     sizes=(256, 512, 768, 1024), grad_fraction: float = 0.3, start: float = 0.0):
    """Synthetic request stream: Poisson arrivals at ``rate`` per second,
    random scene, random view on the radius-2.5 sphere at a size from
    ``sizes``, ``grad_fraction`` of them forward + backward with N(0,1)
    upstream gradients."""
    t = start
    out = []
    for i in range(n):
        t += rng.exponential(1.0 / rate)
        res = int(rng.choice(sizes))
        cam = _camera.on_sphere(rng, res, res)
        want = bool(rng.uniform() < grad_fraction)
        up = None
        if want:
            up = (rng.normal(size=(3, res, res)).astype(np.float32),
                  rng.normal(size=(res, res)).astype(np.float32),
                  rng.normal(size=(res, res)).astype(np.float32))
        out.append(Request(i, int(rng.integers(n_scenes)), cam, want, t, up))
    return out


def latency_of(results: dict) -> tuple:
    lat = np.array([r.latency for r in results.values()]) * 1e3
    return float(np.percentile(lat, 50)), float(np.percentile(lat, 99))


__all__ = ["Server", "Request", "Result", "poisson_requests", "latency_of"]
