"""Benchmark of the tetrahedron splatting rasterizer: forward + backward
throughput in Mpixel/s.

Workload (default): the 128^3 structured grid (12,582,912 tets, 2,146,689
vertices) with the three-sphere SDF, 4 views at 512x512, s = 175, 16x16 tiles.
One step = pre-filter (view independent) + forward of all views + backward of
all views, the inputs resident in HBM.  The seeded synthetic inputs come from
``synth``; the upstream gradient is seeded N(0, 1).

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on
the same workload instead (one view per step, bounded sample).
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = ("fwd+bwd Mpixel/s (128³ grid, 4×512² views) vs plain path; "
          "serve p50/p99 latency")
UNIT = "Mpixel/s"

# FP32 work per fragment of the blend kernels: the forward's chord test (18
# flop) and opacity and compositing (30 flop, of which 4 are special-function
# operations: two exponentials and two reciprocals); the backward's ~150 flop
# of which 5 are special-function operations (the recomputed opacity and
# 1 / (1 - alpha)).  FMA-pipe flop and MUFU operations are set against the
# peaks the build measures with its own microbenchmarks (libtets_peaks.so).
FWD_FLOP_PER_FRAG = 48
BWD_FLOP_PER_FRAG = 150
FWD_MUFU_PER_FRAG = 4
BWD_MUFU_PER_FRAG = 5

# DRAM bytes (read + write) per launch of the blend kernels on this workload,
# from one ncu capture (profiles/blend_spheres128_4x512.md), keyed by the
# sha256 prefix of the kernel source they were taken on and the tile size: a
# changed kernel reports no traffic until it is captured again.
KERNEL_TRAFFIC = {
    "d610ca1a9a522701": {8: {"blend_fwd": 141488128, "blend_bwd_px": 151716736}},
}


# Issue rate and occupancy of the blend kernels from one `ncu --set full`
# capture each on the one-view case of this workload (tile 8,
# profiles/blend_spheres128_4x512.md), keyed like KERNEL_TRAFFIC.
KERNEL_NCU_ONE_VIEW = {
    "d610ca1a9a522701": {8: {
        "blend_fwd": {"issued_warps_per_scheduler": 0.48, "achieved_occupancy": 0.220,
                      "warp_instructions": 47448529, "ms": 0.1231},
        "blend_bwd_px": {"issued_warps_per_scheduler": 0.27, "achieved_occupancy": 0.422,
                         "warp_instructions": 14462974, "ms": 0.0536}}},
}


def kernel_source_hash() -> str:
    import hashlib
    path = os.path.join(ROOT, "paper_2406_01579_b300", "csrc", "blend.cu")
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--s", type=float, default=175.0)
    ap.add_argument("--tile", type=int, default=0,
                    help="tile edge 8, 16 or 32; 0: picked by the library's autotuner on this batch")
    ap.add_argument("--blend-segment", type=int, default=0,
                    help="list entries per backward segment (0: autotuned, or the library "
                         "default with --tile)")
    ap.add_argument("--blend-warps", type=int, default=0,
                    help="warps per block of the blend kernels (0: autotuned, or the library "
                         "default with --tile)")
    ap.add_argument("--frag-cap", type=int, default=0,
                    help="per-pixel fragment lists for the backward (0: library default, "
                         "-1: none)")
    ap.add_argument("--hull", type=int, default=0, choices=[0, 1],
                    help="tile test against the projected tet (1) or bbox rects only (0)")
    ap.add_argument("--res", type=int, default=512)
    ap.add_argument("--views", type=int, default=4)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the normal-map step and the geometry-term timings")
    ap.add_argument("--workload", default="spheres128", choices=["spheres128", "batched", "serve"])
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--serve-rates", default="200,500,1000,2000")
    ap.add_argument("--no-workloads", action="store_true",
                    help="skip the batched-uneven and serving summaries of the default line")
    ap.add_argument("--line-serve-requests", type=int, default=1000,
                    help="requests per rate of the serving summary in the default line")
    return ap.parse_args()


def workload_name(a):
    return (f"spheres128: 128^3 grid x6 tets (12,582,912 tets, 2,146,689 vertices), "
            f"{a.views} views at {a.res}x{a.res}, s={a.s:g}, tile {a.tile}, "
            f"backward segment {a.blend_segment or 256}, {a.blend_warps or 4} warps per blend block, "
            + (f"per-pixel fragment lists of {a.frag_cap or 128}" if a.frag_cap >= 0
               else "no per-pixel fragment lists")
            + f"{', hull test' if a.hull else ', bbox rects'}")


# ---------------------------------------------------------------------------
# clocks
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("timestamp,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        # the raw samples; the JSON line carries their summary
        self.path = os.path.join(os.environ.get("TTS_CLOCKS_DIR", tempfile.gettempdir()),
                                 f"tts_clocks_rank{gpu_index}.csv")
        self.gpu = gpu_index

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv",
                 "-lms", "20"], stdout=self.fh, stderr=subprocess.DEVNULL)
            # wait for the first sample so that the timed region is covered
            t0 = time.time()
            while time.time() - t0 < 10:
                self.fh.flush()
                if len(open(self.path).read().splitlines()) >= 2:
                    break
                time.sleep(0.02)
        except Exception:
            self.proc = None
        self.window = [None, None]

    def mark(self, i):
        self.window[i] = time.time()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        import datetime
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        rows = []
        for line in open(self.path).read().splitlines()[1:]:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                ts = datetime.datetime.strptime(parts[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
                rows.append((ts, float(parts[1].split()[0]), float(parts[2].split()[0]), parts))
            except ValueError:
                continue
        lo, hi = self.window
        inside = [r for r in rows if lo is not None and lo - 0.03 <= r[0] <= hi + 0.03]
        if not inside and rows:   # timed region shorter than the sampling period
            inside = [min(rows, key=lambda r: abs(r[0] - lo))] if lo is not None else rows[-1:]
        for ts, c, cm, parts in inside:
            sm.append(c)
            smax.append(cm)
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
def run_ours(a, rank, world):
    import torch

    import synth
    from paper_2406_01579_b300 import Params, Rasterizer, SceneTensors, _lib
    from paper_2406_01579_b300.multirank import (allreduce_grads, job_mpix_s, max_over_ranks,
                                                 rank_cameras)
    from paper_2406_01579_b300.pipeline import HostStepPipeline

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    sc = synth.scene_spheres128(res=a.res, n_views=a.views)
    # weak scaling: each rank renders its own views of the scene
    sc.cams = rank_cameras(sc.cams, rank, a.res, a.res)
    st = SceneTensors(*(torch.from_numpy(x).to(dev) for x in (sc.V, sc.T, sc.f, sc.rgb)))
    tune = None
    if a.tile == 0:
        # the library's autotuner: tile, then backward segment, then warps per block
        from paper_2406_01579_b300.autotune import autotune
        best, times = autotune([st], [(c, 0) for c in sc.cams],
                               Params(s=a.s, hull=bool(a.hull)), cache_path=None)
        a.tile = best["tile"]
        if a.blend_segment == 0:
            a.blend_segment = best["blend_segment"]
        if a.blend_warps == 0:
            a.blend_warps = best["blend_warps"]
        if a.frag_cap == 0:
            a.frag_cap = best["frag_cap"]
        tune = {"picked": best,
                "ms_per_step": {k: {str(c): round(t, 4) for c, t in v.items()}
                                for k, v in times.items()}}
    params = Params(s=a.s, tile=a.tile, blend_segment=a.blend_segment, hull=bool(a.hull),
                    blend_warps=a.blend_warps, frag_cap=a.frag_cap)
    r = Rasterizer([st], [(c, 0) for c in sc.cams], params, device=dev)
    r.forward()
    r.shrink_to_fit(1.15)
    r.forward()
    ups = synth.upstream_grads(2 + rank, sc.cams)
    gi = torch.from_numpy(np.concatenate([u[0].ravel() for u in ups])).to(dev)
    ga = torch.from_numpy(np.concatenate([u[1].ravel() for u in ups])).to(dev)
    gd = torch.from_numpy(np.concatenate([u[2].ravel() for u in ups])).to(dev)
    img, alpha, depth = r._outputs()
    grads = [(torch.empty_like(st.V), torch.empty_like(st.f), torch.empty_like(st.rgb))]
    L = r.lib
    import ctypes
    stream = torch.cuda.current_stream(dev)
    sp = stream.cuda_stream
    dV = (ctypes.c_void_p * 1)(grads[0][0].data_ptr())
    df = (ctypes.c_void_p * 1)(grads[0][1].data_ptr())
    dc = (ctypes.c_void_p * 1)(grads[0][2].data_ptr())
    b = r.batch()
    bp = ctypes.byref(b)
    stages = ["prefilter", "bin", "blend_fwd", "blend_bwd", "scatter_bwd"]
    outs = _lib.tts_outputs()
    outs.image, outs.alpha, outs.depth, outs.normal = (img.data_ptr(), alpha.data_ptr(),
                                                        depth.data_ptr(), None)
    ups_c = _lib.tts_upstream()
    ups_c.dimage, ups_c.dalpha, ups_c.ddepth, ups_c.dnormal = (gi.data_ptr(), ga.data_ptr(),
                                                               gd.data_ptr(), None)

    def step(ev=None):
        """One training step through the public entry points (pre-filter,
        render forward, render backward); with ev, the same work through the
        per-stage entry points with an event between stages (stage timing)."""
        if ev is None:
            _lib.check(L.tts_prepare_scene(bp, sp))
            _lib.check(L.tts_render_fwd_ex(bp, ctypes.byref(outs), sp))
            _lib.check(L.tts_render_bwd_ex(bp, ctypes.byref(ups_c), dV, df, dc, sp))
            allreduce_grads(grads, dist)     # the scene's gradient over all ranks' views
            return
        ev[0].record(stream)
        _lib.check(L.tts_prepare_scene(bp, sp))
        ev[1].record(stream)
        _lib.check(L.tts_bin_views(bp, sp))
        ev[2].record(stream)
        _lib.check(L.tts_blend_fwd(bp, img.data_ptr(), alpha.data_ptr(), depth.data_ptr(), sp))
        ev[3].record(stream)
        _lib.check(L.tts_blend_bwd(bp, gi.data_ptr(), ga.data_ptr(), gd.data_ptr(), sp))
        ev[4].record(stream)
        _lib.check(L.tts_scatter_bwd(bp, dV, df, dc, sp))
        ev[5].record(stream)
        allreduce_grads(grads, dist)

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(a.warmup, 3)):
        step()
    info = r.info()
    assert info.status == 0, f"status {info.status}"
    barrier()
    clk = ClockSampler(dev.index)
    clk.start()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(6)] for _ in range(a.steps)]
    n0 = L.tts_launch_count()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    clk.mark(0)
    t_start.record(stream)
    for k in range(a.steps):
        step()
    t_end.record(stream)
    barrier()
    clk.mark(1)
    time.sleep(0.05)
    clocks = clk.stop()
    launches = L.tts_launch_count() - n0
    elapsed = t_start.elapsed_time(t_end) / 1e3
    # stage breakdown: the same steps again, with events between the stages
    for k in range(a.steps):
        step(evs[k])
    barrier()
    stage_ms = {s: statistics.mean(evs[k][i].elapsed_time(evs[k][i + 1]) for k in range(a.steps))
                for i, s in enumerate(stages)}
    info = r.info()
    assert info.status == 0, f"status {info.status}"
    pixels_per_step = sum(c.width * c.height for c in sc.cams)
    value = job_mpix_s(pixels_per_step, a.steps, elapsed, dist, dev)
    elapsed = max_over_ranks(elapsed, dist, dev)
    # fragments met by the forward (per-pixel counters of the last step)
    Tp, Lp, Np = ctypes.c_void_p(), ctypes.c_void_p(), ctypes.c_void_p()
    _lib.check(L.tts_debug_pixels(bp, ctypes.byref(Tp), ctypes.byref(Lp), ctypes.byref(Np), sp))
    nfrag = int(r._ws_slice(Np.value, 4 * r.total_pixels, torch.int32).sum().item())
    lasts = int(r._ws_slice(Lp.value, 4 * r.total_pixels, torch.int32).sum().item())
    # per-kernel times (events after each launch) and the step's counts
    kt = kernel_times(L, step, dev)
    d = r.debug_lists()
    surv_ids = d["surv"][0].long()
    counts = {"K": int(st.T.shape[0]), "N": int(st.V.shape[0]), "surv": int(info.n_surv[0]),
              "views": len(sc.cams), "keys": int(info.n_keys),
              "tiles": int(d["ranges"].shape[0]), "fragments": nfrag,
              "surv_vertices": int(torch.unique(st.T[surv_ids].reshape(-1)).numel()),
              "visible_slots": int(torch.unique(d["vals"]).numel())}
    del d
    fl = r.debug_frag_lists()
    if fl is not None:   # the backward's per-pixel fragment lists
        nbl = fl[1].long()
        counts.update(blended=int(nbl.sum().item()),
                      listed_pixels=int(((nbl > 0) & (nbl <= fl[3])).sum().item()),
                      overflow_pixels=int((nbl > fl[3]).sum().item()), frag_cap=fl[3])
        # (view, survivor) slots with a blended fragment: those the record ->
        # vertex adjoint reads (exact when no pixel is past the cap)
        lists = fl[0]
        used = torch.arange(lists.shape[1], device=lists.device)[None, :] < nbl[:, None]
        counts["touched_slots"] = int(torch.unique(lists[used]).numel())
    del fl
    res = {
        "kernel_ms": kt, "counts": counts,
        "autotune_ms": tune,
        "elapsed": elapsed, "value": value, "stage_ms": stage_ms, "launches": launches,
        "clocks": clocks, "nfrag": nfrag, "entries_walked": lasts, "n_keys": int(info.n_keys),
        "n_surv": int(info.n_surv[0]), "long_lists": int(info.long_lists),
        "pixels_per_step": pixels_per_step,
    }

    # the same step captured once in a CUDA graph and replayed
    try:
        gstep = r.capture_step((img, alpha, depth), (gi, ga, gd), grads)
        for _ in range(3):
            gstep.replay()
            allreduce_grads(grads, dist)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(a.steps):
            gstep.replay()
            allreduce_grads(grads, dist)
        e1.record(stream)
        barrier()
        tg = e0.elapsed_time(e1) / 1e3
        res["graph"] = job_mpix_s(pixels_per_step, a.steps, tg, dist, dev)
        del gstep
    except Exception as exc:  # capture unsupported: report eager only
        res["graph_error"] = repr(exc)[:200]

    # the paper's resort window (N_w = 5), same step
    if not a.no_plain and rank == 0:
        from paper_2406_01579_b300 import Params as _P
        rw = Rasterizer([st], [(c, 0) for c in sc.cams], _P(s=a.s, tile=a.tile, resort_window=5),
                        device=dev)
        rw.forward()
        rw.shrink_to_fit(1.15)
        outw = rw._outputs()
        for _ in range(3):
            rw.step(outw, (gi, ga, gd), grads)
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        nsw = max(3, a.steps // 2)
        for _ in range(nsw):
            rw.step(outw, (gi, ga, gd), grads)
        e1.record(stream)
        barrier()
        res["window5"] = pixels_per_step * nsw / (e0.elapsed_time(e1) / 1e3) / 1e6
        del rw, outw

    # plain single-view path: one view per call, everything per call
    if not a.no_plain and rank == 0:
        plains = [Rasterizer([st], [(c, 0)], params, device=dev) for c in sc.cams]
        for p_ in plains:
            p_.forward()
            p_.shrink_to_fit(1.15)
        for p_, (ui, ua, ud) in zip(plains, ups):
            p_._gi = torch.from_numpy(ui.ravel()).to(dev)
            p_._ga = torch.from_numpy(ua.ravel()).to(dev)
            p_._gd = torch.from_numpy(ud.ravel()).to(dev)

        def plain_step():
            for p_ in plains:
                p_.forward(prepare=True, check_status=False)
                p_.backward(p_._gi, p_._ga, p_._gd, grads=grads)

        for _ in range(3):
            plain_step()
        torch.cuda.synchronize(dev)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ns = max(3, a.steps // 2)
        e0.record(stream)
        for _ in range(ns):
            plain_step()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        tp = e0.elapsed_time(e1) / 1e3
        res["plain"] = pixels_per_step * ns / tp / 1e6
        del plains

    if not a.no_extras and rank == 0:
        res["extras"] = extras(a, st, sc, params, ups, dev, barrier)

    # end to end through the public API with host buffers
    if not a.no_e2e:
        hV = torch.from_numpy(sc.V).pin_memory()
        hf = torch.from_numpy(sc.f).pin_memory()
        hc = torch.from_numpy(sc.rgb).pin_memory()
        hgi, hga, hgd = gi.cpu().pin_memory(), ga.cpu().pin_memory(), gd.cpu().pin_memory()
        odV = torch.empty(grads[0][0].shape, dtype=torch.float32).pin_memory()
        odf = torch.empty(grads[0][1].shape, dtype=torch.float32).pin_memory()
        odc = torch.empty(grads[0][2].shape, dtype=torch.float32).pin_memory()
        bi = sum(x.numel() * 4 for x in (hV, hf, hc, hgi, hga, hgd))
        bo = sum(x.numel() * 4 for x in (odV, odf, odc))

        # every step copies its inputs in and its gradients out; the copies
        # of neighbouring steps overlap the compute (HostStepPipeline)
        pipe = HostStepPipeline(
            r, reduce_grads=(lambda g: allreduce_grads(g, dist)) if dist is not None else None)

        def e2e_step():
            pipe.step([(hV, hf, hc)], (hgi, hga, hgd), [(odV, odf, odc)])

        pipe.begin()
        for _ in range(3):
            e2e_step()
        pipe.end()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        pipe.begin()
        for _ in range(a.steps):
            e2e_step()
        pipe.end()
        e1.record(stream)
        barrier()
        te = e0.elapsed_time(e1) / 1e3
        res["e2e"] = {"value": job_mpix_s(pixels_per_step, a.steps, te, dist, dev), "unit": UNIT,
                      "h2d_bytes_per_step": bi, "d2h_bytes_per_step": bo,
                      "overlap": "copies of neighbouring steps overlap compute (two buffer sets)"}
        r.set_scenes([st])

        # the same with the scene resident (a training loop keeps the grid's
        # parameters and their gradients on the device for its optimizer):
        # every step copies its upstream gradients in from pinned host memory
        # (two buffer sets, step i+1's copy under step i's compute) and reads
        # back one scalar of its result (the sum of dL/df)
        h2d = torch.cuda.Stream(device=dev)
        hup = (hgi, hga, hgd)
        ubufs = [tuple(torch.empty(x.shape, dtype=x.dtype, device=dev) for x in hup)
                 for _ in range(2)]
        ev_in = [torch.cuda.Event() for _ in range(2)]
        ev_used = [torch.cuda.Event() for _ in range(2)]
        hsum = torch.empty(1, dtype=torch.float32).pin_memory()
        out_r = r._outputs()

        def resident_step(i):
            b = i & 1
            if i >= 2:
                h2d.wait_event(ev_used[b])       # step i-2 has consumed buffer set b
            with torch.cuda.stream(h2d):
                for d, h in zip(ubufs[b], hup):
                    d.copy_(h, non_blocking=True)
                ev_in[b].record(h2d)
            stream.wait_event(ev_in[b])
            r.step(out_r, ubufs[b], grads)
            ev_used[b].record(stream)
            hsum.copy_(grads[0][1].sum().reshape(1), non_blocking=True)

        h2d.wait_stream(stream)
        for i in range(3):
            resident_step(i)
        torch.cuda.synchronize(dev)
        barrier()
        e0.record(stream)
        h2d.wait_stream(stream)
        for i in range(a.steps):
            resident_step(i)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        tr = e0.elapsed_time(e1) / 1e3
        res["e2e_resident"] = {
            "value": job_mpix_s(pixels_per_step, a.steps, tr, dist, dev), "unit": UNIT,
            "h2d_bytes_per_step": sum(x.numel() * 4 for x in hup), "d2h_bytes_per_step": 4,
            "what": "scene parameters and gradients resident on the device; per step the "
                    "upstream gradients from pinned host memory in, one scalar of the result "
                    "(sum of dL/df) out"}
    # the quick serve (a small mix with the benchmark scene) when the full
    # serving summary does not run
    if not a.no_serve and rank == 0 and (a.no_workloads or world > 1):
        res["serve"] = quick_serve(a, st, dev)
    res["sc"] = sc
    if dist is not None:
        dist.barrier()
    return res


# ---------------------------------------------------------------------------
# ALU peaks (own microbenchmarks) and per-kernel times
# ---------------------------------------------------------------------------
def measure_alu_peaks(dev, target_ms=25.0):
    """FP32 FMA TFLOP/s and ex2 / rcp MUFU Gop/s of this GPU, each the best of
    three launches of register-resident dependency chains (libtets_peaks.so)
    sized to about target_ms, timed with CUDA events; the SM clock is sampled
    meanwhile."""
    import ctypes

    import torch
    path = os.path.join(ROOT, "paper_2406_01579_b300", "libtets_peaks.so")
    L = ctypes.CDLL(path)
    L.tts_peak_fma.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                               ctypes.POINTER(ctypes.c_double), ctypes.c_void_p]
    L.tts_peak_mufu.argtypes = [ctypes.c_int] + L.tts_peak_fma.argtypes
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = 8 * sms, 256
    out = torch.empty(blocks * threads, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    ops = ctypes.c_double()

    def launch(which, iters):
        if which == "fma":
            rc = L.tts_peak_fma(blocks, threads, iters, out.data_ptr(), ctypes.byref(ops),
                                stream.cuda_stream)
        else:
            rc = L.tts_peak_mufu(0 if which == "ex2" else 1, blocks, threads, iters,
                                 out.data_ptr(), ctypes.byref(ops), stream.cuda_stream)
        assert rc == 0, f"peak kernel {which} failed"
        return ops.value

    def timed(which, iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        n = launch(which, iters)
        e1.record(stream)
        e1.synchronize()
        return n, e0.elapsed_time(e1)

    clk = ClockSampler(dev.index)
    clk.start()
    clk.mark(0)
    res = {}
    for which in ("fma", "ex2", "rcp"):
        timed(which, 16)                           # warm-up
        _, ms = timed(which, 64)
        iters = max(64, int(64 * target_ms / max(ms, 1e-3)))
        runs = [timed(which, iters) for _ in range(3)]
        res[which] = runs[0][0] / (min(t for _, t in runs) / 1e3)
    clk.mark(1)
    clocks = clk.stop()
    # sanity: the chains' results are finite and no rate exceeds twice its
    # nominal bound at the maximum clock (FMA: 128 lanes x 2 flop per SM and
    # clock; MUFU: 32 lanes per SM and clock)
    assert bool(torch.isfinite(out).all()), "peak kernels produced non-finite values"
    nominal = {"fma": sms * 128 * 2 * 2.032e9, "ex2": sms * 32 * 2.032e9, "rcp": sms * 32 * 2.032e9}
    for k, v in res.items():
        assert v < 2.0 * nominal[k], f"{k} peak {v:.3e}/s is above twice its nominal bound"
    return {"fma_tflops": res["fma"] / 1e12, "ex2_gops": res["ex2"] / 1e9,
            "rcp_gops": res["rcp"] / 1e9, "mufu_gops": min(res["ex2"], res["rcp"]) / 1e9,
            "launch": f"{blocks} blocks x {threads} threads, 8 independent chains per thread",
            "clocks": clocks}


def kernel_times(L, step, dev, n_steps=10):
    """Per-kernel times of one step: the library records an event after each
    of its kernel launches (tts_debug_kernel_events); the time of kernel i is
    the gap between events i-1 and i (the events keep the kernels from
    overlapping, so the sum exceeds the pipelined step a little).  Mean over
    n_steps steps; names from the runtime."""
    import ctypes
    import re

    import torch
    stream = torch.cuda.current_stream(dev)
    nmax = 64
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(nmax + 1)]
    for e in evs:
        e.record(stream)            # creates the CUDA events
    torch.cuda.synchronize(dev)
    handles = (ctypes.c_void_p * nmax)(*[e.cuda_event for e in evs[1:]])
    tot, names = None, None
    for _ in range(n_steps):
        _lib_check(L.tts_debug_kernel_events(handles, nmax))
        evs[0].record(stream)
        step()
        torch.cuda.synchronize(dev)
        buf = (ctypes.c_char_p * nmax)()
        n = L.tts_debug_kernel_events_used(buf, nmax)
        ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(n)]
        nm = []
        for i in range(n):
            raw = (buf[i] or b"?").decode(errors="replace")
            m = re.search(r"k_[a-z0-9_]+", raw)     # the name inside a mangled symbol
            nm.append(m.group(0) if m else raw)
        if tot is None:
            tot, names = ms, nm
        else:
            tot = [x + y for x, y in zip(tot, ms)]
    _lib_check(L.tts_debug_kernel_events(None, 0))
    out = {}
    for name, t in zip(names, tot):
        out[name] = out.get(name, 0.0) + t / n_steps
    return out


def _lib_check(rc):
    assert rc == 0, f"library call failed ({rc})"


def kernel_rooflines(kt, counts, peaks, hbm_gbs):
    """Per kernel: algorithmic bytes (HBM-bound kernels) or FMA-pipe flop and
    MUFU operations (blend kernels) per launch over its event-timed duration,
    against the measured peaks.  The byte counts are the data each kernel must
    move at least (unique reads and writes), from the step's counts."""
    K, N, S, NV = counts["K"], counts["N"], counts["surv"], counts["views"]
    U, keys, tiles = counts["surv_vertices"], counts["keys"], counts["tiles"]
    slots, vis, frag = NV * S, counts["visible_slots"], counts["fragments"]
    chunks = (K + 2047) // 2048
    model = {
        # K1: tet indices + vertex SDF (unique) + flag per tet
        "k_prefilter_flags": ("hbm", 16 * K + 4 * N + K),
        "k_prefilter_scan": ("hbm", 8 * chunks),
        # flags + survivor ids and their vertex ids (read and written)
        "k_prefilter_compact": ("hbm", K + 16 * S + 20 * S),
        # K2: survivor ids + vertex ids + the survivors' vertices (28 B) once;
        # per (view, survivor) the record (96 B), depth bits and tile rect
        "k_preprocess": ("hbm", 20 * S + 28 * U + slots * (96 + 4 + 16)),
        # K3: per tile a count read, a range, a cursor and a class entry written
        "k_tile_scan": ("hbm", 20 * tiles),
        # K4: per slot its rect and depth bits; per key 8 B written
        "k_place": ("hbm", 20 * slots + 8 * keys),
        # K5: per key 8 B read, 4 B written
        "k_tile_sort": ("hbm", 12 * keys),
        "k_worklist_count": ("hbm", 24 * tiles),
        "k_worklist_place": ("hbm", 24 * tiles),
        # K8: touched flags of all slots; for each touched slot (a blended
        # fragment's; every visible slot when that count is missing) its
        # record gradient read and cleared (96 B each way), bbox corner and
        # vertex ids (16 B each) and flag cleared; the survivors' vertices read
        # and their gradients written (28 B each way)
        "k_tet_bwd": ("hbm", slots + (96 + 96 + 16 + 16 + 1) * counts.get("touched_slots", vis)
                      + 56 * U),
        "k_blend_fwd": ("alu", (frag * (FWD_FLOP_PER_FRAG - FWD_MUFU_PER_FRAG),
                                frag * FWD_MUFU_PER_FRAG)),
        "k_blend_bwd": ("alu", (frag * (BWD_FLOP_PER_FRAG - BWD_MUFU_PER_FRAG),
                                frag * BWD_MUFU_PER_FRAG)),
    }
    if "k_blend_bwd_px" in kt:
        # per-pixel fragment lists: the pixel-list kernel does the backward of
        # every listed pixel, the list walk only that of pixels past the cap
        # (the work split by their blended fragments; all of it to the
        # pixel-list kernel when none is past the cap)
        share = 1.0
        if counts.get("overflow_pixels", 0) > 0:
            share = counts["listed_pixels"] / max(counts["listed_pixels"] + counts["overflow_pixels"], 1)
        bf, bm = model.pop("k_blend_bwd")[1]
        model["k_blend_bwd_px"] = ("alu", (bf * share, bm * share))
        if share < 1.0:
            model["k_blend_bwd"] = ("alu", (bf * (1 - share), bm * (1 - share)))
    out = []
    for name, ms in sorted(kt.items(), key=lambda x: -x[1]):
        rec = {"kernel": name, "ms": round(ms, 5)}
        if name in model and ms > 0:
            bound, work = model[name]
            if bound == "hbm":
                ach = work / (ms / 1e3) / 1e9
                rec.update(bound="hbm", bytes=int(work), achieved=ach, peak=hbm_gbs, unit="GB/s",
                           frac=ach / hbm_gbs)
            else:
                flop, mufu = work
                af = flop / (ms / 1e3) / 1e12
                am = mufu / (ms / 1e3) / 1e9
                ff, fm = af / peaks["fma_tflops"], am / peaks["mufu_gops"]
                rec.update(bound="alu", fma_flop=int(flop), mufu_ops=int(mufu),
                           achieved=af, peak=peaks["fma_tflops"], unit="TFLOP/s", frac=max(ff, fm),
                           fma_frac=ff, mufu_frac=fm, mufu_gops=am)
        out.append(rec)
    return out


def extras(a, st, sc, params, ups, dev, barrier):
    """Timings beside the headline step on the same 128^3 grid: the step with
    the Eq. 2 normal map as a fourth channel, and the geometry terms (unique
    edges, Sec. 4.2 regularizers with gradients, Marching Tetrahedra, the
    App. B.1 coarse-to-fine bounds and refit)."""
    import ctypes
    import dataclasses

    import torch

    from paper_2406_01579_b300 import Rasterizer, _lib, fit_grid
    from paper_2406_01579_b300.geometry import Regularizers, tet_edges

    stream = torch.cuda.current_stream(dev)
    out = {}

    def timed(fn, n):
        for _ in range(2):
            fn()
        barrier()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(n):
            fn()
        e1.record(stream)
        barrier()
        return e0.elapsed_time(e1) / n

    # the step with the normal map (upstream dL/dnormal ~ N(0, 1))
    rn = Rasterizer([st], [(c, 0) for c in sc.cams], dataclasses.replace(params, normals=True),
                    device=dev)
    rn.forward()
    rn.shrink_to_fit(1.15)
    on = rn._outputs()
    g = np.random.default_rng(7)
    upn = [torch.from_numpy(np.concatenate([u[i].ravel() for u in ups])).to(dev) for i in range(3)]
    upn.append(torch.from_numpy(g.normal(size=3 * rn.total_pixels).astype(np.float32)).to(dev))
    gr = [(torch.empty_like(st.V), torch.empty_like(st.f), torch.empty_like(st.rgb))]
    ms = timed(lambda: rn.step(on, upn, gr), max(3, a.steps // 2))
    out["normals_step_mpix_s"] = rn.total_pixels / (ms / 1e3) / 1e6
    del rn, on
    # unique edges (topology, once per grid) and the regularizers
    N, K = st.V.shape[0], st.T.shape[0]
    out["edges_ms"] = timed(lambda: tet_edges(st.T, N), 2)
    E = tet_edges(st.T, N)
    reg = Regularizers(N, dev)
    dV, df = torch.empty_like(st.V), torch.empty_like(st.f)
    out["regularizers_ms"] = timed(lambda: reg(st.V, st.T, st.f, E, 1.0, 1.0, grads=(dV, df)), 5)
    out["n_edges"] = int(E.shape[0])
    # Marching Tetrahedra: outputs sized by a first call, then the timed calls
    L = _lib.load()
    nb = ctypes.c_size_t(0)
    _lib.check(L.tts_marching_tets_workspace_size(K, E.shape[0], ctypes.byref(nb)))
    ws = torch.empty(int(nb.value), dtype=torch.uint8, device=dev)
    counts = torch.zeros(2, dtype=torch.int64, device=dev)
    dummy = torch.empty(3, dtype=torch.float32, device=dev)
    dummyi = torch.empty(3, dtype=torch.int32, device=dev)
    args = (st.V.data_ptr(), st.T.data_ptr(), st.f.data_ptr(), N, K, E.data_ptr(), E.shape[0])
    _lib.check(L.tts_marching_tets(*args, dummy.data_ptr(), None, 0, dummyi.data_ptr(), 0,
                                   counts.data_ptr(), ws.data_ptr(), ws.numel(), stream.cuda_stream))
    nv, nt = (int(x) for x in counts.cpu())
    verts = torch.empty((nv, 3), dtype=torch.float32, device=dev)
    tris = torch.empty((nt, 3), dtype=torch.int32, device=dev)

    def mt():
        _lib.check(L.tts_marching_tets(*args, verts.data_ptr(), None, nv, tris.data_ptr(), nt,
                                       counts.data_ptr(), ws.data_ptr(), ws.numel(),
                                       stream.cuda_stream))
    out["marching_tets_ms"] = timed(mt, 5)
    out["mesh"] = {"vertices": nv, "triangles": nt}
    # Sec. 3.3's device radix sort on this step's (tile, depth) keys, in the
    # order the binning emits them (slot-major, then tile), beside the
    # binning's own per-tile on-chip ordering (part of the headline step) and
    # a library sort (torch.sort, all 64 key bits) of the same keys
    rk = Rasterizer([st], [(c, 0) for c in sc.cams], params, device=dev)
    rk.forward()
    d = rk.debug_lists()
    k = d["keys"].cpu().numpy().view(np.uint64)
    v = d["vals"].cpu().numpy()
    order = np.lexsort((k >> np.uint64(d["depth_bits"]), v))
    kin = torch.from_numpy(k[order].view(np.int64).copy()).to(dev)
    vin = torch.from_numpy(v[order].copy()).to(dev)
    bits = int(d["info"].sort_bits)
    need = ctypes.c_size_t(0)
    _lib.check(L.tts_sort_pairs_scratch_size(kin.numel(), ctypes.byref(need)))
    scratch = torch.empty(int(need.value), dtype=torch.uint8, device=dev)
    kout, vout = torch.empty_like(kin), torch.empty_like(vin)

    def radix():
        _lib.check(L.tts_sort_pairs(kin.data_ptr(), vin.data_ptr(), kout.data_ptr(),
                                    vout.data_ptr(), kin.numel(), bits, scratch.data_ptr(),
                                    scratch.numel(), stream.cuda_stream))
    out["radix_sort_ms"] = timed(radix, 5)
    out["radix_sort_matches_binning"] = bool(torch.equal(kout, d["keys"]) and torch.equal(vout, d["vals"]))

    def lib_sort():
        sk, idx = torch.sort(kin, stable=True)
        return sk, vin[idx]
    out["torch_sort_ms"] = timed(lib_sort, 5)
    out["sort_keys"] = int(kin.numel())
    out["sort_bits"] = bits
    del rk, kin, vin, kout, vout, scratch
    # coarse-to-fine pre-filter: bounds of the first round's survivors, refit
    rb = Rasterizer([st], [(sc.cams[0], 0)], params, device=dev)
    rb.prepare()
    V2 = torch.empty_like(st.V)
    out["coarse_to_fine_ms"] = timed(
        lambda: fit_grid(st.V, [-1.0] * 3, [1.0] * 3, rb.survivor_bounds()[0], 0.05, out=V2), 5)
    del rb
    # walk statistics of one untimed step (TTS_FLAG_COUNT), with bbox rects and
    # with the hull test: keys, list groups scanned, candidates staged (forward
    # and list-walk backward), blended fragments of the pixel-list backward
    walks = {}
    for hull in (False, True):
        pw = dataclasses.replace(params, hull=hull, count_walk=True)
        rw = Rasterizer([st], [(c, 0) for c in sc.cams], pw, device=dev)
        rw.forward()
        rw.shrink_to_fit(1.15)
        ow = rw._outputs()
        uw = tuple(torch.from_numpy(np.concatenate([u[i].ravel() for u in ups])).to(dev)
                   for i in range(3))
        gw = [(torch.empty_like(st.V), torch.empty_like(st.f), torch.empty_like(st.rgb))]
        rw.debug_walk_counts(reset=True)
        rw.step(ow, uw, gw)
        w = rw.debug_walk_counts(reset=True)
        w["keys"] = int(rw.info().n_keys)
        fl = rw.debug_frag_lists()
        if fl is not None:
            w["blended"] = int(fl[1].long().sum().item())
        walks["hull" if hull else "bbox"] = w
        del rw, ow, gw
    out["walk_counts"] = walks
    return out


def resident_scenes(rng, n_list, dev):
    """Scenes of the given grid resolutions (sphere or torus SDF + noise); the
    grid's vertex positions and tet indices are shared on the device by the
    scenes of one resolution."""
    import torch

    import synth
    from paper_2406_01579_b300 import SceneTensors
    out, grid = [], {}
    for n in n_list:
        V, T, f, rgb = synth.random_scene(rng, int(n), "sphere" if rng.uniform() < 0.5 else "torus")
        if int(n) not in grid:
            grid[int(n)] = (torch.from_numpy(V).to(dev), torch.from_numpy(T).to(dev))
        Vd, Td = grid[int(n)]
        out.append(SceneTensors(Vd, Td, torch.from_numpy(f).to(dev), torch.from_numpy(rgb).to(dev)))
    return out


def quick_serve(a, big_scene, dev, n_requests=300, rate=200.0):
    """Served latency on a small mix: the benchmark scene plus 7 resident
    scenes of 32^3..96^3, 300 requests at 200 req/s, 30% forward+backward,
    views 256^2..1024^2."""
    from paper_2406_01579_b300 import Params
    from paper_2406_01579_b300.serve import Server, poisson_requests
    rng = np.random.default_rng(44)
    scenes = [big_scene] + resident_scenes(rng, [32, 48, 64, 96, 32, 48, 64], dev)
    srv = Server(scenes, Params(s=a.s, tile=a.tile), hbm_budget=120e9, max_views=16, streams=3)
    srv.run(poisson_requests(np.random.default_rng(1), 48, rate, len(scenes), pinned=True),
            on_result=lambda r: None)   # warm-up
    srv.run(poisson_requests(np.random.default_rng(3), 100, 4 * rate, len(scenes), pinned=True),
            on_result=lambda r: None)
    srv.reserve()
    reqs = poisson_requests(np.random.default_rng(2), n_requests, rate, len(scenes), pinned=True)
    _, stats = srv.run(reqs, on_result=lambda r: None)
    stats.update({"rate_req_s": rate, "scenes": len(scenes),
                  "mix": "views 256..1024 px, 30% fwd+bwd, 128^3 + 7 scenes of 32..96^3"})
    return stats


# ---------------------------------------------------------------------------
# the oracle (CPU) on a bounded sample of the same workload
# ---------------------------------------------------------------------------
def oracle_step(sc, view_ids, a, upstream, nthreads=0, tile=None):
    import oracle
    tile = a.tile if tile is None else tile
    op = oracle.make_params(s=float(np.float32(a.s)), tile=tile,
                            prefilter_thresh=float(np.float32(1 / 255)),
                            alpha_skip=float(np.float32(1 / 255)),
                            alpha_cap=float(np.float32(0.99)), t_eps=float(np.float32(1e-4)))
    surv, _, _ = oracle.prefilter(sc.T, sc.f, op)
    px = 0
    for v in view_ids:
        cam = sc.cams[v]
        bins = oracle.bin_view(surv, sc.T, sc.V, cam, tile, hull=bool(a.hull))
        oracle.render(sc.V, sc.T, sc.f, sc.rgb, cam, op, surv=surv, bins=bins,
                      upstream=upstream[v], nthreads=nthreads)
        px += cam.width * cam.height
    return px


def cpu_baseline(a, sc=None, min_seconds=10.0, max_steps=6):
    """The oracle as it stands on the host cores: whole steps of the same
    workload (pre-filter + all views: bin, FP64 render, adjoint), repeated
    until about min_seconds of CPU work."""
    import synth
    if sc is None:
        sc = synth.scene_spheres128(res=a.res, n_views=a.views)
    ups = synth.upstream_grads(2, sc.cams)
    views = list(range(len(sc.cams)))
    t = time.perf_counter()
    px, steps = 0, 0
    while steps < max_steps and (steps == 0 or time.perf_counter() - t < min_seconds):
        px += oracle_step(sc, views, a, ups)
        steps += 1
    dt = time.perf_counter() - t
    return {"value": px / dt / 1e6, "unit": UNIT, "cores": len(os.sched_getaffinity(0)),
            "kind": "oracle",
            "sample": f"{steps} whole steps of the same workload (pre-filter of the full grid + "
                      f"all {len(views)} views: bin, FP64 render, adjoint); {dt:.1f} s"}


def cpu_configs(a, sc3):
    """The oracle on the three single-GPU configurations, on all host cores
    and on one thread (the render and its adjoint are the OpenMP part; the
    pre-filter and the binning run on one thread in both): 16^3 sphere at
    128^2, 64^3 torus at 512^2, and one of the 4 views of the 128^3 scene
    (with the pre-filter of the whole grid).  Each entry repeats whole steps
    until about `budget` seconds; about 25 s in all on 16 cores."""
    import synth
    tile = a.tile if a.tile else 8
    out = {}
    cases = (("sphere16_128", synth.scene_sphere16(), 16, (1.0, 1.0)),
             ("torus64_512", synth.scene_torus64(), tile, (2.0, 0.1)),
             ("spheres128_512_one_view", sc3, tile, (0.1, 0.1)))
    for name, sc, t, (b_all, b_one) in cases:
        ups = synth.upstream_grads(2, sc.cams[:1])
        rec = {}
        for label, nth, budget in (("all_cores", 0, b_all), ("one_thread", 1, b_one)):
            t0 = time.perf_counter()
            px, steps = 0, 0
            while steps == 0 or (steps < 20 and time.perf_counter() - t0 < budget):
                px += oracle_step(sc, [0], a, ups, nthreads=nth, tile=t)
                steps += 1
            dt = time.perf_counter() - t0
            rec[label] = {"value": px / dt / 1e6, "unit": UNIT, "ms_per_step": dt / steps * 1e3,
                          "steps": steps,
                          "cores": len(os.sched_getaffinity(0)) if nth == 0 else 1}
        rec["tile"] = t
        out[name] = rec
    return out


def run_single_views(a, dev):
    """The two single-view configurations on the GPU (16^3 sphere at 128^2,
    64^3 torus at 512^2): one view per call, pre-filter + forward + backward,
    the tile picked by the autotuner, eager and as a replayed CUDA graph of
    the step.  Each step is timed alone with CUDA events, after a write of
    256 MB (more than L2) that evicts the previous step's data."""
    import torch

    import synth
    from paper_2406_01579_b300 import Params, Rasterizer, SceneTensors
    from paper_2406_01579_b300.autotune import autotune_tile
    flush = torch.empty(64 << 20, dtype=torch.float32, device=dev)
    out = {}
    for name, sc in (("sphere16_128", synth.scene_sphere16()),
                     ("torus64_512", synth.scene_torus64())):
        st = SceneTensors(*(torch.from_numpy(x).to(dev) for x in (sc.V, sc.T, sc.f, sc.rgb)))
        views = [(sc.cams[0], 0)]
        tile, _ = autotune_tile([st], views, Params(s=a.s), reps=3, cache_path=None)
        r = Rasterizer([st], views, Params(s=a.s, tile=tile), device=dev)
        r.forward()
        r.shrink_to_fit(1.15)
        o = r._outputs()
        up = tuple(torch.randn(n, device=dev) for n in (3 * r.total_pixels, r.total_pixels,
                                                           r.total_pixels))
        g = [(torch.empty_like(st.V), torch.empty_like(st.f), torch.empty_like(st.rgb))]
        for _ in range(3):
            r.step(o, up, g)
        def timed(run):
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(a.steps)]
            for e0, e1 in ev:
                flush.fill_(1.0)
                e0.record()
                run()
                e1.record()
            torch.cuda.synchronize(dev)
            return sum(e0.elapsed_time(e1) for e0, e1 in ev) / len(ev)

        ms = timed(lambda: r.step(o, up, g))
        graph = r.capture_step(o, up, g)
        ms_g = timed(graph.replay)
        out[name] = {"value": r.total_pixels / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_step": ms,
                     "graph_mpix_s": r.total_pixels / (ms_g / 1e3) / 1e6, "graph_ms_per_step": ms_g,
                     "steps": a.steps, "tile": tile, "l2": "flushed before every step"}
        del r, o, g, graph
    return out


def run_reference(a):
    import synth
    if a.tile == 0:
        # the autotuner (a GPU measurement) is not run on this arm: the tile it
        # picks on this workload
        a.tile = 8
    sc = synth.scene_spheres128(res=a.res, n_views=a.views)
    ups = synth.upstream_grads(2, sc.cams)
    for k in range(a.warmup):
        oracle_step(sc, [k % len(sc.cams)], a, ups)
    t = time.perf_counter()
    px = 0
    for k in range(a.steps):
        px += oracle_step(sc, [k % len(sc.cams)], a, ups)
    dt = time.perf_counter() - t
    v = px / dt / 1e6
    sample = ("each step: pre-filter of the full grid + one of the 4 views (bin, FP64 render, "
              "adjoint), views in turn")
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": workload_name(a)},
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": len(os.sched_getaffinity(0)),
                            "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_batched(a, emit=True, steps=None):
    """16 scenes of uneven resolution (32..128)^3, 1-8 views each at
    256^2..1024^2, tile size autotuned, one CUDA graph per step (pre-filter +
    forward + backward of all views); compared with the plain single-view
    path on the same views.  Prints its JSON line (emit) or returns it."""
    import torch

    import synth
    from paper_2406_01579_b300 import Params, Rasterizer
    from paper_2406_01579_b300.autotune import autotune
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(3)
    ns = [int(rng.choice([32, 48, 64, 96, 128])) for _ in range(16)]
    scenes = resident_scenes(rng, ns, dev)
    views = []
    for si in range(16):
        for _ in range(int(rng.integers(1, 9))):
            res = int(rng.choice([256, 512, 768, 1024]))
            views.append((synth.random_camera(rng, res, res), si))
    params = Params(s=a.s)
    best, times = autotune(scenes, views, params, reps=2, cache_path=None)
    params = Params(s=a.s, **best)
    r = Rasterizer(scenes, views, params)
    r.forward()
    r.shrink_to_fit(1.15)
    r.forward()
    out = r._outputs()
    up = tuple(torch.randn(n, device=dev) for n in (3 * r.total_pixels, r.total_pixels,
                                                       r.total_pixels))
    grads = [(torch.empty_like(x.V), torch.empty_like(x.f), torch.empty_like(x.rgb)) for x in scenes]
    g = r.capture_step(out, up, grads)
    for _ in range(3):
        g.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    nsteps = steps or a.steps
    e0.record()
    for _ in range(nsteps):
        g.replay()
    e1.record()
    torch.cuda.synchronize()
    t = e0.elapsed_time(e1) / 1e3
    px = r.total_pixels
    # plain path: every view alone, everything per call
    plains = []
    for c, si in views:
        p_ = Rasterizer([scenes[si]], [(c, 0)], params)
        p_.forward()
        p_.shrink_to_fit(1.15)
        plains.append(p_)
    gr1 = [[(torch.empty_like(scenes[si].V), torch.empty_like(scenes[si].f),
             torch.empty_like(scenes[si].rgb))] for _, si in views]
    ups1 = [tuple(torch.randn(n, device=dev) for n in (3 * p_.total_pixels, p_.total_pixels,
                                                          p_.total_pixels)) for p_ in plains]
    outs1 = [p_._outputs() for p_ in plains]

    def plain_step():
        for p_, o, u_, g_ in zip(plains, outs1, ups1, gr1):
            p_.step(o, u_, g_)

    plain_step()
    torch.cuda.synchronize()
    e0.record()
    nplain = max(2, nsteps // 4)
    for _ in range(nplain):
        plain_step()
    e1.record()
    torch.cuda.synchronize()
    tp = e0.elapsed_time(e1) / 1e3 / nplain
    info = r.info()
    rec = {
        "metric": METRIC, "value": px * nsteps / t / 1e6, "unit": UNIT, "n_gpus": 1,
        "steps": nsteps, "ms_per_step": t / nsteps * 1e3, "higher_is_better": True,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"batched uneven: 16 scenes n={ns}, {len(views)} views "
                               f"256..1024 px, s={a.s:g}, one CUDA graph per step",
                   "autotune": {"picked": best,
                                "ms_per_step": {k: {str(c): round(t, 3) for c, t in v.items()}
                                                for k, v in times.items()}}},
        "plain_path_mpix_s": px / tp / 1e6, "batched_vs_plain": (px * nsteps / t) / (px / tp),
        "status": int(info.status), "keys": int(info.n_keys)}
    del g, r, plains, scenes
    torch.cuda.empty_cache()
    if emit:
        print(json.dumps(rec))
    return rec


def run_serve(a, emit=True, requests=None):
    """Serving: 64 resident scenes (32..128)^3, Poisson arrivals, 30%
    forward+backward, views 256^2..1024^2, HBM budget 120 GB.  Prints its
    JSON line (emit) or returns it."""
    import torch

    from paper_2406_01579_b300 import Params
    from paper_2406_01579_b300.serve import Server, poisson_requests
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(4)
    ns = [int(rng.choice([32, 48, 64, 96, 128])) for _ in range(64)]
    scenes = resident_scenes(rng, ns, dev)
    # mixed request sizes: the tile the autotuner picks on the headline workload
    tile = a.tile if a.tile else 8
    srv = Server(scenes, Params(s=a.s, tile=tile), hbm_budget=120e9, max_views=16, streams=3)
    # warm-up: batches as large as the highest rate makes them, so the slots'
    # buffers have grown before the timed runs
    srv.run(poisson_requests(np.random.default_rng(1), 64, 500.0, len(scenes), pinned=True),
            on_result=lambda r: None)
    srv.run(poisson_requests(np.random.default_rng(3), 300, 4000.0, len(scenes), pinned=True),
            on_result=lambda r: None)
    srv.reserve()
    out = []
    nreq = requests or a.serve_requests
    for rate in [float(x) for x in a.serve_rates.split(",")]:
        reqs = poisson_requests(np.random.default_rng(int(rate)), nreq, rate, len(scenes),
                                pinned=True)
        _, st = srv.run(reqs, on_result=lambda r: None)
        st["rate_req_s"] = rate
        out.append(st)
        del reqs
    rec = {"metric": "serve p50/p99 latency (ms) and Mpixel/s", "unit": "ms",
           "config": {"workload": f"serve: 64 resident scenes n={sorted(set(ns))}, "
                                  "views 256..1024 px, 30% fwd+bwd, budget 120 GB, "
                                  "upstream gradients from pinned host tensors",
                      "requests_per_rate": nreq, "tile": tile},
           "rates": out}
    del srv, scenes
    torch.cuda.empty_cache()
    if emit:
        print(json.dumps(rec))
    return rec


def main():
    a = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if a.impl == "reference":
        if rank == 0:
            run_reference(a)
        return
    if a.workload == "batched":
        run_batched(a)
        return
    if a.workload == "serve":
        run_serve(a)
        return
    res = run_ours(a, rank, world)
    if rank != 0:
        return
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    hbm = float(peaks.get("hbm_gbs", 6400.0))
    hbm_src = "MEASURED_PEAKS.json hbm_gbs (of measured)" if "hbm_gbs" in peaks else \
        "fallback 6.4 TB/s (of fallback)"
    import torch
    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    alu = measure_alu_peaks(dev)
    roof = kernel_rooflines(res["kernel_ms"], res["counts"], alu, hbm)
    st = res["stage_ms"]
    dom = max(st, key=st.get)
    # the dominant kernel of the step (by its event-timed duration)
    top = max((x for x in roof if "frac" in x), key=lambda x: x["ms"])
    rk = top["kernel"]
    traffic = KERNEL_TRAFFIC.get(kernel_source_hash(), {}).get(a.tile, {}).get(
        rk.replace("k_", "", 1))
    if top["bound"] == "alu":
        roofline = {"kernel": rk, "bound": "alu", "achieved": top["achieved"],
                    "peak": alu["fma_tflops"], "unit": "TFLOP/s", "frac": top["frac"],
                    "traffic": traffic,
                    "fma": {"achieved_tflops": top["achieved"], "peak_tflops": alu["fma_tflops"],
                            "frac": top["fma_frac"]},
                    "mufu": {"achieved_gops": top["mufu_gops"], "peak_gops": alu["mufu_gops"],
                             "frac": top["mufu_frac"]},
                    "peak_source": "measured by this benchmark (FMA and ex2/rcp chains, "
                                   "libtets_peaks.so), of measured",
                    "ms_per_launch": top["ms"]}
    else:
        roofline = {"kernel": rk, "bound": "hbm", "achieved": top["achieved"], "peak": hbm,
                    "unit": "GB/s", "frac": top["frac"], "traffic": traffic,
                    "peak_source": hbm_src, "ms_per_launch": top["ms"]}
    workloads = None
    if not a.no_workloads and world == 1:
        workloads = {"single_view": run_single_views(a, torch.device("cuda", 0)),
                     "batched_uneven": run_batched(a, emit=False, steps=max(5, a.steps // 4)),
                     "serve": run_serve(a, emit=False, requests=a.line_serve_requests)}
    out = {
        "metric": METRIC, "value": res["value"], "unit": UNIT, "n_gpus": world,
        "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": res["elapsed"] / a.steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": workload_name(a), "global_views": a.views * world,
                   "l2": "inputs larger than L2 (tet indices 201 MB, per-step records "
                         f"{res['n_surv'] * a.views * 96 / 1e6:.0f} MB)",
                   "parallelism": f"dp{world} (own views per GPU; vertex gradients all-reduced)",
                   "autotune": res.get("autotune_ms")},
        "roofline": roofline,
        "rooflines": roof,
        "ncu_one_view": KERNEL_NCU_ONE_VIEW.get(kernel_source_hash(), {}).get(a.tile),
        "alu_peaks": alu,
        "hbm_peak_source": hbm_src,
        "step_counts": res["counts"],
        "stage_ms": st, "dominant_stage": dom,
        "plain_path_mpix_s": res.get("plain"),
        "graph_mpix_s": res.get("graph"),
        "resort_window5_mpix_s": res.get("window5"),
        "serve": res.get("serve"),
        "gpu_launches": res["launches"],
        "fragments_per_step": res["nfrag"], "keys_per_step": res["n_keys"],
        "survivors": res["n_surv"], "long_lists": res["long_lists"],
        "mtet_per_s": 12582912 * a.steps / res["elapsed"] / 1e6,
        "clocks": res["clocks"],
    }
    if workloads is not None:
        out["workloads"] = workloads
    if "extras" in res:
        out["extras"] = res["extras"]
        w = res["extras"].get("walk_counts", {}).get("hull" if a.hull else "bbox")
        if w:
            # the forward's per-entry reject tests: overhead, not algorithmic
            # work (the roofline counts fragments); counts of one untimed
            # TTS_FLAG_COUNT step over the timed forward's mean duration
            fwd_s = st["blend_fwd"] / 1e3
            out["reject_tests"] = {
                "entries_tested": 32 * w["fwd_groups"], "candidates_staged": w["fwd_candidates"],
                "blended": w.get("blended"), "entries_tested_per_s": 32 * w["fwd_groups"] / fwd_s,
                "candidates_per_s": w["fwd_candidates"] / fwd_s,
                "note": "bbox tests of list entries (groups of 32) and candidates the forward "
                        "staged; their chord tests at the block's pixels are overhead"}
    if "e2e" in res:
        out["e2e"] = res["e2e"]
    if "e2e_resident" in res:
        out["e2e_resident"] = res["e2e_resident"]
    if not a.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(a, res["sc"])
        out["cpu_baseline"]["configs"] = cpu_configs(a, res["sc"])
    print(json.dumps(out))


if __name__ == "__main__":
    main()
