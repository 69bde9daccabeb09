"""Autotuner of the launch configuration.

Times a whole step (pre-filter + forward + backward, or forward only) of the
actual batch for each candidate and keeps the fastest:

  autotune_tile  the tile size (8, 16, 32);
  autotune       a coordinate search over the tile size (library defaults
                 otherwise), then the backward's list-segment length for the
                 best tile, then the warps per block of the blend kernels,
                 then the backward's per-pixel fragment list capacity (the
                 knobs that change the scheduling, not the result).

The hot path's per-tile depth sort is a comparison (merge) sort, so it has
no digit-width knob.  Decisions are cached in a JSON file (when a path is
given) keyed by the batch shape: the sorted view sizes, the survivor count
(two significant digits), s and the searched knobs.
"""

from __future__ import annotations

import dataclasses
import json
import math
import os

import torch

from .rasterizer import Params, Rasterizer

# No cache file unless the caller names one (here or in TTS_AUTOTUNE_CACHE).
DEFAULT_CACHE = os.environ.get("TTS_AUTOTUNE_CACHE") or None


def _round2(x: int) -> int:
    if x <= 0:
        return 0
    e = int(math.floor(math.log10(x))) - 1
    return int(round(x / 10 ** e) * 10 ** e)


def shape_key(views, n_surv: int, params: Params, with_backward: bool) -> str:
    sizes = sorted((int(c.width), int(c.height)) for c, _ in views)
    return json.dumps({"views": sizes, "surv": _round2(n_surv), "s": round(float(params.s), 3),
                       "bwd": bool(with_backward)}, sort_keys=True)


def _time_step(r: Rasterizer, with_backward: bool, reps: int) -> float:
    out = r._outputs()
    up = (torch.randn(3 * r.total_pixels, device=r.device),
          torch.randn(r.total_pixels, device=r.device), torch.randn(r.total_pixels, device=r.device))
    grads = [(torch.empty_like(s.V), torch.empty_like(s.f), torch.empty_like(s.rgb))
             for s in r.scenes]

    def run():
        if with_backward:
            r.step(out, up, grads)
        else:
            r.prepare()
            r.forward_raw(out)

    for _ in range(2):
        run()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        run()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def autotune_tile(scenes, views, params: Params, candidates=(8, 16, 32), with_backward=True,
                  reps: int = 5, cache_path: str | None = DEFAULT_CACHE):
    """Returns (best tile, {tile: ms per step}).  Uses and updates the cache."""
    probe = Rasterizer(scenes, views, dataclasses.replace(params, tile=16))
    probe.forward()
    n_surv = int(sum(probe.info().n_surv[i] for i in range(len(scenes))))
    key = shape_key(views, n_surv, params, with_backward)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        try:
            cache = json.load(open(cache_path))
        except (OSError, ValueError):
            cache = {}
    if key in cache:
        return int(cache[key]["tile"]), {int(k): v for k, v in cache[key]["ms"].items()}
    times = {}
    for t in candidates:
        p = dataclasses.replace(params, tile=t, forward_only=not with_backward)
        r = Rasterizer(scenes, views, p)
        r.forward()
        r.shrink_to_fit(1.25)
        r.forward()
        times[t] = _time_step(r, with_backward, reps)
        del r
    best = min(times, key=times.get)
    if cache_path:
        cache[key] = {"tile": best, "ms": {str(k): v for k, v in times.items()}}
        os.makedirs(os.path.dirname(cache_path) or ".", exist_ok=True)
        tmp = cache_path + ".tmp"
        with open(tmp, "w") as fh:
            json.dump(cache, fh, indent=1)
        os.replace(tmp, cache_path)
    return best, times


def _load_cache(path):
    if path and os.path.exists(path):
        try:
            return json.load(open(path))
        except (OSError, ValueError):
            return {}
    return {}


def _store_cache(path, cache):
    if not path:
        return
    os.makedirs(os.path.dirname(path) or ".", exist_ok=True)
    tmp = path + ".tmp"
    with open(tmp, "w") as fh:
        json.dump(cache, fh, indent=1)
    os.replace(tmp, path)


def autotune(scenes, views, params: Params, tiles=(8, 16, 32), segments=(128, 256, 512),
             warps=(2, 4, 8), frag_caps=(128, 255, -1), with_backward=True, reps: int = 5,
             cache_path: str | None = DEFAULT_CACHE):
    """Coordinate search of (tile, blend_segment, blend_warps, frag_cap): the
    tile with the library defaults for the others, then the segment length at
    that tile, then the warps per block, then the per-pixel fragment list
    capacity of the backward (-1: none) at all three (forward-only searches
    skip the last).  Returns ({"tile", "blend_segment", "blend_warps",
    "frag_cap"}, {knob: {candidate: ms per step}}).  Uses and updates the
    cache."""
    probe = Rasterizer(scenes, views, dataclasses.replace(params, tile=16))
    probe.forward()
    n_surv = int(sum(probe.info().n_surv[i] for i in range(len(scenes))))
    del probe
    if not with_backward:
        frag_caps = ()
    key = json.dumps({"shape": shape_key(views, n_surv, params, with_backward),
                      "tiles": list(tiles), "segments": list(segments), "warps": list(warps),
                      "frag_caps": list(frag_caps)}, sort_keys=True)
    cache = _load_cache(cache_path)
    if key in cache:
        c = cache[key]
        return dict(c["best"]), {k: {int(a): b for a, b in v.items()} for k, v in c["ms"].items()}

    def time_cfg(**kw):
        p = dataclasses.replace(params, forward_only=not with_backward, **kw)
        r = Rasterizer(scenes, views, p)
        r.forward()
        r.shrink_to_fit(1.25)
        r.forward()
        t = _time_step(r, with_backward, reps)
        del r
        return t

    best = {"tile": int(params.tile), "blend_segment": 0, "blend_warps": 0,
            "frag_cap": int(params.frag_cap)}
    ms = {"tile": {}, "blend_segment": {}, "blend_warps": {}, "frag_cap": {}}
    for t in tiles:
        ms["tile"][t] = time_cfg(tile=t, blend_segment=0, blend_warps=0)
    best["tile"] = min(ms["tile"], key=ms["tile"].get)
    for g in segments:
        ms["blend_segment"][g] = time_cfg(tile=best["tile"], blend_segment=g, blend_warps=0)
    best["blend_segment"] = min(ms["blend_segment"], key=ms["blend_segment"].get)
    for w in warps:
        ms["blend_warps"][w] = time_cfg(tile=best["tile"], blend_segment=best["blend_segment"],
                                        blend_warps=w)
    best["blend_warps"] = min(ms["blend_warps"], key=ms["blend_warps"].get)
    for fc in frag_caps:
        ms["frag_cap"][fc] = time_cfg(tile=best["tile"], blend_segment=best["blend_segment"],
                                      blend_warps=best["blend_warps"], frag_cap=fc)
    if ms["frag_cap"]:
        best["frag_cap"] = min(ms["frag_cap"], key=ms["frag_cap"].get)
    cache[key] = {"best": best, "ms": {k: {str(a): b for a, b in v.items()} for k, v in ms.items()}}
    _store_cache(cache_path, cache)
    return best, ms
