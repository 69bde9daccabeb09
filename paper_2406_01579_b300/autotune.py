"""Tile-size autotuner.

Times a whole step (pre-filter + forward + backward, or forward only) of the
actual batch for each candidate tile size and keeps the fastest.  Decisions
are cached in a JSON file keyed by the batch shape: the sorted view sizes,
the survivor count (two significant digits) and s.
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
