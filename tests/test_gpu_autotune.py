"""The tile-size autotuner times each candidate on the real batch, returns a
candidate, and answers later calls for the same shape from its JSON cache."""

import json

import numpy as np
import pytest

import synth
from paper_2406_01579_b300 import Params
from paper_2406_01579_b300.autotune import autotune_tile
from parity import to_dev

pytestmark = pytest.mark.gpu


def test_autotune_picks_and_caches(tmp_path):
    sc = to_dev(synth.scene_sphere16())
    rng = np.random.default_rng(2)
    views = [(synth.random_camera(rng, 256, 256), 0) for _ in range(2)]
    cache = str(tmp_path / "tune.json")
    best, times = autotune_tile([sc], views, Params(s=175.0), candidates=(8, 16, 32), reps=2,
                                cache_path=cache)
    assert best in (8, 16, 32) and set(times) == {8, 16, 32}
    assert best == min(times, key=times.get)
    data = json.load(open(cache))
    assert len(data) == 1
    best2, times2 = autotune_tile([sc], views, Params(s=175.0), cache_path=cache)
    assert best2 == best and times2 == times


def test_autotune_searches_segment_and_warps(tmp_path):
    """The coordinate search times the tile, then the backward segment and the
    warps per block at the best tile; the picked configuration renders the
    same image as the defaults (the knobs only schedule the work)."""
    import torch

    from paper_2406_01579_b300 import Rasterizer
    from paper_2406_01579_b300.autotune import autotune
    sc = to_dev(synth.scene_sphere16())
    rng = np.random.default_rng(4)
    views = [(synth.random_camera(rng, 192, 192), 0) for _ in range(2)]
    cache = str(tmp_path / "tune.json")
    best, ms = autotune([sc], views, Params(s=120.0), tiles=(8, 16), segments=(64, 256),
                        warps=(2, 4, 8), reps=2, cache_path=cache)
    assert set(ms["tile"]) == {8, 16} and set(ms["blend_segment"]) == {64, 256}
    assert set(ms["blend_warps"]) == {2, 4, 8}
    assert best["tile"] == min(ms["tile"], key=ms["tile"].get)
    assert best["blend_warps"] == min(ms["blend_warps"], key=ms["blend_warps"].get)
    again, ms2 = autotune([sc], views, Params(s=120.0), tiles=(8, 16), segments=(64, 256),
                          warps=(2, 4, 8), cache_path=cache)
    assert again == best and ms2 == ms
    ref = Rasterizer([sc], views, Params(s=120.0, tile=best["tile"])).forward()
    got = Rasterizer([sc], views, Params(s=120.0, **best)).forward()
    for a, b in zip(ref, got):
        assert torch.allclose(a, b, atol=1e-6, rtol=0)
