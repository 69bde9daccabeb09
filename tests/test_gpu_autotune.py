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
