"""Pins of the oracle's coarse-to-fine pre-filter (App. B.1): survivor bounds
against what Eq. 1 implies for a sphere, and the grid refit against its
closed form."""

import numpy as np
import pytest

import oracle
import synth


@pytest.mark.parametrize("s", [60.0, 175.0, 620.0])
def test_sphere_survivor_bounds(s):
    """A survivor has alpha_max >= 1/255, so sigmoid(-s f_min) >= 1/255, i.e.
    some vertex has f <= ln(254)/s; for f = |x| - r every survivor vertex is
    within r + ln(254)/s + (tet diameter) of the centre.  The tets around the
    extreme points (+-r on each axis) survive, so the bounds reach +-r."""
    n, r = 16, 0.55
    V = synth.grid_vertices(n)
    T = synth.grid_tets(n)
    f = (np.linalg.norm(V.astype(np.float64), axis=1) - r).astype(np.float32)
    surv, _, _ = oracle.prefilter(T, f, oracle.make_params(s=s))
    b = oracle.survivor_bounds(V, T, surv)
    h = 2.0 / n
    outer = r + np.log(254.0) / s + h * np.sqrt(3.0)
    assert (b[3:] >= r).all() and (b[:3] <= -r).all()
    assert (b[3:] <= outer).all() and (b[:3] >= -outer).all()
    # the bounds are attained by survivor vertices
    P = V[T[surv]].reshape(-1, 3)
    for a in range(3):
        assert b[a] in P[:, a] and b[3 + a] in P[:, a]


def test_empty_survivors():
    V = synth.grid_vertices(2)
    T = synth.grid_tets(2)
    b = oracle.survivor_bounds(V, T, np.zeros(0, np.int32))
    assert np.isposinf(b[:3]).all() and np.isneginf(b[3:]).all()
    np.testing.assert_array_equal(oracle.fit_grid(V, [-1] * 3, [1] * 3, b), V)


def test_fit_grid_closed_form():
    V = synth.grid_vertices(4)
    aabb = np.array([-0.3, -0.2, 0.1, 0.5, 0.4, 0.3], np.float32)
    pad = 0.1
    out = oracle.fit_grid(V, [-1.0] * 3, [1.0] * 3, aabb, pad)
    ext = aabb[3:].astype(np.float64) - aabb[:3]
    lo = aabb[:3] - pad * ext
    hi = aabb[3:] + pad * ext
    # corners of the grid box go to the corners of the widened bounds, the
    # centre to the centre, and grid lines stay equally spaced
    assert np.abs(out.min(0) - lo).max() < 1e-15 and np.abs(out.max(0) - hi).max() < 1e-15
    c = np.argmin(np.abs(V.astype(np.float64)).sum(1))
    np.testing.assert_allclose(out[c], 0.5 * (lo + hi), atol=1e-15)
    xs = np.unique(out[:, 0])
    np.testing.assert_allclose(np.diff(xs), (hi[0] - lo[0]) / 4, rtol=1e-12)
    # identity when the bounds equal the grid box
    same = oracle.fit_grid(V, [-1.0] * 3, [1.0] * 3, np.array([-1, -1, -1, 1, 1, 1], np.float32), 0.0)
    np.testing.assert_array_equal(same, V.astype(np.float64))


def test_second_round_is_finer():
    """After the refit the same sphere is covered by smaller tets: more
    survivors, each smaller."""
    n, r, s = 16, 0.35, 175.0
    V = synth.grid_vertices(n)
    T = synth.grid_tets(n)
    sdf = lambda X: (np.linalg.norm(X.astype(np.float64), axis=1) - r).astype(np.float32)
    p = oracle.make_params(s=s)
    surv1, _, _ = oracle.prefilter(T, sdf(V), p)
    b = oracle.survivor_bounds(V, T, surv1)
    V2 = oracle.fit_grid(V, [-1.0] * 3, [1.0] * 3, b, 0.05).astype(np.float32)
    surv2, _, _ = oracle.prefilter(T, sdf(V2), p)
    assert len(surv2) > 2 * len(surv1)
    b2 = oracle.survivor_bounds(V2, T, surv2)
    assert (b2[3:] >= r).all() and (b2[:3] <= -r).all()
