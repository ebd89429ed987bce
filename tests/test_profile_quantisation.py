"""The quantised cubic CDF of step (b) (reading R3: F(u) = 1/2 + u (3/4 - u^2/4)
on u in (-1, 1), scaled by ONE = 4096 and rounded to the nearest integer) stays
in [0, ONE] for every binary32 u when each step is one round-to-nearest binary32
operation in the written order; the device code relies on it and applies no
clamp.  numpy's float32 arithmetic is that sequence (one IEEE operation per
step, no contraction).  The extremes lie next to -1 and 1: every binary32 value
in the last 2^22 representable steps below 1 and above -1 is checked, and a
seeded sample of the rest of the interval.  (An exhaustive run over every u in
(-1, 1), about 2.1e9 values, takes about a minute in C and found the same.)"""
import numpy as np

ONE = 4096


def _q(u: np.ndarray) -> np.ndarray:
    u = u.astype(np.float32)
    a = u * u
    b = np.float32(0.25) * a
    c = np.float32(0.75) - b
    d = u * c
    F = np.float32(0.5) + d
    s = F * np.float32(ONE)
    return np.rint(s).astype(np.int64)          # round half to even, as cvt.rni


def _below_one(count: int) -> np.ndarray:
    """The `count` largest binary32 values below 1."""
    top = np.float32(1.0).view(np.int32)
    return (top - np.arange(1, count + 1, dtype=np.int32)).view(np.float32)


def test_quantised_cdf_in_range_next_to_the_ends():
    near = _below_one(1 << 22)
    assert near.min() > 0.0 and near.max() < 1.0
    for u in (near, -near):
        q = _q(u)
        assert q.min() >= 0 and q.max() <= ONE
    # the ends are reached: ONE just below 1, 0 just above -1
    assert _q(near[:1])[0] == ONE and _q(-near[:1])[0] == 0


def test_quantised_cdf_in_range_on_a_sample():
    rng = np.random.default_rng(20241219)
    u = rng.uniform(-1.0, 1.0, 4_000_000).astype(np.float32)
    u = u[(u > -1.0) & (u < 1.0)]
    q = _q(u)
    assert q.min() >= 0 and q.max() <= ONE


def test_quantised_cdf_monotone_across_window_edges():
    """Adjacent binary32 u may give q one unit out of order (rounding of c in
    u * c), but the edges of a fill window are at least dz / (sqrt(5) sigma_max)
    = 0.25 / (sqrt(5) 10) = 0.01118 apart in u (0.0111 here, below that with
    room for the rounding of the edges), and at that distance q never
    decreases: the window's per-bin weights Q_{i+1} - Q_i are never negative."""
    rng = np.random.default_rng(5)
    u = rng.uniform(-1.0, 1.0 - 0.0111, 4_000_000).astype(np.float32)
    v = (u + np.float32(0.0111)).astype(np.float32)
    keep = (u > -1.0) & (v < 1.0)
    assert np.all(_q(v[keep]) >= _q(u[keep]))
    # and next to the ends, where F is flattest
    near = _below_one(1 << 16)
    for lo in (-near, near - np.float32(0.0111)):
        lo = lo[(lo > -1.0) & (lo + np.float32(0.0111) < 1.0)]
        assert np.all(_q(lo + np.float32(0.0111)) >= _q(lo))


def test_quantised_cdf_values_at_simple_points():
    u = np.array([0.0, 0.5, -0.5], np.float32)
    # F(0) = 1/2, F(1/2) = 1/2 + 1/2 (3/4 - 1/16) = 27/32, F(-1/2) = 5/32
    assert list(_q(u)) == [ONE // 2, 27 * ONE // 32, 5 * ONE // 32]
