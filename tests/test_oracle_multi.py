"""Pins of the GPU-flavour multi-vertex fit in the oracle (Sec. 3.5, weight
w_ij with competing vertices at their seeds, |dz| < 0.5 um rule, duplicate
removal; readings R12-R15 in oracle/pv_oracle.c).

The weight's constants are pinned through closed forms at chi2 = 0: alone, a
track has w = 1 / (1 + exp(-chi2_cut / 2)); with a competing seed that also
fits it exactly, w = 1 / (2 + exp(-chi2_cut / 2)).  Both fix ndof = 2 sum w - 3
of a noise-free vertex."""
import math

import numpy as np

import oracle
from paper_2412_14966_gb300 import synthetic

M = oracle.default_mv_params()
W_ALONE = 1.0 / (1.0 + math.exp(-M.chi2_cut / 2))
W_PAIR = 1.0 / (2.0 + math.exp(-M.chi2_cut / 2))


def _exact_vertex(rng, P, n, cov_xx=1e-3, min_slope=0.0):
    """Noise-free tracks through P whose states are exactly representable
    (slopes of magnitude at least min_slope in x and y)."""
    mag = rng.uniform(min_slope, 0.3, (n, 2)) * rng.choice([-1.0, 1.0], (n, 2))
    slopes = np.round(mag * 256) / 256
    d = np.round(rng.uniform(-8, 8, n) * 64) / 64
    return synthetic.straight_tracks(P, slopes, P[2] + d, cov_xx=cov_xx)


def _seeds(zs, xs=None, ys=None, cap=64):
    K = len(zs)
    f = {k: np.zeros((1, cap), np.float32) for k in ("x", "y", "z")}
    f["z"][0, :K] = zs
    if xs is not None:
        f["x"][0, :K] = xs
        f["y"][0, :K] = ys
    f["n"] = np.array([K], np.int32)
    return f


def _run(events_tracks, seeds, m=None, p=None):
    batch = synthetic.batch_from_events([events_tracks])
    return oracle.mv_fit_batch(batch, seeds, p or oracle.default_params(), m or M)


def _P(x, y, z):
    return (float(np.float32(x)), float(np.float32(y)), float(np.float32(z)))


def test_isolated_noise_free_vertex_weights_and_position():
    rng = np.random.default_rng(1)
    P = _P(0.0125, -0.0075, 23.5)
    t = _exact_vertex(rng, P, 12)
    r = _run(t, _seeds([P[2] + 0.08]))
    assert r["status"][0, 0] & oracle.CONVERGED
    np.testing.assert_allclose([r["x"][0, 0], r["y"][0, 0], r["z"][0, 0]], P, atol=1e-6)
    assert r["n_tracks"][0, 0] == 12
    # every track at chi2 = 0 with no competitor: w = 1 / (1 + e^{-chi2_cut/2})
    assert abs(r["ndof"][0, 0] - (2 * 12 * W_ALONE - 3)) < 1e-6
    assert np.all(r["track_vertex"] == 0)
    assert r["status"][0, 0] & oracle.ACCEPTED


def test_constant_weights_give_the_weighted_least_squares_covariance():
    """At convergence on noise-free tracks every weight is W_ALONE, so
    C = (W_ALONE * A^T A)^{-1} for the whitened design matrix A."""
    rng = np.random.default_rng(2)
    P = _P(0.0, 0.0, -12.25)
    t = _exact_vertex(rng, P, 9, cov_xx=4e-4)
    r = _run(t, _seeds([P[2]]))
    rows = []
    for i in range(9):
        d = P[2] - float(t["z"][i])
        vxx = float(t["cxx"][i]) + d * d * float(t["ctxtx"][i])
        vyy = float(t["cyy"][i]) + d * d * float(t["ctyty"][i])
        rows.append(np.array([-1.0, 0.0, float(t["tx"][i])]) / math.sqrt(vxx))
        rows.append(np.array([0.0, -1.0, float(t["ty"][i])]) / math.sqrt(vyy))
    A = np.array(rows)
    C = np.linalg.inv(W_ALONE * A.T @ A)
    got = r["cov"][0, 0]
    want = np.array([C[0, 0], C[0, 1], C[1, 1], C[0, 2], C[1, 2], C[2, 2]])
    np.testing.assert_allclose(got, want, rtol=1e-6, atol=1e-14)


def test_two_seeds_on_one_point_share_every_track_and_one_is_a_duplicate():
    """Both seeds fit every track exactly: w = 1 / (2 + e^{-chi2_cut/2}) < 0.5,
    so neither vertex keeps a track; the second is rejected as a duplicate of
    the first (equal track counts keep the earlier one, R15)."""
    rng = np.random.default_rng(3)
    P = _P(0.0, 0.0, 5.0)
    t = _exact_vertex(rng, P, 10)
    r = _run(t, _seeds([P[2], P[2]]))
    for k in range(2):
        assert abs(r["ndof"][0, k] - (2 * 10 * W_PAIR - 3)) < 1e-6
        assert r["n_tracks"][0, k] == 0
    assert not r["status"][0, 0] & oracle.DUPLICATE
    assert r["status"][0, 0] & oracle.REJ_NTRK
    assert r["status"][0, 1] & oracle.DUPLICATE
    assert not r["status"][0, 1] & oracle.ACCEPTED
    assert np.all(r["track_vertex"] == -1)


def test_separated_vertices_fit_like_single_vertices():
    """Vertices 20 mm apart, tracks with slopes of at least 0.05 (so each
    passes more than 1 mm from the other vertex): competitor terms and the
    other vertex's tracks have vanishing weight, so each fit equals the fit of
    its own tracks alone."""
    rng = np.random.default_rng(4)
    P0, P1 = _P(0.01, 0.0, -10.0), _P(-0.01, 0.02, 10.0)
    t0 = _exact_vertex(rng, P0, 8, min_slope=0.05)
    t1 = _exact_vertex(rng, P1, 11, min_slope=0.05)
    both = {k: np.concatenate([t0[k], t1[k]]) for k in t0}
    r = _run(both, _seeds([P0[2] + 0.05, P1[2] - 0.05]))
    a0 = _run(t0, _seeds([P0[2] + 0.05]))
    a1 = _run(t1, _seeds([P1[2] - 0.05]))
    for k, a in ((0, a0), (1, a1)):
        for f in ("x", "y", "z"):
            assert abs(r[f][0, k] - a[f][0, 0]) < 1e-9
        np.testing.assert_allclose(r["cov"][0, k], a["cov"][0, 0], rtol=1e-9)
        assert r["n_iter"][0, k] == a["n_iter"][0, 0]
    assert np.array_equal(r["track_vertex"], np.r_[np.zeros(8), np.ones(11)].astype(np.int32))
    assert np.all(r["status"][0, :2] & oracle.ACCEPTED)


def test_duplicate_rule_keeps_the_vertex_with_more_tracks():
    """Two noisy vertices 60 um apart in z (far inside 5 sigma): the one with
    fewer tracks is rejected; 30 mm apart: both are kept."""
    rng = np.random.default_rng(5)
    def noisy(P, n):
        t = _exact_vertex(rng, P, n, cov_xx=0.03 ** 2)
        t["x"] = (t["x"] + rng.normal(0, 0.03, n)).astype(np.float32)
        t["y"] = (t["y"] + rng.normal(0, 0.03, n)).astype(np.float32)
        return t
    A, B = _P(0.0, 0.0, 1.0), _P(0.0, 0.0, 1.06)
    ta, tb = noisy(A, 6), noisy(B, 14)
    both = {k: np.concatenate([ta[k], tb[k]]) for k in ta}
    r = _run(both, _seeds([A[2], B[2]]))
    dz = r["z"][0, 1] - r["z"][0, 0]
    assert dz * dz < 25 * (r["cov"][0, 0, 5] + r["cov"][0, 1, 5])
    small, large = (0, 1) if r["n_tracks"][0, 0] < r["n_tracks"][0, 1] else (1, 0)
    assert r["status"][0, small] & oracle.DUPLICATE
    assert not r["status"][0, large] & oracle.DUPLICATE
    far = {k: np.concatenate([ta[k], noisy(_P(0.0, 0.0, 31.0), 14)[k]]) for k in ta}
    r2 = _run(far, _seeds([A[2], 31.0]))
    assert not np.any(r2["status"][0, :2] & oracle.DUPLICATE)


def test_stop_rule_looks_at_dz_only():
    """R13: the GPU rule stops on |dz| < 0.5 um alone.  A tolerance of 0.5 um
    stops no later than the tight one, and a larger dz tolerance never adds
    iterations."""
    rng = np.random.default_rng(6)
    P = _P(0.0, 0.0, 0.0)
    t = _exact_vertex(rng, P, 10, cov_xx=0.03 ** 2)
    t["x"] = (t["x"] + rng.normal(0, 0.03, 10)).astype(np.float32)
    t["y"] = (t["y"] + rng.normal(0, 0.03, 10)).astype(np.float32)
    iters = [_run(t, _seeds([0.3]), oracle.default_mv_params(dz_tol=tol, max_iter=100))["n_iter"][0, 0]
             for tol in (1e-1, 1e-2, 0.5e-3, 1e-6, 1e-9)]
    assert iters == sorted(iters)
    tight = _run(t, _seeds([0.3]), oracle.default_mv_params(dz_tol=1e-12, max_iter=200))
    std = _run(t, _seeds([0.3]))
    assert abs(std["z"][0, 0] - tight["z"][0, 0]) < 0.5e-3


def test_permutation_and_translation_invariance():
    rng = np.random.default_rng(7)
    P0, P1 = _P(0.0, 0.01, -3.0), _P(0.02, 0.0, -2.2)
    def noisy(P, n):
        t = _exact_vertex(rng, P, n, cov_xx=0.02 ** 2)
        t["x"] = (t["x"] + rng.normal(0, 0.02, n)).astype(np.float32)
        t["y"] = (t["y"] + rng.normal(0, 0.02, n)).astype(np.float32)
        return t
    t = {k: np.concatenate([noisy(P0, 9)[k], noisy(P1, 7)[k]]) for k in ("x", "y", "z", "tx", "ty",
                                                                        "cxx", "cxtx", "ctxtx",
                                                                        "cyy", "cyty", "ctyty")}
    s = _seeds([-3.05, -2.15])
    r = _run(t, s)
    perm = rng.permutation(len(t["x"]))
    rp = _run({k: v[perm] for k, v in t.items()}, s)
    for f in ("x", "y", "z"):
        np.testing.assert_allclose(rp[f][0, :2], r[f][0, :2], atol=1e-12)
    assert np.array_equal(rp["n_tracks"][0, :2], r["n_tracks"][0, :2])
    assert np.array_equal(rp["track_vertex"], r["track_vertex"][perm])
    # shift everything by (dx, dy, dz) with dz a multiple of a coarse power of
    # two so that the float32 states shift exactly
    dx, dy, dz = 0.25, -0.125, 8.0
    tt = dict(t)
    tt["x"] = (t["x"] + dx).astype(np.float32)
    tt["y"] = (t["y"] + dy).astype(np.float32)
    tt["z"] = (t["z"] + dz).astype(np.float32)
    st = _seeds(np.float32(s["z"][0, :2] + dz), np.float32([dx, dx]), np.float32([dy, dy]))
    p = oracle.default_params(x_b=dx, y_b=dy)
    rt = _run(tt, st, p=p)
    for f, d in (("x", dx), ("y", dy), ("z", dz)):
        np.testing.assert_allclose(rt[f][0, :2] - d, r[f][0, :2], atol=2e-6)


def test_first_step_onto_the_common_point_stops_at_once():
    """Noise-free tracks and a seed displaced in x only: whatever the weights,
    the weighted least-squares point of tracks through P is P, so the first
    step lands on P with dz = 0 while dchi2 is large; the GPU rule (R13, no
    dchi2 condition) stops after that one iteration."""
    rng = np.random.default_rng(8)
    P = _P(0.0, 0.0, 7.5)
    t = _exact_vertex(rng, P, 10, cov_xx=1e-4)
    r = _run(t, _seeds([P[2]], [0.04], [0.0]))
    assert r["n_iter"][0, 0] == 1
    assert r["status"][0, 0] & oracle.CONVERGED
    np.testing.assert_allclose([r["x"][0, 0], r["y"][0, 0], r["z"][0, 0]], P, atol=1e-7)


def test_track_count_threshold_is_half():
    """R14: a track counts for a vertex from w = 0.5 on.  An extra track about
    2 sigma from a noise-free vertex (chi2 ~ 3.6 < chi2_cut, w ~ 0.55) counts;
    at 2.3 sigma (chi2 > chi2_cut, w < 0.5) it does not."""
    rng = np.random.default_rng(9)
    P = _P(0.0, 0.0, 0.0)
    t = _exact_vertex(rng, P, 10, cov_xx=1e-4, min_slope=0.05)
    counts = []
    for nsig in (2.02, 2.3):
        extra = synthetic.straight_tracks((nsig * 0.01, 0.0, 0.0), [[0.11, -0.13]], [3.0],
                                          cov_xx=1e-4)
        both = {k: np.concatenate([t[k], extra[k]]) for k in t}
        r = _run(both, _seeds([0.0]))
        counts.append(int(r["n_tracks"][0, 0]))
        w_extra = (r["ndof"][0, 0] + 3) / 2 - 10 * W_ALONE     # approximately
        assert (w_extra > 0.5) == (nsig < 2.2), (nsig, w_extra)
    assert counts == [11, 10]


def test_duplicate_separation_is_in_units_of_the_z_variances():
    """R15 compares dz^2 with 25 (C_zz + C_zz'): two poorly measured vertices
    2 mm apart whose summed z variance S satisfies |dz| < 25 S < dz^2 are
    distinct (a rule linear in dz would merge them)."""
    rng = np.random.default_rng(10)
    for trial in range(40):
        def noisy(P, n):
            slopes = rng.uniform(0.15, 0.25, (n, 2)) * rng.choice([-1.0, 1.0], (n, 2))
            tt = synthetic.straight_tracks(P, slopes, P[2] + rng.uniform(-5, 5, n), cov_xx=0.01)
            tt["x"] = (tt["x"] + rng.normal(0, 0.1, n)).astype(np.float32)
            tt["y"] = (tt["y"] + rng.normal(0, 0.1, n)).astype(np.float32)
            return tt
        A, B = _P(0.0, 0.0, 0.0), _P(0.0, 0.0, 2.0)
        ta, tb = noisy(A, 5), noisy(B, 5)
        both = {k: np.concatenate([ta[k], tb[k]]) for k in ta}
        r = _run(both, _seeds([A[2], B[2]]))
        if np.any(r["status"][0, :2] & oracle.SINGULAR):
            continue
        dz = abs(r["z"][0, 1] - r["z"][0, 0])
        S = r["cov"][0, 0, 5] + r["cov"][0, 1, 5]
        if dz < 25 * S < dz * dz:
            assert not np.any(r["status"][0, :2] & oracle.DUPLICATE)
            return
    raise AssertionError("no discriminating configuration found")
