"""Pins of steps (d2)-(d3): the adaptive vertex fit (Sec. 3.5, Eqs. chi2,
chi2_definition, r_i, H, Newton step, C, deltachisq, tukey; reading R7) and
the final selection."""
import numpy as np
import pytest
from scipy import optimize

import oracle
from paper_2412_14966_gb300 import synthetic
from tests import helpers


def _toy_vertex(rng, n, vtx, res=0.03, outliers=0):
    """n noisy tracks from vtx plus outliers from elsewhere (float32 states)."""
    tx = rng.uniform(-0.3, 0.3, n + outliers)
    ty = rng.uniform(-0.3, 0.3, n + outliers)
    zs = vtx[2] + rng.uniform(-10, 10, n + outliers)
    ox = np.full(n + outliers, vtx[0]); oy = np.full(n + outliers, vtx[1])
    oz = np.full(n + outliers, vtx[2])
    if outliers:
        ox[n:] += rng.normal(0, 0.5, outliers)
        oz[n:] += rng.uniform(-3, 3, outliers)
    cols = {
        "x": ox + tx * (zs - oz) + rng.normal(0, res, n + outliers),
        "y": oy + ty * (zs - oz) + rng.normal(0, res, n + outliers),
        "z": zs, "tx": tx, "ty": ty,
        "cxx": np.full(n + outliers, res * res), "cxtx": np.zeros(n + outliers),
        "ctxtx": np.full(n + outliers, 1e-6),
        "cyy": np.full(n + outliers, res * res), "cyty": np.zeros(n + outliers),
        "ctyty": np.full(n + outliers, 1e-6),
    }
    return {k: np.ascontiguousarray(v.astype(np.float32)) for k, v in cols.items()}


def test_noise_free_tracks_fit_their_common_point():
    rng = np.random.default_rng(1)
    P = (0.012, -0.007, 23.4)
    slopes = np.stack([rng.uniform(-0.3, 0.3, 12), rng.uniform(-0.3, 0.3, 12)], 1)
    # exactly representable states
    slopes = np.round(slopes * 256) / 256
    d = np.round(rng.uniform(-8, 8, 12) * 64) / 64
    Pr = (np.float32(P[0]), np.float32(P[1]), np.float32(P[2]))
    t = synthetic.straight_tracks((float(Pr[0]), float(Pr[1]), float(Pr[2])), slopes,
                                  float(Pr[2]) + d, cov_xx=1e-3)
    r = oracle.fit_tracks(t, (0.0, 0.0, float(Pr[2]) + 0.1), oracle.default_params())
    assert r["status"] & oracle.CONVERGED
    np.testing.assert_allclose(r["x"], [float(Pr[0]), float(Pr[1]), float(Pr[2])], atol=2e-6)
    assert r["n_tracks"] == 12
    assert abs(r["ndof"] - (2 * 12 - 3)) < 1e-3
    assert r["chi2"] < 1e-3


def test_unit_weights_equal_linear_least_squares():
    """With chi2_max -> infinity all weights are 1 and one Newton step is the
    exact linear least-squares solution (Sec. 3.5); compare with lstsq on the
    whitened system and with the covariance (A^T A)^-1."""
    rng = np.random.default_rng(2)
    t = _toy_vertex(rng, 15, (0.01, 0.02, -40.0), outliers=2)
    # correlated position/slope errors make W depend on the sign of z_seed - z_trk
    t["cxtx"] = np.full(len(t["x"]), 2e-5, np.float32)
    t["cyty"] = np.full(len(t["x"]), -1.5e-5, np.float32)
    seed = (0.0, 0.0, -40.2)
    p = oracle.default_params(chi2_max=1e30, max_iter=1, dchi2_tol=1e30, dz_tol=1e30)
    r = oracle.fit_tracks(t, seed, p)
    wx, wy = helpers.track_weights_at(t, np.float64(np.float32(seed[2])))
    x = t["x"].astype(np.float64); y = t["y"].astype(np.float64)
    z = t["z"].astype(np.float64)
    tx = t["tx"].astype(np.float64); ty = t["ty"].astype(np.float64)
    n = len(x)
    # residual rows: x_i + (zv - z_i) tx_i - xv = 0  ->  [-1, 0, tx] a = -(x_i - z_i tx_i)
    A = np.zeros((2 * n, 3)); bvec = np.zeros(2 * n)
    A[:n, 0] = -1; A[:n, 2] = tx; bvec[:n] = -(x - z * tx)
    A[n:, 1] = -1; A[n:, 2] = ty; bvec[n:] = -(y - z * ty)
    sw = np.sqrt(np.concatenate([wx, wy]))
    sol, *_ = np.linalg.lstsq(A * sw[:, None], bvec * sw, rcond=None)
    np.testing.assert_allclose(r["x"], sol, atol=1e-9, rtol=0)
    Cref = np.linalg.inv((A * sw[:, None]).T @ (A * sw[:, None]))
    cov = r["cov"]
    got = np.array([[cov[0], cov[1], cov[3]], [cov[1], cov[2], cov[4]], [cov[3], cov[4], cov[5]]])
    np.testing.assert_allclose(got, Cref, rtol=1e-9, atol=1e-15)
    # chi2 of the new solution is the least-squares minimum (Eq. deltachisq)
    res = (A * sw[:, None]) @ sol - bvec * sw
    assert abs(r["chi2"] - res @ res) < 1e-8 * max(1.0, res @ res)


@pytest.mark.parametrize("seed_id", range(6))
def test_tukey_fixed_point_minimises_robust_objective(seed_id):
    """Run to convergence, the fit sits at a minimum of the Tukey objective
    sum rho(chi2_i), rho' = w (weights frozen at the seed's W, Sec. 3.5):
    brute-force minimisation of that objective finds the same point."""
    rng = np.random.default_rng(100 + seed_id)
    n = int(rng.integers(2, 7))
    vtx = (rng.normal(0, 0.02), rng.normal(0, 0.02), rng.uniform(-50, 50))
    t = _toy_vertex(rng, n, vtx, res=0.02, outliers=int(rng.integers(0, 3)))
    seed = (0.0, 0.0, float(np.float32(vtx[2] + rng.normal(0, 0.05))))
    p = oracle.tight_params()
    r = oracle.fit_tracks(t, seed, p)
    if not (r["status"] & oracle.CONVERGED):
        pytest.skip("fit did not converge on this toy")
    wx, wy = helpers.track_weights_at(t, np.float64(np.float32(seed[2])))

    def obj(a):
        return float(helpers.tukey_rho(helpers.chi2_terms(t, a, wx, wy), p.chi2_max).sum())

    # brute force: dense grid around the seed, then a simplex refinement
    best = None
    for dx in np.linspace(-0.06, 0.06, 13):
        for dy in np.linspace(-0.06, 0.06, 13):
            for dzz in np.linspace(-0.3, 0.3, 13):
                a = (seed[0] + dx, seed[1] + dy, seed[2] + dzz)
                v = obj(a)
                if best is None or v < best[0]:
                    best = (v, a)
    res = optimize.minimize(obj, best[1], method="Nelder-Mead",
                            options={"xatol": 1e-10, "fatol": 1e-14, "maxiter": 20000})
    # the fit's fixed point is a stationary point; it must be the same minimum
    # that brute force finds near the seed (objective values agree) and the
    # position agrees to 0.01 um
    assert obj(r["x"]) <= res.fun + 1e-9
    np.testing.assert_allclose(r["x"], res.x, atol=1e-5)


def test_gradient_vanishes_at_convergence():
    rng = np.random.default_rng(3)
    t = _toy_vertex(rng, 30, (0.0, 0.01, 5.0), outliers=3)
    seed = (0.0, 0.0, 5.05)
    p = oracle.tight_params()
    r = oracle.fit_tracks(t, seed, p)
    wx, wy = helpers.track_weights_at(t, np.float64(np.float32(seed[2])))

    def obj(a):
        return float(helpers.tukey_rho(helpers.chi2_terms(t, a, wx, wy), p.chi2_max).sum())

    # gradient divided by the curvature = distance to the stationary point
    for k in range(3):
        e = np.zeros(3); e[k] = 1e-6
        g = (obj(r["x"] + e) - obj(r["x"] - e)) / 2e-6
        e[k] = 1e-4
        h = (obj(r["x"] + e) - 2 * obj(r["x"]) + obj(r["x"] - e)) / 1e-8
        assert h > 0
        assert abs(g / h) < 1e-7


def test_weights_in_unit_interval_and_counts():
    rng = np.random.default_rng(4)
    t = _toy_vertex(rng, 20, (0.0, 0.0, 0.0), outliers=5)
    r = oracle.fit_tracks(t, (0.0, 0.0, 0.02), oracle.default_params())
    n = len(t["x"])
    assert 0 <= r["n_tracks"] <= n
    # ndof = 2 sum w - 3 with w in [0, 1]
    assert -3 <= r["ndof"] <= 2 * r["n_tracks"] - 3 + 1e-9
    assert r["chi2"] >= -1e-9


def test_covariance_symmetric_positive_definite():
    rng = np.random.default_rng(5)
    t = _toy_vertex(rng, 25, (0.0, 0.0, -100.0))
    r = oracle.fit_tracks(t, (0.0, 0.0, -100.05), oracle.default_params())
    c = r["cov"]
    C = np.array([[c[0], c[1], c[3]], [c[1], c[2], c[4]], [c[3], c[4], c[5]]])
    assert np.all(np.linalg.eigvalsh(C) > 0)


def test_permutation_and_translation():
    rng = np.random.default_rng(6)
    t = _toy_vertex(rng, 25, (0.01, -0.01, 10.0), outliers=2)
    p = oracle.default_params()
    r = oracle.fit_tracks(t, (0.0, 0.0, 10.1), p)
    perm = rng.permutation(len(t["x"]))
    r2 = oracle.fit_tracks({k: np.ascontiguousarray(v[perm]) for k, v in t.items()},
                           (0.0, 0.0, 10.1), p)
    np.testing.assert_allclose(r2["x"], r["x"], atol=1e-12, rtol=0)
    np.testing.assert_allclose(r2["cov"], r["cov"], rtol=1e-10)
    # translate tracks, seed and beam by (dx, dy, dz) with exactly representable shifts
    dx, dy, dz = 0.25, -0.125, 16.0
    t3 = dict(t)
    t3["x"] = (t["x"] + np.float32(dx)).astype(np.float32)
    t3["y"] = (t["y"] + np.float32(dy)).astype(np.float32)
    t3["z"] = (t["z"] + np.float32(dz)).astype(np.float32)
    p3 = oracle.default_params(x_b=dx, y_b=dy)
    r3 = oracle.fit_tracks(t3, (dx, dy, 10.1 + dz), p3)
    np.testing.assert_allclose(r3["x"], r["x"] + np.array([dx, dy, dz]), atol=2e-6)
    assert r3["status"] == r["status"]


def test_pulls_have_unit_width():
    """Statistical sanity of C: (fit - truth) / sqrt(C_ii) ~ N(0, 1)."""
    rng = np.random.default_rng(7)
    pulls = []
    p = oracle.default_params()
    for _ in range(1500):
        vtx = (rng.normal(0, 0.015), rng.normal(0, 0.015), rng.normal(0, 40))
        t = _toy_vertex(rng, 25, vtx, res=0.03)
        r = oracle.fit_tracks(t, (0.0, 0.0, vtx[2] + rng.normal(0, 0.05)), p)
        if not (r["status"] & oracle.CONVERGED):
            continue
        c = r["cov"]
        pulls.append([(r["x"][0] - vtx[0]) / np.sqrt(c[0]),
                      (r["x"][1] - vtx[1]) / np.sqrt(c[2]),
                      (r["x"][2] - vtx[2]) / np.sqrt(c[5])])
    pulls = np.array(pulls)
    assert len(pulls) > 1400
    sd = pulls.std(axis=0)
    mean = pulls.mean(axis=0)
    # Tukey down-weighting of tails makes the pulls slightly wider than 1
    assert np.all(sd > 0.9) and np.all(sd < 1.2), sd
    assert np.all(np.abs(mean) < 0.1), mean


def test_convergence_status_and_iteration_cap():
    rng = np.random.default_rng(8)
    t = _toy_vertex(rng, 20, (0.0, 0.0, 0.0), outliers=4)
    r = oracle.fit_tracks(t, (0.0, 0.0, 0.2), oracle.default_params(max_iter=1))
    assert r["status"] & oracle.MAXITER and r["n_iter"] == 1
    r = oracle.fit_tracks(t, (0.0, 0.0, 0.2), oracle.default_params())
    assert r["status"] & oracle.CONVERGED and 1 <= r["n_iter"] <= 10


def test_convergence_needs_both_conditions():
    """x86 rule of Sec. 3.5: converged only if |dchi2| < 0.01 AND |dz| < 1 um."""
    rng = np.random.default_rng(18)
    t = _toy_vertex(rng, 20, (0.0, 0.0, 0.0), outliers=4)
    seed = (0.0, 0.0, 0.2)
    loose_z = oracle.fit_tracks(t, seed, oracle.default_params(dz_tol=1e30, dchi2_tol=1e-12,
                                                               max_iter=100))
    loose_c = oracle.fit_tracks(t, seed, oracle.default_params(dz_tol=1e-10, dchi2_tol=1e30,
                                                               max_iter=100))
    assert loose_z["n_iter"] > 2 and loose_c["n_iter"] > 2


def test_singular_when_no_track_has_weight():
    rng = np.random.default_rng(9)
    t = _toy_vertex(rng, 5, (0.0, 0.0, 0.0), res=0.001)
    r = oracle.fit_tracks(t, (0.0, 0.0, 5.0), oracle.default_params())  # 5 mm away
    assert r["status"] & oracle.SINGULAR
    assert not (r["status"] & oracle.ACCEPTED)


def test_final_selection():
    """0.3 mm beamline cut for pp vertices only (Sec. 3.5) and the minimal
    track counts 4 (pp) / 3 (gas) of Table smog-pp."""
    p = oracle.default_params()
    slopes = [(0.1, 0.0), (-0.1, 0.05), (0.0, 0.2), (0.2, -0.2), (-0.15, -0.1)]

    def fit_at(vtx, n):
        zs = [vtx[2] + 1.0 + 0.5 * i for i in range(n)]
        t = synthetic.straight_tracks(vtx, slopes[:n], zs, cov_xx=1e-3)
        return oracle.fit_tracks(t, (vtx[0], vtx[1], vtx[2] + 0.01), p)

    assert fit_at((0.29, 0.0, 10.0), 5)["status"] & oracle.ACCEPTED
    r = fit_at((0.31, 0.0, 10.0), 5)
    assert r["status"] & oracle.REJ_BEAM and not r["status"] & oracle.ACCEPTED
    r = fit_at((0.0, 0.0, 10.0), 3)
    assert r["status"] & oracle.REJ_NTRK
    assert fit_at((0.0, 0.0, 10.0), 4)["status"] & oracle.ACCEPTED
    # gas region: no beamline cut, 3 tracks suffice
    assert fit_at((1.0, 0.0, -400.0), 3)["status"] & oracle.ACCEPTED
    assert fit_at((1.0, 0.0, -400.0), 2)["status"] & oracle.REJ_NTRK


def test_tracks_with_non_finite_variance_are_not_used():
    """Reading R10: a track enters the fit only with finite, positive
    extrapolated variances; otherwise the fit is that of the other tracks."""
    rng = np.random.default_rng(19)
    t = _toy_vertex(rng, 12, (0.0, 0.0, 3.0))
    p = oracle.default_params()
    ref = oracle.fit_tracks({k: v[1:] for k, v in t.items()}, (0.0, 0.0, 3.02), p)
    for field, val in (("cyy", np.inf), ("cxx", np.nan), ("cxx", -1.0)):
        bad = {k: v.copy() for k, v in t.items()}
        bad[field][0] = val
        r = oracle.fit_tracks(bad, (0.0, 0.0, 3.02), p)
        np.testing.assert_allclose(r["x"], ref["x"], atol=1e-12)
        assert r["n_tracks"] == ref["n_tracks"]


def test_degenerate_normal_matrix_is_singular():
    """Reading R11: one weighted track, or tracks sharing one direction, leave
    the vertex position along the track undetermined: SINGULAR at the first
    iteration instead of a step along the null direction."""
    p = oracle.default_params()
    one = synthetic.straight_tracks((0.0, 0.0, 5.0), [(0.1, -0.05)], [6.0], cov_xx=1e-3)
    r = oracle.fit_tracks(one, (0.0, 0.0, 5.01), p)
    assert r["status"] & oracle.SINGULAR and r["n_iter"] == 1
    par = synthetic.straight_tracks((0.0, 0.0, 5.0), [(0.1, -0.05)] * 4, [6.0, 7.0, 3.0, 4.0],
                                    cov_xx=1e-3)
    par["x"] = (par["x"] + np.float32([0.0, 0.01, -0.01, 0.02])).astype(np.float32)
    r = oracle.fit_tracks(par, (0.0, 0.0, 5.01), p)
    assert r["status"] & oracle.SINGULAR
    # two tracks at a clear angle are enough
    two = synthetic.straight_tracks((0.0, 0.0, 5.0), [(0.1, -0.05), (-0.2, 0.1)], [6.0, 7.0],
                                    cov_xx=1e-3)
    r = oracle.fit_tracks(two, (0.0, 0.0, 5.01), p)
    assert not (r["status"] & oracle.SINGULAR)
    np.testing.assert_allclose(r["x"], [0.0, 0.0, 5.0], atol=1e-5)
