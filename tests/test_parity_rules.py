"""The GPU parity rule for ill-conditioned covariances (tests/gpu_common.py),
checked on the CPU: the oracle's covariance spread under one-ulp moves of the
binary32 inputs is small for well-determined vertices and large only for the
degenerate few-track fits the rule exists for."""
import numpy as np

import oracle
from paper_2412_14966_gb300 import synthetic
from tests import gpu_common as G


def _setup():
    b = synthetic.workload_nominal(n_events=2000, seed=7)
    p = oracle.default_params()
    f = oracle.find_batch(b, p)
    return b, p, f, oracle.fit_batch(b, f, p)


def test_spread_small_for_well_determined_vertices():
    b, p, f, r = _setup()
    spreads = []
    for e in range(0, b.n_events, 16):
        for k in range(f["n"][e]):
            if r["n_tracks"][e, k] >= 10 and not r["status"][e, k] & oracle.SINGULAR:
                spreads.append(G.cov_spread(b, f, p, e, k))
    spreads = np.asarray(spreads)
    assert len(spreads) > 100
    # about one ulp of input moves a typical covariance by a few 1e-6 (a track
    # near chi2_max makes the tail); none reaches the tolerance itself
    assert np.median(spreads) < G.TOL_COV / G.ILL_FACTOR
    assert spreads.max() < G.TOL_COV


def test_spread_large_for_a_degenerate_two_track_fit():
    b, p, f, r = _setup()
    e, k = 170, 2
    assert r["n_tracks"][e, k] == 2 and r["status"][e, k] & oracle.REJ_NTRK
    sp = G.cov_spread(b, f, p, e, k)
    assert sp > G.TOL_COV
    # deterministic: the perturbation draws are seeded by the vertex
    assert G.cov_spread(b, f, p, e, k) == sp


def test_spread_zero_without_perturbation_effect():
    """Noise-free tracks through one point with unit weights: the fit is
    linear least squares, so a one-ulp move of the inputs moves the
    covariance by about one ulp only."""
    rng = np.random.default_rng(3)
    n = 12
    tx, ty = rng.uniform(-0.3, 0.3, n), rng.uniform(-0.3, 0.3, n)
    z = rng.uniform(-5, 5, n)
    v = (0.01, -0.02, 1.5)
    t = {"x": v[0] + tx * (z - v[2]), "y": v[1] + ty * (z - v[2]), "z": z, "tx": tx, "ty": ty,
         "cxx": np.full(n, 1e-4), "cxtx": np.zeros(n), "ctxtx": np.full(n, 1e-8),
         "cyy": np.full(n, 1e-4), "cyty": np.zeros(n), "ctyty": np.full(n, 1e-8)}
    t = {k: np.asarray(a, np.float32) for k, a in t.items()}
    batch = synthetic.batch_from_events([t])
    p = oracle.default_params()
    found = {"x": np.array([[0.0]]), "y": np.array([[0.0]]), "z": np.array([[1.4]]),
             "track_cluster": np.zeros(n, np.int32)}
    assert G.cov_spread(batch, found, p, 0, 0) < 1e-6
