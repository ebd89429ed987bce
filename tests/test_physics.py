"""The physics harness (Sec. 4 figures of merit on synthetic truth): its
matching and counting on hand-made outputs whose answer follows from their
construction, and a statistical sanity check of the oracle's reconstruction
on the nominal workload (pulls of unit width, high efficiency).  CPU only."""
import numpy as np
import pytest

import oracle
from paper_2412_14966_gb300 import physics, synthetic


@pytest.fixture(scope="module")
def batch():
    return synthetic.workload_nominal(n_events=300, seed=31)


def _perfect(batch, sz=0.05, sxy=0.01):
    """One accepted vertex per reconstructible truth PV, at its position."""
    E = batch.n_events
    K = 64
    x = np.zeros((E, K)); y = np.zeros((E, K)); z = np.zeros((E, K))
    cov = np.zeros((E, K, 6)); st = np.zeros((E, K), np.int32); n = np.zeros(E, np.int32)
    for p in range(len(batch.pv_event)):
        if batch.pv_secondary[p]:
            continue
        need = 3 if batch.pv_gas[p] else 4
        if batch.pv_ntracks[p] < need:
            continue
        e = batch.pv_event[p]
        k = n[e]
        x[e, k], y[e, k], z[e, k] = batch.pv_pos[p]
        cov[e, k] = (sxy ** 2, 0.0, sxy ** 2, 0.0, 0.0, sz ** 2)
        st[e, k] = physics.ACCEPTED
        n[e] += 1
    return x, y, z, cov, st, n


def test_perfect_reconstruction(batch):
    x, y, z, cov, st, n = _perfect(batch)
    m = physics.evaluate(batch, x, y, z, cov, st, n)
    assert m["efficiency"] == 1.0 and m["fake_rate"] == 0.0
    assert m["matched"] == m["reconstructible"] == m["reconstructed"]
    assert m["pp"]["resolution_um"] == {"x": 0.0, "y": 0.0, "z": 0.0}


def test_secondaries_and_small_pvs_are_not_reconstructible(batch):
    m = physics.evaluate(batch, *_perfect(batch))
    pp = ~batch.pv_gas & ~batch.pv_secondary
    assert m["reconstructible"] == int((pp & (batch.pv_ntracks >= 4)).sum())
    assert batch.pv_secondary.any()


def test_a_vertex_beyond_five_sigma_is_a_fake(batch):
    x, y, z, cov, st, n = _perfect(batch)
    # an event whose other vertices are far from the first one
    e = next(e for e in range(batch.n_events)
             if n[e] >= 2 and np.min(np.abs(z[e, 1:n[e]] - z[e, 0])) > 1.0)
    z[e, 0] += 5.01 * 0.05                # just beyond 5 sigma_z
    m = physics.evaluate(batch, x, y, z, cov, st, n)
    R = m["reconstructible"]
    assert m["matched"] == R - 1 and m["reconstructed"] == R
    z[e, 0] -= 0.02 * 0.05                # now 4.99 sigma: matched again
    m = physics.evaluate(batch, x, y, z, cov, st, n)
    assert m["matched"] == R and m["fake_rate"] == 0.0


def test_duplicates_keep_the_closest_and_count_the_other_as_fake(batch):
    x, y, z, cov, st, n = _perfect(batch)
    e = int(np.nonzero(n >= 1)[0][0])
    k = n[e]
    x[e, k], y[e, k], z[e, k] = x[e, 0], y[e, 0], z[e, 0] + 0.03
    cov[e, k] = cov[e, 0]
    st[e, k] = physics.ACCEPTED
    n[e] += 1
    m = physics.evaluate(batch, x, y, z, cov, st, n)
    assert m["efficiency"] == 1.0
    assert m["reconstructed"] == m["matched"] + 1
    assert m["pp"]["resolution_um"]["z"] == 0.0      # the exact one was kept


def test_rejected_vertices_are_not_counted(batch):
    x, y, z, cov, st, n = _perfect(batch)
    e = int(np.nonzero(n >= 1)[0][0])
    st[e, 0] = oracle.REJ_BEAM
    m = physics.evaluate(batch, x, y, z, cov, st, n)
    assert m["reconstructed"] == m["reconstructible"] - 1 == m["matched"]


def test_oracle_reconstruction_is_sane_on_the_nominal_workload():
    """Unit-width pulls (the covariance estimates the scatter) and high
    efficiency with a small fake rate on the synthetic pp workload."""
    b = synthetic.workload_nominal(n_events=1500, seed=5)
    p = oracle.default_params()
    ref = oracle.find_batch(b, p)
    fit = oracle.fit_batch(b, ref, p)
    m = physics.evaluate(b, fit["x"], fit["y"], fit["z"], fit["cov"], fit["status"], ref["n"],
                         fit["n_tracks"])
    assert m["efficiency"] > 0.93 and m["fake_rate"] < 0.05, m
    assert m["efficiency_isolated"] > m["efficiency_close"]
    assert m["efficiency_rank"]["1"] > m["efficiency_rank"]["5"]
    for a in "xyz":
        assert 0.85 < m["pp"]["pull_width"][a] < 1.15, m["pp"]
        assert abs(m["pp"]["pull_mean"][a]) < 0.1, m["pp"]
