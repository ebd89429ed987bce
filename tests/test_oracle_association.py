"""Pins of step (d1): explicit track-to-cluster association through partition
points and the removal loop (Sec. 3.4, reading R6)."""
import numpy as np

import oracle

P = oracle.default_params()
GAS = oracle.gas_bin(P)


def closest_cluster(c, lo, hi):
    """Index of the cluster closest to bin c (distance to the interval
    [lo, hi] in bins; ties go to the lower cluster)."""
    best, bestd = -1, None
    for k in range(len(lo)):
        d = max(lo[k] - c, 0, c - hi[k])
        if bestd is None or d < bestd:
            best, bestd = k, d
    return best


def test_partition_equals_closest_cluster_bruteforce():
    rng = np.random.default_rng(5)
    for trial in range(200):
        K = int(rng.integers(1, 9))
        starts = np.sort(rng.choice(np.arange(1100, 3300, 7), K, replace=False))
        lo = starts
        hi = starts + rng.integers(0, 6, K)
        binmax = lo + (hi - lo) // 2
        # enough tracks everywhere so nothing is removed
        center = np.concatenate([np.repeat(binmax, 5), rng.integers(1000, 3400, 60)])
        r = oracle.associate_bins(center, lo, hi, binmax, P)
        assert r["n"] == K and r["keep"].all()
        for t, c in enumerate(center):
            assert r["cluster"][t] == closest_cluster(int(c), lo, hi), (trial, t, c)


def test_unfilled_tracks_never_assigned():
    lo = np.array([1500, 2000]); hi = lo + 2; bm = lo + 1
    center = np.array([-1, 1501, 1501, 1501, 2001, 2001, 2001, -1])
    r = oracle.associate_bins(center, lo, hi, bm, P)
    assert r["cluster"][0] == -1 and r["cluster"][-1] == -1
    assert list(r["cluster"][1:-1]) == [0, 0, 0, 1, 1, 1]


def test_small_cluster_between_two_large_is_absorbed():
    """A cluster with fewer than 3 tracks (pp) is removed and its tracks go to
    the neighbours by the new partition point."""
    lo = np.array([2000, 2010, 2020]); hi = lo + 2; bm = lo + 1
    center = np.array([2001] * 5 + [2011, 2012] + [2021] * 5 + [2017])
    r = oracle.associate_bins(center, lo, hi, bm, P)
    assert r["n"] == 2 and list(r["keep"]) == [True, False, True]
    # new partition point between clusters 0 and 2: floor((2002 + 2020) / 2) = 2011
    exp = [0] * 5 + [0, 1] + [1] * 5 + [1]
    assert list(r["cluster"]) == exp


def test_gas_cluster_keeps_two_tracks():
    """2 tracks suffice below z = -300 mm (SMOG2 region), not above."""
    lo = np.array([500, 2000]); hi = lo + 2; bm = lo + 1
    center = np.array([501, 501, 2001, 2001] + [2501] * 6)
    lo = np.append(lo, 2500); hi = np.append(hi, 2502); bm = np.append(bm, 2501)
    r = oracle.associate_bins(center, lo, hi, bm, P)
    assert list(r["keep"]) == [True, False, True]


def test_fewest_tracks_removed_first_then_recount():
    """Only one cluster is removed per pass: the one with fewest tracks.
    After its tracks move, a neighbour may reach the threshold."""
    lo = np.array([2000, 2006, 2030]); hi = lo.copy(); bm = lo.copy()
    # cluster 0: 2 tracks, cluster 1: 1 track, cluster 2: 5 tracks
    center = np.array([2000, 2000, 2006] + [2030] * 5)
    r = oracle.associate_bins(center, lo, hi, bm, P)
    # pass 1 removes cluster 1 (1 track); its track then joins cluster 0,
    # which reaches 3 tracks and survives
    assert list(r["keep"]) == [True, False, True]
    assert list(r["cluster"]) == [0, 0, 0] + [1] * 5


def test_tie_removes_lowest_z():
    lo = np.array([2000, 2100, 2200]); hi = lo.copy(); bm = lo.copy()
    center = np.array([2000, 2000, 2100, 2100] + [2200] * 5)
    r = oracle.associate_bins(center, lo, hi, bm, P)
    # clusters 0 and 1 both have 2 tracks: cluster 0 goes first; then its
    # tracks join cluster 1, which reaches 4 and survives
    assert list(r["keep"]) == [False, True, True]


def test_everything_removed():
    lo = np.array([2000, 2100]); hi = lo.copy(); bm = lo.copy()
    center = np.array([2000, 2100])
    r = oracle.associate_bins(center, lo, hi, bm, P)
    assert r["n"] == 0 and list(r["cluster"]) == [-1, -1]


def test_batch_assignment_consistent_with_seeds():
    """On real events every filled track is assigned, every surviving cluster
    has enough tracks, and the mapping matches the closest-cluster rule."""
    from paper_2412_14966_gb300 import synthetic
    b = synthetic.workload_small(n_events=10)
    f = oracle.find_batch(b, P)
    prep = oracle.prepare_f32(b.tracks, P)
    for e in range(10):
        sl = slice(b.offsets[e], b.offsets[e + 1])
        n = f["n"][e]
        tc = f["track_cluster"][sl]
        filled = prep["filled"][sl] > 0
        if n > 0:
            assert (tc[filled] >= 0).all()
        assert (tc[~filled] == -1).all()
        lo, hi = f["lo"][e, :n], f["hi"][e, :n]
        for k in range(n):
            need = P.min_assoc_gas if f["bin"][e, k] < GAS else P.min_assoc_pp
            assert (tc == k).sum() >= need
        for t in np.nonzero(filled)[0]:
            assert tc[t] == closest_cluster(int(prep["center"][sl][t]), lo, hi)
