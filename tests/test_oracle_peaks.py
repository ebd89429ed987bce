"""Pins of step (c): proto-clusters, dip splitting and the seed position
(Sec. 3.3, readings R4, R5, R9) on hand-built histograms whose answer follows
from their construction."""
import numpy as np
import pytest

import oracle

ONE = oracle.ONE
P = oracle.default_params()
NB = oracle.num_bins(P)


def hist_with(values_at: dict) -> np.ndarray:
    h = np.zeros(NB, np.uint32)
    for b, v in values_at.items():
        h[b] = v
    return h


def zmid(i):
    return P.z_min + (i + 0.5) * P.dz


def place(start, values):
    return {start + k: v for k, v in enumerate(values)}


def test_single_symmetric_peak():
    h = hist_with(place(2000, [1000, 3000, 5000, 3000, 1000]))
    s = oracle.seeds_from_hist(h, P)
    assert s["n"] == 1
    assert (s["lo"][0], s["hi"][0], s["bin"][0]) == (2000, 2004, 2002)
    assert s["z"][0] == np.float32(zmid(2002))


@pytest.mark.parametrize("frac", [0.25, -0.25, 0.125, -0.375, 0.0])
def test_parabola_vertex_is_recovered(frac):
    """For bin contents on a parabola A - B (j - j0)^2, delta of Sec. 3.3 is the
    exact vertex offset: z_seed = z_min + (j0 + 1/2) dz."""
    i = 2100
    j0 = i + frac
    B = 64
    vals = {}
    for j in range(i - 3, i + 4):
        v = 40000 - B * (j - j0) ** 2
        assert float(v).is_integer()
        vals[j] = int(v)
    s = oracle.seeds_from_hist(hist_with(vals), P)
    assert s["n"] == 1 and s["bin"][0] == i
    assert s["z"][0] == np.float32(P.z_min + (j0 + 0.5) * P.dz)


def test_delta_limits():
    """delta -> +-1/2 as a neighbour approaches the maximum (Sec. 3.3)."""
    s = oracle.seeds_from_hist(hist_with(place(1500, [5000, 20000, 19999, 3000])), P)
    d = (s["z"][0] - zmid(1501)) / P.dz
    assert 0.49 < d <= 0.5
    s = oracle.seeds_from_hist(hist_with(place(1500, [3000, 19999, 20000, 5000])), P)
    d = (s["z"][0] - zmid(1502)) / P.dz
    assert -0.5 <= d < -0.49


def test_deep_dip_splits_two_clusters():
    """Two peaks separated by a dip well below both maxima, each with more than
    2.5 tracks of integral: split at the minimum, which goes to the left piece."""
    vals = [1000, 4000, 8000, 4000, 1500, 4000, 8000, 4000, 1000]
    s = oracle.seeds_from_hist(hist_with(place(2000, vals)), P)
    assert s["n"] == 2
    assert list(s["lo"]) == [2000, 2005]
    assert list(s["hi"]) == [2004, 2008]
    assert list(s["bin"]) == [2002, 2006]


def test_shallow_dip_does_not_split():
    """A dip at >= 80% of the smaller neighbouring maximum is not significant."""
    vals = [1000, 4000, 8000, 7000, 6400, 7000, 8000, 4000, 1000]
    s = oracle.seeds_from_hist(hist_with(place(2000, vals)), P)
    assert s["n"] == 1
    assert (s["lo"][0], s["hi"][0]) == (2000, 2008)
    assert s["bin"][0] == 2002  # lowest index among equal maxima


def test_dip_just_below_ratio_splits():
    vals = [1000, 4000, 8000, 7000, 6399, 7000, 8000, 4000, 1000]
    s = oracle.seeds_from_hist(hist_with(place(2000, vals)), P)
    assert s["n"] == 2


def test_small_side_peak_is_not_split_off():
    """A deep dip but a side piece below the 2.5-track integral: no split
    (Sec. 3.3: splitting only if the seed cluster's track integral is above the
    threshold)."""
    vals = [2000, 6000, 12000, 6000, 1000, 1500, 2500, 1500, 500]
    s = oracle.seeds_from_hist(hist_with(place(2000, vals)), P)
    assert s["n"] == 1
    assert (s["lo"][0], s["hi"][0], s["bin"][0]) == (2000, 2008, 2002)


def test_low_integral_cluster_dropped_and_gas_threshold():
    """A cluster with 2 tracks of integral is dropped in the pp region (< 2.5)
    but kept in the gas region (>= 1.75), Table smog-pp."""
    two_tracks = [1000, 3000, 2192, 1000, 1000]     # sums to 8192 = 2 tracks
    assert sum(two_tracks) == 2 * ONE
    s = oracle.seeds_from_hist(hist_with(place(2500, two_tracks)), P)
    assert s["n"] == 0
    s = oracle.seeds_from_hist(hist_with(place(500, two_tracks)), P)
    assert s["n"] == 1 and s["bin"][0] == 501


def test_threshold_is_strict_and_separates_proto_clusters():
    """Proto-clusters are maximal runs of bins strictly above the threshold;
    a bin equal to it separates them.  Seeds come out z-ordered."""
    thr = P.bin_threshold
    vals = [3000, 9000, 3000, thr, 3000, 9000, 3000]
    s = oracle.seeds_from_hist(hist_with(place(1200, vals)), P)
    assert s["n"] == 2
    assert list(s["lo"]) == [1200, 1204] and list(s["hi"]) == [1202, 1206]
    vals[3] = thr + 1
    s = oracle.seeds_from_hist(hist_with(place(1200, vals)), P)
    # now one proto-cluster with a deep dip at the middle bin: split there
    assert s["n"] == 2
    assert list(s["hi"]) == [1203, 1206]


def test_peaks_two_bins_apart_are_separable():
    """The minimal peak distance is two bins (Sec. 3.2)."""
    vals = [4000, 12000, 2000, 12000, 4000]
    s = oracle.seeds_from_hist(hist_with(place(2000, vals)), P)
    assert s["n"] == 2 and list(s["bin"]) == [2001, 2003]


def test_plateau_minimum_leftmost_goes_left():
    vals = [3000, 12000, 3000, 1000, 1000, 1000, 3000, 12000, 3000]
    s = oracle.seeds_from_hist(hist_with(place(2000, vals)), P)
    assert s["n"] == 2
    assert list(s["hi"]) == [2003, 2008] and list(s["lo"]) == [2000, 2004]


def test_three_peaks_walk_in_z_order():
    """The first dip splits off the first peak; the small middle peak cannot
    stand alone at the second dip, so it stays with the last peak."""
    vals = [3000, 12000, 3000, 300, 3000, 4000, 300, 3000, 12000, 3000]
    s = oracle.seeds_from_hist(hist_with(place(2000, vals)), P)
    # dip 2003: left 18300 and right 25300 are both >= 10240 -> split;
    # dip 2006: left piece [2004, 2006] = 7300 < 10240 -> no split
    assert s["n"] == 2
    assert list(s["lo"]) == [2000, 2004]
    assert list(s["hi"]) == [2003, 2009]
    assert list(s["bin"]) == [2001, 2008]


def test_split_integral_includes_the_minimum_bin():
    """The left piece [start, m] holds the minimum bin: its integral is tested
    with it.  Here the left piece reaches exactly 2.5 tracks only with it."""
    left = [2000, 5000, 2240, 1000]            # 10240 = 2.5 * ONE with the minimum
    assert sum(left) == 10240
    vals = left + [4000, 9000, 4000]
    s = oracle.seeds_from_hist(hist_with(place(2000, vals)), P)
    assert s["n"] == 2 and list(s["hi"]) == [2003, 2006]
    # and the right piece is tested without it: exactly 2.5 tracks after it
    vals = [4000, 9000, 4000, 1000] + [2000, 5240, 3000]
    assert sum(vals[4:]) == 10240
    s = oracle.seeds_from_hist(hist_with(place(2000, vals)), P)
    assert s["n"] == 2 and list(s["lo"]) == [2000, 2004]
    vals[5] -= 1
    assert oracle.seeds_from_hist(hist_with(place(2000, vals)), P)["n"] == 1


def test_left_maximum_restarts_after_a_split():
    """After a split the open piece's maximum is the peak right of the split,
    so a later dip is judged against it, not against the earlier peak."""
    vals = [3000, 6000, 3000, 1000, 8000, 20000, 12000, 20000, 8000, 3000]
    s = oracle.seeds_from_hist(hist_with(place(2000, vals)), P)
    assert s["n"] == 3
    assert list(s["lo"]) == [2000, 2004, 2007]
    assert list(s["hi"]) == [2003, 2006, 2009]


def _split_reference(N, a, b, p, gas_bin):
    """Second formulation of reading R5: compress plateaus into runs, list the
    alternating extrema, then walk the minima in z order."""
    runs = []  # (value, first bin)
    for i in range(a, b + 1):
        if runs and runs[-1][0] == N[i]:
            continue
        runs.append((int(N[i]), i))
    vals = [r[0] for r in runs]
    mins, maxs = [], []
    for k in range(len(runs)):
        left = vals[k - 1] if k > 0 else -1
        right = vals[k + 1] if k + 1 < len(runs) else -1
        if vals[k] > left and vals[k] > right:
            maxs.append(k)
        elif vals[k] < left and vals[k] < right and k > 0 and k + 1 < len(runs):
            mins.append(k)
    pieces = []
    s = a
    first_max = maxs[0]
    L = vals[first_max]
    for mk in mins:
        nxt = min(x for x in maxs if x > mk)
        R = vals[nxt]
        m = runs[mk][1]
        T = int(round((p.min_integral_gas if m < gas_bin else p.min_integral_pp) * ONE))
        if (int(p.dip_den) * int(N[m]) < int(p.dip_num) * min(L, R)
                and int(N[s:m + 1].astype(np.int64).sum()) >= T
                and int(N[m + 1:b + 1].astype(np.int64).sum()) >= T):
            pieces.append((s, m))
            s = m + 1
            L = R
        else:
            L = max(L, R)
    pieces.append((s, b))
    return pieces


def _seeds_reference(N, p):
    gas_bin = oracle.gas_bin(p)
    out = []
    i = 0
    while i < len(N):
        if N[i] > p.bin_threshold:
            a = i
            while i + 1 < len(N) and N[i + 1] > p.bin_threshold:
                i += 1
            for lo, hi in _split_reference(N, a, i, p, gas_bin):
                im = lo + int(np.argmax(N[lo:hi + 1]))
                T = int(round((p.min_integral_gas if im < gas_bin else p.min_integral_pp) * ONE))
                if int(N[lo:hi + 1].astype(np.int64).sum()) >= T:
                    out.append((lo, hi, im))
        i += 1
    return out


def test_random_histograms_against_extrema_formulation():
    """Random wiggly histograms (sums of bumps with noise and plateaus)."""
    rng = np.random.default_rng(21)
    for trial in range(300):
        N = np.zeros(NB, np.int64)
        for _ in range(rng.integers(1, 8)):
            c = rng.integers(20, NB - 20)
            w = rng.integers(1, 6)
            amp = rng.integers(500, 20000)
            for j in range(c - 3 * w, c + 3 * w + 1):
                N[j] += int(amp * np.exp(-0.5 * ((j - c) / w) ** 2))
        noise = rng.integers(-300, 300, NB)
        N = np.maximum(N + np.where(N > 0, noise, 0), 0)
        # plateaus
        k = rng.integers(0, NB - 5)
        N[k:k + 3] = N[k]
        N = N.astype(np.uint32)
        s = oracle.seeds_from_hist(N, P)
        ref = _seeds_reference(N, P)
        got = list(zip(s["lo"].tolist(), s["hi"].tolist(), s["bin"].tolist()))
        assert got == ref, trial
        # invariants: z order, delta in [-1/2, 1/2], disjoint pieces
        for k in range(s["n"]):
            assert s["lo"][k] <= s["bin"][k] <= s["hi"][k]
            d = (float(s["z"][k]) - zmid(int(s["bin"][k]))) / P.dz
            assert -0.5 - 1e-6 <= d <= 0.5 + 1e-6
            if k:
                assert s["hi"][k - 1] < s["lo"][k]
                assert s["z"][k - 1] < s["z"][k]


def test_seed_xy_on_beamline():
    p = oracle.default_params(x_b=0.5, y_b=-0.25, tx_b=1e-3, ty_b=-2e-3)
    h = hist_with(place(2000, [1000, 3000, 9000, 3000, 1000]))
    from paper_2412_14966_gb300 import synthetic
    # a single-event batch with no tracks cannot carry a histogram, so check
    # the seed z from the histogram and the beam relation on a real event
    b = synthetic.workload_small(n_events=2)
    f = oracle.find_batch(b, p)
    for e in range(2):
        for k in range(f["n"][e]):
            z = f["z"][e, k]
            assert f["x"][e, k] == np.float32(np.float32(0.5) + np.float32(1e-3) * z)
            assert f["y"][e, k] == np.float32(np.float32(-0.25) + np.float32(-2e-3) * z)
    assert oracle.seeds_from_hist(h, p)["n"] == 1


# --- the x86 flavour: recursive splitting (reading R16) ---------------------

P_REC = oracle.default_params(split_mode=1)


def _pieces(h, p):
    s = oracle.seeds_from_hist(h, p)
    return [(int(a), int(b)) for a, b in zip(s["lo"], s["hi"])]


def test_recursive_split_looks_at_the_two_largest_maxima():
    """N = 8000, 6000, 10000, 8000, 10000.  In z order the first dip (6000)
    is significant against min(8000, 10000) (30000 < 32000) and both sides hold
    2.5 tracks, so the GPU flavour splits [0,1] | [2,4]; the dip 8000 between
    the last two maxima is not (40000 < 40000 fails).  The x86 flavour looks
    only between the two largest maxima (bins 2 and 4), finds 8000, and keeps
    one piece."""
    h = hist_with(place(2000, [8000, 6000, 10000, 8000, 10000]))
    assert _pieces(h, P) == [(2000, 2001), (2002, 2004)]
    assert _pieces(h, P_REC) == [(2000, 2004)]


def test_recursive_split_recurses_on_both_sides():
    """N = 4000, 6000, 4000, 6000, 2000, 10000, 300, 4000.  The two largest
    maxima are 10000 (bin 5) and the first 6000 (bin 1, lower position on the
    tie); the smallest bin between them is 2000 (bin 4): significant and both
    sides hold 2.5 tracks (22000 and 14300), so split after bin 4.  Left
    [0,4]: maxima 6000 at bins 1 and 3, minimum 4000 between, significant but
    the right side (6000 + 2000) is below 2.5 tracks: no split.  Right [5,7]:
    maxima 10000 and 4000, dip 300, right side 4000 too small: no split."""
    h = hist_with(place(2000, [4000, 6000, 4000, 6000, 2000, 10000, 300, 4000]))
    assert _pieces(h, P_REC) == [(2000, 2004), (2005, 2007)]
    assert _pieces(h, P) == [(2000, 2002), (2003, 2007)]


def test_recursive_split_agrees_on_single_peaks_and_clear_pairs():
    """One maximum: one piece in both flavours; two well separated maxima with
    a deep dip: the same split in both."""
    one = hist_with(place(3000, [1000, 3000, 6000, 9000, 6000, 3000, 1000]))
    assert _pieces(one, P_REC) == _pieces(one, P) == [(3000, 3006)]
    two = hist_with(place(3000, [2000, 6000, 12000, 6000, 1000, 6000, 12000, 6000, 2000]))
    assert _pieces(two, P_REC) == _pieces(two, P) == [(3000, 3004), (3005, 3008)]


def test_recursive_split_splits_each_side_again():
    """Three equal peaks with deep dips: the first split lies between the
    first two maxima (equal values: lower positions first), and the right side
    is split again between its two maxima; both flavours give three pieces."""
    h = hist_with(place(2000, [2000, 6000, 12000, 6000, 1000, 6000, 12000, 6000, 1500, 6000, 12000,
                               6000, 2000]))
    want = [(2000, 2004), (2005, 2008), (2009, 2012)]
    assert _pieces(h, P_REC) == want
    assert _pieces(h, P) == want
