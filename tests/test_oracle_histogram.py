"""Pins of step (b): the per-track profile and the event histogram (Sec. 3.2,
reading R3: cubic CDF of the variance-matched Epanechnikov kernel)."""
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2412_14966_gb300 import synthetic
from tests import helpers

ONE = oracle.ONE


def _edges(first, n, p):
    return [p.z_min + (first + k) * p.dz for k in range(n + 1)]


def test_paper_constants_golden():
    """Default parameters equal the values printed in the paper."""
    with open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")) as f:
        g = json.load(f)
    p = oracle.default_params()
    assert p.z_min == g["histogram_z_min_mm"]["value"]
    assert p.z_max == g["histogram_z_max_mm"]["value"]
    assert p.dz == g["bin_width_mm"]["value"]
    assert math.isclose(p.sigma_max_pp, g["sigma_max_pp_mm"]["value"])
    assert p.sigma_max_gas == g["sigma_max_gas_mm"]["value"]
    assert p.z_gas == g["gas_region_upper_z_mm"]["value"]
    assert p.min_integral_pp == g["min_cluster_integral_pp"]["value"]
    assert p.min_integral_gas == g["min_cluster_integral_gas"]["value"]
    assert p.min_pv_tracks_pp == g["min_tracks_pv_pp"]["value"]
    assert p.min_pv_tracks_gas == g["min_tracks_pv_gas"]["value"]
    assert p.min_assoc_pp == g["min_assoc_tracks_pp"]["value"]
    assert p.min_assoc_gas == g["min_assoc_tracks_gas"]["value"]
    assert p.chi2_max == g["tukey_chi2_max"]["value"]
    assert p.dchi2_tol == g["converge_dchi2"]["value"]
    assert p.dz_tol == g["converge_dz_mm"]["value"]
    assert p.max_iter == g["max_iterations"]["value"]
    assert p.max_r_beam == g["max_beamline_distance_mm"]["value"]
    assert oracle.num_bins(p) == g["n_bins"]["value"]
    assert oracle.gas_bin(p) == 1000


@pytest.mark.parametrize("sigma", [0.02, 0.11, 0.25, 0.6, 1.4, 4.0, 9.5])
def test_profile_sums_to_one_track(sigma):
    """Away from the range ends each track adds exactly ONE (the weights of a
    track add up to unity, Sec. 3.2)."""
    p = oracle.default_params()
    rng = np.random.default_rng(int(sigma * 1000))
    for z in rng.uniform(-400, 200, 50):
        first, w = oracle.track_profile(np.float32(z), np.float32(sigma), p)
        assert int(w.sum()) == ONE
        assert (w >= 0).all()


@pytest.mark.parametrize("sigma", [0.05, 0.2, 0.7, 1.5, 6.0])
def test_profile_equals_kernel_integral(sigma):
    """Each bin's weight is the integral over the bin of the Epanechnikov
    density with variance sigma^2, up to the 1/ONE quantisation at each edge.
    The integral is computed by quadrature, independently of the cubic CDF."""
    p = oracle.default_params()
    rng = np.random.default_rng(7 + int(sigma * 100))
    for z in rng.uniform(-300, 200, 20):
        zf = float(np.float32(z))
        first, w = oracle.track_profile(zf, np.float32(sigma), p)
        e = _edges(first, len(w), p)
        for k in range(len(w)):
            ref = helpers.epanechnikov_bin_integral(e[k], e[k + 1], zf, float(np.float32(sigma)))
            assert abs(w[k] / ONE - ref) <= 1.01 / ONE + 1e-6, (z, k, w[k] / ONE, ref)


@pytest.mark.parametrize("sigma", [0.05, 0.2, 0.7, 1.5])
def test_profile_approximates_gaussian(sigma):
    """The cubic profile approximates the Gaussian bin integrals of Sec. 3.2:
    the variance-matched Epanechnikov CDF is within 0.032 of the normal CDF,
    so a bin differs by at most 2 * 0.032 plus quantisation."""
    p = oracle.default_params()
    for z in (-123.456, 0.1, 17.3):
        zf = float(np.float32(z))
        first, w = oracle.track_profile(zf, np.float32(sigma), p)
        e = _edges(first, len(w), p)
        worst = 0.0
        for k in range(len(w)):
            g = helpers.gaussian_bin_integral(e[k], e[k + 1], zf, float(np.float32(sigma)))
            worst = max(worst, abs(w[k] / ONE - g))
        assert worst < 0.064 + 2.0 / ONE
        # the Gaussian mass outside the window is small
        g_in = helpers.gaussian_bin_integral(e[0], e[-1], zf, float(np.float32(sigma)))
        assert g_in > 0.97


@pytest.mark.parametrize("sigma", [0.3, 0.8, 2.0])
def test_profile_mean_and_variance(sigma):
    """The profile's mean is z_poca and its variance sigma^2 + dz^2/12."""
    p = oracle.default_params()
    zf = float(np.float32(12.3456))
    first, w = oracle.track_profile(zf, np.float32(sigma), p)
    mids = np.array(_edges(first, len(w), p)[:-1]) + 0.5 * p.dz
    m = (w * mids).sum() / ONE
    v = (w * (mids - m) ** 2).sum() / ONE
    assert abs(m - zf) < 0.01 * sigma + 2e-3
    assert abs(v / (sigma ** 2 + p.dz ** 2 / 12) - 1) < 0.02 + 0.01 / sigma


def test_profile_mirror_symmetry_at_bin_centre():
    p = oracle.default_params()
    for i in (400, 2200, 3000):
        zc = p.z_min + (i + 0.5) * p.dz
        for sigma in (0.1, 0.37, 1.2):
            first, w = oracle.track_profile(zc, np.float32(sigma), p)
            assert first + len(w) - 1 - i == i - first
            assert np.abs(w.astype(np.int64) - w[::-1].astype(np.int64)).max() <= 1


def test_profile_narrow_goes_to_one_bin():
    p = oracle.default_params()
    for z in (-10.37, 0.0, 55.55):
        first, w = oracle.track_profile(np.float32(z), np.float32(1e-8), p)
        assert len(w) == 1 and w[0] == ONE
        assert first == int(math.floor((np.float32(z) - p.z_min) / p.dz))


def test_profile_at_range_end_loses_outside_mass():
    """A track near z_max keeps only the mass inside the histogram."""
    p = oracle.default_params()
    first, w = oracle.track_profile(np.float32(299.9), np.float32(0.3), p)
    nb = oracle.num_bins(p)
    inside = [w[k] for k in range(len(w)) if 0 <= first + k < nb]
    outside = [w[k] for k in range(len(w)) if not (0 <= first + k < nb)]
    assert sum(outside) > 0 and sum(inside) + sum(outside) == ONE
    ref = helpers.epanechnikov_bin_integral(p.z_min, p.z_max, float(np.float32(299.9)),
                                            float(np.float32(0.3)))
    assert abs(sum(inside) / ONE - ref) < 1.5 / ONE


def _event_hist(tracks, p):
    b = synthetic.batch_from_events([tracks])
    return oracle.find_batch(b, p, want_hist=True)["hist"][0]


def test_histogram_is_sum_of_track_profiles():
    """The histogram of an event is the bin-wise sum of the filled tracks'
    profiles (with cuts applied per track)."""
    b = synthetic.workload_small(n_events=3)
    p = oracle.default_params()
    f = oracle.find_batch(b, p, want_hist=True)
    prep = oracle.prepare_f32(b.tracks, p)
    nb = oracle.num_bins(p)
    for e in range(3):
        ref = np.zeros(nb, np.int64)
        for t in range(b.offsets[e], b.offsets[e + 1]):
            if not prep["filled"][t]:
                continue
            first, w = oracle.track_profile(prep["zpoca"][t], prep["sigma"][t], p)
            for k, wk in enumerate(w):
                if 0 <= first + k < nb:
                    ref[first + k] += int(wk)
        np.testing.assert_array_equal(f["hist"][e].astype(np.int64), ref)


def test_histogram_total_and_permutation():
    b = synthetic.workload_small(n_events=4)
    p = oracle.default_params()
    f = oracle.find_batch(b, p, want_hist=True)
    prep = oracle.prepare_f32(b.tracks, p)
    for e in range(4):
        sl = slice(b.offsets[e], b.offsets[e + 1])
        n_filled = int(prep["filled"][sl].sum())
        total = int(f["hist"][e].astype(np.int64).sum())
        # every filled track adds ONE unless it sits at a range end
        assert total <= n_filled * ONE
        assert total >= n_filled * ONE - 2 * ONE
    # permutation of tracks inside each event: identical histograms
    rng = np.random.default_rng(3)
    perm = np.concatenate([rng.permutation(np.arange(b.offsets[e], b.offsets[e + 1]))
                           for e in range(4)])
    b2 = synthetic.EventBatch(tracks={k: v[perm] for k, v in b.tracks.items()},
                              offsets=b.offsets, pv_event=b.pv_event, pv_pos=b.pv_pos,
                              pv_ntracks=b.pv_ntracks, pv_secondary=b.pv_secondary,
                              pv_gas=b.pv_gas, track_pv=b.track_pv[perm])
    f2 = oracle.find_batch(b2, p, want_hist=True)
    np.testing.assert_array_equal(f["hist"], f2["hist"])
    np.testing.assert_array_equal(f["z"], f2["z"])
    np.testing.assert_array_equal(f["n"], f2["n"])
    # the assignment follows the tracks
    np.testing.assert_array_equal(f["track_cluster"][perm], f2["track_cluster"])
