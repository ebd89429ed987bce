"""Pins of the x86 flavour's profile (Sec. 3.2, reading R17): template
histograms chosen by sigma_poca.  Each template is checked against a Gaussian
integrated over the bins by Simpson's rule (no error function involved),
against the variance of a binned Gaussian (Sheppard's correction), and for the
class grid, symmetry, unit sum, minimal width and placement on the bin of
z_poca."""
import math

import numpy as np
import pytest

import oracle
from paper_2412_14966_gb300 import synthetic

ONE = oracle.ONE
P = oracle.default_params(profile_mode=1)
P_CUBIC = oracle.default_params()
TPL = oracle.template_table(P)
K = len(TPL["sigma"])
DZ = P.dz


def _simpson_bin_mass(a, b, s, n=400):
    """Mass of N(0, s^2) on [a, b] by composite Simpson's rule."""
    x = np.linspace(a, b, 2 * n + 1)
    f = np.exp(-0.5 * (x / s) ** 2) / (s * math.sqrt(2.0 * math.pi))
    h = (b - a) / (2 * n)
    return h / 3.0 * (f[0] + f[-1] + 4.0 * f[1:-1:2].sum() + 2.0 * f[2:-1:2].sum())


def _weights(k):
    return np.diff(TPL["q"][k])


def test_class_grid_is_geometric():
    """sigma_k = 0.01 mm * 2^(k/4); class k starts at the geometric mean of
    sigma_{k-1} and sigma_k; the grid reaches the p-gas sigma_poca limit."""
    for k in range(K):
        assert abs(TPL["sigma"][k] / (0.01 * 2.0 ** (k / 4)) - 1.0) < 1e-12
    assert TPL["bound"][0] == 0.0
    for k in range(1, K):
        gm = math.sqrt(TPL["sigma"][k - 1] * TPL["sigma"][k])
        assert abs(TPL["bound"][k] / gm - 1.0) < 1e-12
    assert TPL["sigma"][-1] >= P.sigma_max_gas


@pytest.mark.parametrize("k", range(K))
def test_template_is_the_binned_gaussian(k):
    """Every bin weight is ONE times the Gaussian mass of the bin (centred on
    the middle bin) within the two roundings of the cumulative values."""
    s = TPL["sigma"][k]
    H = TPL["half"][k]
    w = _weights(k)
    assert len(w) == 2 * H + 1 and w.sum() == ONE and (w >= 0).all()
    for i in range(2 * H + 1):
        off = i - H
        a, b = (off - 0.5) * DZ, (off + 0.5) * DZ
        if i == 0:
            a = -12.0 * s - 12.0 * DZ         # the outer bins also take the tails
        if i == 2 * H:
            b = 12.0 * s + 12.0 * DZ
        m = _simpson_bin_mass(a, b, s, n=400 if b - a < 20 * s else 4000)
        assert abs(w[i] - ONE * m) <= 1.0 + 1e-6, (k, i, w[i], ONE * m)


@pytest.mark.parametrize("k", range(K))
def test_template_symmetry_and_minimal_width(k):
    """Q[i] + Q[2H+1-i] = ONE (the Gaussian is symmetric about the bin
    centre); the tail beyond the outer edge is below half a unit and the tail
    beyond the next edge inwards is not (H is the smallest such width)."""
    q = TPL["q"][k]
    H = TPL["half"][k]
    assert (q[::-1] + q == ONE).all()
    s = TPL["sigma"][k]
    tail_out = _simpson_bin_mass(-30.0 * s - 30 * DZ, -(H + 0.5) * DZ, s, n=20000)
    assert ONE * tail_out < 0.5 + 1e-6
    if H > 0:
        tail_in = _simpson_bin_mass(-30.0 * s - 30 * DZ, -(H - 0.5) * DZ, s, n=20000)
        assert ONE * tail_in >= 0.5 - 1e-6


@pytest.mark.parametrize("k", [k for k in range(K) if 0.25 <= 0.01 * 2 ** (k / 4)])
def test_template_variance_is_sheppard_corrected(k):
    """A Gaussian of sigma binned with width dz has variance sigma^2 + dz^2/12
    (Sheppard's correction, exact up to exponentially small terms for
    sigma >= dz); the integer template keeps it to its quantisation error."""
    s = TPL["sigma"][k]
    H = TPL["half"][k]
    w = _weights(k).astype(np.float64)
    off = (np.arange(2 * H + 1) - H) * DZ
    assert abs(np.sum(w * off) / ONE) < 1e-12
    var = np.sum(w * off ** 2) / ONE
    assert abs(var / (s * s + DZ * DZ / 12.0) - 1.0) < 0.02, (k, var, s)


def test_class_boundaries_select_the_template():
    """sigma_poca just below class k's lower bound takes class k - 1's
    template, at the bound class k's; the template is centred on the bin of
    z_poca whatever the position inside the bin."""
    for k in (5, 17, 24, 33, 40):
        b = TPL["bound"][k]
        lo = np.nextafter(np.float32(b), np.float32(0.0))
        while float(lo) >= b:
            lo = np.nextafter(lo, np.float32(0.0))
        hi = np.float32(b)
        while float(hi) < b:
            hi = np.nextafter(hi, np.float32(np.inf))
        f_lo, w_lo = oracle.track_profile(0.1, float(lo), P)
        f_hi, w_hi = oracle.track_profile(0.1, float(hi), P)
        assert np.array_equal(w_lo, _weights(k - 1)) and np.array_equal(w_hi, _weights(k))
        c = int((0.1 - P.z_min) / DZ)
        assert f_lo == c - TPL["half"][k - 1] and f_hi == c - TPL["half"][k]
    c = 2400
    zs = [P.z_min + (c + u) * DZ for u in (0.01, 0.37, 0.5, 0.93)]
    prof = [oracle.track_profile(z, 0.4, P) for z in zs]
    assert all(f == prof[0][0] and np.array_equal(w, prof[0][1]) for f, w in prof)


def test_event_histogram_adds_templates_and_drops_outside_bins():
    """A filled track adds its template at its bin (bins outside the range
    lose their share); an event's histogram is the sum over its tracks."""
    rng = np.random.default_rng(5)
    ev = []
    for z in (-549.9, 12.0, -420.0):
        sl = rng.uniform(0.05, 0.3, (6, 2)) * rng.choice([-1.0, 1.0], (6, 2))
        ev.append(synthetic.straight_tracks((0.0, 0.0, z), sl, z + rng.uniform(20, 200, 6),
                                            cov_xx=4e-3))
    batch = synthetic.batch_from_events(ev)
    r = oracle.find_batch(batch, P, want_hist=True)
    prep = oracle.prepare_f32(batch.tracks, P)
    nb = oracle.num_bins(P)
    off = batch.offsets
    for e in range(batch.n_events):
        h = np.zeros(nb, np.int64)
        for t in range(off[e], off[e + 1]):
            if not prep["filled"][t]:
                continue
            f, w = oracle.track_profile(prep["zpoca"][t], prep["sigma"][t], P)
            assert f == prep["j0"][t] and f + len(w) - 1 == prep["j1"][t]
            for i, v in enumerate(w):
                if 0 <= f + i < nb:
                    h[f + i] += v
        assert np.array_equal(h, r["hist"][e].astype(np.int64)), e
    assert r["hist"][0].sum() < 6 * ONE      # the first event's tracks reach below z_min


def test_template_seeds_find_the_same_vertices():
    """On the nominal workload both profiles find nearly the same seeds: the
    two are approximations of one Gaussian profile (Sec. 3.2)."""
    batch = synthetic.workload_nominal(n_events=400, seed=21)
    a = oracle.find_batch(batch, P_CUBIC)
    b = oracle.find_batch(batch, P)
    same_n = np.mean(a["n"] == b["n"])
    assert same_n > 0.85, same_n
    near = []
    for e in np.nonzero(a["n"] == b["n"])[0]:
        n = a["n"][e]
        near.append(np.abs(a["z"][e, :n] - b["z"][e, :n]).max(initial=0.0))
    assert np.quantile(near, 0.95) < 0.25, np.quantile(near, 0.95)
