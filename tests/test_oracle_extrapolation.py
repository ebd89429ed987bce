"""Pins of step (a): z_poca (Eq. zpocadef), V_xy(z) (Eq. Vxy) and sigma_poca
(Sec. 3.1).  CPU only."""
import math

import numpy as np
import pytest

import oracle
from paper_2412_14966_gb300 import synthetic
from tests import helpers


def _tracks_through(points, slopes, dz_state):
    """Noise-free tracks through the given 3D points, states moved by dz_state."""
    n = len(points)
    cols = {k: np.zeros(n) for k in synthetic.TRACK_FIELDS}
    for i, ((px, py, pz), (tx, ty), d) in enumerate(zip(points, slopes, dz_state)):
        cols["x"][i] = px + tx * d
        cols["y"][i] = py + ty * d
        cols["z"][i] = pz + d
        cols["tx"][i] = tx
        cols["ty"][i] = ty
        cols["cxx"][i] = cols["cyy"][i] = 1e-3
        cols["ctxtx"][i] = cols["ctyty"][i] = 1e-6
    return cols


def _as_f32(cols):
    return {k: np.ascontiguousarray(v.astype(np.float32)) for k, v in cols.items()}


def test_zpoca_of_tracks_through_the_beamline():
    """A track through the beamline point at z0 has its closest approach at z0."""
    rng = np.random.default_rng(11)
    n = 200
    z0 = rng.uniform(-500, 250, n)
    slopes = np.stack([rng.uniform(-0.3, 0.3, n), rng.uniform(-0.3, 0.3, n)], 1)
    slopes[np.hypot(slopes[:, 0], slopes[:, 1]) < 0.02] = 0.05
    # exactly representable geometry so that binary32 inputs are exact
    z0 = np.round(z0 * 8) / 8
    d = np.round(rng.uniform(-10, 10, n) * 8) / 8
    slopes = np.round(slopes * 1024) / 1024
    pts = [(0.0, 0.0, z) for z in z0]
    t = _as_f32(_tracks_through(pts, slopes, d))
    p = oracle.default_params()
    r64 = oracle.prepare_f64(t, p)
    np.testing.assert_allclose(r64["zpoca"], z0, atol=1e-9)
    r32 = oracle.prepare_f32(t, p)
    # binary32: a few ulp of |z| plus the state's own rounding divided by |t|
    np.testing.assert_allclose(r32["zpoca"], z0, atol=2e-4)


def test_zpoca_invariant_along_the_track():
    """Moving the state along its own straight line leaves z_poca unchanged."""
    rng = np.random.default_rng(12)
    n = 100
    x = rng.normal(0, 0.05, n); y = rng.normal(0, 0.05, n); z = rng.uniform(-100, 100, n)
    tx = rng.uniform(-0.3, 0.3, n); ty = rng.uniform(-0.3, 0.3, n)
    p = oracle.default_params()
    out = []
    for shift in (0.0, 7.25, -13.5):
        cols = {k: np.zeros(n) for k in synthetic.TRACK_FIELDS}
        cols.update(x=x + tx * shift, y=y + ty * shift, z=z + shift, tx=tx, ty=ty)
        cols["cxx"][:] = 1e-3; cols["cyy"][:] = 1e-3
        out.append(oracle.prepare_f64(_as_f32(cols), p)["zpoca"])
    # inputs are rounded to binary32, so agreement is at the input rounding level
    np.testing.assert_allclose(out[1], out[0], atol=5e-5)
    np.testing.assert_allclose(out[2], out[0], atol=5e-5)


@pytest.mark.parametrize("beam", [(0.0, 0.0, 0.0, 0.0), (0.4, -0.3, 2e-3, -1.5e-3),
                                  (1.092, 0.472, 0.0, 0.0)])
def test_zpoca_equals_bruteforce_closest_approach(beam):
    """Against the closest approach found by minimising the transverse distance
    between track and beamline on a grid (reading R1 for tilted beams)."""
    rng = np.random.default_rng(13)
    n = 40
    cols = {k: np.zeros(n) for k in synthetic.TRACK_FIELDS}
    cols["x"] = rng.normal(0, 0.3, n) + beam[0]
    cols["y"] = rng.normal(0, 0.3, n) + beam[1]
    cols["z"] = rng.uniform(-200, 200, n)
    cols["tx"] = rng.uniform(-0.3, 0.3, n)
    cols["ty"] = rng.uniform(-0.3, 0.3, n)
    cols["cxx"][:] = 1e-3; cols["cyy"][:] = 1e-3
    t = _as_f32(cols)
    p = oracle.default_params(x_b=beam[0], y_b=beam[1], tx_b=beam[2], ty_b=beam[3])
    z64 = oracle.prepare_f64(t, p)["zpoca"]
    z32 = oracle.prepare_f32(t, p)["zpoca"]
    for i in range(n):
        zb = helpers.closest_approach_z_bruteforce(
            float(t["x"][i]), float(t["y"][i]), float(t["z"][i]), float(t["tx"][i]),
            float(t["ty"][i]), beam=beam, half_range=2000.0)
        assert abs(z64[i] - zb) < 1e-6, (i, z64[i], zb)
        # the pinned binary32 sequence, within its rounding
        assert abs(z32[i] - zb) < 2e-3 + 1e-5 * abs(zb), (i, z32[i], zb)


def test_covariance_extrapolation_monte_carlo():
    """V_xx(z) of Eq. Vxy (diagonal block) against the sample variance of x
    propagated along sampled straight lines."""
    rng = np.random.default_rng(14)
    V = np.array([[4e-3, 3e-5], [3e-5, 2e-6]])  # (x, tx) covariance with correlation
    L = np.linalg.cholesky(V)
    s = rng.standard_normal((400_000, 2)) @ L.T
    for dz in (-12.0, 0.0, 5.0, 30.0):
        x_at = s[:, 0] + dz * s[:, 1]
        wx, _ = helpers.track_weights_at(
            {"z": np.array([0.0]), "cxx": np.array([V[0, 0]]), "cxtx": np.array([V[0, 1]]),
             "ctxtx": np.array([V[1, 1]]), "cyy": np.array([1.0]), "cyty": np.array([0.0]),
             "ctyty": np.array([0.0])}, dz)
        assert abs(np.var(x_at) * wx[0] - 1.0) < 0.01


def test_sigma_poca_monte_carlo():
    """sigma_poca = sqrt(V_xx / |t - t_b|^2) (Sec. 3.1) equals the spread of the
    closest-approach z under position noise of equal x, y variance."""
    rng = np.random.default_rng(15)
    p = oracle.default_params()
    for tx, ty, sig in ((0.1, 0.05, 0.03), (-0.25, 0.2, 0.05), (0.02, -0.03, 0.01)):
        cols = {k: np.zeros(1) for k in synthetic.TRACK_FIELDS}
        cols.update(x=np.array([0.0]), y=np.array([0.0]), z=np.array([10.0]),
                    tx=np.array([tx]), ty=np.array([ty]))
        cols["cxx"][:] = sig * sig; cols["cyy"][:] = sig * sig
        cols["ctxtx"][:] = 1e-6; cols["ctyty"][:] = 1e-6
        o = oracle.prepare_f64(_as_f32(cols), p)
        n = 400_000
        px = rng.normal(0, sig, n)
        py = rng.normal(0, sig, n)
        zs = 10.0 + helpers.closest_approach_minimiser(px, py, np.float64(np.float32(tx)),
                                                       np.float64(np.float32(ty)))
        assert abs(np.std(zs) / o["sigma"][0] - 1.0) < 0.01


def test_sigma_uses_covariance_at_zpoca():
    """With slope variance the uncertainty grows with the distance between the
    state and z_poca as V_xx(z_poca) of Eq. Vxy (reading R2)."""
    p = oracle.default_params()
    base = {k: np.zeros(2) for k in synthetic.TRACK_FIELDS}
    base.update(x=np.array([0.2, 0.2]), y=np.array([0.0, 0.0]), z=np.array([0.0, 0.0]),
                tx=np.array([0.2, 0.2]), ty=np.array([0.0, 0.0]))
    base["cxx"][:] = 1e-4; base["cyy"][:] = 1e-4
    base["ctxtx"][:] = np.array([0.0, 1e-4])
    o = oracle.prepare_f64(_as_f32(base), p)
    d = o["zpoca"][0] - 0.0
    assert abs(d + 1.0) < 1e-6  # z_poca = -x/tx = -1 mm
    vxx1 = 1e-4 + d * d * np.float64(np.float32(1e-4))
    assert math.isclose(o["sigma"][1], math.sqrt(vxx1) / np.float64(np.float32(0.2)),
                        rel_tol=1e-6)
    assert o["sigma"][1] > o["sigma"][0]


def test_sigma_with_correlated_state_monte_carlo():
    """The state sits 5 mm upstream of z_poca and (x, tx) are correlated: the
    spread of z_poca follows V_xx propagated by +5 mm (Eq. Vxy with dz =
    z_poca - z_trk), which differs strongly from propagation by -5 mm."""
    rng = np.random.default_rng(16)
    p = oracle.default_params()
    tx, ty = 0.2, -0.1
    V = np.array([[4e-3, 5e-4], [5e-4, 1e-4]])
    cols = {k: np.zeros(1) for k in synthetic.TRACK_FIELDS}
    # line through (0, 0, 5): state at z = 0
    cols.update(x=np.array([-5 * tx]), y=np.array([-5 * ty]), z=np.array([0.0]),
                tx=np.array([tx]), ty=np.array([ty]))
    cols["cxx"][:] = V[0, 0]; cols["cxtx"][:] = V[0, 1]; cols["ctxtx"][:] = V[1, 1]
    cols["cyy"][:] = V[0, 0]; cols["cyty"][:] = V[0, 1]; cols["ctyty"][:] = V[1, 1]
    o = oracle.prepare_f64(_as_f32(cols), p)
    o32 = oracle.prepare_f32(_as_f32(cols), p)
    assert abs(o["zpoca"][0] - 5.0) < 1e-5
    assert abs(o32["sigma"][0] / o["sigma"][0] - 1.0) < 1e-5
    L = np.linalg.cholesky(V)
    n = 400_000
    sx = rng.standard_normal((n, 2)) @ L.T
    sy = rng.standard_normal((n, 2)) @ L.T
    # sampled lines evaluated at z = 5 (position noise there), nominal slopes
    px = sx[:, 0] + 5.0 * sx[:, 1]
    py = sy[:, 0] + 5.0 * sy[:, 1]
    tx32, ty32 = np.float64(np.float32(tx)), np.float64(np.float32(ty))
    zs = 5.0 + helpers.closest_approach_minimiser(px, py, tx32, ty32)
    # x and y carry the same variance, as the paper's formula assumes
    assert abs(np.std(zs) / o["sigma"][0] - 1.0) < 0.01


def test_contract_mode_close_to_binary64():
    """The pinned binary32 sequence stays within binary32 rounding of the
    binary64 values on realistic tracks."""
    b = synthetic.workload_small(n_events=20)
    p = oracle.default_params()
    r32 = oracle.prepare_f32(b.tracks, p)
    r64 = oracle.prepare_f64(b.tracks, p)
    ok = r32["filled"] > 0
    err = np.abs(r32["zpoca"][ok] - r64["zpoca"][ok])
    assert err.max() < 2e-3  # mm; |z| up to ~200 mm, t down to ~0.03
    rel = np.abs(r32["sigma"][ok] / r64["sigma"][ok] - 1.0)
    assert rel.max() < 1e-5


def test_fill_conditions():
    """Tracks are filled only with z_poca inside [-550, 300) mm and sigma_poca
    below 1.5 mm (pp) or 10 mm (z_poca < -300 mm), Sec. 3.2, and with a slope
    relative to the beam (reading R1: parallel tracks have no z_poca)."""
    p = oracle.default_params()
    rows = [  # (x, z, tx, sigma_xy) -> expected filled; z_poca = z - x/tx
        (0.0, 0.0, 0.1, 0.10, 1),      # sigma_poca 1.0 mm, pp -> filled
        (0.0, 0.0, 0.1, 0.16, 0),      # 1.6 mm > 1.5 (pp) -> not filled
        (0.0, -400.0, 0.1, 0.5, 1),    # 5 mm in the gas region -> filled
        (0.0, -400.0, 0.1, 1.2, 0),    # 12 mm > 10 -> not filled
        (0.0, 299.9, 0.2, 0.01, 1),    # inside the range
        (0.0, 300.1, 0.2, 0.01, 0),    # above the range
        (0.0, -550.2, 0.2, 0.01, 0),   # below the range
        (0.0, 10.0, 0.0, 0.01, 0),     # parallel to the beam
        (float("nan"), 10.0, 0.1, 0.01, 0),
    ]
    cols = {k: np.zeros(len(rows)) for k in synthetic.TRACK_FIELDS}
    for i, (x, z, tx, s, _) in enumerate(rows):
        cols["x"][i] = x; cols["z"][i] = z; cols["tx"][i] = tx
        cols["cxx"][i] = cols["cyy"][i] = s * s
    r = oracle.prepare_f32(_as_f32(cols), p)
    assert list(r["filled"]) == [e[-1] for e in rows]
