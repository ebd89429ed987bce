"""Independent reference computations used to pin the oracle.

None of these re-types the oracle's formulas: each one computes the quantity
from its plain definition (a closest approach found by minimising a distance,
an integral found by quadrature, a least-squares problem solved by a library
routine, an M-estimator minimised numerically, ...).
"""
from __future__ import annotations

import math

import numpy as np


def closest_approach_z_bruteforce(x, y, z, tx, ty, beam=(0.0, 0.0, 0.0, 0.0),
                                  half_range=400.0):
    """z at which the transverse distance between the straight track and the
    beamline is smallest, found by a coarse grid then golden-section search."""
    xb, yb, txb, tyb = beam

    def d2(zz):
        dx = (x + tx * (zz - z)) - (xb + txb * zz)
        dy = (y + ty * (zz - z)) - (yb + tyb * zz)
        return dx * dx + dy * dy

    grid = np.linspace(z - half_range, z + half_range, 80001)
    vals = d2(grid)
    i = int(np.argmin(vals))
    a = grid[max(i - 1, 0)]
    b = grid[min(i + 1, len(grid) - 1)]
    gr = (math.sqrt(5.0) - 1.0) / 2.0
    c = b - gr * (b - a)
    d = a + gr * (b - a)
    for _ in range(200):
        if d2(c) < d2(d):
            b = d
        else:
            a = c
        c = b - gr * (b - a)
        d = a + gr * (b - a)
    return 0.5 * (a + b)


def closest_approach_minimiser(px, py, dx, dy):
    """Minimiser z* of |p + z d|^2 for 2-vectors p, d (the textbook quadratic
    minimum, -p.d / d.d); used vectorised in Monte Carlo checks."""
    return -(px * dx + py * dy) / (dx * dx + dy * dy)


def epanechnikov_bin_integral(lo, hi, mu, sigma, n=64):
    """Integral over [lo, hi] of the Epanechnikov density with mean mu and
    variance sigma^2 (support mu +- sqrt(5) sigma), by Gauss-Legendre quadrature
    on the part of the bin inside the support."""
    s = math.sqrt(5.0) * sigma
    a = max(lo, mu - s)
    b = min(hi, mu + s)
    if b <= a:
        return 0.0
    xg, wg = np.polynomial.legendre.leggauss(n)
    xs = 0.5 * (b - a) * xg + 0.5 * (a + b)
    u = (xs - mu) / s
    dens = 0.75 * (1.0 - u * u) / s
    return float(0.5 * (b - a) * np.sum(wg * dens))


def gaussian_bin_integral(lo, hi, mu, sigma):
    """Integral over [lo, hi] of N(mu, sigma^2), via math.erf."""
    c = 1.0 / (sigma * math.sqrt(2.0))
    return 0.5 * (math.erf((hi - mu) * c) - math.erf((lo - mu) * c))


def tukey_rho(c2, c2max):
    """Objective whose derivative in chi2 is the Tukey bi-square weight
    (1 - chi2/chi2max)^2 for chi2 < chi2max, and 0 above."""
    c2 = np.asarray(c2, dtype=np.float64)
    inside = c2 < c2max
    r = np.full_like(c2, c2max / 3.0)
    f = 1.0 - c2[inside] / c2max
    r[inside] = (c2max / 3.0) * (1.0 - f ** 3)
    return r


def track_weights_at(tracks: dict, zs: float):
    """Diagonal weights 1/V_xx, 1/V_yy of each track extrapolated to zs by
    propagating the covariance of (x, tx) along the straight line x + dz*tx
    (J V J^T with J = (1, dz))."""
    d = zs - tracks["z"].astype(np.float64)
    vxx = (tracks["cxx"].astype(np.float64) + 2 * d * tracks["cxtx"].astype(np.float64)
           + d * d * tracks["ctxtx"].astype(np.float64))
    vyy = (tracks["cyy"].astype(np.float64) + 2 * d * tracks["cyty"].astype(np.float64)
           + d * d * tracks["ctyty"].astype(np.float64))
    return 1.0 / vxx, 1.0 / vyy


def chi2_terms(tracks: dict, alpha, wx, wy):
    """Per-track chi2 of a vertex at alpha: the transverse offset of each line
    at z = alpha_z from (alpha_x, alpha_y), weighted by wx, wy."""
    x = tracks["x"].astype(np.float64); y = tracks["y"].astype(np.float64)
    z = tracks["z"].astype(np.float64)
    tx = tracks["tx"].astype(np.float64); ty = tracks["ty"].astype(np.float64)
    rx = x + (alpha[2] - z) * tx - alpha[0]
    ry = y + (alpha[2] - z) * ty - alpha[1]
    return rx * rx * wx + ry * ry * wy
