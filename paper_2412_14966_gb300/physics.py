"""Physics figures of merit of a primary-vertex reconstruction against the
truth of a synthetic batch (Sec. 4 of arXiv:2412.14966): efficiency, fake
rate, position resolution and pulls, overall and by the paper's categories
that synthetic truth supports (isolated / close, multiplicity rank, at least
ten tracks, pp / p-gas).

Definitions, restated from Sec. 4:
  * a true PV is reconstructible when it produced at least four tracks (pp)
    or three (p-gas);
  * a reconstructed PV matches a reconstructible one when their z differ by
    less than five times the reconstructed z uncertainty; a true PV keeps
    only its closest match.  Matching is one-to-one: candidate pairs are
    taken in increasing |dz| and each side is used once (the paper does not
    say what happens when one reconstructed PV is the closest match of two
    true ones);
  * efficiency = matched / reconstructible, fake rate = (reconstructed -
    matched) / reconstructed, resolution = standard deviation of
    reconstructed - true position over matched PVs, pull = that difference
    divided by the reconstructed uncertainty;
  * a true PV is "close" when another reconstructible PV of its event lies
    within 10 mm in z, else "isolated"; the multiplicity rank orders the
    reconstructible PVs of an event by track count.
Displaced ("secondary") truth vertices are not PVs: they are never
reconstructible, and a reconstructed vertex on one counts as a fake.

numpy only; it evaluates outputs, it computes nothing of the method."""
from __future__ import annotations

import numpy as np

ACCEPTED = 32


def _pairs(zr, szr, zt):
    """Candidate (rec, true) pairs of one event, closest first."""
    out = []
    for i in range(len(zr)):
        for j in range(len(zt)):
            d = abs(zr[i] - zt[j])
            if d < 5.0 * szr[i]:
                out.append((d, i, j))
    out.sort()
    return out


def evaluate(batch, x, y, z, cov, status, n_per_event, n_tracks=None,
             min_tracks_pp: int = 4, min_tracks_gas: int = 3, close_mm: float = 10.0) -> dict:
    """Figures of merit of the accepted vertices (status & ACCEPTED) of a
    batch.  x, y, z, status: [n_events, capacity]; cov: [n_events, capacity,
    6] (xx, xy, yy, xz, yz, zz); n_per_event: [n_events]; n_tracks (optional,
    [n_events, capacity]) gives the fake rate of vertices with at least ten
    tracks."""
    E = batch.n_events
    rcible = (~batch.pv_secondary) & np.where(batch.pv_gas, batch.pv_ntracks >= min_tracks_gas,
                                              batch.pv_ntracks >= min_tracks_pp)
    pv_by_event = [[] for _ in range(E)]
    for p in np.nonzero(rcible)[0]:
        pv_by_event[int(batch.pv_event[p])].append(int(p))
    matched_true = np.zeros(len(rcible), bool)
    close = np.zeros(len(rcible), bool)
    rank = np.full(len(rcible), -1, np.int64)
    d_pos, d_sig, d_gas = [], [], []
    n_rec = n_rec_matched = n_rec10 = n_rec10_matched = 0
    for e in range(E):
        n = int(n_per_event[e])
        acc = [k for k in range(n) if status[e, k] & ACCEPTED]
        pvs = pv_by_event[e]
        zt = batch.pv_pos[pvs, 2] if pvs else np.zeros(0)
        for a, p in enumerate(pvs):
            close[p] = bool(np.any((np.abs(zt - zt[a]) < close_mm) & (np.arange(len(pvs)) != a)))
        order = sorted(range(len(pvs)), key=lambda a: -int(batch.pv_ntracks[pvs[a]]))
        for r_, a in enumerate(order):
            rank[pvs[a]] = r_
        zr = np.array([z[e, k] for k in acc], np.float64)
        szr = np.array([np.sqrt(max(cov[e, k, 5], 0.0)) for k in acc], np.float64)
        used_r, used_t = set(), set()
        for d, i, j in _pairs(zr, szr, zt):
            if i in used_r or j in used_t:
                continue
            used_r.add(i)
            used_t.add(j)
            k, p = acc[i], pvs[j]
            matched_true[p] = True
            c = cov[e, k]
            d_pos.append((x[e, k] - batch.pv_pos[p, 0], y[e, k] - batch.pv_pos[p, 1],
                          z[e, k] - batch.pv_pos[p, 2]))
            d_sig.append((np.sqrt(max(c[0], 0.0)), np.sqrt(max(c[2], 0.0)),
                          np.sqrt(max(c[5], 0.0))))
            d_gas.append(bool(batch.pv_gas[p]))
        n_rec += len(acc)
        n_rec_matched += len(used_r)
        if n_tracks is not None:
            big = [i for i, k in enumerate(acc) if n_tracks[e, k] >= 10]
            n_rec10 += len(big)
            n_rec10_matched += sum(1 for i in big if i in used_r)

    def eff(mask):
        m = rcible & mask
        return float(matched_true[m].sum() / m.sum()) if m.any() else None

    d_pos = np.asarray(d_pos, np.float64).reshape(-1, 3)
    d_sig = np.asarray(d_sig, np.float64).reshape(-1, 3)
    d_gas = np.asarray(d_gas, bool)

    def res(sel):
        if sel.sum() < 2:
            return None
        dp, ds = d_pos[sel], d_sig[sel]
        pull = dp / np.where(ds > 0, ds, np.nan)
        return {"resolution_um": {a: float(1e3 * np.std(dp[:, i])) for i, a in enumerate("xyz")},
                "pull_mean": {a: float(np.nanmean(pull[:, i])) for i, a in enumerate("xyz")},
                "pull_width": {a: float(np.nanstd(pull[:, i])) for i, a in enumerate("xyz")},
                "matched": int(sel.sum())}

    pp = ~batch.pv_gas
    out = {
        "reconstructible": int(rcible.sum()),
        "reconstructed": int(n_rec),
        "matched": int(n_rec_matched),
        "efficiency": eff(np.ones_like(rcible)),
        "efficiency_pp": eff(pp),
        "efficiency_gas": eff(batch.pv_gas),
        "efficiency_isolated": eff(~close),
        "efficiency_close": eff(close),
        "efficiency_ge10_tracks": eff(batch.pv_ntracks >= 10),
        "efficiency_rank": {f"{r + 1}": eff(rank == r) for r in (0, 2, 4)},
        "fake_rate": float((n_rec - n_rec_matched) / n_rec) if n_rec else None,
        "fake_rate_ge10_tracks": (float((n_rec10 - n_rec10_matched) / n_rec10)
                                  if n_tracks is not None and n_rec10 else None),
        "pp": res(~d_gas),
        "gas": res(d_gas),
    }
    return out
