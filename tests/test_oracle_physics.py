"""Sanity of the whole oracle chain on synthetic truth, with the figures of
merit defined in Sec. 4 (reconstructible PV: >= 4 tracks (pp); match within
5 sigma in z; efficiency; fake rate).  Not a pin of the paper's numbers (its
samples are not available); it catches a chain that is wired wrongly."""
import numpy as np

import oracle
from paper_2412_14966_gb300 import synthetic


def _efficiency(b, f, v):
    acc = (v["status"] & oracle.ACCEPTED) > 0
    n_match = n_rcible = n_rec = 0
    for e in range(b.n_events):
        sel = (b.pv_event == e) & (b.pv_ntracks >= 4) & ~b.pv_secondary
        truth = b.pv_pos[sel][:, 2]
        rec = [(v["z"][e, k], np.sqrt(v["cov"][e, k, 5])) for k in range(f["n"][e]) if acc[e, k]]
        n_rcible += len(truth)
        n_rec += len(rec)
        used = set()
        for zt in truth:
            cand = [(abs(zr - zt), k) for k, (zr, sz) in enumerate(rec)
                    if abs(zr - zt) < 5 * sz and k not in used]
            if cand:
                used.add(min(cand)[1])
                n_match += 1
    return n_match / n_rcible, 1 - n_match / max(n_rec, 1)


def test_efficiency_and_fake_rate_small_workload():
    b = synthetic.workload_small()
    p = oracle.default_params()
    f, v = oracle.find_fit(b, p)
    eff, fake = _efficiency(b, f, v)
    assert eff > 0.80, eff
    assert fake < 0.15, fake


def test_secondaries_rejected_by_beamline_cut():
    """Vertices displaced by > 0.3 mm transversely are not accepted."""
    b = synthetic.generate(200, 42, mu=2.0, mean_tracks=28, secondary_frac=0.5)
    p = oracle.default_params()
    f, v = oracle.find_fit(b, p)
    acc = (v["status"] & oracle.ACCEPTED) > 0
    r = np.hypot(v["x"], v["y"])
    assert (r[acc] <= 0.3).all()
    assert ((v["status"] & oracle.REJ_BEAM) > 0).sum() > 5


def test_fixed_target_events_found():
    b = synthetic.generate(100, 43, mu=3.0, mean_tracks=20, gas_event_frac=1.0)
    p = oracle.default_params()
    f, v = oracle.find_fit(b, p)
    acc = (v["status"] & oracle.ACCEPTED) > 0
    assert acc.sum() > 0.6 * len(b.pv_event)
    assert (v["z"][acc] < -300).all()
