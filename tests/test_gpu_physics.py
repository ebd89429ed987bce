"""Physics figures of merit (Sec. 4) of the CUDA path on synthetic truth:
the same as the oracle's reconstruction of the same events (the outputs agree
by the parity tests, so the figures must too), the p-gas figures of the
pp + p-gas overlay, and the beamline-offset scan of Sec. 4 (relative
efficiency when the beamline given to the method is off by 20 and 50 um)."""
import numpy as np
import pytest

import oracle
from paper_2412_14966_gb300 import physics, synthetic
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pv():
    import paper_2412_14966_gb300 as pv
    from paper_2412_14966_gb300 import build
    build.build()
    return pv


def _gpu_metrics(pv, batch, beam=(0.0, 0.0, 0.0, 0.0)):
    ctx = pv.Context(device=0, beamline=beam)
    s, v = G.gpu_find_fit(ctx, batch)
    ctx.close()
    E = batch.n_events
    return physics.evaluate(batch, v["x"][:E], v["y"][:E], v["z"][:E], v["cov"][:E],
                            v["status"][:E], v["n_per_event"][:E], v["n_tracks"][:E])


def _oracle_metrics(batch, beam=(0.0, 0.0, 0.0, 0.0)):
    p = G.oracle_params_for(beam=beam)
    ref = oracle.find_batch(batch, p)
    fit = oracle.fit_batch(batch, ref, p)
    return physics.evaluate(batch, fit["x"], fit["y"], fit["z"], fit["cov"], fit["status"],
                            ref["n"], fit["n_tracks"])


@pytest.mark.parametrize("name", ["nominal", "overlay"])
def test_figures_of_merit_match_the_oracle(pv, name):
    batch = (synthetic.workload_nominal(n_events=3000, seed=41) if name == "nominal"
             else synthetic.workload_overlay(n_events=1500, seed=42))
    g = _gpu_metrics(pv, batch)
    r = _oracle_metrics(batch)
    print(name, {k: g[k] for k in ("efficiency", "efficiency_gas", "fake_rate")}, g["pp"])
    assert abs(g["matched"] - r["matched"]) <= max(2, 1e-3 * r["matched"])
    assert abs(g["reconstructed"] - r["reconstructed"]) <= max(2, 1e-3 * r["reconstructed"])
    assert g["efficiency"] > 0.93 and g["fake_rate"] < 0.05
    for region in ("pp", "gas"):
        if r[region] is None:
            continue
        for a in "xyz":
            rg, rr = g[region]["resolution_um"][a], r[region]["resolution_um"][a]
            assert abs(rg - rr) <= 0.01 * rr + 0.05, (region, a, rg, rr)
    if name == "overlay":
        assert g["efficiency_gas"] > 0.9


def test_beamline_offset_scan(pv):
    """Sec. 4: the efficiency stays within 1% of nominal for a beamline off
    by up to 50 um (the seeds sit on the beamline; the fit moves them)."""
    batch = synthetic.workload_nominal(n_events=3000, seed=43)
    base = _gpu_metrics(pv, batch)["efficiency"]
    rel = {}
    for d in (0.02, 0.05):
        rel[d] = _gpu_metrics(pv, batch, beam=(d, d, 0.0, 0.0))["efficiency"] / base
    print("relative efficiency", rel)
    assert rel[0.02] > 0.995 and rel[0.05] > 0.985
