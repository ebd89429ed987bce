"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.  Bit-exact for z_poca, sigma_poca, histogram bins, seeds,
cluster bounds and track assignment; within 0.1 um (x, y), 0.5 um (z) and 1e-4
relative covariance for the fit."""
import numpy as np
import pytest

import oracle
from paper_2412_14966_gb300 import synthetic
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pv():
    import paper_2412_14966_gb300 as pv
    from paper_2412_14966_gb300 import build
    build.build()
    return pv


@pytest.fixture(scope="module")
def ctx(pv):
    c = pv.Context(device=0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def small():
    return synthetic.workload_small()


def test_extrapolation_bit_exact(ctx, pv, small):
    import torch
    tracks = pv.Tracks.from_batch(small)
    zp, sg, cb = ctx.extrapolate_batch(tracks)
    torch.cuda.synchronize()
    ref = oracle.prepare_f32(small.tracks, oracle.default_params())
    assert np.array_equal(zp.cpu().numpy().view(np.int32), ref["zpoca"].view(np.int32))
    fin = np.isfinite(ref["sigma"])
    assert np.array_equal(sg.cpu().numpy()[fin].view(np.int32), ref["sigma"][fin].view(np.int32))
    assert np.array_equal(cb.cpu().numpy(), np.where(ref["filled"] > 0, ref["center"], -1))


@pytest.mark.parametrize("name", ["small", "nominal500", "pileup200", "mixture500"])
def test_histogram_bit_exact(ctx, pv, name):
    """Every bin of every event's histogram (Sec. 3.2, reading R3) against the
    oracle: the small workload, 500 nominal events, 200 high pile-up events
    (~1,200 tracks each) and 500 events of the fixed-target mixture (p-gas
    windows up to 180 bins)."""
    import torch
    batch = {"small": lambda: synthetic.workload_small(),
             "nominal500": lambda: synthetic.workload_nominal(n_events=500, seed=21),
             "pileup200": lambda: synthetic.generate(200, 22, mu=40.0, mean_tracks=28.0,
                                                     name="pileup-200"),
             "mixture500": lambda: synthetic.workload_mixture(n_events=500, seed=23)}[name]()
    tracks = pv.Tracks.from_batch(batch)
    h = ctx.histogram_batch(tracks)
    torch.cuda.synchronize()
    ref = oracle.find_batch(batch, oracle.default_params(), want_hist=True)
    got = h.cpu().numpy().view(np.uint32)
    bad = np.nonzero(got != ref["hist"])
    assert len(bad[0]) == 0, (bad[0][:5], bad[1][:5])
    assert (ref["hist"].sum(axis=1) > 0).all() or name == "small"


@pytest.mark.parametrize("fused", [True, False])
def test_find_and_fit_small_workload(ctx, pv, small, fused):
    s, v = G.gpu_find_fit(ctx, small, fused=fused)
    p = oracle.default_params()
    ref = oracle.find_batch(small, p)
    G.assert_find_equal(s, ref, small)
    fit = oracle.fit_batch(small, ref, p)
    worst, nd = G.assert_fit_close(v, fit, ref["n"], lambda: G.tight_refit(pv, small, s, ref),
                                   cond=(small, ref, p))
    print("worst", worst, "iteration mismatches", nd)


def test_plain_path_equals_fused(pv, small):
    import torch
    a = pv.Context(device=0)
    b = pv.Context(device=0, path=pv.PATH_PLAIN)
    sa, va = G.gpu_find_fit(a, small)
    sb, vb = G.gpu_find_fit(b, small)
    E = small.n_events
    assert np.array_equal(sa["n_per_event"][:E], sb["n_per_event"][:E])
    assert np.array_equal(sa["track_vertex"][:small.n_tracks], sb["track_vertex"][:small.n_tracks])
    for e in range(E):
        n = sa["n_per_event"][e]
        for k in ("x", "y", "z", "bin_lo", "bin_hi", "bin_max"):
            assert np.array_equal(sa[k][e, :n], sb[k][e, :n]), (e, k)
        for k in ("x", "y", "z", "cov", "chi2", "ndof", "n_tracks", "n_iter", "status"):
            assert np.array_equal(va[k][e, :n], vb[k][e, :n]), (e, k)
    a.close(); b.close()
    torch.cuda.synchronize()


def test_nominal_workload_full_size(ctx, pv):
    """10,000 events at the benchmark's launch configuration, every event
    against the oracle."""
    batch = synthetic.workload_nominal()
    s, v = G.gpu_find_fit(ctx, batch)
    p = oracle.default_params()
    ref = oracle.find_batch(batch, p)
    G.assert_find_equal(s, ref, batch)
    fit = oracle.fit_batch(batch, ref, p)
    worst, nd = G.assert_fit_close(v, fit, ref["n"], lambda: G.tight_refit(pv, batch, s, ref),
                                   cond=(batch, ref, p))
    print("worst", {k: worst[k] for k in ("xy", "z", "cov")}, "ill-conditioned", worst["ill"],
          "fixed-point comparisons", nd)
    n = s["n_per_event"][:batch.n_events]
    assert n.min() >= 0 and n.max() <= 64
    for e in range(batch.n_events):
        z = s["z"][e, :n[e]]
        assert np.all(np.diff(z) > 0)
        assert np.all(np.isfinite(v["z"][e, :n[e]]))


def test_mixture_with_fixed_target(ctx, pv):
    """Uneven events and the p-gas region (Table smog-pp), every event
    against the oracle."""
    batch = synthetic.workload_mixture(n_events=3000)
    s, v = G.gpu_find_fit(ctx, batch)
    p = oracle.default_params()
    ref = oracle.find_batch(batch, p)
    G.assert_find_equal(s, ref, batch)
    assert (ref["z"][ref["n"] > 0] < -300).any()
    fit = oracle.fit_batch(batch, ref, p)
    G.assert_fit_close(v, fit, ref["n"], lambda: G.tight_refit(pv, batch, s, ref), cond=(batch, ref, p))


def test_high_pileup_events(ctx, pv):
    """~1,200 tracks per event (global-scratch path), overlapping vertices."""
    batch = synthetic.generate(24, 3, mu=40.0, mean_tracks=28.0, name="pileup-24")
    s, v = G.gpu_find_fit(ctx, batch)
    p = oracle.default_params()
    ref = oracle.find_batch(batch, p)
    G.assert_find_equal(s, ref, batch)
    fit = oracle.fit_batch(batch, ref, p)
    G.assert_fit_close(v, fit, ref["n"], lambda: G.tight_refit(pv, batch, s, ref), cond=(batch, ref, p))


@pytest.mark.parametrize("beam", [(0.35, -0.2, 1.5e-3, -0.8e-3), (1.092, 0.472, 0.0, 0.0)])
def test_displaced_and_tilted_beamline(pv, beam):
    """Nonzero beam position and slope exercise the beam terms of Eq. zpocadef
    (reading R1) and the seed position on the beamline."""
    batch = synthetic.workload_small(n_events=60, seed=5)
    ctx = pv.Context(device=0, beamline=beam)
    s, v = G.gpu_find_fit(ctx, batch)
    p = G.oracle_params_for(beam=beam)
    ref = oracle.find_batch(batch, p)
    G.assert_find_equal(s, ref, batch)
    fit = oracle.fit_batch(batch, ref, p)
    G.assert_fit_close(v, fit, ref["n"], lambda: G.tight_refit(pv, batch, s, ref, beam=beam),
                       cond=(batch, ref, p))
    ctx.close()


def test_kahan_accumulation_within_tolerance(pv, small):
    ctx = pv.Context(device=0, accum_mode=pv.ACCUM_KAHAN)
    s, v = G.gpu_find_fit(ctx, small)
    p = oracle.default_params()
    ref = oracle.find_batch(small, p)
    G.assert_find_equal(s, ref, small)
    fit = oracle.fit_batch(small, ref, p)
    G.assert_fit_close(v, fit, ref["n"], lambda: G.tight_refit(pv, small, s, ref,
                                                        accum_mode=pv.ACCUM_KAHAN),
                       cond=(small, ref, p))
    ctx.close()


def test_deterministic_and_alone_equals_mix(ctx, pv):
    """Per-event results do not depend on the rest of the batch or on
    scheduling: bit-identical alone and in the mix, run after run."""
    batch = synthetic.workload_mixture(n_events=800, seed=9)
    s1, v1 = G.gpu_find_fit(ctx, batch)
    s2, v2 = G.gpu_find_fit(ctx, batch)
    for k in ("x", "y", "z", "cov", "status", "n_iter"):
        for e in range(batch.n_events):
            n = v1["n_per_event"][e]
            assert np.array_equal(v1[k][e, :n], v2[k][e, :n]), (k, e)
    pick = np.array([5, 17, 400, 401, 799, 3])
    sub = batch.subset(pick)
    s3, v3 = G.gpu_find_fit(ctx, sub)
    for i, e in enumerate(pick):
        n = v1["n_per_event"][e]
        assert v3["n_per_event"][i] == n
        for k in ("x", "y", "z", "cov", "chi2", "status", "n_iter"):
            assert np.array_equal(v3[k][i, :n], v1[k][e, :n]), (k, e)


def test_edge_cases(ctx, pv):
    import torch
    rng = np.random.default_rng(4)
    ev = []
    ev.append(synthetic.straight_tracks((0.0, 0.0, 1.0), [(0.1, 0.0)], [2.0]))          # 1 track
    ev.append({k: np.zeros(0, np.float32) for k in synthetic.TRACK_FIELDS})            # empty
    # 100 well separated vertices of 5 tracks: more seeds than the capacity
    many = [synthetic.straight_tracks((0.0, 0.0, -240.0 + 4.5 * i),
                                      rng.uniform(-0.3, 0.3, (5, 2)),
                                      -240.0 + 4.5 * i + rng.uniform(-5, 5, 5), cov_xx=4e-4)
            for i in range(100)]
    ev.append({k: np.concatenate([m[k] for m in many]) for k in synthetic.TRACK_FIELDS})
    # NaN / parallel / out-of-range tracks mixed into a normal event
    base = synthetic.workload_small(n_events=1, seed=8)
    t = {k: v.copy() for k, v in base.tracks.items()}
    t["x"][0] = np.nan
    t["tx"][1] = 0.0; t["ty"][1] = 0.0
    t["z"][2] = 1e6
    t["cyy"][3] = np.inf
    ev.append(t)
    # one event of 5,000 tracks
    big = synthetic.generate(1, 77, mu=170.0, mean_tracks=28.0)
    ev.append({k: v for k, v in big.tracks.items()})
    batch = synthetic.batch_from_events(ev)
    s, v = G.gpu_find_fit(ctx, batch)
    p = oracle.default_params()
    ref = oracle.find_batch(batch, p)
    assert ref["event_status"][2] & oracle.EV_SEED_OVERFLOW
    G.assert_find_equal(s, ref, batch)
    fit = oracle.fit_batch(batch, ref, p)
    G.assert_fit_close(v, fit, ref["n"], lambda: G.tight_refit(pv, batch, s, ref), cond=(batch, ref, p))
    # empty batch
    empty = synthetic.batch_from_events([])
    tr = pv.Tracks.from_batch(empty)
    ctx.fit_batch(tr)
    torch.cuda.synchronize()


def test_bad_offsets_flagged(ctx, pv):
    import torch
    batch = synthetic.workload_small(n_events=4, seed=2)
    tracks = pv.Tracks.from_batch(batch)
    offs = batch.offsets.copy()
    offs[2] = offs[1] - 1          # event 1 ends before it starts; event 2 starts earlier
    bad = pv.Tracks(tracks.cols, torch.from_numpy(offs).cuda())
    out = ctx.fit_batch(bad)
    torch.cuda.synchronize()
    o = out.numpy()
    assert o["event_status"][1] == pv.EV_BAD_OFFSETS and o["n_per_event"][1] == 0
    assert o["event_status"][0] != pv.EV_BAD_OFFSETS


@pytest.mark.parametrize("pinned", [True, False])
def test_run_host_equals_device_path(ctx, pv, small, pinned):
    """Pinned host outputs are written by the kernels in place, pageable ones
    through a device staging buffer; both equal the device path."""
    import torch
    s, v = G.gpu_find_fit(ctx, small)
    host = pv.Tracks.from_host(small, pinned=pinned)
    out = pv.Vertices.empty(small.n_events, small.n_tracks, host=True, pinned=pinned)
    ctx.run_host(host, out)
    o = out.numpy()
    for e in range(small.n_events):
        n = v["n_per_event"][e]
        for k in ("x", "y", "z", "cov", "status", "n_iter"):
            assert np.array_equal(o[k][e, :n], v[k][e, :n]), (k, e)
    assert np.array_equal(o["track_vertex"][:small.n_tracks], v["track_vertex"][:small.n_tracks])


@pytest.mark.parametrize("tilted", [False, True])
def test_pp_plus_gas_overlay(pv, tilted):
    """pp events each overlaid with one p-gas PV (the paper's pp + p-gas
    sample), around a straight or a displaced and inclined beamline (Eq.
    zpocadef with beam slopes, reading R1): every event against the oracle."""
    beam = synthetic.TILTED_BEAM if tilted else (0.0, 0.0, 0.0, 0.0)
    batch = synthetic.workload_overlay(n_events=1000, seed=7, beam=beam)
    ctx = pv.Context(device=0, beamline=beam)
    s, v = G.gpu_find_fit(ctx, batch)
    ctx.close()
    p = G.oracle_params_for(beam=beam)
    ref = oracle.find_batch(batch, p)
    G.assert_find_equal(s, ref, batch)
    # both regions produce seeds
    zs = ref["z"][np.arange(64)[None, :] < ref["n"][:, None]]
    assert (zs < -300).sum() > 0.8 * batch.n_events and (zs > -300).sum() > batch.n_events
    fit = oracle.fit_batch(batch, ref, p)
    G.assert_fit_close(v, fit, ref["n"], lambda: G.tight_refit(pv, batch, s, ref, beam=beam),
                       cond=(batch, ref, p))


@pytest.mark.parametrize("path", ["fused", "plain"])
def test_recursive_split_flavour(pv, path):
    """The x86 flavour of the peak search (Sec. 3.3, reading R16) through the
    fused and the plain path: seeds bit-exact and the fit within tolerance on
    the nominal workload and the pp + p-gas overlay (both regions' minimal
    integrals).  The two flavours part on a few percent of the events."""
    cfg = dict(split_mode=pv.SPLIT_RECURSIVE)
    if path == "plain":
        cfg["path"] = pv.PATH_PLAIN
    for batch in (synthetic.workload_nominal(n_events=1500, seed=14),
                  synthetic.workload_overlay(n_events=800, seed=13)):
        ctx = pv.Context(device=0, **cfg)
        s, v = G.gpu_find_fit(ctx, batch)
        ctx.close()
        p = oracle.default_params(split_mode=1)
        ref = oracle.find_batch(batch, p)
        G.assert_find_equal(s, ref, batch)
        ref0 = oracle.find_batch(batch, oracle.default_params())
        assert (ref0["n"] != ref["n"]).any()
        fit = oracle.fit_batch(batch, ref, p)
        G.assert_fit_close(v, fit, ref["n"], lambda: G.tight_refit(pv, batch, s, ref, **cfg),
                           cond=(batch, ref, p))


def _sigma_ladder_events():
    """Events whose tracks' sigma_poca runs through every template class (log-
    uniform from 5 um to 9.5 mm, p-gas region) and, capped at 1.5 mm, the pp
    region; also tracks near both ends of the histogram."""
    rng = np.random.default_rng(17)
    ev = []
    for z0, smax in ((-420.0, 9.5), (0.0, 1.45), (-549.8, 9.5), (299.7, 1.45)):
        n = 120
        sig = np.exp(rng.uniform(np.log(0.005), np.log(smax), n))
        t = rng.uniform(0.05, 0.3, (n, 2)) * rng.choice([-1.0, 1.0], (n, 2))
        tt = np.sqrt((t ** 2).sum(axis=1))
        e = synthetic.straight_tracks((0.0, 0.0, z0), t, z0 + rng.uniform(-1.0, 1.0, n),
                                      cov_xx=1.0, cov_tt=1e-12)
        e["cxx"] = ((sig * tt) ** 2).astype(np.float32)
        e["cyy"] = e["cxx"].copy()
        ev.append(e)
    return synthetic.batch_from_events(ev)


def test_template_profile_histogram_bit_exact(pv):
    """The x86 profile (Sec. 3.2, reading R17): the device's template table
    (built with the device's erfc) and fill give the oracle's histograms bit
    for bit, for sigma_poca in every template class and at the range ends."""
    import torch
    batch = _sigma_ladder_events()
    p = oracle.default_params(profile_mode=1)
    prep = oracle.prepare_f32(batch.tracks, p)
    tpl = oracle.template_table(p)
    classes = {int(np.searchsorted(tpl["bound"], s, side="right") - 1)
               for s, f in zip(prep["sigma"], prep["filled"]) if f}
    assert len(classes) == len(tpl["sigma"])
    ctx = pv.Context(device=0, profile_mode=pv.PROFILE_TEMPLATE)
    h = ctx.histogram_batch(pv.Tracks.from_batch(batch))
    torch.cuda.synchronize()
    ctx.close()
    ref = oracle.find_batch(batch, p, want_hist=True)
    assert np.array_equal(h.cpu().numpy().view(np.uint32), ref["hist"])
    # the events through the fused find (its own fill) against the oracle
    ctx = pv.Context(device=0, profile_mode=pv.PROFILE_TEMPLATE)
    s, v = G.gpu_find_fit(ctx, batch)
    ctx.close()
    G.assert_find_equal(s, oracle.find_batch(batch, p), batch)


@pytest.mark.parametrize("split", [0, 1])
@pytest.mark.parametrize("path", ["fused", "plain"])
def test_template_profile_flavour(pv, path, split):
    """The x86 profile alone and with the x86 split (the full x86 flavour of
    steps b and c) through both paths: seeds bit-exact and the fit within
    tolerance on the nominal workload and the pp + p-gas overlay."""
    cfg = dict(profile_mode=pv.PROFILE_TEMPLATE, split_mode=split)
    if path == "plain":
        cfg["path"] = pv.PATH_PLAIN
    for batch in (synthetic.workload_nominal(n_events=1500, seed=15),
                  synthetic.workload_overlay(n_events=800, seed=16)):
        ctx = pv.Context(device=0, **cfg)
        s, v = G.gpu_find_fit(ctx, batch)
        ctx.close()
        p = oracle.default_params(profile_mode=1, split_mode=split)
        ref = oracle.find_batch(batch, p)
        G.assert_find_equal(s, ref, batch)
        fit = oracle.fit_batch(batch, ref, p)
        G.assert_fit_close(v, fit, ref["n"], lambda: G.tight_refit(pv, batch, s, ref, **cfg),
                           cond=(batch, ref, p))


@pytest.mark.parametrize("case", ["nominal", "mixture", "unsplittable", "pageable", "plain",
                                  "mixed", "x86"])
def test_run_host_pipeline_equals_device_path(pv, case):
    """pv_run_host splits batches of 4,096 events or more into event chunks
    whose copies overlap the kernels; the results equal the device path's bit
    for bit (events are independent).  A batch whose offsets do not rise runs
    as one chunk and still matches (its bad event flagged the same way).
    Outputs in pinned memory are written in place, pageable ones (and all of
    the plain path's) are staged and copied back; "mixed" has both kinds in one
    call.  Pinned inputs are read in place by the find kernel of the GPU
    flavour, which leaves the device copy for the fit; pageable inputs, the
    plain path and the x86 flavour copy them in by event chunks."""
    import torch
    if case in ("nominal", "pageable", "plain", "mixed", "x86"):
        batch = synthetic.workload_nominal(n_events=9000, seed=12)
    elif case == "mixture":
        batch = synthetic.workload_mixture(n_events=5000, seed=13)
    else:
        batch = synthetic.workload_nominal(n_events=4500, seed=14)
        off = batch.offsets.copy()
        off[-1] = off[-1] + 5            # the last event ends past the last track
        batch.offsets = off
    cfg = dict(use_graph=1)
    if case == "plain":
        cfg = dict(path=pv.PATH_PLAIN)
    elif case == "x86":
        cfg = dict(use_graph=1, split_mode=pv.SPLIT_RECURSIVE, profile_mode=pv.PROFILE_TEMPLATE)
    ctx = pv.Context(device=0, **cfg)
    s, v = G.gpu_find_fit(ctx, batch)
    host = pv.Tracks.from_host(batch, pinned=case != "pageable")
    out = pv.Vertices.empty(batch.n_events, batch.n_tracks, host=True, pinned=case != "pageable")
    if case == "mixed":
        for k in ("cov", "status", "track_vertex"):
            out.a[k] = torch.empty_like(out.a[k], pin_memory=False)
    for a in out.a.values():
        a.fill_(-7)
    ctx.run_host(host, out)
    ctx.close()
    o = out.numpy()
    E = batch.n_events
    assert np.array_equal(o["n_per_event"][:E], v["n_per_event"][:E])
    assert np.array_equal(o["event_status"][:E], v["event_status"][:E])
    for e in range(E):
        n = v["n_per_event"][e]
        for k in ("x", "y", "z", "cov", "chi2", "status", "n_iter", "n_tracks"):
            assert np.array_equal(o[k][e, :n], v[k][e, :n]), (k, e)
    nt = len(batch.tracks["x"])
    owned = np.zeros(nt, bool)
    for e in range(E):
        b0, b1 = batch.offsets[e], batch.offsets[e + 1]
        if 0 <= b0 <= b1 <= nt:
            owned[b0:b1] = True
    assert np.array_equal(o["track_vertex"][:nt][owned], v["track_vertex"][:nt][owned])
    if case == "unsplittable":
        assert o["event_status"][E - 1] == pv.EV_BAD_OFFSETS


def _comb_event(n_peaks=40, rising=True):
    """One event whose histogram is a single proto-cluster of n_peaks narrow
    peaks (k + 3 tracks each, one bin wide, 1 mm apart in the p-gas region) on
    a floor of 24 broad tracks: rising to the right, the recursive split (the
    two largest maxima are the two rightmost peaks at every level) nests
    n_peaks - 1 pending right-hand sides."""
    ev = []
    t = np.array([[0.3, 0.0]])
    for k in range(n_peaks):
        z = -450.0 + k * 1.0 + 0.125
        m = (k if rising else n_peaks - 1 - k) + 3
        ev.append(synthetic.straight_tracks((0.0, 0.0, z), np.repeat(t, m, 0), np.full(m, z),
                                            cov_xx=(0.02 * 0.3) ** 2, cov_tt=1e-14))
    for j in range(24):
        z = -462.0 + 2.5 * j
        ev.append(synthetic.straight_tracks((0.0, 0.0, z), t, [z], cov_xx=(8.0 * 0.3) ** 2,
                                            cov_tt=1e-14))
    return {k: np.concatenate([e[k] for e in ev]) for k in synthetic.TRACK_FIELDS}


@pytest.mark.parametrize("path", ["fused", "plain"])
def test_recursive_split_deep_comb_on_the_gpu(pv, path):
    """The x86 flavour's recursive split to depth 39 on the device (and a
    falling comb, which splits at the top level every time): seeds, bounds and
    assignments bit-exact with the oracle, every peak a seed."""
    batch = synthetic.batch_from_events([_comb_event(), _comb_event(rising=False),
                                         _comb_event(25)])
    p = oracle.default_params(split_mode=1)
    ref = oracle.find_batch(batch, p, want_hist=True)
    # each comb is one proto-cluster: every bin from its first to its last
    # peak is above the threshold
    for e, npk in enumerate((40, 40, 25)):
        h = ref["hist"][e]
        assert ref["n"][e] == npk
        lo, hi = ref["lo"][e, 0], ref["hi"][e, npk - 1]
        assert np.all(h[lo:hi + 1] > p.bin_threshold), e
    cfg = dict(split_mode=pv.SPLIT_RECURSIVE)
    if path == "plain":
        cfg["path"] = pv.PATH_PLAIN
    ctx = pv.Context(device=0, **cfg)
    s, v = G.gpu_find_fit(ctx, batch)
    ctx.close()
    G.assert_find_equal(s, ref, batch)


def _long_event(n_broad=840, z0=-290.0, step=0.5, peaks=14):
    """One event whose histogram is a single proto-cluster of about 1,700 bins:
    broad pp tracks (sigma_poca 1.2 mm) every 0.5 mm over 420 mm lift every bin
    above the threshold, and narrow peaks of 12 + k tracks every 29 mm split it."""
    t = np.array([[0.3, 0.0]])
    ev = []
    for j in range(n_broad):
        z = z0 + step * j
        ev.append(synthetic.straight_tracks((0.0, 0.0, z), t, [z], cov_xx=(1.2 * 0.3) ** 2,
                                            cov_tt=1e-14))
    for k in range(peaks):
        z = z0 + 15.0 + 29.0 * k + 0.125
        m = 12 + k
        ev.append(synthetic.straight_tracks((0.0, 0.0, z), np.repeat(t, m, 0), np.full(m, z),
                                            cov_xx=(0.05 * 0.3) ** 2, cov_tt=1e-14))
    return {k: np.concatenate([e[k] for e in ev]) for k in synthetic.TRACK_FIELDS}


@pytest.mark.parametrize("path", ["fused", "plain"])
def test_recursive_split_longer_than_its_scratch_on_the_gpu(pv, path):
    """The recursive split's scratch in the find kernel holds 1,536 bins of
    proto-clusters; a longer one splits without scratch (each piece found by
    descending from the top), one that still fits beside it with: seeds,
    bounds and assignments bit-exact with the oracle either way."""
    batch = synthetic.batch_from_events([_long_event(), _comb_event(), _long_event(peaks=9),
                                         _comb_event(25, rising=False)])
    p = oracle.default_params(split_mode=1)
    ref = oracle.find_batch(batch, p, want_hist=True)
    h = ref["hist"][0]
    above = h > p.bin_threshold
    assert int(above.sum()) > 1536 and ref["n"][0] == 14
    cfg = dict(split_mode=pv.SPLIT_RECURSIVE)
    if path == "plain":
        cfg["path"] = pv.PATH_PLAIN
    ctx = pv.Context(device=0, **cfg)
    s, v = G.gpu_find_fit(ctx, batch)
    ctx.close()
    G.assert_find_equal(s, ref, batch)
