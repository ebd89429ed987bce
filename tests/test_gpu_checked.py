"""The checked build (the library compiled with PV_CHECKED=1: its kernels test
the indices of their main shared- and global-memory accesses, skip and count
any that would leave its buffer) stands in for a memory checker.  On the
parity workloads, every path and both flavours, no index leaves its buffer,
and the results equal the default build's bit for bit (the checks change no
arithmetic).  The multi-vertex kernels write their binary32 sums as plain
expressions, which the compiler may contract into fused multiply-adds
differently when the checks change the surrounding code; their vertex lists
must agree and the positions meet the fit tolerances."""
import numpy as np
import pytest

from paper_2412_14966_gb300 import synthetic

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "cov", "n_tracks", "n_iter", "status")


def _batches():
    rng = np.random.default_rng(4)
    edge = [synthetic.straight_tracks((0.0, 0.0, 1.0), rng.uniform(-0.3, 0.3, (0, 2)), []),
            synthetic.straight_tracks((0.0, 0.0, 1.0), rng.uniform(-0.3, 0.3, (1, 2)), [3.0])]
    big = synthetic.generate(1, 11, mu=30.0, mean_tracks=28.0)
    edge.append({k: v for k, v in big.tracks.items()})
    return {
        "small": synthetic.workload_small(),
        "nominal": synthetic.workload_nominal(n_events=800, seed=6),
        "pileup": synthetic.generate(12, 3, mu=40.0, mean_tracks=28.0, name="pileup-12"),
        "overlay": synthetic.workload_overlay(n_events=300, seed=8),
        "edge": synthetic.batch_from_events(edge),
    }


def _collect(pv, batches):
    """Every entry point on every batch; numpy results keyed by (batch, what)."""
    import torch
    out = {}
    for name, b in batches.items():
        E = b.n_events
        t = pv.Tracks.from_batch(b)
        runs = [("fused", {}), ("plain", dict(path=pv.PATH_PLAIN)),
                ("x86", dict(split_mode=pv.SPLIT_RECURSIVE, profile_mode=pv.PROFILE_TEMPLATE))]
        for what, cfg in runs:
            ctx = pv.Context(device=0, **cfg)
            seeds = ctx.find_batch(t)
            two = ctx.fit_batch(t, seeds)
            fused = ctx.fit_batch(t)
            torch.cuda.synchronize()
            out[(name, what, "seeds")] = seeds.numpy()
            out[(name, what, "two_step")] = two.numpy()
            out[(name, what, "fused")] = fused.numpy()
            if what == "fused":
                out[(name, what, "multi")] = ctx.fit_multi(t).numpy()
                out[(name, what, "hist")] = {"h": ctx.histogram_batch(t).cpu().numpy()}
            if what == "x86":
                out[(name, what, "hist")] = {"h": ctx.histogram_batch(t).cpu().numpy()}
            torch.cuda.synchronize()
            ctx.close()
        out[(name, "n")] = (E, b.n_tracks)
    return out


def _close_multi(a, b, E):
    """Vertex counts equal; positions within 0.1 um (x, y) and 0.5 um (z) on
    all but a few vertices (slowly settling fits amplify rounding)."""
    if not np.array_equal(a["n_per_event"][:E], b["n_per_event"][:E]):
        return False
    live = np.arange(a["x"].shape[1])[None, :] < a["n_per_event"][:E, None]
    bad = np.zeros(int(live.sum()), bool)
    for k, tol in (("x", 1e-4), ("y", 1e-4), ("z", 5e-4)):
        u, v = a[k][:E][live].astype(np.float64), b[k][:E][live].astype(np.float64)
        both_nan = np.isnan(u) & np.isnan(v)     # singular vertices carry no position
        with np.errstate(invalid="ignore"):
            bad |= ~both_nan & ~(np.abs(u - v) < tol)
    return bad.sum() <= max(2, 0.002 * live.sum())


def _same(a, b, E, n_tracks):
    if "h" in a:
        return np.array_equal(a["h"], b["h"])
    if not np.array_equal(a["n_per_event"][:E], b["n_per_event"][:E]):
        return False
    if not np.array_equal(a["track_vertex"][:n_tracks], b["track_vertex"][:n_tracks]):
        return False
    for e in range(E):
        n = a["n_per_event"][e]
        for k in FIELDS:
            if k in a and not np.array_equal(a[k][e, :n], b[k][e, :n]):
                return False
    return True


def test_checked_build_finds_no_bad_index_and_changes_nothing():
    import paper_2412_14966_gb300 as pv
    from paper_2412_14966_gb300 import build
    default_lib = build.build()
    checked_lib = build.build(checked=True)
    batches = _batches()
    saved = pv.LIB_PATH
    try:
        pv._LIB = None
        pv.LIB_PATH = default_lib
        assert pv.check_report() == (False, 0, 0)
        ref = _collect(pv, batches)
        pv._LIB = None
        pv.LIB_PATH = checked_lib
        assert pv.check_report() == (True, 0, 0)
        got = _collect(pv, batches)
        report = pv.check_report()
    finally:
        pv._LIB = None
        pv.LIB_PATH = saved
    assert report == (True, 0, 0), report
    differ = [k for k in ref if k[1] != "n" and k[2] != "multi" and
              not _same(ref[k], got[k], *ref[(k[0], "n")])]
    differ += [k for k in ref if k[1] != "n" and k[2] == "multi" and
               not _close_multi(ref[k], got[k], ref[(k[0], "n")][0])]
    assert not differ, differ
