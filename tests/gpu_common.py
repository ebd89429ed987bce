"""Shared helpers of the GPU parity tests: run the CUDA path through the C ABI
and compare with the oracle."""
from __future__ import annotations

import numpy as np

import oracle

TOL_XY = 1e-4     # mm (0.1 um)
TOL_Z = 5e-4      # mm (0.5 um)
TOL_COV = 1e-4    # relative to sqrt(C_ii C_jj)

COV_IDX = ((0, 0), (0, 1), (1, 1), (0, 2), (1, 2), (2, 2))


def oracle_params_for(ctx_cfg: dict | None = None, beam=(0.0, 0.0, 0.0, 0.0), **kw):
    p = oracle.default_params(x_b=beam[0], y_b=beam[1], tx_b=beam[2], ty_b=beam[3])
    for k, v in (ctx_cfg or {}).items():
        if hasattr(p, k):
            setattr(p, k, v)
    for k, v in kw.items():
        setattr(p, k, v)
    return p


def gpu_find_fit(ctx, batch, fused=True, two_step=False):
    """Returns (seeds dict, vertices dict) as numpy, from the C ABI."""
    import torch

    import paper_2412_14966_gb300 as pv
    tracks = pv.Tracks.from_batch(batch)
    seeds = ctx.find_batch(tracks)
    if fused:
        verts = ctx.fit_batch(tracks)
    else:
        verts = ctx.fit_batch(tracks, seeds)
    torch.cuda.synchronize()
    return seeds.numpy(), verts.numpy()


def assert_find_equal(gpu: dict, ref: dict, batch, events=None):
    """Seeds, cluster bounds and track assignment: bit-exact."""
    E = batch.n_events
    events = range(E) if events is None else events
    assert np.array_equal(gpu["n_per_event"][:E], ref["n"]), _first_diff(gpu["n_per_event"][:E], ref["n"])
    assert np.array_equal(gpu["event_status"][:E], ref["event_status"])
    tv = gpu["track_vertex"][:batch.n_tracks]
    assert np.array_equal(tv, ref["track_cluster"]), _first_diff(tv, ref["track_cluster"])
    for e in events:
        n = ref["n"][e]
        for k, rk in (("bin_lo", "lo"), ("bin_hi", "hi"), ("bin_max", "bin")):
            if k in gpu:
                assert np.array_equal(gpu[k][e, :n], ref[rk][e, :n]), (e, k)
        for k in ("x", "y", "z"):
            g = np.ascontiguousarray(gpu[k][e, :n]).view(np.int32)
            r = np.ascontiguousarray(ref[k][e, :n]).view(np.int32)
            assert np.array_equal(g, r), (e, k, gpu[k][e, :n], ref[k][e, :n])


def _first_diff(a, b):
    d = np.nonzero(a != b)[0]
    return f"first difference at {d[:5]}: {a[d[:5]]} vs {b[d[:5]]}" if len(d) else ""


def fit_mismatches(gpu: dict, ref: dict, n_seeds: np.ndarray, cond=None):
    """Per-vertex comparison.  Returns (list of (e, k) whose iteration counts
    differ, dict of worst errors over vertices with equal counts).  A
    covariance outside TOL_COV is accepted only for an ill-conditioned vertex
    (``cond`` = (batch, found, params); see cov_spread) within ILL_FACTOR times
    the oracle's own spread; those vertices are listed under "ill"."""
    worst = {"xy": 0.0, "z": 0.0, "cov": 0.0, "ill": []}
    differ = []
    for e in range(len(n_seeds)):
        for k in range(n_seeds[e]):
            gs, rs = int(gpu["status"][e, k]), int(ref["status"][e, k])
            g_sing, r_sing = bool(gs & oracle.SINGULAR), bool(rs & oracle.SINGULAR)
            assert g_sing == r_sing, (e, k, gs, rs)
            if r_sing:
                continue
            if gpu["n_iter"][e, k] != ref["n_iter"][e, k]:
                differ.append((e, k))
                continue
            worst["xy"] = max(worst["xy"], abs(gpu["x"][e, k] - ref["x"][e, k]),
                              abs(gpu["y"][e, k] - ref["y"][e, k]))
            worst["z"] = max(worst["z"], abs(gpu["z"][e, k] - ref["z"][e, k]))
            ce = cov_error(gpu["cov"][e, k], ref["cov"][e, k])
            if ce >= TOL_COV and cond is not None:
                spread = cov_spread(*cond, e, k)
                assert spread >= TOL_COV / ILL_FACTOR and ce < ILL_FACTOR * spread, (e, k, ce, spread)
                worst["ill"].append((e, k, ce, spread))
            else:
                worst["cov"] = max(worst["cov"], ce)
            assert gs == rs, (e, k, gs, rs, gpu["n_tracks"][e, k], ref["n_tracks"][e, k])
            assert gpu["n_tracks"][e, k] == ref["n_tracks"][e, k], (e, k)
    return differ, worst


def cov_error(g, r) -> float:
    """Largest |C_gpu - C_ref| / sqrt(C_ii C_jj) over the 6 elements."""
    diag = {0: r[0], 1: r[2], 2: r[5]}
    err = 0.0
    for q, (i, j) in enumerate(COV_IDX):
        err = max(err, abs(float(g[q]) - float(r[q])) / np.sqrt(diag[i] * diag[j]))
    return err


# An ill-conditioned covariance: one whose oracle value moves by more than
# TOL_COV / ILL_FACTOR when the vertex's binary32 track inputs move by one ulp.
# Binary32 per-track arithmetic cannot pin such a covariance to TOL_COV (a
# track with chi2 just below chi2_max, whose Tukey weight (1 - chi2/chi2_max)^2
# carries most of the z information, is the typical case); it is compared at
# ILL_FACTOR times that spread instead.
ILL_FACTOR = 10.0


def vertex_tracks(batch, found: dict, e: int, k: int) -> dict:
    b0, b1 = int(batch.offsets[e]), int(batch.offsets[e + 1])
    idx = b0 + np.nonzero(found["track_cluster"][b0:b1] == k)[0]
    return {kk: vv[idx] for kk, vv in batch.tracks.items()}


def cov_spread(batch, found: dict, p, e: int, k: int, n_draw: int = 8) -> float:
    """Largest change of the oracle's covariance of vertex (e, k) (cov_error
    measure) over n_draw refits whose binary32 track inputs are each moved by
    one ulp in a random direction."""
    t = vertex_tracks(batch, found, e, k)
    seed = (found["x"][e, k], found["y"][e, k], found["z"][e, k])
    base = oracle.fit_tracks(t, seed, p)
    rng = np.random.default_rng(1000 * e + k)
    worst = 0.0
    for _ in range(n_draw):
        tp = {}
        for kk, v in t.items():
            v = np.asarray(v, np.float32)
            up = rng.integers(0, 2, v.shape).astype(bool)
            tp[kk] = np.where(up, np.nextafter(v, np.float32(np.inf)),
                              np.nextafter(v, np.float32(-np.inf))).astype(np.float32)
        r = oracle.fit_tracks(tp, seed, p)
        if r["status"] & oracle.SINGULAR:
            continue
        worst = max(worst, cov_error(r["cov"], base["cov"]))
    return worst


def assert_fit_close(gpu, ref, n_seeds, tight_pair=None, cond=None):
    """Tolerances on every vertex whose iteration counts agree; the others are
    refitted on both sides to full convergence (``tight_pair`` = callable
    returning (gpu_tight, ref_tight)) and compared there.  ``cond`` =
    (batch, found, params) enables the ill-conditioned rule of
    fit_mismatches."""
    differ, worst = fit_mismatches(gpu, ref, n_seeds, cond)
    assert worst["xy"] < TOL_XY, worst
    assert worst["z"] < TOL_Z, worst
    assert worst["cov"] < TOL_COV, worst
    n_total = int(np.sum(n_seeds))
    if differ:
        assert tight_pair is not None, f"{len(differ)} iteration-count mismatches"
        # fixed points are compared where the paper's stopping rule was not decisive
        assert len(differ) <= max(3, 0.05 * n_total), (len(differ), n_total)
        gt, rt = tight_pair()
        for e, k in differ:
            assert abs(gt["x"][e, k] - rt["x"][e, k]) < TOL_XY, (e, k)
            assert abs(gt["y"][e, k] - rt["y"][e, k]) < TOL_XY, (e, k)
            assert abs(gt["z"][e, k] - rt["z"][e, k]) < TOL_Z, (e, k)
            assert cov_error(gt["cov"][e, k], rt["cov"][e, k]) < TOL_COV, (e, k)
    return worst, len(differ)


def _ulp_moved(t: dict, rng) -> dict:
    out = {}
    for kk, v in t.items():
        v = np.asarray(v, np.float32)
        up = rng.integers(0, 2, v.shape).astype(bool)
        out[kk] = np.where(up, np.nextafter(v, np.float32(np.inf)),
                           np.nextafter(v, np.float32(-np.inf))).astype(np.float32)
    return out


def mv_spread(batch, found: dict, p, e: int, k: int, n_draw: int = 8):
    """The multi-vertex analogue of cov_spread: the largest change of the
    oracle's fitted x/y, z (mm) and covariance of vertex (e, k) over n_draw
    refits of event e whose binary32 track inputs are each moved by one ulp
    (the seeds stay).  Returns (xy, z, cov)."""
    from paper_2412_14966_gb300 import synthetic
    b0, b1 = int(batch.offsets[e]), int(batch.offsets[e + 1])
    t = {kk: vv[b0:b1] for kk, vv in batch.tracks.items()}
    seeds = {kk: found[kk][e:e + 1] for kk in ("x", "y", "z")}
    seeds["n"] = found["n"][e:e + 1]
    base = oracle.mv_fit_batch(synthetic.batch_from_events([t]), seeds, p)
    rng = np.random.default_rng(1000 * e + k)
    wxy = wz = wc = 0.0
    for _ in range(n_draw):
        r = oracle.mv_fit_batch(synthetic.batch_from_events([_ulp_moved(t, rng)]), seeds, p)
        if r["status"][0, k] & oracle.SINGULAR:
            continue
        wxy = max(wxy, abs(r["x"][0, k] - base["x"][0, k]), abs(r["y"][0, k] - base["y"][0, k]))
        wz = max(wz, abs(r["z"][0, k] - base["z"][0, k]))
        wc = max(wc, cov_error(r["cov"][0, k], base["cov"][0, k]))
    return wxy, wz, wc
