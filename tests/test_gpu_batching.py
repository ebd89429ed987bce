"""Batching: the fused path's launch shape (block sizes and grids, chosen by
hand or by the autotuner per event-size bucket) and CUDA-graph replay do not
change any result, bit for bit."""
import numpy as np
import pytest

from paper_2412_14966_gb300 import synthetic

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "cov", "chi2", "ndof", "n_tracks", "n_iter", "status")


def _run(ctx, tracks, pv, out=None):
    import torch
    o = ctx.fit_batch(tracks, out=out)
    torch.cuda.synchronize()
    return o.numpy()


def _same(a, b, batch):
    E = batch.n_events
    assert np.array_equal(a["n_per_event"][:E], b["n_per_event"][:E])
    assert np.array_equal(a["track_vertex"][:batch.n_tracks], b["track_vertex"][:batch.n_tracks])
    for e in range(E):
        n = a["n_per_event"][e]
        for k in FIELDS:
            assert np.array_equal(a[k][e, :n], b[k][e, :n]), (k, e)


def test_every_launch_shape_gives_identical_results():
    import paper_2412_14966_gb300 as pv
    from paper_2412_14966_gb300 import build
    build.build()
    batch = synthetic.workload_mixture(n_events=1500, seed=21)
    ctx = pv.Context(device=0)
    tracks = pv.Tracks.from_batch(batch)
    ref = _run(ctx, tracks, pv)
    bucket = 0
    for fi in (64, 96, 128, 256):
        for ft in (128, 256):
            ctx.set_launch_config(bucket, fi, ft)
            assert ctx.launch_config(tracks)[:2] == (fi, ft)
            _same(_run(ctx, tracks, pv), ref, batch)
    with pytest.raises(pv.PVError):
        ctx.set_launch_config(bucket, 100, 256)
    ctx.close()


def test_graph_replay_equals_direct_launch():
    import paper_2412_14966_gb300 as pv
    batch = synthetic.workload_nominal(n_events=2000, seed=22)
    direct = pv.Context(device=0)
    graph = pv.Context(device=0, use_graph=1)
    tracks = pv.Tracks.from_batch(batch)
    ref = _run(direct, tracks, pv)
    out = pv.Vertices.empty(batch.n_events, batch.n_tracks)
    for _ in range(3):                       # capture once, replay twice
        _same(_run(graph, tracks, pv, out=out), ref, batch)
    out2 = pv.Vertices.empty(batch.n_events, batch.n_tracks)   # new arguments: new graph
    _same(_run(graph, tracks, pv, out=out2), ref, batch)
    other = synthetic.workload_small(n_events=50, seed=23)
    t2 = pv.Tracks.from_batch(other)
    _same(_run(graph, t2, pv), _run(direct, t2, pv), other)
    direct.close()
    graph.close()


def test_autotuner_sets_the_bucket_of_its_sample():
    import paper_2412_14966_gb300 as pv
    ctx = pv.Context(device=0)
    small = synthetic.workload_nominal(n_events=3000, seed=24)          # ~159 tracks/event
    pileup = synthetic.generate(60, 25, mu=40.0, mean_tracks=28.0)      # ~1,270 tracks/event
    ts, tp = pv.Tracks.from_batch(small), pv.Tracks.from_batch(pileup)
    ref_s, ref_p = _run(ctx, ts, pv), _run(ctx, tp, pv)
    cfg_p = ctx.autotune(tp)
    assert cfg_p[0] in (64, 96, 128, 256) and cfg_p[1] in (128, 256)
    assert ctx.launch_config(ts)[:2] == (128, 256)        # bucket 0 untouched
    cfg_s = ctx.autotune(ts)
    assert cfg_s[0] in (64, 96, 128, 256) and cfg_s[1] in (128, 256)
    _same(_run(ctx, ts, pv), ref_s, small)
    _same(_run(ctx, tp, pv), ref_p, pileup)
    ctx.close()
