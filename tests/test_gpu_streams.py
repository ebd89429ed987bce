"""Calls on one context from several CUDA streams: the context keeps one set
of scratch memory per stream, so device calls whose work overlaps on the GPU
do not share counters, work lists or per-track arrays.  Two batches run again
and again on two streams at once give the results they give one after the
other, bit for bit, on the fused and the plain path and for the multi-vertex
fit."""
import numpy as np
import pytest

from paper_2412_14966_gb300 import synthetic

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "z", "cov", "chi2", "ndof", "n_tracks", "n_iter", "status")


def _same(a: dict, b: dict, batch):
    E = batch.n_events
    assert np.array_equal(a["n_per_event"][:E], b["n_per_event"][:E])
    assert np.array_equal(a["track_vertex"][:batch.n_tracks], b["track_vertex"][:batch.n_tracks])
    K = a["x"].shape[1]
    live = np.arange(K)[None, :] < b["n_per_event"][:E, None]
    for k in KEYS:
        g = np.ascontiguousarray(a[k][:E]).view(np.int32)
        r = np.ascontiguousarray(b[k][:E]).view(np.int32)
        m = live[..., None] if g.ndim == 3 else live
        assert not np.any(m & (g != r)), k


@pytest.mark.parametrize("entry", ["fused", "plain", "multi"])
def test_overlapping_calls_on_two_streams(entry):
    import torch

    import paper_2412_14966_gb300 as pv
    from paper_2412_14966_gb300 import build
    build.build()
    cfg = dict(path=pv.PATH_PLAIN) if entry == "plain" else {}
    ctx = pv.Context(device=0, **cfg)
    batches = [synthetic.workload_nominal(n_events=3000, seed=31),
               synthetic.workload_mixture(n_events=3000, seed=32)]
    tracks = [pv.Tracks.from_batch(b) for b in batches]
    run = ctx.fit_multi if entry == "multi" else ctx.fit_batch
    main = torch.cuda.current_stream()
    refs = []
    for t, b in zip(tracks, batches):
        o = pv.Vertices.empty(b.n_events, b.n_tracks)
        run(t, out=o, stream=main)
        torch.cuda.synchronize()
        refs.append(o.numpy())
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = [pv.Vertices.empty(b.n_events, b.n_tracks) for b in batches]
    for rep in range(4):
        for i in range(2):
            run(tracks[i], out=outs[i], stream=streams[i])
        torch.cuda.synchronize()
        for i in range(2):
            _same(outs[i].numpy(), refs[i], batches[i])
    ctx.close()
