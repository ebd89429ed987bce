"""The allocation-free entry point, pv_find_fit_static.

It serves callers that cannot allocate device memory while they run (a
real-time loop cannot afford cudaMalloc / cudaFree, which may synchronise the
whole device; some applications hand all device memory to their own
allocator at start-up).  It runs the same fused find + fit as pv_fit_batch
with seeds == NULL, but with the library's static device scratch.  Here its
output is compared, through the C ABI, with the allocating entry point's on
two calls in a row, within the parity tolerances, and an oversized batch must
be refused with PV_ERR_CAPACITY.
"""
import numpy as np
import pytest

from paper_2412_14966_gb300 import synthetic
from tests import gpu_common as G

pytestmark = pytest.mark.gpu


def _compare(out: dict, ref: dict, batch):
    E = batch.n_events
    assert np.array_equal(out["n_per_event"][:E], ref["n_per_event"][:E])
    assert np.array_equal(out["event_status"][:E], ref["event_status"][:E])
    assert np.array_equal(out["track_vertex"][:batch.n_tracks], ref["track_vertex"][:batch.n_tracks])
    for e in range(E):
        n = ref["n_per_event"][e]
        assert np.array_equal(out["status"][e, :n], ref["status"][e, :n]), e
        assert np.array_equal(out["n_tracks"][e, :n], ref["n_tracks"][e, :n]), e
        ok = (ref["status"][e, :n] & 4) == 0        # singular vertices carry no fit
        assert np.all(np.abs(out["x"][e, :n] - ref["x"][e, :n])[ok] < G.TOL_XY), e
        assert np.all(np.abs(out["y"][e, :n] - ref["y"][e, :n])[ok] < G.TOL_XY), e
        assert np.all(np.abs(out["z"][e, :n] - ref["z"][e, :n])[ok] < G.TOL_Z), e
        for k in np.nonzero(ok)[0]:
            assert G.cov_error(out["cov"][e, k], ref["cov"][e, k]) < G.TOL_COV, (e, k)


def _scratch_bytes(batch, capacity=64):
    """Scratch a batch needs: 31 B per track (fit inputs 16 + 8, center bin
    2, vertex index 1, vertex-ordered track index 4), and 32 B per entry of
    the four vertex work lists (size classes of at least 1, 9, 17 and 33
    tracks; each holds at most min(tracks / that minimum, slots), slots being
    the smaller of tracks and events x capacity), each array 16-byte aligned."""
    def r16(v):
        return (v + 15) // 16 * 16
    n = batch.n_tracks
    slots = min(n, batch.n_events * capacity)
    work = sum(min(n // m, slots) for m in (1, 9, 17, 33))
    return 256 + r16(16 * n) + r16(8 * n) + r16(2 * n) + r16(n) + r16(4 * n) + r16(32 * work)


def test_static_scratch_entry_point_matches_allocating_one():
    import torch

    import paper_2412_14966_gb300 as pv
    from paper_2412_14966_gb300 import build
    build.build()
    ctx = pv.Context(device=0)
    # about 157k tracks, including events above 256 tracks (they use the
    # per-track scratch arrays); the batch's scratch fits in the 8 MiB array
    batch = synthetic.workload_nominal(n_events=1000, seed=11)
    assert _scratch_bytes(batch) <= 8 << 20 and (batch.event_sizes() > 256).any()
    tracks = pv.Tracks.from_batch(batch)
    ref = ctx.fit_batch(tracks)
    torch.cuda.synchronize()
    ref = ref.numpy()
    for _ in range(2):
        out = ctx.find_fit_static(tracks)
        torch.cuda.synchronize()
        _compare(out.numpy(), ref, batch)
    # a batch whose scratch would not fit is refused, not truncated
    big = synthetic.workload_nominal(n_events=1600, seed=12)
    assert _scratch_bytes(big) > 8 << 20
    with pytest.raises(pv.PVError) as err:
        ctx.find_fit_static(pv.Tracks.from_batch(big))
    assert err.value.code == pv.PV_ERR_CAPACITY
    ctx.close()
