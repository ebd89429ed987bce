"""The allocation-free entry point, pv_find_fit_static.

It serves callers that cannot allocate device memory while they run (a
real-time loop cannot afford cudaMalloc / cudaFree, which may synchronise the
whole device; some applications hand all device memory to their own
allocator at start-up).  It runs the same fused find + fit as pv_fit_batch
with seeds == NULL, but with the library's static device scratch.  Here it
runs first on a fresh context: two calls in a row, through the C ABI, must
leave the context without device memory and the device's free memory
unchanged, and give the allocating entry point's results bit for bit (same
kernels, and a vertex's result does not depend on where its scratch lives).
An oversized batch must be refused with PV_ERR_CAPACITY.
"""
import numpy as np
import pytest

from paper_2412_14966_gb300 import synthetic

pytestmark = pytest.mark.gpu

KEYS = ("x", "y", "z", "cov", "chi2", "ndof", "n_tracks", "n_iter", "status",
        "bin_lo", "bin_hi", "bin_max")


def _assert_identical(out: dict, ref: dict, batch):
    E = batch.n_events
    assert np.array_equal(out["n_per_event"][:E], ref["n_per_event"][:E])
    assert np.array_equal(out["event_status"][:E], ref["event_status"][:E])
    assert np.array_equal(out["track_vertex"][:batch.n_tracks], ref["track_vertex"][:batch.n_tracks])
    K = out["x"].shape[1]
    live = np.arange(K)[None, :] < ref["n_per_event"][:E, None]
    for k in KEYS:
        g = np.ascontiguousarray(out[k][:E]).view(np.int32)
        r = np.ascontiguousarray(ref[k][:E]).view(np.int32)
        if g.ndim == 3:
            bad = np.nonzero(live[..., None] & (g != r))
        else:
            bad = np.nonzero(live & (g != r))
        assert len(bad[0]) == 0, (k, bad[0][:5], bad[1][:5])


def _scratch_bytes(batch, capacity=64):
    """Scratch a batch needs: 31 B per track (fit inputs 16 + 8, center bin
    2, vertex index 1, place in vertex order 4), and 32 B per entry of the
    four vertex work lists (size classes of at least 1, 9, 17 and 33 tracks;
    each holds at most min(tracks / that minimum, slots), slots being the
    smaller of tracks and events x capacity), each array 16-byte aligned."""
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
    # about 157k tracks, including events above 256 tracks (they use the
    # per-track scratch arrays); the batch's scratch fits in the 8 MiB array
    batch = synthetic.workload_nominal(n_events=1000, seed=11)
    assert _scratch_bytes(batch) <= 8 << 20 and (batch.event_sizes() > 256).any()
    tracks = pv.Tracks.from_batch(batch)
    outs = [pv.Vertices.empty(batch.n_events, batch.n_tracks) for _ in range(3)]
    ctx = pv.Context(device=0)
    # one call on a few events loads the kernels (the driver may allocate
    # device memory for code on a first launch)
    warm = synthetic.workload_small(n_events=8, seed=3)
    ctx.find_fit_static(pv.Tracks.from_batch(warm))
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    got = []
    for i in range(2):
        ctx.find_fit_static(tracks, out=outs[i])
        torch.cuda.synchronize()
        got.append(outs[i].numpy())
    assert torch.cuda.mem_get_info()[0] == free0
    assert ctx.device_bytes() == 0
    # the allocating entry point on its own context, bit for bit
    ref_ctx = pv.Context(device=0)
    ref_ctx.fit_batch(tracks, out=outs[2])
    torch.cuda.synchronize()
    assert ref_ctx.device_bytes() > 0
    ref = outs[2].numpy()
    for g in got:
        _assert_identical(g, ref, batch)
    # a batch whose scratch would not fit is refused, not truncated
    big = synthetic.workload_nominal(n_events=1600, seed=12)
    assert _scratch_bytes(big) > 8 << 20
    with pytest.raises(pv.PVError) as err:
        ctx.find_fit_static(pv.Tracks.from_batch(big))
    assert err.value.code == pv.PV_ERR_CAPACITY
    ref_ctx.close()
    ctx.close()
