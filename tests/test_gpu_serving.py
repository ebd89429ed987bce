"""Serving through pv_submit / pv_poll: requests of uneven size are admitted as
the device memory pool frees up, their events run side by side in the
persistent serving kernel, and every result is bit-identical to the same
request run alone.  The serving kernel's wait for work is bounded: with
nothing submitted it ends on its own (PV_ERR_TIMEOUT) and the context stays
usable."""
import time

import numpy as np
import pytest

from paper_2412_14966_gb300 import synthetic

pytestmark = pytest.mark.gpu

FIELDS = ("x", "y", "z", "cov", "chi2", "ndof", "n_tracks", "n_iter", "status")


def _requests(pv, n_req, seed):
    """Device-resident requests drawn from the uneven mixture workload."""
    rng = np.random.default_rng(seed)
    mix = synthetic.workload_mixture(n_events=3000, seed=seed)
    reqs = []
    start = 0
    for _ in range(n_req):
        k = int(rng.integers(1, 400))
        ev = np.arange(start, start + k) % mix.n_events
        start += k
        b = mix.subset(ev)
        reqs.append((b, pv.Tracks.from_batch(b)))
    return reqs


def _same(a: dict, b: dict, batch):
    E = batch.n_events
    assert np.array_equal(a["n_per_event"][:E], b["n_per_event"][:E])
    assert np.array_equal(a["track_vertex"][:batch.n_tracks], b["track_vertex"][:batch.n_tracks])
    for e in range(E):
        n = a["n_per_event"][e]
        for k in FIELDS:
            assert np.array_equal(a[k][e, :n], b[k][e, :n]), (k, e)


def _wait(ctx, tickets, limit_s=60.0):
    t0 = time.time()
    pending = set(tickets)
    while pending:
        for t in list(pending):
            if ctx.poll(t):
                pending.discard(t)
        assert time.time() - t0 < limit_s, f"{len(pending)} requests not done"
        time.sleep(0.0005)


def test_served_results_equal_alone_results():
    import torch

    import paper_2412_14966_gb300 as pv
    from paper_2412_14966_gb300 import build
    build.build()
    reqs = _requests(pv, 24, seed=5)
    alone = pv.Context(device=0)
    ref = []
    for b, t in reqs:
        ref.append(alone.fit_batch(t).numpy())
    torch.cuda.synchronize()
    alone.close()
    # a pool that holds only a few requests at a time forces queueing
    biggest = max(b.n_tracks for b, _ in reqs)
    ctx = pv.Context(device=0, pool_bytes=int(3 * (48 * biggest + 32 * 64 * 400)))
    outs = [pv.Vertices.empty(b.n_events, b.n_tracks) for b, _ in reqs]
    tickets = []
    for (b, t), o in zip(reqs, outs):
        while True:
            rc, tk = ctx.submit_nowait(t, o)
            if rc == pv.PV_OK:
                tickets.append(tk)
                break
            time.sleep(0.0002)      # queue full: let requests finish
    _wait(ctx, tickets)
    torch.cuda.synchronize()
    for (b, _), o, r in zip(reqs, outs, ref):
        _same(o.numpy(), r, b)
    lat = [ctx.latency_ns(t) for t in tickets]
    assert all(v > 0 for v in lat)
    with pytest.raises(pv.PVError) as err:       # a retired ticket is unknown
        ctx.poll(tickets[0])
    assert err.value.code == pv.PV_ERR_NOTFOUND
    ctx.close()


def test_request_larger_than_pool_is_refused():
    import paper_2412_14966_gb300 as pv
    ctx = pv.Context(device=0, pool_bytes=1 << 20)
    b = synthetic.workload_nominal(n_events=2000, seed=3)
    t = pv.Tracks.from_batch(b)
    o = pv.Vertices.empty(b.n_events, b.n_tracks)
    with pytest.raises(pv.PVError) as err:
        ctx.submit(t, o)
    assert err.value.code == pv.PV_ERR_NOMEM
    # a small request still goes through the same context
    small = synthetic.workload_small(n_events=5, seed=4)
    ts = pv.Tracks.from_batch(small)
    os_ = pv.Vertices.empty(small.n_events, small.n_tracks)
    tk = ctx.submit(ts, os_)
    _wait(ctx, [tk])
    ctx.close()


def test_interleaved_submit_and_poll_keeps_results():
    """Requests submitted while earlier ones run (continuous batching)."""
    import torch

    import paper_2412_14966_gb300 as pv
    reqs = _requests(pv, 40, seed=9)
    alone = pv.Context(device=0)
    ref = [alone.fit_batch(t).numpy() for _, t in reqs]
    torch.cuda.synchronize()
    alone.close()
    ctx = pv.Context(device=0)
    outs = [pv.Vertices.empty(b.n_events, b.n_tracks) for b, _ in reqs]
    live = []
    done = []
    for i, ((b, t), o) in enumerate(zip(reqs, outs)):
        live.append((i, ctx.submit(t, o)))
        # poll a little between arrivals
        for j, tk in list(live):
            if ctx.poll(tk):
                live.remove((j, tk))
                done.append(j)
    _wait(ctx, [tk for _, tk in live])
    torch.cuda.synchronize()
    for (b, _), o, r in zip(reqs, outs, ref):
        _same(o.numpy(), r, b)
    ctx.close()


def test_idle_server_ends_on_its_own_and_the_context_stays_usable():
    """A serving kernel started with no request waits for work at most its idle
    bound (here max_spin_ns = 0.2 ms), then ends with PV_ERR_TIMEOUT; a request
    submitted afterwards starts it again and completes with the batched
    path's results."""
    import torch

    import paper_2412_14966_gb300 as pv
    ctx = pv.Context(device=0, max_spin_ns=200_000)
    ctx.serve_start()
    t0 = time.time()
    while True:
        running, last = ctx.serve_status()
        if not running:
            break
        assert time.time() - t0 < 10.0, "serving kernel did not end"
        time.sleep(0.001)
    assert last == pv.PV_ERR_TIMEOUT
    b = synthetic.workload_mixture(n_events=300, seed=11)
    t = pv.Tracks.from_batch(b)
    ref_ctx = pv.Context(device=0)
    ref = ref_ctx.fit_batch(t).numpy()
    ref_ctx.close()
    o = pv.Vertices.empty(b.n_events, b.n_tracks)
    tk = ctx.submit(t, o)
    _wait(ctx, [tk])
    torch.cuda.synchronize()
    _same(o.numpy(), ref, b)
    assert ctx.latency_ns(tk) > 0
    ctx.close()


def test_serving_follows_the_context_settings():
    """The serving kernel runs the context's flavour and accumulation mode:
    x86 flavour with binary64 sums, bit-identical to the batched path."""
    import torch

    import paper_2412_14966_gb300 as pv
    cfg = dict(split_mode=pv.SPLIT_RECURSIVE, profile_mode=pv.PROFILE_TEMPLATE,
               accum_mode=pv.ACCUM_FP64)
    reqs = _requests(pv, 6, seed=13)
    alone = pv.Context(device=0, **cfg)
    ref = [alone.fit_batch(t).numpy() for _, t in reqs]
    torch.cuda.synchronize()
    alone.close()
    ctx = pv.Context(device=0, **cfg)
    outs = [pv.Vertices.empty(b.n_events, b.n_tracks) for b, _ in reqs]
    tickets = [ctx.submit(t, o) for (b, t), o in zip(reqs, outs)]
    _wait(ctx, tickets)
    torch.cuda.synchronize()
    for (b, _), o, r in zip(reqs, outs, ref):
        _same(o.numpy(), r, b)
    ctx.close()
