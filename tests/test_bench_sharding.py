"""The multi-GPU benchmark's host logic on two gloo ranks (CPU): every rank
takes its own independent events (no data-path exchange), the whole-job
figure is the sum of the ranks' events over the slowest rank's time, and the
reference arm runs on rank 0 only.  The method treats events independently,
so the ranks' per-shard results equal the oracle on the concatenated shards."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
N_EV = 24
STEPS = 7


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist = bench._init_dist(world, backend="gloo")
    batch = bench.shard_workload(rank, n_events=N_EV)
    seconds = 1.0 + 0.5 * rank                     # rank 1 is the slow one
    events_all, total_s, value = bench.aggregate(dist, float(batch.n_events * STEPS), seconds)
    # the reference arm: ranks other than 0 leave at once without output
    class A:
        steps, warmup = 1, 0
    ref_rc = bench.run_reference(A) if rank != 0 else 0
    f, fit = oracle.find_fit(batch, oracle.default_params())
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), events_all=events_all, total_s=total_s,
             value=value, ref_rc=ref_rc, z=batch.tracks["z"], n=f["n"], tv=f["track_cluster"],
             vz=fit["z"], vx=fit["x"])
    bench._barrier(dist)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_aggregate(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r = [np.load(tmp_path / f"rank{i}.npz") for i in range(world)]
    for q in r:
        assert float(q["events_all"]) == world * N_EV * STEPS
        assert float(q["total_s"]) == 1.5
        assert float(q["value"]) == pytest.approx(world * N_EV * STEPS / 1.5)
    assert int(r[1]["ref_rc"]) == 0
    # independent shards: different events on each rank
    assert not np.array_equal(r[0]["z"][:50], r[1]["z"][:50])
    # per-shard results equal the oracle on the two shards run as one batch
    sys.path.insert(0, ROOT)
    import bench
    both = bench.shard_workload(0, N_EV).concat(bench.shard_workload(1, N_EV))
    f, fit = oracle.find_fit(both, oracle.default_params())
    assert np.array_equal(f["n"], np.concatenate([r[0]["n"], r[1]["n"]]))
    assert np.array_equal(f["track_cluster"], np.concatenate([r[0]["tv"], r[1]["tv"]]))
    K = fit["z"].shape[1]
    for i in range(world):
        k = r[i]["vz"].shape[1]
        assert k <= K
        sl = slice(i * N_EV, (i + 1) * N_EV)
        assert np.array_equal(fit["z"][sl, :k], r[i]["vz"])
        assert np.array_equal(fit["x"][sl, :k], r[i]["vx"])


def test_reference_worker_takes_a_bounded_sample():
    """A reference-arm worker processes the first `take` events of its range
    (its whole range when take is None), reps times, and counts them."""
    sys.path.insert(0, ROOT)
    import bench
    oracle.build()
    bench._pool_init(2, N_EV)
    half = N_EV // 2
    assert bench._pool_run((0, 1, None)) == half
    assert bench._pool_run((1, 2, 3)) == 6
    assert bench._pool_run((1, 1, 10 * N_EV)) == half
