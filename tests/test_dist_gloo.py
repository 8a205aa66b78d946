"""The multi-replica path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Under torchrun every rank runs an independent terrain ("replicas only": one
terrain has no exchange step); the only cross-rank work is the reduction of the
timings (max over ranks) and of the processed particle-steps (sum over ranks),
which these ranks exercise with the same function the benchmark calls.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, local = bench._dist()
        # rank-dependent timings and work: rank 1 is the slower replica
        times, units = bench.aggregate(w, [10.0 + 5.0 * r, 2.0 - r], 1000.0 * (r + 1))
        dist.barrier()
        q.put((r, w, local, times, units))
    finally:
        dist.destroy_process_group()


def _run(world):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return sorted(out)


def test_two_rank_reduction_takes_max_time_and_total_work():
    out = _run(2)
    for r, (rank, w, local, times, units) in enumerate(out):
        assert (rank, w, local) == (r, 2, r)
        assert times == [15.0, 2.0]          # slowest replica's timed region and e2e loop
        assert units == 3000.0               # particle-steps of both replicas
    # whole-job throughput as the benchmark reports it
    assert out[0][4] / (out[0][3][0] * 1e-3) == pytest.approx(3000.0 / 0.015)


def test_single_rank_needs_no_process_group():
    import bench
    times, units = bench.aggregate(1, [3.0, 4.0], 123.0)
    assert times == [3.0, 4.0] and units == 123.0
