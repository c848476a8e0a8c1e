"""The N > 1 path of bench.py (replicas only: each rank solves its own copy,
no data-path collective) on CPU with the gloo backend, world size 2: the
timing is the max over ranks and the work is summed."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench._barrier()                 # the barrier around every timed region
    dev_ms = 100.0 + 50.0 * rank     # rank 1 is slower
    e2e = 1.0 + rank
    work = 10.0 * (rank + 1)
    out = bench.aggregate_replicas(dev_ms, e2e, work, world, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, out))


def test_replica_aggregation_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert res[r] == (150.0, 2.0, 30.0)


def test_single_rank_passthrough():
    import bench
    assert bench.aggregate_replicas(5.0, 0.5, 7, 1) == (5.0, 0.5, 7)


def test_reference_arm_only_rank0_reports(monkeypatch):
    import bench
    args = type("A", (), dict(workload="full8", cpu_rows=100, warmup=0, steps=1))()
    assert bench.run_reference(args, 1, 2) is None


def test_barrier_is_a_no_op_in_one_process():
    import bench
    assert not dist.is_initialized()
    bench._barrier()
