"""The N > 1 path of bench.py on CPU: two gloo ranks, each with its own replica
of the workload, meet only at the maximum of their step times; the job's
throughput is the units all ranks processed over the slowest rank's time."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    try:
        local_ms = 10.0 + 5.0 * rank
        mx = bench.max_over_ranks(local_ms, dist)
        sysr = bench.replica_workload(rank)
        rate = bench.aggregate_rate(sysr.n * 12, mx, world)
        out.put((rank, mx, rate, float(sysr.x[0, :16].sum())))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_max_time_and_aggregate():
    world = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][1] == res[1][1] == 15.0                   # both ranks see the slowest time
    n = 256000
    assert res[0][2] == pytest.approx(world * n * 12 / 0.015)
    assert res[0][3] != res[1][3]                           # independent replicas (own seeds)
