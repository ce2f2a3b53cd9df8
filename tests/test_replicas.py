"""The N > 1 path of bench.py: independent replicas, one per rank, with no
data-path collective; only the timing reductions cross ranks.  Run as two
gloo ranks on the CPU."""
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # Rank r processed 1000 (r + 1) units in 10 (r + 1) ms.
        units, ms = 1000.0 * (rank + 1), 10.0 * (rank + 1)
        out.put((rank, bench.reduce_max(ms, world), bench.reduce_sum(units, world),
                 bench.replica_rate(units, ms, world)))
        bench.barrier(world)
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_aggregate_whole_job_rate():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(2))
    for rank, mx, sm, rate in res:
        assert mx == 20.0 and sm == 3000.0
        assert rate == pytest.approx(3000.0 / 0.020)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(5.0, 1) == 5.0 and bench.reduce_sum(7.0, 1) == 7.0
    assert bench.replica_rate(100.0, 10.0, 1) == pytest.approx(1e4)
