"""Multi-rank path of bench.py on CPU: two gloo ranks, each running its own
independent resonators (weak scaling, no data-path collective); the job rate
counts every rank's work over the slowest rank's time."""
import os
import socket

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import sys
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    local_ms = 100.0 * (rank + 1)          # rank 1 is the slow one
    value, total_ms = bench.weak_scaling_rate(local_ms, 1000, world)
    # each rank's resonators are its own: seeds differ per rank
    seeds = [r.seed for r in bench.workload(rank)]
    q.put((rank, value, total_ms, seeds, bench.dist_env()))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_weak_scaling_rate_uses_the_slowest_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (_, v0, t0, s0, e0), (_, v1, t1, s1, e1) = out
    assert t0 == t1 == pytest.approx(200.0)
    assert v0 == v1 == pytest.approx(2 * 1000 / 0.2)
    assert set(s0).isdisjoint(s1)
    assert e0 == (0, 0, 2) and e1 == (1, 1, 2)
