"""The N > 1 path of bench.py on CPU: world-size-2 gloo process groups.

Every rank runs its own replica of the workload (no data-path collective);
the only cross-rank steps are barriers and the maximum of the timed
interval, and the reference arm runs on rank 0 alone.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    mine = [3.5, 7.25][rank]
    got = bench.max_over_ranks(mine)
    dist.barrier()
    ws, r, local = bench.dist_env()
    value = bench.job_throughput(1e9, ws, 10, got)
    # the reference arm: rank 0 only; others return without work
    class A:
        steps, warmup, gpus = 1, 0, world
    ran = None
    if r != 0:
        bench.run_reference(A())
        ran = "skipped"
    q.put((rank, got, ws, r, local, value, ran))
    dist.destroy_process_group()


@pytest.mark.timeout(120)
def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=100) for _ in procs)
    for p in procs:
        p.join(timeout=30)
        assert p.exitcode == 0
    for rank, got, ws, r, local, value, ran in out:
        assert got == 7.25 and ws == 2 and r == rank == local
        assert value == pytest.approx(1e9 * 2 * 10 / 7.25e-3 / 1e9)
    assert out[1][6] == "skipped"


def test_single_rank_is_a_no_op():
    import bench
    assert bench.max_over_ranks(4.0) == 4.0
    assert bench.job_throughput(2e9, 1, 5, 1000.0) == pytest.approx(10.0)
