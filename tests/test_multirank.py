"""The multi-rank path of bench.py on CPU (gloo, world size 2).

The GEMM is not sharded (replicas only), so the only cross-rank steps are the
barrier around the timed region and the max over ranks of the elapsed time;
the whole-job value is the total work of all ranks over the slowest rank's
time."""
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
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    bench.barrier(world)
    secs = 1.0 + rank          # rank 1 is the slow one
    value, t_max = bench.aggregate(1e12, 4, secs, world)
    bench.barrier(world)
    dist.destroy_process_group()
    q.put((rank, value, t_max))


@pytest.mark.timeout(120)
def test_two_rank_aggregation_uses_slowest_rank():
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
    for rank, value, t_max in out:
        assert t_max == 2.0                        # max over ranks
        assert abs(value - 1e12 * 4 * 2 / 2.0 / 1e12) < 1e-12   # 4 TFLOP/s whole job
