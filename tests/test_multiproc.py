"""The N > 1 path of the benchmark is replicas only (independent solves per rank, no data-path collective);
its host-side aggregation — the max over ranks of the timed region and the whole-job throughput — runs
here on two CPU processes with the gloo backend."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    # rank r "timed" 100 + 50 r ms for 4 steps
    ms = bench.reduce_max(100.0 + 50.0 * rank, "cpu")
    out.put((rank, ms, bench.job_throughput(4, world, ms * 1e-3)))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_aggregate_with_gloo():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    world = 2
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, thr in res:
        assert ms == 150.0                       # the slowest rank's time on every rank
        assert thr == pytest.approx(2 * 4 / 0.150)  # all ranks' steps over that time


def test_single_process_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.5, "cpu") == 3.5
    assert bench.job_throughput(5, 1, 2.0) == 2.5
