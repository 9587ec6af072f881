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


def test_roofline_of_the_dominant_class_and_every_class():
    """bench.roofline: the dominant class (by time) against its bound's peak, and every class beside it."""
    import bench
    stats = {"gemm": {"ms": 200.0, "launches": 4000, "flops": 1.0e11, "bytes": 1.0e9},
             "eigen": {"ms": 260.0, "launches": 1800, "flops": 1.2e8, "bytes": 1.0e6},
             "tt_misc": {"ms": 30.0, "launches": 4000, "flops": 2.0e8, "bytes": 3.0e9},
             "khatri_rao": {"ms": 0.0, "launches": 0, "flops": 0.0, "bytes": 0.0}}
    out = bench.roofline(stats, fp64_peak=1.25)
    assert out["kernel_class"] == "eigen" and out["bound"] == "alu"
    assert abs(out["achieved"] - 1.2e8 / 0.26 / 1e12) <= 1e-12
    assert abs(out["frac"] - out["achieved"] / 1.25) <= 1e-12
    assert abs(out["share"] - 260.0 / 490.0) <= 1e-12
    by = out["by_class"]
    assert set(by) == {"gemm", "eigen", "tt_misc"}  # classes without launches are left out
    assert by["gemm"]["bound"] == "alu" and abs(by["gemm"]["frac"] - 0.4) <= 1e-4
    peaks, _ = bench.measured_peaks()
    assert by["tt_misc"]["bound"] == "hbm" and by["tt_misc"]["unit"] == "GB/s"
    assert abs(by["tt_misc"]["achieved"] - 100.0) <= 0.01
    assert abs(by["tt_misc"]["frac"] - 100.0 / float(peaks["hbm_gbs"])) <= 1e-4


def test_default_workload_has_its_stored_oracle_solve(monkeypatch):
    """The default bench options match the oracle's stored solve (tests/golden), so the CPU baseline and the
    reference arm time the same workload instead of reporting it unavailable; the stored counts are consistent."""
    import sys
    import bench
    monkeypatch.setattr(sys, "argv", ["bench.py"])
    args = bench.parse()
    got = bench.oracle_applies_per_solve(args)
    assert got is not None
    applies, g = got
    assert applies == sum(g["applies_by_rank"].values())
    assert set(g["applies_by_rank"]) <= {str(r) for r in range(args.rank_start, args.rank + 1, args.rank_step)}
    assert g["rel_resid"] <= args.tt_tol
