"""Benchmark: low-rank (TT) vs full-format Fourier–Galerkin homogenisation on GB300.

Workload (default): d = 3, N = 243 per axis, isotropic lognormal conductivity a = exp(g), g a seeded
periodic Gaussian random field (squared-exponential covariance, correlation length 0.2, variance 1,
seed 19020745), E = (1, 0, 0).  The coefficient is compressed on the GPU to TT rank r_A (default 10,
the coefficient rank the paper uses for its stochastic material) and the full-format solver gets the
expansion of that TT coefficient, so both solve the same problem.

One step = one complete TT solve from u = 0 at the metric's accuracy: the rank-adapting minimal-residual
iteration Sec. 4.3 proposes (truncation rank 10, raised by 5 up to the cap 20 whenever the residual stagnates,
restarting from the best iterate; the material and P~^-1 products truncated by the randomised rounding, every
other truncation deterministic), stopped when the relative residual reaches 3e-4 at the cap (A_eff's error is
quadratic in the field's, about 6 x the squared residual for E = e_1 here, so this reaches A_eff within 1e-6),
then A_eff: every hot-path stage — mode-wise gradient FFTs, material products, truncations, divergence sums,
exponential-sum preconditioner, TT inner products, A_eff.  value = TT solves per second over the timed steps (whole job:
summed over ranks under torchrun, timed by the slowest rank), uninstrumented; one extra profiled solve gives
the kernel classes and the roofline.  The full-format FP64 PCG solve (tol 1e-8) of the same problem is timed
beside it (p50/p99) and gives the A_eff reference; so is the LRFG_MIXED full solve.

Timing: W untimed warm-up steps, then K steps each bracketed by CUDA events on the library's stream,
with a 512 MiB buffer written between steps to flush L2 (the TT state is a few MiB and would otherwise
stay in L2).  nvidia-smi samples clocks during the timed region.

    python bench.py [--steps K] [--warmup W] [--rank r] [--sketch-over p] [--tt-tol t] [--N 243]
                    [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import collections
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "solves/s and CG op-applies/s at A_eff rel err ≤1e-6, low-rank vs full; p50/p99"
SEED = 19020745


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=5)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--N", type=int, default=243)
    p.add_argument("--rank", type=int, default=20, help="the rank cap of the TT solve")
    p.add_argument("--rank-start", type=int, default=10,
                   help="rank-adapting MinRes (Sec. 4.3): start rank (0: the fixed rank --rank throughout)")
    p.add_argument("--rank-step", type=int, default=5, help="rank increase when the residual stagnates")
    p.add_argument("--coeff-rank", type=int, default=10)
    p.add_argument("--pinv-eps", type=float, default=0.1)
    p.add_argument("--maxit", type=int, default=80)
    p.add_argument("--sketch-over", type=int, default=10,
                   help="oversampling of the randomised rounding of the products (0: deterministic rounding)")
    p.add_argument("--tt-tol", type=float, default=3e-4,
                   help="relative residual at which the TT solve stops (A_eff error ~ 4-6 x its square)")
    p.add_argument("--tensor-tol", type=float, default=2e-4,
                   help="relative residual of the six solves of the homogenised tensor (the ratio of A_eff's error "
                        "to the squared residual depends on E: about 6 for E = e_1, up to about 18 for e_2 here)")
    p.add_argument("--stop-on-increase", type=int, default=0,
                   help="also stop after this many iterations without a new smallest residual (1: the paper's rule, "
                        "Sec. 4.3; 0: off)")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-tensor", action="store_true",
                   help="leave out the homogenised tensor's six solves (a reported extra, not the timed step)")
    p.add_argument("--micro", type=int, default=8,
                   help="microstructures of the workload's recipe solved together in lockstep (0: skip)")
    p.add_argument("--format", choices=["tt", "tucker"], default="tt",
                   help="low-rank solution format of the timed solve (the coefficient is the same rank-10 TT; a "
                        "Tucker problem compresses it by HOSVD)")
    p.add_argument("--workload", choices=["c2", "c3", "c4", "c5"], default="c2",
                   help="c2: lognormal SE-GRF, coefficient TT rank 10 (default, N=243); c3: tanh-smoothed cube of "
                        "contrast 100, coefficient rank 2 (N=1215 unless --N is given); c4: a batch of seeded "
                        "microstructures of mixed N and rank through the serving executor; c5: a Poisson stream "
                        "of requests (d in {2,3}, N 63-729, rank tolerance 1e-6-1e-4) served as they arrive")
    p.add_argument("--count", type=int, default=64, help="c4: requests in the batch")
    p.add_argument("--group", type=int, default=8,
                   help="c4: requests of one shape the executor solves together in lockstep (1: one at a time)")
    p.add_argument("--c4-rank-step", type=int, default=1, help="c4: TT ranks drawn over the multiples of this step")
    p.add_argument("--c4-prec", choices=["fp64", "mixed"], default="fp64", help="c4: solve precision")
    p.add_argument("--c4-sketch-over", type=int, default=0,
                   help="c4: oversampling of the randomised rounding of the products (0: deterministic rounding)")
    p.add_argument("--workers", type=int, default=8, help="c4/c5: executor worker streams")
    p.add_argument("--rate", type=float, default=200.0, help="c5: mean arrival rate (requests/s)")
    p.add_argument("--rank-cap", type=int, default=30, help="c5: rank cap of the tolerance truncation")
    p.add_argument("--c3-full", choices=["none", "mixed", "fp64"], default="mixed",
                   help="c3: full-format anchor solve on the expanded coefficient")
    p.add_argument("--case", choices=["tt_apply", "tt_solve", "full_apply", "full_apply_mixed"], default=None,
                   help="run two operator applications (tt_solve: one TT solve, the timed step) of the workload and "
                        "exit (a small program for profilers)")
    return p.parse_args()


def reduce_max(value: float, device) -> float:
    """Max of value over the ranks of the default process group (the value itself without one): the timing
    rule for N > 1 replicas (every rank times its own steps; the job takes as long as the slowest)."""
    import torch
    import torch.distributed as dist
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of N independent replicas: all ranks' units over the slowest rank's time."""
    return world * units_per_rank / seconds


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def workload_config(args):
    fmt = "Tucker" if args.format == "tucker" else "TT"
    rnd = (f"randomised rounding of the products (oversampling {args.sketch_over})" if args.sketch_over > 0
           else "deterministic rounding")
    sched = (f"rank-adapting MinRes, rank {args.rank_start} -> {args.rank} in steps of {args.rank_step}"
             if args.rank_start > 0 else f"rank {args.rank} MinRes")
    return {"workload": f"d=3 N={args.N}^3 lognormal SE-GRF (l=0.2, var=1, seed {SEED}), E=(1,0,0); "
                        f"{fmt} {sched} ({rnd}, stop at relative residual {args.tt_tol:g}) "
                        f"vs full FP64 PCG (tol 1e-8)",
            "d": 3, "N": args.N, "coeff_tt_rank": args.coeff_rank, "format": args.format, "tt_rank": args.rank,
            "rank_start": args.rank_start, "rank_step": args.rank_step,
            "sketch_over": args.sketch_over, "tt_tol": args.tt_tol, "stop_on_increase": args.stop_on_increase,
            "pinv_eps": args.pinv_eps, "precision": "fp64", "l2": "flushed between steps (512 MiB write)",
            "sketch_seeds": f"0..{max(args.steps, 1) - 1}, one per timed step"}


def make_coefficient(N):
    from synthetic import lognormal_grf
    return lognormal_grf(3, N, ell=0.2, var=1.0, seed=SEED)


# -------------------------------------------------------------------------------------------------
# clocks
# -------------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = "index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, device):
        self.device = device
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.device}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [l for l in out.splitlines() if l.strip()]
        return False

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in getattr(self, "lines", []):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


# -------------------------------------------------------------------------------------------------
# roofline of the dominant kernel class
# -------------------------------------------------------------------------------------------------
def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# FP64 arithmetic classes are bound by the FP64 pipe.  Its rate is measured on the device at run time
# (lrfg_probe_fp64: FMA loops over 8 blocks per SM); the derived figure, 2 FP64 FMA per clock per SM (4 flop/clk/SM)
# x 152 SMs x 2.07 GHz = 1.26 TFLOP/s, is the fallback when no measurement is passed in.
FP64_DERIVED_TFLOPS = 152 * 2.070 * 4 / 1e3
ALU_CLASSES = {"fft_fibres", "fibre_operator", "gauss_multi", "r2c_rows", "c2r_rows", "rows_fused", "gemm", "eigen",
               "gram_factor", "sketch"}


def class_rooflines(stats, classes):
    """Achieved HBM bandwidth of memory-bound kernel classes against the measured copy peak."""
    peaks, src = measured_peaks()
    out = {}
    for k in classes:
        v = stats.get(k)
        if not v or not v["launches"] or v["ms"] <= 0:
            continue
        gbs = v["bytes"] / (v["ms"] * 1e-3) / 1e9
        out[k] = {"achieved_gbs": round(gbs, 1), "frac": round(gbs / float(peaks["hbm_gbs"]), 3),
                  "launches": v["launches"], "ms": round(v["ms"], 3)}
    return out


def roofline(stats, fp64_peak=None):
    peaks, src = measured_peaks()
    dom = max(stats, key=lambda k: stats[k]["ms"])
    s = stats[dom]
    per_launch_ms = s["ms"] / max(s["launches"], 1)
    if dom in ALU_CLASSES:
        achieved = s["flops"] / (s["ms"] * 1e-3) / 1e12 if s["ms"] > 0 else 0.0
        peak = fp64_peak if fp64_peak else FP64_DERIVED_TFLOPS
        source = ("measured FP64 FMA rate of this GPU (lrfg_probe_fp64, in this run)" if fp64_peak else
                  "derived FP64 pipe rate (2 DFMA/clk/SM x 152 SMs x 2.07 GHz)")
        out = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
               "peak_source": source}
    else:
        achieved = s["bytes"] / (s["ms"] * 1e-3) / 1e9 if s["ms"] > 0 else 0.0
        peak = float(peaks["hbm_gbs"])
        out = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
               "peak_source": src}
    total = sum(v["ms"] for v in stats.values())
    out.update({"kernel_class": dom, "launches": s["launches"], "avg_launch_ms": per_launch_ms,
                "share": s["ms"] / total if total > 0 else None, "traffic": None})
    # every class beside it, against the same denominators (a latency-bound class shows a small fraction: its
    # launches are one block per small matrix, and its time is the length of a sequential algorithm)
    alu_peak = fp64_peak if fp64_peak else FP64_DERIVED_TFLOPS
    out["by_class"] = {}
    for k, v in stats.items():
        if not v["launches"] or v["ms"] <= 0:
            continue
        if k in ALU_CLASSES:
            a = v["flops"] / (v["ms"] * 1e-3) / 1e12
            out["by_class"][k] = {"bound": "alu", "achieved": round(a, 5), "unit": "TFLOP/s", "frac": round(a / alu_peak, 5),
                                  "share": round(v["ms"] / total, 4), "avg_launch_us": round(1e3 * v["ms"] / v["launches"], 1)}
        else:
            a = v["bytes"] / (v["ms"] * 1e-3) / 1e9
            out["by_class"][k] = {"bound": "hbm", "achieved": round(a, 2), "unit": "GB/s",
                                  "frac": round(a / float(peaks["hbm_gbs"]), 5), "share": round(v["ms"] / total, 4),
                                  "avg_launch_us": round(1e3 * v["ms"] / v["launches"], 1)}
    return out


# -------------------------------------------------------------------------------------------------
# CPU baseline: the oracle as it stands
# -------------------------------------------------------------------------------------------------
GOLDEN = os.path.join(ROOT, "tests", "golden", "lognormal_243.json")


_ORACLE_CACHE = {}


def _oracle_operator(args, rank):
    """The oracle's truncated operator of the workload at truncation rank `rank` and its right-hand side (the
    coefficient compressed once by the oracle's TT-SVD, one operator per rank, kept for later samples)."""
    from oracle import lowrank as lr
    key = ("coeff", args.N, args.coeff_rank)
    if key not in _ORACLE_CACHE:
        _ORACLE_CACHE[key] = lr.tt_svd(make_coefficient(args.N), rmax=args.coeff_rank)
    okey = ("op", args.N, args.coeff_rank, rank, args.sketch_over, args.pinv_eps)
    if okey not in _ORACLE_CACHE:
        sketch = (args.sketch_over, 0) if args.sketch_over > 0 else None
        op = lr.LowRankGaNi(_ORACLE_CACHE[key], (args.N,) * 3, fmt="tt", rank=rank, pinv_eps=args.pinv_eps,
                            sketch=sketch)
        _ORACLE_CACHE[okey] = (op, op.rhs(np.array([1.0, 0.0, 0.0])))
    return _ORACLE_CACHE[okey]


def oracle_apply_seconds(args, n_applies, rank=None):
    """Time oracle applications of the truncated TT operator (Eq. (Pls_lowrank)) of the workload at truncation
    rank `rank` (default the cap), with the randomised rounding of the products when the workload uses it,
    starting from the right-hand side."""
    op, x = _oracle_operator(args, rank or args.rank)
    times = []
    for _ in range(n_applies):
        t0 = time.perf_counter()
        x = op.apply(x)
        times.append(time.perf_counter() - t0)
    return times


def oracle_applies_per_solve(args):
    """Operator applications of one oracle solve of this workload, from the oracle's own complete run stored
    in tests/golden/lognormal_243.json (written by tests/golden/make_golden.py, which calls only the oracle);
    None when the stored run is not this configuration."""
    try:
        g = json.load(open(GOLDEN))["tt_sketch"][str(args.rank)]
    except (OSError, KeyError, ValueError):
        return None
    o = g["opts"]
    same = (args.N == 243 and args.coeff_rank == 10 and o["rank"] == args.rank and o["sketch_over"] == args.sketch_over
            and o["tol"] == args.tt_tol and o["pinv_eps"] == args.pinv_eps and o["maxit"] == args.maxit
            and int(o["stop_on_increase"]) == int(args.stop_on_increase)
            and int(o.get("rank_start", 0)) == args.rank_start and int(o.get("rank_step", 0)) == args.rank_step)
    return (g["applies"], g) if same else None


def oracle_solve_seconds(args, g, per_rank):
    """Seconds of one oracle solve of the workload: per_rank oracle applications timed at each truncation rank
    the stored solve used, times its applications at that rank (the median of each rank's sample)."""
    by_rank = g.get("applies_by_rank") or {str(args.rank): g["applies"]}
    total, parts = 0.0, []
    for r, n in sorted(by_rank.items(), key=lambda kv: int(kv[0])):
        t = statistics.median(oracle_apply_seconds(args, per_rank, rank=int(r)))
        total += n * t
        parts.append(f"{n} at rank {r} ({t:.2f} s each)")
    return total, parts


def cpu_cores():
    try:
        from threadpoolctl import threadpool_info
        n = max((i.get("num_threads", 1) for i in threadpool_info()), default=1)
        return int(n)
    except Exception:
        return os.cpu_count() or 1


# -------------------------------------------------------------------------------------------------
# our arm
# -------------------------------------------------------------------------------------------------
def timed_solves(P, E, n, stream, flush, clk=None):
    """n solves, each bracketed by CUDA events on the library's stream with L2 flushed before it; P is one problem
    or a list of problems taken in turn; returns (per-solve ms, results)."""
    import torch
    Ps = P if isinstance(P, list) else [P]
    ms, res = [], []
    for i in range(n):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res.append(Ps[i % len(Ps)].solve(E, want_field=False)[0])
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    return ms, res


def pct(v, q):
    return float(np.percentile(v, q))


def run_ours(args):
    import torch
    import paper_1902_07455_gb300 as lrfg

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1902_07455_gb300 import build
    build.build()
    ctx = lrfg.Context(local)
    fp64_fma, fp64_dmma = ctx.probe_fp64()
    E = [1.0, 0.0, 0.0]
    A = make_coefficient(args.N)
    A_dev = torch.as_tensor(A, device=f"cuda:{local}")
    a_tt = ctx.tt_compress(A_dev, args.coeff_rank)
    a_full = ctx.tt_expand(a_tt)
    del A_dev
    stream = ctx.stream
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=f"cuda:{local}")

    # full-format FP64 PCG (tol 1e-8) on the same coefficient: the A_eff reference and the comparison solver
    Pfull = ctx.problem(a_full, lrfg.FULL, tol=1e-8, maxit=2000)
    full_res, _ = Pfull.solve(E, want_field=False)
    full_ms, _ = timed_solves(Pfull, E, 3, stream, flush)
    f_in = ctx.field_from_full(torch.randn((args.N,) * 3, dtype=torch.float64, device=f"cuda:{local}"))
    f_out = Pfull.apply(f_in)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        Pfull.apply_into(f_in, f_out)
    torch.cuda.synchronize()
    full_apply_s = (time.perf_counter() - t0) / 5
    # the same solve with LRFG_MIXED: FP32 storage and FFTs, FP64 scalars, to a 1e-5 residual
    Pmix = ctx.problem(a_full, lrfg.FULL, tol=1e-5, maxit=2000, prec=lrfg.MIXED)
    mix_res, _ = Pmix.solve(E, want_field=False)
    mix_ms, _ = timed_solves(Pmix, E, 3, stream, flush)
    Pmix.apply_into(f_in, f_out)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        Pmix.apply_into(f_in, f_out)
    torch.cuda.synchronize()
    mix_apply_s = (time.perf_counter() - t0) / 5
    # per-class HBM rooflines of one solve in each precision
    full_classes = ["rows_fused", "r2c_rows", "c2r_rows", "fft_fibres", "pointwise", "reduce"]
    full_roof = {}
    for name, P in (("f64", Pfull), ("mixed", Pmix)):
        ctx.profile_reset()
        ctx.profile(True)
        P.solve(E, want_field=False)
        ctx.profile(False)
        full_roof[name] = class_rooflines(ctx.profile_read(), full_classes)
    f_in.free()
    f_out.free()

    # the low-rank solve that is timed (the workload's step): TT rank r, randomised rounding of the products,
    # stopped at the residual tolerance; step i draws its sketch from SplitMix64 stream i, so the steps sample
    # the randomised rounding (its iteration count moves with the sketch and with rounding near the residual
    # floor) instead of repeating one bitwise-identical solve
    lr_fmt = lrfg.TUCKER if args.format == "tucker" else lrfg.TT
    Ptts = [ctx.problem(a_tt, lr_fmt, rank=args.rank, pinv_eps=args.pinv_eps, tol=args.tt_tol, maxit=args.maxit,
                        stop_on_increase=args.stop_on_increase, sketch_over=args.sketch_over,
                        rank_start=args.rank_start, rank_step=args.rank_step, sketch_seed=s)
            for s in range(max(args.steps, 1))]
    Ptt = Ptts[0]
    for i in range(args.warmup):
        Ptts[i % len(Ptts)].solve(E, want_field=False)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    with ClockSampler(local) as clk:
        step_ms, results = timed_solves(Ptts, E, args.steps, stream, flush)
    torch.cuda.synchronize()
    launches = ctx.launch_count() - launches0
    total_ms = sum(step_ms)
    if world > 1:
        total_ms = reduce_max(total_ms, f"cuda:{local}")
        dist.barrier()
    res = results[-1]
    applies = sum(r.applies for r in results)
    errs = [abs(r.Aeff - full_res.Aeff) / full_res.Aeff for r in results]
    rel_err = max(errs)
    # one more solve, profiled (CUDA events around every launch), for the kernel classes and the roofline
    ctx.profile_reset()
    ctx.profile(True)
    prof_res, _ = Ptt.solve(E, want_field=False)
    ctx.profile(False)
    stats = ctx.profile_read()

    # the same TT solve with LRFG_MIXED (FP32 fibre transforms and sketch side in the steps, FP64 residual)
    Pmx = ctx.problem(a_tt, lr_fmt, rank=args.rank, pinv_eps=args.pinv_eps, tol=args.tt_tol, maxit=args.maxit,
                      stop_on_increase=args.stop_on_increase, sketch_over=args.sketch_over, prec=lrfg.MIXED,
                      rank_start=args.rank_start, rank_step=args.rank_step)
    Pmx.solve(E, want_field=False)
    Pmx1 = ctx.problem(a_tt, lr_fmt, rank=args.rank, pinv_eps=args.pinv_eps, tol=args.tt_tol, maxit=args.maxit,
                       stop_on_increase=args.stop_on_increase, sketch_over=args.sketch_over, prec=lrfg.MIXED,
                       rank_start=args.rank_start, rank_step=args.rank_step, sketch_seed=1)
    mx_ms, mx_res = timed_solves([Pmx, Pmx1], E, 2, stream, flush)
    tt_mixed = {"solves_per_s": 2e3 / sum(mx_ms), "p50_ms": pct(mx_ms, 50), "p99_ms": pct(mx_ms, 99),
                "sketch_seeds": [0, 1], "iters": [r.iters for r in mx_res], "applies": [r.applies for r in mx_res],
                "converged": [bool(r.converged) for r in mx_res], "ms": [round(m, 2) for m in mx_ms],
                "aeff": mx_res[-1].Aeff,
                "aeff_rel_err": max(abs(r.Aeff - full_res.Aeff) / full_res.Aeff for r in mx_res)}
    Pmx1.free()
    # the homogenised tensor (Eq. (homog)): the d (d + 1) / 2 = 6 solves of the polarisation fields, TT in
    # lockstep (lrfg_problem_solve_many: one launch sequence for all six) against six full FP64 solves
    tensor = None if args.no_tensor else homogenised_tensor(ctx, args, a_tt, lr_fmt, Pfull, stream, flush)
    Pmx.free()

    # a batch of microstructures of this workload's recipe (seeds SEED + 1 .. SEED + count), one TT solve each
    # with the timed step's options, solved together in lockstep (lrfg_problems_solve), against their full FP64
    # solves
    micro = microstructure_batch(ctx, args, lr_fmt, stream, flush, count=args.micro)

    # the configuration of the previous measurements: TT rank 10, deterministic rounding, stop on increase
    P10 = ctx.problem(a_tt, lr_fmt, rank=10, pinv_eps=args.pinv_eps, tol=1e-12, maxit=60, stop_on_increase=True)
    P10.solve(E, want_field=False)
    ms10, r10 = timed_solves(P10, E, 2, stream, flush)
    P10.free()

    # end to end through the C ABI with host buffers: lrfg_solve with the coefficient carriages in host
    # memory (copied in each call) and the result read back to the host; call i draws its sketch from stream i,
    # as timed step i does, so the two numbers cover the same solves
    host_cores = [c.cpu().numpy() for c in a_tt.cores]
    e2e_ms = []
    for i in range(max(args.steps, 1)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r_e2e = solve_host(ctx, host_cores, args, E, seed=i)
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    h2d = sum(c.nbytes for c in host_cores)
    d2h = 8 * 2 + 4 * 8  # the lrfg_result fields read back (A_eff, residual, counters)

    line = None
    if rank == 0:
        solves_per_s = job_throughput(args.steps, world, total_ms * 1e-3)
        line = {
            "metric": METRIC, "value": solves_per_s, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args),
            "tt_op_applies_per_s": world * applies / (total_ms * 1e-3),
            "tt_applies_per_solve": applies / args.steps,
            "tt_iters": res.iters, "tt_rel_resid": res.rel_resid, "tt_aeff": res.Aeff, "full_aeff": full_res.Aeff,
            "aeff_rel_err": rel_err, "meets_1e-6": rel_err <= 1e-6,
            "per_step": {"sketch_seed": list(range(len(results))), "iters": [r.iters for r in results],
                         "applies": [r.applies for r in results], "converged": [bool(r.converged) for r in results],
                         "ms": [round(m, 2) for m in step_ms],
                         "aeff_rel_err": [float("%.3g" % e) for e in errs]},
            "p50_ms": pct(step_ms, 50), "p99_ms": pct(step_ms, 99),
            "full": {"solves_per_s": 1e3 / statistics.median(full_ms), "p50_ms": pct(full_ms, 50),
                     "p99_ms": pct(full_ms, 99), "iters": full_res.iters, "tol": 1e-8,
                     "op_applies_per_s": 1.0 / full_apply_s},
            "full_solves_per_s": 1e3 / statistics.median(full_ms),
            "full_mixed": {"solves_per_s": 1e3 / statistics.median(mix_ms), "p50_ms": pct(mix_ms, 50),
                           "p99_ms": pct(mix_ms, 99), "iters": mix_res.iters, "op_applies_per_s": 1.0 / mix_apply_s,
                           "tol": 1e-5, "aeff": mix_res.Aeff,
                           "aeff_rel_err_vs_f64": abs(mix_res.Aeff - full_res.Aeff) / full_res.Aeff},
            "tt_vs_full_fp64": solves_per_s / world / (1e3 / statistics.median(full_ms)),
            "tt_mixed": tt_mixed,
            "homogenised_tensor_6_solves": tensor,
            "microstructure_batch": micro,
            "tt_rank10_deterministic": {"solves_per_s": 1e3 / statistics.median(ms10), "iters": r10[-1].iters,
                                        "aeff_rel_err": abs(r10[-1].Aeff - full_res.Aeff) / full_res.Aeff},
            "full_class_rooflines": full_roof,
            "coeff_ranks": Ptt.coeff_ranks(),
            "e2e": {"value": len(e2e_ms) * 1e3 / sum(e2e_ms), "unit": "solves/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "aeff": r_e2e, "ms": [round(m, 2) for m in e2e_ms],
                    "sketch_seeds": list(range(len(e2e_ms)))},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "fp64_measured_tflops": {"fma": fp64_fma, "dmma": fp64_dmma},
            "roofline": roofline(stats, fp64_fma),
            "profiled_solve": {"note": "one extra solve with CUDA events around every launch (not timed above)",
                               "iters": prof_res.iters, "applies": prof_res.applies},
            "kernel_classes": {k: {"ms": round(v["ms"], 3), "launches": v["launches"],
                                   "gflop": round(v["flops"] / 1e9, 3)} for k, v in stats.items() if v["launches"]},
        }
    for P in Ptts:
        P.free()
    Pfull.free()
    Pmix.free()
    ctx.close()
    if world > 1:
        dist.destroy_process_group()
    return line


def homogenised_tensor(ctx, args, a_tt, lr_fmt, Pfull, stream, flush):
    """The homogenised tensor (Eq. (homog)): the d (d + 1) / 2 = 6 solves of the polarisation fields, TT in lockstep
    (lrfg_problem_solve_many: one launch sequence for all six), FP64 and LRFG_MIXED, against six full FP64 solves."""
    import torch
    import paper_1902_07455_gb300 as lrfg
    Es6 = [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0], [1.0, 1.0, 0.0], [1.0, 0.0, 1.0], [0.0, 1.0, 1.0]]
    P6 = ctx.problem(a_tt, lr_fmt, rank=args.rank, pinv_eps=args.pinv_eps, tol=args.tensor_tol, maxit=args.maxit,
                     stop_on_increase=args.stop_on_increase, sketch_over=args.sketch_over,
                     rank_start=args.rank_start, rank_step=args.rank_step)
    P6.solve_many(Es6)
    tensor_ms, tensor_tt = [], None
    for _ in range(2):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tensor_tt = P6.solve_many(Es6)
        e1.record(stream)
        e1.synchronize()
        tensor_ms.append(e0.elapsed_time(e1))
    full6_ms, full6 = 0.0, []
    for E6 in Es6:
        ms1, r1 = timed_solves(Pfull, E6, 1, stream, flush)
        full6_ms += ms1[0]
        full6.append(r1[0])
    tensor = {"tol": args.tensor_tol,
              "tt_lockstep": {"solves_per_s": 6e3 / min(tensor_ms), "seconds": min(tensor_ms) / 1e3,
                              "iters": [r.iters for r in tensor_tt]},
              "full_fp64": {"solves_per_s": 6e3 / full6_ms, "seconds": full6_ms / 1e3},
              "max_rel_err_vs_full": max(abs(a.Aeff - b.Aeff) / b.Aeff for a, b in zip(tensor_tt, full6))}
    tensor["tt_vs_full_fp64"] = tensor["tt_lockstep"]["solves_per_s"] / tensor["full_fp64"]["solves_per_s"]
    P6.free()
    Pmx6 = ctx.problem(a_tt, lr_fmt, rank=args.rank, pinv_eps=args.pinv_eps, tol=args.tensor_tol, maxit=args.maxit,
                       stop_on_increase=args.stop_on_increase, sketch_over=args.sketch_over, prec=lrfg.MIXED,
                       rank_start=args.rank_start, rank_step=args.rank_step)
    Pmx6.solve_many(Es6)
    flush.fill_(1.0)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    mx6 = Pmx6.solve_many(Es6)
    e1.record(stream)
    e1.synchronize()
    tensor["tt_mixed_lockstep"] = {"solves_per_s": 6e3 / e0.elapsed_time(e1),
                                   "max_rel_err_vs_full": max(abs(a.Aeff - b.Aeff) / b.Aeff for a, b in zip(mx6, full6))}
    tensor["tt_mixed_vs_full_fp64"] = tensor["tt_mixed_lockstep"]["solves_per_s"] / tensor["full_fp64"]["solves_per_s"]
    tensor["meets_1e-6"] = max(tensor["max_rel_err_vs_full"], tensor["tt_mixed_lockstep"]["max_rel_err_vs_full"]) <= 1e-6
    Pmx6.free()
    return tensor


def microstructure_batch(ctx, args, lr_fmt, stream, flush, count=8):
    """`count` seeded microstructures of the workload's recipe (lognormal SE-GRF, seeds SEED + 1 ..), each
    compressed to the coefficient rank: their TT solves (the timed step's options) together in lockstep through
    lrfg_problems_solve, FP64 and LRFG_MIXED, against their full FP64 solves one after the other."""
    import torch
    import paper_1902_07455_gb300 as lrfg
    from synthetic import lognormal_grf
    if count < 1:
        return None
    E = [1.0, 0.0, 0.0]
    dev = f"cuda:{torch.cuda.current_device()}"
    coeffs, fulls = [], []
    for i in range(count):
        A = torch.as_tensor(lognormal_grf(3, args.N, ell=0.2, var=1.0, seed=SEED + 1 + i), device=dev)
        a = ctx.tt_compress(A, args.coeff_rank)
        del A
        coeffs.append(a)
    full_ms = 0.0
    for a in coeffs:
        a_full = ctx.tt_expand(a)
        P = ctx.problem(a_full, lrfg.FULL, tol=1e-8, maxit=2000)
        ms1, r1 = timed_solves(P, E, 1, stream, flush)
        full_ms += ms1[0]
        fulls.append(r1[0].Aeff)
        P.free()
        del a_full
    out = {"count": count, "seeds": [SEED + 1 + i for i in range(count)],
           "full_fp64": {"solves_per_s": count * 1e3 / full_ms, "seconds": full_ms / 1e3}}
    for name, prec in (("tt_lockstep", lrfg.FP64), ("tt_mixed_lockstep", lrfg.MIXED)):
        Ps = [ctx.problem(a, lr_fmt, rank=args.rank, pinv_eps=args.pinv_eps, tol=args.tt_tol, maxit=args.maxit,
                          stop_on_increase=args.stop_on_increase, sketch_over=args.sketch_over, prec=prec,
                          rank_start=args.rank_start, rank_step=args.rank_step) for a in coeffs]
        lrfg.Problem.solve_together(Ps, [E] * count)
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        rs = lrfg.Problem.solve_together(Ps, [E] * count)
        e1.record(stream)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        errs = [abs(r.Aeff - f) / f for r, f in zip(rs, fulls)]
        out[name] = {"solves_per_s": count * 1e3 / ms, "seconds": ms / 1e3, "iters": [r.iters for r in rs],
                     "max_rel_err_vs_full": max(errs), "meets_1e-6": max(errs) <= 1e-6,
                     "vs_full_fp64": (count * 1e3 / ms) / out["full_fp64"]["solves_per_s"]}
        for P in Ps:
            P.free()
    return out


def solve_host(ctx, host_cores, args, E, seed=0):
    """One lrfg_solve call with host-resident coefficient carriages (the public C ABI); `seed`: the SplitMix64
    stream of the randomised rounding's sketch."""
    import ctypes as C
    from paper_1902_07455_gb300 import _lib as L
    c = L.lrfg_coeff()
    c.d = 3
    for j in range(3):
        c.N[j] = host_cores[j].shape[1]
    c.fmt = L.LRFG_TT
    c.on_device = 0
    c.tt.d = 3
    keep = [np.ascontiguousarray(h) for h in host_cores]
    for j in range(3):
        c.tt.N[j] = keep[j].shape[1]
        c.tt.cores[j] = keep[j].ctypes.data
    rr = [1] + [k.shape[2] for k in keep[:-1]] + [1]
    for j in range(4):
        c.tt.r[j] = rr[j]
    o = L.lrfg_opts()
    o.fmt = L.LRFG_TUCKER if args.format == "tucker" else L.LRFG_TT
    o.prec, o.rank, o.pinv_eps = L.LRFG_FP64, args.rank, args.pinv_eps
    o.tol, o.maxit, o.stop_on_increase = args.tt_tol, args.maxit, args.stop_on_increase
    o.sketch_over, o.sketch_seed = args.sketch_over, seed
    o.rank_start, o.rank_step = args.rank_start, args.rank_step
    res = L.lrfg_result()
    Ed = (C.c_double * 3)(*E)
    st = ctx.lib.lrfg_solve(ctx.h, C.byref(c), Ed, C.byref(o), C.byref(res), None)
    if st not in (L.LRFG_OK, L.LRFG_ENOCONV):
        ctx.check(st)
    return res.Aeff


def add_cpu_baseline(line, args):
    # a bounded sample: oracle applications of the same truncated operator (about 10-30 s of CPU work), scaled
    # to solves/s by the applications per solve of the oracle's own complete solve of this workload (stored),
    # or else by the GPU run's count of the same algorithm
    stored = oracle_applies_per_solve(args)
    if stored:
        sec, parts = oracle_solve_seconds(args, stored[1], 3)
        line["cpu_baseline"] = {"value": 1.0 / sec, "unit": "solves/s", "cores": cpu_cores(), "kind": "oracle",
                                "sample": f"3 oracle applications of the TT operator at N={args.N}^3 at each truncation "
                                          f"rank of the oracle's own complete solve of this workload (tests/golden), "
                                          f"weighted by its applications there: " + ", ".join(parts)}
        return
    t = oracle_apply_seconds(args, 8)
    per_apply = statistics.median(t)
    n_app = line["tt_applies_per_solve"]
    line["cpu_baseline"] = {"value": 1.0 / (per_apply * n_app), "unit": "solves/s", "cores": cpu_cores(),
                            "kind": "oracle",
                            "sample": f"{len(t)} oracle applications of the rank-{args.rank} TT operator at N={args.N}^3 "
                                      f"({per_apply:.2f} s each, median), times {n_app} applications per solve from "
                                      f"the GPU run's solves (same algorithm)"}


# -------------------------------------------------------------------------------------------------
# reference arm: the oracle, timed on the host cores
# -------------------------------------------------------------------------------------------------
def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return None
    # each step: one oracle application of the workload's operator at every truncation rank of the oracle's own
    # complete solve of this workload (stored in tests/golden), weighted by its applications at that rank: the
    # seconds of one oracle solve; the value is the inverse of the median step
    stored = oracle_applies_per_solve(args)
    if stored is None:
        return {"impl": "reference", "unavailable": "no stored oracle solve of this configuration (run "
                                                   "tests/golden/make_golden.py for it)"}
    n_app, g = stored
    by_rank = g.get("applies_by_rank") or {str(args.rank): n_app}
    times = []
    for step in range(args.warmup + args.steps):
        sec = sum(n * oracle_apply_seconds(args, 1, rank=int(r))[0] for r, n in by_rank.items())
        if step >= args.warmup:
            times.append(sec)
    value = 1.0 / statistics.median(times)
    cores = cpu_cores()
    return {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": workload_config(args),
            "oracle_solve": {"applies": n_app, "iters": g["iters"], "aeff": g["Aeff"]},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step one oracle application of the TT operator at N={args.N}^3 at each "
                                       f"truncation rank of the oracle's own complete solve of this workload "
                                       f"(tests/golden), times its {n_app} applications split by rank "
                                       f"{dict(sorted(by_rank.items(), key=lambda kv: int(kv[0])))}"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def c3_bounds(N, contrast):
    """Voigt and Reuss bounds of the smoothed cube: arithmetic and harmonic means of the grid samples
    (computed slice by slice; the grid is never held whole)."""
    from synthetic import smoothed_cube
    _, terms, w = smoothed_cube(3, N, contrast=contrast, full=False)
    h = terms[1][0]
    arith = 1.0 + (contrast - 1.0) * float(np.mean(h)) ** 3
    hh = np.outer(h, h)
    inv = 0.0
    for i in range(N):
        inv += float(np.sum(1.0 / (1.0 + (contrast - 1.0) * h[i] * hh)))
    return arith, 1.0 / (inv / float(N) ** 3)


def run_c3(args):
    """The large smoothed-cube workload: d = 3 tanh-smoothed cube (|x| < 0.3, width 2/N, contrast 100;
    coefficient of TT rank 2 built on the GPU from its two separable terms), TT MinRes solve at rank r; the
    full-format solve on the expanded coefficient (FP32 storage, or FP64) as the anchor; Voigt-Reuss bounds."""
    import torch
    import paper_1902_07455_gb300 as lrfg
    from paper_1902_07455_gb300 import build
    from synthetic import smoothed_cube
    build.build()
    N = args.N
    contrast = 100.0
    ctx = lrfg.Context(0)
    _, terms, w = smoothed_cube(3, N, contrast=contrast, full=False)
    rank1 = [lrfg.TTensor.from_numpy([np.asarray(f, dtype=np.float64).reshape(1, N, 1) for f in t]) for t in terms]
    a_tt = ctx.tt_add(w[0], rank1[0], w[1], rank1[1])
    E = [1.0, 0.0, 0.0]
    P = ctx.problem(a_tt, lrfg.TT, rank=args.rank, pinv_eps=args.pinv_eps, tol=1e-12, maxit=args.maxit)
    stream = ctx.stream
    for _ in range(args.warmup):
        P.solve(E, want_field=False)
    torch.cuda.synchronize()
    launches0 = ctx.launch_count()
    ctx.profile_reset()
    ctx.profile(True)
    step_ms, results = [], []
    with ClockSampler(0) as clk:
        for _ in range(args.steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            results.append(P.solve(E, want_field=False)[0])
            e1.record(stream)
            e1.synchronize()
            step_ms.append(e0.elapsed_time(e1))
    ctx.profile(False)
    stats = ctx.profile_read()
    launches = ctx.launch_count() - launches0
    res = results[-1]
    arith, harm = c3_bounds(N, contrast)
    anchor = None
    if args.c3_full != "none":
        a_full = ctx.tt_expand(a_tt)
        prec = lrfg.MIXED if args.c3_full == "mixed" else lrfg.FP64
        tol = 1e-5 if args.c3_full == "mixed" else 1e-8
        Pf = ctx.problem(a_full, lrfg.FULL, tol=tol, maxit=5000, prec=prec)
        del a_full
        fr, _ = Pf.solve(E, want_field=False)
        anchor = {"precision": args.c3_full, "tol": tol, "aeff": fr.Aeff, "iters": fr.iters, "seconds": fr.seconds,
                  "solves_per_s": 1.0 / fr.seconds}
        Pf.free()
    total_ms = sum(step_ms)
    line = {
        "metric": METRIC, "value": args.steps / (total_ms * 1e-3), "unit": "solves/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"d=3 N={N}^3 tanh-smoothed cube |x|<0.3 width 2/N contrast 100 (coefficient TT "
                               f"rank 2), E=(1,0,0); TT rank {args.rank} MinRes", "d": 3, "N": N,
                   "tt_rank": args.rank, "pinv_eps": args.pinv_eps, "precision": "fp64"},
        "tt_iters": res.iters, "tt_applies_per_solve": sum(r.applies for r in results) / args.steps,
        "tt_aeff": res.Aeff, "voigt": arith, "reuss": harm, "within_bounds": harm <= res.Aeff <= arith,
        "full_anchor": anchor,
        "aeff_rel_err_vs_anchor": abs(res.Aeff - anchor["aeff"]) / anchor["aeff"] if anchor else None,
        "p50_ms": float(np.percentile(step_ms, 50)), "p99_ms": float(np.percentile(step_ms, 99)),
        "gpu_launches": launches, "clocks": clk.summary(), "roofline": roofline(stats),
        "kernel_classes": {k: {"ms": round(v["ms"], 3), "launches": v["launches"]} for k, v in stats.items()
                           if v["launches"]},
    }
    print(json.dumps(line))
    P.free()
    ctx.close()


def c4_requests(count, seed=SEED, rank_step=1):
    """Seeded batch: half lognormal SE-GRF (l uniform in [0.1, 0.3], variance (ln(contrast)/4)^2 so that
    exp(+-2 sigma) spans the contrast), half tanh-smoothed inclusions (sphere or cube, radius / half-side
    uniform in [0.15, 0.35]); contrast log-uniform in [5, 100]; N uniform in {45, 81, 135, 243}; TT rank
    uniform in [5, 30] (rank_step > 1: uniform over the multiples of rank_step there).  Grid coefficients
    (lognormal, sphere) are TT-compressed to rank 10 on the GPU here, before timing; the cube is its exact
    rank-2 TT.  Each request: (TT carriages on the host, rank, description)."""
    import torch
    import paper_1902_07455_gb300 as lrfg
    from synthetic import lognormal_grf, smoothed_cube, smoothed_sphere
    rng = np.random.Generator(np.random.PCG64(seed))
    ctx = lrfg.Context(0)
    out = []
    for i in range(count):
        N = int(rng.choice([45, 81, 135, 243]))
        if rank_step > 1:
            r = rank_step * int(rng.integers(-(-5 // rank_step), 30 // rank_step + 1))
        else:
            r = int(rng.integers(5, 31))
        contrast = float(np.exp(rng.uniform(np.log(5.0), np.log(100.0))))
        if i % 2 == 0:
            ell = float(rng.uniform(0.1, 0.3))
            a = lognormal_grf(3, N, ell=ell, var=(np.log(contrast) / 4.0) ** 2, seed=seed + i)
            desc = f"lognormal l={ell:.2f}"
        else:
            size = float(rng.uniform(0.15, 0.35))
            if rng.integers(0, 2) == 0:
                a = smoothed_sphere(3, N, contrast=contrast, radius=size)
                desc = f"sphere R={size:.2f}"
            else:
                _, terms, w = smoothed_cube(3, N, contrast=contrast, c=size, full=False)
                cores = [np.asarray(f, dtype=np.float64).reshape(1, N, 1) for f in terms[0]]
                cores2 = [np.asarray(f, dtype=np.float64).reshape(1, N, 1) for f in terms[1]]
                tt = ctx.tt_add(w[0], lrfg.TTensor.from_numpy(cores), w[1], lrfg.TTensor.from_numpy(cores2))
                out.append((tt.numpy(), r, f"cube c={size:.2f} contrast={contrast:.1f} N={N} r={r}"))
                continue
        tt = ctx.tt_compress(torch.as_tensor(a, device="cuda:0"), 10)
        out.append((tt.numpy(), r, f"{desc} contrast={contrast:.1f} N={N} r={r}"))
    ctx.close()
    return out


def run_batch(B, reqs, maxit, pinv_eps, prec=0, sketch_over=0):
    """Submit every request at once to executor B; returns (seconds from first submission to last
    completion, BatchResults)."""
    import paper_1902_07455_gb300 as lrfg
    t0 = time.perf_counter()
    tickets = [B.submit(c, [1.0, 0.0, 0.0], lrfg.TT, rank=r, pinv_eps=pinv_eps, tol=1e-12, maxit=maxit, prec=prec,
                        sketch_over=sketch_over) for c, r, _ in reqs]
    res = [B.wait(t) for t in tickets]
    return time.perf_counter() - t0, res


def run_c4(args):
    """Batched throughput: `count` microstructures of mixed N and rank (c4_requests), every request
    submitted at once to the executor; value = solves/s from first submission to last completion (host
    clock, coefficient upload from host memory included: end to end by construction).  The same batch
    through one worker gives the serial figure."""
    from paper_1902_07455_gb300 import build
    build.build()
    t_gen = time.perf_counter()
    reqs = c4_requests(args.count, rank_step=args.c4_rank_step)
    t_gen = time.perf_counter() - t_gen
    import paper_1902_07455_gb300 as lrfg
    prec = lrfg.MIXED if args.c4_prec == "mixed" else lrfg.FP64
    kw = dict(prec=prec, sketch_over=args.c4_sketch_over)
    # a warm pass (plans, twiddles and pools of every worker context), then the timed pass
    with lrfg.Batch(0, workers=args.workers, group=args.group) as B:
        run_batch(B, reqs, args.maxit, args.pinv_eps, **kw)
        with ClockSampler(0) as clk:
            dt, res = run_batch(B, reqs, args.maxit, args.pinv_eps, **kw)
    # one worker, one request at a time: warmed on the largest requests, then the whole batch
    big = sorted(reqs, key=lambda q: -q[0][1].shape[1] * q[1] ** 2)[:4]
    with lrfg.Batch(0, workers=1) as B1:
        run_batch(B1, big, args.maxit, args.pinv_eps, **kw)
        dt1, res1 = run_batch(B1, reqs, args.maxit, args.pinv_eps, **kw)
    lat = [b.total_s for b in res]
    same = all(a.result.Aeff == b.result.Aeff and a.result.iters == b.result.iters for a, b in zip(res, res1))
    diff = max(abs(a.result.Aeff - b.result.Aeff) / abs(b.result.Aeff) for a, b in zip(res, res1))
    line = {
        "metric": METRIC, "value": len(reqs) / dt, "unit": "solves/s", "n_gpus": 1, "steps": 1,
        "warmup": 1, "ms_per_step": 1e3 * dt, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if prec == lrfg.FP64 else "f32+f64", "data": "synthetic",
        "config": {"workload": f"batch of {len(reqs)} seeded d=3 microstructures (half lognormal SE-GRF, half "
                               f"tanh-smoothed sphere/cube inclusions, contrast 5-100), N in {{45,81,135,243}}, "
                               f"TT rank 5-30" + (f" in steps of {args.c4_rank_step}" if args.c4_rank_step > 1 else "")
                               + f", coefficient TT rank 10 (cube: exact 2), TT MinRes, "
                               + ("FP64" if prec == lrfg.FP64 else "LRFG_MIXED (FP32 transforms and sketch side, "
                                                                   "FP64 residual)"),
                   "count": len(reqs), "workers": args.workers, "group": args.group, "maxit": args.maxit,
                   "pinv_eps": args.pinv_eps, "sketch_over": args.c4_sketch_over, "precision": args.c4_prec},
        "serial_solves_per_s": len(reqs) / dt1, "overlap_speedup": dt1 / dt,
        "bitwise_equal_to_serial": same, "max_rel_aeff_diff_vs_serial": diff,
        "groups": sorted(collections.Counter(b.group for b in res).items()),
        "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
        "run_s_sum": sum(b.run_s for b in res), "iters_mean": float(np.mean([b.result.iters for b in res])),
        "e2e": {"value": len(reqs) / dt, "unit": "solves/s",
                "h2d_bytes_per_step": int(sum(sum(c.nbytes for c in cs) for cs, _, _ in reqs)),
                "d2h_bytes_per_step": 48 * len(reqs)},
        "clocks": clk.summary(), "input_generation_s": t_gen,
        "requests": [{"desc": d, "aeff": b.result.Aeff, "iters": b.result.iters, "run_s": round(b.run_s, 4)}
                     for (_, _, d), b in zip(reqs, res)],
    }
    print(json.dumps(line), flush=True)


SMOOTH_N = [63, 75, 81, 105, 125, 135, 147, 175, 189, 225, 243, 245, 315, 343, 375, 405, 441, 525, 567, 625, 675,
            729]  # odd sizes in [63, 729] with prime factors 3, 5, 7 only


def separable_tt(terms, weights):
    """TT carriages of sum_i weights[i] * outer(terms[i]) (rank = number of terms): the first carriage
    holds the weighted first factors, the others are block diagonal / block columns."""
    R, d = len(terms), len(terms[0])
    N = [len(v) for v in terms[0]]
    cores = []
    for j in range(d):
        a = 1 if j == 0 else R
        b = 1 if j == d - 1 else R
        c = np.zeros((a, N[j], b))
        for i in range(R):
            v = np.asarray(terms[i][j], dtype=np.float64) * (weights[i] if j == 0 else 1.0)
            c[0 if j == 0 else i, :, 0 if j == d - 1 else i] = v
        cores.append(c)
    return cores


def c5_requests(count, rate, seed=SEED + 5):
    """Seeded request stream: exponential gaps of mean 1/rate; d in {2, 3} with equal probability; N uniform
    over SMOOTH_N; rank tolerance log-uniform in [1e-6, 1e-4]; contrast log-uniform in [5, 100].  d = 2:
    lognormal SE-GRF (grid, variance (ln(contrast)/4)^2), tanh-smoothed square (separable) or disc
    (grid); d = 3: tanh-smoothed cube (separable, exact TT rank 2), laminate (rank 1), or for N <= 135 a
    lognormal SE-GRF (grid).  Grid coefficients go to the executor as grid values (TT-compressed with the
    request's tolerance on the GPU, inside the request).  Each request: (arrival offset in s, coefficient,
    d, rank_tol, description)."""
    from synthetic import laminate, lognormal_grf, smoothed_cube, smoothed_sphere
    rng = np.random.Generator(np.random.PCG64(seed))
    t = 0.0
    out = []
    for i in range(count):
        t += float(rng.exponential(1.0 / rate))
        d = int(rng.integers(2, 4))
        N = int(rng.choice(SMOOTH_N))
        rtol = float(10.0 ** rng.uniform(-6.0, -4.0))
        contrast = float(np.exp(rng.uniform(np.log(5.0), np.log(100.0))))
        size = float(rng.uniform(0.15, 0.35))
        kind = int(rng.integers(0, 3))
        if d == 2 and kind == 0:
            coeff = lognormal_grf(2, N, ell=float(rng.uniform(0.1, 0.3)), var=(np.log(contrast) / 4.0) ** 2,
                                  seed=seed + i)
            desc = "lognormal"
        elif d == 2 and kind == 1:
            _, terms, w = smoothed_cube(2, N, contrast=contrast, c=size, full=False)
            coeff, desc = separable_tt(terms, w), "square"
        elif d == 2:
            coeff, desc = smoothed_sphere(2, N, contrast=contrast, radius=size), "disc"
        elif kind == 0 and N <= 135:
            coeff = lognormal_grf(3, N, ell=float(rng.uniform(0.1, 0.3)), var=(np.log(contrast) / 4.0) ** 2,
                                  seed=seed + i)
            desc = "lognormal"
        elif kind == 1:
            _, terms, w = laminate(3, N, contrast=contrast, c=size, full=False)
            coeff, desc = separable_tt(terms, w), "laminate"
        else:
            _, terms, w = smoothed_cube(3, N, contrast=contrast, c=size, full=False)
            coeff, desc = separable_tt(terms, w), "cube"
        out.append((t, coeff, d, rtol, f"d={d} N={N} {desc} contrast={contrast:.1f} rank_tol={rtol:.1e}"))
    return out


def run_c5(args):
    """Serving: requests arrive on a seeded Poisson clock (c5_requests) and are submitted to the executor at
    their arrival times by the host; each is a TT solve with the request's rank tolerance (rank cap
    --rank-cap).  Latency = arrival to completion (queueing for a worker and HBM included); value =
    completed requests / (last completion - first arrival)."""
    import paper_1902_07455_gb300 as lrfg
    from paper_1902_07455_gb300 import build
    build.build()
    t_gen = time.perf_counter()
    reqs = c5_requests(args.count, args.rate)
    t_gen = time.perf_counter() - t_gen

    def serve(B, stream):
        tickets = []
        t0 = time.perf_counter()
        for t_arr, coeff, d, rtol, _ in stream:
            delay = t_arr - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            E = [1.0] + [0.0] * (d - 1)
            tickets.append(B.submit(coeff, E, lrfg.TT, rank=args.rank_cap, pinv_eps=args.pinv_eps, tol=1e-10,
                                    maxit=args.maxit, rank_tol=rtol, coeff_rank=args.coeff_rank))
        res = []
        for i, t in enumerate(tickets):
            res.append(B.wait(t))
            print(f"c5 {i} {stream[i][4]} run {res[-1].run_s:.3f} s latency {res[-1].total_s:.3f} s "
                  f"ranks {res[-1].result.ranks} iters {res[-1].result.iters}", file=sys.stderr, flush=True)
        return time.perf_counter() - t0, res

    with lrfg.Batch(0, workers=args.workers) as B:
        serve(B, [(0.0,) + r[1:] for r in reqs[: min(len(reqs), 2 * args.workers)]])  # warm the contexts
        with ClockSampler(0) as clk:
            span, res = serve(B, reqs)
    lat = np.array([b.total_s for b in res])
    queue = np.array([b.queue_s for b in res])
    h2d = int(sum(sum(c.nbytes for c in q[1]) if isinstance(q[1], list) else q[1].nbytes for q in reqs))
    line = {
        "metric": METRIC, "value": len(res) / span, "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 1,
        "ms_per_step": 1e3 * span, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"serving: {len(reqs)} requests, Poisson arrivals at {args.rate:g}/s, d in {{2,3}}, "
                               f"N in 3-5-7-smooth sizes 63-729, TT MinRes with rank tolerance 1e-6-1e-4 "
                               f"(cap {args.rank_cap}), grid coefficients TT-compressed to rank <= {args.coeff_rank}, "
                               f"FP64", "count": len(reqs), "rate": args.rate, "coeff_rank": args.coeff_rank,
                   "workers": args.workers, "maxit": args.maxit, "rank_cap": args.rank_cap},
        "latency_p50_s": float(np.percentile(lat, 50)), "latency_p99_s": float(np.percentile(lat, 99)),
        "queue_p50_s": float(np.percentile(queue, 50)), "queue_p99_s": float(np.percentile(queue, 99)),
        "run_p50_s": float(np.percentile([b.run_s for b in res], 50)),
        "offered_rate": len(reqs) / reqs[-1][0], "arrival_span_s": reqs[-1][0],
        "e2e": {"value": len(res) / span, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": 48 * len(res)},
        "clocks": clk.summary(), "input_generation_s": t_gen,
        "requests": [{"desc": q[4], "aeff": b.result.Aeff, "iters": b.result.iters, "ranks": b.result.ranks,
                      "run_s": round(b.run_s, 4), "latency_s": round(b.total_s, 4)} for q, b in zip(reqs, res)],
    }
    print(json.dumps(line), flush=True)


def run_case(args):
    """Two applications of one operator of the benchmark workload (coefficient compressed to rank
    coeff-rank on the GPU): the launch sequence a profiler capture of one kernel needs, and nothing else."""
    import torch
    import paper_1902_07455_gb300 as lrfg
    from paper_1902_07455_gb300 import build
    build.build()
    ctx = lrfg.Context(0)
    A = torch.as_tensor(make_coefficient(args.N), device="cuda:0")
    a_tt = ctx.tt_compress(A, args.coeff_rank)
    if args.case == "tt_solve":
        P = ctx.problem(a_tt, lrfg.TT, rank=args.rank, pinv_eps=args.pinv_eps, tol=args.tt_tol, maxit=args.maxit,
                        stop_on_increase=args.stop_on_increase, sketch_over=args.sketch_over,
                        rank_start=args.rank_start, rank_step=args.rank_step)
        r, _ = P.solve([1.0, 0.0, 0.0], want_field=False)
        print(json.dumps({"case": args.case, "N": args.N, "iters": r.iters, "aeff": r.Aeff, "ok": True}))
        P.free()
        ctx.close()
        return
    if args.case == "tt_apply":
        P = ctx.problem(a_tt, lrfg.TT, rank=args.rank, pinv_eps=args.pinv_eps, sketch_over=args.sketch_over)
        x = P.rhs([1.0, 0.0, 0.0])
    else:
        prec = lrfg.MIXED if args.case == "full_apply_mixed" else lrfg.FP64
        P = ctx.problem(ctx.tt_expand(a_tt), lrfg.FULL, prec=prec)
        x = ctx.field_from_full(torch.randn((args.N,) * 3, dtype=torch.float64, device="cuda:0"))
    for _ in range(2):
        y = P.apply(x)
    torch.cuda.synchronize()
    print(json.dumps({"case": args.case, "N": args.N, "ok": True}))
    y.free()
    x.free()
    P.free()
    ctx.close()


def main():
    args = parse()
    if args.workload == "c3" and "--N" not in sys.argv:
        args.N = 1215
    if args.case:
        run_case(args)
        return
    if args.workload == "c3" and args.impl == "ours":
        run_c3(args)
        return
    if args.workload == "c4" and args.impl == "ours":
        run_c4(args)
        return
    if args.workload == "c5" and args.impl == "ours":
        if "--count" not in sys.argv:
            args.count = 200
        run_c5(args)
        return
    if args.impl == "reference":
        line = run_reference(args)
    else:
        line = run_ours(args)
        if line is not None and not args.no_cpu_baseline and dist_env()[0] == 1:
            add_cpu_baseline(line, args)
    if line is not None:
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
