"""Write stored oracle values for the full-size parity tests (calls only oracle/ and synthetic/).

    python tests/golden/make_golden.py [--N 243] [--ranks 5 10]

Workload: d = 3, N^3 grid, lognormal SE-GRF coefficient (l = 0.2, variance 1, seed 19020745) compressed
by the oracle's TT-SVD to rank 10; the full-format reference solves the expansion of that TT coefficient
(the comparison protocol of Sec. 4.1); E = (1, 0, 0).  Output: tests/golden/lognormal_<N>.json with
the full PCG A_eff (tolerance 1e-8), its iteration count, and the TT minimal-residual A_eff at each rank
(exponential-sum accuracy 0.1, stop when the residual fails to decrease, at most 60 iterations); and the
benchmark's TT solve: the rank-adapting minimal-residual iteration (Sec. 4.3; rank 10, raised by 5 to the cap 20
when the residual stagnates) with the randomised rounding of the material and P~^-1 products (oversampling 10,
SplitMix64 stream 0), stopped at the relative residual 3e-4, at most 80 iterations,
with its iterations, operator applications (in total and per truncation rank) and run time (``--sketch-only`` adds just that entry to an existing
file).
"""
import argparse
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fourier_galerkin as fg  # noqa: E402
from oracle import lowrank as lr  # noqa: E402
from synthetic import lognormal_grf  # noqa: E402


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--N", type=int, default=243)
    p.add_argument("--ranks", type=int, nargs="*", default=[5, 10])
    p.add_argument("--coeff-rank", type=int, default=10)
    p.add_argument("--sketch-only", action="store_true")
    p.add_argument("--tensor-only", action="store_true",
                   help="add the full-format homogenised tensor (Eq. (homog)) to an existing file")
    args = p.parse_args()
    N = args.N
    E = np.array([1.0, 0.0, 0.0])
    A = lognormal_grf(3, N, ell=0.2, var=1.0, seed=19020745)
    a_tt = lr.tt_svd(A, rmax=args.coeff_rank)
    A_r = lr.tt_full(a_tt)
    path = os.path.join(HERE, f"lognormal_{N}.json")
    if args.tensor_only:
        # the full-format fields of E = e_1, e_2, e_3 (tol 1e-8); the problem is linear in E, so the field of
        # e_a + e_b is u_a + u_b and every entry of the tensor follows from the three solves
        out = json.load(open(path))
        t0 = time.time()
        fields = [fg.solve_gani(A_r, np.eye(3)[a], tol=1e-8, maxit=2000)["uh"] for a in range(3)]
        T = np.zeros((3, 3))
        for a in range(3):
            T[a, a] = fg.homogenised_coefficient(fields[a], A_r, np.eye(3)[a])
        for a in range(3):
            for b in range(a + 1, 3):
                Eab = np.eye(3)[a] + np.eye(3)[b]
                q = fg.homogenised_coefficient(fields[a] + fields[b], A_r, Eab)
                T[a, b] = T[b, a] = 0.5 * (q - T[a, a] - T[b, b])
        out["full_tensor"] = {"A": T.tolist(), "tol": 1e-8, "seconds": time.time() - t0}
        print("full_tensor", out["full_tensor"], flush=True)
        with open(path, "w") as f:
            json.dump(out, f, indent=1)
        print(path)
        return
    if args.sketch_only:
        out = json.load(open(path))
    else:
        out = {"workload": f"d=3 N={N}^3 lognormal SE-GRF l=0.2 var=1 seed 19020745, coefficient TT rank "
                           f"{args.coeff_rank} (oracle TT-SVD), E=(1,0,0)",
               "coeff_ranks": lr.tt_ranks(a_tt), "coeff_mean": float(A_r.mean())}
        t0 = time.time()
        full = fg.solve_gani(A_r, E, tol=1e-8, maxit=2000)
        out["full"] = {"Aeff": full["Aeff"], "iters": full["iters"], "rel_resid": full["rel_resid"],
                       "seconds": time.time() - t0, "tol": 1e-8}
        print("full", out["full"], flush=True)
        out["tt"] = {}
        for r in args.ranks:
            t0 = time.time()
            op = lr.LowRankGaNi(a_tt, (N, N, N), fmt="tt", rank=r, pinv_eps=0.1)
            res = lr.minres(op, E, maxit=60)
            out["tt"][str(r)] = {"Aeff": res["Aeff"], "iters": res["iters"], "rel_resid": res["rel_resid"],
                                 "seconds": time.time() - t0}
            print("tt", r, out["tt"][str(r)], flush=True)
    # the benchmark's TT solve (randomised rounding of the products, residual tolerance)
    opts = {"rank": 20, "rank_start": 10, "rank_step": 5, "pinv_eps": 0.1, "sketch_over": 10, "sketch_seed": 0,
            "tol": 3e-4, "stop_on_increase": 0, "maxit": 80}
    op = lr.LowRankGaNi(a_tt, (N, N, N), fmt="tt", rank=opts["rank"], pinv_eps=opts["pinv_eps"],
                        sketch=(opts["sketch_over"], opts["sketch_seed"]))
    count = {"applies": 0, "by_rank": {}}
    plain_apply = op.apply

    def counted(v):
        count["applies"] += 1
        key = str(op.rank)  # the current truncation rank of the rank-adapting iteration
        count["by_rank"][key] = count["by_rank"].get(key, 0) + 1
        return plain_apply(v)
    op.apply = counted
    t0 = time.time()
    res = lr.minres_rank_adaptive(op, E, opts["rank_start"], opts["rank_step"], tol=opts["tol"], maxit=opts["maxit"],
                                  stop_on_increase=opts["stop_on_increase"])
    out["tt_sketch"] = {"20": {"Aeff": res["Aeff"], "iters": res["iters"], "rel_resid": res["rel_resid"],
                               "rank": res["rank"], "applies": count["applies"], "applies_by_rank": count["by_rank"],
                               "seconds": time.time() - t0, "opts": opts}}
    print("tt_sketch", out["tt_sketch"], flush=True)
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
    print(path)


if __name__ == "__main__":
    main()
