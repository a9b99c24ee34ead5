"""Oracle step counts of plain GMRES(200) (complex128, tol 1e-6) on held-out
problems of the benchmark's workloads, for the side-by-side report of Krylov
steps (GPU counts come from bench.py's `plain` object).  TEST INFRASTRUCTURE
ONLY: calls the oracle and the seeded input generators, nothing of the CUDA
path.

    python -m oracle.iterations_report [--procs 8]                       # 64 held-out 128x128 problems
    python -m oracle.iterations_report --workload splitter256 --count 4  # held-out 256x256 at 1300 / 1550 nm
"""
from __future__ import annotations

import argparse
import json
import os


def _one(args):
    workload, j = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import fdfd, gmres
    from paper_1902_00090_gb300 import inputs
    if workload == "pca128":
        g = inputs.grid_128()
        eps = inputs.trajectory_set(g, 2, 32, 16)[28 * 16 + j]
        label = "128x128"
    else:
        # the two-wavelength workload: permittivity j // 2 of held-out
        # trajectory 256 (seed PCG64(3256)), at 1300 nm (even j) or 1550 nm
        lam = (1300e-9, 1550e-9)[j % 2]
        g = inputs.grid_for(256, 256, wavelength=lam)
        eps = inputs.trajectory_eps(g, 3, 256)[j // 2]
        label = f"256x256 {int(round(lam * 1e9))} nm, step {j // 2}"
    A = fdfd.operator_for(g, eps).tocsr()
    b = fdfd.source_for(g)
    _, info = gmres.plain_gmres(A, b, tol=1e-6, restart=200, maxit=20000)
    return j, label, info.iters, info.cycles, info.true_rel_residual


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    p.add_argument("--count", type=int, default=64)
    p.add_argument("--workload", default="pca128", choices=["pca128", "splitter256"])
    a = p.parse_args()
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(min(a.procs, a.count)) as pool:
        res = sorted(pool.map(_one, [(a.workload, j) for j in range(a.count)]))
    its = [r[2] for r in res]
    print(json.dumps({"solver": "oracle plain GMRES(200), complex128, tol 1e-6, cap 20000",
                      "workload": a.workload, "problems": len(res),
                      "iters_mean": sum(its) / len(its), "iters_min": min(its), "iters_max": max(its),
                      "per_problem": [{"j": r[0], "problem": r[1], "iters": r[2], "cycles": r[3],
                                       "true_rel_residual": r[4]} for r in res]}))


if __name__ == "__main__":
    main()
