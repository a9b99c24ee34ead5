"""Oracle step counts of plain GMRES(200) on the benchmark's 64 held-out 128x128
problems (complex128, tol 1e-6), for the side-by-side report of Krylov steps
(GPU counts come from bench.py's `plain` object).  TEST INFRASTRUCTURE ONLY:
calls the oracle and the seeded input generators, nothing of the CUDA path.

    python -m oracle.iterations_report [--procs 8]
"""
from __future__ import annotations

import argparse
import json
import os


def _one(args):
    j, = args
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import fdfd, gmres
    from paper_1902_00090_gb300 import inputs
    g = inputs.grid_128()
    eps = inputs.trajectory_set(g, 2, 32, 16)[28 * 16 + j]
    A = fdfd.operator_for(g, eps).tocsr()
    b = fdfd.source_for(g)
    _, info = gmres.plain_gmres(A, b, tol=1e-6, restart=200, maxit=20000)
    return j, info.iters, info.cycles, info.true_rel_residual


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--procs", type=int, default=os.cpu_count() or 1)
    p.add_argument("--count", type=int, default=64)
    a = p.parse_args()
    import multiprocessing as mp
    with mp.get_context("spawn").Pool(a.procs) as pool:
        res = sorted(pool.map(_one, [(j,) for j in range(a.count)]))
    its = [r[1] for r in res]
    print(json.dumps({"solver": "oracle plain GMRES(200), complex128, tol 1e-6", "problems": len(res),
                      "iters_mean": sum(its) / len(its), "iters_min": min(its), "iters_max": max(its),
                      "per_problem": [{"j": r[0], "iters": r[1], "cycles": r[2], "true_rel_residual": r[3]}
                                      for r in res]}))


if __name__ == "__main__":
    main()
