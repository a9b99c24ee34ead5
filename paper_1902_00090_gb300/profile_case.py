"""Fixed-size solver run for kernel profiling (ncu) and quick timing.

Solves `--solves` held-out 128x128 problems of the synthetic trajectory set
(seeded), batched, with an iteration cap so that the run is short and every
launch sees the same Krylov-basis sizes from run to run.  Augmentation uses
`--k` random vectors (the kernels' work does not depend on their quality).

    python -m paper_1902_00090_gb300.profile_case --solves 64 --maxit 120 --k 20
"""
from __future__ import annotations

import argparse
import time

import numpy as np


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--solves", type=int, default=64)
    p.add_argument("--n", type=int, default=128)
    p.add_argument("--maxit", type=int, default=120)
    p.add_argument("--restart", type=int, default=200)
    p.add_argument("--k", type=int, default=20)
    p.add_argument("--precision", default="c64")
    p.add_argument("--repeat", type=int, default=1)
    p.add_argument("--orth", default=None, choices=[None, "cgs2", "dcgs2"])
    p.add_argument("--profile", action="store_true", help="print per-kernel-class time and GB/s")
    p.add_argument("--graphs", default="on", choices=["on", "off"],
                   help="step loop as a CUDA graph (on) or launched by the host (off)")
    p.add_argument("--basis", default="f32", choices=["f32", "f16"], help="Krylov basis storage (complex64)")
    a = p.parse_args()

    import torch
    import paper_1902_00090_gb300 as ddg
    from paper_1902_00090_gb300 import inputs

    g = inputs.grid_for(a.n, a.n)
    eps = inputs.trajectory_set(g, 2, (a.solves + 15) // 16)[: a.solves]
    ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for e in eps]
    bs = [ddg.fdfd_source(op, g.i_src, g.sigma_src, g.j_src) for op in ops]
    ctx = ddg.Context(orthogonalization=a.orth)
    ctx.set_graphs(a.graphs == "on")
    ctx.set_basis_storage(a.basis)
    U = None
    if a.k > 0:
        U = torch.as_tensor(inputs.random_complex(g.D, 7, shape=(a.k, g.D)), device="cuda")
    for r in range(a.repeat):
        if a.profile and r == a.repeat - 1:
            ctx.profile_enable(True)
        torch.cuda.synchronize()
        t0 = time.time()
        if U is None:
            xs, infos, st = ddg.gmres_solve_batched(ctx, ops, bs, tol=1e-6, restart=a.restart, maxit=a.maxit,
                                                    precision=a.precision)
        else:
            xs, infos, st = ddg.augmented_gmres_solve_batched(ctx, ops, bs, [U] * len(ops), tol=1e-6,
                                                              restart=a.restart, maxit=a.maxit,
                                                              precision=a.precision)
        torch.cuda.synchronize()
        dt = time.time() - t0
        print(f"run {r}: {len(ops)} solves, {dt * 1e3:.1f} ms, iters mean "
              f"{np.mean([i['iters'] for i in infos]):.1f}, status {st}, launches {ctx.launches}")
    if a.profile:
        for name, (ms, by, n) in ctx.profile_read().items():
            if n:
                print(f"  {name:10s} {n:6d} launches {ms:9.2f} ms  {by / max(ms, 1e-9) / 1e6:8.1f} GB/s "
                      f" {ms * 1e3 / n:8.1f} us/launch")


if __name__ == "__main__":
    main()
