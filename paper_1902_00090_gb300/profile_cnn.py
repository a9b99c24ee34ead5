"""Fixed-size run of the subspace CNN's forward pass, for kernel profiling (ncu)
and quick timing.

Predicts the subspaces of `--batch` 128x128 problems of the synthetic
trajectory set with the default network (6 levels, 32-128 channels, k = 8,
He-initialised weights: the kernels' work does not depend on their values).

    python -m paper_1902_00090_gb300.profile_cnn --batch 64 --repeat 5
"""
from __future__ import annotations

import argparse
import time


def main():
    p = argparse.ArgumentParser()
    p.add_argument("--batch", type=int, default=64)
    p.add_argument("--n", type=int, default=128)
    p.add_argument("--k", type=int, default=8)
    p.add_argument("--repeat", type=int, default=5)
    p.add_argument("--tensor-cores", default="on", choices=["on", "off"])
    a = p.parse_args()

    import torch
    import paper_1902_00090_gb300 as ddg
    from paper_1902_00090_gb300 import inputs

    g = inputs.grid_for(a.n, a.n)
    eps = inputs.trajectory_set(g, 2, (a.batch + 15) // 16)[: a.batch]
    ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for e in eps]
    P = ddg.Predictor(k=a.k)
    P.init_he(seed=0)
    P.set_tensor_cores(a.tensor_cores == "on")
    src = (g.i_src, g.sigma_src, g.j_src)
    U = [torch.empty((a.k, g.D), dtype=torch.complex128, device="cuda") for _ in ops]
    for r in range(a.repeat):
        torch.cuda.synchronize()
        t0 = time.time()
        P.predict(ops, src, U=U)
        torch.cuda.synchronize()
        print(f"run {r}: {a.batch} predictions, {(time.time() - t0) * 1e3:.2f} ms, launches {P.launches}")


if __name__ == "__main__":
    main()
