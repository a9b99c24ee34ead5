"""Writes oracle_regression.txt: outputs of the CPU oracle on small seeded
problems, kept so that a change to the oracle's arithmetic shows up in the
CPU tests.  Calls only oracle/ and the seeded input generators.

    python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

from oracle import fdfd, gmres, pca  # noqa: E402
from paper_1902_00090_gb300 import inputs  # noqa: E402


def cases():
    """(name, grid, eps) of the regression problems."""
    out = []
    for n, npml, seed in [(16, 3, 0), (24, 4, 1), (32, 6, 2)]:
        g = inputs.Grid(nx=n, ny=n + 3, npml=npml, i_src=2 * npml, sigma_src=n / 8, slab_cells=2)
        eps = inputs.background_eps(g) + 0.5 * np.random.default_rng(seed).random((g.ny, g.nx))
        out.append((f"n{n}_s{seed}", g, eps))
    return out


def main():
    lines = ["# oracle outputs; rows n*: name plain_iters plain_cycles plain_true_res aug_iters "
             "aug_first_step aug_true_res (GMRES(25) to 1e-8, 3 random V vectors, first-cycle policy); "
             "row pca32: sigma_1..sigma_4 of 12 trajectory fields on a 32x32 grid"]
    for name, g, eps in cases():
        A = fdfd.operator_for(g, eps)
        b = fdfd.source_for(g)
        _, ip = gmres.plain_gmres(A, b, tol=1e-8, restart=25, maxit=5000)
        V = inputs.random_complex(g.D, 7, shape=(3, g.D)).T
        _, ia = gmres.augmented_gmres(A, b, V, tol=1e-8, restart=25, maxit=5000, aug_cycles=1)
        lines.append(f"{name} {ip.iters} {ip.cycles} {ip.true_rel_residual:.12e} {ia.iters} "
                     f"{ia.first_step_rel_residual:.12e} {ia.true_rel_residual:.12e}")
    g = inputs.grid_for(32, 32, npml=6, i_src=8, sigma_src=3.0, slab_cells=4)
    F = []
    for e in inputs.trajectory_eps(g, 7, 0, steps=12):
        F.append(np.linalg.solve(fdfd.operator_for(g, e).toarray(), fdfd.source_for(g)))
    _, s = pca.pca_basis(np.stack(F, axis=1), 4)
    lines.append("pca32 " + " ".join(f"{v:.12e}" for v in s[:4]))
    with open(os.path.join(HERE, "oracle_regression.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
