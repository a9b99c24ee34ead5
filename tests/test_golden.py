"""Fixtures under tests/golden/: a value the paper prints (the size of its
linear system) and stored outputs of the oracle on small seeded problems
(written by tests/golden/make_golden.py, which calls only oracle/)."""
import importlib.util
import os

import numpy as np

from oracle import fdfd, gmres, pca
from paper_1902_00090_gb300 import inputs

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def rows(name):
    with open(os.path.join(HERE, name)) as f:
        return [ln.split() for ln in f if ln.strip() and not ln.startswith("#")]


def test_paper_grid_has_one_unknown_per_cell():
    # Fig. 1: 20 nm cells, 229 x 90 = 20,610 unknowns (2D TM, Ez only)
    (nx, ny, dx_nm, unknowns), = [tuple(int(v) for v in r) for r in rows("paper_grid.txt")]
    g = inputs.Grid(nx=nx, ny=ny, dx=dx_nm * 1e-9, npml=10, i_src=20, sigma_src=6.0, slab_cells=8)
    A = fdfd.operator_for(g, inputs.background_eps(g))
    b = fdfd.source_for(g)
    assert A.shape == (unknowns, unknowns) and b.shape == (unknowns,)
    assert A.nnz <= 5 * unknowns


def test_oracle_reproduces_its_stored_outputs():
    spec = importlib.util.spec_from_file_location("make_golden", os.path.join(HERE, "make_golden.py"))
    mk = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mk)
    stored = {r[0]: r[1:] for r in rows("oracle_regression.txt")}
    for name, g, eps in mk.cases():
        A = fdfd.operator_for(g, eps)
        b = fdfd.source_for(g)
        _, ip = gmres.plain_gmres(A, b, tol=1e-8, restart=25, maxit=5000)
        V = inputs.random_complex(g.D, 7, shape=(3, g.D)).T
        _, ia = gmres.augmented_gmres(A, b, V, tol=1e-8, restart=25, maxit=5000, aug_cycles=1)
        it, cyc, res, ait, afirst, ares = stored[name]
        assert abs(ip.iters - int(it)) <= 1 and abs(ia.iters - int(ait)) <= 1
        assert np.isclose(ip.true_rel_residual, float(res), rtol=1e-3)
        assert np.isclose(ia.first_step_rel_residual, float(afirst), rtol=1e-10)
        assert np.isclose(ia.true_rel_residual, float(ares), rtol=1e-3)
    g = inputs.grid_for(32, 32, npml=6, i_src=8, sigma_src=3.0, slab_cells=4)
    F = [np.linalg.solve(fdfd.operator_for(g, e).toarray(), fdfd.source_for(g))
         for e in inputs.trajectory_eps(g, 7, 0, steps=12)]
    _, s = pca.pca_basis(np.stack(F, axis=1), 4)
    assert np.allclose(s[:4], [float(v) for v in stored["pca32"]], rtol=1e-10)
