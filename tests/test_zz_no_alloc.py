"""gmres_solve_noalloc: the allocation-free solve gives gmres_solve's results.

Callers whose device memory belongs entirely to another allocator, or that
cannot afford the device synchronisation of cudaMalloc/cudaFree, use this
entry point: it keeps its workspace in a static device array instead of
allocating.  Checked through the C ABI against gmres_solve on two calls in a
row (the array keeps the previous call's contents), in both precisions.
"""
import numpy as np
import pytest

from oracle import fdfd
from paper_1902_00090_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1902_00090_gb300 as ddg  # noqa: E402


def _problem(n, seed):
    g = inputs.Grid(nx=n, ny=n, npml=10 if n >= 64 else 4, i_src=20 if n >= 64 else 6,
                    sigma_src=6.0 if n >= 64 else 2.0)
    eps = inputs.bernoulli_eps(g, seed) if n == 128 else inputs.background_eps(g) + \
        np.random.default_rng(seed).random((g.ny, g.nx))
    op = ddg.fdfd_operator(g, torch.as_tensor(eps, device="cuda"))
    b = ddg.fdfd_source(op, g.i_src, g.sigma_src, g.j_src)
    return g, eps, op, b


@pytest.mark.parametrize("prec,n,restart", [("c64", 128, 200), ("c128", 64, 100)])
def test_noalloc_matches_gmres_solve_twice(prec, n, restart):
    ctx = ddg.Context()
    for call, seed in enumerate((0, 1)):
        g, eps, op, b = _problem(n, seed)
        x_ref, i_ref, s_ref = ddg.gmres_solve(ctx, op, b, tol=1e-6, restart=restart, maxit=5000,
                                              precision=prec)
        x, info, st = ddg.gmres_solve_noalloc(op, b, tol=1e-6, restart=restart, maxit=5000, precision=prec)
        assert st == s_ref == 0, (call, st, info)
        assert info["iters"] == i_ref["iters"] and info["cycles"] == i_ref["cycles"]
        xr, xn = x_ref.cpu().numpy(), x.cpu().numpy()
        assert np.linalg.norm(xn - xr) <= 1e-12 * np.linalg.norm(xr)
        A = fdfd.operator_for(g, eps)
        bh = b.cpu().numpy()
        assert np.linalg.norm(bh - A @ xn) / np.linalg.norm(bh) <= 1e-6


def test_noalloc_rejects_sizes_beyond_its_buffer():
    g, eps, op, b = _problem(128, 0)
    with pytest.raises(ddg.DdgError) as e:
        ddg.gmres_solve_noalloc(op, b, tol=1e-6, restart=200, precision="c128")
    assert e.value.status == 1 and "static" in str(e.value)
    # a rejected call leaves the entry point usable
    x, info, st = ddg.gmres_solve_noalloc(op, b, tol=1e-6, restart=200, precision="c64")
    assert st == 0 and info["converged"]
