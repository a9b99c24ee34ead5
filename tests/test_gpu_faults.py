"""Failure detection on the GPU without a GPU fault.

(a) The solver's bounded device waits: with a wait limit of zero the Arnoldi
kernels' waits for bulk copies of basis columns run out almost at once; each
block that gives up stops its reduction, still waits (at the default 1 s bound)
for the copies it issued, and raises a flag that the host reads: the call
returns DDG_ETIMEOUT, and the same context then solves correctly.
(b) Allocation failure, made on the host: a workspace limit below what a
solve needs makes the call return DDG_ENOMEM without allocating; the context
works again once the limit is lifted.
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

DDG_ENOMEM, DDG_ETIMEOUT = 2, 6


def problems(n=8, side=128):
    g = inputs.grid_for(side, side)
    eps = inputs.trajectory_set(g, 2, (n + 15) // 16)[:n]
    ops = [ddg.fdfd_operator(g, torch.as_tensor(e, device="cuda")) for e in eps]
    bs = [ddg.fdfd_source(op, g.i_src, g.sigma_src, g.j_src) for op in ops]
    return g, eps, ops, bs


def true_residual(g, eps, x):
    A = fdfd.operator_for(g, eps)
    b = fdfd.source_for(g)
    return np.linalg.norm(b - A @ x) / np.linalg.norm(b)


@pytest.mark.parametrize("graphs", [True, False])
def test_wait_limit_runs_out_and_the_context_stays_usable(graphs):
    # 32 solves of 256x256 with the FP32 basis: the reduction kernel streams
    # at the bandwidth limit, so its copies are regularly still in flight when
    # a block comes to use them, and a wait limit of zero runs out
    g, eps, ops, bs = problems(32, 256)
    ctx = ddg.Context()
    ctx.set_basis_storage("f32")
    ctx.set_graphs(graphs)
    ctx.set_wait_limit(0)
    with pytest.raises(ddg.DdgError) as ei:
        ddg.gmres_solve_batched(ctx, ops, bs, tol=1e-6, restart=200, maxit=400, precision="c64")
    assert ei.value.status == DDG_ETIMEOUT
    assert "time limit" in str(ei.value)
    # the default limit again: the same context solves, and the device is sane
    g, eps, ops, bs = problems()
    ctx.set_wait_limit(10**9)
    xs, infos, st = ddg.gmres_solve_batched(ctx, ops[:2], bs[:2], tol=1e-6, restart=200, maxit=5000,
                                            precision="c64")
    assert st == 0
    for e, x in zip(eps[:2], xs):
        assert true_residual(g, e, x.cpu().numpy()) <= 1e-6


def test_half_basis_with_a_zero_wait_limit_stays_usable():
    # the half-precision basis leaves the reduction latency-bound: its copies
    # have mostly landed when they are used, so a zero limit may or may not run
    # out; either way the call returns, and the context then solves correctly
    g, eps, ops, bs = problems(32, 256)
    ctx = ddg.Context()
    ctx.set_basis_storage("f16")
    ctx.set_wait_limit(0)
    try:
        ddg.gmres_solve_batched(ctx, ops, bs, tol=1e-6, restart=200, maxit=400, precision="c64")
    except ddg.DdgError as e:
        assert e.status == DDG_ETIMEOUT
    ctx.set_wait_limit(10**9)
    g, eps, ops, bs = problems()
    xs, infos, st = ddg.gmres_solve_batched(ctx, ops[:2], bs[:2], tol=1e-6, restart=200, maxit=5000,
                                            precision="c64")
    assert st == 0
    for e, x in zip(eps[:2], xs):
        assert true_residual(g, e, x.cpu().numpy()) <= 1e-6


def test_wait_limit_is_checked():
    ctx = ddg.Context()
    for bad in (-1, 10**11):
        with pytest.raises(ddg.DdgError):
            ctx.set_wait_limit(bad)


def test_workspace_limit_gives_enomem_and_can_be_lifted():
    g, eps, ops, bs = problems(4)
    ctx = ddg.Context()
    ctx.set_workspace_limit(1 << 20)      # 1 MiB: far below four 128x128 GMRES(200) bases
    with pytest.raises(ddg.DdgError) as ei:
        ddg.gmres_solve_batched(ctx, ops, bs, tol=1e-6, restart=200, maxit=5000, precision="c64")
    assert ei.value.status == DDG_ENOMEM and "limit" in str(ei.value)
    assert ctx.workspace_bytes == 0
    ctx.set_workspace_limit(0)
    xs, infos, st = ddg.gmres_solve_batched(ctx, ops, bs, tol=1e-6, restart=200, maxit=5000, precision="c64")
    assert st == 0 and all(i["converged"] for i in infos)
    held = ctx.workspace_bytes
    assert held > (1 << 20)
    # a limit below the workspace held frees it; one at least as large keeps solving
    ctx.set_workspace_limit(held)
    assert ctx.workspace_bytes == held
    xs2, infos2, st2 = ddg.gmres_solve_batched(ctx, ops, bs, tol=1e-6, restart=200, maxit=5000, precision="c64")
    assert st2 == 0 and ctx.workspace_bytes == held
    ctx.set_workspace_limit(1 << 20)
    assert ctx.workspace_bytes == 0
