"""Recycling along design trajectories (gmres_solve_trajectories) against the
oracle: step t of each trajectory is the oracle's augmented GMRES with the
subspace [U | x_{t-1}] (U the problem's predicted vectors, x_{t-1} the
trajectory's previous solution as the GPU computed it), in complex128."""
import numpy as np
import pytest

from oracle import fdfd, gmres, losses
from paper_1902_00090_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1902_00090_gb300 as ddg  # noqa: E402

G = inputs.Grid(nx=48, ny=40, npml=6, i_src=12, sigma_src=4.0, slab_cells=4, design=(12, 36, 16, 24))


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=torch.complex128)


@pytest.mark.parametrize("k", [0, 2])
def test_trajectory_recycling_matches_oracle(k):
    n_traj, n_steps, tol = 2, 3, 1e-8
    eps = [inputs.trajectory_eps(G, 2, 40 + r, steps=n_steps) for r in range(n_traj)]
    ops = [[ddg.fdfd_operator(G, torch.as_tensor(e, device="cuda")) for e in tr] for tr in eps]
    bs = [[ddg.fdfd_source(op, G.i_src, G.sigma_src, G.j_src) for op in tr] for tr in ops]
    U = None
    if k:
        U = [[dev(inputs.random_complex(G.D, 100 * r + t, shape=(k, G.D))) for t in range(n_steps)]
             for r in range(n_traj)]
    ctx = ddg.Context()
    ctx.set_fallback(2.0)              # as the oracle: never fall back
    ctx.set_augmented_cycles(10**6)    # and keep the subspace in every cycle
    x, infos, st = ddg.gmres_solve_trajectories(ctx, ops, bs, U, tol=tol, restart=30, maxit=3000,
                                                precision="c128")
    assert st == 0
    b = fdfd.source_for(G)
    for r in range(n_traj):
        for t in range(n_steps):
            A = fdfd.operator_for(G, eps[r][t])
            xh = x[r][t].cpu().numpy()
            inf = infos[r][t]
            assert np.linalg.norm(b - A @ xh) / np.linalg.norm(b) <= tol
            cols = ([U[r][t].cpu().numpy()] if k else []) + ([x[r][t - 1].cpu().numpy()[None]] if t else [])
            if not cols:
                xo, io = gmres.plain_gmres(A, b, tol=tol, restart=30, maxit=3000)
            else:
                V = np.concatenate(cols).T
                xo, io = gmres.augmented_gmres(A, b, V, tol=tol, restart=30, maxit=3000)
                # the V-only step: Eq. 6's minimum over the recycled subspace
                assert abs(inf["first_step_rel_residual"] - np.sqrt(losses.residual_loss(A, V, b))) <= 1e-10
            assert abs(inf["iters"] - io.iters) <= 1, (r, t, inf, io)
            assert np.linalg.norm(xh - xo) / np.linalg.norm(xo) <= 1e-6
            if t:
                # the previous design's field is a good start: most of the
                # residual is gone before the first Krylov step
                assert inf["first_step_rel_residual"] < 0.5


def test_trajectory_recycling_rejects_bad_arguments():
    ops = [[ddg.fdfd_operator(G, torch.as_tensor(inputs.background_eps(G), device="cuda"))]]
    bs = [[ddg.fdfd_source(ops[0][0], G.i_src, G.sigma_src, G.j_src)]]
    big = [[dev(inputs.random_complex(G.D, 1, shape=(32, G.D)))]]
    with pytest.raises(ddg.DdgError):
        ddg.gmres_solve_trajectories(ddg.Context(), ops, bs, big)     # k + 1 = 33 columns > 32


def test_queue_over_trajectories_equals_one_call():
    # gmres_solve_queue_trajectories: groups of trajectories on concurrent
    # lanes, each group solved by gmres_solve_trajectories; every solve's
    # result is that of its own trajectory, bitwise, in any group
    n_traj, n_steps = 3, 2
    eps = [inputs.trajectory_eps(G, 2, 50 + r, steps=n_steps) for r in range(n_traj)]
    ops = [[ddg.fdfd_operator(G, torch.as_tensor(e, device="cuda")) for e in tr] for tr in eps]
    bs = [[ddg.fdfd_source(op, G.i_src, G.sigma_src, G.j_src) for op in tr] for tr in ops]
    U = [[dev(inputs.random_complex(G.D, 200 + 10 * r + t, shape=(2, G.D))) for t in range(n_steps)]
         for r in range(n_traj)]
    ctx = ddg.Context()
    x1, i1, s1 = ddg.gmres_solve_trajectories(ctx, ops, bs, U, tol=1e-7, restart=30, maxit=3000, precision="c64")
    lanes = [ddg.Context(), ddg.Context()]
    x2, i2, s2 = ddg.gmres_solve_queue_trajectories(lanes, ops, bs, U, traj_per_group=1, tol=1e-7, restart=30,
                                                    maxit=3000, precision="c64")
    assert s1 == s2 == 0
    for r in range(n_traj):
        for t in range(n_steps):
            assert i1[r][t] == i2[r][t]
            assert torch.equal(x1[r][t], x2[r][t])
