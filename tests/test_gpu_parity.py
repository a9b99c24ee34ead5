"""GPU parity: the CUDA library (through its C ABI) against the CPU oracle.

Bars: operator and source element by element (FP64 round-off, FP32 round-off
for the complex64 stencil); solves by the true relative residual recomputed
with the oracle's sparse operator (<= tol) and the relative L2 distance to the
oracle's direct solution (<= 1e-5 at tol = 1e-6, i.e. forward-error factor 10).
"""
import dataclasses

import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fdfd, gmres, losses
from paper_1902_00090_gb300 import inputs

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_1902_00090_gb300 as ddg  # noqa: E402


@pytest.fixture(scope="module")
def ctx():
    c = ddg.Context()
    c.set_fallback(2.0)           # parity with the oracle's augmented method: never fall back,
    c.set_augmented_cycles(10**6)  # and keep V in every restart cycle
    return c


def dev(a, dtype=torch.complex128):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    return t.detach().cpu().numpy()


def rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


GRIDS = [
    inputs.Grid(nx=37, ny=29, npml=5, i_src=9, sigma_src=3.0),      # ragged: not a multiple of any tile
    inputs.Grid(nx=128, ny=128),
    inputs.Grid(nx=192, ny=64, npml=10, i_src=20),
    inputs.Grid(nx=3, ny=5, npml=1, i_src=1, sigma_src=1.0, slab_cells=1),   # smallest allowed
    # even widths take the two-cells-per-thread complex64 stencil: a row that
    # ends inside a warp, the smallest such row, and rows over several blocks
    inputs.Grid(nx=38, ny=9, npml=3, i_src=5, sigma_src=2.0, slab_cells=2),
    inputs.Grid(nx=4, ny=5, npml=1, i_src=1, sigma_src=1.0, slab_cells=1),
    inputs.Grid(nx=1030, ny=6, npml=2, i_src=9, sigma_src=2.0, slab_cells=2),
    # the stencil's four-row groups: fewer rows than one group (row ny wraps to
    # row 0, rows past it feed no output), and a last group with one row
    inputs.Grid(nx=6, ny=3, npml=1, i_src=1, sigma_src=1.0, slab_cells=1),
    inputs.Grid(nx=520, ny=13, npml=2, i_src=9, sigma_src=2.0, slab_cells=2),
]


def problem(g, seed=0):
    rng = np.random.default_rng(seed)
    eps = inputs.background_eps(g) + 3.0 * rng.random((g.ny, g.nx))
    return eps


@pytest.mark.parametrize("g", GRIDS, ids=lambda g: f"{g.nx}x{g.ny}")
def test_operator_matches_oracle(g):
    eps = problem(g)
    A = fdfd.operator_for(g, eps)
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    x = inputs.random_complex(g.D, seed=1)
    y = host(ddg.fdfd_apply(op, dev(x)))
    yo = A @ x
    assert np.max(np.abs(y - yo)) <= 1e-13 * np.max(np.abs(yo))
    y32 = host(ddg.fdfd_apply_c64(op, dev(x, torch.complex64)))
    assert rel(y32, yo) <= 2e-6


@pytest.mark.parametrize("g", GRIDS[:3], ids=lambda g: f"{g.nx}x{g.ny}")
def test_source_matches_oracle(g):
    eps = problem(g)
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    b = host(ddg.fdfd_source(op, g.i_src, g.sigma_src, g.j_src))
    bo = fdfd.source_for(g)
    assert np.max(np.abs(b - bo)) <= 1e-15 * np.max(np.abs(bo))


def test_operator_rejects_bad_eps():
    g = inputs.Grid(nx=16, ny=16, npml=3, i_src=4)
    for bad in (-1.0, 0.0, float("nan"), float("inf")):
        eps = inputs.background_eps(g)
        eps[3, 5] = bad
        with pytest.raises(ddg.DdgError) as e:
            ddg.fdfd_operator(g, dev(eps, torch.float64))
        assert e.value.status == 1


def small(n=16, npml=3, seed=0):
    g = inputs.Grid(nx=n, ny=n, npml=npml, i_src=n // 4, sigma_src=n / 8, slab_cells=max(2, n // 16))
    rng = np.random.default_rng(seed)
    eps = inputs.background_eps(g) + 0.5 * rng.random((g.ny, g.nx))
    return g, eps, fdfd.operator_for(g, eps), fdfd.source_for(g)


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_dense_direct_16x16(ctx, prec):
    g, eps, A, b = small(16)
    x_ref = np.linalg.solve(A.toarray(), b)
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    tol = 1e-12 if prec == "c128" else 1e-10
    x, info, st = ddg.gmres_solve(ctx, op, dev(b), tol=tol, restart=60, maxit=3000, precision=prec)
    assert st == 0 and info["converged"]
    assert rel(host(x), x_ref) <= (1e-10 if prec == "c128" else 1e-8)
    assert np.linalg.norm(b - A @ host(x)) / np.linalg.norm(b) <= tol


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_longest_restart(ctx, prec):
    # restart 1024 (the largest accepted): the Arnoldi kernels' shared memory
    # (Givens staging, coefficient vectors, back substitution) exceeds 48 KB
    g, eps, A, b = small(32, npml=6, seed=2)
    x_ref = spla.spsolve(A.tocsc(), b)
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    x, info, st = ddg.gmres_solve(ctx, op, dev(b), tol=1e-8, restart=1024, maxit=5000, precision=prec)
    assert st == 0 and info["converged"] and info["cycles"] <= (2 if prec == "c128" else 3)
    assert np.linalg.norm(b - A @ host(x)) / np.linalg.norm(b) <= 1e-8
    assert rel(host(x), x_ref) <= 1e-6
    xo, io = gmres.plain_gmres(A, b, tol=1e-8, restart=1024, maxit=5000)
    print(f"restart 1024 {prec}: {info['iters']} GPU iterations, oracle {io.iters}")


def test_plain_iterations_match_oracle_c128(ctx):
    # Same algorithm in the same precision: equal Krylov step counts (up to a
    # step at a tolerance crossing) and the same solution.
    g, eps, A, b = small(32, npml=6, seed=1)
    xo, io = gmres.plain_gmres(A, b, tol=1e-9, restart=25, maxit=3000)
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    x, info, st = ddg.gmres_solve(ctx, op, dev(b), tol=1e-9, restart=25, maxit=3000)
    assert st == 0
    assert abs(info["iters"] - io.iters) <= 1
    assert info["cycles"] == io.cycles
    assert rel(host(x), xo) <= 1e-6


@pytest.fixture(scope="module")
def config1():
    g = inputs.grid_128()
    eps = inputs.bernoulli_eps(g, 0)
    A = fdfd.operator_for(g, eps)
    b = fdfd.source_for(g)
    xd = spla.spsolve(A.tocsc(), b)
    return g, eps, A, b, xd


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_config1_plain_full_size(ctx, config1, prec):
    g, eps, A, b, xd = config1
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    bd = ddg.fdfd_source(op, g.i_src, g.sigma_src, g.j_src)
    x, info, st = ddg.gmres_solve(ctx, op, bd, tol=1e-6, restart=200, maxit=5000, precision=prec)
    assert st == 0 and info["converged"]
    xh = host(x)
    true_res = np.linalg.norm(b - A @ xh) / np.linalg.norm(b)
    assert true_res <= 1e-6
    assert abs(true_res - info["true_rel_residual"]) <= 1e-9
    assert rel(xh, xd) <= 1e-5
    # oracle GMRES(200) needs 1534 Krylov steps on this problem
    assert 1300 <= info["iters"] <= 2200


def rand_V(D, N, seed):
    return inputs.random_complex(D, seed, shape=(N, D))


def test_fp32_only_to_1e4(ctx, config1):
    # DDG_C64_ONLY: no FP64 refinement; the solver judges convergence on an FP32
    # residual, so the FP64 residual recomputed by the oracle meets the
    # tolerance up to FP32 round-off, and the field is within the measured
    # forward-error factor (3.6 at 1e-6 on this problem) times the tolerance.
    g, eps, A, b, xd = config1
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    x, info, st = ddg.gmres_solve(ctx, op, dev(b), tol=1e-4, restart=200, maxit=5000, precision="c64_only")
    assert st == 0 and info["converged"]
    xh = host(x)
    r = np.linalg.norm(b - A @ xh) / np.linalg.norm(b)
    assert r <= 1.02e-4
    assert abs(r - info["true_rel_residual"]) <= 2e-6
    assert rel(xh, xd) <= 1e-3
    # the same problem through the refinement path stops at the same tolerance
    x2, info2, st2 = ddg.gmres_solve(ctx, op, dev(b), tol=1e-4, restart=200, maxit=5000, precision="c64")
    assert st2 == 0 and abs(info2["iters"] - info["iters"]) <= 0.1 * info["iters"] + 5


def test_fp32_only_augmented(ctx):
    # augmented path in DDG_C64_ONLY with a subspace holding a nearby solution
    g, eps, A, b = small(48, npml=6, seed=5)
    # the subspace: the solution of a nearby problem (eps perturbed) and noise
    eps2 = eps + 0.05 * np.random.default_rng(6).random(eps.shape)
    x2 = spla.spsolve(fdfd.operator_for(g, eps2).tocsc(), b)
    V = np.stack([x2, inputs.random_complex(g.D, 41)])
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    x, info, st = ddg.augmented_gmres_solve(ctx, op, dev(b), dev(V), tol=1e-4, restart=60, maxit=5000,
                                            precision="c64_only")
    assert st == 0 and info["converged"]
    assert np.linalg.norm(b - A @ host(x)) / np.linalg.norm(b) <= 1.02e-4
    assert info["first_step_rel_residual"] < 0.5


def test_augmented_matches_oracle_c128(ctx):
    g, eps, A, b = small(24, npml=4, seed=9)
    V = rand_V(g.D, 4, 9)
    xo, io = gmres.augmented_gmres(A, b, V.T, tol=1e-9, restart=30)
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    x, info, st = ddg.augmented_gmres_solve(ctx, op, dev(b), dev(V), tol=1e-9, restart=30)
    assert st == 0 and info["converged"] and not info["fallback_used"]
    assert abs(info["iters"] - io.iters) <= 1
    assert rel(host(x), xo) <= 1e-6
    lres = losses.residual_loss(A, V.T, b)
    assert abs(info["first_step_rel_residual"] - np.sqrt(lres)) <= 1e-10
    assert abs(info["first_step_rel_residual"] - io.first_step_rel_residual) <= 1e-10


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_augmented_solution_in_V_needs_no_krylov_step(ctx, prec):
    g, eps, A, b = small(24, npml=4, seed=6)
    xd = spla.spsolve(A.tocsc(), b)
    V = np.stack([inputs.random_complex(g.D, 1), xd, inputs.random_complex(g.D, 2)])
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    x, info, st = ddg.augmented_gmres_solve(ctx, op, dev(b), dev(V), tol=1e-6, restart=30,
                                            precision=prec)
    assert st == 0 and info["converged"]
    if prec == "c128":
        assert info["first_step_rel_residual"] <= 1e-12
        assert info["iters"] == 0
    else:
        assert info["first_step_rel_residual"] <= 1e-6
    assert rel(host(x), xd) <= 1e-6


def test_rank_deficient_V_falls_back_to_plain(ctx):
    g, eps, A, b = small(24, npml=4, seed=3)
    v = inputs.random_complex(g.D, 5)
    V = np.stack([v, 2.0 * v, inputs.random_complex(g.D, 6)])   # duplicate direction
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    x, info, st = ddg.augmented_gmres_solve(ctx, op, dev(b), dev(V), tol=1e-8, restart=30)
    assert st == 0 and info["converged"] and info["fallback_used"] == 1
    assert np.linalg.norm(b - A @ host(x)) / np.linalg.norm(b) <= 1e-8


def test_zero_rhs_gives_zero_solution(ctx):
    g, eps, A, b = small(16)
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    x0 = dev(inputs.random_complex(g.D, 3))
    x, info, st = ddg.gmres_solve(ctx, op, dev(np.zeros(g.D, complex)), x=x0, tol=1e-6)
    assert st == 0 and info["converged"] and info["iters"] == 0
    assert np.all(host(x) == 0)


def test_iteration_cap_reports_no_convergence(ctx):
    g, eps, A, b = small(32, npml=6)
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    x, info, st = ddg.gmres_solve(ctx, op, dev(b), tol=1e-12, restart=10, maxit=37)
    assert st == 4 and not info["converged"]
    assert info["iters"] == 37
    res = np.linalg.norm(b - A @ host(x)) / np.linalg.norm(b)
    assert abs(res - info["true_rel_residual"]) <= 1e-9 and res < 1.0


def test_initial_guess_is_used(ctx):
    g, eps, A, b = small(16)
    xd = np.linalg.solve(A.toarray(), b)
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    x, info, st = ddg.gmres_solve(ctx, op, dev(b), x=dev(xd), tol=1e-8)
    assert st == 0 and info["iters"] == 0


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_batched_uneven_sizes_match_single_solves(ctx, prec):
    specs = [(16, 3, 0), (37, 5, 1), (64, 8, 2), (24, 4, 3), (16, 3, 4)]
    ops, bs, As, bos = [], [], [], []
    for n, L, seed in specs:
        g = inputs.Grid(nx=n, ny=n + 3, npml=L, i_src=2 * L, sigma_src=n / 8, slab_cells=2)
        rng = np.random.default_rng(seed)
        eps = inputs.background_eps(g) + rng.random((g.ny, g.nx))
        ops.append(ddg.fdfd_operator(g, dev(eps, torch.float64)))
        As.append(fdfd.operator_for(g, eps))
        bo = fdfd.source_for(g)
        bos.append(bo)
        bs.append(dev(bo))
    xs, infos, st = ddg.gmres_solve_batched(ctx, ops, bs, tol=1e-8, restart=40, precision=prec)
    assert st == 0
    for i in range(len(specs)):
        x1, info1, _ = ddg.gmres_solve(ctx, ops[i], bs[i], tol=1e-8, restart=40, precision=prec)
        assert infos[i]["iters"] == info1["iters"]
        assert np.array_equal(host(xs[i]), host(x1))           # same kernels, same order: bitwise
        xh = host(xs[i])
        assert np.linalg.norm(bos[i] - As[i] @ xh) / np.linalg.norm(bos[i]) <= 1e-8


def test_batched_augmented_uneven(ctx):
    specs = [(24, 4, 0), (33, 5, 1), (40, 5, 2)]
    ops, bs, Us, As, bos = [], [], [], [], []
    for n, L, seed in specs:
        g = inputs.Grid(nx=n, ny=n, npml=L, i_src=2 * L, sigma_src=n / 8, slab_cells=2)
        rng = np.random.default_rng(seed)
        eps = inputs.background_eps(g) + rng.random((g.ny, g.nx))
        ops.append(ddg.fdfd_operator(g, dev(eps, torch.float64)))
        A = fdfd.operator_for(g, eps)
        As.append(A)
        bo = fdfd.source_for(g)
        bos.append(bo)
        bs.append(dev(bo))
        # a useful subspace: the solution of a perturbed problem plus noise
        A2 = fdfd.operator_for(g, eps * 1.01)
        Us.append(dev(np.stack([spla.spsolve(A2.tocsc(), bo), inputs.random_complex(g.D, seed)])))
    direct = [spla.spsolve(A.tocsc(), bo) for A, bo in zip(As, bos)]
    for prec in ("c128", "c64"):
        xs, infos, st = ddg.augmented_gmres_solve_batched(ctx, ops, bs, Us, tol=1e-7, restart=30,
                                                          precision=prec)
        assert st == 0
        for i in range(len(specs)):
            xh = host(xs[i])
            assert np.linalg.norm(bos[i] - As[i] @ xh) / np.linalg.norm(bos[i]) <= 1e-7
            # the field: within the forward-error factor 10 of the tolerance of the direct solution
            assert rel(xh, direct[i]) <= 1e-6
            assert infos[i]["first_step_rel_residual"] < 0.5


def test_pca_fit_matches_oracle_svd(ctx):
    from oracle import pca
    rng = np.random.default_rng(0)
    D, M, k = 3000, 90, 12
    F = (rng.standard_normal((D, M)) + 1j * rng.standard_normal((D, M))) * (0.8 ** np.arange(M))
    Uo, so = pca.pca_basis(F, k)
    U, sig = ddg.pca_fit(ctx, dev(F.T), k)
    Ug = host(U).T
    assert np.allclose(sig, so[:k], rtol=1e-10)
    assert np.linalg.norm(Ug.conj().T @ Ug - np.eye(k)) <= 1e-10
    assert np.linalg.norm(Ug @ Ug.conj().T - Uo @ Uo.conj().T, 2) <= 1e-8
    assert abs(pca.captured_energy(Ug, F) - pca.captured_energy(Uo, F)) <= 1e-10


def test_pca_fit_on_solved_training_fields(ctx):
    # fields solved by the library itself (the config-2 training flow, small)
    from oracle import pca
    g = inputs.grid_for(64, 64, i_src=20)
    eps_set = inputs.trajectory_set(g, 2, 4, steps=12)
    ops = [ddg.fdfd_operator(g, dev(e, torch.float64)) for e in eps_set]
    bs = [ddg.fdfd_source(op, g.i_src, g.sigma_src, g.j_src) for op in ops]
    xs, infos, st = ddg.gmres_solve_batched(ctx, ops, bs, tol=1e-10, restart=100, maxit=20000)
    assert st == 0
    F = torch.stack(xs)
    U, sig = ddg.pca_fit(ctx, F, 8)
    Uo, so = pca.pca_basis(host(F).T, 8)
    gap_ok = so[7] > 1.05 * so[8]
    assert np.allclose(sig, so[:8], rtol=1e-8)
    if gap_ok:
        Ug = host(U).T
        assert np.linalg.norm(Ug @ Ug.conj().T - Uo @ Uo.conj().T, 2) <= 1e-6


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_delayed_reorthogonalisation_matches_cgs2(prec):
    # Same Krylov space and Hessenberg matrix in exact arithmetic: equal step
    # counts up to a step at a tolerance crossing, both at the tolerance.
    g, eps, A, b = small(48, npml=6, seed=11)
    rng = np.random.default_rng(11)
    V = rand_V(g.D, 3, 11)
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    res = {}
    for scheme in ("cgs2", "dcgs2"):
        c = ddg.Context(orthogonalization=scheme)
        c.set_fallback(2.0)
        x, info, st = ddg.gmres_solve(c, op, dev(b), tol=1e-8, restart=40, maxit=4000, precision=prec)
        xa, ia, sa = ddg.augmented_gmres_solve(c, op, dev(b), dev(V), tol=1e-8, restart=40, maxit=4000,
                                               precision=prec)
        assert st == 0 and sa == 0
        for xx in (x, xa):
            assert np.linalg.norm(b - A @ host(xx)) / np.linalg.norm(b) <= 1e-8
        res[scheme] = (info["iters"], ia["iters"])
    for k in range(2):
        a_, b_ = res["cgs2"][k], res["dcgs2"][k]
        assert abs(a_ - b_) <= max(2, 0.03 * a_), res


def test_dcgs2_is_default_and_matches_oracle_steps(ctx):
    g, eps, A, b = small(32, npml=6, seed=1)
    xo, io = gmres.plain_gmres(A, b, tol=1e-9, restart=25, maxit=3000)
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    c = ddg.Context(orthogonalization="cgs2")
    x1, i1, _ = ddg.gmres_solve(c, op, dev(b), tol=1e-9, restart=25, maxit=3000)
    x2, i2, _ = ddg.gmres_solve(ctx, op, dev(b), tol=1e-9, restart=25, maxit=3000)
    assert abs(i1["iters"] - io.iters) <= 1 and abs(i2["iters"] - io.iters) <= 1
    assert rel(host(x2), xo) <= 1e-6


def test_poor_subspace_falls_back_to_plain_after_its_step():
    # V-only residual above the threshold: the solve keeps the least-squares
    # step over V (Eq. 3 with K empty) and continues as plain GMRES (Eq. 2).
    g, eps, A, b = small(32, npml=6, seed=12)
    V = rand_V(g.D, 3, 12)
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    c = ddg.Context()
    c.set_fallback(0.5)
    x, info, st = ddg.augmented_gmres_solve(c, op, dev(b), dev(V), tol=1e-9, restart=25, maxit=3000)
    assert st == 0 and info["converged"] and info["fallback_used"] == 1
    assert info["first_step_rel_residual"] > 0.5
    # oracle: the same V step, then plain GMRES from it
    AV = np.column_stack([A @ V[n] for n in range(V.shape[0])])
    z, *_ = np.linalg.lstsq(AV, b, rcond=None)
    x1 = V.T @ z
    xo, io = gmres.plain_gmres(A, b, x0=x1, tol=1e-9, restart=25, maxit=3000)
    assert abs(info["iters"] - io.iters) <= 1
    assert rel(host(x), xo) <= 1e-6
    # a threshold >= 1 keeps the augmented method
    c.set_fallback(2.0)
    x2, i2, s2 = ddg.augmented_gmres_solve(c, op, dev(b), dev(V), tol=1e-9, restart=25, maxit=3000)
    assert s2 == 0 and i2["fallback_used"] == 0


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_first_cycle_augmented_then_plain(prec):
    # default restart reading: the paper's method in the first cycle, plain GMRES after
    g, eps, A, b = small(32, npml=6, seed=14)
    A2 = fdfd.operator_for(g, eps * 1.01)
    V = np.stack([spla.spsolve(A2.tocsc(), b), inputs.random_complex(g.D, 14)])
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    c = ddg.Context()
    x, info, st = ddg.augmented_gmres_solve(c, op, dev(b), dev(V), tol=1e-9, restart=25, maxit=3000,
                                            precision=prec)
    assert st == 0 and info["converged"] and not info["fallback_used"]
    xo, io = gmres.augmented_gmres(A, b, V.T, tol=1e-9, restart=25, maxit=3000, aug_cycles=1)
    assert np.linalg.norm(b - A @ host(x)) / np.linalg.norm(b) <= 1e-9
    if prec == "c128":
        assert abs(info["iters"] - io.iters) <= 1
        assert rel(host(x), xo) <= 1e-6


@pytest.mark.parametrize("prec", ["c64", "c128"])
def test_graph_step_loop_matches_host_loop(prec):
    # The graph-driven solve (every restart cycle inside one graph launch,
    # device-side WHILE and IF nodes over the same kernels) and the
    # host-driven loop launch the same kernels in the same order: equal fields
    # bit for bit, equal step and cycle counts, including cycles that end
    # mid-way (restart 30, several cycles; solves stopping at different steps)
    # and solves stopped by the iteration cap.
    g = inputs.grid_for(64, 64)
    eps = inputs.trajectory_set(g, 2, 3, steps=3)
    ops = [ddg.fdfd_operator(g, dev(e, torch.float64)) for e in eps]
    bs = [ddg.fdfd_source(op, g.i_src, g.sigma_src, g.j_src) for op in ops]
    U = dev(inputs.random_complex(g.D, 5, shape=(4, g.D)))
    out = {}
    for graphs in (True, False):
        c = ddg.Context()
        c.set_graphs(graphs)
        xs, infos, st = ddg.gmres_solve_batched(c, ops, bs, tol=1e-6, restart=30, maxit=4000, precision=prec)
        xa, infa, sta = ddg.augmented_gmres_solve_batched(c, ops, bs, [U] * len(ops), tol=1e-6, restart=30,
                                                          maxit=4000, precision=prec)
        # the iteration cap inside a cycle (the graph's loops end on their counters)
        xc, infc, stc = ddg.gmres_solve_batched(c, ops, bs, tol=1e-6, restart=30, maxit=45, precision=prec)
        assert st == 0 and sta == 0 and stc == 4
        out[graphs] = (np.stack([host(x) for x in xs + xa + xc]),
                       [(i["iters"], i["cycles"], i["converged"]) for i in infos + infa + infc])
    assert out[True][1] == out[False][1]
    assert np.array_equal(out[True][0], out[False][0])


@pytest.fixture(scope="module")
def ctx_f16():
    c = ddg.Context()
    c.set_basis_storage("f16")
    return c


def test_half_basis_full_size(ctx_f16, config1):
    # Krylov basis stored in IEEE half: the FP64 true residual still judges
    # convergence, so the solution meets the same bars as the FP32 basis
    g, eps, A, b, xd = config1
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    x, info, st = ddg.gmres_solve(ctx_f16, op, dev(b), tol=1e-6, restart=200, maxit=5000, precision="c64")
    assert st == 0 and info["converged"]
    xh = host(x)
    assert np.linalg.norm(b - A @ xh) / np.linalg.norm(b) <= 1e-6
    assert rel(xh, xd) <= 1e-5
    x32, info32, _ = ddg.gmres_solve(ddg.Context(), op, dev(b), tol=1e-6, restart=200, maxit=5000, precision="c64")
    print(f"half basis: {info['iters']} steps, FP32 basis: {info32['iters']} steps")
    assert info["iters"] <= 1.25 * info32["iters"] + 10


def test_half_basis_augmented_and_batched(ctx_f16):
    # uneven batch, augmented, both cycle policies' first cycle; FP32-only too
    g = inputs.grid_for(64, 64)
    eps = inputs.trajectory_set(g, 2, 3, steps=3)
    ops = [ddg.fdfd_operator(g, dev(e, torch.float64)) for e in eps]
    bs = [ddg.fdfd_source(op, g.i_src, g.sigma_src, g.j_src) for op in ops]
    As = [fdfd.operator_for(g, e) for e in eps]
    bo = fdfd.source_for(g)
    x_near = spla.spsolve(As[0].tocsc(), bo)
    U = dev(np.stack([x_near, inputs.random_complex(g.D, 9)]))
    direct = [spla.spsolve(A.tocsc(), bo) for A in As]
    for prec, tol in (("c64", 1e-6), ("c64_only", 1e-4)):
        xs, infos, st = ddg.augmented_gmres_solve_batched(ctx_f16, ops, bs, [U] * len(ops), tol=tol, restart=50,
                                                          maxit=6000, precision=prec)
        assert st == 0
        for A, x, i, xd in zip(As, xs, infos, direct):
            assert i["converged"]
            assert np.linalg.norm(bo - A @ host(x)) / np.linalg.norm(bo) <= tol * 1.02
            # the field against the direct solution: the 1e-5 bar at 1e-6 (and 1e-3 at 1e-4)
            assert rel(host(x), xd) <= 10 * tol


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_jacobi_preconditioner_matches_oracle(prec):
    # the data-free baseline: right Jacobi preconditioner, against the oracle's
    # preconditioned GMRES (same steps and cycles in c128; the solution meets
    # the tolerance of A f = b in both precisions; augmentation still works)
    g, eps, A, b = small(32, npml=6, seed=1)
    tol = 1e-9 if prec == "c128" else 1e-6
    xo, io = gmres.plain_gmres(A, b, tol=tol, restart=25, maxit=20000, minv=1.0 / A.diagonal())
    c = ddg.Context()
    c.set_preconditioner("jacobi")
    op = ddg.fdfd_operator(g, dev(eps, torch.float64))
    x, info, st = ddg.gmres_solve(c, op, dev(b), tol=tol, restart=25, maxit=20000, precision=prec)
    assert st == 0 and info["converged"]
    assert np.linalg.norm(b - A @ host(x)) / np.linalg.norm(b) <= tol
    if prec == "c128":
        assert abs(info["iters"] - io.iters) <= 1 and info["cycles"] == io.cycles
        assert rel(host(x), xo) <= 1e-6
    V = np.stack([spla.spsolve(A.tocsc(), b) + 1e-3 * inputs.random_complex(g.D, 3), inputs.random_complex(g.D, 4)])
    xa, ia, sta = ddg.augmented_gmres_solve(c, op, dev(b), dev(V), tol=tol, restart=25, maxit=20000, precision=prec)
    assert sta == 0 and ia["converged"]
    assert np.linalg.norm(b - A @ host(xa)) / np.linalg.norm(b) <= tol


@pytest.mark.parametrize("augmented", [False, True])
def test_solve_queue_matches_one_batched_call(augmented):
    # groups of 2 solves on 2 lanes (3 groups, each lane its own context,
    # stream and host thread): every solve bitwise equal to the same solve in
    # one batched call, with the same step count
    specs = [(16, 3, 0), (37, 5, 1), (64, 8, 2), (24, 4, 3), (16, 3, 4), (30, 4, 5)]
    ops, bs = [], []
    for n, L, seed in specs:
        g = inputs.Grid(nx=n, ny=n + 3, npml=L, i_src=2 * L, sigma_src=n / 8, slab_cells=2)
        rng = np.random.default_rng(seed)
        eps = inputs.background_eps(g) + rng.random((g.ny, g.nx))
        ops.append(ddg.fdfd_operator(g, dev(eps, torch.float64)))
        bs.append(ddg.fdfd_source(ops[-1], g.i_src, g.sigma_src, g.j_src))
    U = [dev(inputs.random_complex(o.D, 10 + s, shape=(3, o.D))) for s, o in enumerate(ops)] if augmented else None
    lanes = [ddg.Context(), ddg.Context()]
    xq, iq, stq = ddg.gmres_solve_queue(lanes, ops, bs, U=U, width=2, tol=1e-8, restart=40, precision="c64")
    one = ddg.Context()
    if augmented:
        xb, ib, stb = ddg.augmented_gmres_solve_batched(one, ops, bs, U, tol=1e-8, restart=40, precision="c64")
    else:
        xb, ib, stb = ddg.gmres_solve_batched(one, ops, bs, tol=1e-8, restart=40, precision="c64")
    assert stq == 0 and stb == 0
    for s in range(len(specs)):
        assert iq[s]["iters"] == ib[s]["iters"] and iq[s]["converged"]
        assert np.array_equal(host(xq[s]), host(xb[s]))
    # a cap that no solve meets: every info filled, status DDG_ENOCONV
    xc, ic, stc = ddg.gmres_solve_queue(lanes, ops, bs, U=U, width=4, tol=1e-12, restart=10, maxit=5,
                                        precision="c64")
    assert stc == 4 and all(0 < i["iters"] <= 5 and not i["converged"] for i in ic)


def test_autotuner_times_the_library_and_picks_a_measured_candidate(tmp_path):
    from paper_1902_00090_gb300 import autotune
    specs = [(16, 3, 0), (24, 4, 1), (16, 3, 2), (24, 4, 3)]
    ops, bs = [], []
    for n, L, seed in specs:
        g = inputs.Grid(nx=n, ny=n, npml=L, i_src=2 * L, sigma_src=n / 8, slab_cells=2)
        eps = inputs.background_eps(g) + np.random.default_rng(seed).random((g.ny, g.nx))
        ops.append(ddg.fdfd_operator(g, dev(eps, torch.float64)))
        bs.append(ddg.fdfd_source(ops[-1], g.i_src, g.sigma_src, g.j_src))
    lanes = [ddg.Context(), ddg.Context()]
    cache = str(tmp_path / "tune.json")
    r = autotune.tune_queue(lanes, ops, bs, sample=4, widths=(1, 2, 4), tol=1e-8, restart=30,
                            precision="c64", basis="f32", cache_path=cache)
    assert not r["cached"] and r["solves_per_s"] > 0
    assert (r["width"], r["lanes"]) in [(w, l) for w, l, _ in r["timings"]]
    assert len(r["timings"]) == 5 and all(v > 0 for _, _, v in r["timings"])
    r2 = autotune.tune_queue(lanes, ops, bs, sample=4, widths=(1, 2, 4), tol=1e-8, restart=30,
                             precision="c64", basis="f32", cache_path=cache)
    assert r2["cached"] and (r2["width"], r2["lanes"]) == (r["width"], r["lanes"])


@pytest.mark.parametrize("prec", ["c128", "c64"])
def test_restart_policy_per_wavelength_matches_oracle(prec):
    # one batch, one device at two wavelengths, two restart policies: all four
    # vectors in the first cycle, then the leading two kept (1550 nm, the
    # default) or plain GMRES (1300 nm); each solve against the oracle with
    # the same policy (c128: steps +-1 and the solution; c64: the tolerance)
    ctx = ddg.Context()
    ctx.set_fallback(2.0)
    ctx.set_augmented_policy(1, keep=2)
    ctx.set_augmented_policy(1, keep=0, wavelength=1300e-9)
    ops, bs, Vs, refs = [], [], [], []
    for lam, keep in ((1300e-9, 0), (1550e-9, 2)):
        g0, eps, _, _ = small(24, npml=4, seed=21)
        g = dataclasses.replace(g0, wavelength=lam)
        A, b = fdfd.operator_for(g, eps), fdfd.source_for(g)
        V = rand_V(g.D, 4, 22)
        xo, io = gmres.augmented_gmres(A, b, V.T, tol=1e-9, restart=20, maxit=4000, aug_cycles=1, aug_keep=keep)
        assert io.converged
        ops.append(ddg.fdfd_operator(g, dev(eps, torch.float64)))
        bs.append(ddg.fdfd_source(ops[-1], g.i_src, g.sigma_src, g.j_src))
        Vs.append(dev(V))
        refs.append((A, b, xo, io))
    tol = 1e-9 if prec == "c128" else 1e-7
    xs, infos, st = ddg.augmented_gmres_solve_batched(ctx, ops, bs, Vs, tol=tol, restart=20, maxit=4000,
                                                      precision=prec)
    assert st == 0
    for x, info, (A, b, xo, io) in zip(xs, infos, refs):
        assert np.linalg.norm(b - A @ host(x)) / np.linalg.norm(b) <= tol
        if prec == "c128":
            assert abs(info["iters"] - io.iters) <= 1, (info, io.iters)
            assert rel(host(x), xo) <= 1e-6
    # the two policies differ on this problem: so the per-wavelength entry was used
    assert refs[0][3].iters != gmres.augmented_gmres(refs[0][0], refs[0][1], Vs[0].cpu().numpy().T, tol=1e-9,
                                                     restart=20, maxit=4000, aug_cycles=1, aug_keep=2)[1].iters
