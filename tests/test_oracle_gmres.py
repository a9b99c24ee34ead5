"""Pins of the oracle GMRES (Eq. 2) and data-driven GMRES (Eqs. 3-4, S1-S7)."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fdfd, gmres, losses
from paper_1902_00090_gb300 import inputs


def small_problem(n=16, npml=3, seed=0):
    g = inputs.Grid(nx=n, ny=n, npml=npml, i_src=n // 4, sigma_src=n / 8, slab_cells=max(2, n // 16))
    rng = np.random.default_rng(seed)
    eps = inputs.background_eps(g)
    eps += 0.5 * rng.random(eps.shape)
    A = fdfd.operator_for(g, eps)
    b = fdfd.source_for(g)
    return g, A, b


def test_givens_rotation_zeroes_second_entry():
    rng = np.random.default_rng(1)
    for _ in range(20):
        a, b = rng.standard_normal(2) + 1j * rng.standard_normal(2)
        c, s, r = gmres.givens(a, b)
        u, v = gmres.apply_rotation(c, s, a, b)
        assert abs(v) < 1e-15 * abs(r) and abs(u - r) < 1e-14 * abs(r)
        assert abs(c * c + abs(s) ** 2 - 1) < 1e-14 and np.isreal(c)
    c, s, r = gmres.givens(0.0, 2.0 + 0j)
    assert abs(gmres.apply_rotation(c, s, 0.0, 2.0)[1]) == 0


def test_givens_least_squares_matches_library():
    rng = np.random.default_rng(2)
    k = 30
    H = np.triu(rng.standard_normal((k + 1, k)) + 1j * rng.standard_normal((k + 1, k)), -1)
    beta = 2.5
    y, res = gmres.lstsq_givens(H, beta)
    e1 = np.zeros(k + 1, complex)
    e1[0] = beta
    y_ref, *_ = np.linalg.lstsq(H, e1, rcond=None)
    assert np.linalg.norm(y - y_ref) <= 1e-12 * np.linalg.norm(y_ref)
    assert abs(res - np.linalg.norm(H @ y_ref - e1)) <= 1e-12 * beta


def test_dense_direct_solve_16x16():
    g, A, b = small_problem(16)
    x_ref = np.linalg.solve(A.toarray(), b)
    x, info = gmres.plain_gmres(A, b, tol=1e-13, restart=60, maxit=2000)
    assert info.converged
    assert np.linalg.norm(x - x_ref) <= 1e-10 * np.linalg.norm(x_ref)


def test_residual_monotone_within_and_across_cycles():
    g, A, b = small_problem(32, npml=6, seed=1)
    x, info = gmres.plain_gmres(A, b, tol=1e-9, restart=25, maxit=3000)
    assert info.converged and info.cycles >= 3
    for est in info.cycle_estimates:
        assert np.all(np.diff(est) <= 1e-12 * est[0])
    th = np.array(info.true_history)
    assert np.all(np.diff(th) <= 1e-12)


def test_matches_scipy_gmres_solution():
    g, A, b = small_problem(32, npml=6, seed=2)
    x, info = gmres.plain_gmres(A, b, tol=1e-10, restart=40, maxit=4000)
    xs, code = spla.gmres(A, b, rtol=1e-10, restart=40, maxiter=200)
    assert code == 0
    xd = spla.spsolve(A.tocsc(), b)
    assert np.linalg.norm(x - xd) <= 1e-7 * np.linalg.norm(xd)
    assert np.linalg.norm(x - xs) <= 1e-7 * np.linalg.norm(xd)


def test_single_cycle_is_krylov_minimiser():
    # Eq. 2 directly: after k steps f_k = K (K^+ ...) with K the Krylov matrix;
    # compare with the least-squares minimiser over an explicitly built Krylov basis.
    g, A, b = small_problem(16, seed=4)
    k = 12
    x, info = gmres.plain_gmres(A, b, tol=1e-300, restart=k, maxit=k)
    K = np.empty((b.size, k), complex)
    v = b / np.linalg.norm(b)
    for i in range(k):
        K[:, i] = v
        v = A @ v
        v /= np.linalg.norm(v)
    AK = A @ K
    z, *_ = np.linalg.lstsq(AK, b, rcond=None)
    ref = K @ z
    assert np.linalg.norm(x - ref) <= 1e-8 * np.linalg.norm(ref)


def test_augmented_with_no_vectors_is_plain_gmres():
    g, A, b = small_problem(24, npml=4, seed=5)
    x1, i1 = gmres.plain_gmres(A, b, tol=1e-8, restart=30)
    x2, i2 = gmres.augmented_gmres(A, b, np.zeros((b.size, 0), complex), tol=1e-8, restart=30)
    assert i1.iters == i2.iters
    assert np.linalg.norm(x1 - x2) <= 1e-12 * np.linalg.norm(x1)


def test_solution_in_subspace_needs_no_krylov_step():
    g, A, b = small_problem(24, npml=4, seed=6)
    xd = spla.spsolve(A.tocsc(), b)
    rng = np.random.default_rng(0)
    V = np.column_stack([rng.standard_normal(b.size) + 1j * rng.standard_normal(b.size),
                         xd, rng.standard_normal(b.size) + 0j])
    x, info = gmres.augmented_gmres(A, b, V, tol=1e-10, restart=30)
    assert info.first_step_rel_residual <= 1e-12
    assert info.iters == 0 and info.converged
    assert np.linalg.norm(x - xd) <= 1e-10 * np.linalg.norm(xd)


def _aug_run(seed=7, N=5, k=20):
    g, A, b = small_problem(24, npml=4, seed=seed)
    rng = np.random.default_rng(seed)
    V = rng.standard_normal((b.size, N)) + 1j * rng.standard_normal((b.size, N))
    x, info, last = gmres.augmented_gmres(A, b, V, tol=1e-300, restart=k, maxit=k,
                                          keep_basis=True)
    return A, b, V, x, info, last


def test_augmented_invariants():
    A, b, V, x, info, last = _aug_run()
    C, Q, H, B = last["C"], last["Q"], last["H"], last["B"]
    k = H.shape[1]
    assert np.linalg.norm(C.conj().T @ Q) <= 1e-12                 # C^H Q = 0
    assert np.linalg.norm(Q.conj().T @ Q - np.eye(k + 1)) <= 1e-12
    AQ = A @ Q[:, :k]
    S3 = AQ - Q @ H - C @ B                                          # Eq. S3
    assert np.linalg.norm(S3) <= 1e-12 * spla.norm(A) * np.sqrt(k)
    assert np.allclose(np.tril(H, -2), 0)


def test_block_least_squares_S7_decouples():
    A, b, V, x, info, last = _aug_run(seed=8)
    H, B, c_r, beta = last["H"], last["B"], last["c_r"], last["beta"]
    N, k = B.shape
    M = np.zeros((N + k + 1, N + k), complex)
    M[:N, :N] = np.eye(N)
    M[:N, N:] = B
    M[N:, N:] = H
    rhs = np.concatenate([c_r, beta * np.eye(k + 1)[0]])
    sol, *_ = np.linalg.lstsq(M, rhs, rcond=None)
    assert np.linalg.norm(sol[:N] - last["xa"]) <= 1e-10 * np.linalg.norm(sol)
    assert np.linalg.norm(sol[N:] - last["y"]) <= 1e-10 * np.linalg.norm(sol)


def test_first_step_residual_is_residual_loss():
    g, A, b = small_problem(24, npml=4, seed=9)
    rng = np.random.default_rng(9)
    V = rng.standard_normal((b.size, 4)) + 1j * rng.standard_normal((b.size, 4))
    x, info = gmres.augmented_gmres(A, b, V, tol=1e-8, restart=30)
    assert info.converged
    lres = losses.residual_loss(A, V, b)
    assert abs(info.first_step_rel_residual - np.sqrt(lres)) <= 1e-10


def test_least_squares_residual_equals_true_residual():
    A, b, V, x, info, last = _aug_run(seed=10)
    true = np.linalg.norm(b - A @ x)
    est = info.cycle_estimates[-1][-1]
    assert abs(true - est) <= 1e-9 * np.linalg.norm(b)


def test_losses_range_and_extremes():
    rng = np.random.default_rng(11)
    D = 200
    V = rng.standard_normal((D, 3)) + 1j * rng.standard_normal((D, 3))
    f_in = V @ np.array([1.0, -2j, 0.5])
    assert losses.projection_loss(V, f_in) <= 1e-24
    Qv, _ = np.linalg.qr(V)
    f_perp = rng.standard_normal(D) + 0j
    f_perp -= Qv @ (Qv.conj().T @ f_perp)
    assert abs(losses.projection_loss(V, f_perp) - 1.0) <= 1e-12
    f = rng.standard_normal(D) + 1j * rng.standard_normal(D)
    assert 0.0 <= losses.projection_loss(V, f) <= 1.0


def test_augmented_first_cycle_then_plain_reading():
    # aug_cycles = 1: the first cycle is the paper's method, the rest plain GMRES
    g, A, b = small_problem(24, npml=4, seed=13)
    rng = np.random.default_rng(13)
    V = rng.standard_normal((b.size, 3)) + 1j * rng.standard_normal((b.size, 3))
    x1, i1 = gmres.augmented_gmres(A, b, V, tol=1e-9, restart=20, maxit=20)
    xp, ip = gmres.plain_gmres(A, b, x0=x1, tol=1e-9, restart=20, maxit=4000)
    x, info = gmres.augmented_gmres(A, b, V, tol=1e-9, restart=20, maxit=4000, aug_cycles=1)
    assert info.converged and info.iters == i1.iters + ip.iters
    assert np.linalg.norm(x - xp) <= 1e-12 * np.linalg.norm(xp)


def test_augmented_keeps_leading_columns_after_the_first_cycle():
    # aug_cycles = 1, aug_keep = j: after the first cycle every cycle minimises
    # over V[:, :j] + its Krylov space, so its residual is orthogonal to
    # A V[:, :j] (the least-squares condition), and not to the dropped columns;
    # keeping every column is the solve that keeps V throughout
    g, A, b = small_problem(24, npml=4, seed=14)
    rng = np.random.default_rng(14)
    V = rng.standard_normal((b.size, 4)) + 1j * rng.standard_normal((b.size, 4))
    x, info = gmres.augmented_gmres(A, b, V, tol=1e-12, restart=20, maxit=40, aug_cycles=1, aug_keep=2)
    assert info.cycles == 2 and not info.converged
    r = b - A @ x
    C2, _ = np.linalg.qr(A @ V[:, :2])
    assert np.linalg.norm(C2.conj().T @ r) <= 1e-10 * np.linalg.norm(r)
    C4, _ = np.linalg.qr(A @ V)
    assert np.linalg.norm(C4[:, 2:].conj().T @ r) >= 1e-6 * np.linalg.norm(r)
    xa, ia = gmres.augmented_gmres(A, b, V, tol=1e-9, restart=20, maxit=4000, aug_cycles=1, aug_keep=4)
    xk, ik = gmres.augmented_gmres(A, b, V, tol=1e-9, restart=20, maxit=4000)
    assert ia.converged and ia.iters == ik.iters
    assert np.linalg.norm(xa - xk) <= 1e-8 * np.linalg.norm(xk)
    # aug_keep = 0 is the first-cycle-then-plain reading
    x0, i0 = gmres.augmented_gmres(A, b, V, tol=1e-9, restart=20, maxit=4000, aug_cycles=1, aug_keep=0)
    xp, ip = gmres.augmented_gmres(A, b, V, tol=1e-9, restart=20, maxit=4000, aug_cycles=1)
    assert np.array_equal(x0, xp) and i0.iters == ip.iters


def test_right_preconditioned_gmres():
    # The data-free baseline: GMRES on A M^-1 with M = diag(A) (Jacobi).
    # M = I reproduces the plain solve exactly; Jacobi reaches the direct
    # solution, and its single cycle minimises ||b - A M^-1 y|| over the
    # Krylov space of A M^-1 (checked against an explicit basis).
    g, A, b = small_problem(16, seed=4)
    x_ref = np.linalg.solve(A.toarray(), b)
    x0, i0 = gmres.plain_gmres(A, b, tol=1e-10, restart=40, maxit=4000)
    x1, i1 = gmres.plain_gmres(A, b, tol=1e-10, restart=40, maxit=4000, minv=np.ones(g.D))
    assert np.array_equal(x0, x1) and i0.iters == i1.iters
    minv = 1.0 / A.diagonal()
    xj, ij = gmres.plain_gmres(A, b, tol=1e-10, restart=40, maxit=4000, minv=minv)
    assert ij.converged and np.linalg.norm(xj - x_ref) / np.linalg.norm(x_ref) <= 1e-8
    # one cycle of j steps: the residual equals the minimum over the Krylov space of A M^-1
    j = 12
    xc, ic = gmres.plain_gmres(A, b, tol=1e-300, restart=j, maxit=j, minv=minv)
    B = A @ np.diag(minv)
    K = np.column_stack([np.linalg.matrix_power(B, p) @ b for p in range(j)])
    Qk, _ = np.linalg.qr(K)
    y, *_ = np.linalg.lstsq(B @ Qk, b, rcond=None)
    assert np.isclose(np.linalg.norm(b - A @ xc), np.linalg.norm(b - B @ Qk @ y), rtol=1e-6)
