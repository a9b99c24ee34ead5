"""Oracle GMRES and data-driven GMRES, complex128.  TEST INFRASTRUCTURE ONLY.

plain_gmres     -- Eq. 2: f_i = argmin over K_i(A, b) of ||A f - b||, built with
                   the Arnoldi iteration (Eq. S2 with N = 0), restarted every m
                   steps from the current iterate (the paper does not restart;
                   restarting is the reading used for GMRES(m)).
augmented_gmres -- Eqs. 3-4 and the supplement: f_i = argmin over
                   range(V) + K_i(A~, b~) with A~ = P_perp A, b~ = P_perp b,
                   P_perp = I - C C^H from the thin QR A V = C R (Eq. S1 item 5),
                   Arnoldi on A~ (Eq. S2), the Hessenberg matrix of Eq. S4, the
                   block least-squares problem of Eq. S7 and f = V R^-1 x + Q y.

The small least-squares problems ("QR factorization", end of the supplement's
derivation) are solved with complex Givens rotations (Golub & Van Loan,
Matrix Computations, Sec. 5.1.8: c real, s complex), one rotation per Arnoldi
step.  `lstsq_givens` exposes that step on its own so that it can be checked
against a library least-squares solve.

Gram-Schmidt: Eq. S2 is classical Gram-Schmidt (all coefficients q_j^H A~ q_i
taken from the same vector).  With reorth=True the same projection is applied
a second time and the two coefficient vectors are summed ("twice is enough",
CGS2); this keeps Q orthonormal to working precision over long cycles.

Restarts of the augmented method (the paper is silent): V, C and R^-1 are kept;
every cycle solves the residual equation A d = r, r = b - A f, with the same
augmentation, i.e. c_r = C^H r, r~ = r - C c_r, q_1 = r~/||r~||, and
d = V R^-1 (c_r - B y) + Q y.  On the first cycle from f = 0 this is exactly the
paper's method.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np


@dataclass
class GmresInfo:
    converged: bool = False
    iters: int = 0                    # Arnoldi steps (matvecs with A in the Krylov loop)
    cycles: int = 0
    true_rel_residual: float = np.inf
    first_step_rel_residual: float = np.nan   # ||b~|| / ||b|| (augmented only)
    breakdown: bool = False
    est_history: list = field(default_factory=list)   # |g_{j+1}| / ||b|| per step
    true_history: list = field(default_factory=list)  # true ||r|| / ||b|| per cycle start
    cycle_estimates: list = field(default_factory=list)  # per cycle: list of |g_{j+1}|


def givens(a: complex, b: complex):
    """Complex Givens rotation (c real, s complex) with
    [[c, s], [-conj(s), c]] @ [a, b] = [r, 0]."""
    if b == 0:
        return 1.0, 0.0 + 0.0j, a
    if a == 0:
        return 0.0, np.conj(b) / abs(b), abs(b)
    t = np.hypot(abs(a), abs(b))
    ph = a / abs(a)
    c = abs(a) / t
    s = ph * np.conj(b) / t
    return c, s, ph * t


def apply_rotation(c: float, s: complex, u: complex, v: complex):
    return c * u + s * v, -np.conj(s) * u + c * v


def lstsq_givens(H: np.ndarray, beta: float):
    """min_y || H y - beta e1 || for an upper-Hessenberg (k+1) x k matrix H,
    by Givens rotations; returns (y, residual norm)."""
    k = H.shape[1]
    g = np.zeros(k + 1, dtype=np.complex128)
    g[0] = beta
    R = H.astype(np.complex128).copy()
    cs = np.zeros(k)
    sn = np.zeros(k, dtype=np.complex128)
    for j in range(k):
        for i in range(j):
            R[i, j], R[i + 1, j] = apply_rotation(cs[i], sn[i], R[i, j], R[i + 1, j])
        cs[j], sn[j], R[j, j] = givens(R[j, j], R[j + 1, j])
        R[j + 1, j] = 0.0
        g[j], g[j + 1] = apply_rotation(cs[j], sn[j], g[j], g[j + 1])
    y = back_substitute(R[:k, :k], g[:k])
    return y, abs(g[k])


def back_substitute(R: np.ndarray, g: np.ndarray) -> np.ndarray:
    """Solve the upper-triangular system R y = g."""
    k = R.shape[0]
    y = np.zeros(k, dtype=np.complex128)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - R[i, i + 1:] @ y[i + 1:]) / R[i, i]
    return y


def _cgs(Q: np.ndarray, w: np.ndarray, reorth: bool):
    """Eq. S2 projection of w against the columns of Q (classical GS), optionally twice."""
    h = Q.conj().T @ w
    w = w - Q @ h
    if reorth:
        h2 = Q.conj().T @ w
        w = w - Q @ h2
        h = h + h2
    return h, w


def plain_gmres(A, b: np.ndarray, x0=None, tol: float = 1e-6, restart: int = 200,
                maxit: int = 5000, reorth: bool = True, breakdown_tol: float = 1e-14,
                keep_basis: bool = False, minv: np.ndarray = None):
    """Restarted GMRES(m) for A f = b (Eq. 2).  A: anything with A @ x.

    Stops when the true relative residual ||b - A f|| / ||b|| <= tol (checked at
    the start of every cycle) or after maxit Arnoldi steps.  Inside a cycle the
    Arnoldi loop stops as soon as the least-squares residual |g_{j+1}| is
    <= tol ||b||.  Returns (f, info); with keep_basis, also (Q, H) of the last cycle.

    minv: a diagonal right preconditioner M^-1 (the data-free baseline, e.g. the
    inverse diagonal of A, Jacobi): GMRES on A M^-1 y = r, f += M^-1 y.  The
    residuals are those of A f = b, so the stopping rule is unchanged.
    """
    b = np.asarray(b, dtype=np.complex128)
    D = b.shape[0]
    x = np.zeros(D, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    nb = np.linalg.norm(b)
    info = GmresInfo()
    m = restart
    last = None
    if nb == 0.0:
        info.converged, info.true_rel_residual = True, 0.0
        return (x, info, last) if keep_basis else (x, info)
    while True:
        r = b - A @ x
        beta = np.linalg.norm(r)
        info.true_rel_residual = beta / nb
        info.true_history.append(beta / nb)
        if beta <= tol * nb:
            info.converged = True
            break
        if info.iters >= maxit or info.breakdown:
            break
        info.cycles += 1
        Q = np.zeros((D, m + 1), dtype=np.complex128, order="F")
        H = np.zeros((m + 1, m), dtype=np.complex128)
        R = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        Q[:, 0] = r / beta
        k = 0
        est = []
        for j in range(m):
            w = A @ (Q[:, j] if minv is None else minv * Q[:, j])
            nw = np.linalg.norm(w)
            h, w = _cgs(Q[:, :j + 1], w, reorth)
            H[:j + 1, j] = h
            H[j + 1, j] = np.linalg.norm(w)
            # Givens QR of H, one new column per step
            R[:j + 2, j] = H[:j + 2, j]
            for i in range(j):
                R[i, j], R[i + 1, j] = apply_rotation(cs[i], sn[i], R[i, j], R[i + 1, j])
            cs[j], sn[j], R[j, j] = givens(R[j, j], R[j + 1, j])
            R[j + 1, j] = 0.0
            g[j], g[j + 1] = apply_rotation(cs[j], sn[j], g[j], g[j + 1])
            k = j + 1
            info.iters += 1
            est.append(abs(g[j + 1]))
            info.est_history.append(abs(g[j + 1]) / nb)
            if H[j + 1, j].real <= breakdown_tol * nw:
                info.breakdown = True
                break
            Q[:, j + 1] = w / H[j + 1, j]
            if abs(g[j + 1]) <= tol * nb or info.iters >= maxit:
                break
        y = back_substitute(R[:k, :k], g[:k])
        d = Q[:, :k] @ y
        x = x + (d if minv is None else minv * d)
        info.cycle_estimates.append(est)
        last = (Q[:, :k + 1], H[:k + 1, :k])
    return (x, info, last) if keep_basis else (x, info)


@dataclass
class Augmentation:
    """Eq. S1 item 5: A V = C R with C orthonormal (D x N) and R upper triangular."""
    V: np.ndarray
    C: np.ndarray
    R: np.ndarray
    Rinv: np.ndarray


def augmentation_setup(A, V: np.ndarray) -> Augmentation:
    """Thin QR of A V and the stored inverse of R (supplement, notation item 5)."""
    V = np.asarray(V, dtype=np.complex128)
    if V.shape[1] == 0:
        z = np.zeros((V.shape[0], 0), dtype=np.complex128)
        return Augmentation(V=V, C=z, R=np.zeros((0, 0)), Rinv=np.zeros((0, 0)))
    AV = np.column_stack([A @ V[:, n] for n in range(V.shape[1])])
    C, R = np.linalg.qr(AV, mode="reduced")
    return Augmentation(V=V, C=C, R=R, Rinv=np.linalg.inv(R))


def augmented_gmres(A, b: np.ndarray, V: np.ndarray, x0=None, tol: float = 1e-6,
                    restart: int = 200, maxit: int = 5000, reorth: bool = True,
                    breakdown_tol: float = 1e-14, keep_basis: bool = False,
                    aug_cycles: int | None = None, aug_keep: int = 0):
    """Data-driven GMRES (Eq. 3) with the update rule of the supplement.

    aug_cycles (restart reading): None keeps V in every cycle; an integer c runs
    the augmented method in the first max(c, 1) cycles and continues from the
    current iterate afterwards, as plain GMRES (Eq. 2) when aug_keep = 0, else
    as data-driven GMRES with the leading aug_keep columns of V (their own
    thin QR, Eq. S1).

    Returns (f, info); with keep_basis also a dict holding C, Q, H, B of the last
    cycle for invariant checks (C^H Q = 0, Eq. S3).
    """
    b = np.asarray(b, dtype=np.complex128)
    D = b.shape[0]
    aug = augmentation_setup(A, V)
    C, Rinv, V = aug.C, aug.Rinv, aug.V
    N = C.shape[1]
    x = np.zeros(D, dtype=np.complex128) if x0 is None else np.array(x0, dtype=np.complex128)
    nb = np.linalg.norm(b)
    info = GmresInfo()
    m = restart
    last = None
    if nb == 0.0:
        info.converged, info.true_rel_residual = True, 0.0
        return (x, info, last) if keep_basis else (x, info)
    while True:
        r = b - A @ x
        rn = np.linalg.norm(r)
        info.true_rel_residual = rn / nb
        info.true_history.append(rn / nb)
        if rn <= tol * nb:
            info.converged = True
            break
        if info.iters >= maxit or info.breakdown:
            break
        if aug_cycles is not None and info.cycles >= max(1, aug_cycles):
            # the augmented cycles are done: plain GMRES, or data-driven GMRES
            # with the leading aug_keep vectors, from the current iterate
            if aug_keep > 0:
                xp, ip = augmented_gmres(A, b, V[:, :aug_keep], x0=x, tol=tol, restart=restart,
                                         maxit=maxit - info.iters, reorth=reorth, breakdown_tol=breakdown_tol)
            else:
                xp, ip = plain_gmres(A, b, x0=x, tol=tol, restart=restart, maxit=maxit - info.iters,
                                     reorth=reorth, breakdown_tol=breakdown_tol)
            x = xp
            info.iters += ip.iters
            info.cycles += ip.cycles
            info.converged = ip.converged
            info.true_rel_residual = ip.true_rel_residual
            info.est_history += ip.est_history
            info.true_history += ip.true_history[1:]
            info.cycle_estimates += ip.cycle_estimates
            break
        info.cycles += 1
        # b~ = P_perp r (Eq. 4 applied to the residual equation)
        c_r = C.conj().T @ r
        bt = r - C @ c_r
        beta = np.linalg.norm(bt)
        if info.cycles == 1:
            info.first_step_rel_residual = beta / nb
        if beta <= breakdown_tol * rn:
            # the residual lies in span(A V): the V step alone solves it
            x = x + V @ (Rinv @ c_r)
            info.breakdown = True
            continue
        Q = np.zeros((D, m + 1), dtype=np.complex128, order="F")
        H = np.zeros((m + 1, m), dtype=np.complex128)
        B = np.zeros((N, m), dtype=np.complex128)
        R = np.zeros((m + 1, m), dtype=np.complex128)
        cs = np.zeros(m)
        sn = np.zeros(m, dtype=np.complex128)
        g = np.zeros(m + 1, dtype=np.complex128)
        g[0] = beta
        Q[:, 0] = bt / beta
        k = 0
        est = []
        for j in range(m):
            w = A @ Q[:, j]
            nw = np.linalg.norm(w)
            # A~ q_j = P_perp A q_j; B[:, j] = C^H A q_j (the C^H A Q block of Eq. S7)
            bj = C.conj().T @ w
            w = w - C @ bj
            h, w = _cgs(Q[:, :j + 1], w, reorth)
            if reorth:
                bj2 = C.conj().T @ w
                w = w - C @ bj2
                bj = bj + bj2
            B[:, j] = bj
            H[:j + 1, j] = h
            H[j + 1, j] = np.linalg.norm(w)
            R[:j + 2, j] = H[:j + 2, j]
            for i in range(j):
                R[i, j], R[i + 1, j] = apply_rotation(cs[i], sn[i], R[i, j], R[i + 1, j])
            cs[j], sn[j], R[j, j] = givens(R[j, j], R[j + 1, j])
            R[j + 1, j] = 0.0
            g[j], g[j + 1] = apply_rotation(cs[j], sn[j], g[j], g[j + 1])
            k = j + 1
            info.iters += 1
            est.append(abs(g[j + 1]))
            info.est_history.append(abs(g[j + 1]) / nb)
            if H[j + 1, j].real <= breakdown_tol * nw:
                info.breakdown = True
                break
            Q[:, j + 1] = w / H[j + 1, j]
            if abs(g[j + 1]) <= tol * nb or info.iters >= maxit:
                break
        y = back_substitute(R[:k, :k], g[:k])
        xa = c_r - B[:, :k] @ y
        x = x + V @ (Rinv @ xa) + Q[:, :k] @ y
        info.cycle_estimates.append(est)
        last = dict(C=C, Q=Q[:, :k + 1], H=H[:k + 1, :k], B=B[:, :k], c_r=c_r,
                    beta=beta, y=y, xa=xa, Rinv=Rinv)
    return (x, info, last) if keep_basis else (x, info)


def v_only_residual(A, b: np.ndarray, V: np.ndarray) -> float:
    """min over f in range(V) of ||A f - b|| / ||b|| (the square root of Eq. 6's loss)."""
    AV = np.column_stack([A @ V[:, n] for n in range(V.shape[1])])
    z, *_ = np.linalg.lstsq(AV, b, rcond=None)
    return np.linalg.norm(AV @ z - b) / np.linalg.norm(b)
