"""Oracle FDFD operator and source (Sec. II, Eq. 1).  TEST INFRASTRUCTURE ONLY.

Eq. 1 with the time convention exp(+i omega t) (implied by the source term
-i omega mu0 J) is, for the 2D TM polarisation (Ez only, one unknown per cell,
as in the paper's 229x90 = 20,610-unknown example of Fig. 1):

    -(d/dx d/dx + d/dy d/dy) Ez - (omega/c)^2 eps Ez = -i omega mu0 Jz.

Discretisation (the paper: Yee grid, PML, periodic boundaries):
  * Ez sits at integer nodes p = i, the H components at half nodes p = i + 1/2;
    both directions are periodic (indices mod nx, ny).
  * Stretched-coordinate PML: d/dx -> (1/s_x) d/dx with s(p) = 1 - i sigma'(p),
    sigma'(p) = sigma_max' (delta(p)/L)^m, delta(p) = max(L - p, p - (n - L), 0)
    the depth into the PML in cells (L = npml), and the graded-PML rule
    sigma_max' = -(m + 1) ln R / (2 k0 h L).  The minus sign in s makes the
    outgoing waves exp(-i k x) of the exp(+i omega t) convention decay.
  * Everything is multiplied by h^2, so A has the dimensionless coefficient
    (k0 h)^2 eps and b = -i (k0 h) g, g the source profile; relative residuals
    and relative errors do not depend on these global factors.

The operator is assembled from its definition as a product of sparse matrices:
    A = -( Sxb^-1 Dxb Sxf^-1 Dxf + Syb^-1 Dyb Syf^-1 Dyf ) - (k0 h)^2 diag(eps)
with Df the forward difference x_{i+1} - x_i and Db the backward difference
x_i - x_{i-1} (both periodic), Sf = diag(s(i + 1/2)), Sb = diag(s(i)).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def k0h(dx: float, wavelength: float) -> float:
    """Free-space wavenumber times the cell size."""
    return 2.0 * np.pi / wavelength * dx


def pml_depth(p: np.ndarray, n: int, L: int) -> np.ndarray:
    """Depth into the PML (cells) at coordinate p on a periodic line of n cells."""
    return np.maximum(np.maximum(L - p, p - (n - L)), 0.0)


def stretch(n: int, L: int, kh: float, order: float, R: float):
    """Complex stretch factors (s at integer nodes, s at half nodes), complex128.

    s(p) = 1 - i sigma_max' (delta(p)/L)^order with
    sigma_max' = -(order + 1) ln(R) / (2 kh L).
    """
    sb = np.ones(n, dtype=np.complex128)
    sf = np.ones(n, dtype=np.complex128)
    if L <= 0:
        return sb, sf
    smax = -(order + 1.0) * np.log(R) / (2.0 * kh * L)
    p = np.arange(n, dtype=np.float64)
    sb = 1.0 - 1j * smax * (pml_depth(p, n, L) / L) ** order
    sf = 1.0 - 1j * smax * (pml_depth(p + 0.5, n, L) / L) ** order
    return sb, sf


def _fwd_diff(n: int) -> sp.csr_matrix:
    """(Df x)_i = x_{i+1} - x_i, periodic."""
    e = np.ones(n)
    return sp.diags([-e, e[:-1], e[:1]], [0, 1, -(n - 1)], shape=(n, n), format="csr") \
        if n > 1 else sp.csr_matrix((1, 1))


def _bwd_diff(n: int) -> sp.csr_matrix:
    """(Db x)_i = x_i - x_{i-1}, periodic."""
    e = np.ones(n)
    return sp.diags([e, -e[:-1], -e[:1]], [0, -1, n - 1], shape=(n, n), format="csr") \
        if n > 1 else sp.csr_matrix((1, 1))


def operator(eps: np.ndarray, dx: float, wavelength: float, npml_x: int, npml_y: int,
             order: float = 3.0, R: float = 1e-8) -> sp.csr_matrix:
    """Sparse complex128 A (D x D, D = nx ny, cell (i, j) at row j nx + i)."""
    ny, nx = eps.shape
    kh = k0h(dx, wavelength)
    sxb, sxf = stretch(nx, npml_x, kh, order, R)
    syb, syf = stretch(ny, npml_y, kh, order, R)
    Lx = sp.diags(1.0 / sxb) @ _bwd_diff(nx) @ sp.diags(1.0 / sxf) @ _fwd_diff(nx)
    Ly = sp.diags(1.0 / syb) @ _bwd_diff(ny) @ sp.diags(1.0 / syf) @ _fwd_diff(ny)
    lap = sp.kron(sp.identity(ny), Lx) + sp.kron(Ly, sp.identity(nx))
    A = -lap - kh * kh * sp.diags(eps.reshape(-1).astype(np.complex128))
    return sp.csr_matrix(A, dtype=np.complex128)


def operator_for(grid, eps: np.ndarray) -> sp.csr_matrix:
    """Operator for an inputs.Grid description (same PML on x and y)."""
    return operator(eps, grid.dx, grid.wavelength, grid.npml, grid.npml,
                    grid.pml_order, grid.pml_R)


def source(nx: int, ny: int, dx: float, wavelength: float, i_src: int,
           sigma: float, j_c: float) -> np.ndarray:
    """b = -i (k0 h) g with g a Gaussian line current along y on column i_src."""
    j = np.arange(ny, dtype=np.float64)
    prof = np.exp(-((j - j_c) ** 2) / (2.0 * sigma * sigma))
    g = np.zeros((ny, nx), dtype=np.complex128)
    g[:, i_src] = prof
    return (-1j * k0h(dx, wavelength) * g).reshape(-1)


def source_for(grid) -> np.ndarray:
    return source(grid.nx, grid.ny, grid.dx, grid.wavelength, grid.i_src,
                  grid.sigma_src, grid.j_src)
