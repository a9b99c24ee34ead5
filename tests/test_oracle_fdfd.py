"""Pins of the oracle FDFD operator and source (Sec. II, Eq. 1) against closed forms."""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import fdfd


def test_plane_wave_is_eigenvector_of_periodic_operator():
    # No PML: A = -Laplacian_h - (k0 h)^2 eps on a periodic grid.  A discrete plane
    # wave exp(2 pi i (a i / nx + c j / ny)) has eigenvalue
    # 4 sin^2(pi a / nx) + 4 sin^2(pi c / ny) - (k0 h)^2 eps.
    nx, ny, dx, lam, eps0 = 24, 16, 40e-9, 1550e-9, 2.1
    eps = np.full((ny, nx), eps0)
    A = fdfd.operator(eps, dx, lam, 0, 0)
    kh = 2 * np.pi / lam * dx
    i = np.arange(nx)[None, :]
    j = np.arange(ny)[:, None]
    for a, c in [(0, 0), (1, 0), (0, 3), (5, 7), (11, 2), (12, 8)]:
        p = np.exp(2j * np.pi * (a * i / nx + c * j / ny)).reshape(-1)
        lam_ex = 4 * np.sin(np.pi * a / nx) ** 2 + 4 * np.sin(np.pi * c / ny) ** 2 - kh ** 2 * eps0
        err = np.linalg.norm(A @ p - lam_ex * p) / np.linalg.norm(p)
        assert err <= 1e-13 * max(1.0, abs(lam_ex))


def test_pml_operator_symmetrised_by_integer_node_stretch():
    # With the stretch s(i) at integer nodes and s(i+1/2) at half nodes,
    # diag(sxb_i syb_j) A is complex symmetric (the half-node factors sit between
    # a difference and its transpose).  A wrong stagger or a transposed index breaks it.
    rng = np.random.default_rng(3)
    nx, ny, L = 20, 14, 4
    eps = 2.1 + 10.15 * rng.random((ny, nx))
    dx, lam = 40e-9, 1550e-9
    A = fdfd.operator(eps, dx, lam, L, L)
    kh = 2 * np.pi / lam * dx
    sxb, _ = fdfd.stretch(nx, L, kh, 3.0, 1e-8)
    syb, _ = fdfd.stretch(ny, L, kh, 3.0, 1e-8)
    S = sp.diags(np.kron(syb, np.ones(nx)) * np.kron(np.ones(ny), sxb))
    M = (S @ A).toarray()
    assert np.abs(M - M.T).max() <= 1e-13 * np.abs(M).max()
    assert np.abs(M - M.conj().T).max() > 1e-3   # complex symmetric, not Hermitian


def test_stretch_profile_closed_form():
    # s = 1 in the interior; at the outer edge s = 1 - i sigma_max' with the
    # graded-PML rule sigma_max' = -(m+1) ln R / (2 k0 h L); depth (cells) is
    # measured from the inner PML edge towards the periodic wrap point.
    n, L, kh, m, R = 40, 8, 0.2, 3.0, 1e-8
    sb, sf = fdfd.stretch(n, L, kh, m, R)
    smax = 4.0 * np.log(1e8) / (2 * 0.2 * 8)
    assert np.allclose(sb[L:n - L + 1], 1.0)
    assert abs(sb[0] - (1 - 1j * smax)) < 1e-12
    assert abs(sf[n - 1] - (1 - 1j * smax * (7.5 / 8) ** 3)) < 1e-12   # p = n - 1/2
    assert abs(sb[1] - (1 - 1j * smax * (7 / 8) ** 3)) < 1e-12
    assert abs(sb[n - 1] - sb[1]) < 1e-12                               # mirror about the wrap


def _green_1d(npml, nx=480, eps0=2.1):
    # y-uniform problem: ny = 1, no PML in y, unit line source on column i_s.
    dx, lam = 40e-9, 1550e-9
    eps = np.full((1, nx), eps0)
    A = fdfd.operator(eps, dx, lam, npml, 0)
    i_s = nx // 2
    b = np.zeros(nx, dtype=complex)
    b[i_s] = 1.0
    x = spla.spsolve(A.tocsc(), b)
    kh = 2 * np.pi / lam * dx
    theta = np.arccos(1 - kh * kh * eps0 / 2)
    i = np.arange(nx)
    G = np.exp(-1j * theta * np.abs(i - i_s)) / (2j * np.sin(theta))
    return x, G, i_s


@pytest.mark.parametrize("npml", [10, 20, 40])
def test_one_dimensional_green_function(npml):
    # Discrete 1D Helmholtz Green's function for the outgoing (exp(-i k x)) wave.
    x, G, i_s = _green_1d(npml)
    inner = slice(npml + 20, len(x) - npml - 20)
    err = np.linalg.norm(x[inner] - G[inner]) / np.linalg.norm(G[inner])
    assert err < {10: 1.5e-4, 20: 1e-5, 40: 1e-6}[npml]


def test_green_error_falls_with_pml_thickness():
    errs = []
    for npml in (6, 12, 24):
        x, G, _ = _green_1d(npml)
        inner = slice(60, len(x) - 60)
        errs.append(np.linalg.norm(x[inner] - G[inner]) / np.linalg.norm(G[inner]))
    assert errs[0] > errs[1] > errs[2]


def test_field_decays_through_pml():
    npml = 20
    x, _, i_s = _green_1d(npml)
    a = np.abs(x)
    right = a[len(x) - npml - 1:]            # into the right PML up to the wrap point
    left = a[:npml + 1][::-1]                # into the left PML from its inner edge
    assert np.all(np.diff(right) < 0) and np.all(np.diff(left[: npml]) < 0)
    assert right[-1] < 1e-3 * a[i_s]


def test_source_profile():
    from paper_1902_00090_gb300 import inputs
    g = inputs.grid_128()
    b = fdfd.source_for(g).reshape(g.ny, g.nx)
    nz = np.nonzero(np.abs(b) > 0)
    assert set(nz[1]) == {g.i_src}
    col = b[:, g.i_src]
    assert np.argmax(np.abs(col)) == g.ny // 2
    assert np.allclose(np.abs(col[g.ny // 2 - 5]), np.abs(col[g.ny // 2 + 5]))
    assert np.allclose(col.real, 0.0)


def test_source_amplitude_and_gaussian_width():
    # b = -i (k0 h) J (Eq. 1 times h^2 up to mu0 c): at the profile's centre
    # |b| = k0 h = 2 pi dx / lambda, the phase is -i, and one sigma away the
    # Gaussian has fallen to exp(-1/2); checked at two wavelengths and sizes
    from paper_1902_00090_gb300 import inputs
    for g in (inputs.grid_128(), inputs.grid_for(256, 256, wavelength=1300e-9)):
        b = fdfd.source_for(g).reshape(g.ny, g.nx)
        jc = int(g.j_src)
        kh = 2.0 * np.pi * g.dx / g.wavelength
        assert abs(b[jc, g.i_src] - (-1j * kh)) <= 1e-15 * kh
        s = int(g.sigma_src)
        assert abs(abs(b[jc + s, g.i_src]) / kh - np.exp(-0.5)) <= 1e-14
