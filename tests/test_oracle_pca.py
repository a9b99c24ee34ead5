"""Pins of the oracle PCA basis (Sec. III) against the method of snapshots."""
import numpy as np

from oracle import pca


def test_pca_matches_method_of_snapshots():
    rng = np.random.default_rng(0)
    D, M, k = 400, 60, 8
    # fields with a decaying spectrum so that the k-th gap is clear
    F = (rng.standard_normal((D, M)) + 1j * rng.standard_normal((D, M))) * (0.7 ** np.arange(M))
    U, s = pca.pca_basis(F, k)
    # independent route: eigenvectors of the Gram matrix F^H F, U = F W S^-1
    G = F.conj().T @ F
    lam, W = np.linalg.eigh(G)
    order = np.argsort(lam)[::-1][:k]
    U2 = F @ W[:, order] / np.sqrt(lam[order])
    P1, P2 = U @ U.conj().T, U2 @ U2.conj().T
    assert np.linalg.norm(P1 - P2, 2) <= 1e-9
    assert np.allclose(s[:k] ** 2, lam[order], rtol=1e-10)
    e = pca.captured_energy(U, F)
    assert abs(e - (s[:k] ** 2).sum() / (s ** 2).sum()) <= 1e-12
    assert np.linalg.norm(U.conj().T @ U - np.eye(k)) <= 1e-12


def test_pca_is_uncentred():
    # A constant offset field must show up as the leading component.
    rng = np.random.default_rng(1)
    D, M = 300, 40
    base = rng.standard_normal(D) + 1j * rng.standard_normal(D)
    F = base[:, None] * 10 + 0.1 * (rng.standard_normal((D, M)) + 0j)
    U, s = pca.pca_basis(F, 1)
    cos = abs(np.vdot(U[:, 0], base)) / np.linalg.norm(base)
    assert cos > 0.999
