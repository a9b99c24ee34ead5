"""Oracle principal components of training fields.  TEST INFRASTRUCTURE ONLY.

Sec. III ("Principal component analysis"): the augmentation vectors are the
leading principal components of the simulated training fields, computed by an
incomplete singular value decomposition of the matrix whose columns are the
field vectors.  The paper mentions no mean subtraction and no per-field
normalisation, so the decomposition is of F = [f^(1) ... f^(M)] itself
(uncentred): v_1..v_N are its N leading left singular vectors.
"""
from __future__ import annotations

import numpy as np


def pca_basis(F: np.ndarray, k: int):
    """Top-k left singular vectors of F (D x M, complex) and all singular values."""
    U, s, _ = np.linalg.svd(np.asarray(F, dtype=np.complex128), full_matrices=False)
    return U[:, :k], s


def captured_energy(U: np.ndarray, F: np.ndarray) -> float:
    """||U^H F||_F^2 / ||F||_F^2 for orthonormal U."""
    return float(np.linalg.norm(U.conj().T @ F) ** 2 / np.linalg.norm(F) ** 2)
