"""Oracle training losses of the subspace predictor.  TEST INFRASTRUCTURE ONLY.

Eq. 5 (projection loss):  l_proj = min over f in range(V) of ||f - f_k||^2 / ||f_k||^2.
Eq. 6 (residual loss):    l_res  = min over f in range(V) of ||A f - b||^2 / ||b||^2.

Both are written as their definitions: a library least-squares solve over the
coefficients of V, then the relative squared residual.
"""
from __future__ import annotations

import numpy as np


def projection_loss(V: np.ndarray, f: np.ndarray) -> float:
    z, *_ = np.linalg.lstsq(V, f, rcond=None)
    return float(np.linalg.norm(V @ z - f) ** 2 / np.linalg.norm(f) ** 2)


def residual_loss(A, V: np.ndarray, b: np.ndarray) -> float:
    AV = np.column_stack([A @ V[:, n] for n in range(V.shape[1])])
    z, *_ = np.linalg.lstsq(AV, b, rcond=None)
    return float(np.linalg.norm(AV @ z - b) ** 2 / np.linalg.norm(b) ** 2)
