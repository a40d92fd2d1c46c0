"""The all-at-once system and the alpha-circulant preconditioner (oracle).

Block vectors have shape (ell, N): row t-1 holds x_t.
"""
from __future__ import annotations

from typing import Callable

import numpy as np

Apply = Callable[[np.ndarray], np.ndarray]   # N-vector -> N-vector (A times it)


def aao_apply(A: Apply, x: np.ndarray) -> np.ndarray:
    """y = script-A x (Eq. 1): y_t = A x_t - x_{t-1}, with x_0 = 0."""
    ell = x.shape[0]
    y = np.empty_like(x)
    for t in range(ell):
        y[t] = A(x[t])
        if t > 0:
            y[t] -= x[t - 1]
    return y


def aao_dense(A: np.ndarray, ell: int) -> np.ndarray:
    """Dense script-A: A on the diagonal blocks, -I on the sub-diagonal (Eq. 1)."""
    N = A.shape[0]
    M = np.zeros((ell * N, ell * N))
    for t in range(ell):
        M[t * N:(t + 1) * N, t * N:(t + 1) * N] = A
        if t > 0:
            M[t * N:(t + 1) * N, (t - 1) * N:t * N] = -np.eye(N)
    return M


def c_alpha(ell: int, alpha: float) -> np.ndarray:
    """C_alpha: ones on the sub-diagonal, alpha in the top-right corner (Eq. 2)."""
    C = np.zeros((ell, ell))
    for t in range(1, ell):
        C[t, t - 1] = 1.0
    C[0, ell - 1] = alpha
    return C


def p_alpha_dense(A: np.ndarray, ell: int, alpha: float) -> np.ndarray:
    """P_alpha = I_ell (x) A + C_alpha (x) (-I_N)  (Eq. 2)."""
    N = A.shape[0]
    return np.kron(np.eye(ell), A) - np.kron(c_alpha(ell, alpha), np.eye(N))


def p_alpha_apply(A: Apply, x: np.ndarray, alpha: float) -> np.ndarray:
    """y = P_alpha x: as script-A x, plus -alpha x_ell in the first block (Eq. 2)."""
    y = aao_apply(A, x)
    y[0] = y[0] - alpha * x[-1]
    return y
