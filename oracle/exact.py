"""The exact solution of the all-at-once system (oracle).

Eq. 1 is equivalent to ell sequential solves with the SPD block A
(Section 1): x_1 = A^{-1} b_1, x_t = A^{-1}(b_t + x_{t-1}).  This is the
definition the iterative solvers are checked against.
"""
from __future__ import annotations

from typing import Callable

import numpy as np
import scipy.linalg as sla

Op = Callable[[np.ndarray], np.ndarray]


def cg(A: Op, b: np.ndarray, tol: float = 1e-14, maxit: int = 100000) -> np.ndarray:
    """Plain conjugate gradients (Hestenes-Stiefel) for SPD A, x_0 = 0, to ||r||/||b|| < tol."""
    x = np.zeros_like(b)
    r = b.copy()
    p = r.copy()
    rr = float(np.vdot(r, r).real)
    bb = rr
    if bb == 0.0:
        return x
    for _ in range(maxit):
        Ap = A(p)
        a = rr / float(np.vdot(p, Ap).real)
        x += a * p
        r -= a * Ap
        rr_new = float(np.vdot(r, r).real)
        if rr_new <= tol * tol * bb:
            break
        p = r + (rr_new / rr) * p
        rr = rr_new
    return x


def sequential_solve_dense(A: np.ndarray, b: np.ndarray) -> np.ndarray:
    """x = script-A^{-1} b for b of shape (ell, N), by ell LU solves with A."""
    lu = sla.lu_factor(A)
    x = np.zeros_like(b)
    prev = np.zeros(b.shape[1])
    for t in range(b.shape[0]):
        prev = sla.lu_solve(lu, b[t] + prev)
        x[t] = prev
    return x


def sequential_solve_cg(A: Op, b: np.ndarray, tol: float = 1e-14) -> np.ndarray:
    """x = script-A^{-1} b by ell CG solves with A (large N)."""
    x = np.zeros_like(b)
    prev = np.zeros(b.shape[1])
    for t in range(b.shape[0]):
        prev = cg(A, b[t] + prev, tol=tol)
        x[t] = prev
    return x
