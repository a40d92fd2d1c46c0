"""Chebyshev semi-iteration on B = A - lambda I (oracle; Section 3).

The paper gives CI through its error polynomial (proof of Proposition 1):
after p steps from x_0 = 0 the error is
    e_p = T_p((theta - B)/delta) / T_p(theta/delta) e_0,
with theta the centre and delta the half-width of the spectral segment S_j.
The recurrence below is the textbook one (Saad, Iterative Methods for Sparse
Linear Systems, Chebyshev acceleration), written for a complex centre:

    sigma1 = theta/delta,  rho_0 = 1/sigma1
    x_0 = 0,  r_0 = f,  d_0 = f/theta
    for k = 0 .. p-1:
        x_{k+1} = x_k + d_k
        r_{k+1} = r_k - B d_k
        rho_{k+1} = 1/(2 sigma1 - rho_k)
        d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1}/delta) r_{k+1}

No inner stopping test: a fixed p makes the preconditioner a fixed linear
operator (Section 5, NC1).

Degenerate segment (delta = 0, the spectrum of B is the single point theta,
e.g. a one-cell grid where A = I): the recurrence's limit as delta -> 0 is
the exact solve, x_k = f/theta for every k >= 1; that limit is returned.
"""
from __future__ import annotations

from typing import Callable, List, Optional

import numpy as np


def chebyshev_solve(B: Callable[[np.ndarray], np.ndarray], f: np.ndarray, theta: complex,
                    delta: float, p: int, history: Optional[List[np.ndarray]] = None) -> np.ndarray:
    """Return x_p for B x = f after p Chebyshev steps from x_0 = 0.

    ``history``, if given, receives x_1 .. x_p.
    """
    f = np.asarray(f, dtype=complex)
    x = np.zeros_like(f)
    if p <= 0:
        return x
    if delta == 0.0:
        x = f / theta
        if history is not None:
            history.extend(x.copy() for _ in range(p))
        return x
    sigma1 = theta / delta
    rho = 1.0 / sigma1
    r = f.copy()
    d = f / theta
    for k in range(p):
        x = x + d
        if history is not None:
            history.append(x.copy())
        if k == p - 1:
            break
        r = r - B(d)
        rho_next = 1.0 / (2.0 * sigma1 - rho)
        d = rho_next * rho * d + (2.0 * rho_next / delta) * r
        rho = rho_next
    return x
