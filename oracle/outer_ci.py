"""Chebyshev semi-iteration as the outer solver (oracle; Sections 2 and 5).

The paper solves the preconditioned system P^{-1} script-A x = P^{-1} b (Eq. 3)
by Chebyshev semi-iteration over the interval of Corollary 1,
[1, mu_N^ell / (mu_N^ell - alpha)], keeping that interval even when P is
applied inexactly (Section 5), from x_0 = 0, stopping when
||b - script-A x|| / ||b|| < tol.

Recurrence (the textbook one, as for the inner solves), with M = P^{-1}:
    theta = (l_max + l_min)/2, delta = (l_max - l_min)/2, sigma1 = theta/delta
    r_0 = b - A x_0, z_0 = M r_0, d_0 = z_0/theta, rho_0 = 1/sigma1
    x_{k+1} = x_k + d_k;  r_{k+1} = r_k - A d_k;  z_{k+1} = M r_{k+1}
    rho_{k+1} = 1/(2 sigma1 - rho_k)
    d_{k+1} = rho_{k+1} rho_k d_k + (2 rho_{k+1}/delta) z_{k+1}
Each iteration costs one script-A product and one preconditioner apply
(Table 1).
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

Op = Callable[[np.ndarray], np.ndarray]


@dataclass
class CiResult:
    x: np.ndarray
    its: int
    converged: bool
    resid: float
    history: List[float] = field(default_factory=list)


def corollary1_interval(mu_min: float, ell: int, alpha: float):
    """[1, mu_N^ell/(mu_N^ell - alpha)]: extreme eigenvalues of P_alpha^{-1} script-A (Corollary 1)."""
    m = mu_min ** ell
    return 1.0, m / (m - alpha)


def outer_ci(Aop: Op, Mop: Op, b: np.ndarray, l_min: float, l_max: float, tol: float, max_its: int,
             x0: Optional[np.ndarray] = None, fixed_its: Optional[int] = None) -> CiResult:
    """Chebyshev semi-iteration on M A x = M b over [l_min, l_max]; residual in the unpreconditioned norm."""
    x = np.zeros_like(b) if x0 is None else x0.copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return CiResult(np.zeros_like(b), 0, True, 0.0, [])
    theta = 0.5 * (l_max + l_min)
    delta = 0.5 * (l_max - l_min)
    r = b - Aop(x)
    z = Mop(r)
    if delta == 0.0:                      # single-point interval: Richardson with step 1/theta
        sigma1, rho = np.inf, 0.0
    else:
        sigma1 = theta / delta
        rho = 1.0 / sigma1
    d = z / theta
    hist = []
    its = 0
    nmax = fixed_its if fixed_its is not None else max_its
    while its < nmax:
        x = x + d
        r = r - Aop(d)
        its += 1
        rel = np.linalg.norm(r) / bnorm
        hist.append(rel)
        if fixed_its is None and rel < tol:
            return CiResult(x, its, True, rel, hist)
        z = Mop(r)
        if delta == 0.0:
            d = z / theta
        else:
            rho_next = 1.0 / (2.0 * sigma1 - rho)
            d = rho_next * rho * d + (2.0 * rho_next / delta) * z
            rho = rho_next
    rel = np.linalg.norm(b - Aop(x)) / bnorm
    return CiResult(x, its, rel < tol, rel, hist)
