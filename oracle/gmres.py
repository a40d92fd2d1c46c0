"""Right-preconditioned flexible GMRES (oracle).

The paper's outer solver is Chebyshev semi-iteration on Eq. 3; this library
solves the same preconditioned system with right-preconditioned FGMRES (the
preconditioned vectors Z_j are kept), modified Gram-Schmidt Arnoldi and Givens
rotations.  The convergence measure is the paper's relative residual
||b - script-A x|| / ||b|| with x_0 = 0 (Section 5).

Restarted form: a cycle of at most ``restart`` Arnoldi steps; after each
cycle (or when the Givens estimate drops below tol) the explicit residual is
formed; the solve stops when that explicit residual is below tol.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import Callable, List, Optional

import numpy as np

Op = Callable[[np.ndarray], np.ndarray]


@dataclass
class GmresResult:
    x: np.ndarray
    outer_its: int
    converged: bool
    resid_explicit: float
    history: List[float] = field(default_factory=list)   # Givens estimates, relative


def fgmres(Aop: Op, Mop: Op, b: np.ndarray, tol: float, max_outer: int,
           restart: Optional[int] = None, x0: Optional[np.ndarray] = None,
           fixed_its: Optional[int] = None,
           callback: Optional[Callable[[int], None]] = None) -> GmresResult:
    """Solve Aop(x) = b with right preconditioner Mop (x = Mop-preconditioned Krylov).

    ``fixed_its``: run exactly that many Arnoldi steps in one cycle (no early
    stop, no restart) and return the iterate; used for step-by-step parity.
    ``callback``: called with the running Arnoldi step count after every step
    (a timing hook; it sees no vectors and changes nothing).
    """
    shape = b.shape
    bnorm = np.linalg.norm(b)
    x = np.zeros(shape) if x0 is None else x0.astype(float).copy()
    if bnorm == 0.0:
        return GmresResult(x, 0, True, 0.0, [])
    m = restart if restart is not None else max_outer
    if fixed_its is not None:
        m = fixed_its
        max_outer = fixed_its
    total = 0
    history: List[float] = []
    while True:
        r = b - Aop(x)
        beta = np.linalg.norm(r)
        if fixed_its is None and beta / bnorm < tol:
            return GmresResult(x, total, True, beta / bnorm, history)
        if total >= max_outer:
            return GmresResult(x, total, False, beta / bnorm, history)
        V = [r / beta]
        Z = []
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        k = 0
        while k < m and total < max_outer:
            z = Mop(V[k])
            Z.append(z)
            w = Aop(z)
            for i in range(k + 1):                      # modified Gram-Schmidt
                H[i, k] = np.vdot(V[i], w).real
                w = w - H[i, k] * V[i]
            hnext = np.linalg.norm(w)
            H[k + 1, k] = hnext
            for i in range(k):                          # apply earlier rotations
                a, c = H[i, k], H[i + 1, k]
                H[i, k] = cs[i] * a + sn[i] * c
                H[i + 1, k] = -sn[i] * a + cs[i] * c
            a, c = H[k, k], H[k + 1, k]
            rr = np.hypot(a, c)
            cs[k], sn[k] = (1.0, 0.0) if rr == 0.0 else (a / rr, c / rr)
            H[k, k] = rr
            H[k + 1, k] = 0.0
            g[k + 1] = -sn[k] * g[k]
            g[k] = cs[k] * g[k]
            k += 1
            total += 1
            history.append(abs(g[k]) / bnorm)
            if callback is not None:
                callback(total)
            # happy breakdown: the Krylov space is invariant, the iterate is exact
            breakdown = hnext <= 1e-14 * beta
            if k < m and not breakdown:
                V.append(w / hnext)
            if breakdown or (fixed_its is None and abs(g[k]) / bnorm < tol):
                break
        y = np.linalg.solve(np.triu(H[:k, :k]), g[:k]) if k > 0 else np.zeros(0)
        for i in range(k):
            x = x + y[i] * Z[i]
        if fixed_its is not None:
            res = np.linalg.norm(b - Aop(x)) / bnorm
            return GmresResult(x, total, res < tol, res, history)
