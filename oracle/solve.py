"""Putting the oracle pieces together for one instance (test infrastructure).

``make_block_op`` turns face arrays into the N-vector map x -> A x on flat
vectors; ``solve`` runs right-preconditioned FGMRES on Eq. 1 with P_NC
(Eq. 5 + inner CI) as the preconditioner.
"""
from __future__ import annotations

from typing import Optional, Sequence, Union

import numpy as np

from .allatonce import aao_apply
from .gmres import GmresResult, fgmres
from .operator import MU_MIN_NEUMANN, fv_apply, gershgorin_mu_max
from .precond import pnc_apply


def make_block_op(kx, ky, kz, shape):
    """Return A as a map on flat length-N vectors (real or complex)."""
    def A(v):
        return fv_apply(v.reshape(shape), kx, ky, kz).reshape(-1)
    return A


def precond_op(kx, ky, kz, shape, alpha: float, p: Union[int, Sequence[int]],
               mu_max: Optional[float] = None, mu_min: float = MU_MIN_NEUMANN):
    A = make_block_op(kx, ky, kz, shape)
    mmax = gershgorin_mu_max(kx, ky, kz, shape) if mu_max is None else mu_max
    return lambda r: pnc_apply(A, r, alpha, mu_min, mmax, p)


def solve(kx, ky, kz, shape, ell: int, alpha: float, b: np.ndarray, p, tol: float,
          max_outer: int, restart: Optional[int] = None, mu_max: Optional[float] = None,
          fixed_its: Optional[int] = None, callback=None) -> GmresResult:
    """FGMRES on script-A x = b (Eq. 1) right-preconditioned by P_NC^{-1}."""
    A = make_block_op(kx, ky, kz, shape)
    M = precond_op(kx, ky, kz, shape, alpha, p, mu_max)
    return fgmres(lambda x: aao_apply(A, x), M, b, tol, max_outer, restart=restart,
                  fixed_its=fixed_its, callback=callback)
