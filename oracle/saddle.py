"""P_SP: the saddle-point reformulation of the shifted solves (Section 4), oracle.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).

Eq. 5 needs y_j = (A - lambda_j I)^{-1} v_j for every frequency.  Section 4 solves them in
real arithmetic with a fixed number K of Krylov iterations each:
  * real shifts (j = 0 and j = ell/2): preconditioned CG on A - lambda_j I;
  * complex shifts: the real system of twice the size (the saddle-point system of Section 4)
        S = [[Phi, Psi], [Psi, -Phi]],  Phi = Im(lambda) I,  Psi = A - Re(lambda) I,
        S [Re x; -Im x] = [-Im b; Re b],
    by MINRES with the block-diagonal preconditioner P_D = diag(Phi + Psi, Phi + Psi)
    (Section 4's theorem: the spectrum of P_D^{-1} S lies in [-1, -1/sqrt 2] u [1/sqrt 2, 1]).
    Phi must be positive definite, so a shift with Im(lambda) < 0 is solved through its
    conjugate: (A - lambda) x = b  <=>  (A - conj lambda) conj x = conj b.
The paper applies the SPD blocks approximately with one V-cycle of an algebraic multigrid
(HSL_MI20).  This library uses its own multigrid for the same operators, defined here and run
identically on the GPU:
  * levels: pairwise aggregation of the structured grid (2 x 2 cells in 2D, 2 x 2 x 2 in 3D,
    ceil(n/2) per axis), the coarse operator being the Galerkin product R B P with
    piecewise-constant P and R = P^T.  For B = (1 + c) I + K this keeps the form
    B_H = (1 + c) W_H + K_H: W_H sums the cells of an aggregate and each coarse face sums the fine
    face diffusivities crossing it;
  * smoother: weighted Jacobi, omega = 2/3, NU sweeps before and after the coarse correction
    (a symmetric V-cycle, so it is an SPD preconditioner for CG and MINRES);
  * coarsest level (every side <= 4 cells): NU_COARSE Jacobi sweeps from zero.
Grids are 1D, 2D (fields of shape (n1, n0)) or 3D (fields of shape (n2, n1, n0)).
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import List, Optional

import numpy as np

from .precond import forward_transform, inverse_transform
from .spectral import scaled_roots

OMEGA = 2.0 / 3.0
NU = 2
NU_COARSE = 16
COARSEST = 4


@dataclass
class Level:
    w: np.ndarray    # cell weights, the level's field shape (1 on the finest level)
    kx: np.ndarray   # face diffusivities along x (last axis): one fewer entry along it
    ky: np.ndarray   # along y (second-last axis)
    kz: Optional[np.ndarray] = None   # along z (first axis of a 3D field), None in 1D/2D


def _faces(L: Level):
    """(axis, face array) pairs of a level; x is the last axis."""
    nd = L.w.ndim
    out = [(nd - 1, L.kx), (nd - 2, L.ky)]
    if L.kz is not None:
        out.append((0, L.kz))
    return out


def _agg_index(shape):
    """Aggregate index of every cell of a field of this shape (2 per axis)."""
    return tuple(ix // 2 for ix in np.indices(shape))


def _coarse_faces(k: np.ndarray, axis: int, cshape) -> np.ndarray:
    """Coarse faces along `axis`: the fine faces between cells 2I+1 and 2I+2 along the axis
    cross from aggregate I to I+1; summed over the aggregate's cells along the other axes."""
    cn = cshape[axis]
    shp = list(cshape)
    shp[axis] = max(cn - 1, 0)
    kc = np.zeros(shp)
    if cn > 1:
        sel = np.take(k, np.arange(1, 2 * cn - 2, 2), axis=axis)
        idx = list(np.indices(sel.shape))
        for a in range(sel.ndim):
            if a != axis:
                idx[a] = idx[a] // 2
        np.add.at(kc, tuple(idx), sel)
    return kc


def hierarchy(kx: np.ndarray, ky: np.ndarray, shape, kz: Optional[np.ndarray] = None) -> List[Level]:
    """Aggregation levels; kx, ky, kz in the (n2, n1, n0-1) / (n2, n1-1, n0) / (n2-1, n1, n0)
    layout.  1D/2D grids (n2 = 1) give fields of shape (n1, n0), 3D grids (n2, n1, n0)."""
    n2, n1, n0 = shape
    if n2 == 1:
        lv = [Level(np.ones((n1, n0)), kx[0].astype(float).copy(), ky[0].astype(float).copy())]
    else:
        if kz is None:
            raise ValueError("a 3D grid needs its z faces")
        lv = [Level(np.ones((n2, n1, n0)), kx.astype(float).copy(), ky.astype(float).copy(),
                    kz.astype(float).copy())]
    while max(lv[-1].w.shape) > COARSEST:
        f = lv[-1]
        cshape = tuple((m + 1) // 2 for m in f.w.shape)
        w = np.zeros(cshape)
        np.add.at(w, _agg_index(f.w.shape), f.w)                      # cells of each aggregate
        fc = {a: _coarse_faces(k, a, cshape) for a, k in _faces(f)}
        nd = len(cshape)
        lv.append(Level(w, fc[nd - 1], fc[nd - 2], fc.get(0) if f.kz is not None else None))
    return lv


def level_apply(L: Level, c: float, x: np.ndarray) -> np.ndarray:
    """B x = (1 + c) W x + K x on one level (x of the level's field shape)."""
    y = (1.0 + c) * L.w * x
    for a, k in _faces(L):
        if k.size:
            n = x.shape[a]
            f = k * (np.take(x, np.arange(1, n), axis=a) - np.take(x, np.arange(0, n - 1), axis=a))
            lo = [slice(None)] * x.ndim
            hi = [slice(None)] * x.ndim
            lo[a] = slice(0, n - 1)
            hi[a] = slice(1, n)
            y[tuple(lo)] -= f
            y[tuple(hi)] += f
    return y


def level_diag(L: Level, c: float) -> np.ndarray:
    d = (1.0 + c) * L.w.copy()
    for a, k in _faces(L):
        if k.size:
            n = d.shape[a]
            lo = [slice(None)] * d.ndim
            hi = [slice(None)] * d.ndim
            lo[a] = slice(0, n - 1)
            hi[a] = slice(1, n)
            d[tuple(lo)] += k
            d[tuple(hi)] += k
    return d


def jacobi(L: Level, c: float, b: np.ndarray, x: np.ndarray, sweeps: int) -> np.ndarray:
    d = level_diag(L, c)
    for _ in range(sweeps):
        x = x + OMEGA * (b - level_apply(L, c, x)) / d
    return x


def restrict(b: np.ndarray, coarse_shape) -> np.ndarray:
    """Sum of b over each aggregate (R = P^T)."""
    r = np.zeros(coarse_shape)
    np.add.at(r, _agg_index(b.shape), b)
    return r


def prolong(xc: np.ndarray, fine_shape) -> np.ndarray:
    """Every fine cell takes its aggregate's value (piecewise-constant P)."""
    return xc[_agg_index(fine_shape)]


def vcycle(levels: List[Level], c: float, b: np.ndarray, q: int = 0) -> np.ndarray:
    """One symmetric V-cycle for B = (1 + c) I + K from level q, zero initial guess."""
    L = levels[q]
    x = np.zeros_like(b)
    if q == len(levels) - 1:
        return jacobi(L, c, b, x, NU_COARSE)
    x = jacobi(L, c, b, x, NU)
    r = b - level_apply(L, c, x)
    xc = vcycle(levels, c, restrict(r, levels[q + 1].w.shape), q + 1)
    x = x + prolong(xc, L.w.shape)
    return jacobi(L, c, b, x, NU)


def pcg(levels: List[Level], c: float, b: np.ndarray, iters: int) -> np.ndarray:
    """iters steps of CG on B = (1 + c) I + K preconditioned by one V-cycle, x_0 = 0."""
    x = np.zeros_like(b)
    r = b.copy()
    z = vcycle(levels, c, r)
    p = z.copy()
    rz = float(np.vdot(r, z))
    for k in range(iters):
        if rz == 0.0:
            break
        q = level_apply(levels[0], c, p)
        a = rz / float(np.vdot(p, q))
        x = x + a * p
        r = r - a * q
        if k == iters - 1:
            break
        z = vcycle(levels, c, r)
        rz_new = float(np.vdot(r, z))
        p = z + (rz_new / rz) * p
        rz = rz_new
    return x


def saddle_apply(levels: List[Level], lam: complex, u: np.ndarray, v: np.ndarray):
    """S [u; v] with Phi = Im(lam) I, Psi = A - Re(lam) I."""
    phi = lam.imag
    pu = level_apply(levels[0], -lam.real, u)
    pv = level_apply(levels[0], -lam.real, v)
    return phi * u + pv, pu - phi * v


def minres(levels: List[Level], lam: complex, fu: np.ndarray, fv: np.ndarray, iters: int):
    """iters steps of preconditioned MINRES on S [u; v] = [fu; fv] from zero, preconditioner
    P_D = diag(B, B) applied by one V-cycle per block, B = Phi + Psi = (1 + c) I + K with
    c = Im(lam) - Re(lam).  Lanczos process in the P_D^{-1} inner product, QR of the
    tridiagonal by Givens rotations, and the short solution recurrence (Paige and Saunders)."""
    c_pd = lam.imag - lam.real

    def prec(a, b):
        return vcycle(levels, c_pd, a), vcycle(levels, c_pd, b)

    xu, xv = np.zeros_like(fu), np.zeros_like(fv)
    vu_old, vv_old = np.zeros_like(fu), np.zeros_like(fv)
    vu, vv = fu.copy(), fv.copy()
    zu, zv = prec(vu, vv)
    gamma = np.sqrt(float(np.vdot(zu, vu) + np.vdot(zv, vv)))
    gamma_old = 1.0
    eta = gamma
    s_old = s = 0.0
    c_old = c = 1.0
    wu_old, wv_old = np.zeros_like(fu), np.zeros_like(fv)
    wu, wv = np.zeros_like(fu), np.zeros_like(fv)
    for _ in range(iters):
        if gamma == 0.0:
            break
        zu, zv = zu / gamma, zv / gamma
        su, sv = saddle_apply(levels, lam, zu, zv)
        delta = float(np.vdot(su, zu) + np.vdot(sv, zv))
        nu_ = su - (delta / gamma) * vu - (gamma / gamma_old) * vu_old
        nv_ = sv - (delta / gamma) * vv - (gamma / gamma_old) * vv_old
        zu_n, zv_n = prec(nu_, nv_)
        gamma_n = np.sqrt(max(float(np.vdot(zu_n, nu_) + np.vdot(zv_n, nv_)), 0.0))
        a0 = c * delta - c_old * s * gamma
        a1 = np.hypot(a0, gamma_n)
        a2 = s * delta + c_old * c * gamma
        a3 = s_old * gamma
        c_n, s_n = a0 / a1, gamma_n / a1
        wu_n = (zu - a3 * wu_old - a2 * wu) / a1
        wv_n = (zv - a3 * wv_old - a2 * wv) / a1
        xu = xu + c_n * eta * wu_n
        xv = xv + c_n * eta * wv_n
        eta = -s_n * eta
        vu_old, vv_old, vu, vv = vu, vv, nu_, nv_
        zu, zv = zu_n, zv_n
        gamma_old, gamma = gamma, gamma_n
        wu_old, wv_old, wu, wv = wu, wv, wu_n, wv_n
        c_old, c, s_old, s = c, c_n, s, s_n
    return xu, xv


def shifted_solve(levels: List[Level], lam: complex, b: np.ndarray, iters: int, real: bool) -> np.ndarray:
    """Approximate (A - lam I)^{-1} b for one frequency (b complex of the field shape);
    real: the shift is real (frequencies 0 and ell/2), solved by CG."""
    if real:
        xr = pcg(levels, -lam.real, b.real.copy(), iters)
        xi = pcg(levels, -lam.real, b.imag.copy(), iters) if np.any(b.imag) else np.zeros_like(xr)
        return xr + 1j * xi
    conj = lam.imag < 0.0
    lp = np.conj(lam) if conj else lam
    bp = np.conj(b) if conj else b
    u, v = minres(levels, lp, -bp.imag.copy(), bp.real.copy(), iters)   # [Re x; -Im x]
    x = u - 1j * v
    return np.conj(x) if conj else x


def psp_apply(kx, ky, shape, r: np.ndarray, alpha: float, iters: int, kz=None) -> np.ndarray:
    """z = P_SP^{-1} r: Eq. 5 with every shifted solve replaced by iters Krylov steps (Section 4)."""
    ell = r.shape[0]
    levels = hierarchy(kx, ky, shape, kz)
    fshape = levels[0].w.shape
    lam = scaled_roots(ell, alpha)
    v = forward_transform(r, alpha)
    y = np.zeros_like(v)
    for j in range(ell):
        real = (j == 0) or (2 * j == ell)
        lj = complex(lam[j].real, 0.0) if real else complex(lam[j])
        y[j] = shifted_solve(levels, lj, v[j].reshape(fshape), iters, real).reshape(-1)
    return inverse_transform(y, alpha)
