"""Applying P_alpha^{-1} through the time DFT (oracle; Section 2.2, Section 3).

Eq. 5:  P_alpha^{-1} = (Gamma^{-1} U (x) I)(I (x) A - Lambda (x) I)^{-1}(U* Gamma (x) I).

Steps for a real block vector r of shape (ell, N):
  1. s_t = gamma_t r_t                                   (Gamma)
  2. v_j = ell^{-1/2} sum_t s_t exp(-2 pi i (t-1)(j-1)/ell)  (U*, naive DFT,
     all ell frequencies, no symmetry shortcut)
  3. y_j = (A - lambda_j I)^{-1} v_j, either exactly or by p steps of CI
     (Eq. 7 per frequency; P_NC when approximated by CI)
  4. zhat_t = ell^{-1/2} sum_j y_j exp(+2 pi i (t-1)(j-1)/ell)   (U)
  5. z_t = Re(zhat_t)/gamma_t                             (Gamma^{-1})
For real r and even ell the y_j come in conjugate pairs, so zhat is real up to
rounding; step 5 checks that.
"""
from __future__ import annotations

from typing import Callable, Sequence, Union

import numpy as np

from .chebyshev import chebyshev_solve
from .spectral import cheb_interval, gamma, scaled_roots

Apply = Callable[[np.ndarray], np.ndarray]


def forward_transform(r: np.ndarray, alpha: float) -> np.ndarray:
    """Steps 1-2: v = (U* Gamma (x) I) r, by the naive DFT sum."""
    ell = r.shape[0]
    g = gamma(ell, alpha)
    v = np.zeros(r.shape, dtype=complex)
    for j in range(ell):
        for t in range(ell):
            v[j] += np.exp(-2j * np.pi * t * j / ell) * (g[t] * r[t])
    return v / np.sqrt(ell)


def inverse_transform(y: np.ndarray, alpha: float, check_real: bool = True) -> np.ndarray:
    """Steps 4-5: z = (Gamma^{-1} U (x) I) y, returning the real part."""
    ell = y.shape[0]
    g = gamma(ell, alpha)
    zh = np.zeros(y.shape, dtype=complex)
    for t in range(ell):
        for j in range(ell):
            zh[t] += np.exp(2j * np.pi * t * j / ell) * y[j]
    zh /= np.sqrt(ell)
    if check_real:
        scale = max(np.abs(zh).max(), 1e-300)
        if np.abs(zh.imag).max() > 1e-10 * scale:
            raise AssertionError("inverse DFT is not real: conjugate symmetry broken")
    return zh.real / g[:, None]


def pnc_apply(A: Apply, r: np.ndarray, alpha: float, mu_min: float, mu_max: float,
              p: Union[int, Sequence[int]]) -> np.ndarray:
    """z = P_NC^{-1} r: Eq. 5 with each block solve replaced by p steps of CI.

    ``p`` is one count for every frequency (NC1) or a list of ell counts (NC2,
    Algorithm 1).  CI on B_j = A - lambda_j I uses the segment of Lemma 2.
    """
    ell = r.shape[0]
    lam = scaled_roots(ell, alpha)
    ps = [int(p)] * ell if np.isscalar(p) else [int(q) for q in p]
    v = forward_transform(r, alpha)
    y = np.zeros_like(v)
    for j in range(ell):
        theta, delta = cheb_interval(mu_min, mu_max, lam[j])
        lj = lam[j]
        y[j] = chebyshev_solve(lambda w, lj=lj: A(w) - lj * w, v[j], theta, delta, ps[j])
    return inverse_transform(y, alpha)


def palpha_exact_apply(A_dense: np.ndarray, r: np.ndarray, alpha: float) -> np.ndarray:
    """z = P_alpha^{-1} r through Eq. 5 with exact (dense) block solves."""
    ell = r.shape[0]
    N = A_dense.shape[0]
    lam = scaled_roots(ell, alpha)
    v = forward_transform(r, alpha)
    y = np.zeros_like(v)
    for j in range(ell):
        y[j] = np.linalg.solve(A_dense - lam[j] * np.eye(N), v[j])
    return inverse_transform(y, alpha)


def neumann_dct_eigenvalues(kappa: Sequence[float], shape) -> np.ndarray:
    """Eigenvalues of A = I + K for spatially constant face diffusivities, one per axis.

    The finite-volume Neumann operator with constant kappa_a on axis a is a sum of scaled 1D
    Neumann Laplacians (diagonal 2, ends 1, off-diagonals -1), each diagonalised by the
    orthonormal DCT-II with eigenvalues 4 sin^2(pi k / (2 n_a)), k = 0..n_a-1; A is
    diagonalised by their tensor product (the decomposition A = X Phi X^T of Section 2.2).
    shape = (n2, n1, n0); kappa = (kappa_x, kappa_y, kappa_z); returns Phi with that shape.
    """
    n2, n1, n0 = shape
    ev = [4.0 * np.sin(np.pi * np.arange(n) / (2.0 * n)) ** 2 for n in (n0, n1, n2)]
    phi = np.ones(shape)
    phi += kappa[0] * ev[0][None, None, :]
    phi += kappa[1] * ev[1][None, :, None]
    phi += kappa[2] * ev[2][:, None, None]
    return phi


def palpha_dct_apply(kappa: Sequence[float], shape, r: np.ndarray, alpha: float) -> np.ndarray:
    """z = P_alpha^{-1} r exactly, for spatially constant face diffusivities (Section 2.2).

    Eq. 5 with A = X Phi X^T: the shifted solves (A - lambda_j I) y_j = v_j become
    y_j = X (Phi - lambda_j)^{-1} X^T v_j, X the orthonormal DCT-II along every axis
    (scipy.fft.dctn / idctn, type 2, norm 'ortho').  This is the paper's best-case
    preconditioner, applied without a dense factorisation.
    """
    from scipy.fft import dctn, idctn

    ell = r.shape[0]
    lam = scaled_roots(ell, alpha)
    phi = neumann_dct_eigenvalues(kappa, shape)
    v = forward_transform(r, alpha)
    y = np.zeros_like(v)
    for j in range(ell):
        vj = v[j].reshape(shape)
        vh = dctn(vj.real, type=2, norm="ortho") + 1j * dctn(vj.imag, type=2, norm="ortho")
        yh = vh / (phi - lam[j])
        y[j] = (idctn(yh.real, type=2, norm="ortho") + 1j * idctn(yh.imag, type=2, norm="ortho")).reshape(-1)
    return inverse_transform(y, alpha)
