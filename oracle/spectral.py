"""Scalar parameters and convergence results of the method (oracle).

Notation follows the paper: ell blocks, shifts lambda_j (Section 2.2), Gamma
scaling, U Fourier matrix, B_j = A - lambda_j I (Eq. 8), spectrum of A in
[mu_N, mu_1] = [mu_min, mu_max].
"""
from __future__ import annotations

import numpy as np


def scaled_roots(ell: int, alpha: float) -> np.ndarray:
    """Shifts lambda_j, j = 1..ell, paired with U's columns (Section 2.2, Eq. 4).

    Reading of Eq. 4: with U_j = ell^{-1/2} (exp(+2 pi i (t-1)(j-1)/ell))_t,
    the alpha-circulant C_alpha equals Gamma^{-1} U Lambda U* Gamma only when
    lambda_j = alpha^{1/ell} exp(-2 pi i (j-1)/ell).  lambda_1 = alpha^{1/ell},
    lambda_{ell/2+1} = -alpha^{1/ell}, lambda_{ell+2-j} = conj(lambda_j).
    """
    j = np.arange(ell)
    return alpha ** (1.0 / ell) * np.exp(-2j * np.pi * j / ell)


def gamma(ell: int, alpha: float) -> np.ndarray:
    """Diagonal of Gamma_alpha: alpha^{(t-1)/ell}, t = 1..ell (Section 2.2)."""
    return alpha ** (np.arange(ell) / ell)


def fourier_matrix(ell: int) -> np.ndarray:
    """U with columns U_j = ell^{-1/2} (exp(2 pi i (t-1)(j-1)/ell))_{t=1..ell} (Section 2.2)."""
    t = np.arange(ell)[:, None]
    j = np.arange(ell)[None, :]
    return np.exp(2j * np.pi * t * j / ell) / np.sqrt(ell)


def cheb_interval(mu_min: float, mu_max: float, lam: complex):
    """Centre theta and half-width delta of the segment S_j (Lemma 2).

    The spectrum of B_j lies on [mu_min - lambda_j, mu_max - lambda_j]; its
    centre is (mu_max + mu_min)/2 - lambda_j and its half-length
    (mu_max - mu_min)/2.
    """
    return 0.5 * (mu_max + mu_min) - lam, 0.5 * (mu_max - mu_min)


def chebyshev_T(p: int, x):
    """T_p(x) for complex x: ((x + s)^p + (x - s)^p)/2 with s = sqrt(x^2 - 1) (Theorem 4).

    The sum is symmetric in the branch of s, so either square root gives T_p.
    """
    x = np.asarray(x, dtype=complex)
    s = np.sqrt(x * x - 1.0)
    return 0.5 * ((x + s) ** p + (x - s) ** p)


def error_bound(p: int, mu_min: float, mu_max: float, lam: complex) -> float:
    """|T_p((xi_1 + xi_N)/(xi_1 - xi_N))|^{-1}, xi_1 = mu_max - lam, xi_N = mu_min - lam.

    Proposition 1: bound on ||e_p|| / ||e_0|| for CI on B_j after p steps.
    """
    xi1 = mu_max - lam
    xiN = mu_min - lam
    return float(1.0 / abs(chebyshev_T(p, (xi1 + xiN) / (xi1 - xiN))))


def asymptotic_factor(mu_min: float, mu_max: float, lam: complex) -> float:
    """1 / |x + sqrt(x^2 - 1)|, x = (xi_1 + xi_N)/(xi_1 - xi_N), principal-real-part root.

    Lemma 3 and the proof of Theorem 4: the asymptotic convergence factor of
    CI on B_j.
    """
    xi1 = mu_max - lam
    xiN = mu_min - lam
    x = complex((xi1 + xiN) / (xi1 - xiN))
    s = np.sqrt(x * x - 1.0)
    if s.real < 0:
        s = -s
    return float(1.0 / abs(x + s))


def sigma_bound(mu_min: float, mu_max: float, lam: complex) -> float:
    """sigma_j = (sqrt(k) - 1)/(sqrt(k) + 1), k = condition number of Re(B_j) (Eq. 13)."""
    k = (mu_max - np.real(lam)) / (mu_min - np.real(lam))
    r = np.sqrt(k)
    return float((r - 1.0) / (r + 1.0))


def axelsson_iterations(eps: float, v_min: float, v_max: float) -> float:
    """p* of Theorem 3: iterations for CI on an SPD matrix with spectrum in [v_min, v_max]."""
    q = np.sqrt(v_min / v_max)
    return float(np.log(1.0 / eps + np.sqrt(1.0 / eps ** 2 - 1.0)) / np.log((1.0 + q) / (1.0 - q)))


def assign_iterations(ell: int, nx: int, mu_max: float, mu_min: float, alpha: float,
                      eta: float) -> np.ndarray:
    """Algorithm 1: share ell*n_x*eta inner iterations by ln(sigma_1)/ln(sigma_j)."""
    lam = scaled_roots(ell, alpha)
    sig = np.array([sigma_bound(mu_min, mu_max, l) for l in lam])
    r = np.log(sig[0]) / np.log(sig)
    r = r / r.sum()
    return np.floor(r * ell * nx * eta).astype(np.int64)


def preconditioned_extremes(mu_min: float, ell: int, alpha: float):
    """Corollary 1: for 0 < alpha < mu_N^ell, spectrum of P^{-1} script-A is in [1, mu_N^ell/(mu_N^ell - alpha)]."""
    m = mu_min ** ell
    return 1.0, m / (m - alpha)


def preconditioned_eigenvalues(mu: np.ndarray, ell: int, alpha: float) -> np.ndarray:
    """Theorem 1: 1 with multiplicity (ell-1)N, and mu_j^ell/(mu_j^ell - alpha)."""
    N = len(mu)
    m = np.asarray(mu) ** ell
    return np.concatenate([np.ones((ell - 1) * N), m / (m - alpha)])
