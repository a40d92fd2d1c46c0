"""Pins for oracle/allatonce.py and the spectral results of Section 2."""
import numpy as np
import pytest

from oracle import allatonce as aao
from oracle import operator as op
from oracle import spectral as spc
from paper_2506_03947_gb300 import inputs


def _small_A(N=6, kappa=1.5):
    P = inputs.make_problem("t", 1, (N,), 6, 1e-2, 1, 0.0, (0.0,), 0, 1, kappa0=kappa)
    A = op.fv_dense(P.kx, P.ky, P.kz, P.shape)
    mu = 1 + 4 * kappa * np.sin(np.pi * np.arange(N) / (2 * N)) ** 2   # DCT closed form
    return A, mu


def test_aao_dense_and_apply_agree():
    A, _ = _small_A()
    ell = 6
    M = aao.aao_dense(A, ell)
    x = np.random.default_rng(0).standard_normal((ell, A.shape[0]))
    y = aao.aao_apply(lambda v: A @ v, x)
    np.testing.assert_allclose(M @ x.ravel(), y.ravel(), atol=1e-12)
    # block lower bidiagonal: A on the diagonal, -I below (Eq. 1)
    N = A.shape[0]
    np.testing.assert_array_equal(M[N:2 * N, 0:N], -np.eye(N))
    np.testing.assert_array_equal(M[0:N, N:2 * N], 0)


def test_palpha_differs_from_aao_by_corner_block():
    A, _ = _small_A()
    ell, N = 6, A.shape[0]
    for alpha in (1.0, 0.3, 1e-2):
        Pd = aao.p_alpha_dense(A, ell, alpha)
        E1 = np.kron(np.eye(ell)[:, [0]], np.eye(N))
        El = np.kron(np.eye(ell)[:, [ell - 1]], np.eye(N))
        # P_alpha = script-A - alpha E_1 E_ell^T (proof of Lemma 1)
        np.testing.assert_allclose(Pd, aao.aao_dense(A, ell) - alpha * E1 @ El.T, atol=0)
        x = np.random.default_rng(1).standard_normal((ell, N))
        np.testing.assert_allclose(Pd @ x.ravel(), aao.p_alpha_apply(lambda v: A @ v, x, alpha).ravel(),
                                   atol=1e-12)
    np.testing.assert_array_equal(aao.p_alpha_dense(A, ell, 0.0), aao.aao_dense(A, ell))


@pytest.mark.parametrize("ell", [4, 6, 10, 12])
@pytest.mark.parametrize("alpha", [1.0, 1e-2, 1e-5])
def test_kronecker_factorisation_reproduces_c_alpha(ell, alpha):
    # Eq. 4: C_alpha = Gamma^{-1} U Lambda U* Gamma with the shift pairing of spectral.scaled_roots
    U = spc.fourier_matrix(ell)
    G = np.diag(spc.gamma(ell, alpha))
    Lam = np.diag(spc.scaled_roots(ell, alpha))
    np.testing.assert_allclose(U @ U.conj().T, np.eye(ell), atol=1e-13)
    C = np.linalg.inv(G) @ U @ Lam @ U.conj().T @ G
    np.testing.assert_allclose(C, aao.c_alpha(ell, alpha), atol=1e-12 / min(alpha, 1.0) ** ((ell - 1) / ell))


def test_printed_sign_pairing_does_not_reproduce_c_alpha():
    # As printed, lambda_j = alpha^{1/ell} exp(+2 pi i (j-1)/ell) with the same U; that pairing
    # gives C_alpha's transpose-like matrix instead, which is why the conjugate pairing is used.
    ell, alpha = 6, 1.0
    U = spc.fourier_matrix(ell)
    lam_printed = alpha ** (1 / ell) * np.exp(2j * np.pi * np.arange(ell) / ell)
    C = U @ np.diag(lam_printed) @ U.conj().T
    assert np.abs(C - aao.c_alpha(ell, alpha)).max() > 0.5


def test_full_kronecker_form_of_palpha():
    A, _ = _small_A(N=4)
    ell, alpha, N = 6, 0.05, 4
    U = spc.fourier_matrix(ell)
    G = np.diag(spc.gamma(ell, alpha))
    Lam = np.diag(spc.scaled_roots(ell, alpha))
    left = np.kron(np.linalg.inv(G) @ U, np.eye(N))
    mid = np.kron(np.eye(ell), A) - np.kron(Lam, np.eye(N))
    right = np.kron(U.conj().T @ G, np.eye(N))
    np.testing.assert_allclose(left @ mid @ right, aao.p_alpha_dense(A, ell, alpha), atol=1e-11)


def test_lemma1_sherman_morrison_woodbury():
    A, _ = _small_A(N=5)
    ell, alpha, N = 6, 0.2, 5
    Ad = aao.aao_dense(A, ell)
    Ainv = np.linalg.inv(Ad)
    E1 = np.kron(np.eye(ell)[:, [0]], np.eye(N))
    El = np.kron(np.eye(ell)[:, [ell - 1]], np.eye(N))
    Aml = np.linalg.matrix_power(np.linalg.inv(A), ell)
    np.testing.assert_allclose(El.T @ Ainv @ E1, Aml, atol=1e-13)        # E_l^T A^{-1} E_1 = A^{-l}
    Z = (np.eye(N) - alpha * Aml) / alpha
    smw = Ainv + Ainv @ E1 @ np.linalg.inv(Z) @ El.T @ Ainv
    np.testing.assert_allclose(smw, np.linalg.inv(aao.p_alpha_dense(A, ell, alpha)), atol=1e-11)


@pytest.mark.parametrize("alpha", [0.5, 1e-2])
def test_theorem1_and_corollary1_spectrum(alpha):
    A, mu = _small_A(N=8)
    ell = 6
    M = np.linalg.solve(aao.p_alpha_dense(A, ell, alpha), aao.aao_dense(A, ell))
    ev = np.sort(np.linalg.eigvals(M).real)
    assert np.abs(np.linalg.eigvals(M).imag).max() < 1e-8
    np.testing.assert_allclose(ev, np.sort(spc.preconditioned_eigenvalues(mu, ell, alpha)), atol=1e-8)
    lo, hi = spc.preconditioned_extremes(mu.min(), ell, alpha)
    assert ev[0] == pytest.approx(lo, abs=1e-8) and ev[-1] == pytest.approx(hi, rel=1e-8)
    # Remark 1 (Lin-Ng): |lambda - 1| <= alpha/(1 - eta') for alpha <= eta' < 1 (mu_min >= 1 here)
    eta_p = max(alpha, 0.6)
    assert np.abs(ev - 1).max() <= alpha / (1 - eta_p) + 1e-12
