"""Pins for oracle/operator.py: closed forms, invariants, two independent assemblies."""
import numpy as np
import pytest

from oracle import operator as op
from paper_2506_03947_gb300 import inputs


def _rand_faces(shape, seed):
    rng = np.random.default_rng(seed)
    n2, n1, n0 = shape
    kx = rng.uniform(0.1, 3.0, (n2, n1, n0 - 1))
    ky = rng.uniform(0.1, 3.0, (n2, n1 - 1, n0))
    kz = rng.uniform(0.1, 3.0, (n2 - 1, n1, n0))
    return kx, ky, kz


def test_1d_constant_kappa_eigenvalues_are_dct_closed_form():
    # Neumann 3-point FV with constant kappa: eigenvectors are the DCT-II modes,
    # eigenvalues 1 + 4 kappa sin^2(pi k / (2N)), k = 0..N-1 (standard result).
    N, kappa = 64, 5.0
    P = inputs.make_problem("t", 1, (N,), 10, 1e-2, 1, 0.0, (0.0,), 0, 1, kappa0=kappa)
    A = op.fv_dense(P.kx, P.ky, P.kz, P.shape)
    k = np.arange(N)
    closed = 1.0 + 4.0 * kappa * np.sin(np.pi * k / (2 * N)) ** 2
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(A)), np.sort(closed), rtol=0, atol=1e-11)
    # DCT-II mode k is an eigenvector
    i = np.arange(N)
    for kk in (0, 1, 7, N - 1):
        v = np.cos(np.pi * kk * (i + 0.5) / N)
        np.testing.assert_allclose(A @ v, closed[kk] * v, atol=1e-11)


@pytest.mark.parametrize("shape", [(1, 1, 9), (1, 5, 7), (3, 4, 5), (1, 1, 1), (1, 2, 1)])
def test_apply_dense_sparse_agree(shape):
    kx, ky, kz = _rand_faces(shape, 3)
    N = int(np.prod(shape))
    A = op.fv_dense(kx, ky, kz, shape)
    As = op.fv_sparse(kx, ky, kz, shape).toarray()
    np.testing.assert_allclose(A, As, atol=1e-14)
    np.testing.assert_allclose(A, A.T, atol=0)
    x = np.random.default_rng(4).standard_normal(N)
    np.testing.assert_allclose(op.fv_apply(x.reshape(shape), kx, ky, kz).ravel(), A @ x, atol=1e-12)
    xc = x + 1j * np.random.default_rng(5).standard_normal(N)
    np.testing.assert_allclose(op.fv_apply(xc.reshape(shape), kx, ky, kz).ravel(), A @ xc, atol=1e-12)


def test_neumann_constant_vector_and_mu_min():
    P = inputs.config_2d(n=12)
    A = op.fv_dense(P.kx, P.ky, P.kz, P.shape)
    ones = np.ones(P.N)
    np.testing.assert_allclose(A @ ones, ones, atol=1e-12)   # K 1 = 0
    ev = np.linalg.eigvalsh(A)
    assert abs(ev[0] - op.MU_MIN_NEUMANN) < 1e-10
    assert ev[-1] <= op.gershgorin_mu_max(P.kx, P.ky, P.kz, P.shape) + 1e-12


def test_gershgorin_1d_constant():
    N, kappa = 32, 5.0
    P = inputs.make_problem("t", 1, (N,), 10, 1e-2, 1, 0.0, (0.0,), 0, 1, kappa0=kappa)
    assert op.gershgorin_mu_max(P.kx, P.ky, P.kz, P.shape) == pytest.approx(1 + 4 * kappa)
    # 3D: interior cells have 6 faces
    P3 = inputs.make_problem("t", 3, (4, 4, 4), 10, 1e-2, 1, 0.0, (0.0,), 0, 1, kappa0=kappa)
    assert op.gershgorin_mu_max(P3.kx, P3.ky, P3.kz, P3.shape) == pytest.approx(1 + 12 * kappa)


@pytest.mark.parametrize("nx,ell", [(12, 10), (9, 6)])
def test_dirichlet_operator_matches_appendix_a(nx, ell):
    # Appendix A: mu_ij = 1 + (4 nu/h^2)(sin^2(i pi/(2(nx+1))) + sin^2(j pi/(2(nx+1))))
    A = op.dirichlet_sparse(nx, ell).toarray()
    nu, h = op.dirichlet_params(nx, ell)
    assert nu == pytest.approx(0.04 / (2 * ell - 4))
    s = np.sin(np.arange(1, nx + 1) * np.pi / (2 * (nx + 1))) ** 2
    closed = 1 + 4 * nu / h ** 2 * (s[:, None] + s[None, :]).ravel()
    np.testing.assert_allclose(np.sort(np.linalg.eigvalsh(A)), np.sort(closed), atol=1e-10)
    mn, mx = op.dirichlet_mu_bounds(nx, ell)
    assert mn == pytest.approx(closed.min(), abs=1e-12) and mn > 1.0
    assert mx == pytest.approx(closed.max(), abs=1e-12)
    # eigenvectors V_i (x) V_j of Appendix A
    i = np.arange(1, nx + 1)
    V = np.sqrt(2.0 / (nx + 1)) * np.sin(np.outer(i, i) * np.pi / (nx + 1))
    X = np.kron(V[:, 1], V[:, 2])
    mu = 1 + 4 * nu / h ** 2 * (s[1] + s[2])
    np.testing.assert_allclose(A @ X, mu * X, atol=1e-10)
