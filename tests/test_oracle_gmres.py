"""Pins for oracle/gmres.py, oracle/exact.py and oracle/solve.py."""
import numpy as np
import pytest

from oracle import allatonce as aao
from oracle import exact
from oracle import operator as op
from oracle import precond as pc
from oracle import solve
from oracle.gmres import fgmres
from paper_2506_03947_gb300 import inputs


def test_sequential_solve_equals_dense_solve():
    P = inputs.config_2d(n=5)
    A = op.fv_dense(P.kx, P.ky, P.kz, P.shape)
    x = exact.sequential_solve_dense(A, P.b)
    xd = np.linalg.solve(aao.aao_dense(A, P.ell), P.b.ravel()).reshape(P.ell, P.N)
    np.testing.assert_allclose(x, xd, atol=1e-12 * np.abs(xd).max())
    xc = exact.sequential_solve_cg(lambda v: A @ v, P.b)
    np.testing.assert_allclose(xc, xd, atol=1e-11 * np.abs(xd).max())


def test_gmres_minimises_residual_over_krylov_space():
    # Unpreconditioned GMRES after k steps = least-squares minimiser over K_k(M, b) (brute force)
    rng = np.random.default_rng(0)
    n = 30
    M = np.eye(n) * 3 + rng.standard_normal((n, n)) * 0.3
    b = rng.standard_normal(n)
    for k in (1, 3, 6):
        res = fgmres(lambda v: M @ v, lambda v: v, b, 1e-30, k, fixed_its=k)
        K = np.stack([np.linalg.matrix_power(M, i) @ b for i in range(k)], axis=1)
        Q, _ = np.linalg.qr(K)
        c, *_ = np.linalg.lstsq(M @ Q, b, rcond=None)
        np.testing.assert_allclose(res.x, Q @ c, atol=1e-10)
        assert res.history[-1] == pytest.approx(np.linalg.norm(b - M @ res.x) / np.linalg.norm(b), rel=1e-8)


def test_config1_solution_against_dense_lu():
    # 1D, N = 256, ell = 10, alpha = 1e-2, 20 inner iterations, GMRES to 1e-10; ell*N = 2560
    P = inputs.config_1d()
    A = op.fv_dense(P.kx, P.ky, P.kz, P.shape)
    xd = np.linalg.solve(aao.aao_dense(A, P.ell), P.b.ravel()).reshape(P.ell, P.N)
    res = solve.solve(P.kx, P.ky, P.kz, P.shape, P.ell, P.alpha, P.b, P.inner_its, 1e-10, 64)
    assert res.converged and res.resid_explicit < 1e-10
    assert res.outer_its <= 8
    assert np.linalg.norm(res.x - xd) / np.linalg.norm(xd) < 1e-9


def test_exact_preconditioner_small_alpha_converges_in_few_steps():
    # spectrum of P_alpha^{-1} script-A clusters within ~alpha of 1 (Theorem 1, Remark 1)
    P = inputs.config_2d(n=6, alpha=1e-6)
    A = op.fv_dense(P.kx, P.ky, P.kz, P.shape)
    res = fgmres(lambda x: aao.aao_apply(lambda v: A @ v, x),
                 lambda r: pc.palpha_exact_apply(A, r, 1e-6), P.b, 1e-8, 10)
    assert res.converged and res.outer_its <= 3


def test_restarted_and_fixed_modes():
    P = inputs.config_2d(n=10)
    full = solve.solve(P.kx, P.ky, P.kz, P.shape, P.ell, P.alpha, P.b, 10, 1e-8, 64)
    rst = solve.solve(P.kx, P.ky, P.kz, P.shape, P.ell, P.alpha, P.b, 10, 1e-8, 200, restart=5)
    assert full.converged and rst.converged
    assert rst.outer_its >= full.outer_its
    fx = solve.solve(P.kx, P.ky, P.kz, P.shape, P.ell, P.alpha, P.b, 10, 1e-8, 64,
                     fixed_its=full.outer_its)
    np.testing.assert_allclose(fx.x, full.x, atol=1e-12 * np.abs(full.x).max())
