"""Pins of the P_SP oracle (Section 4): the saddle-point reformulation, the spectrum of the
block-diagonally preconditioned system, and the Krylov and multigrid building blocks, each
against something other than the oracle itself."""
import numpy as np
import pytest
import scipy.sparse.linalg as sla

from oracle import operator as op
from oracle import precond as pc
from oracle import saddle as sd
from oracle import spectral as spc
from paper_2506_03947_gb300 import inputs


def _problem(n, seed=3):
    return inputs.make_problem("s", 2, n, 6, 1e-2, 1, 0.5, (4.0, 4.0), seed, seed + 1)


def _dense_S(A, lam):
    N = A.shape[0]
    Psi = A - lam.real * np.eye(N)
    Phi = lam.imag * np.eye(N)
    return np.block([[Phi, Psi], [Psi, -Phi]]), Phi, Psi


@pytest.mark.parametrize("j", [1, 2])
def test_saddle_reformulation_solves_the_complex_shifted_system(j):
    # S [Re x; -Im x] = [-Im b; Re b]  <=>  (A - lambda) x = b  (Section 4)
    P = _problem((9, 7))
    A = op.fv_dense(P.kx, P.ky, P.kz, P.shape)
    lam = np.conj(spc.scaled_roots(6, 0.3)[j])          # Im > 0
    b = np.random.default_rng(1).standard_normal(P.N) + 1j * np.random.default_rng(2).standard_normal(P.N)
    S, _, _ = _dense_S(A, lam)
    sol = np.linalg.solve(S, np.concatenate([-b.imag, b.real]))
    x = sol[:P.N] - 1j * sol[P.N:]
    ref = np.linalg.solve(A - lam * np.eye(P.N), b)
    assert np.abs(x - ref).max() < 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("alpha", [1e-2, 0.5])
def test_block_diagonal_preconditioned_spectrum(alpha):
    # Section 4's theorem: eig(P_D^{-1} S) in [-1, -1/sqrt 2] u [1/sqrt 2, 1], P_D = diag(Phi+Psi)
    P = _problem((6, 5))
    A = op.fv_dense(P.kx, P.ky, P.kz, P.shape)
    for lam in np.conj(spc.scaled_roots(6, alpha)[1:3]):
        S, Phi, Psi = _dense_S(A, lam)
        B = Phi + Psi
        PD = np.block([[B, np.zeros_like(B)], [np.zeros_like(B), B]])
        ev = np.linalg.eigvals(np.linalg.solve(PD, S)).real
        a = np.abs(ev)
        assert a.min() >= 1 / np.sqrt(2) - 1e-12 and a.max() <= 1 + 1e-12


def test_galerkin_coarse_operator():
    # each coarse level is R B P with piecewise-constant P (dense products), for any shift
    P = _problem((11, 7))
    lv = sd.hierarchy(P.kx, P.ky, P.shape)
    c = 0.37
    for q in range(len(lv) - 1):
        f, g = lv[q], lv[q + 1]
        m1, m0 = f.w.shape
        c1, c0 = g.w.shape
        Pm = np.zeros((m1 * m0, c1 * c0))
        for j in range(m1):
            for i in range(m0):
                Pm[i + m0 * j, (i // 2) + c0 * (j // 2)] = 1.0
        Bf = np.column_stack([sd.level_apply(f, c, e.reshape(m1, m0)).ravel() for e in np.eye(m1 * m0)])
        Bc = np.column_stack([sd.level_apply(g, c, e.reshape(c1, c0)).ravel() for e in np.eye(c1 * c0)])
        assert np.abs(Pm.T @ Bf @ Pm - Bc).max() < 1e-12 * np.abs(Bc).max()


def test_vcycle_is_symmetric_positive_definite():
    P = _problem((13, 10))
    lv = sd.hierarchy(P.kx, P.ky, P.shape)
    rng = np.random.default_rng(5)
    for c in (-0.6, 0.4):
        a, b = rng.standard_normal((10, 13)), rng.standard_normal((10, 13))
        va, vb = sd.vcycle(lv, c, a), sd.vcycle(lv, c, b)
        assert abs(np.vdot(va, b) - np.vdot(a, vb)) < 1e-12 * np.abs(va).max() * np.abs(b).sum()
        assert np.vdot(va, a) > 0 and np.vdot(vb, b) > 0


def test_pcg_matches_scipy_cg_iterates():
    P = _problem((16, 12))
    lv = sd.hierarchy(P.kx, P.ky, P.shape)
    c = -0.6
    b = np.random.default_rng(6).standard_normal((12, 16))
    N = b.size
    Aop = sla.LinearOperator((N, N), matvec=lambda v: sd.level_apply(lv[0], c, v.reshape(12, 16)).ravel())
    Mop = sla.LinearOperator((N, N), matvec=lambda v: sd.vcycle(lv, c, v.reshape(12, 16)).ravel())
    for k in (1, 3, 7):
        ref, _ = sla.cg(Aop, b.ravel(), rtol=0.0, atol=0.0, maxiter=k, M=Mop)
        x = sd.pcg(lv, c, b, k)
        assert np.abs(x.ravel() - ref).max() < 1e-10 * np.abs(ref).max()


def test_minres_matches_scipy_minres_iterates():
    P = _problem((10, 8))
    lv = sd.hierarchy(P.kx, P.ky, P.shape)
    lam = complex(np.conj(spc.scaled_roots(6, 1e-2)[1]))
    rng = np.random.default_rng(7)
    fu, fv = rng.standard_normal((8, 10)), rng.standard_normal((8, 10))
    N = fu.size
    c_pd = lam.imag - lam.real

    def S(v):
        su, sv = sd.saddle_apply(lv, lam, v[:N].reshape(8, 10), v[N:].reshape(8, 10))
        return np.concatenate([su.ravel(), sv.ravel()])

    def M(v):
        return np.concatenate([sd.vcycle(lv, c_pd, v[:N].reshape(8, 10)).ravel(),
                               sd.vcycle(lv, c_pd, v[N:].reshape(8, 10)).ravel()])

    Sop = sla.LinearOperator((2 * N, 2 * N), matvec=S)
    Mop = sla.LinearOperator((2 * N, 2 * N), matvec=M)
    for k in (1, 2, 5, 9):
        ref, _ = sla.minres(Sop, np.concatenate([fu.ravel(), fv.ravel()]), rtol=0.0, maxiter=k, M=Mop)
        xu, xv = sd.minres(lv, lam, fu, fv, k)
        x = np.concatenate([xu.ravel(), xv.ravel()])
        assert np.abs(x - ref).max() < 1e-9 * np.abs(ref).max(), k


def test_psp_tends_to_exact_palpha():
    P = _problem((20, 14))
    A = op.fv_dense(P.kx, P.ky, P.kz, P.shape)
    r = np.random.default_rng(1).standard_normal((P.ell, P.N))
    ze = pc.palpha_exact_apply(A, r, P.alpha)
    errs = [np.abs(sd.psp_apply(P.kx, P.ky, P.shape, r, P.alpha, k) - ze).max() / np.abs(ze).max()
            for k in (10, 20, 50)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-9


# ---- 3D grids: 2 x 2 x 2 aggregates -------------------------------------------------------

def _problem3(n, seed=13):
    return inputs.make_problem("s3", 3, n, 6, 1e-2, 1, 0.5, (3.0, 3.0, 2.0), seed, seed + 1)


def test_3d_finest_level_is_the_operator():
    # level 0 with c = 0 is A = I + K of the finite-volume operator module (Eq. 1's A)
    P = _problem3((7, 5, 4))
    lv = sd.hierarchy(P.kx, P.ky, P.shape, P.kz)
    A = op.fv_dense(P.kx, P.ky, P.kz, P.shape)
    x = np.random.default_rng(3).standard_normal(P.N)
    y = sd.level_apply(lv[0], 0.0, x.reshape(P.shape)).ravel()
    assert np.abs(y - A @ x).max() < 1e-12 * np.abs(A @ x).max()
    assert [L.w.shape for L in lv] == [(4, 5, 7), (2, 3, 4)]


def test_3d_galerkin_coarse_operator():
    P = _problem3((9, 6, 5))
    lv = sd.hierarchy(P.kx, P.ky, P.shape, P.kz)
    c = 0.29
    assert len(lv) == 3
    for q in range(len(lv) - 1):
        f, g = lv[q], lv[q + 1]
        fs, cs = f.w.shape, g.w.shape
        nf, nc = int(np.prod(fs)), int(np.prod(cs))
        Pm = np.zeros((nf, nc))
        for k in range(fs[0]):
            for j in range(fs[1]):
                for i in range(fs[2]):
                    Pm[i + fs[2] * (j + fs[1] * k), (i // 2) + cs[2] * ((j // 2) + cs[1] * (k // 2))] = 1.0
        Bf = np.column_stack([sd.level_apply(f, c, e.reshape(fs)).ravel() for e in np.eye(nf)])
        Bc = np.column_stack([sd.level_apply(g, c, e.reshape(cs)).ravel() for e in np.eye(nc)])
        assert np.abs(Pm.T @ Bf @ Pm - Bc).max() < 1e-12 * np.abs(Bc).max()


def test_3d_vcycle_is_symmetric_positive_definite():
    P = _problem3((10, 7, 6))
    lv = sd.hierarchy(P.kx, P.ky, P.shape, P.kz)
    rng = np.random.default_rng(15)
    shp = lv[0].w.shape
    for c in (-0.6, 0.4):
        a, b = rng.standard_normal(shp), rng.standard_normal(shp)
        va, vb = sd.vcycle(lv, c, a), sd.vcycle(lv, c, b)
        assert abs(np.vdot(va, b) - np.vdot(a, vb)) < 1e-12 * np.abs(va).max() * np.abs(b).sum()
        assert np.vdot(va, a) > 0 and np.vdot(vb, b) > 0


def test_3d_krylov_iterates_match_scipy():
    P = _problem3((9, 8, 6))
    lv = sd.hierarchy(P.kx, P.ky, P.shape, P.kz)
    shp = lv[0].w.shape
    N = P.N
    rng = np.random.default_rng(16)
    c = -0.6
    b = rng.standard_normal(shp)
    Aop = sla.LinearOperator((N, N), matvec=lambda v: sd.level_apply(lv[0], c, v.reshape(shp)).ravel())
    Mop = sla.LinearOperator((N, N), matvec=lambda v: sd.vcycle(lv, c, v.reshape(shp)).ravel())
    for k in (1, 4):
        ref, _ = sla.cg(Aop, b.ravel(), rtol=0.0, atol=0.0, maxiter=k, M=Mop)
        assert np.abs(sd.pcg(lv, c, b, k).ravel() - ref).max() < 1e-10 * np.abs(ref).max()
    lam = complex(np.conj(spc.scaled_roots(6, 1e-2)[1]))
    c_pd = lam.imag - lam.real
    fu, fv = rng.standard_normal(shp), rng.standard_normal(shp)

    def S(v):
        su, sv = sd.saddle_apply(lv, lam, v[:N].reshape(shp), v[N:].reshape(shp))
        return np.concatenate([su.ravel(), sv.ravel()])

    def M(v):
        return np.concatenate([sd.vcycle(lv, c_pd, v[:N].reshape(shp)).ravel(),
                               sd.vcycle(lv, c_pd, v[N:].reshape(shp)).ravel()])

    Sop = sla.LinearOperator((2 * N, 2 * N), matvec=S)
    Mop2 = sla.LinearOperator((2 * N, 2 * N), matvec=M)
    for k in (2, 6):
        ref, _ = sla.minres(Sop, np.concatenate([fu.ravel(), fv.ravel()]), rtol=0.0, maxiter=k, M=Mop2)
        xu, xv = sd.minres(lv, lam, fu, fv, k)
        assert np.abs(np.concatenate([xu.ravel(), xv.ravel()]) - ref).max() < 1e-9 * np.abs(ref).max(), k


def test_3d_psp_tends_to_exact_palpha():
    P = _problem3((6, 5, 4))
    A = op.fv_dense(P.kx, P.ky, P.kz, P.shape)
    r = np.random.default_rng(17).standard_normal((P.ell, P.N))
    ze = pc.palpha_exact_apply(A, r, P.alpha)
    errs = [np.abs(sd.psp_apply(P.kx, P.ky, P.shape, r, P.alpha, k, P.kz) - ze).max() / np.abs(ze).max()
            for k in (8, 16, 40)]
    assert errs[0] > errs[1] > errs[2] and errs[2] < 1e-9
