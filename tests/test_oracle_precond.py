"""Pins for oracle/precond.py: dense P_alpha^{-1}, closed-form P_NC^{-1}, symmetry, limits."""
import numpy as np
import pytest
import scipy.fft as sfft

from oracle import allatonce as aao
from oracle import operator as op
from oracle import precond as pc
from oracle import spectral as spc
from paper_2506_03947_gb300 import inputs


def test_dft_round_trip_and_conjugate_symmetry():
    rng = np.random.default_rng(0)
    for ell in (4, 6, 10):
        r = rng.standard_normal((ell, 7))
        v = pc.forward_transform(r, 0.03)
        for j in range(1, ell):
            np.testing.assert_allclose(v[ell - j], np.conj(v[j]), atol=1e-13)
        np.testing.assert_allclose(v[0].imag, 0, atol=1e-13)
        np.testing.assert_allclose(v[ell // 2].imag, 0, atol=1e-13)
        np.testing.assert_allclose(pc.inverse_transform(v, 0.03), r, atol=1e-12)
        # against numpy's FFT of the scaled vector (library routine, same convention)
        s = spc.gamma(ell, 0.03)[:, None] * r
        np.testing.assert_allclose(v, np.fft.fft(s, axis=0) / np.sqrt(ell), atol=1e-13)


@pytest.mark.parametrize("ell,alpha", [(4, 0.5), (6, 1e-2), (10, 1e-2), (10, 0.3)])
def test_exact_dft_path_equals_dense_inverse(ell, alpha):
    P = inputs.config_2d(n=4, ell=ell, alpha=alpha)
    A = op.fv_dense(P.kx, P.ky, P.kz, P.shape)
    r = np.random.default_rng(1).standard_normal((ell, P.N))
    z = pc.palpha_exact_apply(A, r, alpha)
    zd = np.linalg.solve(aao.p_alpha_dense(A, ell, alpha), r.ravel()).reshape(ell, P.N)
    np.testing.assert_allclose(z, zd, atol=1e-11 * np.abs(zd).max())


def _pnc_closed_form_1d(r, N, kappa, ell, alpha, p):
    # 1D constant kappa: P_NC^{-1} = (G^{-1}U x V) diag(q(mu_k - lambda_j)) (U*G x V^T),
    # V the orthonormal DCT-II, q(z) = (1 - Omega_p(z))/z, Omega_p the Chebyshev error polynomial.
    mu = 1 + 4 * kappa * np.sin(np.pi * np.arange(N) / (2 * N)) ** 2
    lam = spc.scaled_roots(ell, alpha)
    g = spc.gamma(ell, alpha)
    s = g[:, None] * r
    v = np.fft.fft(s, axis=0) / np.sqrt(ell)                 # U* over t
    vh = sfft.dct(v.real, type=2, norm="ortho", axis=1) + 1j * sfft.dct(v.imag, type=2, norm="ortho", axis=1)
    out = np.zeros_like(vh)
    for j in range(ell):
        th, de = spc.cheb_interval(1.0, 1 + 4 * kappa, lam[j])
        zk = mu - lam[j]
        om = spc.chebyshev_T(p, (th - zk) / de) / spc.chebyshev_T(p, th / de)
        out[j] = (1 - om) / zk * vh[j]
    y = sfft.idct(out.real, type=2, norm="ortho", axis=1) + 1j * sfft.idct(out.imag, type=2, norm="ortho", axis=1)
    zt = np.fft.ifft(y, axis=0) * np.sqrt(ell)
    return zt.real / g[:, None]


@pytest.mark.parametrize("p", [1, 2, 7, 20])
@pytest.mark.parametrize("alpha", [0.5, 1e-2])
def test_pnc_matches_closed_form_1d(p, alpha):
    N, kappa, ell = 32, 5.0, 10
    P = inputs.make_problem("t", 1, (N,), ell, alpha, p, 0.0, (0.0,), 0, 1, kappa0=kappa)
    A = lambda v: op.fv_apply(v.reshape(P.shape), P.kx, P.ky, P.kz).ravel()
    r = np.random.default_rng(3).standard_normal((ell, N))
    z = pc.pnc_apply(A, r, alpha, 1.0, 1 + 4 * kappa, p)
    zc = _pnc_closed_form_1d(r, N, kappa, ell, alpha, p)
    np.testing.assert_allclose(z, zc, atol=1e-11 * np.abs(zc).max())


def test_pnc_tends_to_exact_palpha_and_is_linear():
    P = inputs.config_2d(n=6, ell=6, alpha=0.1)
    Ad = op.fv_dense(P.kx, P.ky, P.kz, P.shape)
    A = lambda v: Ad @ v
    mu_max = op.gershgorin_mu_max(P.kx, P.ky, P.kz, P.shape)
    rng = np.random.default_rng(4)
    r1, r2 = rng.standard_normal((2, 6, P.N))
    z_exact = pc.palpha_exact_apply(Ad, r1, 0.1)
    prev = np.inf
    for p in (5, 20, 80, 300):
        e = np.abs(pc.pnc_apply(A, r1, 0.1, 1.0, mu_max, p) - z_exact).max()
        assert e < prev
        prev = e
    assert prev < 1e-9 * np.abs(z_exact).max()
    za = pc.pnc_apply(A, 2.0 * r1 - 3.0 * r2, 0.1, 1.0, mu_max, 9)
    zb = 2.0 * pc.pnc_apply(A, r1, 0.1, 1.0, mu_max, 9) - 3.0 * pc.pnc_apply(A, r2, 0.1, 1.0, mu_max, 9)
    np.testing.assert_allclose(za, zb, atol=1e-11 * np.abs(zb).max())


def test_single_cell_degenerate_segment_is_exact():
    # N = 1: A = I, the segment of Lemma 2 is one point; CI's delta -> 0 limit is the exact solve
    P = inputs.make_problem("t", 1, (1,), 4, 0.3, 1, 0.0, (0.0,), 0, 1)
    A = op.fv_dense(P.kx, P.ky, P.kz, P.shape)
    assert op.gershgorin_mu_max(P.kx, P.ky, P.kz, P.shape) == 1.0
    r = np.random.default_rng(9).standard_normal((4, 1))
    for p in (1, 2, 5):
        z = pc.pnc_apply(lambda v: A @ v, r, 0.3, 1.0, 1.0, p)
        np.testing.assert_allclose(z, pc.palpha_exact_apply(A, r, 0.3), atol=1e-13)


def _constant_faces(shape, kap):
    n2, n1, n0 = shape
    kx = np.full((n2, n1, max(n0 - 1, 0)), kap[0])
    ky = np.full((n2, max(n1 - 1, 0), n0), kap[1])
    kz = np.full((max(n2 - 1, 0), n1, n0), kap[2])
    return kx, ky, kz


@pytest.mark.parametrize("shape,kap", [((1, 1, 9), (4.0, 0.0, 0.0)), ((1, 6, 7), (3.0, 2.0, 0.0)),
                                       ((3, 4, 5), (1.5, 2.5, 0.7))])
def test_dct_eigenvalues_are_the_spectrum_of_constant_kappa_A(shape, kap):
    # the closed form of the separable Neumann operator against a dense symmetric eigensolver
    kx, ky, kz = _constant_faces(shape, kap)
    ev = np.sort(np.linalg.eigvalsh(op.fv_dense(kx, ky, kz, shape)))
    phi = np.sort(pc.neumann_dct_eigenvalues(kap, shape).ravel())
    assert np.abs(ev - phi).max() < 1e-12 * ev.max()
    assert abs(phi.min() - 1.0) < 1e-15   # mu_min = 1 (the constant mode)


@pytest.mark.parametrize("alpha", [0.5, 1e-2])
@pytest.mark.parametrize("shape,kap", [((1, 6, 7), (3.0, 2.0, 0.0)), ((3, 4, 5), (1.5, 2.5, 0.7))])
def test_dct_palpha_equals_dense_palpha_and_inverts_palpha(shape, kap, alpha):
    # best-case P_alpha^{-1} through the spatial DCT equals the dense-solve path of Eq. 5 and
    # is the inverse of P_alpha (Eq. 2) applied as script-A plus the circulant corner
    ell = 6
    kx, ky, kz = _constant_faces(shape, kap)
    A = op.fv_dense(kx, ky, kz, shape)
    r = np.random.default_rng(4).standard_normal((ell, A.shape[0]))
    z_dct = pc.palpha_dct_apply(kap, shape, r, alpha)
    z_dense = pc.palpha_exact_apply(A, r, alpha)
    assert np.abs(z_dct - z_dense).max() < 1e-12 * np.abs(z_dense).max()
    back = aao.p_alpha_apply(lambda v: A @ v, z_dct, alpha)
    assert np.abs(back - r).max() < 1e-11 * np.abs(r).max()
