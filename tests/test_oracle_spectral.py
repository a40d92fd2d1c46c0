"""Pins for oracle/spectral.py: printed roots, Tables 2-4, Theorems 3-4, Proposition 1."""
import numpy as np
import pytest

from conftest import read_golden
from oracle import operator as op
from oracle import spectral as spc


def test_printed_roots_and_labelling():
    rows = {r[0]: complex(float(r[1]), float(r[2])) for r in read_golden("roots_l10.txt")}
    lam = spc.scaled_roots(10, 1.0)
    # the printed values (4 decimals) are members of the set, with their conjugates
    for v in rows.values():
        assert np.abs(lam - v).min() < 6e-5
        assert np.abs(lam - np.conj(v)).min() < 6e-5
    for ell, alpha in ((10, 1.0), (10, 1e-2), (6, 0.1), (12, 1e-3)):
        lam = spc.scaled_roots(ell, alpha)
        r = alpha ** (1 / ell)
        assert lam[0] == pytest.approx(r) and lam[ell // 2] == pytest.approx(-r)
        for j in range(1, ell // 2):
            assert lam[ell - j] == pytest.approx(np.conj(lam[j]))
            assert abs(lam[j].imag) > 0
        # real parts decrease from lambda_1 to lambda_{ell/2+1} (Section 3)
        assert np.all(np.diff(lam[: ell // 2 + 1].real) < 0)
    np.testing.assert_allclose(spc.gamma(4, 1e-4), [1, 1e-1, 1e-2, 1e-3])


def test_chebyshev_polynomial_definitions_agree():
    th = np.linspace(0, np.pi, 7)
    for p in (0, 1, 2, 5, 17):
        np.testing.assert_allclose(spc.chebyshev_T(p, np.cos(th)).real, np.cos(p * th), atol=1e-12)
        x = np.array([1.5, 3.0, 40.0])
        np.testing.assert_allclose(spc.chebyshev_T(p, x).real, np.cosh(p * np.arccosh(x)), rtol=1e-12)
    # three-term recurrence for complex arguments
    z = np.array([1.3 + 0.4j, -2.0 + 1.0j, 0.2 - 3.0j])
    t0, t1 = np.ones_like(z), z
    for p in range(2, 12):
        t0, t1 = t1, 2 * z * t1 - t0
        np.testing.assert_allclose(spc.chebyshev_T(p, z), t1, rtol=1e-11)


def test_theorem3_iterations_match_table2_real_roots():
    # Theorem 3's p* for lambda = +-1 against Table 2's counted CI iterations (n_x = 100, alpha = 1)
    mn, mx = op.dirichlet_mu_bounds(100, 10)
    for row in read_golden("table2_ci_iterations.txt"):
        eps = float(row[0])
        n_plus, n_minus = int(row[1]), int(row[6])
        p_plus = spc.axelsson_iterations(eps, mn - 1.0, mx - 1.0)
        p_minus = spc.axelsson_iterations(eps, mn + 1.0, mx + 1.0)
        assert abs(p_plus - n_plus) <= max(6, 0.02 * n_plus), (eps, p_plus, n_plus)
        assert abs(p_minus - n_minus) <= 3, (eps, p_minus, n_minus)


def test_theorem4_bound_and_ordering():
    mn, mx = op.dirichlet_mu_bounds(100, 10)
    for alpha in (1.0, 1e-2):
        lam = spc.scaled_roots(10, alpha)
        sig = [spc.sigma_bound(mn, mx, l) for l in lam]
        rho = [spc.asymptotic_factor(mn, mx, l) for l in lam]
        for j in range(10):
            if abs(lam[j].imag) > 1e-12:
                assert rho[j] < sig[j]                                # Eq. 13, strict for complex shifts
            else:
                assert rho[j] == pytest.approx(sig[j], rel=1e-12)     # equal for real shifts
        # conjugates share sigma; smaller real part gives smaller sigma (Section 3.2 remarks)
        for j in range(1, 5):
            assert sig[j] == pytest.approx(sig[10 - j])
        assert np.all(np.diff(sig[:6]) < 0)


def test_proposition1_bound_tends_to_asymptotic_factor():
    mn, mx = 1.0, 180.0
    lam = spc.scaled_roots(10, 1e-2)[2]
    rho = spc.asymptotic_factor(mn, mx, lam)
    prev = None
    for p in (50, 200, 800):
        b = spc.error_bound(p, mn, mx, lam) ** (1.0 / p)
        if prev is not None:
            assert abs(b - rho) < abs(prev - rho)
        prev = b
    assert prev == pytest.approx(rho, rel=2e-3)
    # p = 1: |T_1(x)|^{-1} = |xi_1 - xi_N| / |xi_1 + xi_N| (Proposition 2)
    xi1, xiN = mx - lam, mn - lam
    assert spc.error_bound(1, mn, mx, lam) == pytest.approx(abs(xi1 - xiN) / abs(xi1 + xiN))


def test_algorithm1_and_budget_reproduce_tables_3_and_4():
    # Table 1 budget: script-A costs ell matvecs, NC1 costs ell*n_x*eta, NC2 the Algorithm 1 total.
    rows = read_golden("nc_matvec_counts.txt")
    assert len(rows) == 114
    for tab, meth, ell, nx, alpha, eta, its, mv in rows:
        ell, nx, alpha, eta, its, mv = int(ell), int(nx), float(alpha), float(eta), int(its), int(mv)
        if meth == "NC1":
            per = ell + int(round(ell * nx * eta))
        else:
            mn, mx = op.dirichlet_mu_bounds(nx, ell)
            per = ell + int(spc.assign_iterations(ell, nx, mx, mn, alpha, eta).sum())
        assert its * per == mv, (tab, meth, ell, nx, alpha, eta)


def test_algorithm1_allocation_shape():
    mn, mx = op.dirichlet_mu_bounds(100, 10)
    a = spc.assign_iterations(10, 100, mx, mn, 1.0, 0.1)
    # lambda = 1 gets the most, lambda = -1 the least; conjugate pairs equal (Section 5.2 text)
    assert a[0] == 30 and a[5] == 4
    assert all(a[j] == a[10 - j] for j in range(1, 5))
