"""The seeded input recipe (paper_2506_03947_gb300/inputs.py) against its stated properties.

The oracle and the CUDA path both take their inputs from this module, so a mistake here would
go unnoticed by parity tests; these check the recipe itself. They cover:
  * the correlation the Gaussian filter produces;
  * the standardisation;
  * faces as geometric means of cell diffusivities;
  * the constant case kappa = 50 / ell;
  * the block structure of b;
  * determinism by seed;
  * the workloads' sizes and seeds.
"""
import numpy as np
import pytest

from paper_2506_03947_gb300 import inputs


def _autocorr_x(g, lag):
    a = g[0]
    return float(np.mean(a * np.roll(a, -lag, axis=1)))


def test_gaussian_field_is_standardised():
    g = inputs.gaussian_field((1, 96, 128), (16.0, 16.0), seed=3)
    assert abs(g.mean()) < 1e-12 and abs(g.std() - 1.0) < 1e-12


@pytest.mark.parametrize("corr", [4.0, 8.0])
def test_gaussian_field_correlation_is_exp_minus_d2_over_2lc2(corr):
    # Filtering white noise with a Gaussian of standard deviation s gives the correlation
    # exp(-d^2 / (4 s^2)); with s = Lc / sqrt(2) that is exp(-d^2 / (2 Lc^2)). A filter of width
    # Lc (a plausible slip) would give exp(-1/4) = 0.78 at d = Lc instead of exp(-1/2) = 0.61.
    g = inputs.gaussian_field((1, 512, 512), (corr, corr), seed=11)
    for lag in (int(corr / 2), int(corr), int(2 * corr)):
        expect = np.exp(-lag * lag / (2.0 * corr * corr))
        assert abs(_autocorr_x(g, lag) - expect) < 0.06, (lag, _autocorr_x(g, lag), expect)


def test_anisotropic_correlation_lengths_follow_the_axes():
    # corr is given in (x, y, z) order while arrays are (z, y, x): a swap would exchange these
    g = inputs.gaussian_field((1, 512, 512), (8.0, 2.0), seed=5)
    cx = float(np.mean(g[0] * np.roll(g[0], -4, axis=1)))
    cy = float(np.mean(g[0] * np.roll(g[0], -4, axis=0)))
    assert abs(cx - np.exp(-16.0 / 128.0)) < 0.06 and abs(cy - np.exp(-16.0 / 8.0)) < 0.06


def test_faces_are_geometric_means_of_cell_diffusivities():
    shape = (3, 5, 7)
    g = np.random.default_rng(0).standard_normal(shape)
    k0, sig = 2.5, 0.7
    kx, ky, kz = inputs.face_diffusivities(g, k0, sig)
    kc = k0 * np.exp(sig * g)
    assert kx.shape == (3, 5, 6) and ky.shape == (3, 4, 7) and kz.shape == (2, 5, 7)
    assert np.allclose(kx, np.sqrt(kc[:, :, :-1] * kc[:, :, 1:]), rtol=1e-14)
    assert np.allclose(ky, np.sqrt(kc[:, :-1, :] * kc[:, 1:, :]), rtol=1e-14)
    assert np.allclose(kz, np.sqrt(kc[:-1] * kc[1:]), rtol=1e-14)


@pytest.mark.parametrize("ell", [4, 10, 16])
def test_constant_case_is_fifty_over_ell(ell):
    P = inputs.make_problem("c", 2, (12, 8), ell, 1e-2, 5, 0.0, (16.0, 16.0), 1, 2)
    assert inputs.kappa0_for(ell) == 50.0 / ell
    assert np.all(P.kx == 50.0 / ell) and np.all(P.ky == 50.0 / ell) and P.kz.size == 0
    assert P.kx.shape == (1, 8, 11) and P.ky.shape == (1, 7, 12)


def test_rhs_block_structure():
    b = inputs.rhs(200000, 10, seed=4)
    assert b.shape == (10, 200000) and not np.any(b[1:])
    assert abs(b[0].mean()) < 0.01 and abs(b[0].std() - 1.0) < 0.01


def test_problems_are_deterministic_by_seed():
    a = inputs.config_2d(n=64)
    b = inputs.config_2d(n=64)
    c = inputs.config_2d(n=64, seed_field=99)
    assert np.array_equal(a.kx, b.kx) and np.array_equal(a.b, b.b)
    assert not np.array_equal(a.kx, c.kx) and np.array_equal(a.b, c.b)


def test_workload_sizes_and_seeds():
    P = inputs.config_1d()
    assert (P.dim, P.n, P.ell, P.alpha, P.inner_its, P.tol) == (1, (256, 1, 1), 10, 1e-2, 20, 1e-10)
    assert np.all(P.kx == 5.0)
    big = inputs.config_2d_large()
    assert (big.n, big.ell, big.alpha, big.inner_its, big.N) == ((1024, 1024, 1), 10, 1e-2, 40, 1048576)
    assert np.array_equal(big.b, inputs.rhs(big.N, 10, 22))
    P3 = inputs.config_3d(n=16)
    assert P3.b.shape == (8, 10, 16 ** 3) and P3.inner_its == 15
    assert np.array_equal(P3.b[3], inputs.rhs(16 ** 3, 10, 35))


def test_batch_specs_draw_from_the_stated_sets():
    specs = inputs.batch_specs(64, 42)
    assert specs == inputs.batch_specs(64, 42) and len(specs) == 64
    assert {n for n, _, _, _ in specs} <= {128, 192, 256, 384, 512}
    assert {l for _, l, _, _ in specs} <= {6, 8, 10, 12}
    assert {a for _, _, a, _ in specs} <= {1e-1, 1e-2}
    assert all(0.2 <= s <= 1.0 for _, _, _, s in specs)
    # every size and ell occurs in the 64 draws
    assert len({n for n, _, _, _ in specs}) == 5 and len({l for _, l, _, _ in specs}) == 4
