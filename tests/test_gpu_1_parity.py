"""GPU parity of the two operators behind the C ABI against the oracle.

aao_matvec (Eq. 1) and aao_precond_apply (Eq. 5 with p Chebyshev steps per
frequency) are compared element by element with oracle/ on the same seeded
inputs, on shapes that span several thread-block tiles with ragged edges, the
degenerate one-cell grid, 1D/2D/3D stencils and every supported ell.
"""
import numpy as np
import pytest

from gpu_util import (U64, ensure_lib, log_record, make_solver, oracle_ops, precond_err, precond_tol, to_dev,
                      torch_cuda)
from oracle import allatonce, operator, precond
from paper_2506_03947_gb300 import inputs

pytestmark = pytest.mark.gpu

SHAPES = [
    ("1d_n256_l10", lambda: inputs.config_1d()),
    ("1d_n1_l4", lambda: inputs.make_problem("n1", 1, (1,), 4, 0.3, 1, 0.0, (0.0,), 0, 1)),
    ("1d_n300_l6", lambda: inputs.make_problem("r", 1, (300,), 6, 1e-2, 1, 0.8, (8.0,), 5, 6)),
    ("2d_3x5_l4", lambda: inputs.make_problem("s", 2, (3, 5), 4, 0.5, 1, 0.5, (2.0, 2.0), 7, 8)),
    ("2d_37x29_l10", lambda: inputs.make_problem("r", 2, (37, 29), 10, 1e-2, 1, 0.5, (16.0, 16.0), 3, 4)),
    ("2d_64x64_l8", lambda: inputs.config_2d(n=64, ell=8, alpha=1e-1)),
    ("2d_70x9_l12", lambda: inputs.make_problem("r", 2, (70, 9), 12, 1e-3, 1, 1.0, (4.0, 4.0), 9, 10)),
    ("3d_5x4x3_l6", lambda: inputs.make_problem("c", 3, (5, 4, 3), 6, 1e-2, 1, 0.7, (8.0, 8.0, 4.0), 11, 12)),
    ("3d_33x9x7_l10", lambda: inputs.make_problem("c", 3, (33, 9, 7), 10, 1e-2, 1, 0.7, (8.0, 8.0, 4.0), 13, 14)),
    ("2d_20x20_l14", lambda: inputs.make_problem("r", 2, (20, 20), 14, 1e-2, 1, 0.5, (16.0, 16.0), 15, 16)),
    ("2d_20x20_l16", lambda: inputs.make_problem("r", 2, (20, 20), 16, 1e-2, 1, 0.5, (16.0, 16.0), 17, 18)),
]


def _rand_block(P, seed):
    return np.random.default_rng(seed).standard_normal((P.ell, P.N))


@pytest.mark.parametrize("name,mk", SHAPES, ids=[s[0] for s in SHAPES])
def test_matvec_parity(name, mk):
    torch = torch_cuda()
    P = mk()
    A, _ = oracle_ops(P)
    x = _rand_block(P, 1)
    ref = allatonce.aao_apply(A, x)
    s = make_solver(P, 0, 3)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    s.matvec(xd, yd)
    y = yd.cpu().numpy()
    err = np.abs(y - ref).max() / np.abs(ref).max()
    log_record({"test": "matvec", "case": name, "err": err})
    # the same sums in a different order: a few ulps of the largest term (mu_max |x|)
    bound = 16 * U64 * operator.gershgorin_mu_max(P.kx, P.ky, P.kz, P.shape)
    assert err <= bound, (err, bound)


@pytest.mark.parametrize("name,mk", SHAPES, ids=[s[0] for s in SHAPES])
def test_spectral_bounds_match_oracle(name, mk):
    P = mk()
    s = make_solver(P, 1, 3, device_faces=False)
    mu_min, mu_max = s.bounds()
    assert mu_min == 1.0
    ref = operator.gershgorin_mu_max(P.kx, P.ky, P.kz, P.shape)
    assert abs(mu_max - ref) <= 1e-14 * ref


@pytest.mark.parametrize("prec", [0, 1], ids=["fp64", "mixed"])
@pytest.mark.parametrize("p", [1, 2, 3, 4, 7, 20])
@pytest.mark.parametrize("name,mk", SHAPES, ids=[s[0] for s in SHAPES])
def test_precond_parity(name, mk, p, prec):
    torch = torch_cuda()
    P = mk()
    A, mu_max = oracle_ops(P)
    r = _rand_block(P, 2)
    ref = precond.pnc_apply(A, r, P.alpha, 1.0, mu_max, p)
    s = make_solver(P, prec, p)
    rd = to_dev(r)
    zd = torch.empty_like(rd)
    s.precond_apply(rd, zd)
    z = zd.cpu().numpy()
    err = precond_err(z, ref, P.ell, P.alpha)
    tol = precond_tol(prec, p)
    log_record({"test": "precond", "case": name, "p": p, "prec": prec, "err": err, "tol": tol,
                "ratio": err / tol})
    assert err <= tol, (err, tol)


def test_precond_host_pointers_match_device_pointers():
    torch = torch_cuda()
    P = inputs.config_2d(n=40)
    s = make_solver(P, 1, 9)
    r = _rand_block(P, 3)
    z_host = np.zeros_like(r)
    s.precond_apply(r, z_host)                  # numpy (host) buffers: staged by the library
    rd = to_dev(r)
    zd = torch.empty_like(rd)
    s.precond_apply(rd, zd)
    np.testing.assert_array_equal(zd.cpu().numpy(), z_host)


def test_precond_unaligned_device_buffers():
    # r read element by element may sit at any 8-byte boundary; a device z that is not 16-byte
    # aligned (the inverse transform stores two doubles at a time) is staged and copied on the
    # device, so both give the bits of the aligned apply
    torch = torch_cuda()
    binding = ensure_lib()
    for prec, p in ((1, 9), (1, 2), (0, 5)):
        P = inputs.config_2d(n=40)
        s = make_solver(P, prec, p)
        L = P.ell * P.N
        rd = to_dev(_rand_block(P, 4))
        zd = torch.empty_like(rd)
        s.precond_apply(rd, zd)
        rbuf = torch.zeros(L + 1, dtype=torch.float64, device="cuda")
        zbuf = torch.full((L + 1,), float("nan"), dtype=torch.float64, device="cuda")
        r1, z1 = rbuf[1:], zbuf[1:]
        r1.copy_(rd.reshape(-1))
        assert z1.data_ptr() % 16 == 8 and r1.data_ptr() % 16 == 8
        s.precond_apply(r1, z1)
        assert torch.equal(z1, zd.reshape(-1)), prec
        assert torch.isnan(zbuf[0])                       # nothing written before z
        # a pointer that is not 8-byte aligned is refused before any device work
        lib = binding.load_library()
        rc = lib.aao_precond_apply(s.h, rd.data_ptr() + 4, zd.data_ptr())
        assert rc == binding.AAO_EINVAL
        assert b"8-byte" in lib.aao_last_error(s.h)
        rc = lib.aao_matvec(s.h, rd.data_ptr(), zd.data_ptr() + 4)
        assert rc == binding.AAO_EINVAL


def test_precond_is_deterministic():
    torch = torch_cuda()
    P = inputs.config_2d(n=48)
    for prec in (0, 1):
        s = make_solver(P, prec, 11)
        rd = to_dev(_rand_block(P, 4))
        z1 = torch.empty_like(rd)
        z2 = torch.empty_like(rd)
        s.precond_apply(rd, z1)
        s.precond_apply(rd, z2)
        assert torch.equal(z1, z2)


def test_mixed_precond_is_close_to_exact_palpha_for_large_p():
    # p large: P_NC^{-1} -> P_alpha^{-1} (Eq. 5 with exact block solves); both precisions
    torch = torch_cuda()
    P = inputs.config_2d(n=8, ell=6, alpha=0.1)
    Ad = operator.fv_dense(P.kx, P.ky, P.kz, P.shape)
    r = _rand_block(P, 5)
    ref = precond.palpha_exact_apply(Ad, r, P.alpha)
    for prec, tol in ((0, 1e-9), (1, 2e-4)):
        s = make_solver(P, prec, 400)
        rd = to_dev(r)
        zd = torch.empty_like(rd)
        s.precond_apply(rd, zd)
        err = np.abs(zd.cpu().numpy() - ref).max() / np.abs(ref).max()
        assert err < tol, (prec, err)


def test_invalid_diffusivity_rejected_on_device():
    torch_cuda()
    binding = ensure_lib()
    P = inputs.config_2d(n=6)
    for bad in (np.nan, -1.0, 0.0, np.inf):
        kx = P.kx.ravel().copy()
        kx[3] = bad
        with pytest.raises(binding.AaoError) as ei:
            binding.Solver(2, P.n, kx, P.ky.ravel(), None, P.ell, P.alpha)
        assert ei.value.status == binding.AAO_EINVAL
