"""The two kernels of the fused four-step Chebyshev sweep (2D mixed path).

aao_set_step_kernel selects the shared-memory tile kernel or the persistent
TMA-fed kernel; both compute Chebyshev steps k .. k+3 of Eq. 7 on every
frequency.  Each is compared with the oracle's P_NC^{-1} (Eq. 5 with p
Chebyshev steps per frequency) on grids that span several 120 x 16 tiles
with ragged right and bottom edges, and with each other.
"""
import numpy as np
import pytest

from gpu_util import ensure_lib, log_record, make_solver, oracle_ops, precond_err, precond_tol, to_dev, torch_cuda
from oracle import precond
from paper_2506_03947_gb300 import inputs

pytestmark = pytest.mark.gpu

# (n0, n1, ell): n0 % 4 == 0 keeps the fused path; tiles are 120 x 16 interior cells
GRIDS = [
    (260, 70, 10),   # 3 x 5 tiles, ragged both ways
    (128, 33, 4),    # two tile columns, one 8-column tail
    (376, 17, 16),   # 4 x 2 tiles, one-row tail
    (120, 16, 6),    # exactly one tile
    (64, 64, 8),     # narrower than a tile
]


def _problem(n0, n1, ell, seed):
    return inputs.make_problem("g%dx%d" % (n0, n1), 2, (n0, n1), ell, 1e-2, 1, 0.6, (16.0, 16.0), seed, seed + 1)


def _apply(s, r):
    torch = torch_cuda()
    rd = to_dev(r)
    zd = torch.empty_like(rd)
    s.precond_apply(rd, zd)
    return zd.cpu().numpy()


@pytest.mark.parametrize("p", [7, 12, 21])
@pytest.mark.parametrize("n0,n1,ell", GRIDS, ids=["%dx%d_l%d" % g for g in GRIDS])
def test_step_kernels_match_oracle_and_each_other(n0, n1, ell, p):
    binding = ensure_lib()
    P = _problem(n0, n1, ell, 100 + n0 + n1 + ell)
    A, mu_max = oracle_ops(P)
    r = np.random.default_rng(7).standard_normal((P.ell, P.N))
    ref = precond.pnc_apply(A, r, P.alpha, 1.0, mu_max, p)
    s = make_solver(P, 1, p)
    assert s.step_kernel() == binding.AAO_STEP_STREAM      # the default without a tune cache
    s.set_step_kernel(binding.AAO_STEP_TMA)
    assert s.step_kernel() == binding.AAO_STEP_TMA
    z_tma = _apply(s, r)
    s.set_step_kernel(binding.AAO_STEP_TILE)
    assert s.step_kernel() == binding.AAO_STEP_TILE
    z_tile = _apply(s, r)
    tol = precond_tol(1, p)
    e_tma = precond_err(z_tma, ref, P.ell, P.alpha)
    e_tile = precond_err(z_tile, ref, P.ell, P.alpha)
    e_pair = precond_err(z_tma, z_tile, P.ell, P.alpha)
    s.set_step_kernel(binding.AAO_STEP_STREAM)
    assert s.step_kernel() == binding.AAO_STEP_STREAM
    z_str = _apply(s, r)
    e_str = precond_err(z_str, ref, P.ell, P.alpha)
    e_str_pair = precond_err(z_str, z_tma, P.ell, P.alpha)
    log_record({"test": "step_kernels", "case": "%dx%d_l%d" % (n0, n1, ell), "p": p, "err_tma": e_tma,
                "err_tile": e_tile, "err_stream": e_str, "tma_vs_tile": e_pair, "stream_vs_tma": e_str_pair,
                "bitwise": bool(np.array_equal(z_tma, z_tile)),
                "bitwise_stream": bool(np.array_equal(z_tma, z_str)), "tol": tol, "ratio": e_tma / tol})
    assert e_tma <= tol, (e_tma, tol)
    assert e_tile <= tol, (e_tile, tol)
    assert e_str <= tol, (e_str, tol)
    # same FP32 operations in the same order: at most rounding-order noise
    assert e_pair <= 64 * np.finfo(np.float32).eps, e_pair
    assert e_str_pair <= 64 * np.finfo(np.float32).eps, e_str_pair


STREAM_CONFIGS = [(4, 64, 4, 8), (4, 16, 3, 6), (4, 28, 4, 6), (4, 40, 3, 8), (4, 100, 4, 8), (4, 52, 3, 6),
                  (4, 46, 3, 12), (4, 88, 4, 12),
                  # H + 9 a multiple of 6: the skewed level schedule
                  (4, 87, 3, 8), (4, 15, 4, 8), (4, 33, 3, 8), (4, 3, 3, 8),
                  # five rows in flight (the ring slot of row t - 1 is refilled once its x_{k-1} is read)
                  (4, 87, 5, 8), (4, 88, 5, 8), (4, 15, 5, 8), (4, 3, 5, 8)]


@pytest.mark.parametrize("cfg", STREAM_CONFIGS, ids=["S%d_H%d_D%d_NW%d" % c for c in STREAM_CONFIGS])
def test_stream_kernel_configurations_match_oracle(cfg):
    # every supported (H, D, NW) of the warp-strip kernel computes the same steps: segments that
    # do not divide the grid, several units per warp (ring slots reused across units)
    binding = ensure_lib()
    P = _problem(376, 130, 10, 31)
    A, mu_max = oracle_ops(P)
    r = np.random.default_rng(12).standard_normal((P.ell, P.N))
    p = 21
    ref = precond.pnc_apply(A, r, P.alpha, 1.0, mu_max, p)
    s = make_solver(P, 1, p)
    s.set_step_kernel(binding.AAO_STEP_STREAM)
    s.set_stream_config(*cfg)
    assert s.stream_config() == dict(zip(("S", "H", "D", "NW"), cfg))
    z = _apply(s, r)
    err = precond_err(z, ref, P.ell, P.alpha)
    tol = precond_tol(1, p)
    log_record({"test": "stream_configs", "cfg": list(cfg), "err": err, "tol": tol, "ratio": err / tol})
    assert err <= tol, (err, tol)


def test_stream_config_rules():
    binding = ensure_lib()
    P = _problem(64, 64, 8, 9)
    s = make_solver(P, 1, 9)
    # H + 8 and H + 9 both off a multiple of 6; the skewed schedule (H + 9) at 6 or 12 warps
    for bad in ((4, 62, 4, 8), (4, 24, 4, 8), (2, 64, 4, 8), (4, 64, 6, 8), (4, 64, 4, 9), (4, 0, 3, 8),
                (4, 63, 4, 12), (4, 63, 3, 6), (4, 64, 5, 12), (2, 62, 5, 8)):
        with pytest.raises(binding.AaoError):
            s.set_stream_config(*bad)
    s64 = make_solver(P, 0, 9)
    with pytest.raises(binding.AaoError):
        s64.set_step_kernel(binding.AAO_STEP_STREAM)


def test_tma_kernel_is_deterministic_and_repeatable():
    P = _problem(260, 70, 10, 5)
    r = np.random.default_rng(8).standard_normal((P.ell, P.N))
    s = make_solver(P, 1, 20)
    z1 = _apply(s, r)
    z2 = _apply(s, r)
    np.testing.assert_array_equal(z1, z2)


def test_step_kernel_selection_rules():
    binding = ensure_lib()
    P2 = _problem(64, 64, 8, 9)
    s64 = make_solver(P2, 0, 9)             # FP64: no fused path
    assert s64.step_kernel() == binding.AAO_STEP_AUTO
    with pytest.raises(binding.AaoError):
        s64.set_step_kernel(binding.AAO_STEP_TMA)
    with pytest.raises(binding.AaoError):
        s64.set_step_kernel(binding.AAO_STEP_TILE)
    P3 = inputs.make_problem("odd", 2, (30, 12), 6, 1e-2, 1, 0.5, (8.0, 8.0), 3, 4)   # n0 % 4 != 0
    s_odd = make_solver(P3, 1, 9)
    assert s_odd.step_kernel() == binding.AAO_STEP_AUTO
    with pytest.raises(binding.AaoError):
        s_odd.set_step_kernel(binding.AAO_STEP_TMA)
    sm = make_solver(P2, 1, 9)
    with pytest.raises(binding.AaoError):
        sm.set_step_kernel(7)
    sm.set_step_kernel(binding.AAO_STEP_TILE)
    sm.set_step_kernel(binding.AAO_STEP_AUTO)
    assert sm.step_kernel() == binding.AAO_STEP_STREAM


def test_full_solve_with_either_kernel_agrees():
    # whole FGMRES solve (Section 5) with each kernel: same iterations, same solution to solver tolerance
    torch = torch_cuda()
    binding = ensure_lib()
    P = _problem(260, 70, 10, 11)
    b = to_dev(P.b)
    out = {}
    for kind in (binding.AAO_STEP_TMA, binding.AAO_STEP_TILE, binding.AAO_STEP_STREAM):
        s = make_solver(P, 1, 20)
        s.set_step_kernel(kind)
        x = torch.zeros_like(b)
        s.solve(b, x, 1e-8, 60)
        out[kind] = (x.cpu().numpy(), s.stats()["outer_its"])
    xa, ia = out[binding.AAO_STEP_TMA]
    xb, ib = out[binding.AAO_STEP_TILE]
    xc, ic = out[binding.AAO_STEP_STREAM]
    assert ia == ib == ic
    assert np.abs(xa - xb).max() / np.abs(xb).max() < 1e-7
    assert np.abs(xc - xb).max() / np.abs(xb).max() < 1e-7


def test_expired_tma_wait_reports_timeout_and_handle_recovers():
    # fault injection without a GPU fault: a zero wait limit makes the persistent kernel's
    # first wait on its copies expire; it lets the copies land, records the expiry and
    # returns; the call reports AAO_ETIMEOUT, and with the default limit the same handle
    # again produces the reference result
    binding = ensure_lib()
    P = _problem(260, 70, 10, 13)
    r = np.random.default_rng(9).standard_normal((P.ell, P.N))
    s = make_solver(P, 1, 20)
    s.set_step_kernel(binding.AAO_STEP_TMA)
    z_ref = _apply(s, r)
    s.set_wait_limit(0)
    with pytest.raises(binding.AaoError) as ei:
        _apply(s, r)
    assert ei.value.status == binding.AAO_ETIMEOUT
    s.set_wait_limit(binding.DEFAULT_WAIT_CYCLES)
    np.testing.assert_array_equal(_apply(s, r), z_ref)
    with pytest.raises(binding.AaoError):
        s.set_wait_limit(-1)
