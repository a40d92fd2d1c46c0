"""Parity at the full size of the 3D multi-right-hand-side workload: 128^3 cells
(N = 2,097,152), ell = 10, alpha = 1e-2, anisotropic lognormal diffusivity
(sigma 0.7, correlation lengths 8/8/4), p = 15, eight right-hand sides.

Whole-vector checks the oracle can afford at this size (the script-A matvec and
the explicit residual of each solve), and sampled preconditioner outputs: p
Chebyshev steps apply a degree p-1 polynomial in the 7-point operator A, so
z = P_NC^{-1} r at a cell depends on r only within p - 1 cells of it, and the
oracle evaluates it on a window of radius p around each sample.
"""
import numpy as np
import pytest

from gpu_util import log_record, make_solver, precond_err, precond_tol, to_dev, torch_cuda
from oracle import allatonce, operator, precond, solve
from paper_2506_03947_gb300 import inputs

pytestmark = pytest.mark.gpu

P_INNER = 15


@pytest.fixture(scope="module")
def problem():
    return inputs.config_3d()


@pytest.fixture(scope="module")
def block_op(problem):
    return solve.make_block_op(problem.kx, problem.ky, problem.kz, problem.shape)


def _window3(P, c, R):
    n0, n1, n2 = P.n
    cz, cy, cx = c
    z0, z1 = max(0, cz - R), min(n2, cz + R + 1)
    y0, y1 = max(0, cy - R), min(n1, cy + R + 1)
    x0, x1 = max(0, cx - R), min(n0, cx + R + 1)
    kx = P.kx[z0:z1, y0:y1, x0:x1 - 1]
    ky = P.ky[z0:z1, y0:y1 - 1, x0:x1]
    kz = P.kz[z0:z1 - 1, y0:y1, x0:x1]
    return (z0, z1, y0, y1, x0, x1), kx, ky, kz


def test_matvec_full_size_3d(problem, block_op):
    torch = torch_cuda()
    P = problem
    x = np.random.default_rng(1).standard_normal((P.ell, P.N))
    ref = allatonce.aao_apply(block_op, x)
    s = make_solver(P, 1, P_INNER)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    s.matvec(xd, yd)
    err = np.abs(yd.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-13


@pytest.mark.parametrize("prec", [1, 0], ids=["mixed", "fp64"])
def test_precond_sampled_full_size_3d(problem, prec):
    torch = torch_cuda()
    P = problem
    p = P_INNER
    mu_max = operator.gershgorin_mu_max(P.kx, P.ky, P.kz, P.shape)
    r = np.random.default_rng(2).standard_normal((P.ell, P.N))
    s = make_solver(P, prec, p)
    rd = to_dev(r)
    zd = torch.empty_like(rd)
    s.precond_apply(rd, zd)
    n0, n1, n2 = P.n
    z = zd.cpu().numpy().reshape(P.ell, n2, n1, n0)
    r4 = r.reshape(P.ell, n2, n1, n0)
    rng = np.random.default_rng(3)
    samples = [(0, 0, 0), (n2 - 1, n1 - 1, n0 - 1), (0, n1 // 2, n0 - 1), (n2 // 2, 0, n0 // 2)] + \
        [tuple(int(v) for v in rng.integers(0, n0, 3)) for _ in range(3)]
    tol = precond_tol(prec, p)
    worst = 0.0
    for c in samples:
        (z0, z1, y0, y1, x0, x1), kx, ky, kz = _window3(P, c, p)
        shape = (z1 - z0, y1 - y0, x1 - x0)
        rw = r4[:, z0:z1, y0:y1, x0:x1].reshape(P.ell, -1)
        Aw = solve.make_block_op(kx, ky, kz, shape)
        zw = precond.pnc_apply(Aw, rw, P.alpha, 1.0, mu_max, p).reshape(P.ell, *shape)
        ref = zw[:, c[0] - z0, c[1] - y0, c[2] - x0]
        got = z[:, c[0], c[1], c[2]]
        worst = max(worst, precond_err(got, ref, P.ell, P.alpha))
    log_record({"test": "precond_fullsize_3d", "prec": prec, "err": worst, "tol": tol, "ratio": worst / tol})
    assert worst <= tol, (worst, tol)


def test_solves_full_size_3d(problem, block_op):
    # the first and last right-hand sides, mixed path, residual certified by the oracle's
    # script-A; the FP64 GPU path on the first one: same iterations (+-2), same solution
    torch = torch_cuda()
    P = problem
    s = make_solver(P, 1, P_INNER)
    xs = {}
    for i in (0, P.b.shape[0] - 1):
        b = P.b[i]
        bd = to_dev(b)
        xd = torch.zeros_like(bd)
        s.solve(bd, xd, 1e-8, 64)
        st = s.stats()
        x = xd.cpu().numpy()
        res = np.linalg.norm(b - allatonce.aao_apply(block_op, x)) / np.linalg.norm(b)
        log_record({"test": "solve_fullsize_3d", "rhs": i, "its": st["outer_its"], "resid": res})
        assert st["converged"] and res <= 1e-8
        xs[i] = (x, st["outer_its"])
    s.close()
    s64 = make_solver(P, 0, P_INNER)
    bd = to_dev(P.b[0])
    xd = torch.zeros_like(bd)
    s64.solve(bd, xd, 1e-8, 64)
    x64, its64 = xd.cpu().numpy(), s64.stats()["outer_its"]
    x32, its32 = xs[0]
    d = np.linalg.norm(x32 - x64) / np.linalg.norm(x64)
    log_record({"test": "mixed_vs_fp64_fullsize_3d", "its32": its32, "its64": its64, "rel_diff": d})
    assert its32 <= its64 + 2
    assert d <= 1e-7


def test_multi_rhs_full_size_3d(problem, block_op):
    # the eight right-hand sides of the workload together (aao_solve_multi): every residual
    # certified by the oracle's script-A, the same iterations as a single solve (+-1), and the
    # first and last solutions equal to the single solves' to solver tolerance
    torch = torch_cuda()
    P = problem
    s = make_solver(P, 1, P_INNER)
    bs = [to_dev(P.b[i]) for i in range(P.b.shape[0])]
    xs = [torch.zeros_like(b) for b in bs]
    s.solve_multi(bs, xs, 1e-8, 64)
    its = []
    for i in range(len(bs)):
        st = s.multi_stats(i)
        x = xs[i].cpu().numpy()
        res = np.linalg.norm(P.b[i] - allatonce.aao_apply(block_op, x)) / np.linalg.norm(P.b[i])
        log_record({"test": "multi_rhs_fullsize_3d", "rhs": i, "its": st["outer_its"], "resid": res})
        assert st["converged"] and res <= 1e-8
        its.append(st["outer_its"])
    for i in (0, len(bs) - 1):
        x1 = torch.zeros_like(bs[i])
        s.solve(bs[i], x1, 1e-8, 64)
        assert abs(s.stats()["outer_its"] - its[i]) <= 1
        d = float(torch.linalg.norm(x1 - xs[i]) / torch.linalg.norm(x1))
        assert d <= 1e-7, d
    s.close()
