"""Parity at the full benchmark size: 2D 1024 x 1024 (N = 1,048,576), ell = 10,
alpha = 1e-2, lognormal diffusivity, in the launch configuration bench.py
times (mixed precision, p = 40 and p = 10; FP64 for comparison).

Whole-vector checks the oracle can afford at this size (the script-A matvec,
the explicit residual, the exact solution by sequential CG solves), plus
sampled preconditioner outputs: z = P_NC^{-1} r at a cell depends only on r
within p - 1 cells of it (p Chebyshev steps apply a degree p-1 polynomial in
A, a nearest-neighbour stencil), so the oracle evaluates it on a window of
radius p around each sample.
"""
import numpy as np
import pytest

from gpu_util import log_record, make_solver, precond_err, precond_tol, to_dev, torch_cuda
from oracle import allatonce, exact, operator, precond, solve
from paper_2506_03947_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def problem():
    return inputs.config_2d_large()


@pytest.fixture(scope="module")
def exact_solution(problem):
    A = operator.fv_sparse(problem.kx, problem.ky, problem.kz, problem.shape)
    return exact.sequential_solve_cg(lambda v: A @ v, problem.b, tol=1e-13)


def _window(P, cy, cx, R):
    n = P.n[0]
    y0, y1 = max(0, cy - R), min(n, cy + R + 1)
    x0, x1 = max(0, cx - R), min(n, cx + R + 1)
    kx = P.kx[:, y0:y1, x0:x1 - 1]
    ky = P.ky[:, y0:y1 - 1, x0:x1]
    kz = P.kz[:, :0, :]
    return (y0, y1, x0, x1), kx, ky, kz


def test_matvec_full_size(problem):
    torch = torch_cuda()
    P = problem
    x = np.random.default_rng(1).standard_normal((P.ell, P.N))
    A = solve.make_block_op(P.kx, P.ky, P.kz, P.shape)
    ref = allatonce.aao_apply(A, x)
    s = make_solver(P, 1, 40)
    xd = to_dev(x)
    yd = torch.empty_like(xd)
    s.matvec(xd, yd)
    err = np.abs(yd.cpu().numpy() - ref).max() / np.abs(ref).max()
    assert err < 1e-13


@pytest.mark.parametrize("prec", [1, 0], ids=["mixed", "fp64"])
@pytest.mark.parametrize("p", [40, 10])
def test_precond_sampled_full_size(problem, p, prec):
    torch = torch_cuda()
    P = problem
    mu_max = operator.gershgorin_mu_max(P.kx, P.ky, P.kz, P.shape)
    r = np.random.default_rng(2).standard_normal((P.ell, P.N))
    s = make_solver(P, prec, p)
    rd = to_dev(r)
    zd = torch.empty_like(rd)
    s.precond_apply(rd, zd)
    z = zd.cpu().numpy().reshape(P.ell, P.n[1], P.n[0])
    n = P.n[0]
    rng = np.random.default_rng(3)
    samples = [(0, 0), (n - 1, n - 1), (0, n // 2), (n // 2, n - 1)] + \
        [tuple(int(v) for v in rng.integers(0, n, 2)) for _ in range(4)]
    tol = precond_tol(prec, p)
    r3 = r.reshape(P.ell, P.n[1], P.n[0])
    worst = 0.0
    for cy, cx in samples:
        (y0, y1, x0, x1), kx, ky, kz = _window(P, cy, cx, p)
        shape = (1, y1 - y0, x1 - x0)
        rw = r3[:, y0:y1, x0:x1].reshape(P.ell, -1)
        Aw = solve.make_block_op(kx, ky, kz, shape)
        zw = precond.pnc_apply(Aw, rw, P.alpha, 1.0, mu_max, p).reshape(P.ell, y1 - y0, x1 - x0)
        ref = zw[:, cy - y0, cx - x0]
        got = z[:, cy, cx]
        err = precond_err(got, ref, P.ell, P.alpha)
        worst = max(worst, err)
    log_record({"test": "precond_fullsize", "p": p, "prec": prec, "err": worst, "tol": tol, "ratio": worst / tol})
    assert worst <= tol, (worst, tol)


def test_solve_full_size_mixed_vs_fp64(problem, exact_solution):
    torch = torch_cuda()
    P = problem
    A = solve.make_block_op(P.kx, P.ky, P.kz, P.shape)
    bnorm = np.linalg.norm(P.b)
    results = {}
    for prec in (1, 0):
        for p in (40, 10):
            s = make_solver(P, prec, p)
            bd = to_dev(P.b)
            xd = torch.zeros_like(bd)
            s.solve(bd, xd, 1e-8, 64)
            st = s.stats()
            x = xd.cpu().numpy()
            res = np.linalg.norm(P.b - allatonce.aao_apply(A, x)) / bnorm
            err = np.linalg.norm(x - exact_solution) / np.linalg.norm(exact_solution)
            results[(prec, p)] = (st["outer_its"], res, err, x)
            log_record({"test": "solve_fullsize", "prec": prec, "p": p, "its": st["outer_its"],
                        "resid": res, "err_exact": err})
            s.close()
            assert st["converged"]
            assert res <= 1e-8
            assert err <= 1e-7
    for p in (40, 10):
        its32, its64 = results[(1, p)][0], results[(0, p)][0]
        assert its32 <= its64 + 2
        d = np.linalg.norm(results[(1, p)][3] - results[(0, p)][3]) / np.linalg.norm(results[(0, p)][3])
        log_record({"test": "mixed_vs_fp64_fullsize", "p": p, "rel_diff": d})
        assert d <= 1e-7
