"""The paper's outer solver (Chebyshev semi-iteration on P^{-1} script-A over Corollary 1's
interval) on the GPU against oracle/outer_ci.py."""
import numpy as np
import pytest

from gpu_util import log_record, make_solver, oracle_ops, to_dev, torch_cuda
from oracle import allatonce, exact, operator, precond, solve
from oracle.outer_ci import corollary1_interval, outer_ci
from paper_2506_03947_gb300 import inputs

pytestmark = pytest.mark.gpu


def _oracle_ci(P, p, tol, max_its, fixed=None):
    A, mu_max = oracle_ops(P)
    lo, hi = corollary1_interval(1.0, P.ell, P.alpha)
    M = lambda r: precond.pnc_apply(A, r, P.alpha, 1.0, mu_max, p)
    return outer_ci(lambda x: allatonce.aao_apply(A, x), M, P.b, lo, hi, tol, max_its, fixed_its=fixed)


@pytest.mark.parametrize("k", [1, 3, 8])
def test_fp64_fixed_iterations_match_oracle(k):
    torch = torch_cuda()
    P = inputs.config_2d(n=32)
    ref = _oracle_ci(P, 10, 1e-30, k, fixed=k)
    s = make_solver(P, 0, 10)
    bd = to_dev(P.b)
    xd = torch.zeros_like(bd)
    s.solve_ci(bd, xd, 0.5, k, fixed_its=k)
    err = np.linalg.norm(xd.cpu().numpy() - ref.x) / np.linalg.norm(ref.x)
    log_record({"test": "ci_fixed", "k": k, "err": err})
    assert err <= 1e-10
    np.testing.assert_allclose(s.stats()["hist"], ref.history, rtol=1e-7, atol=1e-14)


@pytest.mark.parametrize("alloc", [None, "nc2"])
def test_converged_fp64_and_mixed(alloc):
    torch = torch_cuda()
    from oracle import spectral
    P = inputs.config_2d(n=48)
    _, mu_max = oracle_ops(P)
    p = 10 if alloc is None else [int(v) for v in spectral.assign_iterations(P.ell, 48, mu_max, 1.0, P.alpha, 0.2)]
    ref = _oracle_ci(P, p, 1e-8, 200)
    assert ref.converged
    xe = exact.sequential_solve_cg(solve.make_block_op(P.kx, P.ky, P.kz, P.shape), P.b)
    out = {}
    for prec in (0, 1):
        s = make_solver(P, prec, 10)
        if alloc:
            s.set_inner_alloc(p)
        bd = to_dev(P.b)
        xd = torch.zeros_like(bd)
        s.solve_ci(bd, xd, 1e-8, 200)
        out[prec] = (s.stats(), xd.cpu().numpy())
    st64, x64 = out[0]
    st32, x32 = out[1]
    e64 = np.linalg.norm(x64 - ref.x) / np.linalg.norm(ref.x)
    e32 = np.linalg.norm(x32 - xe) / np.linalg.norm(xe)
    log_record({"test": "ci_converged", "alloc": str(alloc), "its_oracle": ref.its, "its64": st64["outer_its"],
                "its32": st32["outer_its"], "e64_oracle": e64, "e32_exact": e32})
    assert st64["outer_its"] == ref.its and e64 <= 1e-10
    assert st32["converged"] and st32["outer_its"] <= st64["outer_its"] + 2
    assert e32 <= 1e-7
    A = solve.make_block_op(P.kx, P.ky, P.kz, P.shape)
    assert np.linalg.norm(P.b - allatonce.aao_apply(A, x32)) / np.linalg.norm(P.b) <= 1e-8
