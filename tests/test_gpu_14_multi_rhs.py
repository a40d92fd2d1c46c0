"""Several right-hand sides of one operator solved together (aao_solve_multi).

The right-hand sides run as a batch of views of the handle that share its face coefficients;
the single Chebyshev steps load each tile's stencil once for all of them.  Each solution is
checked against the oracle's exact solution of Eq. 1 (sequential solves) and against the same
right-hand side solved alone; the second call reuses the views and reproduces the first bit for
bit.
"""
import numpy as np
import pytest

from gpu_util import ensure_lib, log_record, make_solver, to_dev, torch_cuda
from oracle import allatonce, exact, operator, solve
from paper_2506_03947_gb300 import inputs

pytestmark = pytest.mark.gpu


def _exact(P, b):
    A = operator.fv_sparse(P.kx, P.ky, P.kz, P.shape)
    return exact.sequential_solve_cg(lambda v: A @ v, b)


CASES = [
    ("3d_40x32x24_l10_p6", lambda: inputs.make_problem("m3", 3, (40, 32, 24), 10, 1e-2, 6, 0.7, (8.0, 8.0, 4.0), 71,
                                                       [72, 73, 74]), 6),
    ("2d_96x64_l8_p12", lambda: inputs.make_problem("m2", 2, (96, 64), 8, 1e-2, 12, 0.5, (16.0, 16.0), 75,
                                                    [76, 77, 78, 79]), 12),
]


@pytest.mark.parametrize("name,mk,p", CASES, ids=[c[0] for c in CASES])
def test_multi_rhs_matches_oracle_and_single_solves(name, mk, p):
    torch = torch_cuda()
    P = mk()
    s = make_solver(P, 1, p, restart=48)
    nr = P.b.shape[0]
    bs = [to_dev(P.b[i]) for i in range(nr)]
    xs = [torch.zeros_like(b) for b in bs]
    s.solve_multi(bs, xs, 1e-8, 200)
    A = solve.make_block_op(P.kx, P.ky, P.kz, P.shape)
    for i in range(nr):
        st = s.multi_stats(i)
        x = xs[i].cpu().numpy()
        res = np.linalg.norm(P.b[i] - allatonce.aao_apply(A, x)) / np.linalg.norm(P.b[i])
        xe = _exact(P, P.b[i])
        err = np.linalg.norm(x - xe) / np.linalg.norm(xe)
        x1 = torch.zeros_like(bs[i])
        s.solve(bs[i], x1, 1e-8, 200)
        its1 = s.stats()["outer_its"]
        log_record({"test": "multi_rhs", "case": name, "rhs": i, "its": st["outer_its"], "its_single": its1,
                    "resid": res, "err": err})
        assert st["converged"] and res <= 1e-8 and err <= 1e-7
        assert abs(st["outer_its"] - its1) <= 1
    # the views are reused: the same solve again gives the same bits
    xs2 = [torch.zeros_like(b) for b in bs]
    s.solve_multi(bs, xs2, 1e-8, 200)
    for a, b in zip(xs, xs2):
        assert torch.equal(a, b)
    s.close()


def test_multi_rhs_argument_checks():
    torch = torch_cuda()
    binding = ensure_lib()
    P = inputs.make_problem("a", 2, (32, 32), 6, 1e-2, 6, 0.5, (16.0, 16.0), 81, [82, 83])
    bs = [to_dev(P.b[i]) for i in range(2)]
    xs = [torch.zeros_like(b) for b in bs]
    s64 = make_solver(P, 0, 6)
    with pytest.raises(binding.AaoError):
        s64.solve_multi(bs, xs, 1e-8, 50)                  # FP64 handle
    s = make_solver(P, 1, 6)
    with pytest.raises(binding.AaoError):
        s.solve_multi(bs, [bs[0], xs[1]], 1e-8, 50)        # b and x alias
    with pytest.raises(binding.AaoError):
        s.multi_stats(0)                                   # no multi solve yet
    s.solve_multi(bs, xs, 1e-8, 50)
    assert s.multi_stats(1)["converged"]


def test_multi_rhs_profile_counts_middle_steps():
    """Event timing of the single Chebyshev steps k = 2 .. p-1 (one span of p - 2 launches per
    Arnoldi step; the last of them writes x_p for the inverse-transform launch); the profiled
    solve runs without graphs and gives the same bits."""
    torch = torch_cuda()
    P = inputs.make_problem("m3p", 3, (40, 32, 24), 10, 1e-2, 7, 0.7, (8.0, 8.0, 4.0), 91, [92, 93, 94])
    p = 7
    s = make_solver(P, 1, p, restart=48)
    nr = P.b.shape[0]
    bs = [to_dev(P.b[i]) for i in range(nr)]
    assert s.multi_profile() == {"launches": 0, "ms": 0.0, "bytes": 0.0}
    xs = [torch.zeros_like(b) for b in bs]
    s.solve_multi(bs, xs, 1e-8, 200)
    s.multi_profile_enable(True)
    xp = [torch.zeros_like(b) for b in bs]
    s.solve_multi(bs, xp, 1e-8, 200)
    prof = s.multi_profile()
    s.multi_profile_enable(False)
    its = [s.multi_stats(i)["outer_its"] for i in range(nr)]
    for a, b in zip(xs, xp):
        assert torch.equal(a, b)
    spans, rem = divmod(prof["launches"], p - 2)
    assert rem == 0 and max(its) <= spans <= sum(its)
    N, ell = P.N, P.ell
    one = sum((3.0 if k == 2 else 4.0) * 4.0 * ell * N + 12.0 * N for k in range(2, p))
    full = sum((3.0 if k == 2 else 4.0) * 4.0 * ell * N * nr + 12.0 * N for k in range(2, p))
    assert spans * one <= prof["bytes"] <= spans * full + 1.0
    assert prof["ms"] > 0.0
    log_record({"test": "multi_rhs_profile", "spans": spans, "its": its, "ms": prof["ms"],
                "gbs": prof["bytes"] / (prof["ms"] * 1e-3) / 1e9})
    s.close()
