"""Schedule of the warp-strip sweep: every p, the two-step final launch, the inverse transform.

The α-scaling, the forward transform and step 1 run as one launch (the transform of a one-cell
ring recomputed per block).  With the warp-strip kernel, steps 2 .. p-1 of Eq. 7 run as launches
of S steps (step 2 alone first when their count is odd, one two-step launch for a remainder of
two); the final launch writes x_p alone and a separate kernel applies Eq. 5's inverse transform
and Gamma^{-1}.  Each apply is compared with the oracle's P_NC^{-1} and with the persistent TMA
kernel (whose last step is fused with the inverse transform), for every residue of p - 2 modulo
4, with the launch count of the schedule checked, and for several two-step configurations.
"""
import numpy as np
import pytest

from gpu_util import ensure_lib, log_record, make_solver, oracle_ops, precond_err, precond_tol, to_dev, torch_cuda
from oracle import precond
from paper_2506_03947_gb300 import inputs

pytestmark = pytest.mark.gpu


def _problem(n0, n1, ell, seed):
    return inputs.make_problem("g%dx%d" % (n0, n1), 2, (n0, n1), ell, 1e-2, 1, 0.6, (16.0, 16.0), seed, seed + 1)


def _apply_counted(s, r):
    torch = torch_cuda()
    binding = ensure_lib()
    rd = to_dev(r)
    zd = torch.empty_like(rd)
    s.precond_apply(rd, zd)            # warm-up (graphs and staging)
    torch.cuda.synchronize()
    c0 = binding.aao_kernel_launch_count()
    s.precond_apply(rd, zd)
    torch.cuda.synchronize()
    return zd.cpu().numpy(), binding.aao_kernel_launch_count() - c0


def _expected_launches(p, S):
    """The transform with step 1 (one launch), [step 2 alone], the S-step launches, [the two-step
    launch], the inverse transform."""
    R = p - 2
    if R < 2:
        return None
    single = R % 2
    R -= single
    n = R // S if S == 2 else R // 4 + (1 if R % 4 == 2 else 0)
    return 1 + single + n + 1


@pytest.mark.parametrize("p", [3, 4, 5, 6, 7, 8, 9, 12, 13, 40])
def test_stream_schedule_every_p(p):
    binding = ensure_lib()
    P = _problem(260, 70, 10, 211)
    A, mu_max = oracle_ops(P)
    r = np.random.default_rng(p).standard_normal((P.ell, P.N))
    ref = precond.pnc_apply(A, r, P.alpha, 1.0, mu_max, p)
    s = make_solver(P, 1, p)
    s.set_step_kernel(binding.AAO_STEP_STREAM)
    z, nl = _apply_counted(s, r)
    s.set_step_kernel(binding.AAO_STEP_TMA)
    z_tma, _ = _apply_counted(s, r)
    tol = precond_tol(1, p)
    err = precond_err(z, ref, P.ell, P.alpha)
    pair = precond_err(z, z_tma, P.ell, P.alpha)
    exp = _expected_launches(p, 4)
    log_record({"test": "stream_schedule", "p": p, "err": err, "tol": tol, "ratio": err / tol,
                "stream_vs_tma": pair, "launches": nl, "expected": exp})
    assert err <= tol, (err, tol)
    # the fused steps are the tile kernel's operations in the same order; the last step and the
    # inverse transform differ in rounding order only
    assert pair <= 64 * np.finfo(np.float32).eps, pair
    if exp is not None:
        assert nl == exp, (nl, exp)
    else:
        assert np.array_equal(z, z_tma)    # p = 3: the same single-step kernels


TAILS = [(8, 3, 16), (14, 4, 8), (26, 3, 12), (38, 4, 16), (68, 3, 8)]


@pytest.mark.parametrize("tail", TAILS, ids=["H%d_D%d_NW%d" % t for t in TAILS])
def test_two_step_final_launch_configurations(tail):
    binding = ensure_lib()
    P = _problem(376, 130, 12, 223)
    A, mu_max = oracle_ops(P)
    r = np.random.default_rng(5).standard_normal((P.ell, P.N))
    p = 12                                # steps 2 .. 11: two four-step launches and the tail
    ref = precond.pnc_apply(A, r, P.alpha, 1.0, mu_max, p)
    s = make_solver(P, 1, p)
    s.set_step_kernel(binding.AAO_STEP_STREAM)
    s.set_stream_tail(*tail)
    assert s.stream_tail() == {"S": 2, "H": tail[0], "D": tail[1], "NW": tail[2]}
    z, nl = _apply_counted(s, r)
    err = precond_err(z, ref, P.ell, P.alpha)
    tol = precond_tol(1, p)
    log_record({"test": "stream_tail", "tail": list(tail), "err": err, "tol": tol, "ratio": err / tol})
    assert err <= tol, (err, tol)
    assert nl == _expected_launches(p, 4)


def test_two_step_sweep_and_tail_rules():
    binding = ensure_lib()
    P = _problem(200, 96, 8, 227)
    A, mu_max = oracle_ops(P)
    r = np.random.default_rng(3).standard_normal((P.ell, P.N))
    p = 9                                 # step 2 alone, then three two-step launches
    ref = precond.pnc_apply(A, r, P.alpha, 1.0, mu_max, p)
    s = make_solver(P, 1, p)
    s.set_step_kernel(binding.AAO_STEP_STREAM)
    s.set_stream_config(2, 32, 3, 12)
    z, nl = _apply_counted(s, r)
    err = precond_err(z, ref, P.ell, P.alpha)
    assert err <= precond_tol(1, p), err
    assert nl == _expected_launches(p, 2)
    for bad in ((15, 3, 16), (8, 5, 16), (8, 3, 6), (0, 3, 8), (4100, 3, 8)):
        with pytest.raises(binding.AaoError):
            s.set_stream_tail(*bad)
    assert s.stream_tail()["S"] == 2
