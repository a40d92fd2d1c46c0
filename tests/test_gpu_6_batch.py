"""Batched solve (aao_batch_*): many instances with uneven grids, ell and alpha in lockstep.

Each member's result is checked against the oracle (explicit residual, exact solution) and
against the same instance solved alone; CUDA-graph replay must give the same bits as direct
launches.
"""
import numpy as np
import pytest

from gpu_util import ensure_lib, log_record, make_solver, to_dev, torch_cuda
from oracle import allatonce, exact, operator, solve
from paper_2506_03947_gb300 import inputs

pytestmark = pytest.mark.gpu


def _members():
    specs = [(32, 6, 1e-1, 0.3), (48, 8, 1e-2, 0.8), (64, 10, 1e-2, 0.5), (40, 12, 1e-1, 1.0), (96, 10, 1e-1, 0.2),
             (32, 10, 1e-2, 0.6)]
    return [inputs.make_problem("b%d" % i, 2, (n, n), ell, alpha, 12, sig, (16.0, 16.0), 100 + i, 200 + i)
            for i, (n, ell, alpha, sig) in enumerate(specs)]


def _exact(P):
    A = operator.fv_sparse(P.kx, P.ky, P.kz, P.shape)
    return exact.sequential_solve_cg(lambda v: A @ v, P.b)


def test_batch_matches_oracle_and_single_solves():
    torch = torch_cuda()
    binding = ensure_lib()
    probs = _members()
    solvers = [make_solver(P, 1, 12, restart=32) for P in probs]
    bs = [to_dev(P.b) for P in probs]
    xs = [torch.zeros_like(b) for b in bs]
    batch = binding.Batch(solvers, use_graphs=True)
    batch.solve(bs, xs, 1e-8, 200)
    xg = [x.cpu().numpy() for x in xs]
    for i, P in enumerate(probs):
        st = batch.stats(i)
        A = solve.make_block_op(P.kx, P.ky, P.kz, P.shape)
        res = np.linalg.norm(P.b - allatonce.aao_apply(A, xg[i])) / np.linalg.norm(P.b)
        xe = _exact(P)
        err = np.linalg.norm(xg[i] - xe) / np.linalg.norm(xe)
        # the same instance alone
        s1 = make_solver(P, 1, 12, restart=32)
        x1 = torch.zeros_like(bs[i])
        s1.solve(bs[i], x1, 1e-8, 200)
        its1 = s1.stats()["outer_its"]
        log_record({"test": "batch", "i": i, "n": P.n[0], "ell": P.ell, "its": st["outer_its"], "its_single": its1,
                    "resid": res, "err": err})
        assert st["converged"] and res <= 1e-8 and err <= 1e-7
        assert abs(st["outer_its"] - its1) <= 1
        assert st["a_matvecs"] == st["outer_its"] * P.ell * 13 + (st["cycles"] + 1) * P.ell
    # graph replay and direct launches give the same bits
    xs2 = [torch.zeros_like(b) for b in bs]
    batch2 = binding.Batch(solvers, use_graphs=False)
    batch2.solve(bs, xs2, 1e-8, 200)
    for a, b in zip(xs, xs2):
        assert torch.equal(a, b)
    # a second solve with the same batch (graphs reused) reproduces the first
    xs3 = [torch.zeros_like(b) for b in bs]
    batch.solve(bs, xs3, 1e-8, 200)
    for a, b in zip(xs, xs3):
        assert torch.equal(a, b)


@pytest.mark.parametrize("orth", ["mgs", "cgs2"])
def test_batch_orthogonalisation_follows_members(orth):
    # Members on modified Gram-Schmidt (the default): the batch runs one fused MGS launch per
    # basis vector over all members.  Members on CGS2: the batch runs the classical passes.
    # Either way each member converges, certified, within the tolerance of the exact solution,
    # in the iterations it takes alone (+-1: the batch sweeps one Chebyshev step per launch and
    # the single solver four, so their FP32 rounding differs).
    torch = torch_cuda()
    binding = ensure_lib()
    code = binding.AAO_ORTH_MGS if orth == "mgs" else binding.AAO_ORTH_CGS2
    probs = _members()[:4]
    bs = [to_dev(P.b) for P in probs]
    solvers = [make_solver(P, 1, 12, restart=32, orth=code) for P in probs]
    xs = [torch.zeros_like(b) for b in bs]
    batch = binding.Batch(solvers, use_graphs=True)
    batch.solve(bs, xs, 1e-8, 200)
    for i, P in enumerate(probs):
        st = batch.stats(i)
        s1 = make_solver(P, 1, 12, restart=32, orth=code)
        x1 = torch.zeros_like(bs[i])
        s1.solve(bs[i], x1, 1e-8, 200)
        its1 = s1.stats()["outer_its"]
        A = solve.make_block_op(P.kx, P.ky, P.kz, P.shape)
        xg = xs[i].cpu().numpy()
        res = np.linalg.norm(P.b - allatonce.aao_apply(A, xg)) / np.linalg.norm(P.b)
        xe = _exact(P)
        err = np.linalg.norm(xg - xe) / np.linalg.norm(xe)
        log_record({"test": "batch_orth", "orth": orth, "i": i, "its": st["outer_its"], "its_single": its1,
                    "resid": res, "err": err})
        assert st["converged"] and res <= 1e-8 and err <= 1e-7
        assert abs(st["outer_its"] - its1) <= 1


@pytest.mark.parametrize("p", [2, 3, 5, 7, 11])
def test_batch_schedules_over_p(p):
    # The batch's preconditioner schedule depends on p:
    #   p = 2: the last step at k = 1;
    #   p = 3: the last step from x_1 = bhat/theta;
    #   p = 5: single steps only;
    #   p = 7: the transform with step 1, step 2 alone, one four-step launch through the last
    #          step (x_p), the inverse transform;
    #   p = 11: the same with two four-step launches.
    # Each member must reach the oracle's exact solution, certified, in about the iterations it
    # takes alone: within 5 %, or +-1. Small p needs 45-115 iterations with restarts, and the
    # single solver runs fused pairs or four-step launches where the batch runs single steps,
    # so FP32 rounding differs.
    torch = torch_cuda()
    binding = ensure_lib()
    probs = _members()[:3]
    bs = [to_dev(P.b) for P in probs]
    solvers = [make_solver(P, 1, p, restart=64) for P in probs]
    xs = [torch.zeros_like(b) for b in bs]
    batch = binding.Batch(solvers, use_graphs=True)
    batch.solve(bs, xs, 1e-8, 200)
    for i, P in enumerate(probs):
        st = batch.stats(i)
        s1 = make_solver(P, 1, p, restart=64)
        x1 = torch.zeros_like(bs[i])
        s1.solve(bs[i], x1, 1e-8, 200)
        xe = _exact(P)
        err = np.linalg.norm(xs[i].cpu().numpy() - xe) / np.linalg.norm(xe)
        log_record({"test": "batch_p", "p": p, "i": i, "its": st["outer_its"],
                    "its_single": s1.stats()["outer_its"], "err": err})
        assert st["converged"] and err <= 1e-7
        its1 = s1.stats()["outer_its"]
        assert abs(st["outer_its"] - its1) <= max(1, its1 // 20)
        assert st["a_matvecs"] == st["outer_its"] * P.ell * (p + 1) + (st["cycles"] + 1) * P.ell


def test_batch_argument_checks():
    torch_cuda()
    binding = ensure_lib()
    P2 = inputs.config_2d(n=30)                       # n0 % 4 != 0
    with pytest.raises(binding.AaoError):
        binding.Batch([make_solver(P2, 1, 8)])
    P = inputs.config_2d(n=32)
    with pytest.raises(binding.AaoError):
        binding.Batch([make_solver(P, 1, 8), make_solver(P, 1, 9)])   # different inner_its
    with pytest.raises(binding.AaoError):
        binding.Batch([make_solver(P, 0, 8)])                         # FP64 members


def test_batch_warp_strip_queue_matches_tile_sweep():
    # The fused sweeps as one persistent warp-strip launch over all members (any ell), units taken
    # from the device queue, through the last step (a two-step final launch writes x_p, a batched
    # inverse transform follows, and the transform is fused with step 1), against the same batch
    # with the shared-memory tile kernel per ell and the last step fused with the inverse
    # transform: the same steps, in a different rounding order at both ends, so both must reach
    # the exact solution, certified, in the same number of iterations up to one (the queue is
    # reset by its last warp, so every launch of every Arnoldi step covers all units)
    torch = torch_cuda()
    binding = ensure_lib()
    probs = _members()
    solvers = [make_solver(P, 1, 12, restart=32) for P in probs]
    bs = [to_dev(P.b) for P in probs]
    out = {}
    for kind in (binding.AAO_STEP_STREAM, binding.AAO_STEP_TILE):
        xs = [torch.zeros_like(b) for b in bs]
        batch = binding.Batch(solvers, use_graphs=True)
        batch.set_sweep(kind)
        batch.solve(bs, xs, 1e-8, 200)
        out[kind] = ([x.cpu().numpy() for x in xs], [batch.stats(i)["outer_its"] for i in range(len(probs))],
                     [batch.stats(i)["converged"] for i in range(len(probs))])
        batch.close()
    (xa, ia, ca), (xb, ib, cb) = out[binding.AAO_STEP_STREAM], out[binding.AAO_STEP_TILE]
    assert all(ca) and all(cb)
    assert all(abs(a - b) <= 1 for a, b in zip(ia, ib))
    errs = []
    for P, a, b in zip(probs, xa, xb):
        xe = _exact(P)
        ea = np.linalg.norm(a - xe) / np.linalg.norm(xe)
        eb = np.linalg.norm(b - xe) / np.linalg.norm(xe)
        errs.append((ea, eb))
        assert ea <= 1e-7 and eb <= 1e-7
    diff = max(np.abs(a - b).max() / np.abs(b).max() for a, b in zip(xa, xb))
    log_record({"test": "batch_stream_vs_tile", "its": ia, "its_tile": ib, "errs": errs, "rel_diff": diff})


def test_batch_profile_reports_fused_sweeps():
    torch = torch_cuda()
    binding = ensure_lib()
    probs = _members()[:3]
    solvers = [make_solver(P, 1, 12, restart=32) for P in probs]
    bs = [to_dev(P.b) for P in probs]
    xs = [torch.zeros_like(b) for b in bs]
    batch = binding.Batch(solvers, use_graphs=True)
    batch.profile_enable(True)
    batch.solve(bs, xs, 1e-8, 200)
    prof = batch.profile()
    its = max(batch.stats(i)["outer_its"] for i in range(len(probs)))
    # three fused launches per Arnoldi step at p = 12: steps 2..5 (x_{k-1} = bhat/theta, 4 field
    # sets moved), 6..9 (5 sets) and the final two-step launch 10..11 (x_p alone: 4 sets), each
    # with two face arrays
    assert prof["launches"] == 3 * its and prof["ms"] > 0
    cells = sum(P.N * ((4 + 5 + 4) * 4.0 * P.ell + 3 * 8) for P in probs)
    assert 0 < prof["bytes"] <= its * cells * 1.01
    with pytest.raises(binding.AaoError):
        batch.set_sweep(binding.AAO_STEP_STREAM, 4, 62, 3, 8)       # H + 8 not a multiple of 6
    with pytest.raises(binding.AaoError) as ei:
        batch.set_sweep(binding.AAO_STEP_STREAM, 4, 63, 3, 8)       # the skewed schedule: single solver only
    assert "lockstep" in str(ei.value)
    with pytest.raises(binding.AaoError):
        batch.set_sweep(binding.AAO_STEP_STREAM, 4, 64, 5, 8)       # five rows in flight: single solver only
