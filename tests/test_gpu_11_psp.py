"""P_SP on the GPU (Section 4) against the oracle: the preconditioner apply (fixed-iteration
CG on the real shifts, block-diagonally preconditioned MINRES on the saddle-point systems,
aggregation-multigrid V-cycles; 1D, 2D and 3D grids, ragged and degenerate sizes), FGMRES solves
with it, and its limit P_alpha."""
import numpy as np
import pytest

from gpu_util import ensure_lib, log_record, to_dev, torch_cuda
from oracle import allatonce, gmres, operator, precond, saddle
from oracle.solve import make_block_op
from paper_2506_03947_gb300 import inputs

pytestmark = pytest.mark.gpu


def _solver(P, prec, p):
    torch = torch_cuda()
    binding = ensure_lib()
    fk = [torch.from_numpy(np.ascontiguousarray(a.ravel())).cuda() if a.size else None for a in (P.kx, P.ky, P.kz)]
    s = binding.Solver(P.dim, P.n, fk[0], fk[1], fk[2], P.ell, P.alpha, prec=prec, inner_its=p, restart=64,
                       stream=torch.cuda.current_stream().cuda_stream)
    s._faces = fk
    return s


CASES = [
    ("1d_37_l10", lambda: inputs.make_problem("a", 1, (37,), 10, 1e-2, 1, 0.5, (8.0,), 3, 4), 6),
    ("2d_20x14_l6", lambda: inputs.make_problem("b", 2, (20, 14), 6, 1e-2, 1, 0.5, (4.0, 4.0), 5, 6), 10),
    ("2d_64x48_l10", lambda: inputs.make_problem("c", 2, (64, 48), 10, 1e-1, 1, 0.7, (8.0, 8.0), 7, 8), 4),
    ("2d_3x5_l4", lambda: inputs.make_problem("d", 2, (3, 5), 4, 0.5, 1, 0.5, (2.0, 2.0), 9, 10), 3),
    ("3d_20x14x9_l6", lambda: inputs.make_problem("e3", 3, (20, 14, 9), 6, 1e-2, 1, 0.5, (4.0, 4.0, 3.0), 15, 16), 6),
    ("3d_9x5x33_l8", lambda: inputs.make_problem("f3", 3, (9, 5, 33), 8, 1e-1, 1, 0.7, (3.0, 2.0, 6.0), 17, 18), 4),
    ("3d_2x3x2_l4", lambda: inputs.make_problem("g3", 3, (2, 3, 2), 4, 0.5, 1, 0.5, (2.0, 2.0, 2.0), 19, 20), 3),
]


@pytest.mark.parametrize("name,mk,k", CASES, ids=[c[0] for c in CASES])
def test_psp_apply_matches_oracle(name, mk, k):
    torch = torch_cuda()
    binding = ensure_lib()
    P = mk()
    r = np.random.default_rng(2).standard_normal((P.ell, P.N))
    ref = saddle.psp_apply(P.kx, P.ky, P.shape, r, P.alpha, k, P.kz)
    s = _solver(P, binding.AAO_FP64, k)
    s.set_precond_mode(binding.AAO_PRECOND_SP)
    rd = to_dev(r)
    zd = torch.empty_like(rd)
    s.precond_apply(rd, zd)
    err = np.abs(zd.cpu().numpy() - ref).max() / np.abs(ref).max()
    log_record({"test": "psp_apply", "case": name, "k": k, "err": err})
    assert err < 1e-9, err


def test_psp_solve_matches_oracle():
    torch = torch_cuda()
    binding = ensure_lib()
    P = inputs.make_problem("e", 2, (32, 24), 10, 1e-2, 1, 0.5, (8.0, 8.0), 11, 12)
    k = 8
    A = make_block_op(P.kx, P.ky, P.kz, P.shape)
    ref = gmres.fgmres(lambda v: allatonce.aao_apply(A, v),
                       lambda r: saddle.psp_apply(P.kx, P.ky, P.shape, r, P.alpha, k), P.b, 1e-8, 64)
    s = _solver(P, binding.AAO_FP64, k)
    s.set_precond_mode(binding.AAO_PRECOND_SP)
    bd = to_dev(P.b)
    xd = torch.zeros_like(bd)
    s.solve(bd, xd, 1e-8, 64)
    st = s.stats()
    err = np.linalg.norm(xd.cpu().numpy() - ref.x) / np.linalg.norm(ref.x)
    log_record({"test": "psp_solve", "its": st["outer_its"], "its_oracle": ref.outer_its, "err": err})
    assert st["converged"] and st["outer_its"] == ref.outer_its
    assert err < 1e-7
    assert st["a_matvecs"] == st["outer_its"] * (P.ell + P.ell * k) + st["cycles"] * P.ell


def test_psp_tends_to_exact_palpha():
    torch = torch_cuda()
    binding = ensure_lib()
    P = inputs.make_problem("f", 2, (12, 10), 6, 1e-2, 1, 0.5, (4.0, 4.0), 13, 14)
    Ad = operator.fv_dense(P.kx, P.ky, P.kz, P.shape)
    r = np.random.default_rng(3).standard_normal((P.ell, P.N))
    ze = precond.palpha_exact_apply(Ad, r, P.alpha)
    s = _solver(P, binding.AAO_FP64, 60)
    s.set_precond_mode(binding.AAO_PRECOND_SP)
    rd = to_dev(r)
    zd = torch.empty_like(rd)
    s.precond_apply(rd, zd)
    assert np.abs(zd.cpu().numpy() - ze).max() < 1e-8 * np.abs(ze).max()


def test_psp_solve_3d_matches_oracle():
    torch = torch_cuda()
    binding = ensure_lib()
    P = inputs.make_problem("h3", 3, (16, 12, 10), 8, 1e-2, 1, 0.5, (4.0, 4.0, 3.0), 21, 22)
    k = 6
    A = make_block_op(P.kx, P.ky, P.kz, P.shape)
    ref = gmres.fgmres(lambda v: allatonce.aao_apply(A, v),
                       lambda r: saddle.psp_apply(P.kx, P.ky, P.shape, r, P.alpha, k, P.kz), P.b, 1e-8, 64)
    s = _solver(P, binding.AAO_FP64, k)
    s.set_precond_mode(binding.AAO_PRECOND_SP)
    bd = to_dev(P.b)
    xd = torch.zeros_like(bd)
    s.solve(bd, xd, 1e-8, 64)
    st = s.stats()
    err = np.linalg.norm(xd.cpu().numpy() - ref.x) / np.linalg.norm(ref.x)
    log_record({"test": "psp_solve_3d", "its": st["outer_its"], "its_oracle": ref.outer_its, "err": err})
    assert st["converged"] and st["outer_its"] == ref.outer_its
    assert err < 1e-7


def test_psp_mode_rules():
    binding = ensure_lib()
    P = inputs.make_problem("g", 2, (16, 12), 6, 1e-2, 1, 0.5, (4.0, 4.0), 1, 2)
    with pytest.raises(binding.AaoError):
        _solver(P, binding.AAO_MIXED, 5).set_precond_mode(binding.AAO_PRECOND_SP)
    P3 = inputs.make_problem("h", 3, (6, 5, 4), 6, 1e-2, 1, 0.5, (4.0, 4.0, 2.0), 1, 2)
    with pytest.raises(binding.AaoError) as ei:
        _solver(P3, binding.AAO_MIXED, 5).set_precond_mode(binding.AAO_PRECOND_SP)
    assert "FP64" in str(ei.value)
    _solver(P3, binding.AAO_FP64, 5).set_precond_mode(binding.AAO_PRECOND_SP)   # 3D is built
