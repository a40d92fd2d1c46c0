"""Whole-field parity of the persistent four-step kernel on grids with more tiles than SMs.

The persistent kernel gives each CTA tiles blockIdx, blockIdx + gridDim, ... .  A CTA's second
and third tile run code that a single-tile CTA never reaches: the TMA stage parity carried across
tiles, the face-coefficient boxes of the next tile issued during the current tile's second pass,
and the coefficient barrier's phase.  These grids make every CTA (or some of them) take two or
three tiles, and every output value of z = P_NC^{-1} r (Eq. 5 with p Chebyshev steps of Eq. 7 per
frequency, Lemma 2's segment) is compared with the oracle's:

* the 1024 x 1024 bench grid (423 tiles of 120 x 22 over 152 SMs: three rounds), p = 7 (one
  four-step launch whose x_{k-1} is bhat/theta) and p = 40 (that launch, then eight that read a
  stored x_{k-1});
* 1920 x 400 (16 x 19 = 304 tiles: exactly two per CTA), p = 12;
* 1204 x 500 with ell = 16 (11 x 23 = 253 tiles: some CTAs take two, the rest one; ragged right
  and bottom edges), p = 21.
"""
import numpy as np
import pytest

from gpu_util import ensure_lib, log_record, make_solver, oracle_ops, precond_err, precond_tol, to_dev, torch_cuda
from oracle import precond
from paper_2506_03947_gb300 import inputs

pytestmark = pytest.mark.gpu

TILE_X, TILE_Y = 120, 22


def _tiles(n0, n1):
    return ((n0 + TILE_X - 1) // TILE_X) * ((n1 + TILE_Y - 1) // TILE_Y)


CASES = [
    # name, builder, p
    ("bench1024_p7", lambda: inputs.config_2d_large(inner_its=7), 7),
    ("bench1024_p40", lambda: inputs.config_2d_large(inner_its=40), 40),
    ("g1920x400_l10_p12", lambda: inputs.make_problem("g1920x400", 2, (1920, 400), 10, 1e-2, 12, 0.5,
                                                      (16.0, 16.0), 51, 52), 12),
    ("g1204x500_l16_p21", lambda: inputs.make_problem("g1204x500", 2, (1204, 500), 16, 1e-2, 21, 0.8,
                                                      (16.0, 16.0), 53, 54), 21),
]


@pytest.mark.parametrize("name,mk,p", CASES, ids=[c[0] for c in CASES])
def test_persistent_kernel_whole_field_matches_oracle(name, mk, p):
    torch = torch_cuda()
    binding = ensure_lib()
    P = mk()
    A, mu_max = oracle_ops(P)
    r = np.random.default_rng(17).standard_normal((P.ell, P.N))
    ref = precond.pnc_apply(A, r, P.alpha, 1.0, mu_max, p)
    s = make_solver(P, 1, p)
    s.set_step_kernel(binding.AAO_STEP_TMA)
    assert s.step_kernel() == binding.AAO_STEP_TMA
    rd = to_dev(r)
    zd = torch.empty_like(rd)
    s.precond_apply(rd, zd)
    z = zd.cpu().numpy()
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    tiles = _tiles(P.n[0], P.n[1])
    err = precond_err(z, ref, P.ell, P.alpha)
    tol = precond_tol(1, p)
    # where the largest deviation sits (which tile, which block): a failure on a CTA's later
    # tile shows up as a concentrated error on tiles >= nsm
    dev = np.abs(z - ref).reshape(P.ell, P.n[1], P.n[0]) * (P.alpha ** (np.arange(P.ell) / P.ell))[:, None, None]
    t, y, x = np.unravel_index(int(np.argmax(dev)), dev.shape)
    tile = (y // TILE_Y) * ((P.n[0] + TILE_X - 1) // TILE_X) + x // TILE_X
    log_record({"test": "tma_rounds", "case": name, "p": p, "tiles": tiles, "sms": nsm,
                "rounds": (tiles + nsm - 1) // nsm, "err": err, "tol": tol, "ratio": err / tol,
                "argmax_block": int(t), "argmax_tile": int(tile)})
    assert tiles > nsm, (tiles, nsm)
    assert err <= tol, (err, tol, int(t), int(tile))
    # the shared-memory tile kernel computes the same steps in the same order
    s.set_step_kernel(binding.AAO_STEP_TILE)
    z2 = torch.empty_like(rd)
    s.precond_apply(rd, z2)
    e_pair = precond_err(z, z2.cpu().numpy(), P.ell, P.alpha)
    assert e_pair <= 64 * np.finfo(np.float32).eps, e_pair
    s.close()


STREAM_CASES = [
    ("bench1024_p40_lockstep", lambda: inputs.config_2d_large(inner_its=40), 40, (4, 88, 4, 8)),
    ("bench1024_p40_skewed", lambda: inputs.config_2d_large(inner_its=40), 40, (4, 87, 4, 8)),
    ("bench1024_p12_H16", lambda: inputs.config_2d_large(inner_its=12), 12, (4, 16, 3, 6)),
    ("g1204x500_l16_p21_H28", lambda: inputs.make_problem("g1204x500", 2, (1204, 500), 16, 1e-2, 21, 0.8,
                                                          (16.0, 16.0), 53, 54), 21, (4, 28, 4, 6)),
]


@pytest.mark.parametrize("name,mk,p,cfg", STREAM_CASES, ids=[c[0] for c in STREAM_CASES])
def test_stream_kernel_whole_field_matches_oracle(name, mk, p, cfg):
    # the warp-strip kernel over whole fields, with several units per warp (H = 16 on 1024^2:
    # 6080 units over 1216 warps), against the oracle element by element
    torch = torch_cuda()
    binding = ensure_lib()
    P = mk()
    A, mu_max = oracle_ops(P)
    r = np.random.default_rng(19).standard_normal((P.ell, P.N))
    ref = precond.pnc_apply(A, r, P.alpha, 1.0, mu_max, p)
    s = make_solver(P, 1, p)
    s.set_step_kernel(binding.AAO_STEP_STREAM)
    s.set_stream_config(*cfg)
    rd = to_dev(r)
    zd = torch.empty_like(rd)
    s.precond_apply(rd, zd)
    err = precond_err(zd.cpu().numpy(), ref, P.ell, P.alpha)
    tol = precond_tol(1, p)
    log_record({"test": "stream_whole_field", "case": name, "p": p, "cfg": list(cfg), "err": err, "tol": tol,
                "ratio": err / tol})
    assert err <= tol, (err, tol)
    s.close()
