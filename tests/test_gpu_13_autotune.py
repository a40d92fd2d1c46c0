"""The autotuner of the fused sweep on the GPU.

Every candidate it times computes the same preconditioner: each one's z = P_NC^{-1} r (Eq. 5
with p Chebyshev steps of Eq. 7 per frequency, Lemma 2's segment) is compared with the oracle's.
The winner becomes the handle's AAO_STEP_AUTO, and a tune-cache entry is applied by aao_create.
"""
import json

import numpy as np
import pytest

from gpu_util import ensure_lib, log_record, make_solver, oracle_ops, precond_err, precond_tol, to_dev, torch_cuda
from oracle import precond
from paper_2506_03947_gb300 import inputs, tune

pytestmark = pytest.mark.gpu


def _apply(s, r):
    torch = torch_cuda()
    rd = to_dev(r)
    zd = torch.empty_like(rd)
    s.precond_apply(rd, zd)
    return zd.cpu().numpy()


def test_every_candidate_matches_the_oracle():
    binding = ensure_lib()
    P = inputs.make_problem("t", 2, (248, 180), 10, 1e-2, 1, 0.5, (16.0, 16.0), 61, 62)
    p = 16                                # steps 2 .. 15: three four-step launches and a two-step one
    A, mu_max = oracle_ops(P)
    r = np.random.default_rng(21).standard_normal((P.ell, P.N))
    ref = precond.pnc_apply(A, r, P.alpha, 1.0, mu_max, p)
    s = make_solver(P, 1, p)
    best, cands = s.autotune(2)
    sweeps = [c for c in cands if not c["tail"]]
    tails = [c for c in cands if c["tail"]]
    assert len(sweeps) >= 10 and all(c["us_per_apply"] > 0 for c in cands)
    assert best["us_per_apply"] == min(c["us_per_apply"] for c in sweeps)
    assert s.tuning()["tuned"] and s.tuning()["kernel"] == best["kernel"]
    if best["kernel"] == "stream" and best["S"] == 4:
        # the two-step final launch was tuned under the winner; the fastest is the handle's tail
        assert len(tails) >= 6 and all(c["S"] == 2 for c in tails)
        bt = min(tails, key=lambda c: c["us_per_apply"])
        assert s.stream_tail() == {"S": 2, "H": bt["H"], "D": bt["D"], "NW": bt["NW"]}
    tol = precond_tol(1, p)
    kinds = {"tile": binding.AAO_STEP_TILE, "tma": binding.AAO_STEP_TMA, "stream": binding.AAO_STEP_STREAM}
    worst = 0.0
    for c in sweeps:
        s.set_step_kernel(kinds[c["kernel"]])
        if c["kernel"] == "stream":
            s.set_stream_config(c["S"], c["H"], c["D"], c["NW"])
        err = precond_err(_apply(s, r), ref, P.ell, P.alpha)
        worst = max(worst, err)
        assert err <= tol, (c, err, tol)
    if tails:
        s.set_step_kernel(binding.AAO_STEP_STREAM)
        s.set_stream_config(best["S"], best["H"], best["D"], best["NW"])
        for c in tails:
            s.set_stream_tail(c["H"], c["D"], c["NW"])
            err = precond_err(_apply(s, r), ref, P.ell, P.alpha)
            worst = max(worst, err)
            assert err <= tol, (c, err, tol)
    log_record({"test": "autotune_candidates", "n": len(cands), "tails": len(tails), "worst_err": worst,
                "tol": tol, "ratio": worst / tol, "best": best})
    # the tuned default (AAO_STEP_AUTO) is the winner
    s.set_step_kernel(binding.AAO_STEP_AUTO)
    assert s.step_kernel() == kinds[best["kernel"]]


def test_tune_cache_is_applied_by_create(tmp_path):
    torch = torch_cuda()
    binding = ensure_lib()
    P = inputs.make_problem("t", 2, (200, 96), 8, 1e-2, 1, 0.5, (16.0, 16.0), 63, 64)
    path = str(tmp_path / "tune.json")
    dev = torch.cuda.get_device_name()
    tune.save_entry(path, tune.make_entry(dev, 2, P.n, P.ell, binding.AAO_MIXED, 9,
                                          {"kernel": "stream", "S": 2, "H": 32, "D": 4, "NW": 12,
                                           "us_per_apply": 1.0}))
    binding.aao_set_tune_cache(path)
    try:
        s = make_solver(P, 1, 9)
        t = s.tuning()
        assert t == {"kernel": "stream", "S": 2, "H": 32, "D": 4, "NW": 12, "tuned": True}
        A, mu_max = oracle_ops(P)
        r = np.random.default_rng(22).standard_normal((P.ell, P.N))
        err = precond_err(_apply(s, r), precond.pnc_apply(A, r, P.alpha, 1.0, mu_max, 9), P.ell, P.alpha)
        assert err <= precond_tol(1, 9)
        # another grid has no entry: the untuned default
        Q = inputs.make_problem("u", 2, (96, 64), 8, 1e-2, 1, 0.5, (16.0, 16.0), 65, 66)
        assert make_solver(Q, 1, 9).tuning()["tuned"] is False
    finally:
        binding.aao_set_tune_cache(None)
