"""Helpers for the GPU parity tests: build/load the CUDA library, make solvers,
wrap the oracle for a Problem, and compute derived tolerances."""
import json
import os

import numpy as np

U64 = float(np.finfo(np.float64).eps) / 2     # unit roundoff, FP64
U32 = float(np.finfo(np.float32).eps) / 2     # unit roundoff, FP32


def torch_cuda():
    import torch
    if not torch.cuda.is_available():
        import pytest
        pytest.skip("no CUDA device")
    return torch


def ensure_lib():
    from paper_2506_03947_gb300 import build
    build.build()
    from paper_2506_03947_gb300 import binding
    binding.load_library()
    return binding


def faces_or_none(a):
    return a.ravel() if a.size else None


def make_solver(P, prec, p, restart=64, mu_max_override=0.0, device_faces=True, orth=None):
    torch = torch_cuda()
    binding = ensure_lib()
    fk = []
    for a in (P.kx, P.ky, P.kz):
        if a.size == 0:
            fk.append(None)
        elif device_faces:
            fk.append(torch.from_numpy(np.ascontiguousarray(a.ravel())).cuda())
        else:
            fk.append(np.ascontiguousarray(a.ravel()))
    s = binding.Solver(P.dim, P.n, fk[0], fk[1], fk[2], P.ell, P.alpha, prec=prec, inner_its=p,
                       restart=restart, mu_max_override=mu_max_override, orth=orth,
                       stream=torch.cuda.current_stream().cuda_stream)
    s._faces = fk   # keep device copies alive
    return s


def to_dev(a):
    torch = torch_cuda()
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def oracle_ops(P):
    from oracle import allatonce, operator, precond
    from oracle.solve import make_block_op
    A = make_block_op(P.kx, P.ky, P.kz, P.shape)
    mu_max = operator.gershgorin_mu_max(P.kx, P.ky, P.kz, P.shape)
    return A, mu_max


def precond_tol(prec, p, ell=None, alpha=None):
    """Bound on the error of one preconditioner apply as measured by precond_err.

    Rounding model: a Chebyshev step forms A x_k from differences of
    neighbours (relative error about mu_max u) but multiplies that residual by
    g_k = 2 rho_k / delta, about 2/mu_max, so each step adds an error of a few
    units of roundoff relative to |x|; the forward and inverse transforms add a
    few more.  These are many independent roundings, so their sum grows like
    the square root of their number with high probability (probabilistic
    rounding error analysis, Higham and Mary, SIAM J. Sci. Comput. 2019),
    not like their count: after p steps and the two transforms,
        tol = c sqrt(p + 2) u.
    c = 8 in mixed precision, where the FP64 oracle's own rounding is far
    below FP32's; c = 32 in FP64, where the oracle rounds at the same unit as
    the kernels (the comparison sees both), with sums of up to 16 transform
    terms and seven stencil terms in 3D.  Everything up to the unscaling
    Gamma^{-1} happens on zhat_t = gamma_t z_t, so the error is measured there
    (precond_err); Gamma^{-1} is one rounded product per value.
    ``ell`` and ``alpha`` are accepted for call-site symmetry and unused.
    """
    import math
    u = U32 if prec == 1 else U64
    c = 8.0 if prec == 1 else 32.0
    return c * math.sqrt(max(p, 1) + 2) * u


def precond_err(z, ref, ell, alpha):
    """Error of z against the oracle's ref (both (ell, ...)) in the transformed
    domain: max_t max|z_t - ref_t| gamma_t / max_t max|ref_t| gamma_t, with
    gamma_t = alpha^(t/ell) the scaling of Section 2.2 (Eq. 5's Gamma).

    Block t of z is zhat_t / gamma_t, and every rounding error of the apply
    enters zhat; measuring block t after multiplying back by gamma_t gives
    each block its own Gamma^{-1} factor instead of the worst block's.
    """
    import numpy as np
    z = np.asarray(z).reshape(ell, -1)
    ref = np.asarray(ref).reshape(ell, -1)
    g = float(alpha) ** (np.arange(ell) / ell)
    num = (np.abs(z - ref).max(axis=1) * g).max()
    den = (np.abs(ref).max(axis=1) * g).max()
    return float(num / den) if den > 0 else float(num)


def log_record(rec):
    path = os.environ.get("AAO_PARITY_LOG")
    if path:
        with open(path, "a") as f:
            f.write(json.dumps(rec, default=float) + "\n")
