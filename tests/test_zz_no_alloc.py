"""The allocation-free preconditioner apply (aao_precond_apply_noalloc).

For callers that cannot let the library allocate device memory (their memory
belongs to their own pool or a fixed budget on a shared GPU, or they cannot
afford the device-wide synchronisation of cudaMalloc/cudaFree), the library
offers one handle-free apply whose temporaries live in a fixed 16 MiB device
array.  This file checks, through the C ABI, that it gives the same result as
the handle-based aao_precond_apply, on two calls in a row (the second call
reuses the array with the first call's contents still in it), and that a
problem too large for the array is refused with a clear error.

It sits in a file of its own that pytest collects last, and passes both alone
in a fresh process (where its first call does the per-device set-up) and after
the other tests.
"""
import numpy as np
import pytest

from gpu_util import ensure_lib, make_solver, precond_err, precond_tol, to_dev, torch_cuda
from paper_2506_03947_gb300 import inputs

pytestmark = pytest.mark.gpu


def _faces_dev(P):
    torch = torch_cuda()
    return [torch.from_numpy(np.ascontiguousarray(a.ravel())).cuda() if a.size else None
            for a in (P.kx, P.ky, P.kz)]


@pytest.mark.parametrize("prec,p", [(1, 20), (0, 7), (1, 1), (1, 2)], ids=["mixed_p20", "fp64_p7", "mixed_p1", "mixed_p2"])
def test_noalloc_matches_handle_path_twice(prec, p):
    torch = torch_cuda()
    binding = ensure_lib()
    P = inputs.config_2d(n=96, ell=10, alpha=1e-2)
    stream = torch.cuda.current_stream().cuda_stream
    kx, ky, kz = _faces_dev(P)
    ref_solver = make_solver(P, prec, p)
    # both sides are GPU applies, each within precond_tol of the exact P_NC^{-1} r: their
    # difference is within twice that
    tol = 2.0 * precond_tol(prec, p)
    for call in range(2):
        r = to_dev(np.random.default_rng(10 + call).standard_normal((P.ell, P.N)))
        z_ref = torch.empty_like(r)
        ref_solver.precond_apply(r, z_ref)
        z = torch.full_like(r, float("nan"))
        binding.aao_precond_apply_noalloc(P.dim, P.n, kx, ky, kz, P.ell, P.alpha, prec, p, 0.0, r, z, stream)
        torch.cuda.synchronize()
        err = precond_err(z.cpu().numpy(), z_ref.cpu().numpy(), P.ell, P.alpha)
        assert err <= tol, (call, err, tol)


def test_noalloc_3d_and_1d_shapes():
    torch = torch_cuda()
    binding = ensure_lib()
    stream = torch.cuda.current_stream().cuda_stream
    for P in (inputs.make_problem("c", 3, (17, 9, 5), 6, 1e-2, 1, 0.7, (8.0, 8.0, 4.0), 1, 2),
              inputs.config_1d()):
        kx, ky, kz = _faces_dev(P)
        s = make_solver(P, 1, 9)
        r = to_dev(np.random.default_rng(3).standard_normal((P.ell, P.N)))
        z_ref = torch.empty_like(r)
        s.precond_apply(r, z_ref)
        z = torch.empty_like(r)
        binding.aao_precond_apply_noalloc(P.dim, P.n, kx, ky, kz, P.ell, P.alpha, 1, 9, 0.0, r, z, stream)
        err = precond_err(z.cpu().numpy(), z_ref.cpu().numpy(), P.ell, P.alpha)
        assert err <= 2.0 * precond_tol(1, 9)


def test_noalloc_refuses_problems_larger_than_its_array():
    torch = torch_cuda()
    binding = ensure_lib()
    P = inputs.config_2d(n=512, ell=10, alpha=1e-2)        # 262,144 cells: too large for 16 MiB
    kx, ky, kz = _faces_dev(P)
    r = to_dev(np.zeros((P.ell, P.N)))
    z = torch.empty_like(r)
    with pytest.raises(binding.AaoError) as ei:
        binding.aao_precond_apply_noalloc(P.dim, P.n, kx, ky, kz, P.ell, P.alpha, 1, 5, 0.0, r, z,
                                          torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == binding.AAO_EINVAL
    assert "scratch" in str(ei.value) and "bytes" in str(ei.value)
    # host pointers would need staging buffers: refused, not allocated.  The problem is small
    # enough for the array, so the refusal must come from the pointer check.
    Q = inputs.config_2d(n=32, ell=10, alpha=1e-2)
    qx, qy, qz = _faces_dev(Q)
    with pytest.raises(binding.AaoError) as ei:
        binding.aao_precond_apply_noalloc(Q.dim, Q.n, qx, qy, qz, Q.ell, Q.alpha, 1, 5, 0.0,
                                          np.zeros((Q.ell, Q.N)), np.zeros((Q.ell, Q.N)), None)
    assert ei.value.status == binding.AAO_EINVAL
    assert "device pointers" in str(ei.value), str(ei.value)


def test_noalloc_refuses_memory_of_another_device():
    # the kernels run on the current device; another GPU's memory is refused before any launch
    torch = torch_cuda()
    if torch.cuda.device_count() < 2:
        pytest.skip("needs two GPUs")
    binding = ensure_lib()
    Q = inputs.config_2d(n=32, ell=10, alpha=1e-2)
    kx, ky, kz = _faces_dev(Q)
    r = torch.zeros((Q.ell, Q.N), dtype=torch.float64, device="cuda:1")
    z = torch.zeros((Q.ell, Q.N), dtype=torch.float64, device="cuda:0")
    with pytest.raises(binding.AaoError) as ei:
        binding.aao_precond_apply_noalloc(Q.dim, Q.n, kx, ky, kz, Q.ell, Q.alpha, 1, 5, 0.0, r, z,
                                          torch.cuda.current_stream().cuda_stream)
    assert ei.value.status == binding.AAO_EINVAL
    assert "current device" in str(ei.value)


def test_noalloc_refuses_unaligned_buffers():
    # z is written two doubles at a time and r read one at a time: a z off a 16-byte boundary
    # or an r off an 8-byte one is refused before any launch (this entry point stages nothing)
    torch = torch_cuda()
    binding = ensure_lib()
    Q = inputs.config_2d(n=32, ell=10, alpha=1e-2)
    kx, ky, kz = _faces_dev(Q)
    L = Q.ell * Q.N
    buf = torch.zeros(L + 1, dtype=torch.float64, device="cuda")
    r = torch.zeros(L, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    with pytest.raises(binding.AaoError) as ei:
        binding.aao_precond_apply_noalloc(Q.dim, Q.n, kx, ky, kz, Q.ell, Q.alpha, 1, 5, 0.0, r, buf[1:], stream)
    assert ei.value.status == binding.AAO_EINVAL and "16-byte" in str(ei.value)
    # r at an 8-byte offset is accepted and gives the bits of the aligned call
    z0 = torch.empty(L, dtype=torch.float64, device="cuda")
    z1 = torch.empty(L, dtype=torch.float64, device="cuda")
    r.copy_(torch.from_numpy(np.random.default_rng(5).standard_normal(L)).cuda())
    buf[1:].copy_(r)
    binding.aao_precond_apply_noalloc(Q.dim, Q.n, kx, ky, kz, Q.ell, Q.alpha, 1, 5, 0.0, r, z0, stream)
    binding.aao_precond_apply_noalloc(Q.dim, Q.n, kx, ky, kz, Q.ell, Q.alpha, 1, 5, 0.0, buf[1:], z1, stream)
    torch.cuda.synchronize()
    assert torch.equal(z0, z1)

