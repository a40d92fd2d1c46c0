"""CPU checks of the C ABI: the library builds, loads and exports what include/aao.h declares."""
import ctypes
import os
import re

import numpy as np
import pytest

from conftest import ROOT


def _declared_functions():
    src = open(os.path.join(ROOT, "include", "aao.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(aao_[a-z_0-9]+)\s*\(", src)))


@pytest.fixture(scope="module")
def lib():
    from paper_2506_03947_gb300 import build
    build.build()
    from paper_2506_03947_gb300 import binding
    return binding.load_library()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("aao_create", "aao_matvec", "aao_precond_apply", "aao_solve", "aao_get_stats",
                     "aao_last_error", "aao_destroy"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2506_03947_gb300 import binding
    names = _declared_functions()
    assert sorted(binding.EXPORTED) == names
    for n in names:
        assert hasattr(lib, n), n
        assert ctypes.cast(getattr(lib, n), ctypes.c_void_p).value


def test_default_options(lib):
    from paper_2506_03947_gb300 import binding
    o = binding.aao_default_options()
    assert (o.prec, o.inner_its, o.restart, o.orth) == (binding.AAO_MIXED, 20, 64, binding.AAO_ORTH_MGS)
    assert o.mu_max_override == 0.0


def test_invalid_arguments_are_rejected_before_any_device_work(lib):
    from paper_2506_03947_gb300 import binding
    kx = np.ones(7)
    for kwargs, frag in (({"ell": 5}, "ell"), ({"ell": 18}, "ell"), ({"alpha": 1.0}, "alpha"),
                         ({"alpha": 0.0}, "alpha"), ({"dim": 4}, "dim")):
        args = dict(dim=1, n=(8, 1, 1), kx=kx, ky=None, kz=None, ell=10, alpha=1e-2)
        args.update(kwargs)
        with pytest.raises(binding.AaoError) as ei:
            binding.aao_create(**args)
        assert ei.value.status == binding.AAO_EINVAL
        assert frag in str(ei.value)
    with pytest.raises(binding.AaoError) as ei:
        binding.aao_create(2, (4, 4, 1), np.ones(12), None, None, 10, 1e-2)
    assert "ky" in str(ei.value)
    opt = binding.aao_default_options()
    opt.orth = 7
    with pytest.raises(binding.AaoError) as ei:
        binding.aao_create(1, (8, 1, 1), kx, None, None, 10, 1e-2, opt)
    assert ei.value.status == binding.AAO_EINVAL and "orthogonalisation" in str(ei.value)


def test_no_gpu_means_loud_failure(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2506_03947_gb300 import binding
    with pytest.raises(binding.AaoError) as ei:
        binding.aao_create(1, (8, 1, 1), np.ones(7), None, None, 10, 1e-2)
    assert ei.value.status == binding.AAO_ECUDA


def test_assign_iterations_matches_oracle_and_tables(lib):
    # Algorithm 1 on the host side of the library (no device needed) against the oracle,
    # on the paper's operator (Eq. 17) settings of Tables 3 and 4
    from oracle import operator, spectral
    from paper_2506_03947_gb300 import binding
    for ell, nx, alpha, eta in ((10, 100, 1.0, 0.2), (10, 500, 0.01, 0.2), (6, 100, 1.0, 0.3), (16, 100, 0.01, 0.1)):
        mn, mx = operator.dirichlet_mu_bounds(nx, ell)
        got = binding.aao_assign_iterations(ell, nx, mx, mn, alpha, eta)
        ref = spectral.assign_iterations(ell, nx, mx, mn, alpha, eta)
        assert got == [int(v) for v in ref]
    mn, mx = operator.dirichlet_mu_bounds(100, 10)
    assert sum(binding.aao_assign_iterations(10, 100, mx, mn, 1.0, 0.2)) == 193   # Table 3: 3248 = 16 x (10 + 193)
    with pytest.raises(binding.AaoError):
        binding.aao_assign_iterations(9, 100, mx, mn, 1.0, 0.2)


def test_binding_refuses_arrays_of_the_wrong_size_before_any_library_call(lib):
    # The C ABI takes plain pointers and cannot see sizes; the binding knows ell * N and the face
    # counts, and refuses a shorter (or longer) array before the call, so no kernel ever reads
    # past a caller's buffer.
    from paper_2506_03947_gb300 import binding
    with pytest.raises(ValueError, match="kx: expected 7"):
        binding.aao_create(1, (8, 1, 1), np.ones(6), None, None, 10, 1e-2)
    with pytest.raises(ValueError, match="ky: expected 12"):
        binding.aao_create(2, (4, 4, 1), np.ones(12), np.ones(11), None, 10, 1e-2)
    with pytest.raises(ValueError, match="kz: expected 32"):
        binding.aao_create(3, (4, 4, 3), np.ones(36), np.ones(36), np.ones(31), 10, 1e-2)
    s = object.__new__(binding.Solver)           # a handle-less solver: only the checks run
    s.ell, s.n, s.N, s.h = 10, (8, 1, 1), 8, None
    assert s.L == 80
    for call in (lambda: s.solve(np.zeros(79), np.zeros(80), 1e-8, 10),
                 lambda: s.solve(np.zeros(80), np.zeros(81), 1e-8, 10),
                 lambda: s.matvec(np.zeros((10, 7)), np.zeros((10, 8))),
                 lambda: s.precond_apply(np.zeros((10, 8)), np.zeros((9, 8))),
                 lambda: s.solve_fixed(np.zeros(40), np.zeros(80), 3),
                 lambda: s.solve_ci(np.zeros(80), np.zeros(8), 1e-8, 10)):
        with pytest.raises(ValueError, match="expected 80 float64 values"):
            call()
    with pytest.raises(ValueError, match="r: expected 80"):
        binding.aao_precond_apply_noalloc(1, (8, 1, 1), np.ones(7), None, None, 10, 1e-2, 1, 5, 0.0,
                                          np.zeros(8), np.zeros(80))
    b = object.__new__(binding.Batch)
    b.solvers, b.hb = [s, s], None
    with pytest.raises(ValueError, match="one b and one x per member"):
        b.solve([np.zeros(80)], [np.zeros(80), np.zeros(80)], 1e-8, 10)
    with pytest.raises(ValueError, match=r"x\[1\]: expected 80"):
        b.solve([np.zeros(80)] * 2, [np.zeros(80), np.zeros(70)], 1e-8, 10)
