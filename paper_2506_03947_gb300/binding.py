"""Thin ctypes binding of libaao.so (include/aao.h), same names as the C ABI.

Argument marshalling only: every step of the computation runs in the CUDA
library.  Arrays may be torch tensors (CUDA or CPU) or numpy arrays; they must
be contiguous float64.  There is no fallback: if libaao.so is missing or
cannot be loaded, every call raises.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional, Sequence

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libaao.so")

AAO_OK, AAO_EINVAL, AAO_ENOMEM, AAO_ECUDA, AAO_ENOTCONV, AAO_ENUMERIC, AAO_ETIMEOUT = 0, 1, 2, 3, 4, 5, 6
AAO_FP64, AAO_MIXED = 0, 1
AAO_MAX_ELL, AAO_MAX_RESTART, AAO_MAX_HIST = 16, 64, 512

STATUS_NAMES = {0: "AAO_OK", 1: "AAO_EINVAL", 2: "AAO_ENOMEM", 3: "AAO_ECUDA",
                4: "AAO_ENOTCONV", 5: "AAO_ENUMERIC", 6: "AAO_ETIMEOUT"}

# every symbol include/aao.h declares (checked by the CPU test suite)
EXPORTED = ("aao_default_options", "aao_create", "aao_matvec", "aao_precond_apply", "aao_solve",
            "aao_solve_fixed", "aao_get_stats", "aao_get_bounds", "aao_last_error",
            "aao_last_create_error", "aao_kernel_launch_count", "aao_destroy",
            "aao_profile_enable", "aao_profile_get", "aao_precond_apply_noalloc",
            "aao_set_inner_alloc", "aao_assign_iterations", "aao_solve_ci", "aao_batch_create",
            "aao_batch_solve", "aao_batch_get_stats", "aao_batch_last_error", "aao_batch_destroy",
            "aao_set_step_kernel", "aao_get_step_kernel", "aao_set_wait_limit", "aao_set_precond_mode",
            "aao_set_stream_config", "aao_get_stream_config", "aao_set_stream_tail", "aao_get_stream_tail",
            "aao_autotune", "aao_tune_lookup",
            "aao_set_tune_cache", "aao_get_tuning", "aao_batch_set_sweep", "aao_batch_profile_enable",
            "aao_batch_get_profile", "aao_solve_multi", "aao_multi_get_stats", "aao_multi_profile_enable",
            "aao_multi_get_profile")

# preconditioner of the outer solve (aao_set_precond_mode)
AAO_PRECOND_NC, AAO_PRECOND_EXACT_DCT, AAO_PRECOND_SP = 0, 1, 2

# default bound of the persistent kernel's device-side waits, SM clocks
DEFAULT_WAIT_CYCLES = 2000000000

# Arnoldi orthogonalisation (aao_options.orth)
AAO_ORTH_CGS, AAO_ORTH_CGS2, AAO_ORTH_MGS = 0, 1, 2

# four-step kernel selection (aao_set_step_kernel)
AAO_STEP_AUTO, AAO_STEP_TILE, AAO_STEP_TMA, AAO_STEP_STREAM = 0, 1, 2, 3

AAO_NPROF = 9
PROF_NAMES = ("dft", "step_first", "step_second", "step_mid", "step_last", "matvec", "orth", "step_pair",
              "step_quad")


class AaoError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS_NAMES.get(status, str(status)), msg))
        self.status = status


class aao_options(C.Structure):
    _fields_ = [("prec", C.c_int32), ("inner_its", C.c_int32), ("restart", C.c_int32),
                ("orth", C.c_int32), ("mu_max_override", C.c_double), ("stream", C.c_void_p)]


class aao_stats(C.Structure):
    _fields_ = [("outer_its", C.c_int32), ("cycles", C.c_int32), ("converged", C.c_int32),
                ("n_hist", C.c_int32), ("a_matvecs", C.c_int64), ("resid_est", C.c_double),
                ("resid_explicit", C.c_double), ("mu_min", C.c_double), ("mu_max", C.c_double),
                ("hist", C.c_double * AAO_MAX_HIST)]


class aao_tune_entry(C.Structure):
    _fields_ = [("kind", C.c_int32), ("S", C.c_int32), ("H", C.c_int32), ("D", C.c_int32), ("NW", C.c_int32),
                ("tail", C.c_int32), ("us_per_apply", C.c_double)]


class aao_profile(C.Structure):
    _fields_ = [("launches", C.c_int64 * AAO_NPROF), ("ms", C.c_double * AAO_NPROF),
                ("bytes", C.c_double * AAO_NPROF)]


_lib = None


def load_library(path: Optional[str] = None) -> C.CDLL:
    """Load libaao.so once; raise if it is absent (no fallback path exists)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError("libaao.so not found at %s: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`" % p)
    lib = C.CDLL(p)
    vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
    lib.aao_default_options.argtypes = [C.POINTER(aao_options)]
    lib.aao_default_options.restype = None
    lib.aao_create.argtypes = [C.POINTER(vp), i32, C.POINTER(C.c_int64), vp, vp, vp, i32, dbl,
                               C.POINTER(aao_options)]
    lib.aao_create.restype = i32
    lib.aao_matvec.argtypes = [vp, vp, vp]
    lib.aao_matvec.restype = i32
    lib.aao_precond_apply.argtypes = [vp, vp, vp]
    lib.aao_precond_apply.restype = i32
    lib.aao_solve.argtypes = [vp, vp, vp, dbl, i32, i32, i32]
    lib.aao_solve.restype = i32
    lib.aao_solve_fixed.argtypes = [vp, vp, vp, i32, i32]
    lib.aao_solve_fixed.restype = i32
    lib.aao_get_stats.argtypes = [vp, C.POINTER(aao_stats)]
    lib.aao_get_stats.restype = i32
    lib.aao_get_bounds.argtypes = [vp, C.POINTER(dbl), C.POINTER(dbl)]
    lib.aao_get_bounds.restype = i32
    lib.aao_last_error.argtypes = [vp]
    lib.aao_last_error.restype = C.c_char_p
    lib.aao_last_create_error.argtypes = []
    lib.aao_last_create_error.restype = C.c_char_p
    lib.aao_kernel_launch_count.argtypes = []
    lib.aao_kernel_launch_count.restype = i64
    lib.aao_destroy.argtypes = [vp]
    lib.aao_destroy.restype = None
    lib.aao_profile_enable.argtypes = [vp, i32]
    lib.aao_profile_enable.restype = i32
    lib.aao_profile_get.argtypes = [vp, C.POINTER(aao_profile)]
    lib.aao_profile_get.restype = i32
    lib.aao_precond_apply_noalloc.argtypes = [i32, C.POINTER(C.c_int64), vp, vp, vp, i32, dbl, i32, i32,
                                              dbl, vp, vp, vp, C.c_char_p, i32]
    lib.aao_precond_apply_noalloc.restype = i32
    lib.aao_batch_create.argtypes = [C.POINTER(vp), i32, C.POINTER(vp), i32]
    lib.aao_batch_create.restype = i32
    lib.aao_batch_solve.argtypes = [vp, C.POINTER(vp), C.POINTER(vp), dbl, i32]
    lib.aao_batch_solve.restype = i32
    lib.aao_batch_get_stats.argtypes = [vp, i32, C.POINTER(aao_stats)]
    lib.aao_batch_get_stats.restype = i32
    lib.aao_batch_last_error.argtypes = [vp]
    lib.aao_batch_last_error.restype = C.c_char_p
    lib.aao_batch_destroy.argtypes = [vp]
    lib.aao_batch_destroy.restype = None
    lib.aao_solve_ci.argtypes = [vp, vp, vp, dbl, i32, i32, i32, dbl, dbl, i32]
    lib.aao_solve_ci.restype = i32
    lib.aao_set_inner_alloc.argtypes = [vp, C.POINTER(C.c_int32), i32]
    lib.aao_set_inner_alloc.restype = i32
    lib.aao_assign_iterations.argtypes = [i32, C.c_int64, dbl, dbl, dbl, dbl, C.POINTER(C.c_int32)]
    lib.aao_assign_iterations.restype = i32
    lib.aao_set_step_kernel.argtypes = [vp, i32]
    lib.aao_set_step_kernel.restype = i32
    lib.aao_get_step_kernel.argtypes = [vp]
    lib.aao_get_step_kernel.restype = i32
    lib.aao_set_stream_config.argtypes = [vp, i32, i32, i32, i32]
    lib.aao_set_stream_config.restype = i32
    lib.aao_get_stream_config.argtypes = [vp, C.POINTER(C.c_int32)]
    lib.aao_get_stream_config.restype = i32
    lib.aao_set_stream_tail.argtypes = [vp, i32, i32, i32]
    lib.aao_set_stream_tail.restype = i32
    lib.aao_get_stream_tail.argtypes = [vp, C.POINTER(C.c_int32)]
    lib.aao_get_stream_tail.restype = i32
    lib.aao_autotune.argtypes = [vp, i32, C.POINTER(aao_tune_entry), i32, C.POINTER(i32), C.POINTER(aao_tune_entry)]
    lib.aao_autotune.restype = i32
    lib.aao_tune_lookup.argtypes = [C.c_char_p, C.c_char_p, i32, C.POINTER(C.c_int64), i32, i32, i32,
                                    C.POINTER(C.c_int32)]
    lib.aao_tune_lookup.restype = i32
    lib.aao_set_tune_cache.argtypes = [C.c_char_p]
    lib.aao_set_tune_cache.restype = i32
    lib.aao_get_tuning.argtypes = [vp, C.POINTER(C.c_int32)]
    lib.aao_get_tuning.restype = i32
    lib.aao_batch_set_sweep.argtypes = [vp, i32, i32, i32, i32, i32]
    lib.aao_batch_set_sweep.restype = i32
    lib.aao_batch_profile_enable.argtypes = [vp, i32]
    lib.aao_batch_profile_enable.restype = i32
    lib.aao_batch_get_profile.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.aao_batch_get_profile.restype = i32
    lib.aao_solve_multi.argtypes = [vp, i32, C.POINTER(vp), C.POINTER(vp), dbl, i32]
    lib.aao_solve_multi.restype = i32
    lib.aao_multi_get_stats.argtypes = [vp, i32, C.POINTER(aao_stats)]
    lib.aao_multi_get_stats.restype = i32
    lib.aao_multi_profile_enable.argtypes = [vp, i32]
    lib.aao_multi_profile_enable.restype = i32
    lib.aao_multi_get_profile.argtypes = [vp, C.POINTER(C.c_int64), C.POINTER(C.c_double), C.POINTER(C.c_double)]
    lib.aao_multi_get_profile.restype = i32
    lib.aao_set_wait_limit.argtypes = [vp, C.c_int64]
    lib.aao_set_wait_limit.restype = i32
    lib.aao_set_precond_mode.argtypes = [vp, i32]
    lib.aao_set_precond_mode.restype = i32
    _lib = lib
    return lib


def _ptr(a, n: Optional[int] = None, what: str = "array") -> int:
    """Address of a contiguous float64 torch tensor or numpy array (None -> 0).

    n: the number of float64 values the library will access through the pointer.  The C ABI
    takes plain pointers and cannot check sizes, so a shorter array is refused here, before
    any device work."""
    if a is None:
        return 0
    if hasattr(a, "data_ptr"):                       # torch.Tensor
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous():
            raise ValueError("tensors passed to libaao must be contiguous float64")
        size, addr = int(a.numel()), int(a.data_ptr())
    else:
        import numpy as np
        if not isinstance(a, np.ndarray) or a.dtype != np.float64 or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("arrays passed to libaao must be C-contiguous float64 numpy arrays")
        size, addr = int(a.size), int(a.ctypes.data)
    if n is not None and size != n:
        raise ValueError("%s: expected %d float64 values, got %d" % (what, n, size))
    return addr


def _grid(n: Sequence[int]):
    return tuple(int(v) for v in (list(n) + [1, 1, 1])[:3])


def _face_counts(dim: int, n: Sequence[int]):
    """Interior faces per axis (include/aao.h): kx n2*n1*(n0-1), ky n2*(n1-1)*n0, kz (n2-1)*n1*n0."""
    n0, n1, n2 = _grid(n)
    return (n2 * n1 * (n0 - 1), n2 * (n1 - 1) * n0 if dim >= 2 else 0, (n2 - 1) * n1 * n0 if dim == 3 else 0)


def _check(h, rc: int, ok=(AAO_OK,)) -> int:
    if rc not in ok:
        lib = load_library()
        msg = (lib.aao_last_error(h) if h else lib.aao_last_create_error()) or b""
        raise AaoError(rc, msg.decode(errors="replace"))
    return rc


def aao_default_options() -> aao_options:
    opt = aao_options()
    load_library().aao_default_options(C.byref(opt))
    return opt


def aao_create(dim: int, n: Sequence[int], kx, ky, kz, ell: int, alpha: float,
               opt: Optional[aao_options] = None):
    lib = load_library()
    h = C.c_void_p()
    n3 = (C.c_int64 * 3)(*_grid(n))
    fx, fy, fz = _face_counts(int(dim), n)
    px = _ptr(kx, fx if kx is not None else None, "kx")
    py = _ptr(ky, fy if ky is not None else None, "ky")
    pz = _ptr(kz, fz if kz is not None else None, "kz")
    rc = lib.aao_create(C.byref(h), int(dim), n3, px or None, py or None, pz or None, int(ell), float(alpha),
                        C.byref(opt) if opt is not None else None)
    _check(None, rc)
    return h


# L: ell * N, the float64 values of one block vector; None skips the size check.

def aao_matvec(h, x, y, L: Optional[int] = None) -> int:
    return _check(h, load_library().aao_matvec(h, _ptr(x, L, "x"), _ptr(y, L, "y")))


def aao_precond_apply(h, r, z, L: Optional[int] = None) -> int:
    return _check(h, load_library().aao_precond_apply(h, _ptr(r, L, "r"), _ptr(z, L, "z")))


def aao_solve(h, b, x, tol: float, max_outer: int, inner_its: int = 0, use_x0: bool = False,
              allow_notconv: bool = False, L: Optional[int] = None) -> int:
    ok = (AAO_OK, AAO_ENOTCONV) if allow_notconv else (AAO_OK,)
    return _check(h, load_library().aao_solve(h, _ptr(b, L, "b"), _ptr(x, L, "x"), float(tol), int(max_outer),
                                              int(inner_its), 1 if use_x0 else 0), ok)


def aao_solve_fixed(h, b, x, k: int, inner_its: int = 0, L: Optional[int] = None) -> int:
    return _check(h, load_library().aao_solve_fixed(h, _ptr(b, L, "b"), _ptr(x, L, "x"), int(k), int(inner_its)))


def aao_solve_ci(h, b, x, tol: float, max_outer: int, inner_its: int = 0, use_x0: bool = False,
                 l_min: float = 0.0, l_max: float = 0.0, fixed_its: int = 0, allow_notconv: bool = False,
                 L: Optional[int] = None) -> int:
    ok = (AAO_OK, AAO_ENOTCONV) if allow_notconv else (AAO_OK,)
    return _check(h, load_library().aao_solve_ci(h, _ptr(b, L, "b"), _ptr(x, L, "x"), float(tol), int(max_outer),
                                                 int(inner_its), 1 if use_x0 else 0, float(l_min), float(l_max),
                                                 int(fixed_its)),
                  ok)


def aao_get_stats(h) -> dict:
    s = aao_stats()
    _check(h, load_library().aao_get_stats(h, C.byref(s)))
    return {"outer_its": s.outer_its, "cycles": s.cycles, "converged": bool(s.converged),
            "a_matvecs": s.a_matvecs, "resid_est": s.resid_est,
            "resid_explicit": s.resid_explicit, "mu_min": s.mu_min, "mu_max": s.mu_max,
            "hist": [s.hist[i] for i in range(s.n_hist)]}


def aao_get_bounds(h):
    a, b = C.c_double(), C.c_double()
    _check(h, load_library().aao_get_bounds(h, C.byref(a), C.byref(b)))
    return a.value, b.value


def aao_last_error(h) -> str:
    return (load_library().aao_last_error(h) or b"").decode(errors="replace")


def aao_kernel_launch_count() -> int:
    return int(load_library().aao_kernel_launch_count())


def aao_profile_enable(h, on: bool) -> int:
    return _check(h, load_library().aao_profile_enable(h, 1 if on else 0))


def aao_profile_get(h) -> dict:
    p = aao_profile()
    _check(h, load_library().aao_profile_get(h, C.byref(p)))
    return {name: {"launches": int(p.launches[i]), "ms": float(p.ms[i]), "bytes": float(p.bytes[i])}
            for i, name in enumerate(PROF_NAMES)}


def aao_precond_apply_noalloc(dim: int, n: Sequence[int], kx, ky, kz, ell: int, alpha: float,
                              prec: int, inner_its: int, mu_max: float, r, z, stream=None) -> int:
    """Allocation-free, handle-free preconditioner apply (device pointers only)."""
    g = _grid(n)
    n3 = (C.c_int64 * 3)(*g)
    L = int(ell) * g[0] * g[1] * g[2]
    fx, fy, fz = _face_counts(int(dim), n)
    px = _ptr(kx, fx if kx is not None else None, "kx")
    py = _ptr(ky, fy if ky is not None else None, "ky")
    pz = _ptr(kz, fz if kz is not None else None, "kz")
    buf = C.create_string_buffer(512)
    rc = load_library().aao_precond_apply_noalloc(
        int(dim), n3, px or None, py or None, pz or None, int(ell), float(alpha),
        int(prec), int(inner_its), float(mu_max), _ptr(r, L, "r"), _ptr(z, L, "z"), stream, buf, len(buf))
    if rc != AAO_OK:
        raise AaoError(rc, buf.value.decode(errors="replace"))
    return rc


def aao_set_inner_alloc(h, p) -> int:
    arr = (C.c_int32 * len(p))(*[int(v) for v in p])
    return _check(h, load_library().aao_set_inner_alloc(h, arr, len(p)))


def aao_set_step_kernel(h, kind: int) -> int:
    return _check(h, load_library().aao_set_step_kernel(h, int(kind)))


def aao_set_precond_mode(h, mode: int) -> int:
    return _check(h, load_library().aao_set_precond_mode(h, int(mode)))


def aao_set_wait_limit(h, cycles: int) -> int:
    return _check(h, load_library().aao_set_wait_limit(h, int(cycles)))


def aao_get_step_kernel(h) -> int:
    return load_library().aao_get_step_kernel(h)


def aao_set_stream_config(h, S: int, H: int, D: int, NW: int) -> int:
    return _check(h, load_library().aao_set_stream_config(h, int(S), int(H), int(D), int(NW)))


def aao_get_stream_config(h):
    out = (C.c_int32 * 4)()
    _check(h, load_library().aao_get_stream_config(h, out))
    return {"S": out[0], "H": out[1], "D": out[2], "NW": out[3]}


def aao_set_stream_tail(h, H: int, D: int, NW: int) -> int:
    return _check(h, load_library().aao_set_stream_tail(h, int(H), int(D), int(NW)))


def aao_get_stream_tail(h):
    out = (C.c_int32 * 3)()
    _check(h, load_library().aao_get_stream_tail(h, out))
    return {"S": 2, "H": out[0], "D": out[1], "NW": out[2]}


KERNEL_NAMES = {AAO_STEP_AUTO: "auto", AAO_STEP_TILE: "tile", AAO_STEP_TMA: "tma", AAO_STEP_STREAM: "stream"}


def _tune_dict(e):
    return {"kernel": KERNEL_NAMES.get(e.kind, str(e.kind)), "S": e.S, "H": e.H, "D": e.D, "NW": e.NW,
            "tail": bool(e.tail), "us_per_apply": e.us_per_apply}


def aao_autotune(h, reps: int = 3, max_results: int = 256):
    """Time every fused-sweep candidate on the handle; returns (best, all candidates)."""
    res = (aao_tune_entry * max_results)()
    n = C.c_int32(0)
    best = aao_tune_entry()
    _check(h, load_library().aao_autotune(h, int(reps), res, int(max_results), C.byref(n), C.byref(best)))
    return _tune_dict(best), [_tune_dict(res[i]) for i in range(min(n.value, max_results))]


def aao_tune_lookup(path: str, device, dim: int, n: Sequence[int], ell: int, prec: int, p: int):
    """Host-only lookup in a tune cache: the matching entry as a dict, None, or AaoError."""
    out = (C.c_int32 * 5)()
    g = (C.c_int64 * 3)(*_grid(n))
    rc = load_library().aao_tune_lookup(path.encode(), device.encode() if device else None, int(dim), g, int(ell),
                                        int(prec), int(p), out)
    if rc < 0:
        raise AaoError(-rc, "tune cache %s cannot be read or parsed" % path)
    if rc == 0:
        return None
    return {"kernel": KERNEL_NAMES.get(out[0], str(out[0])), "S": out[1], "H": out[2], "D": out[3], "NW": out[4]}


def aao_set_tune_cache(path) -> int:
    return load_library().aao_set_tune_cache(path.encode() if path else None)


def aao_get_tuning(h):
    out = (C.c_int32 * 6)()
    _check(h, load_library().aao_get_tuning(h, out))
    return {"kernel": KERNEL_NAMES.get(out[0], str(out[0])), "S": out[1], "H": out[2], "D": out[3], "NW": out[4],
            "tuned": bool(out[5])}


def aao_assign_iterations(ell: int, nx: int, mu_max: float, mu_min: float, alpha: float, eta: float):
    out = (C.c_int32 * int(ell))()
    rc = load_library().aao_assign_iterations(int(ell), int(nx), float(mu_max), float(mu_min), float(alpha),
                                              float(eta), out)
    if rc != AAO_OK:
        raise AaoError(rc, "aao_assign_iterations: invalid arguments")
    return [int(v) for v in out]


def aao_destroy(h) -> None:
    if h:
        load_library().aao_destroy(h)


def _stats_dict(s):
    return {"outer_its": s.outer_its, "cycles": s.cycles, "converged": bool(s.converged),
            "a_matvecs": s.a_matvecs, "resid_est": s.resid_est,
            "resid_explicit": s.resid_explicit, "mu_min": s.mu_min, "mu_max": s.mu_max,
            "hist": [s.hist[i] for i in range(s.n_hist)]}


class Batch:
    """Batched solve over several Solver objects (aao_batch_*); marshalling only."""

    def __init__(self, solvers, use_graphs=True):
        lib = load_library()
        self.solvers = list(solvers)          # members must outlive the batch
        arr = (C.c_void_p * len(self.solvers))(*[s.h.value if hasattr(s.h, "value") else s.h
                                                for s in self.solvers])
        hb = C.c_void_p()
        rc = lib.aao_batch_create(C.byref(hb), len(self.solvers), arr, 1 if use_graphs else 0)
        if rc != AAO_OK:
            raise AaoError(rc, (lib.aao_last_create_error() or b"").decode(errors="replace"))
        self.hb = hb

    def solve(self, bs, xs, tol, max_outer, allow_notconv=False):
        lib = load_library()
        n = len(self.solvers)
        if len(bs) != n or len(xs) != n:
            raise ValueError("Batch.solve: need one b and one x per member (%d), got %d and %d"
                             % (n, len(bs), len(xs)))
        Ls = [s.ell * s.N for s in self.solvers]
        pb = (C.c_void_p * n)(*[_ptr(v, L, "b[%d]" % i) for i, (v, L) in enumerate(zip(bs, Ls))])
        px = (C.c_void_p * n)(*[_ptr(v, L, "x[%d]" % i) for i, (v, L) in enumerate(zip(xs, Ls))])
        rc = lib.aao_batch_solve(self.hb, pb, px, float(tol), int(max_outer))
        ok = (AAO_OK, AAO_ENOTCONV) if allow_notconv else (AAO_OK,)
        if rc not in ok:
            raise AaoError(rc, (lib.aao_batch_last_error(self.hb) or b"").decode(errors="replace"))
        return rc

    def _check(self, rc):
        if rc != AAO_OK:
            raise AaoError(rc, (load_library().aao_batch_last_error(self.hb) or b"").decode(errors="replace"))
        return rc

    def set_sweep(self, kind, S=4, H=64, D=3, NW=8):
        return self._check(load_library().aao_batch_set_sweep(self.hb, int(kind), int(S), int(H), int(D), int(NW)))

    def profile_enable(self, on=True):
        return self._check(load_library().aao_batch_profile_enable(self.hb, 1 if on else 0))

    def profile(self):
        n = C.c_int64(0)
        ms = C.c_double(0.0)
        by = C.c_double(0.0)
        self._check(load_library().aao_batch_get_profile(self.hb, C.byref(n), C.byref(ms), C.byref(by)))
        return {"launches": n.value, "ms": ms.value, "bytes": by.value}

    def stats(self, i):
        s = aao_stats()
        rc = load_library().aao_batch_get_stats(self.hb, int(i), C.byref(s))
        if rc != AAO_OK:
            raise AaoError(rc, "aao_batch_get_stats")
        return _stats_dict(s)

    def close(self):
        if getattr(self, "hb", None):
            load_library().aao_batch_destroy(self.hb)
            self.hb = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Owns one handle; methods forward to the C ABI (marshalling only)."""

    def __init__(self, dim, n, kx, ky, kz, ell, alpha, prec=AAO_MIXED, inner_its=20, restart=64,
                 orth=None, mu_max_override=0.0, stream=None):
        opt = aao_default_options()
        opt.prec = int(prec)
        opt.inner_its = int(inner_its)
        opt.restart = int(restart)
        if orth is not None:
            opt.orth = int(orth)
        opt.mu_max_override = float(mu_max_override)
        opt.stream = stream
        self.ell = int(ell)
        self.n = tuple(int(v) for v in (list(n) + [1, 1, 1])[:3])
        self.N = self.n[0] * self.n[1] * self.n[2]
        self.h = aao_create(dim, n, kx, ky, kz, ell, alpha, opt)

    @property
    def L(self) -> int:
        """Float64 values of one block vector (ell * N)."""
        return self.ell * self.N

    def matvec(self, x, y):
        return aao_matvec(self.h, x, y, self.L)

    def precond_apply(self, r, z):
        return aao_precond_apply(self.h, r, z, self.L)

    def solve(self, b, x, tol, max_outer, inner_its=0, use_x0=False, allow_notconv=False):
        return aao_solve(self.h, b, x, tol, max_outer, inner_its, use_x0, allow_notconv, self.L)

    def solve_ci(self, b, x, tol, max_outer, inner_its=0, use_x0=False, l_min=0.0, l_max=0.0, fixed_its=0,
                 allow_notconv=False):
        return aao_solve_ci(self.h, b, x, tol, max_outer, inner_its, use_x0, l_min, l_max, fixed_its,
                            allow_notconv, self.L)

    def solve_fixed(self, b, x, k, inner_its=0):
        return aao_solve_fixed(self.h, b, x, k, inner_its, self.L)

    def stats(self):
        return aao_get_stats(self.h)

    def bounds(self):
        return aao_get_bounds(self.h)

    def set_inner_alloc(self, p):
        return aao_set_inner_alloc(self.h, p)

    def set_step_kernel(self, kind):
        return aao_set_step_kernel(self.h, kind)

    def step_kernel(self):
        return aao_get_step_kernel(self.h)

    def set_stream_config(self, S=4, H=88, D=4, NW=8):
        return aao_set_stream_config(self.h, S, H, D, NW)

    def stream_config(self):
        return aao_get_stream_config(self.h)

    def set_stream_tail(self, H, D=3, NW=16):
        return aao_set_stream_tail(self.h, H, D, NW)

    def stream_tail(self):
        return aao_get_stream_tail(self.h)

    def solve_multi(self, bs, xs, tol, max_outer, allow_notconv=False):
        """Several right-hand sides of this operator in lockstep (device arrays, ell*N each)."""
        n = len(bs)
        if len(xs) != n:
            raise ValueError("solve_multi: need one x per b (%d), got %d" % (n, len(xs)))
        pb = (C.c_void_p * n)(*[_ptr(v, self.L, "b[%d]" % i) for i, v in enumerate(bs)])
        px = (C.c_void_p * n)(*[_ptr(v, self.L, "x[%d]" % i) for i, v in enumerate(xs)])
        rc = load_library().aao_solve_multi(self.h, n, pb, px, float(tol), int(max_outer))
        if rc != AAO_OK and not (allow_notconv and rc == AAO_ENOTCONV):
            _check(self.h, rc)
        return rc

    def multi_stats(self, i):
        s = aao_stats()
        _check(self.h, load_library().aao_multi_get_stats(self.h, int(i), C.byref(s)))
        return _stats_dict(s)

    def multi_profile_enable(self, on=True):
        """Event timing of the Chebyshev sweeps of solve_multi (graphs off meanwhile)."""
        _check(self.h, load_library().aao_multi_profile_enable(self.h, 1 if on else 0))

    def multi_profile(self):
        n = C.c_int64(0)
        ms = C.c_double(0.0)
        by = C.c_double(0.0)
        _check(self.h, load_library().aao_multi_get_profile(self.h, C.byref(n), C.byref(ms), C.byref(by)))
        return {"launches": n.value, "ms": ms.value, "bytes": by.value}

    def autotune(self, reps=3):
        return aao_autotune(self.h, reps)

    def tuning(self):
        return aao_get_tuning(self.h)

    def set_wait_limit(self, cycles):
        return aao_set_wait_limit(self.h, cycles)

    def set_precond_mode(self, mode):
        return aao_set_precond_mode(self.h, mode)

    def profile_enable(self, on=True):
        return aao_profile_enable(self.h, on)

    def profile(self):
        return aao_profile_get(self.h)

    def close(self):
        if self.h:
            aao_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
