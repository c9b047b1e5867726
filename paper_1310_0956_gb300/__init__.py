"""Python binding of libwmgct, the GB300 library for wavelet-multigrid
preconditioned Krylov reconstruction in 2D algebraic tomography
(Cools et al., arXiv 1310.0956).

The C ABI is declared in include/wmgct.h. This module only marshals
arguments: every function below calls the C entry point of the same name,
and every step of the computation runs in the library's CUDA kernels. There is
no CPU fallback: if the shared library is missing or fails to load, the calls
raise.

`Plan` is a convenience wrapper taking torch CUDA tensors (device memory and
streams are PyTorch's; the arithmetic is the library's).
"""
from __future__ import annotations

import ctypes as C
import os
import threading

from . import _build

LIB_PATH = _build.LIB

WMG_OK = 0
WMG_NOT_CONVERGED = 1
(WMG_ERR_INVALID_ARG, WMG_ERR_OOM, WMG_ERR_CUDA, WMG_ERR_LEAF_NOT_SPD, WMG_ERR_BREAKDOWN, WMG_ERR_TIMEOUT,
 WMG_ERR_NAN, WMG_ERR_REJECTED) = range(-1, -9, -1)
STATUS_NAMES = {0: "OK", 1: "NOT_CONVERGED", -1: "INVALID_ARG", -2: "OOM", -3: "CUDA_ERROR",
                -4: "LEAF_NOT_SPD", -5: "BREAKDOWN", -6: "TIMEOUT", -7: "NAN", -8: "REJECTED"}

PREC_F64, PREC_F32, PREC_F32_BF16STORE = 0, 1, 2
CYCLE_ADDITIVE, CYCLE_HYBRID, CYCLE_SYMMETRIC, CYCLE_MULTIPLICATIVE = 0, 1, 2, 3
SOLVER_SIRT, SOLVER_CGLS, SOLVER_GMRES, SOLVER_BICGSTAB = 0, 1, 2, 3
KERNEL_STRIP, KERNEL_JOSEPH = 0, 1          # W: exact intersection lengths, or Joseph's kernel
REQ_QUEUED, REQ_RUNNING, REQ_DONE = 0, 1, 2


class WmgError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class wmg_geom(C.Structure):
    _fields_ = [("n", C.c_int32), ("m", C.c_int32), ("angles", C.c_void_p), ("D", C.c_int32),
                ("det_spacing", C.c_double), ("det_offset", C.c_double), ("kernel", C.c_int32)]


class wmg_opts(C.Structure):
    _fields_ = [("levels", C.c_int32), ("nu1", C.c_int32), ("nu2", C.c_int32),
                ("omega", C.c_double), ("lambda_", C.c_double), ("hybrid_depth", C.c_int32),
                ("cycle", C.c_int32), ("precision", C.c_int32)]


class wmg_solve_info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("status", C.c_int32), ("rel_res", C.c_double)]


class wmg_profile_stats(C.Structure):
    _fields_ = [("project_launches", C.c_int32), ("project_ms", C.c_double),
                ("project_images", C.c_double), ("backproject_launches", C.c_int32),
                ("backproject_ms", C.c_double), ("backproject_images", C.c_double),
                ("nnz_per_image", C.c_double), ("project_2h_launches", C.c_int32),
                ("project_2h_ms", C.c_double), ("project_2h_images", C.c_double)]


class wmg_server_config(C.Structure):
    _fields_ = [("hbm_budget", C.c_int64), ("state_bytes", C.c_int64), ("sino_ratio", C.c_double),
                ("max_slots", C.c_int32), ("preconditioned", C.c_int32), ("max_iter", C.c_int32),
                ("rtol", C.c_double), ("restart", C.c_int32), ("opts", wmg_opts)]


class wmg_server_counters(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("admitted", C.c_int64), ("completed", C.c_int64),
                ("rejected", C.c_int64), ("ticks", C.c_int64), ("geometry_setups", C.c_int64),
                ("geometries_evicted", C.c_int64), ("running", C.c_int32), ("queued", C.c_int32),
                ("geometries_cached", C.c_int32), ("state_bytes_capacity", C.c_int64),
                ("state_bytes_used", C.c_int64), ("geometry_bytes_capacity", C.c_int64),
                ("geometry_bytes_used", C.c_int64)]


_lock = threading.Lock()
_lib = None

_vp, _i32, _i64, _dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
_SIGNATURES = {
    "wmg_last_error": (_i32, [C.c_char_p, C.c_size_t]),
    "wmg_version": (_i32, []),
    "wmg_plan_create": (_i32, [C.POINTER(wmg_geom), C.POINTER(wmg_opts), _vp, C.POINTER(_vp)]),
    "wmg_plan_destroy": (_i32, [_vp]),
    "wmg_plan_sizes": (_i32, [_vp, C.POINTER(_i64), C.POINTER(_i64)]),
    "wmg_project": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "wmg_backproject": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "wmg_precond_apply": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "wmg_haar_analysis": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "wmg_haar_synthesis": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "wmg_leaf_inverse": (_i32, [_vp, _i64, _vp, _vp]),
    "wmg_solve": (_i32, [_vp, _i32, _i32, _i32, _vp, _vp, _i32, _dbl, _i32,
                         C.POINTER(wmg_solve_info), C.POINTER(_dbl), _vp]),
    "wmg_solve_x0": (_i32, [_vp, _i32, _i32, _i32, _vp, _vp, _vp, _i32, _dbl, _i32,
                            C.POINTER(wmg_solve_info), C.POINTER(_dbl), _vp]),
    "wmg_state_bytes": (_i32, [_vp, C.POINTER(_i64)]),
    "wmg_state_export": (_i32, [_vp, _vp, _i64, _vp]),
    "wmg_state_import": (_i32, [_vp, _vp, _i64, _vp]),
    "wmg_solve_resume": (_i32, [_vp, _i32, _vp, _vp, _i32, _dbl, C.POINTER(wmg_solve_info), C.POINTER(_dbl),
                                _vp]),
    "wmg_set_allocator": (_i32, [_vp, _vp, _vp]),
    "wmg_plan_nnz": (_i32, [_vp, C.POINTER(_i64)]),
    "wmg_launch_count": (_i64, [_i32]),
    "wmg_plan_get_tuning": (_i32, [_vp, C.POINTER(_i32), C.POINTER(_i32)]),
    "wmg_plan_set_tuning": (_i32, [_vp, _i32, _i32]),
    "wmg_profile_begin": (_i32, [_vp]),
    "wmg_profile_end": (_i32, [_vp, C.POINTER(wmg_profile_stats), _vp]),
    "wmg_project_noalloc": (_i32, [_i32, _i32, _i32, _vp, _vp, _vp]),
    "wmg_measure_peak": (_i32, [_i32, C.POINTER(_dbl), _vp]),
    "wmg_batch_create": (_i32, [C.POINTER(wmg_geom), C.POINTER(wmg_opts), _i32, _vp, C.POINTER(_vp)]),
    "wmg_batch_destroy": (_i32, [_vp]),
    "wmg_batch_sizes": (_i32, [_vp, _i32, C.POINTER(_i64), C.POINTER(_i64)]),
    "wmg_batch_solve": (_i32, [_vp, _i32, _i32, C.POINTER(_vp), C.POINTER(_vp), _i32, _dbl, _i32,
                               C.POINTER(wmg_solve_info), C.POINTER(_dbl), _vp]),
    "wmg_server_create": (_i32, [C.POINTER(wmg_server_config), _vp, C.POINTER(_vp)]),
    "wmg_server_destroy": (_i32, [_vp]),
    "wmg_server_submit": (_i32, [_vp, C.POINTER(wmg_geom), C.POINTER(wmg_opts), _vp, _vp,
                                 C.POINTER(C.c_uint64)]),
    "wmg_server_step": (_i32, [_vp, C.POINTER(_i32)]),
    "wmg_server_poll": (_i32, [_vp, C.c_uint64, C.POINTER(_i32), C.POINTER(wmg_solve_info), C.POINTER(_dbl),
                               C.POINTER(_dbl)]),
    "wmg_server_stats": (_i32, [_vp, C.POINTER(wmg_server_counters)]),
    "wmg_csr_create": (_i32, [_vp, _i32, _vp, C.POINTER(_vp)]),
    "wmg_csr_destroy": (_i32, [_vp]),
    "wmg_csr_info": (_i32, [_vp, C.POINTER(_i64), C.POINTER(_i64), C.POINTER(_i64)]),
    "wmg_csr_apply": (_i32, [_vp, _i32, _vp, _vp, _vp]),
    "wmg_server_footprint": (_i32, [_vp, C.POINTER(wmg_geom), C.POINTER(wmg_opts), C.POINTER(_i64),
                                    C.POINTER(_i64), C.POINTER(_i64)]),
}


def build(force: bool = False) -> str:
    """Compile libwmgct.so for sm_103a (nvcc) in the package's lib/ folder."""
    return _build.build(force=force)


def lib():
    """Load the shared library (building it first if it is out of date)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.build()
            handle = C.CDLL(path)
            for name, (res, args) in _SIGNATURES.items():
                fn = getattr(handle, name)
                fn.restype = res
                fn.argtypes = args
            _lib = handle
        return _lib


def exported_symbols() -> list[str]:
    return list(_SIGNATURES)


def last_error() -> str:
    buf = C.create_string_buffer(1024)
    lib().wmg_last_error(buf, len(buf))
    return buf.value.decode(errors="replace")


# per-problem outcomes a solve reports in its info entries (the problem
# ended, its last iterate in x), as opposed to errors of the call itself
PROBLEM_STATUSES = (WMG_ERR_BREAKDOWN, WMG_ERR_NAN)


def _check(rc: int, allow_not_converged: bool = False, allow=()) -> int:
    if rc in allow:
        return rc
    if rc < 0 or (rc == WMG_NOT_CONVERGED and not allow_not_converged):
        raise WmgError(rc, last_error())
    return rc


# ---- thin wrappers with the C names ----------------------------------------
def wmg_plan_create(geom: wmg_geom, opts: wmg_opts, stream=None) -> C.c_void_p:
    out = _vp()
    _check(lib().wmg_plan_create(C.byref(geom), C.byref(opts), stream, C.byref(out)))
    return out


def wmg_plan_destroy(plan) -> None:
    _check(lib().wmg_plan_destroy(plan))


def wmg_plan_sizes(plan) -> tuple[int, int]:
    N, M = _i64(), _i64()
    _check(lib().wmg_plan_sizes(plan, C.byref(N), C.byref(M)))
    return N.value, M.value


def wmg_project(plan, count, x, b, stream=None):
    _check(lib().wmg_project(plan, count, x, b, stream))


def wmg_backproject(plan, count, b, x, stream=None):
    _check(lib().wmg_backproject(plan, count, b, x, stream))


def wmg_precond_apply(plan, count, s, z, stream=None):
    _check(lib().wmg_precond_apply(plan, count, s, z, stream))


def wmg_haar_analysis(plan, count, x, c, stream=None):
    _check(lib().wmg_haar_analysis(plan, count, x, c, stream))


def wmg_haar_synthesis(plan, count, c, x, stream=None):
    _check(lib().wmg_haar_synthesis(plan, count, c, x, stream))


def wmg_leaf_inverse(plan, k, out, stream=None):
    _check(lib().wmg_leaf_inverse(plan, k, out, stream))


def wmg_solve(plan, solver, preconditioned, count, b, x, max_iter, rtol, restart, info, res_hist,
              stream=None, allow=()) -> int:
    return _check(lib().wmg_solve(plan, solver, preconditioned, count, b, x, max_iter, rtol, restart,
                                  info, res_hist, stream), allow_not_converged=True, allow=allow)


def wmg_solve_x0(plan, solver, preconditioned, count, b, x0, x, max_iter, rtol, restart, info, res_hist,
                 stream=None, allow=()) -> int:
    return _check(lib().wmg_solve_x0(plan, solver, preconditioned, count, b, x0, x, max_iter, rtol, restart,
                                     info, res_hist, stream), allow_not_converged=True, allow=allow)


def wmg_state_bytes(plan) -> int:
    n = _i64()
    _check(lib().wmg_state_bytes(plan, C.byref(n)))
    return n.value


def wmg_state_export(plan, host, nbytes, stream=None) -> None:
    _check(lib().wmg_state_export(plan, host, nbytes, stream))


def wmg_state_import(plan, host, nbytes, stream=None) -> None:
    _check(lib().wmg_state_import(plan, host, nbytes, stream))


def wmg_solve_resume(plan, count, b, x, max_iter, rtol, info, res_hist, stream=None, allow=()) -> int:
    return _check(lib().wmg_solve_resume(plan, count, b, x, max_iter, rtol, info, res_hist, stream),
                  allow_not_converged=True, allow=allow)


_ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_allocator_refs = None


def wmg_set_allocator(alloc, free, ctx=None) -> None:
    """alloc / free: ctypes callbacks of wmg_alloc_fn / wmg_free_fn (or None
    to restore cudaMalloc)."""
    _check(lib().wmg_set_allocator(C.cast(alloc, _vp) if alloc else None,
                                   C.cast(free, _vp) if free else None, ctx))


def _torch_alloc(nbytes, stream, ctx):
    try:
        import torch
        s = stream if stream else torch.cuda.current_stream().cuda_stream
        return torch.cuda.caching_allocator_alloc(int(nbytes), stream=s)
    except Exception:                      # reported to the library as out of memory
        return None


def _torch_free(ptr, nbytes, stream, ctx):
    import torch
    torch.cuda.caching_allocator_delete(ptr)


def use_torch_allocator(enable: bool = True) -> None:
    """Routes the library's later workspace allocations through torch's
    caching allocator (wmg_set_allocator): plans, batches and servers then
    hold torch memory, counted by torch.cuda.memory_allocated and reused
    from its cache. enable=False restores cudaMalloc for later allocations
    (buffers already taken go back to torch when freed)."""
    global _allocator_refs
    if enable:
        refs = (_ALLOC_FN(_torch_alloc), _FREE_FN(_torch_free))
        wmg_set_allocator(refs[0], refs[1])
        # the callbacks stay referenced for the life of the process: buffers
        # taken through them are returned through them
        _allocator_refs = (_allocator_refs or ()) + (refs,)
    else:
        wmg_set_allocator(None, None)


PEAK_FP32_FMA, PEAK_FP32_FMA2, PEAK_FP64_FMA = 0, 1, 2


def wmg_measure_peak(kind, stream=None) -> float:
    """Measured multiply-add peak of the current GPU in TFLOP/s (2 FLOP per
    multiply-add): PEAK_FP32_FMA, PEAK_FP32_FMA2 (paired FP32) or
    PEAK_FP64_FMA."""
    if stream is None:
        import torch
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    v = C.c_double()
    _check(lib().wmg_measure_peak(int(kind), C.byref(v), stream))
    return v.value


def wmg_project_noalloc(n, m, D, x, b, stream=None):
    """Forward projection b = W x without device allocation (FP32,
    equiangular geometry, unit bins; n <= 1024, m <= 4096, D <= 2048). x and
    b are contiguous float32 CUDA tensors of n*n and m*D elements; runs on
    `stream` (default: torch's current stream)."""
    import torch
    bufs = (("x", x, n * n), ("b", b, m * D))
    for name, t, size in bufs:
        if not isinstance(t, torch.Tensor):
            raise TypeError(f"{name} must be a torch tensor")
        if t.numel() != size:
            raise ValueError(f"{name} holds {t.numel()} elements, the geometry needs {size}")
    for name, t, _ in bufs:
        if not (t.is_cuda and t.dtype == torch.float32 and t.is_contiguous()):
            raise TypeError(f"{name} must be a contiguous float32 CUDA tensor")
    if stream is None:
        stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    _check(lib().wmg_project_noalloc(n, m, D, C.c_void_p(x.data_ptr()), C.c_void_p(b.data_ptr()), stream))


def wmg_batch_create(geoms, opts, stream=None) -> C.c_void_p:
    n = len(geoms)
    ga = (wmg_geom * n)(*geoms)
    oa = (wmg_opts * n)(*opts)
    out = _vp()
    _check(lib().wmg_batch_create(ga, oa, n, stream, C.byref(out)))
    return out


def wmg_batch_destroy(batch):
    _check(lib().wmg_batch_destroy(batch))


def wmg_batch_sizes(batch, i) -> tuple[int, int]:
    N, M = _i64(), _i64()
    _check(lib().wmg_batch_sizes(batch, i, C.byref(N), C.byref(M)))
    return N.value, M.value


def wmg_batch_solve(batch, solver, preconditioned, b_ptrs, x_ptrs, max_iter, rtol, restart, info, res_hist,
                    stream=None) -> int:
    n = len(b_ptrs)
    ba = (_vp * n)(*b_ptrs)
    xa = (_vp * n)(*x_ptrs)
    return _check(lib().wmg_batch_solve(batch, solver, preconditioned, ba, xa, max_iter, rtol, restart, info,
                                        res_hist, stream), allow_not_converged=True)


def wmg_plan_nnz(plan) -> int:
    v = _i64()
    _check(lib().wmg_plan_nnz(plan, C.byref(v)))
    return v.value


def wmg_plan_get_tuning(plan) -> tuple[int, int]:
    a, b = _i32(), _i32()
    _check(lib().wmg_plan_get_tuning(plan, C.byref(a), C.byref(b)))
    return a.value, b.value


def wmg_plan_set_tuning(plan, project_ctas, backproject_ctas):
    _check(lib().wmg_plan_set_tuning(plan, project_ctas, backproject_ctas))


def wmg_launch_count(reset: bool = False) -> int:
    return lib().wmg_launch_count(1 if reset else 0)


def wmg_profile_begin(plan):
    _check(lib().wmg_profile_begin(plan))


def wmg_profile_end(plan, stream=None) -> wmg_profile_stats:
    out = wmg_profile_stats()
    _check(lib().wmg_profile_end(plan, C.byref(out), stream))
    return out


def wmg_server_create(cfg: wmg_server_config, stream=None) -> C.c_void_p:
    out = _vp()
    _check(lib().wmg_server_create(C.byref(cfg), stream, C.byref(out)))
    return out


def wmg_server_destroy(srv):
    _check(lib().wmg_server_destroy(srv))


def wmg_server_submit(srv, geom: wmg_geom, opts, b, x) -> int:
    """Returns the ticket; raises WmgError (code -8) when rejected."""
    t = C.c_uint64()
    _check(lib().wmg_server_submit(srv, C.byref(geom), C.byref(opts) if opts is not None else None, b, x,
                                   C.byref(t)))
    return t.value


def wmg_server_step(srv) -> int:
    pending = _i32()
    _check(lib().wmg_server_step(srv, C.byref(pending)))
    return pending.value


def wmg_server_poll(srv, ticket, res_hist=None):
    """Returns (state, info, latency_ms)."""
    state, info, lat = _i32(), wmg_solve_info(), _dbl()
    _check(lib().wmg_server_poll(srv, ticket, C.byref(state), C.byref(info), C.byref(lat), res_hist))
    return state.value, info, lat.value


def wmg_server_stats(srv) -> wmg_server_counters:
    out = wmg_server_counters()
    _check(lib().wmg_server_stats(srv, C.byref(out)))
    return out


def wmg_server_footprint(srv, geom: wmg_geom, opts=None) -> tuple[int, int, int]:
    """(state bytes, cached geometry bytes, setup scratch bytes) of a request."""
    a, b, c = _i64(), _i64(), _i64()
    _check(lib().wmg_server_footprint(srv, C.byref(geom), C.byref(opts) if opts is not None else None,
                                      C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def wmg_csr_create(plan, transposed, stream=None):
    out = _vp()
    _check(lib().wmg_csr_create(plan, 1 if transposed else 0, stream, C.byref(out)))
    return out


def wmg_csr_destroy(csr):
    _check(lib().wmg_csr_destroy(csr))


def wmg_csr_info(csr) -> tuple[int, int, int]:
    r, c, z = _i64(), _i64(), _i64()
    _check(lib().wmg_csr_info(csr, C.byref(r), C.byref(c), C.byref(z)))
    return r.value, c.value, z.value


def wmg_csr_apply(csr, count, x, y, stream=None):
    _check(lib().wmg_csr_apply(csr, count, x, y, stream))


# ---- torch convenience wrapper ---------------------------------------------
class Plan:
    """A plan for one geometry; methods take torch CUDA tensors of the plan's
    dtype (float64 for F64 plans, float32 for F32 plans) holding `count`
    problems back to back, and run on torch's current stream."""

    def __init__(self, n, m, D, levels=3, nu1=1, nu2=1, omega=1.0, lam=0.0, hybrid_depth=2,
                 cycle=CYCLE_SYMMETRIC, precision=PREC_F64, angles=None, det_spacing=1.0,
                 det_offset=0.0, kernel=KERNEL_STRIP):
        import torch
        self._torch = torch
        self._angles = None
        ap = None
        if angles is not None:
            self._angles = (C.c_double * m)(*[float(a) for a in angles])
            ap = C.cast(self._angles, C.c_void_p)
        self.geom = wmg_geom(n, m, ap, D, det_spacing, det_offset, kernel)
        self.opts = wmg_opts(levels, nu1, nu2, omega, lam, hybrid_depth, cycle, precision)
        self.dtype = torch.float64 if precision == PREC_F64 else torch.float32
        self.n, self.m, self.D = n, m, D
        self.N, self.M = n * n, m * D
        self.K = 4 ** (levels - 1) if levels >= 1 else 0
        self.P = (n >> (levels - 1)) ** 2 if levels >= 1 else 0
        import time
        t0 = time.perf_counter()
        self.handle = wmg_plan_create(self.geom, self.opts, self._stream())
        self.setup_s = time.perf_counter() - t0          # plan creation (geometry and leaf setup) is synchronising

    def _stream(self):
        return C.c_void_p(self._torch.cuda.current_stream().cuda_stream)

    def _arg(self, t, size):
        torch = self._torch
        if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == self.dtype and t.is_contiguous()):
            raise TypeError(f"expected a contiguous CUDA tensor of dtype {self.dtype}")
        if t.numel() % size:
            raise ValueError("tensor size is not a multiple of the problem size")
        return C.c_void_p(t.data_ptr()), t.numel() // size

    def _out(self, out, size, cnt):
        """Pointer of a caller-given output holding exactly `cnt` problems."""
        p, c = self._arg(out, size)
        if c != cnt:
            raise ValueError(f"out holds {c} problems, the input {cnt}")
        return p

    def close(self):
        if getattr(self, "handle", None):
            wmg_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def project(self, x, out=None):
        xp, cnt = self._arg(x, self.N)
        out = out if out is not None else self._torch.empty(cnt * self.M, dtype=self.dtype, device=x.device)
        wmg_project(self.handle, cnt, xp, self._out(out, self.M, cnt), self._stream())
        return out

    def backproject(self, b, out=None):
        bp, cnt = self._arg(b, self.M)
        out = out if out is not None else self._torch.empty(cnt * self.N, dtype=self.dtype, device=b.device)
        wmg_backproject(self.handle, cnt, bp, self._out(out, self.N, cnt), self._stream())
        return out

    def precond(self, s, out=None):
        sp, cnt = self._arg(s, self.N)
        out = out if out is not None else self._torch.empty_like(s)
        wmg_precond_apply(self.handle, cnt, sp, self._out(out, self.N, cnt), self._stream())
        return out

    def haar_analysis(self, x, out=None):
        xp, cnt = self._arg(x, self.N)
        out = out if out is not None else self._torch.empty_like(x)
        wmg_haar_analysis(self.handle, cnt, xp, self._out(out, self.N, cnt), self._stream())
        return out

    def haar_synthesis(self, c, out=None):
        cp, cnt = self._arg(c, self.N)
        out = out if out is not None else self._torch.empty_like(c)
        wmg_haar_synthesis(self.handle, cnt, cp, self._out(out, self.N, cnt), self._stream())
        return out

    def leaf_inverse(self, k):
        out = self._torch.empty(self.P * self.P, dtype=self.dtype, device="cuda")
        wmg_leaf_inverse(self.handle, k, C.c_void_p(out.data_ptr()), self._stream())
        return out.view(self.P, self.P)

    def nnz(self) -> int:
        return wmg_plan_nnz(self.handle)

    def tuning(self, project_ctas=None, backproject_ctas=None) -> tuple[int, int]:
        """Launch shapes (CTAs per SM) of the projector / backprojector;
        sets them when both are given."""
        if project_ctas is not None and backproject_ctas is not None:
            wmg_plan_set_tuning(self.handle, project_ctas, backproject_ctas)
        return wmg_plan_get_tuning(self.handle)

    def csr(self, transposed=False):
        """The plan's W (or W^T) stored as CSR: a StoredOperator."""
        return StoredOperator(self, transposed)

    def launch_count(self, reset=False) -> int:
        """Library kernel launches since the last reset (process-wide)."""
        return wmg_launch_count(reset)

    def profile_step(self, b, out, max_iter, rtol, restart, solver=SOLVER_GMRES, preconditioned=True):
        """One solve with CUDA events around every projector / backprojector
        launch; returns per-kernel totals."""
        wmg_profile_begin(self.handle)
        self.solve(b, solver, preconditioned, max_iter, rtol, restart, out=out)
        st = wmg_profile_end(self.handle, self._stream())
        res = {"nnz_per_image": st.nnz_per_image}
        for k in ("project", "backproject", "project_2h"):
            n = getattr(st, k + "_launches")
            ms = getattr(st, k + "_ms")
            imgs = getattr(st, k + "_images")
            res[k] = {"launches": n, "total_ms": ms, "mean_ms": ms / max(n, 1),
                      "images_per_launch": imgs / max(n, 1)}
        return res

    def solve(self, b, solver=SOLVER_CGLS, preconditioned=True, max_iter=100, rtol=1e-4, restart=20,
              out=None, history=False, x0=None, problem_errors=True):
        """Returns (x, info list, residual histories or None, status). x0:
        initial guess (wmg_solve_x0), default 0. problem_errors=False
        returns a problem's breakdown or non-finite data as its info status
        (x holds its last iterate) instead of raising WmgError."""
        allow = () if problem_errors else PROBLEM_STATUSES
        bp, cnt = self._arg(b, self.M)
        out = out if out is not None else self._torch.empty(cnt * self.N, dtype=self.dtype, device=b.device)
        info = (wmg_solve_info * cnt)()
        hist = (C.c_double * (cnt * (max_iter + 1)))() if history else None
        xp = self._out(out, self.N, cnt)
        if x0 is None:
            rc = wmg_solve(self.handle, solver, 1 if preconditioned else 0, cnt, bp, xp, max_iter, rtol, restart,
                           info, hist, self._stream(), allow=allow)
        else:
            x0p, c0 = self._arg(x0, self.N)
            if c0 != cnt:
                raise ValueError("x0 must hold as many images as b has sinograms")
            rc = wmg_solve_x0(self.handle, solver, 1 if preconditioned else 0, cnt, bp, x0p, xp, max_iter, rtol,
                              restart, info, hist, self._stream(), allow=allow)
        return (out,) + self._results(cnt, max_iter, info, hist) + (rc,)

    def _results(self, cnt, max_iter, info, hist):
        infos = [(info[i].iters, info[i].status, info[i].rel_res) for i in range(cnt)]
        hists = None
        if hist is not None:
            import numpy as np
            h = np.frombuffer(hist, dtype=np.float64).reshape(cnt, max_iter + 1)
            hists = [h[i, :infos[i][0] + 1].copy() for i in range(cnt)]
        return infos, hists

    def state_export(self) -> bytes:
        """The state of the last solve (wmg_state_export) as bytes."""
        n = wmg_state_bytes(self.handle)
        buf = C.create_string_buffer(n)
        wmg_state_export(self.handle, buf, n, self._stream())
        return buf.raw

    def state_import(self, state: bytes) -> None:
        """Makes `state` (from state_export of a plan of the same geometry
        and options) this plan's solver state (wmg_state_import)."""
        buf = C.create_string_buffer(bytes(state), len(state))
        wmg_state_import(self.handle, buf, len(state), self._stream())

    def resume(self, b, max_iter, rtol=1e-4, out=None, history=False, problem_errors=True):
        """Continues the plan's solver state to max_iter iterations in total
        (wmg_solve_resume); returns as solve."""
        allow = () if problem_errors else PROBLEM_STATUSES
        bp, cnt = self._arg(b, self.M)
        out = out if out is not None else self._torch.empty(cnt * self.N, dtype=self.dtype, device=b.device)
        info = (wmg_solve_info * cnt)()
        hist = (C.c_double * (cnt * (max_iter + 1)))() if history else None
        xp = self._out(out, self.N, cnt)
        rc = wmg_solve_resume(self.handle, cnt, bp, xp, max_iter, rtol, info, hist, self._stream(), allow=allow)
        return (out,) + self._results(cnt, max_iter, info, hist) + (rc,)


class StoredOperator:
    """W or W^T of a plan assembled as CSR on the device (wmg_csr_*):
    apply(x) multiplies `count` vectors stored back to back."""

    def __init__(self, plan, transposed=False):
        self._plan = plan
        self.handle = wmg_csr_create(plan.handle, transposed, plan._stream())
        self.rows, self.cols, self.nnz = wmg_csr_info(self.handle)

    def apply(self, x, out=None):
        xp, cnt = self._plan._arg(x, self.cols)
        out = out if out is not None else self._plan._torch.empty(cnt * self.rows, dtype=x.dtype, device=x.device)
        wmg_csr_apply(self.handle, cnt, xp, self._plan._out(out, self.rows, cnt), self._plan._stream())
        return out

    def close(self):
        if getattr(self, "handle", None):
            wmg_csr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Problems of different geometries solved together (torch CUDA tensors).
    `problems` is a list of dicts with keys n, m, D and optionally levels,
    lam, angles, det_spacing, det_offset, kernel; the cycle options are
    shared."""

    def __init__(self, problems, nu1=1, nu2=1, omega=1.0, hybrid_depth=1, cycle=CYCLE_HYBRID,
                 precision=PREC_F32):
        import torch
        self._torch = torch
        self._keep = []
        geoms, opts = [], []
        for p in problems:
            ap = None
            if p.get("angles") is not None:
                arr = (C.c_double * p["m"])(*[float(a) for a in p["angles"]])
                self._keep.append(arr)
                ap = C.cast(arr, C.c_void_p)
            geoms.append(wmg_geom(p["n"], p["m"], ap, p["D"], p.get("det_spacing", 1.0), p.get("det_offset", 0.0),
                                  p.get("kernel", KERNEL_STRIP)))
            opts.append(wmg_opts(p.get("levels", 1), nu1, nu2, omega, p.get("lam", 0.0), hybrid_depth, cycle,
                                 precision))
        self.count = len(problems)
        self.dtype = torch.float64 if precision == PREC_F64 else torch.float32
        self.handle = wmg_batch_create(geoms, opts, C.c_void_p(torch.cuda.current_stream().cuda_stream))
        self.sizes = [wmg_batch_sizes(self.handle, i) for i in range(self.count)]

    def close(self):
        if getattr(self, "handle", None):
            wmg_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, bs, solver=SOLVER_GMRES, preconditioned=True, max_iter=100, rtol=1e-4, restart=20,
              outs=None):
        torch = self._torch
        if outs is None:
            outs = [torch.empty(N, dtype=self.dtype, device="cuda") for N, _ in self.sizes]
        if len(bs) != self.count or len(outs) != self.count:
            raise ValueError(f"the batch has {self.count} problems: give as many sinograms and outputs")
        for t, o, (N, M) in zip(bs, outs, self.sizes):
            if t.dtype != self.dtype or t.numel() != M or not t.is_cuda or not t.is_contiguous():
                raise TypeError("sinogram tensors must match the batch's sizes and dtype")
            if o.dtype != self.dtype or o.numel() != N or not o.is_cuda or not o.is_contiguous():
                raise TypeError("output tensors must match the batch's sizes and dtype")
        info = (wmg_solve_info * self.count)()
        rc = wmg_batch_solve(self.handle, solver, 1 if preconditioned else 0, [t.data_ptr() for t in bs],
                             [t.data_ptr() for t in outs], max_iter, rtol, restart, info, None,
                             C.c_void_p(torch.cuda.current_stream().cuda_stream))
        return outs, [(info[i].iters, info[i].status, info[i].rel_res) for i in range(self.count)], rc


class Server:
    """Continuous-batching request server (torch CUDA tensors). Requests are
    dicts with keys n, m, D and optionally levels, lam, angles, det_spacing,
    det_offset, kernel; submit() takes the request's sinogram b and returns a ticket;
    the output image is allocated here and returned by poll() when done."""

    def __init__(self, hbm_budget, max_slots=64, state_bytes=0, sino_ratio=0.0, preconditioned=True,
                 max_iter=200, rtol=1e-4, restart=20, levels=1, nu1=1, nu2=1, omega=1.0, lam=0.0,
                 hybrid_depth=1, cycle=CYCLE_HYBRID, precision=PREC_F32):
        import torch
        self._torch = torch
        self.dtype = torch.float64 if precision == PREC_F64 else torch.float32
        self.max_iter = max_iter
        self.defaults = dict(levels=levels, nu1=nu1, nu2=nu2, omega=omega, lam=lam, hybrid_depth=hybrid_depth,
                             cycle=cycle, precision=precision)
        cfg = wmg_server_config(int(hbm_budget), int(state_bytes), float(sino_ratio), max_slots,
                                1 if preconditioned else 0, max_iter, rtol, restart,
                                wmg_opts(levels, nu1, nu2, omega, lam, hybrid_depth, cycle, precision))
        self._live = {}
        self.handle = wmg_server_create(cfg, C.c_void_p(torch.cuda.current_stream().cuda_stream))

    def close(self):
        if getattr(self, "handle", None):
            wmg_server_destroy(self.handle)
            self.handle = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def submit(self, req, b):
        torch = self._torch
        n, m, D = req["n"], req["m"], req["D"]
        if b.dtype != self.dtype or b.numel() != m * D or not b.is_cuda or not b.is_contiguous():
            raise TypeError("sinogram must be a contiguous CUDA tensor of the server's dtype and size m*D")
        keep = []
        ap = None
        if req.get("angles") is not None:
            arr = (C.c_double * m)(*[float(a) for a in req["angles"]])
            keep.append(arr)
            ap = C.cast(arr, C.c_void_p)
        geom = wmg_geom(n, m, ap, D, req.get("det_spacing", 1.0), req.get("det_offset", 0.0),
                        req.get("kernel", KERNEL_STRIP))
        d = self.defaults
        opts = wmg_opts(req.get("levels", d["levels"]), d["nu1"], d["nu2"], d["omega"], req.get("lam", d["lam"]),
                        d["hybrid_depth"], d["cycle"], d["precision"])
        x = torch.empty(n * n, dtype=self.dtype, device=b.device)
        t = wmg_server_submit(self.handle, geom, opts, C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()))
        self._live[t] = (b, x)
        return t

    def step(self) -> int:
        """One tick; returns the number of requests running or queued."""
        return wmg_server_step(self.handle)

    def poll(self, ticket, history=False):
        """None while the request runs; else (x, (iters, status, rel_res),
        latency_ms[, residual history])."""
        hist = (C.c_double * (self.max_iter + 1))() if history else None
        state, info, lat = wmg_server_poll(self.handle, ticket, hist)
        if state != REQ_DONE:
            return None
        _, x = self._live.pop(ticket)
        res = (x, (info.iters, info.status, info.rel_res), lat)
        if history:
            import numpy as np
            res = res + (np.frombuffer(hist, dtype=np.float64)[:info.iters + 1].copy(),)
        return res

    def footprint(self, req) -> tuple[int, int, int]:
        d = self.defaults
        geom = wmg_geom(req["n"], req["m"], None, req["D"], req.get("det_spacing", 1.0), req.get("det_offset", 0.0),
                        req.get("kernel", KERNEL_STRIP))
        opts = wmg_opts(req.get("levels", d["levels"]), d["nu1"], d["nu2"], d["omega"], req.get("lam", d["lam"]),
                        d["hybrid_depth"], d["cycle"], d["precision"])
        return wmg_server_footprint(self.handle, geom, opts)

    def stats(self) -> dict:
        st = wmg_server_stats(self.handle)
        return {name: getattr(st, name) for name, _ in wmg_server_counters._fields_}
