"""FP64 CPU oracle for the WMG-preconditioned Krylov tomography method.

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the benchmark's
CPU-baseline leg are the only users. The product library never imports it and
it never imports the product library. The arithmetic lives in `wmg_oracle.c`
(plain C, single thread, FP64); this module compiles it with gcc and wraps it
with ctypes on numpy arrays.

Every function follows a passage of Cools et al., arXiv 1310.0956:
  Op.project / backproject    W x and W^T y as SpMVs (Section 2.1, eq. sys);
                              W by exact intersection lengths or by Joseph's
                              interpolating kernel
  sirt                        eq. sirt_it with R, C of Section 2.2.1
  packet_analysis/synthesis   Haar operators eq. intops, eq. intops_wav,
                              eq. 1of4-4of4 applied recursively (Section 3.1.3)
  Wmg.apply                   WTG recursion (Section 3.1.2) with the hybrid
                              residual rule, leaf exact solves (Section 4.1)
  cgls, gmres                 Krylov solvers on the normal equations
                              (Section 2.3.1), right preconditioning for GMRES
  wtg_propagator,             dense error propagators of the wavelet two-grid
  tg_sirt_propagator          scheme (eq. wmg) and the classical TG(1,1)-SIRT
                              scheme (eq. mg_error), and the condition numbers
                              of Section 3.2 (eq. condnr, eq. spec_wavelet,
                              eq. spec_classic). The values Figure 4 prints
                              are for the paper's Joseph kernel and unstated
                              detector width: parity unpinned for those exact
                              values; their orders of magnitude and ordering
                              are checked.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "wmg_oracle.c")
_LIBDIR = os.path.join(_HERE, "lib")
_LIB = os.path.join(_LIBDIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_dp = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64p = np.ctypeslib.ndpointer(dtype=np.int64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")

CYCLE_ADDITIVE = 0
CYCLE_HYBRID = 1
CYCLE_SYMMETRIC = 2
CYCLE_MULTIPLICATIVE = 3


def build(force: bool = False) -> str:
    """Compile the oracle shared library (gcc, -O2, no architecture flags)."""
    os.makedirs(_LIBDIR, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = C.CDLL(build())
        vp = C.c_void_p
        lib.or_op_create.restype = vp
        lib.or_op_create.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                     C.c_void_p, C.c_int]
        lib.or_op_free.argtypes = [vp]
        lib.or_ray_row_k.restype = C.c_int64
        lib.or_ray_row_k.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, vp, C.c_int, C.c_int,
                                     C.c_int, _i32p, _dp, C.c_int64]
        lib.or_ray_row.restype = C.c_int64
        lib.or_ray_row.argtypes = [C.c_int, C.c_int, C.c_int, C.c_double, C.c_double, vp, C.c_int, C.c_int,
                                   _i32p, _dp, C.c_int64]
        lib.or_op_nnz.restype = C.c_int64
        lib.or_op_nnz.argtypes = [vp]
        lib.or_op_export.argtypes = [vp, _i64p, _i32p, _dp]
        lib.or_op_trig.argtypes = [vp, _dp, _dp]
        lib.or_project.argtypes = [vp, _dp, _dp]
        lib.or_backproject.argtypes = [vp, _dp, _dp]
        lib.or_weight_trapezoid.restype = C.c_double
        lib.or_weight_trapezoid.argtypes = [C.c_double, C.c_double, C.c_double]
        lib.or_ne_residual.restype = C.c_double
        lib.or_ne_residual.argtypes = [vp, C.c_double, _dp, _dp]
        lib.or_sirt_scalings.argtypes = [vp, _dp, _dp]
        lib.or_sirt.argtypes = [vp, _dp, _dp, C.c_int, C.c_double, C.c_void_p]
        lib.or_packet_analysis.argtypes = [C.c_int, C.c_int, _dp, _dp]
        lib.or_packet_synthesis.argtypes = [C.c_int, C.c_int, _dp, _dp]
        lib.or_wmg_create.restype = vp
        lib.or_wmg_create.argtypes = [vp, C.c_int, C.c_int, C.c_int, C.c_double, C.c_double,
                                      C.c_int, C.c_int, C.c_int]
        lib.or_wmg_status.restype = C.c_int
        lib.or_wmg_status.argtypes = [vp]
        lib.or_wmg_leaf_export.argtypes = [vp, C.c_int64, _dp]
        lib.or_wmg_dinv_export.argtypes = [vp, _dp]
        lib.or_wmg_free.argtypes = [vp]
        lib.or_wmg_apply.argtypes = [vp, _dp, _dp]
        lib.or_cgls.restype = C.c_int
        lib.or_cgls.argtypes = [vp, vp, C.c_double, _dp, _dp, C.c_int, C.c_int, C.c_double, C.c_void_p]
        lib.or_set_reverse.argtypes = [C.c_int]
        lib.or_bicgstab.restype = C.c_int
        lib.or_bicgstab.argtypes = [vp, vp, C.c_double, _dp, _dp, C.c_int, C.c_int, C.c_double, vp,
                                    C.POINTER(C.c_int)]
        lib.or_gmres.restype = C.c_int
        lib.or_gmres.argtypes = [vp, vp, C.c_double, _dp, _dp, C.c_int, C.c_int, C.c_int, C.c_double,
                                 C.c_void_p]
        _lib = lib
        return lib


SUMMATION_NATURAL, SUMMATION_REVERSED, SUMMATION_PAIRWISE = 0, 1, 2


def set_summation(mode: int) -> None:
    """Order of every later SpMV row sum and dot product: natural, reversed,
    or pairwise (recursive halving). The three evaluate the same arithmetic
    with different rounding; their spread is the floor below which two
    correct FP64 implementations need not agree."""
    if mode not in (SUMMATION_NATURAL, SUMMATION_REVERSED, SUMMATION_PAIRWISE):
        raise ValueError("unknown summation order")
    _load().or_set_reverse(int(mode))


def set_reverse_summation(flag: bool) -> None:
    """Run every later SpMV and dot product in reversed order (a second,
    differently rounded evaluation of the same arithmetic)."""
    set_summation(SUMMATION_REVERSED if flag else SUMMATION_NATURAL)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


def weight_trapezoid(c: float, s: float, delta: float) -> float:
    """Chord of a unit pixel at signed distance `delta` (pixel units) from its
    centre for a line with unit normal (c, s)."""
    return _load().or_weight_trapezoid(c, s, delta)


KERNEL_STRIP = "strip"      # exact pixel-line intersection lengths
KERNEL_JOSEPH = "joseph"    # Joseph's interpolating kernel (Section 2.1)
_METHOD = {KERNEL_STRIP: 0, KERNEL_JOSEPH: 2}


def ray_row(n: int, m: int, D: int, a: int, k: int, dt: float = 1.0, t0: float = 0.0, angles=None,
            kernel: str = KERNEL_STRIP):
    """Row (a, k) of W as (columns, values), built by the same walk as Op
    (Section 2.1) without assembling W: for sampled checks at large sizes."""
    lib = _load()
    cap = 4 * n + 8
    col = np.zeros(cap, np.int32)
    val = np.zeros(cap, np.float64)
    ang = None if angles is None else _f64(angles)
    cnt = lib.or_ray_row_k(n, m, D, dt, t0, None if ang is None else ang.ctypes.data_as(C.c_void_p), a, k,
                           _METHOD[kernel], col, val, cap)
    if cnt < 0:
        raise RuntimeError("row longer than expected")
    return col[:cnt].copy(), val[:cnt].copy()


class Op:
    """Explicit projection matrix W (M x N CSR, FP64) of a parallel-beam
    geometry: n x n image, m angles, D detector bins of spacing `dt` pixels,
    offset `t0` pixels; `angles` None means theta_a = a*pi/m.
    kernel "strip": exact intersection lengths, by the parametric walk
    (method 0) or by brute-force clipping of each line against each pixel
    (method 1, tiny n only); kernel "joseph": Joseph's interpolation along the
    dominant axis (Section 2.1)."""

    def __init__(self, n: int, m: int, D: int, dt: float = 1.0, t0: float = 0.0,
                 angles=None, method: int = 0, kernel: str = KERNEL_STRIP):
        lib = _load()
        if kernel == KERNEL_JOSEPH:
            method = 2
        elif kernel != KERNEL_STRIP:
            raise ValueError("kernel must be 'strip' or 'joseph'")
        self.kernel = kernel
        self.n, self.m, self.D = n, m, D
        self.N, self.M = n * n, m * D
        self._angles = None if angles is None else _f64(angles)
        ap = None if self._angles is None else self._angles.ctypes.data_as(C.c_void_p)
        self._h = lib.or_op_create(n, m, D, dt, t0, ap, method)
        if not self._h:
            raise ValueError("invalid geometry")
        self._lib = lib

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.or_op_free(self._h)
            self._h = None

    @property
    def nnz(self) -> int:
        return self._lib.or_op_nnz(self._h)

    def csr(self):
        nnz = self.nnz
        rowptr = np.zeros(self.M + 1, np.int64)
        col = np.zeros(nnz, np.int32)
        val = np.zeros(nnz, np.float64)
        self._lib.or_op_export(self._h, rowptr, col, val)
        return rowptr, col, val

    def dense(self) -> np.ndarray:
        rowptr, col, val = self.csr()
        W = np.zeros((self.M, self.N))
        for i in range(self.M):
            W[i, col[rowptr[i]:rowptr[i + 1]]] = val[rowptr[i]:rowptr[i + 1]]
        return W

    def trig(self):
        c = np.zeros(self.m)
        s = np.zeros(self.m)
        self._lib.or_op_trig(self._h, c, s)
        return c, s

    def project(self, x) -> np.ndarray:
        y = np.zeros(self.M)
        self._lib.or_project(self._h, _f64(x), y)
        return y

    def backproject(self, y) -> np.ndarray:
        x = np.zeros(self.N)
        self._lib.or_backproject(self._h, _f64(y), x)
        return x

    def ne_residual(self, b, x, lam: float = 0.0) -> float:
        return self._lib.or_ne_residual(self._h, lam, _f64(b), _f64(x))

    def sirt_scalings(self):
        R = np.zeros(self.M)
        Cc = np.zeros(self.N)
        self._lib.or_sirt_scalings(self._h, R, Cc)
        return R, Cc


def packet_analysis(x, n: int, L: int) -> np.ndarray:
    out = np.zeros(n * n)
    _load().or_packet_analysis(n, L, _f64(x), out)
    return out


def packet_synthesis(c, n: int, L: int) -> np.ndarray:
    out = np.zeros(n * n)
    _load().or_packet_synthesis(n, L, _f64(c), out)
    return out


class Wmg:
    """WMG preconditioner B for A = W^T W + lambda I: `levels` = l (L = l-1
    Haar levels, leaves nc x nc with nc = n / 2^L), nu1/nu2 l1-Jacobi sweeps
    (damping omega), cycle ADDITIVE, HYBRID (residual update after the LL
    band at depths < hybrid_depth), SYMMETRIC (hybrid, then the LL band once
    more from the residual of the whole node correction) or MULTIPLICATIVE
    (the fully multiplicative WTG of eq. wmg at depths < hybrid_depth: each
    of LL, LH, HL, HH corrected from the residual the corrections before it
    leave). factor=False keeps the unfactored leaf
    matrices for inspection (apply is then invalid)."""

    def __init__(self, op: Op, levels: int, nu1: int = 0, nu2: int = 0, omega: float = 1.0,
                 lam: float = 0.0, cycle: int = CYCLE_ADDITIVE, hybrid_depth: int = 0,
                 factor: bool = True):
        lib = _load()
        self.op = op
        self.L = levels - 1
        self.nc = op.n >> self.L
        self.K = 4 ** self.L
        self._h = lib.or_wmg_create(op._h, levels, nu1, nu2, omega, lam, cycle, hybrid_depth,
                                    1 if factor else 0)
        if not self._h:
            raise ValueError("invalid WMG parameters")
        self._lib = lib
        self.status = lib.or_wmg_status(self._h)

    def __del__(self):
        if getattr(self, "_h", None):
            self._lib.or_wmg_free(self._h)
            self._h = None

    def leaf(self, k: int) -> np.ndarray:
        P = self.nc * self.nc
        out = np.zeros(P * P)
        self._lib.or_wmg_leaf_export(self._h, k, out)
        return out.reshape(P, P)

    def dinv(self) -> np.ndarray:
        out = np.zeros(self.op.N)
        self._lib.or_wmg_dinv_export(self._h, out)
        return out

    def apply(self, s) -> np.ndarray:
        z = np.zeros(self.op.N)
        self._lib.or_wmg_apply(self._h, _f64(s), z)
        return z


def sirt(op: Op, b, iters: int, lam: float = 0.0, x0=None):
    x = np.zeros(op.N) if x0 is None else _f64(x0).copy()
    hist = np.zeros(iters + 1)
    _load().or_sirt(op._h, _f64(b), x, iters, lam, hist.ctypes.data_as(C.c_void_p))
    return x, hist


def _start(op: Op, x0):
    """The solver's x buffer: x0 (copied) and use_x0 = 1, or zeros and 0."""
    if x0 is None:
        return np.zeros(op.N), 0
    return _f64(x0).copy(), 1


def cgls(op: Op, b, max_iter: int, rtol: float = 0.0, lam: float = 0.0, precond: Wmg = None, x0=None):
    """(Preconditioned) CGLS from x0 (default 0); returns (x, iterations,
    relative NE residual history, relative to the residual of x0)."""
    x, warm = _start(op, x0)
    hist = np.zeros(max_iter + 1)
    k = _load().or_cgls(op._h, precond._h if precond else None, lam, _f64(b), x, warm, max_iter, rtol,
                        hist.ctypes.data_as(C.c_void_p))
    return x, k, hist[:k + 1]


def gmres(op: Op, b, max_iter: int, restart: int = 20, rtol: float = 0.0, lam: float = 0.0,
          precond: Wmg = None, x0=None):
    """Restarted right-preconditioned GMRES on (W^T W + lam) x = W^T b from
    x0 (default 0); returns (x, iterations, relative residual history)."""
    x, warm = _start(op, x0)
    hist = np.zeros(max_iter + 1)
    k = _load().or_gmres(op._h, precond._h if precond else None, lam, _f64(b), x, warm, restart,
                         max_iter, rtol, hist.ctypes.data_as(C.c_void_p))
    return x, k, hist[:k + 1]


def bicgstab(op: Op, b, max_iter: int, rtol: float = 0.0, lam: float = 0.0, precond: Wmg = None, x0=None):
    """Right-preconditioned BiCGStab on (W^T W + lam) x = W^T b, the paper's
    Krylov solver (Section 2.3.1, Section 4), from x0 (default 0); returns
    (x, iterations, relative residual history, status: 0 converged, 1
    iteration cap, -5 breakdown)."""
    x, warm = _start(op, x0)
    hist = np.zeros(max_iter + 1)
    st = C.c_int(0)
    k = _load().or_bicgstab(op._h, precond._h if precond else None, lam, _f64(b), x, warm, max_iter, rtol,
                            hist.ctypes.data_as(C.c_void_p), C.byref(st))
    return x, k, hist[:k + 1], st.value


# ---------------------------------------------------------------------------
# Spectral check (Section 3.2): dense two-grid error propagators for small
# problems, and the condition numbers the paper compares
# ---------------------------------------------------------------------------
def haar_band_restrictions(n: int):
    """The four one-level Haar restrictions I_{h,id}^{2h} (eq. intops_wav,
    eq. 1of4-4of4) as dense (N/4) x N matrices, in the band order LL, LH, HL,
    HH: row-blocks of the packet analysis matrix at depth 1."""
    N = n * n
    Q = np.stack([packet_analysis(np.eye(N)[j], n, 1) for j in range(N)], axis=1)
    return [Q[k * N // 4:(k + 1) * N // 4] for k in range(4)]


def _coarse_correction(A, R):
    """I - I_{2h}^h (A^{2h})^{-1} I_h^{2h} A with the Galerkin A^{2h} = R A R^T."""
    Ac = R @ A @ R.T
    return np.eye(A.shape[0]) - R.T @ np.linalg.solve(Ac, R @ A)


def wtg_propagator(op: Op, lam: float = 0.0) -> np.ndarray:
    """Error propagator of the wavelet two-grid scheme, eq. wmg: the four band
    corrections applied one after the other (LL, LH, HL, HH), each from the
    residual of the corrected iterate (fully multiplicative)."""
    W = op.dense()
    A = W.T @ W + lam * np.eye(op.N)
    E = np.eye(op.N)
    for R in haar_band_restrictions(op.n):
        E = _coarse_correction(A, R) @ E
    return E


def tg_sirt_propagator(op: Op, nu1: int = 1, nu2: int = 1, lam: float = 0.0) -> np.ndarray:
    """Error propagator of the classical two-grid scheme, eq. mg_error:
    S^nu2 (I - I_{2h}^h (A^{2h})^{-1} I_h^{2h} A) S^nu1 with the first-order
    restriction of eq. intops (the Haar LL band) and S the SIRT iteration
    matrix I - C W^T R W (Section 2.2.1)."""
    W = op.dense()
    A = W.T @ W + lam * np.eye(op.N)
    R, C = op.sirt_scalings()
    S = np.eye(op.N) - (C[:, None] * W.T) @ (R[:, None] * W)
    K = _coarse_correction(A, haar_band_restrictions(op.n)[0])
    return np.linalg.matrix_power(S, nu2) @ K @ np.linalg.matrix_power(S, nu1)


def condition_number(M: np.ndarray, symmetric: bool = False) -> float:
    """kappa = max |lambda_i| / min |lambda_i| (eq. condnr)."""
    ev = np.linalg.eigvalsh(M) if symmetric else np.linalg.eigvals(M)
    a = np.abs(ev)
    return float(a.max() / a.min())


def preconditioned_condition_number(E: np.ndarray) -> float:
    """kappa of I - A B A^{-1} for a scheme with error propagator E = I - B A:
    its eigenvalues are 1 - eig(E) (eq. spec_wavelet, eq. spec_classic)."""
    return condition_number(np.eye(E.shape[0]) - E)
