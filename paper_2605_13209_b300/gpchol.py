"""Thin ctypes binding of libgpchol.so (C ABI in include/gpchol.h).

Argument marshalling only: every step of every solve runs in the CUDA
library.  Device matrices are torch tensors in column-major layout (stride
(1, ld)); ``colmajor`` makes one.  The current torch CUDA stream is passed to
each call.  If the library is missing, or there is no GPU, calls raise; there
is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgpchol.so")

GPCH_OK, GPCH_INVALID_ARG, GPCH_NOT_SPD, GPCH_NOT_CONVERGED, GPCH_OOM_BUDGET, GPCH_TIMEOUT, GPCH_CUDA_ERROR = range(7)
GPCH_F64, GPCH_F32 = 0, 1
(PHASE_SE, PHASE_DIAG, PHASE_PANEL, PHASE_TRAILING, PHASE_SOLVE, PHASE_CG_MATVEC, PHASE_CG_VECTOR,
 PHASE_MIXED_TRAILING, PHASE_BATCHED) = range(9)
GPCH_PREC_FP64, GPCH_PREC_BF16, GPCH_PREC_SPLIT_BF16, GPCH_PREC_SPLIT_F16 = 0, 1, 2, 3

_i64 = ctypes.c_int64
_vp = ctypes.c_void_p
_dbl = ctypes.c_double
_int = ctypes.c_int


class GpchError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{status_string(status)}: {msg}")
        self.status = status


class CGStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("converged", ctypes.c_int32), ("relres_max", ctypes.c_double)]


class CGOpts(ctypes.Structure):
    _fields_ = [("variant", ctypes.c_int32), ("products", ctypes.c_int32)]


CG_CLASSIC, CG_SINGLE_REDUCTION = 0, 1
CG_PRODUCTS_FP64, CG_PRODUCTS_DOUBLE_FLOAT, CG_PRODUCTS_TENSOR = 0, 1, 2


class System(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("B", ctypes.c_void_p),
                ("ldb", ctypes.c_int64), ("nrhs", ctypes.c_int32)]


class MSystem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("A", ctypes.c_void_p), ("lda", ctypes.c_int64), ("B", ctypes.c_void_p),
                ("ldb", ctypes.c_int64), ("X", ctypes.c_void_p), ("ldx", ctypes.c_int64), ("nrhs", ctypes.c_int32)]


class BatchStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("steps", ctypes.c_int32), ("backward_error_max", ctypes.c_double)]


class TuneInfo(ctypes.Structure):
    _fields_ = [("source", ctypes.c_int32), ("refined_tile", ctypes.c_int32 * 9),
                ("batch_tile_fp64", ctypes.c_int32 * 9), ("batch_tile_mixed", ctypes.c_int32 * 9),
                ("gpu", ctypes.c_char * 96)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("hbm_budget", ctypes.c_size_t), ("lanes", ctypes.c_int32), ("batch_max_count", ctypes.c_int32),
                ("batch_max_n", ctypes.c_int64), ("solo_prec", ctypes.c_int), ("bwd_tol", ctypes.c_double)]


class Request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("d", ctypes.c_int32), ("nrhs", ctypes.c_int32), ("X", ctypes.c_void_p),
                ("sf2", ctypes.c_double), ("ell", ctypes.c_double), ("sn2", ctypes.c_double), ("B", ctypes.c_void_p),
                ("Xout", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("path", ctypes.c_int32), ("iterations", ctypes.c_int32),
                ("backward_error", ctypes.c_double), ("latency_ms", ctypes.c_double), ("queue_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("completed", ctypes.c_int64), ("failed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("batched_requests", ctypes.c_int64), ("peak_reserved_bytes", ctypes.c_size_t),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("max_ms", ctypes.c_double),
                ("solves_per_s", ctypes.c_double)]


class RefineStats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int32), ("factor_attempts", ctypes.c_int32), ("shift", ctypes.c_double),
                ("backward_error_max", ctypes.c_double)]


_lib = None


def lib() -> ctypes.CDLL:
    """Load libgpchol.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with paper_2605_13209_b300/build.py")
        L = ctypes.CDLL(LIB_PATH)
        L.gpch_create.argtypes = [ctypes.POINTER(_vp), _int, ctypes.c_size_t]
        L.gpch_destroy.argtypes = [_vp]
        L.gpch_status_string.argtypes = [_int]
        L.gpch_status_string.restype = ctypes.c_char_p
        L.gpch_last_error.argtypes = [_vp]
        L.gpch_last_error.restype = ctypes.c_char_p
        L.gpch_version.restype = _int
        L.gpch_workspace_bytes.argtypes = [_vp]
        L.gpch_workspace_bytes.restype = ctypes.c_size_t
        L.gpch_se_matrix.argtypes = [_vp, _i64, _int, _vp, _dbl, _dbl, _dbl, _vp, _i64, _vp]
        L.gpch_chol_factor.argtypes = [_vp, _i64, _int, _vp, _i64, _vp, ctypes.POINTER(_i64)]
        L.gpch_chol_solve.argtypes = [_vp, _i64, _vp, _i64, _vp, _i64, _int, _vp]
        L.gpch_chol_solve_f32.argtypes = [_vp, _i64, _vp, _i64, _vp, _i64, _int, _vp]
        L.gpch_symv_lower.argtypes = [_vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _int, _vp]
        L.gpch_cg_solve.argtypes = [_vp, _i64, _vp, _int, _i64, _vp, _i64, _vp, _i64, _int, _dbl, _int, _int, _vp,
                                    ctypes.POINTER(CGStats)]
        L.gpch_cg_solve_ex.argtypes = [_vp, _i64, _vp, _int, _i64, _vp, _i64, _vp, _i64, _int, _dbl, _int, _int,
                                       ctypes.POINTER(CGOpts), _vp, ctypes.POINTER(CGStats)]
        L.gpch_timing_enable.argtypes = [_vp, _int]
        L.gpch_timing_read.argtypes = [_vp, _int, ctypes.POINTER(_dbl), ctypes.POINTER(_i64), ctypes.POINTER(_dbl)]
        L.gpch_launch_count.argtypes = [_vp]
        L.gpch_launch_count.restype = _i64
        L.gpch_cg_solve_noalloc.argtypes = [_i64, _vp, _int, _i64, _vp, _i64, _vp, _i64, _int, _dbl, _int, _int,
                                             _vp, ctypes.POINTER(CGStats)]
        L.gpch_batched_solve.argtypes = [_vp, _int, ctypes.POINTER(System), _vp, ctypes.POINTER(_i64)]
        L.gpch_server_create.argtypes = [_int, ctypes.POINTER(ServerOpts), ctypes.POINTER(_vp)]
        L.gpch_server_submit.argtypes = [_vp, ctypes.POINTER(Request), ctypes.POINTER(ctypes.c_uint64)]
        L.gpch_server_wait.argtypes = [_vp, ctypes.c_uint64, _dbl, ctypes.POINTER(Result)]
        L.gpch_server_poll.argtypes = [_vp, ctypes.c_uint64, ctypes.POINTER(_int), ctypes.POINTER(Result)]
        L.gpch_server_get_stats.argtypes = [_vp, ctypes.POINTER(ServerStats)]
        L.gpch_server_destroy.argtypes = [_vp]
        L.gpch_syrk_lowprec.argtypes = [_vp, _i64, _i64, _vp, _i64, _vp, _i64, _int, _vp]
        L.gpch_chol_factor_mixed.argtypes = [_vp, _i64, _int, _vp, _i64, _int, _dbl, _vp, _i64, _vp,
                                             ctypes.POINTER(_i64)]
        L.gpch_solve_refined.argtypes = [_vp, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _int, _int, _int, _dbl, _int,
                                         _vp, ctypes.POINTER(RefineStats)]
        L.gpch_logdet.argtypes = [_vp, _i64, _vp, _i64, ctypes.POINTER(_dbl), _vp]
        L.gpch_predict_mean.argtypes = [_vp, _i64, _i64, _int, _vp, _vp, _dbl, _dbl, _vp, _i64, _int, _vp, _i64, _vp]
        L.gpch_chol_factor_ex.argtypes = [_vp, _i64, _int, _vp, _i64, ctypes.c_int32, _vp, ctypes.POINTER(_i64)]
        L.gpch_gemm_fp64_emulated.argtypes = [_vp, _i64, _i64, _i64, _vp, _i64, _vp, _i64, _vp, _i64, _int, _vp]
        L.gpch_autotune.argtypes = [_vp, ctypes.c_char_p, _int, _i64, ctypes.POINTER(TuneInfo)]
        L.gpch_tune_get.argtypes = [_vp, ctypes.POINTER(TuneInfo)]
        L.gpch_batched_solve_mixed.argtypes = [_vp, _int, ctypes.POINTER(MSystem), _dbl, _int, _vp,
                                                ctypes.POINTER(_i64), ctypes.POINTER(BatchStats)]
        L.gpch_block_matvec.argtypes = [_vp, _i64, _i64, _i64, _vp, _int, _i64, _vp, _i64, _vp, _i64, _int,
                                         ctypes.c_int32, _vp]
        L.gpch_cgsr_partials.argtypes = [_vp, _i64, _int, _vp, _i64, _vp, _i64, _vp, _vp]
        L.gpch_cgsr_scalars.argtypes = [_vp, _int, _vp, _vp, _int, _dbl, _int, _vp]
        L.gpch_cgsr_vectors.argtypes = [_vp, _i64, _int, _vp, _vp, _i64, _vp, _vp, _vp, _vp, _i64, _int, _vp]
        L.gpch_cgsr_residual.argtypes = [_vp, _i64, _int, _vp, _vp, _i64, _vp, _vp, _i64, _int, _vp]
        for name in ("gpch_chol_factor_ex", "gpch_gemm_fp64_emulated", "gpch_autotune", "gpch_tune_get", "gpch_batched_solve_mixed", "gpch_block_matvec", "gpch_cgsr_partials", "gpch_cgsr_scalars", "gpch_cgsr_vectors",
                     "gpch_cgsr_residual", "gpch_cg_solve_ex", "gpch_logdet", "gpch_predict_mean", "gpch_create", "gpch_destroy", "gpch_se_matrix", "gpch_chol_factor", "gpch_chol_solve", "gpch_chol_solve_f32", "gpch_symv_lower",
                     "gpch_cg_solve", "gpch_timing_enable", "gpch_timing_read", "gpch_syrk_lowprec",
                     "gpch_chol_factor_mixed", "gpch_solve_refined", "gpch_cg_solve_noalloc",
                     "gpch_batched_solve", "gpch_server_create", "gpch_server_submit", "gpch_server_wait",
                     "gpch_server_poll", "gpch_server_get_stats", "gpch_server_destroy"):
            getattr(L, name).restype = _int
        _lib = L
    return _lib


def status_string(s: int) -> str:
    return lib().gpch_status_string(int(s)).decode()


def _stream(stream=None) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def colmajor(n: int, m: int, dtype=torch.float64, device="cuda", ld: int | None = None) -> torch.Tensor:
    """Empty n x m tensor in column-major layout (stride (1, ld))."""
    ld = n if ld is None else ld
    return torch.empty((m, ld), dtype=dtype, device=device).t()[:n]


def as_colmajor(t: torch.Tensor) -> torch.Tensor:
    """Column-major copy of a 1-D or 2-D tensor (1-D becomes n x 1)."""
    if t.dim() == 1:
        t = t[:, None]
    out = colmajor(t.shape[0], t.shape[1], t.dtype, t.device)
    out.copy_(t)
    return out


def _ld(t: torch.Tensor) -> int:
    if t.dim() != 2 or t.stride(0) != 1:
        raise ValueError("expected a column-major 2-D tensor (stride(0) == 1); use colmajor()/as_colmajor()")
    return max(t.stride(1), 1) if t.shape[1] > 1 else max(t.shape[0], 1)


def _check_cuda(t: torch.Tensor, dtype):
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"expected {dtype}, got {t.dtype}")


class Context:
    """A library context (device, workspace arena, HBM budget)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0):
        self._h = _vp()
        st = lib().gpch_create(ctypes.byref(self._h), int(device), int(hbm_budget_bytes))
        if st != GPCH_OK:
            raise GpchError(st, "gpch_create failed (no usable CUDA device?)")
        self.device = device

    @property
    def handle(self):
        return self._h

    def check(self, st: int):
        if st != GPCH_OK:
            raise GpchError(st, lib().gpch_last_error(self._h).decode())

    def workspace_bytes(self) -> int:
        return int(lib().gpch_workspace_bytes(self._h))

    def timing_enable(self, on: bool = True):
        self.check(lib().gpch_timing_enable(self._h, int(bool(on))))

    def timing_read(self, phase: int):
        """(total_ms, launches, work) of one phase since timing was enabled."""
        ms, n, w = _dbl(0), _i64(0), _dbl(0)
        self.check(lib().gpch_timing_read(self._h, int(phase), ctypes.byref(ms), ctypes.byref(n), ctypes.byref(w)))
        return float(ms.value), int(n.value), float(w.value)

    def launch_count(self) -> int:
        return int(lib().gpch_launch_count(self._h))

    def close(self):
        if self._h:
            lib().gpch_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_default_ctx: Context | None = None


def default_context() -> Context:
    global _default_ctx
    if _default_ctx is None:
        _default_ctx = Context(torch.cuda.current_device())
    return _default_ctx


def se_matrix(X: torch.Tensor, sf2: float, ell: float, sn2: float, A: torch.Tensor | None = None,
              ctx: Context | None = None, stream=None) -> torch.Tensor:
    """A1: squared-exponential covariance of the points X (n x d, row-major,
    float64, CUDA) into a full n x n column-major A."""
    ctx = ctx or default_context()
    _check_cuda(X, torch.float64)
    X = X.contiguous()
    n, d = X.shape
    if A is None:
        A = colmajor(n, n, device=X.device)
    ctx.check(lib().gpch_se_matrix(ctx.handle, n, d, X.data_ptr(), sf2, ell, sn2, A.data_ptr(), _ld(A),
                                   _stream(stream)))
    return A


def chol_factor(A: torch.Tensor, tile: int = 256, ctx: Context | None = None, stream=None,
                raise_on_not_spd: bool = True, update: str = "fp64") -> int:
    """A2-A4: in-place FP64 blocked Cholesky of the column-major A (lower
    triangle).  update: "fp64" (FP64 FMAs) or "fp64_emulated" (step 3 with
    the FP64-accurate tensor-core product).  Returns info (0 on success)."""
    ctx = ctx or default_context()
    _check_cuda(A, torch.float64)
    info = _i64(0)
    upd = {"fp64": 0, "fp64_emulated": 1}[update]
    st = lib().gpch_chol_factor_ex(ctx.handle, A.shape[0], int(tile), A.data_ptr(), _ld(A), upd, _stream(stream),
                                   ctypes.byref(info))
    if st == GPCH_NOT_SPD and not raise_on_not_spd:
        return int(info.value)
    ctx.check(st)
    return int(info.value)


def chol_solve(L: torch.Tensor, B: torch.Tensor, ctx: Context | None = None, stream=None) -> torch.Tensor:
    """A5: solve L L^T X = B in place on the column-major B (n x nrhs)."""
    ctx = ctx or default_context()
    _check_cuda(L, torch.float64)
    _check_cuda(B, torch.float64)
    ctx.check(lib().gpch_chol_solve(ctx.handle, L.shape[0], L.data_ptr(), _ld(L), B.data_ptr(), _ld(B), B.shape[1],
                                    _stream(stream)))
    return B


def chol_solve_f32(L: torch.Tensor, B: torch.Tensor, ctx: Context | None = None, stream=None) -> torch.Tensor:
    """A5 with an FP32 factor (e.g. from chol_factor_mixed): solve L L^T X = B
    in place on the column-major FP64 B (n x nrhs).  Synchronizes the stream."""
    ctx = ctx or default_context()
    _check_cuda(L, torch.float32)
    _check_cuda(B, torch.float64)
    ctx.check(lib().gpch_chol_solve_f32(ctx.handle, L.shape[0], L.data_ptr(), _ld(L), B.data_ptr(), _ld(B),
                                        B.shape[1], _stream(stream)))
    return B


def symv_lower(A: torch.Tensor, X: torch.Tensor, Y: torch.Tensor | None = None, ctx: Context | None = None,
               stream=None) -> torch.Tensor:
    """Y = A X from the lower triangle of the column-major FP64 symmetric A
    (entries above the diagonal never change the result), with double-float
    products: the refined solve's CG product.  X: n x nrhs column-major
    FP64.  Returns Y (n x nrhs, column-major; allocated when not given).
    Enqueued on the stream."""
    ctx = ctx or default_context()
    _check_cuda(A, torch.float64)
    _check_cuda(X, torch.float64)
    n, nrhs = X.shape[0], X.shape[1]
    if Y is None:
        Y = colmajor(n, nrhs, device=X.device)
    _check_cuda(Y, torch.float64)
    ctx.check(lib().gpch_symv_lower(ctx.handle, n, A.data_ptr(), _ld(A), X.data_ptr(), _ld(X), Y.data_ptr(), _ld(Y),
                                    nrhs, _stream(stream)))
    return Y


def logdet(L: torch.Tensor, ctx: Context | None = None, stream=None) -> float:
    """f3: log det A = 2 sum log L_ii from the column-major FP64 factor L
    (as left by chol_factor).  Synchronizes the stream."""
    ctx = ctx or default_context()
    _check_cuda(L, torch.float64)
    out = _dbl(0.0)
    ctx.check(lib().gpch_logdet(ctx.handle, L.shape[0], L.data_ptr(), _ld(L), ctypes.byref(out), _stream(stream)))
    return float(out.value)


def predict_mean(Xs: torch.Tensor, X: torch.Tensor, sf2: float, ell: float, alpha: torch.Tensor,
                 mean: torch.Tensor | None = None, ctx: Context | None = None, stream=None) -> torch.Tensor:
    """f3: GP predictive mean K(Xs, X) alpha (noise-free SE cross
    covariance formed on the fly).  Xs: m x d, X: n x d (row-major float64
    CUDA); alpha: n x nrhs column-major.  Returns mean (m x nrhs,
    column-major)."""
    ctx = ctx or default_context()
    _check_cuda(Xs, torch.float64)
    _check_cuda(X, torch.float64)
    _check_cuda(alpha, torch.float64)
    Xs = Xs.contiguous()
    X = X.contiguous()
    m, d = Xs.shape
    n = X.shape[0]
    if X.shape[1] != d or alpha.shape[0] != n:
        raise ValueError("shape mismatch between Xs, X and alpha")
    nrhs = alpha.shape[1]
    if mean is None:
        mean = colmajor(m, nrhs, device=Xs.device)
    ctx.check(lib().gpch_predict_mean(ctx.handle, m, n, d, Xs.data_ptr(), X.data_ptr(), sf2, ell, alpha.data_ptr(),
                                      _ld(alpha), nrhs, mean.data_ptr(), _ld(mean), _stream(stream)))
    return mean


@dataclass
class CGResult:
    iterations: int
    converged: int
    relres_max: float
    status: int


_CG_VARIANT = {"classic": CG_CLASSIC, "single_reduction": CG_SINGLE_REDUCTION}
_CG_PRODUCTS = {"fp64": CG_PRODUCTS_FP64, "double_float": CG_PRODUCTS_DOUBLE_FLOAT, "tensor": CG_PRODUCTS_TENSOR}


def cg_solve(A: torch.Tensor, B: torch.Tensor, X: torch.Tensor, rtol: float = 1e-10, maxit: int = 10000,
             replace_every: int = 50, ctx: Context | None = None, stream=None,
             raise_on_not_converged: bool = True, variant: str = "classic", products: str = "fp64") -> CGResult:
    """A6-A7: CG (Algorithm 1, left) on the full column-major A (float64 or
    float32), right-hand sides B and start/solution X (n x nrhs, float64).
    variant: "classic" or "single_reduction" (Chronopoulos-Gear); products:
    "fp64", "double_float" (FP32-pipe double-float products) or "tensor"
    (FP64-accurate products on the tensor cores; A symmetric)."""
    ctx = ctx or default_context()
    if A.dtype not in (torch.float64, torch.float32):
        raise ValueError("A must be float64 or float32")
    _check_cuda(A, A.dtype)
    _check_cuda(B, torch.float64)
    _check_cuda(X, torch.float64)
    stats = CGStats()
    dt = GPCH_F64 if A.dtype == torch.float64 else GPCH_F32
    opts = CGOpts(_CG_VARIANT[variant], _CG_PRODUCTS[products])
    st = lib().gpch_cg_solve_ex(ctx.handle, A.shape[0], A.data_ptr(), dt, _ld(A), B.data_ptr(), _ld(B),
                                X.data_ptr(), _ld(X), B.shape[1], rtol, int(maxit), int(replace_every),
                                ctypes.byref(opts), _stream(stream), ctypes.byref(stats))
    if st != GPCH_OK and not (st == GPCH_NOT_CONVERGED and not raise_on_not_converged):
        ctx.check(st)
    return CGResult(stats.iterations, stats.converged, stats.relres_max, st)


def block_matvec(Ablk: torch.Tensor, r0: int, V: torch.Tensor, T: torch.Tensor, products: str = "fp64",
                 ctx: Context | None = None, stream=None) -> torch.Tensor:
    """f4 local product: T = Ablk^T V, rows r0 .. r0+m-1 of A V for the
    symmetric A whose columns r0 .. r0+m-1 are the n x m block Ablk."""
    ctx = ctx or default_context()
    if Ablk.dtype not in (torch.float64, torch.float32):
        raise ValueError("Ablk must be float64 or float32")
    _check_cuda(V, torch.float64)
    _check_cuda(T, torch.float64)
    n, m = Ablk.shape
    dt = GPCH_F64 if Ablk.dtype == torch.float64 else GPCH_F32
    ctx.check(lib().gpch_block_matvec(ctx.handle, n, m, int(r0), Ablk.data_ptr(), dt, _ld(Ablk), V.data_ptr(), _ld(V),
                                      T.data_ptr(), _ld(T), V.shape[1], _CG_PRODUCTS[products], _stream(stream)))
    return T


def cgsr_partials(R: torch.Tensor, W: torch.Tensor, sums: torch.Tensor, ctx: Context | None = None, stream=None):
    ctx = ctx or default_context()
    ctx.check(lib().gpch_cgsr_partials(ctx.handle, R.shape[0], R.shape[1], R.data_ptr(), _ld(R), W.data_ptr(), _ld(W),
                                       sums.data_ptr(), _stream(stream)))


def cgsr_scalars(sums: torch.Tensor, state: torch.Tensor, nrhs: int, first: bool, rtol: float, maxit: int,
                 ctx: Context | None = None, stream=None):
    ctx = ctx or default_context()
    ctx.check(lib().gpch_cgsr_scalars(ctx.handle, int(nrhs), sums.data_ptr(), state.data_ptr(), int(bool(first)),
                                      float(rtol), int(maxit), _stream(stream)))


def cgsr_vectors(state: torch.Tensor, X: torch.Tensor, R: torch.Tensor, W: torch.Tensor, P: torch.Tensor,
                 S: torch.Tensor, replace: bool, ctx: Context | None = None, stream=None):
    ctx = ctx or default_context()
    ctx.check(lib().gpch_cgsr_vectors(ctx.handle, R.shape[0], R.shape[1], state.data_ptr(), X.data_ptr(), _ld(X),
                                      R.data_ptr(), W.data_ptr(), P.data_ptr(), S.data_ptr(), _ld(R),
                                      int(bool(replace)), _stream(stream)))


def cgsr_residual(state: torch.Tensor, B: torch.Tensor, T: torch.Tensor, R: torch.Tensor, all_columns: bool,
                  ctx: Context | None = None, stream=None):
    ctx = ctx or default_context()
    ctx.check(lib().gpch_cgsr_residual(ctx.handle, R.shape[0], R.shape[1], state.data_ptr(), B.data_ptr(), _ld(B),
                                       T.data_ptr(), R.data_ptr(), _ld(R), int(bool(all_columns)), _stream(stream)))


# layout of gpch_cgsr_state: four double[16] arrays, two int32[16] arrays, done, pad
CGSR_STATE_BYTES = 4 * 16 * 8 + 2 * 16 * 4 + 8


def cg_solve_noalloc(A: torch.Tensor, B: torch.Tensor, X: torch.Tensor, rtol: float = 1e-10, maxit: int = 10000,
                     replace_every: int = 50, stream=None) -> CGResult:
    """gpch_cg_solve_noalloc: the CG solve without any device allocation
    (fixed library-owned scratch; n * nrhs <= 262144, nrhs <= 16).  Runs on
    the current CUDA device; no context is involved."""
    if A.dtype not in (torch.float64, torch.float32):
        raise ValueError("A must be float64 or float32")
    _check_cuda(A, A.dtype)
    _check_cuda(B, torch.float64)
    _check_cuda(X, torch.float64)
    stats = CGStats()
    dt = GPCH_F64 if A.dtype == torch.float64 else GPCH_F32
    st = lib().gpch_cg_solve_noalloc(A.shape[0], A.data_ptr(), dt, _ld(A), B.data_ptr(), _ld(B), X.data_ptr(),
                                     _ld(X), B.shape[1], rtol, int(maxit), int(replace_every), _stream(stream),
                                     ctypes.byref(stats))
    if st not in (GPCH_OK, GPCH_NOT_CONVERGED):
        raise GpchError(st, "gpch_cg_solve_noalloc failed")
    return CGResult(stats.iterations, stats.converged, stats.relres_max, st)


_PREC = {"bf16": GPCH_PREC_BF16, "split_bf16": GPCH_PREC_SPLIT_BF16, "split_f16": GPCH_PREC_SPLIT_F16,
         GPCH_PREC_BF16: GPCH_PREC_BF16, GPCH_PREC_SPLIT_BF16: GPCH_PREC_SPLIT_BF16,
         GPCH_PREC_SPLIT_F16: GPCH_PREC_SPLIT_F16}


def syrk_lowprec(P: torch.Tensor, C: torch.Tensor, prec="bf16", ctx: Context | None = None,
                 stream=None) -> torch.Tensor:
    """A4 (mixed): C_lower -= P P^T on the tensor cores (bf16 or split bf16
    products, FP32 accumulation).  P: m x k float32, C: m x m float32, both
    column-major."""
    ctx = ctx or default_context()
    _check_cuda(P, torch.float32)
    _check_cuda(C, torch.float32)
    ctx.check(lib().gpch_syrk_lowprec(ctx.handle, P.shape[0], P.shape[1], P.data_ptr(), _ld(P), C.data_ptr(), _ld(C),
                                      _PREC[prec], _stream(stream)))
    return C


def chol_factor_mixed(A: torch.Tensor, prec="bf16", tile: int = 512, shift: float = 0.0,
                      L: torch.Tensor | None = None, ctx: Context | None = None, stream=None,
                      raise_on_not_spd: bool = True):
    """A8: low-precision factor (FP32 storage) of A + shift I.  Returns (L, info)."""
    ctx = ctx or default_context()
    _check_cuda(A, torch.float64)
    n = A.shape[0]
    if L is None:
        L = colmajor(n, n, dtype=torch.float32, device=A.device)
    info = _i64(0)
    st = lib().gpch_chol_factor_mixed(ctx.handle, n, int(tile), A.data_ptr(), _ld(A), _PREC[prec], float(shift),
                                      L.data_ptr(), _ld(L), _stream(stream), ctypes.byref(info))
    if not (st == GPCH_NOT_SPD and not raise_on_not_spd):
        ctx.check(st)
    return L, int(info.value)


@dataclass
class RefineResult:
    iterations: int
    factor_attempts: int
    shift: float
    backward_error_max: float
    status: int


def solve_refined(A: torch.Tensor, B: torch.Tensor, X: torch.Tensor, prec="split_bf16", tile: int = 512,
                  bwd_tol: float = 1e-12, maxit: int = 500, ctx: Context | None = None, stream=None,
                  raise_on_error: bool = True) -> RefineResult:
    """A8-A9: mixed-precision factor + FP64 PCG refinement to bwd_tol."""
    ctx = ctx or default_context()
    _check_cuda(A, torch.float64)
    _check_cuda(B, torch.float64)
    _check_cuda(X, torch.float64)
    stats = RefineStats()
    st = lib().gpch_solve_refined(ctx.handle, A.shape[0], A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), X.data_ptr(),
                                  _ld(X), B.shape[1], _PREC[prec], int(tile), float(bwd_tol), int(maxit),
                                  _stream(stream), ctypes.byref(stats))
    if raise_on_error:
        ctx.check(st)
    return RefineResult(stats.iterations, stats.factor_attempts, stats.shift, stats.backward_error_max, st)


def batched_solve(As, Bs, ctx: Context | None = None, stream=None, raise_on_not_spd: bool = True):
    """A10: factor (in place) and solve a batch of FP64 systems.  As, Bs:
    lists of column-major float64 CUDA tensors (n x n and n x nrhs); each B
    is overwritten by its solution.  Returns the list of info values."""
    ctx = ctx or default_context()
    if len(As) != len(Bs):
        raise ValueError("As and Bs differ in length")
    arr = (System * len(As))()
    for i, (A, B) in enumerate(zip(As, Bs)):
        _check_cuda(A, torch.float64)
        _check_cuda(B, torch.float64)
        arr[i] = System(A.shape[0], A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), B.shape[1])
    info = (_i64 * max(len(As), 1))()
    st = lib().gpch_batched_solve(ctx.handle, len(As), arr, _stream(stream), info)
    if not (st == GPCH_NOT_SPD and not raise_on_not_spd):
        ctx.check(st)
    return [int(info[i]) for i in range(len(As))]


def gemm_fp64_emulated(A: torch.Tensor, B: torch.Tensor, C: torch.Tensor, lower: bool = False,
                       ctx: Context | None = None, stream=None) -> torch.Tensor:
    """f1: C -= A B^T with FP64-accurate products on the tensor cores (A: m x k,
    B: n x k, C: m x n; column-major float64 CUDA tensors).  lower: only the
    lower triangle of the square C."""
    ctx = ctx or default_context()
    for t in (A, B, C):
        _check_cuda(t, torch.float64)
    m, k = A.shape
    n = B.shape[0]
    if B.shape[1] != k or C.shape[0] != m or C.shape[1] != n:
        raise ValueError("shape mismatch")
    ctx.check(lib().gpch_gemm_fp64_emulated(ctx.handle, m, n, k, A.data_ptr(), _ld(A), B.data_ptr(), _ld(B),
                                            C.data_ptr(), _ld(C), int(bool(lower)), _stream(stream)))
    return C


TUNE_SOURCES = {0: "defaults", 1: "measured", 2: "loaded"}


def _tune_dict(t: TuneInfo) -> dict:
    return {"source": TUNE_SOURCES.get(t.source, str(t.source)), "gpu": t.gpu.decode(),
            "refined_tile": list(t.refined_tile), "batch_tile_fp64": list(t.batch_tile_fp64),
            "batch_tile_mixed": list(t.batch_tile_mixed)}


def autotune(cache_path: str | None = None, force: bool = False, nmax: int = 0, ctx: Context | None = None) -> dict:
    """gpch_autotune: measure (or load from cache_path) the tile choices of
    this device.  Bucket b of each list covers n <= 512 * 2^b."""
    ctx = ctx or default_context()
    t = TuneInfo()
    ctx.check(lib().gpch_autotune(ctx.handle, cache_path.encode() if cache_path else None, int(bool(force)),
                                  int(nmax), ctypes.byref(t)))
    return _tune_dict(t)


def tune_get(ctx: Context | None = None) -> dict:
    ctx = ctx or default_context()
    t = TuneInfo()
    ctx.check(lib().gpch_tune_get(ctx.handle, ctypes.byref(t)))
    return _tune_dict(t)


@dataclass
class BatchResult:
    info: list
    iterations: int
    steps: int
    backward_error_max: float
    status: int


def batched_solve_mixed(As, Bs, Xs, bwd_tol: float = 1e-12, maxit: int = 30, ctx: Context | None = None,
                        stream=None, raise_on_error: bool = True) -> BatchResult:
    """A10 (mixed): FP32 factors with FP64 diagonal leaves and FP64
    iterative refinement for a batch of systems.  As: n x n float64
    (read only), Bs: n x nrhs float64 (read only), Xs: n x nrhs float64
    (solutions), all column-major CUDA tensors."""
    ctx = ctx or default_context()
    if not (len(As) == len(Bs) == len(Xs)):
        raise ValueError("As, Bs and Xs differ in length")
    arr = (MSystem * max(len(As), 1))()
    for i, (A, B, X) in enumerate(zip(As, Bs, Xs)):
        for t in (A, B, X):
            _check_cuda(t, torch.float64)
        arr[i] = MSystem(A.shape[0], A.data_ptr(), _ld(A), B.data_ptr(), _ld(B), X.data_ptr(), _ld(X), B.shape[1])
    info = (_i64 * max(len(As), 1))()
    stats = BatchStats()
    st = lib().gpch_batched_solve_mixed(ctx.handle, len(As), arr, float(bwd_tol), int(maxit), _stream(stream), info,
                                        ctypes.byref(stats))
    if raise_on_error:
        ctx.check(st)
    return BatchResult([int(info[i]) for i in range(len(As))], stats.iterations, stats.steps,
                       stats.backward_error_max, st)


class Server:
    """A11: serving loop with continuous batching (gpch_server_*).  Requests
    are host numpy arrays; the binding keeps them alive until collected."""

    def __init__(self, device: int = 0, hbm_budget: int = 0, lanes: int = 4, batch_max_count: int = 32,
                 batch_max_n: int = 2048, solo_prec="split_bf16", bwd_tol: float = 1e-12):
        import numpy as np  # noqa: F401
        prec = GPCH_PREC_FP64 if solo_prec in ("fp64", GPCH_PREC_FP64) else _PREC[solo_prec]
        self._opts = ServerOpts(int(hbm_budget), int(lanes), int(batch_max_count), int(batch_max_n), prec,
                                float(bwd_tol))
        self._h = _vp()
        st = lib().gpch_server_create(int(device), ctypes.byref(self._opts), ctypes.byref(self._h))
        if st != GPCH_OK:
            raise GpchError(st, "gpch_server_create failed")
        self._keep = {}

    def submit(self, X, B, sf2: float, ell: float, sn2: float) -> int:
        import numpy as np
        X = np.ascontiguousarray(X, dtype=np.float64)
        B = np.asfortranarray(np.atleast_2d(np.asarray(B, dtype=np.float64).T).T)
        out = np.zeros_like(B, order="F")
        n, d = X.shape
        req = Request(n, d, B.shape[1], X.ctypes.data, sf2, ell, sn2, B.ctypes.data, out.ctypes.data)
        t = ctypes.c_uint64(0)
        st = lib().gpch_server_submit(self._h, ctypes.byref(req), ctypes.byref(t))
        if st != GPCH_OK:
            raise GpchError(st, "gpch_server_submit failed")
        self._keep[int(t.value)] = (X, B, out)
        return int(t.value)

    def wait(self, ticket: int, timeout_s: float = 600.0):
        """Returns (solution n x nrhs, result dict)."""
        res = Result()
        st = lib().gpch_server_wait(self._h, ticket, timeout_s, ctypes.byref(res))
        if st == GPCH_TIMEOUT:
            raise GpchError(st, "request still running")
        _, _, out = self._keep.pop(ticket)
        return out, {"status": res.status, "path": res.path, "iterations": res.iterations,
                     "backward_error": res.backward_error, "latency_ms": res.latency_ms, "queue_ms": res.queue_ms}

    def stats(self) -> dict:
        s = ServerStats()
        st = lib().gpch_server_get_stats(self._h, ctypes.byref(s))
        if st != GPCH_OK:
            raise GpchError(st, "gpch_server_get_stats failed")
        return {k: getattr(s, k) for k, _ in ServerStats._fields_}

    def close(self):
        if self._h:
            lib().gpch_server_destroy(self._h)
            self._h = _vp()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
