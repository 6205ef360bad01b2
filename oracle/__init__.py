"""FP64 CPU oracle for the GP solvers (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It wraps ``gp_oracle.c`` (plain C,
FP64, unblocked loops) through ctypes and shares no code with the CUDA
library in ``paper_2605_13209_b300``; that library never imports it.

Each wrapper names the paper passage it follows (Thuering, Strack, Pflueger,
IWOCL '26): Algorithm 1 (left: CG, right: blocked right-looking Cholesky),
Sec. 2.1 (residual replacement), Sec. 2.2 (L L^T = A, forward and back
substitution).  All arrays are numpy float64, column-major (Fortran order)
where they are matrices.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gp_oracle.c")
_LIB = os.path.join(_HERE, "libgporacle.so")

_c_i64 = ctypes.c_int64
_c_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile gp_oracle.c into libgporacle.so (gcc, no FMA contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call([
            "gcc", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
            "-std=c11", "-o", _LIB, _SRC, "-lm",
        ])
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.or_se_matrix.argtypes = [_c_i64, ctypes.c_int, _c_dp, ctypes.c_double, ctypes.c_double,
                                   ctypes.c_double, _c_dp, _c_i64]
        L.or_se_entry.argtypes = [ctypes.c_int, _c_dp, _c_dp, ctypes.c_int, ctypes.c_double,
                                  ctypes.c_double, ctypes.c_double]
        L.or_se_entry.restype = ctypes.c_double
        L.or_cholesky.argtypes = [_c_i64, _c_dp, _c_i64]
        L.or_cholesky.restype = _c_i64
        L.or_blocked_cholesky.argtypes = [_c_i64, _c_i64, _c_dp, _c_i64]
        L.or_blocked_cholesky.restype = _c_i64
        L.or_round_bf16.argtypes = [ctypes.c_double]
        L.or_round_bf16.restype = ctypes.c_double
        L.or_round_f32.argtypes = [ctypes.c_double]
        L.or_round_f32.restype = ctypes.c_double
        L.or_round_f16.argtypes = [ctypes.c_double]
        L.or_round_f16.restype = ctypes.c_double
        L.or_mixed_factor.argtypes = [_c_i64, _c_i64, _c_dp, _c_i64, ctypes.c_int, ctypes.c_double,
                                      _c_dp, _c_i64]
        L.or_mixed_factor.restype = _c_i64
        L.or_forward_sub.argtypes = [_c_i64, _c_dp, _c_i64, _c_dp, _c_i64, ctypes.c_int]
        L.or_back_sub.argtypes = [_c_i64, _c_dp, _c_i64, _c_dp, _c_i64, ctypes.c_int]
        L.or_cg.argtypes = [_c_i64, _c_dp, _c_i64, _c_dp, _c_dp, ctypes.c_double, ctypes.c_int,
                            ctypes.c_int, _c_dp]
        L.or_cg.restype = ctypes.c_int
        L.or_backward_error.argtypes = [_c_i64, _c_dp, _c_i64, _c_dp, _c_dp]
        L.or_backward_error.restype = ctypes.c_double
        L.or_pcg.argtypes = [_c_i64, _c_dp, _c_i64, _c_dp, _c_i64, _c_dp, _c_dp, ctypes.c_double,
                             ctypes.c_double, ctypes.c_int, ctypes.c_int, _c_dp]
        L.or_pcg.restype = ctypes.c_int
        L.or_cg_single_reduction.argtypes = [_c_i64, _c_dp, _c_i64, _c_dp, _c_dp, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, _c_dp]
        L.or_cg_single_reduction.restype = ctypes.c_int
        L.or_gemm_update.argtypes = [_c_i64, _c_i64, _c_i64, _c_dp, _c_i64, _c_dp, _c_i64, _c_dp, _c_i64, ctypes.c_int]
        L.or_logdet.argtypes = [_c_i64, _c_dp, _c_i64, _c_dp]
        L.or_logdet.restype = _c_i64
        L.or_predict_mean.argtypes = [_c_i64, _c_i64, ctypes.c_int, _c_dp, _c_dp, ctypes.c_double, ctypes.c_double,
                                      _c_dp, _c_i64, ctypes.c_int, _c_dp, _c_i64]
        _lib = L
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(_c_dp)


def _fmat(A) -> np.ndarray:
    return np.array(A, dtype=np.float64, order="F", copy=True)


def se_matrix(X, sf2: float, ell: float, sn2: float) -> np.ndarray:
    """Squared-exponential GP kernel matrix of the n x d points X (Sec. 4.1's
    GP covariance matrices, synthetic SE stand-in).  Full n x n, column-major."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    n, d = X.shape
    A = np.zeros((n, n), dtype=np.float64, order="F")
    lib().or_se_matrix(n, d, _p(X), sf2, ell, sn2, _p(A), max(n, 1))
    return A


def se_entry(xi, xj, same: bool, sf2: float, ell: float, sn2: float) -> float:
    """One SE entry K(x_i, x_j) (+ sn2 on the diagonal)."""
    xi = np.ascontiguousarray(xi, dtype=np.float64)
    xj = np.ascontiguousarray(xj, dtype=np.float64)
    return lib().or_se_entry(xi.shape[0], _p(xi), _p(xj), int(bool(same)), sf2, ell, sn2)


def cholesky(A):
    """Textbook unblocked Cholesky, L L^T = A (Sec. 2.2).  Returns (L, info);
    L is lower triangular (strict upper part zeroed)."""
    M = _fmat(A)
    n = M.shape[0]
    info = lib().or_cholesky(n, _p(M), max(n, 1))
    return np.tril(M), int(info)


def blocked_cholesky(A, b: int):
    """Algorithm 1 (right) with block size b.  Returns (L, info)."""
    M = _fmat(A)
    n = M.shape[0]
    info = lib().or_blocked_cholesky(n, b, _p(M), max(n, 1))
    return np.tril(M), int(info)


def round_bf16(x: float) -> float:
    return lib().or_round_bf16(float(x))


def round_f32(x: float) -> float:
    return lib().or_round_f32(float(x))


def round_f16(x: float) -> float:
    return lib().or_round_f16(float(x))


MIXED_MODES = {"fp32": 0, "bf16": 1, "split_bf16": 2, "split_f16": 3}


def mixed_factor(A, b: int, mode: str = "bf16", shift: float = 0.0):
    """Emulated low-precision factor (preconditioner of the refined solve).
    Returns (Lt, info)."""
    M = _fmat(A)
    n = M.shape[0]
    Lt = np.zeros((n, n), dtype=np.float64, order="F")
    info = lib().or_mixed_factor(n, b, _p(M), max(n, 1), MIXED_MODES[mode], shift, _p(Lt), max(n, 1))
    return np.tril(Lt), int(info)


def forward_sub(L, B):
    """Solve L Y = B (Sec. 2.2 forward substitution)."""
    L = _fmat(L)
    Y = _fmat(np.atleast_2d(np.asarray(B, dtype=np.float64).T).T)
    n, nrhs = Y.shape
    lib().or_forward_sub(n, _p(L), max(n, 1), _p(Y), max(n, 1), nrhs)
    return Y.reshape(np.shape(B))


def back_sub(L, B):
    """Solve L^T X = B (Sec. 2.2 back substitution)."""
    L = _fmat(L)
    Y = _fmat(np.atleast_2d(np.asarray(B, dtype=np.float64).T).T)
    n, nrhs = Y.shape
    lib().or_back_sub(n, _p(L), max(n, 1), _p(Y), max(n, 1), nrhs)
    return Y.reshape(np.shape(B))


def chol_solve(L, B):
    """x = L^-T L^-1 b."""
    return back_sub(L, forward_sub(L, B))


def cg(A, b, eps: float, maxit: int, R: int = 50, x0=None):
    """Algorithm 1 (left) with residual replacement every R iterations
    (Sec. 2.1).  Returns (x, iterations, relres)."""
    A = _fmat(A)
    n = A.shape[0]
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    rr = ctypes.c_double(0.0)
    it = lib().or_cg(n, _p(A), max(n, 1), _p(b), _p(x), eps, maxit, R, ctypes.byref(rr))
    return x, int(it), float(rr.value)


def cg_single_reduction(A, b, eps: float, maxit: int, R: int = 50, x0=None):
    """Chronopoulos-Gear single-reduction CG: Algorithm 1 (left) rearranged
    so that an iteration's two inner products follow its one product with A
    (the pipelined CG variants of the paper's related work, Sec. 1).
    Returns (x, iterations, relres)."""
    A = _fmat(A)
    n = A.shape[0]
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    rr = ctypes.c_double(0.0)
    it = lib().or_cg_single_reduction(n, _p(A), max(n, 1), _p(b), _p(x), eps, maxit, R, ctypes.byref(rr))
    return x, int(it), float(rr.value)


def gemm_update(C, A, B, lower: bool = False):
    """C - A B^T with long-double sums, one rounding per entry (Algorithm 1
    step 3 as a definition).  lower: only row >= column entries change."""
    C = _fmat(C)
    A = _fmat(A)
    B = _fmat(B)
    m, k = A.shape
    n = B.shape[0]
    lib().or_gemm_update(m, n, k, _p(A), max(m, 1), _p(B), max(n, 1), _p(C), max(m, 1), int(bool(lower)))
    return C


def logdet(A):
    """log det A = 2 sum_i log L_ii from the textbook factor of an SPD A
    (the GP log-likelihood term of the GP use of Sec. 4.1).  Returns
    (logdet, info); logdet is NaN when info != 0."""
    A = _fmat(A)
    n = A.shape[0]
    out = ctypes.c_double(0.0)
    info = lib().or_logdet(n, _p(A), max(n, 1), ctypes.byref(out))
    return float(out.value), int(info)


def predict_mean(Xs, X, sf2: float, ell: float, alpha):
    """GP predictive mean K(Xs, X) alpha with the noise-free SE cross
    covariance (GP behaviour prediction, Sec. 4.1).  Xs: m x d, X: n x d,
    alpha: n or n x nrhs.  Returns m or m x nrhs."""
    Xs = np.ascontiguousarray(Xs, dtype=np.float64)
    X = np.ascontiguousarray(X, dtype=np.float64)
    a = np.asarray(alpha, dtype=np.float64)
    vec = a.ndim == 1
    a2 = _fmat(a.reshape(-1, 1) if vec else a)
    m, d = Xs.shape
    n = X.shape[0]
    nrhs = a2.shape[1]
    out = np.zeros((m, nrhs), dtype=np.float64, order="F")
    lib().or_predict_mean(m, n, d, _p(Xs), _p(X), sf2, ell, _p(a2), max(n, 1), nrhs, _p(out), max(m, 1))
    return out[:, 0].copy() if vec else out


def pcg(A, Lt, b, bwd_tol: float = 1e-12, eps: float = 1e-13, maxit: int = 500, R: int = 50, x0=None):
    """Preconditioned CG with M = Lt Lt^T (refined solve).  Returns
    (x, iterations, backward_error); iterations < 0 if not converged."""
    A = _fmat(A)
    Lt = _fmat(Lt)
    n = A.shape[0]
    b = np.ascontiguousarray(b, dtype=np.float64)
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    be = ctypes.c_double(0.0)
    it = lib().or_pcg(n, _p(A), max(n, 1), _p(Lt), max(n, 1), _p(b), _p(x), bwd_tol, eps, maxit, R,
                      ctypes.byref(be))
    return x, int(it), float(be.value)


def solve_spd(A, B):
    """x = A^-1 b for an SPD A through LAPACK's Cholesky factor and solve
    (scipy.linalg.cho_factor / cho_solve): a library routine standing in for
    factor() + chol_solve() as the reference solution at sizes where the
    textbook loops take minutes (n >= 8192)."""
    import scipy.linalg
    c = scipy.linalg.cho_factor(np.asarray(A, dtype=np.float64), lower=True, check_finite=False)
    return scipy.linalg.cho_solve(c, np.asarray(B, dtype=np.float64), check_finite=False)


def backward_error(A, x, b) -> float:
    """||Ax-b||_inf / (||A||_inf ||x||_inf + ||b||_inf), long-double residual."""
    A = _fmat(A)
    n = A.shape[0]
    x = np.ascontiguousarray(x, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    return float(lib().or_backward_error(n, _p(A), max(n, 1), _p(x), _p(b)))


def factor_error(L, Lref) -> float:
    """||L - Lref||_F / ||Lref||_F over the lower triangle."""
    L = np.tril(np.asarray(L, dtype=np.float64))
    Lref = np.tril(np.asarray(Lref, dtype=np.float64))
    return float(np.linalg.norm(L - Lref) / np.linalg.norm(Lref))


def forward_error(x, xref) -> float:
    """||x - xref||_2 / ||xref||_2."""
    x = np.asarray(x, dtype=np.float64)
    xref = np.asarray(xref, dtype=np.float64)
    return float(np.linalg.norm(x - xref) / np.linalg.norm(xref))
