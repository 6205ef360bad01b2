"""GPU parity of the FP64-accurate tensor-core product (gpch_gemm_fp64_emulated,
Algorithm 1 step 3 as C -= A B^T) against the oracle's long-double update.

The bound per entry is the splitting's: k 2^-47 2^(e_i + f_j), with 2^e_i
and 2^f_j the powers of two just above the largest |entry| of row i of A
and row j of B, plus FP64 rounding of C; a wrong digit, a dropped class,
a wrong class weight or a lost carry is far above it."""
import math
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
from paper_2605_13209_b300 import gpchol, inputs
from gpu_helpers import ctx, dev, host  # noqa: F401

pytestmark = pytest.mark.gpu


def _scale(X):
    mx = np.abs(X).max(axis=1)
    return np.array([math.ldexp(1.0, math.frexp(v)[1]) if v > 0 else 0.0 for v in mx])


def _check(got, ref, A, B, C, lower=False):
    k = A.shape[1]
    bound = k * 2.0 ** -47 * np.outer(_scale(A), _scale(B)) + 4 * 2.0 ** -53 * (np.abs(C) + np.abs(A) @ np.abs(B).T)
    bound += 1e-300
    err = np.abs(got - ref)
    if lower:
        low = np.tril(np.ones_like(got, dtype=bool))
        assert np.array_equal(got[~low], C[~low])         # strict upper triangle untouched
        err = np.where(low, err, 0.0)
    assert np.all(err <= bound), float(np.max(err / bound))


@pytest.mark.parametrize("m,n,k", [(1, 1, 1), (64, 64, 32), (130, 70, 100), (300, 257, 512), (257, 129, 1100),
                                   (128, 64, 513), (1000, 900, 64)])
def test_emulated_gemm_parity(ctx, m, n, k):
    rng = np.random.default_rng(m * 7 + n * 3 + k)
    A = rng.standard_normal((m, k)) * np.exp(rng.uniform(-20, 0, (m, k)))
    B = rng.standard_normal((n, k)) * np.exp(rng.uniform(-20, 0, (n, k)))
    C = rng.standard_normal((m, n))
    ref = oracle.gemm_update(C, A, B)
    Cd = dev(C)
    gpchol.gemm_fp64_emulated(dev(A), dev(B), Cd, ctx=ctx)
    _check(host(Cd), ref, A, B, C)


@pytest.mark.parametrize("m,k", [(64, 512), (200, 300), (700, 512), (1300, 1024)])
def test_emulated_syrk_lower(ctx, m, k):
    """The SYRK case of step 3: A = B, only the lower triangle of C."""
    rng = np.random.default_rng(m + k)
    P = rng.standard_normal((m, k))
    C = rng.standard_normal((m, m))
    ref = oracle.gemm_update(C, P, P, lower=True)
    Pd = dev(P)
    Cd = dev(C)
    gpchol.gemm_fp64_emulated(Pd, Pd, Cd, lower=True, ctx=ctx)
    _check(host(Cd), ref, P, P, C, lower=True)


def test_emulated_gemm_exact_at_the_largest_digits(ctx):
    """Entries whose digits are the extreme ones (-64 below the top digit,
    -31 on top) make the class sums near 2^24 over k = 512 (class 7:
    14.6e6); the result must still be the kept pairs' exact sum rounded
    once."""
    N = -31 * 128 ** 7 - 64 * sum(128 ** p for p in range(7))
    assert abs(N) < 2 ** 54 and float(N) == N
    v = math.ldexp(float(N), -54)           # row scale 2^0: |v| < 1
    k = 512
    A = np.full((128, k), v)
    B = np.full((64, k), v)
    C = np.zeros((128, 64))
    Cd = dev(C)
    gpchol.gemm_fp64_emulated(dev(A), dev(B), Cd, ctx=ctx)
    got = host(Cd)
    exact = -(Fraction(v) * Fraction(v) * k)
    kept = Fraction(0)
    digits = [-31] + [-64] * 7
    for p in range(8):
        for q in range(8 - p):
            kept += Fraction(digits[p] * digits[q]) * Fraction(128) ** (14 - p - q)
    kept_val = -float(kept * k * Fraction(2) ** -108)
    assert np.all(got == kept_val)                    # the kept pairs, exactly, rounded once
    assert abs(Fraction(kept_val) - exact) <= k * Fraction(2) ** -47


def test_emulated_gemm_special_rows(ctx):
    """A zero row, a row of subnormals, a row with one huge entry."""
    rng = np.random.default_rng(5)
    k = 96
    A = rng.standard_normal((70, k))
    A[3] = 0.0
    A[10] = 5e-310 * rng.standard_normal(k)
    A[20] = 0.0
    A[20, 17] = 1e250
    B = rng.standard_normal((40, k)) * 1e-40
    C = rng.standard_normal((70, 40))
    ref = oracle.gemm_update(C, A, B)
    Cd = dev(C)
    gpchol.gemm_fp64_emulated(dev(A), dev(B), Cd, ctx=ctx)
    got = host(Cd)
    _check(got, ref, A, B, C)
    assert np.array_equal(got[3], C[3])


def test_emulated_update_of_a_cholesky_panel(ctx):
    """Step 3 of Algorithm 1 on an SE system: the trailing update with the
    first 256-column panel of the factor, against the FP64 update."""
    s = inputs.gp_system(1024, 8, 0.5, 1e-3, seed=77)
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    L, _ = oracle.cholesky(A)
    P = np.ascontiguousarray(L[256:, :256])
    C = A[256:, 256:].copy()
    ref = oracle.gemm_update(C, P, P, lower=True)
    Pd, Cd = dev(P), dev(C)
    gpchol.gemm_fp64_emulated(Pd, Pd, Cd, lower=True, ctx=ctx)
    got = host(Cd)
    _check(got, ref, P, P, C, lower=True)
    low = np.tril(np.ones_like(got, dtype=bool))
    assert np.max(np.abs(got - ref)[low]) <= 1e-13 * np.max(np.abs(ref))


@pytest.mark.parametrize("n,tile", [(300, 64), (1000, 256), (2048, 512), (2500, 256)])
def test_cholesky_with_emulated_update(ctx, n, tile):
    """Algorithm 1 (right) with step 3 on the tensor-core product: L within
    1e-12 of the oracle's factor, the solve within 1e-13 backward error,
    the strict upper triangle untouched."""
    s = inputs.gp_system(n, 8, 0.5, 1e-2, nrhs=1, seed=1400 + n)
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    Lref, info = oracle.cholesky(A)
    assert info == 0
    Ad = dev(A)
    assert gpchol.chol_factor(Ad, tile=tile, ctx=ctx, update="fp64_emulated") == 0
    got = host(Ad)
    assert np.array_equal(np.triu(got, 1), np.triu(A, 1))
    assert oracle.factor_error(np.tril(got), Lref) <= 1e-12
    B = dev(s.B)
    gpchol.chol_solve(Ad, B, ctx=ctx)
    assert oracle.backward_error(A, host(B)[:, 0], s.B[:, 0]) <= 1e-13


def test_cholesky_emulated_update_not_spd(ctx):
    s = inputs.gp_system(700, 8, 0.5, 1e-2, seed=1500)
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    A[600, 600] = -1.0
    Ad = dev(A)
    info = gpchol.chol_factor(Ad, tile=256, ctx=ctx, update="fp64_emulated", raise_on_not_spd=False)
    assert info == 601
