"""Pins for the FP64 oracle, against facts fixed by the paper and by
mathematics rather than by the oracle itself: hand-derived closed forms
(tests/golden/closed_forms.json), exact integer factorizations, brute force on
tiny inputs, invariants, and library routines for special cases.

Paper passages: Algorithm 1 (left: CG; right: blocked right-looking
Cholesky), Sec. 2.1 (residual replacement), Sec. 2.2 (L L^T = A, forward and
back substitution)."""
import json
import os

import numpy as np
import pytest
import sympy

import oracle
from paper_2605_13209_b300 import inputs

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "closed_forms.json")))
U = np.finfo(np.float64).eps / 2


def ev(s):
    return float(sympy.N(sympy.sympify(s), 30))


def evm(rows):
    return np.array([[ev(x) for x in r] for r in rows])


def int_lower(n, rng, unit=False, lo=-3, hi=4):
    """Random lower-triangular integer matrix with positive diagonal."""
    L = np.tril(rng.integers(lo, hi, (n, n))).astype(np.float64)
    d = np.ones(n) if unit else rng.integers(1, 5, n).astype(np.float64)
    np.fill_diagonal(L, d)
    return L


# ---------------------------------------------------------------- Cholesky
def test_chol_closed_form_i_plus_vvt():
    g = GOLD["chol_i_plus_vvt"]
    v = np.array([ev(x) for x in g["v"]])
    A = np.eye(3) + np.outer(v, v)
    L, info = oracle.cholesky(A)
    assert info == 0
    np.testing.assert_allclose(L, evm(g["L"]), rtol=4 * U, atol=4 * U)
    Lb, info = oracle.blocked_cholesky(A, 2)
    np.testing.assert_allclose(Lb, evm(g["L"]), rtol=4 * U, atol=4 * U)


@pytest.mark.parametrize("n", [1, 2, 5, 17, 40])
def test_chol_exact_integer_factor(n):
    """A = L0 L0^T with small integers: every intermediate is an integer, so
    the factor must come back bit-exact (catches any index/transpose slip)."""
    rng = np.random.default_rng(n)
    L0 = int_lower(n, rng)
    A = L0 @ L0.T
    L, info = oracle.cholesky(A)
    assert info == 0
    assert np.array_equal(L, L0)
    for b in (1, 3, 8):
        Lb, info = oracle.blocked_cholesky(A, b)
        assert info == 0 and np.array_equal(Lb, L0), b


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8])
def test_chol_brute_force_small(n):
    rng = np.random.default_rng(100 + n)
    X = rng.random((n, 8))
    A = oracle.se_matrix(X, 1.0, 0.5, 1e-2)
    L, info = oracle.cholesky(A)
    assert info == 0
    assert np.all(np.triu(L, 1) == 0) and np.all(np.diag(L) > 0)
    # entrywise brute force: (L L^T)_ij = sum_k L_ik L_jk
    for i in range(n):
        for j in range(n):
            s = sum(L[i, k] * L[j, k] for k in range(n))
            assert abs(s - A[i, j]) <= 8 * U * np.abs(A).max() * n
    Lb, info = oracle.blocked_cholesky(A, 3)
    assert info == 0 and np.max(np.abs(Lb - L)) <= 16 * U * n


def test_chol_diagonal():
    a = np.array([4.0, 9.0, 2.0, 0.25])
    L, info = oracle.cholesky(np.diag(a))
    assert info == 0
    np.testing.assert_array_equal(L, np.diag(np.sqrt(a)))


def test_chol_not_spd_info():
    A = np.array([[1.0, 2.0], [2.0, 1.0]])  # eigenvalues 3, -1: column 2 fails
    _, info = oracle.cholesky(A)
    assert info == 2
    A3 = np.diag([1.0, 1.0, -1.0])
    assert oracle.cholesky(A3)[1] == 3
    assert oracle.blocked_cholesky(A3, 2)[1] == 3
    An = np.diag([1.0, np.nan])
    assert oracle.cholesky(An)[1] == 2


def test_chol_matches_lapack_se():
    """Special case that reduces to a library routine: numpy's LAPACK potrf."""
    sysm = inputs.gp_system(300, 8, 0.5, 1e-2, seed=7)
    A = oracle.se_matrix(sysm.X, sysm.sf2, sysm.ell, sysm.sn2)
    L, info = oracle.cholesky(A)
    assert info == 0
    assert oracle.factor_error(L, np.linalg.cholesky(A)) < 1e-12
    Lb, _ = oracle.blocked_cholesky(A, 64)
    assert oracle.factor_error(Lb, L) < 1e-12


def test_chol_upper_untouched():
    rng = np.random.default_rng(3)
    L0 = int_lower(6, rng)
    A = L0 @ L0.T
    A[np.triu_indices(6, 1)] = 777.0  # upper triangle is not referenced
    M = np.asfortranarray(A.copy())
    info = oracle.lib().or_cholesky(6, oracle._p(M), 6)
    assert info == 0
    assert np.all(M[np.triu_indices(6, 1)] == 777.0)
    assert np.array_equal(np.tril(M), L0)


# ------------------------------------------------------ low-precision factor
def test_round_bf16_matches_torch():
    import torch
    rng = np.random.default_rng(5)
    vals = np.concatenate([rng.standard_normal(2000) * 10.0 ** rng.integers(-6, 6, 2000),
                           [0.0, -0.0, 1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, 1.0 + 2 ** -7 + 2 ** -8,
                            65504.0, 1e-30, -3.0e38]])
    f32 = vals.astype(np.float32)
    ref = torch.from_numpy(f32).to(torch.bfloat16).to(torch.float64).numpy()
    got = np.array([oracle.round_bf16(float(v)) for v in f32])
    np.testing.assert_array_equal(got, ref)
    assert oracle.round_bf16(1.0 + 2 ** -8) == 1.0          # tie -> even
    assert oracle.round_bf16(1.0 + 3 * 2 ** -8) == 1.0 + 2 ** -6   # tie -> even (up)


def test_round_f16_matches_numpy():
    """IEEE binary16 round-to-nearest-even, against numpy's float16
    conversion (normals, subnormals, ties, overflow)."""
    rng = np.random.default_rng(6)
    vals = np.concatenate([rng.standard_normal(3000) * 10.0 ** rng.integers(-9, 5, 3000),
                           [0.0, -0.0, 1.0, 1.0 + 2 ** -11, 1.0 + 3 * 2 ** -11, 2.0 ** -24, 2.0 ** -25,
                            3 * 2.0 ** -26, 2.0 ** -14, 2.0 ** -14 - 2.0 ** -25, 65504.0, 65519.99, 65520.0,
                            -70000.0, 1e-9]])
    with np.errstate(over="ignore"):
        ref = vals.astype(np.float16).astype(np.float64)
    got = np.array([oracle.round_f16(float(v)) for v in vals])
    np.testing.assert_array_equal(got, ref)
    assert oracle.round_f16(1.0 + 2 ** -11) == 1.0                  # tie -> even
    assert oracle.round_f16(1.0 + 3 * 2 ** -11) == 1.0 + 2 ** -9    # tie -> even (up)
    assert oracle.round_f16(2.0 ** -25) == 0.0                      # half the smallest subnormal -> 0


def test_mixed_factor_exact_on_representable_input():
    """Unit-diagonal integer factor: every operand is exact in bfloat16 and
    every product sum is exact, so every mode must return L0 exactly."""
    rng = np.random.default_rng(11)
    L0 = int_lower(24, rng, unit=True, lo=-2, hi=3)
    A = L0 @ L0.T
    for mode in ("fp32", "bf16", "split_bf16", "split_f16"):
        Lt, info = oracle.mixed_factor(A, 8, mode)
        assert info == 0 and np.array_equal(Lt, L0), mode


def test_mixed_factor_error_ordering():
    sysm = inputs.gp_system(192, 8, 0.5, 1e-1, seed=9)
    A = oracle.se_matrix(sysm.X, sysm.sf2, sysm.ell, sysm.sn2)
    L, _ = oracle.cholesky(A)
    errs = {}
    for mode in ("fp32", "split_f16", "split_bf16", "bf16"):
        Lt, info = oracle.mixed_factor(A, 64, mode)
        assert info == 0
        errs[mode] = oracle.factor_error(Lt, L)
    assert errs["fp32"] < 1e-5
    assert errs["fp32"] < errs["split_bf16"] < errs["bf16"] < 0.5
    assert errs["bf16"] > 1e-4   # bfloat16 products really are rounded
    # a scaled binary16 head + tail carries ~22 bits against ~16 for bfloat16
    assert errs["split_f16"] < errs["split_bf16"] / 4 and errs["split_f16"] < 1e-5


def test_mixed_factor_shift():
    """A + delta I is what the shifted factor factors."""
    rng = np.random.default_rng(12)
    L0 = int_lower(10, rng, unit=True, lo=-1, hi=2)
    A = L0 @ L0.T
    Lt, info = oracle.mixed_factor(A - 0.5 * np.eye(10), 4, "fp32", shift=0.5)
    assert info == 0 and np.array_equal(Lt, L0)


# ----------------------------------------------------------- substitution
@pytest.mark.parametrize("n", [1, 7, 33])
def test_substitution_exact_integer(n):
    rng = np.random.default_rng(20 + n)
    L0 = int_lower(n, rng, unit=True)
    x = rng.integers(-5, 6, (n, 3)).astype(np.float64)
    np.testing.assert_array_equal(oracle.forward_sub(L0, L0 @ x), x)
    np.testing.assert_array_equal(oracle.back_sub(L0, L0.T @ x), x)


def test_solve_sherman_morrison():
    g = GOLD["chol_i_plus_vvt"]
    v = np.array([ev(x) for x in g["v"]])
    A = np.eye(3) + np.outer(v, v)
    b = np.array([ev(x) for x in g["b"]])
    L, _ = oracle.cholesky(A)
    x = oracle.chol_solve(L, b)
    np.testing.assert_allclose(x, [ev(s) for s in g["x_sherman_morrison"]], rtol=1e-14, atol=1e-15)


def test_solve_diagonal():
    a = np.array([4.0, 16.0, 0.25])   # perfect squares: sqrt and both divisions exact
    b = np.array([1.0, 1.0, 1.0])
    L, _ = oracle.cholesky(np.diag(a))
    np.testing.assert_array_equal(oracle.chol_solve(L, b), b / a)


def test_solve_matches_library():
    sysm = inputs.gp_system(200, 8, 0.5, 1e-2, nrhs=2, seed=8)
    A = oracle.se_matrix(sysm.X, sysm.sf2, sysm.ell, sysm.sn2)
    L, _ = oracle.cholesky(A)
    X = oracle.chol_solve(L, sysm.B)
    ref = np.linalg.solve(A, sysm.B)
    assert oracle.forward_error(X, ref) < 1e-9
    for r in range(2):
        assert oracle.backward_error(A, X[:, r], sysm.B[:, r]) < 1e-15


# ---------------------------------------------------------------- SE matrix
def test_se_two_points_closed_form():
    g = GOLD["se_two_points"]
    X = np.array([[ev(x) for x in g["x0"]], [ev(x) for x in g["x1"]]])
    K = oracle.se_matrix(X, ev(g["sf2"]), ev(g["ell"]), ev(g["sn2"]))
    np.testing.assert_allclose(K, evm(g["K"]), rtol=4 * U)


def test_se_structure():
    X = inputs.points(64, 8, 3)
    K = oracle.se_matrix(X, 1.5, 0.4, 1e-3)
    assert np.array_equal(K, K.T)
    assert np.all(np.diag(K) == 1.5 + 1e-3)
    assert np.all(K[~np.eye(64, dtype=bool)] < 1.5)
    # far-apart points: K -> (sf2 + sn2) I
    Xf = np.arange(5)[:, None] * np.ones((1, 8)) * 100.0
    Kf = oracle.se_matrix(Xf, 2.0, 0.5, 0.1)
    np.testing.assert_array_equal(Kf, 2.1 * np.eye(5))
    # entry function agrees with the matrix
    for i, j in [(0, 0), (3, 7), (63, 1)]:
        assert oracle.se_entry(X[i], X[j], i == j, 1.5, 0.4, 1e-3) == K[i, j]


# ---------------------------------------------------------------------- CG
def test_cg_first_step_by_hand():
    g = GOLD["cg_first_step"]
    A = evm(g["A"])
    b = np.array([ev(x) for x in g["b"]])
    x1, it, _ = oracle.cg(A, b, 1e-14, 1, R=0)
    assert it == 1
    np.testing.assert_allclose(x1, [ev(s) for s in g["x1"]], rtol=4 * U)
    x, it, rr = oracle.cg(A, b, 1e-12, 50, R=0)
    assert it == g["iterations"]
    np.testing.assert_allclose(x, [ev(s) for s in g["x"]], rtol=1e-14)


def test_cg_diag_three_eigenvalues():
    g = GOLD["cg_diag_123"]
    A = np.diag([ev(x) for x in g["diag"]])
    x, it, rr = oracle.cg(A, np.array([ev(s) for s in g["b"]]), 1e-12, 100, R=0)
    assert it == g["iterations"]
    np.testing.assert_allclose(x, [ev(s) for s in g["x"]], rtol=1e-14)


def test_cg_scaled_identity_one_step():
    b = inputs.rhs(50, 1, 1)[:, 0]
    x, it, rr = oracle.cg(3.0 * np.eye(50), b, 1e-12, 100)
    assert it == 1
    np.testing.assert_allclose(x, b / 3.0, rtol=4 * U)


@pytest.mark.parametrize("k", [2, 5, 9])
def test_cg_k_distinct_eigenvalues(k):
    """A = Q diag(lambda) Q^T, Q a Householder reflector (closed form), with
    k distinct eigenvalues: CG ends within k iterations (exact arithmetic),
    here within k + 1 at eps = 1e-10."""
    n = 60
    rng = np.random.default_rng(k)
    w = rng.standard_normal(n)
    Q = np.eye(n) - 2.0 * np.outer(w, w) / (w @ w)
    lam = np.repeat(np.linspace(1.0, 4.0, k), int(np.ceil(n / k)))[:n]
    A = Q @ np.diag(lam) @ Q.T
    A = 0.5 * (A + A.T)
    b = rng.standard_normal(n)
    x, it, rr = oracle.cg(A, b, 1e-10, 1000, R=0)
    assert it <= k + 1 and rr <= 1e-10
    np.testing.assert_allclose(x, Q @ ((Q.T @ b) / lam), rtol=1e-8, atol=1e-10)


def test_cg_residual_replacement():
    sysm = inputs.gp_system(120, 8, 0.5, 1e-1, seed=4)
    A = oracle.se_matrix(sysm.X, sysm.sf2, sysm.ell, sysm.sn2)
    b = sysm.B[:, 0]
    ref = np.linalg.solve(A, b)
    for R in (0, 1, 7, 50):
        x, it, rr = oracle.cg(A, b, 1e-10, 5000, R=R)
        assert rr <= 1e-10, R
        true_rel = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
        assert true_rel <= 1e-9, R
        assert oracle.forward_error(x, ref) < 1e-6
    # with R = 1 the recurrence residual *is* the true residual each step
    x, it, rr = oracle.cg(A, b, 1e-10, 5000, R=1)
    assert abs(np.linalg.norm(b - A @ x) / np.linalg.norm(b) - rr) <= 1e-14


def test_cg_maxit_and_start_vector():
    sysm = inputs.gp_system(80, 8, 0.5, 1e-2, seed=5)
    A = oracle.se_matrix(sysm.X, sysm.sf2, sysm.ell, sysm.sn2)
    b = sysm.B[:, 0]
    x, it, rr = oracle.cg(A, b, 1e-14, 3)
    assert it == 3 and rr > 1e-14
    # start vector with an exactly zero residual: u0 = 0, the loop never runs
    x, it, rr = oracle.cg(2.0 * np.eye(4), 2.0 * np.ones(4), 1e-10, 10, x0=np.ones(4))
    assert it == 0 and np.array_equal(x, np.ones(4))


# ----------------------------------------------------------- metrics / PCG
def test_backward_error_closed_form():
    A = np.eye(4)
    b = np.ones(4)
    assert oracle.backward_error(A, b, b) == 0.0
    d = 1e-3
    x = b.copy()
    x[0] += d
    assert abs(oracle.backward_error(A, x, b) - d / (2 + d)) < 1e-16


def test_backward_error_nonsymmetric_hand_value():
    """A nonsymmetric 2 x 2 case worked by hand, where the usual slips give
    other values: A = [[1, 4], [2, 0]], x = (1, -2), b = (-6, 2.5).
    Ax - b = (-1, -0.5), so ||r||_inf = 1; ||A||_inf = 5 (row sums 5, 2),
    ||x||_inf = 2, ||b||_inf = 6, and the error is 1 / (5 * 2 + 6) = 1/16
    exactly.  The 1-norm of A would give 1/14, A^T x 3/16, ||x||_1 1/21 and
    a dropped ||b|| term 1/10."""
    A = np.array([[1.0, 4.0], [2.0, 0.0]])
    x = np.array([1.0, -2.0])
    b = np.array([-6.0, 2.5])
    assert oracle.backward_error(A, x, b) == 1.0 / 16.0


def test_pcg_iterates_equal_cg_on_the_transformed_system():
    """Preconditioned CG with M = L L^T on A x = b is CG on the transformed
    system (L^-1 A L^-T) y = L^-1 b with x = L^-T y, iterate by iterate.
    With no stop test and no residual replacement (bwd_tol = eps = 0,
    R = 0) both run exactly k steps; x_k and L^-T y_k must agree to
    rounding for k = 1..4 and a general (non-diagonal) L.  A beta from
    r^T r instead of r^T z, M^-1 applied as L^-1 alone, or a search
    direction built from r instead of z each break the agreement (checked
    by planting each slip in a copy of the oracle)."""
    rng = np.random.default_rng(17)
    n = 8
    G = rng.standard_normal((n, n))
    A = G @ G.T + n * np.eye(n)
    L = np.tril(rng.standard_normal((n, n)) * 0.3) + np.diag(1.0 + rng.random(n))
    b = rng.standard_normal(n)
    Li = np.linalg.inv(L)
    Ah = Li @ A @ Li.T
    Ah = 0.5 * (Ah + Ah.T)
    bh = Li @ b
    for k in range(1, 5):
        x, it, _ = oracle.pcg(A, L, b, bwd_tol=0.0, eps=0.0, maxit=k, R=0)
        y, itc, _ = oracle.cg(Ah, bh, 0.0, k, R=0)
        assert it == -k and itc == k
        xr = Li.T @ y
        assert np.abs(x - xr).max() <= 1e-11 * np.abs(xr).max()


def test_pcg_exact_preconditioner_one_step():
    sysm = inputs.gp_system(100, 8, 0.5, 1e-2, seed=6)
    A = oracle.se_matrix(sysm.X, sysm.sf2, sysm.ell, sysm.sn2)
    L, _ = oracle.cholesky(A)
    x, it, be = oracle.pcg(A, L, sysm.B[:, 0], 1e-12)
    assert it == 1 and be <= 1e-12


def test_pcg_low_precision_preconditioner():
    sysm = inputs.gp_system(256, 8, 0.5, 1e-3, seed=10)
    A = oracle.se_matrix(sysm.X, sysm.sf2, sysm.ell, sysm.sn2)
    b = sysm.B[:, 0]
    Lt, info = oracle.mixed_factor(A, 64, "split_bf16")
    assert info == 0
    x, it, be = oracle.pcg(A, Lt, b, 1e-12)
    assert 1 <= it <= 30 and be <= 1e-12
    _, it_cg, _ = oracle.cg(A, b, 1e-10, 10000)
    assert it < it_cg
    ref = np.linalg.solve(A, b)
    assert oracle.forward_error(x, ref) < 1e-6


def test_solve_spd_matches_textbook_solve():
    """The LAPACK reference solve agrees with the textbook factor and
    substitutions to within the conditioning of the system."""
    s = inputs.gp_system(300, 8, 0.5, 1e-2, nrhs=2, seed=11)
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    L, info = oracle.cholesky(A)
    assert info == 0
    x_ref = oracle.chol_solve(L, s.B)
    x = oracle.solve_spd(A, s.B)
    kappa = np.linalg.cond(A)
    for r in range(2):
        assert oracle.forward_error(x[:, r], x_ref[:, r]) <= 50 * kappa * U


# -------------------------------------------------- single-reduction CG (f2)
def test_cg_single_reduction_first_step_by_hand():
    """Same hand-worked first iteration as classic CG: r = b, w = A r =
    (6, 7), gamma = 5, delta = w^T r = 20, alpha = 1/4, p = r, x_1 = r / 4;
    two distinct eigenvalues, so the second iteration is exact."""
    g = GOLD["cg_first_step"]
    A = evm(g["A"])
    b = np.array([ev(x) for x in g["b"]])
    x1, it, _ = oracle.cg_single_reduction(A, b, 1e-14, 1, R=0)
    assert it == 1
    np.testing.assert_allclose(x1, [ev(s) for s in g["x1"]], rtol=4 * U)
    x, it, _ = oracle.cg_single_reduction(A, b, 1e-14, 50, R=0)
    assert it == g["iterations"]
    np.testing.assert_allclose(x, [ev(s) for s in g["x"]], rtol=1e-14)


def test_cg_single_reduction_diag_three_eigenvalues():
    g = GOLD["cg_diag_123"]
    A = np.diag([ev(x) for x in g["diag"]])
    b = np.array([ev(x) for x in g["b"]])
    x, it, _ = oracle.cg_single_reduction(A, b, 1e-14, 50, R=0)
    assert it == g["iterations"]
    np.testing.assert_allclose(x, [ev(s) for s in g["x"]], rtol=1e-14)


def test_cg_single_reduction_scaled_identity_one_step():
    b = np.array([1.0, -2.0, 3.0, 0.5])
    x, it, rr = oracle.cg_single_reduction(4.0 * np.eye(4), b, 1e-12, 10, R=0)
    assert it == 1 and rr == 0.0
    np.testing.assert_array_equal(x, b / 4.0)


@pytest.mark.parametrize("k", [2, 5, 9])
def test_cg_single_reduction_k_distinct_eigenvalues(k):
    """Householder Q diag(lambda) Q^T with k distinct eigenvalues: the Krylov
    space is exhausted after k steps, so the residual reaches rounding level
    by iteration k (one more allowed for rounding)."""
    rng = np.random.default_rng(300 + k)
    n = 40
    v = rng.standard_normal(n)
    Q = np.eye(n) - 2.0 * np.outer(v, v) / (v @ v)
    lam = np.repeat(np.linspace(1.0, 10.0, k), int(np.ceil(n / k)))[:n]
    A = Q @ np.diag(lam) @ Q.T
    A = 0.5 * (A + A.T)
    b = rng.standard_normal(n)
    x, it, rr = oracle.cg_single_reduction(A, b, 1e-12, 200, R=0)
    assert it <= k + 1
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) < 1e-11


def test_cg_single_reduction_iterates_equal_classic():
    """The rearrangement changes no iterate in exact arithmetic: on a
    well-conditioned SE system, after every iteration count j the two
    algorithms' x agree to rounding level (a wrong beta, a stale alpha in
    the delta - beta gamma / alpha correction, or s not tracking A p breaks
    this at the second iteration)."""
    sysm = inputs.gp_system(120, 8, 0.5, 0.5, seed=31)
    A = oracle.se_matrix(sysm.X, sysm.sf2, sysm.ell, sysm.sn2)
    b = sysm.B[:, 0]
    for j in (1, 2, 3, 5, 8):
        xc, itc, _ = oracle.cg(A, b, 0.0, j, R=0)
        xs, its, _ = oracle.cg_single_reduction(A, b, 0.0, j, R=0)
        assert itc == its == j
        assert oracle.forward_error(xs, xc) < 1e-12, j


def test_cg_single_reduction_replacement_and_convergence():
    """With replacement every 7 iterations the recurrence residual tracks
    the true one, and the stop rule (relative recurrence residual <= eps)
    holds for the true residual too."""
    sysm = inputs.gp_system(200, 8, 0.5, 1e-2, seed=32)
    A = oracle.se_matrix(sysm.X, sysm.sf2, sysm.ell, sysm.sn2)
    b = sysm.B[:, 0]
    x, it, rr = oracle.cg_single_reduction(A, b, 1e-10, 5000, R=7)
    assert rr <= 1e-10
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) < 1e-9
    _, itc, _ = oracle.cg(A, b, 1e-10, 5000, R=7)
    assert abs(it - itc) <= max(3, 0.05 * itc)


# ------------------------------------------------------- GP quantities (f3)
def test_logdet_hand_2x2():
    g = GOLD["logdet_2x2"]
    val, info = oracle.logdet(evm(g["A"]))
    assert info == 0
    assert abs(val - ev(g["logdet"])) <= 8 * U * abs(ev(g["logdet"]))


def test_logdet_determinant_lemma():
    g = GOLD["logdet_i_plus_vvt"]
    v = np.array([ev(x) for x in g["v"]])
    val, info = oracle.logdet(np.eye(3) + np.outer(v, v))
    assert info == 0
    assert abs(val - ev(g["logdet"])) <= 16 * U * abs(ev(g["logdet"]))
    # a longer v: log(1 + v^T v), the factor still of size 50
    rng = np.random.default_rng(41)
    w = rng.standard_normal(50)
    val, _ = oracle.logdet(np.eye(50) + np.outer(w, w))
    assert abs(val - np.log1p(w @ w)) < 1e-12 * abs(np.log1p(w @ w))


def test_logdet_diagonal_and_library():
    a = np.array([0.5, 3.0, 7.0, 1e-3])
    val, info = oracle.logdet(np.diag(a))
    assert info == 0 and abs(val - np.sum(np.log(a))) < 1e-14 * np.sum(np.abs(np.log(a)))
    sysm = inputs.gp_system(150, 8, 0.5, 1e-2, seed=42)
    A = oracle.se_matrix(sysm.X, sysm.sf2, sysm.ell, sysm.sn2)
    sign, ref = np.linalg.slogdet(A)
    val, _ = oracle.logdet(A)
    assert sign == 1.0 and abs(val - ref) < 1e-11 * abs(ref)


def test_logdet_not_spd():
    val, info = oracle.logdet(np.array([[1.0, 2.0], [2.0, 1.0]]))
    assert info == 2 and np.isnan(val)


def test_predict_mean_hand_1d():
    g = GOLD["gp_mean_1d"]
    X = np.array([[ev(x)] for x in g["X"]])
    Xs = np.array([[ev(x)] for x in g["Xs"]])
    alpha = np.array([ev(x) for x in g["alpha"]])
    got = oracle.predict_mean(Xs, X, ev(g["sf2"]), ev(g["ell"]), alpha)
    np.testing.assert_allclose(got, [ev(s) for s in g["mean"]], rtol=8 * U)


def test_predict_mean_at_training_points():
    """With alpha = (K + sn2 I)^-1 y the mean at the training points is
    K alpha = y - sn2 alpha (the noise term is in the system, not in the
    cross covariance): a dropped sf2, a wrong length scale (ell^2 for
    2 ell^2), a transposed cross covariance or an added noise term each
    break it."""
    sysm = inputs.gp_system(180, 8, 0.5, 1e-1, nrhs=2, seed=43)
    A = oracle.se_matrix(sysm.X, 1.7, sysm.ell, sysm.sn2)
    alpha = np.linalg.solve(A, sysm.B)
    mean = oracle.predict_mean(sysm.X, sysm.X, 1.7, sysm.ell, alpha)
    np.testing.assert_allclose(mean, sysm.B - sysm.sn2 * alpha, rtol=0, atol=1e-11 * np.abs(sysm.B).max())


def test_predict_mean_far_point_and_columns():
    sysm = inputs.gp_system(40, 8, 0.5, 1e-2, nrhs=3, seed=44)
    far = np.full((1, 8), 1e3)
    np.testing.assert_array_equal(oracle.predict_mean(far, sysm.X, 1.0, 0.5, sysm.B), np.zeros((1, 3)))
    Xs = inputs.points(7, 8, 45)
    both = oracle.predict_mean(Xs, sysm.X, 1.0, 0.5, sysm.B)
    for r in range(3):
        np.testing.assert_array_equal(both[:, r], oracle.predict_mean(Xs, sysm.X, 1.0, 0.5, sysm.B[:, r]))


# --------------------------------------------- long-double GEMM update (f1)
def test_gemm_update_exact_rationals():
    """Against exact rational arithmetic: C - A B^T entry by entry, rounded
    once to FP64 (long double sums of 12 products carry no error here)."""
    from fractions import Fraction
    rng = np.random.default_rng(61)
    A = rng.standard_normal((5, 12)) * np.exp(rng.uniform(-20, 5, (5, 12)))
    B = rng.standard_normal((4, 12))
    C = rng.standard_normal((5, 4))
    got = oracle.gemm_update(C, A, B)
    for i in range(5):
        for j in range(4):
            ex = Fraction(C[i, j]) - sum(Fraction(A[i, c]) * Fraction(B[j, c]) for c in range(12))
            assert abs(Fraction(got[i, j]) - ex) <= abs(ex) * Fraction(2) ** -52 + Fraction(2) ** -1070


def test_gemm_update_lower_and_library():
    rng = np.random.default_rng(62)
    P = rng.standard_normal((30, 17))
    C = rng.standard_normal((30, 30))
    got = oracle.gemm_update(C, P, P, lower=True)
    ref = C - P @ P.T
    low = np.tril(np.ones((30, 30), dtype=bool))
    np.testing.assert_allclose(got[low], ref[low], rtol=1e-13, atol=1e-13)
    np.testing.assert_array_equal(got[~low], C[~low])      # upper entries untouched
