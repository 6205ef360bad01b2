"""GPU parity of the FP64 path against the oracle: SE matrix (A1), blocked
Cholesky (A2-A4, Algorithm 1 right), substitution (A5), CG (A6-A7,
Algorithm 1 left).  Tolerances: 1e-12 relative in L and 1e-13 relative
backward error for the direct solve; CG to its relative residual rtol."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13209_b300 import gpchol, inputs
from gpu_helpers import ctx, dev, host  # noqa: F401

pytestmark = pytest.mark.gpu

L_TOL = 1e-12
BWD_TOL = 1e-13


def se_system(n, ell=0.5, sn2=1e-2, nrhs=1, seed=0):
    s = inputs.gp_system(n, 8, ell, sn2, nrhs=nrhs, seed=seed)
    return s, oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)


def int_lower_unit(n, rng):
    L = np.tril(rng.integers(-2, 3, (n, n))).astype(np.float64)
    np.fill_diagonal(L, 1.0)
    return L


# ------------------------------------------------------------------ A1
@pytest.mark.parametrize("n", [1, 7, 32, 33, 100, 257])
def test_se_matrix_parity(ctx, n):
    s = inputs.gp_system(n, 8, 0.4, 1e-3, seed=n)
    ref = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    A = gpchol.se_matrix(torch.from_numpy(s.X).cuda(), s.sf2, s.ell, s.sn2, ctx=ctx)
    torch.cuda.synchronize()
    got = host(A)
    assert np.array_equal(got, got.T)
    assert np.all(np.diag(got) == s.sf2 + s.sn2)
    np.testing.assert_allclose(got, ref, rtol=4e-15, atol=1e-300)


def test_se_matrix_lda_and_d(ctx):
    X = inputs.points(50, 3, 9)
    ref = oracle.se_matrix(X, 2.0, 0.7, 0.1)
    A = gpchol.colmajor(50, 50, ld=64)
    A.fill_(7.0)
    gpchol.se_matrix(torch.from_numpy(X).cuda(), 2.0, 0.7, 0.1, A=A, ctx=ctx)
    np.testing.assert_allclose(host(A), ref, rtol=4e-15)


# ------------------------------------------------------------------ A2-A4
@pytest.mark.parametrize("n,tile", [(1, 64), (2, 64), (7, 64), (63, 64), (64, 64), (65, 64), (130, 128),
                                    (255, 128), (256, 256), (257, 256), (600, 192), (1000, 256)])
def test_cholesky_parity(ctx, n, tile):
    _, A = se_system(n, seed=n)
    Lref, info = oracle.cholesky(A)
    assert info == 0
    Ad = dev(A)
    assert gpchol.chol_factor(Ad, tile=tile, ctx=ctx) == 0
    L = np.tril(host(Ad))
    assert np.all(np.diag(L) > 0)
    assert oracle.factor_error(L, Lref) <= L_TOL


@pytest.mark.parametrize("n,tile", [(40, 64), (200, 64), (300, 128)])
def test_cholesky_exact_integer(ctx, n, tile):
    """Unit-diagonal integer factor: every value on the GPU path (including
    the inverted diagonal blocks) is an exactly representable integer, so L
    must come back bit-exact."""
    L0 = int_lower_unit(n, np.random.default_rng(n))
    Ad = dev(L0 @ L0.T)
    assert gpchol.chol_factor(Ad, tile=tile, ctx=ctx) == 0
    assert np.array_equal(np.tril(host(Ad)), L0)


def test_cholesky_upper_untouched_and_lda(ctx):
    n = 150
    _, A = se_system(n, seed=3)
    Ad = gpchol.colmajor(n, n, ld=160)
    Ad.copy_(torch.from_numpy(A))
    iu = np.triu_indices(n, 1)
    Ad[iu] = float("nan")
    assert gpchol.chol_factor(Ad, tile=64, ctx=ctx) == 0
    got = host(Ad)
    assert np.all(np.isnan(got[iu]))
    Lref, _ = oracle.cholesky(A)
    assert oracle.factor_error(np.tril(got), Lref) <= L_TOL


@pytest.mark.parametrize("bad_col", [0, 5, 64, 100, 199])
def test_cholesky_not_spd_info(ctx, bad_col):
    n = 200
    _, A = se_system(n, sn2=1e-1, seed=4)
    A = A.copy()
    A[bad_col, bad_col] = -1.0
    _, info_ref = oracle.cholesky(A)
    Ad = dev(A)
    info = gpchol.chol_factor(Ad, tile=128, ctx=ctx, raise_on_not_spd=False)
    assert info == info_ref and info > 0


def test_cholesky_empty(ctx):
    A = gpchol.colmajor(0, 0)
    assert gpchol.chol_factor(A, tile=64, ctx=ctx) == 0


# ------------------------------------------------------------------ A5
@pytest.mark.parametrize("n,nrhs", [(1, 1), (63, 2), (64, 1), (65, 3), (257, 1), (1000, 16)])
def test_chol_solve_parity(ctx, n, nrhs):
    s, A = se_system(n, nrhs=nrhs, seed=10 + n)
    Lref, _ = oracle.cholesky(A)
    Xref = oracle.chol_solve(Lref, s.B)
    Ld = dev(Lref)
    Bd = dev(s.B)
    gpchol.chol_solve(Ld, Bd, ctx=ctx)
    X = host(Bd).reshape(n, nrhs)
    Xref = np.asarray(Xref).reshape(n, nrhs)
    for r in range(nrhs):
        assert oracle.backward_error(A, X[:, r], s.B[:, r]) <= BWD_TOL
        assert oracle.forward_error(X[:, r], Xref[:, r]) <= 1e-10


def test_chol_solve_exact_integer(ctx):
    rng = np.random.default_rng(77)
    L0 = int_lower_unit(150, rng)
    x = rng.integers(-4, 5, (150, 2)).astype(np.float64)
    Bd = dev(L0 @ (L0.T @ x))
    gpchol.chol_solve(dev(L0), Bd, ctx=ctx)
    assert np.array_equal(host(Bd), x)


def test_factor_then_solve_config1_scale(ctx):
    """n=2048, tile 256 (the small FP64 workload): L within 1e-12 of the
    oracle and backward error within 1e-13."""
    s = inputs.config1()
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    Lref, _ = oracle.cholesky(A)
    Ad = dev(A)
    assert gpchol.chol_factor(Ad, tile=256, ctx=ctx) == 0
    assert oracle.factor_error(np.tril(host(Ad)), Lref) <= L_TOL
    Bd = dev(s.B)
    gpchol.chol_solve(Ad, Bd, ctx=ctx)
    x = host(Bd)[:, 0]
    assert oracle.backward_error(A, x, s.B[:, 0]) <= BWD_TOL


# ------------------------------------------------------------------ A6-A7
@pytest.mark.parametrize("n,R", [(1, 50), (10, 50), (100, 50), (257, 7), (1000, 50), (1000, 1)])
def test_cg_parity(ctx, n, R):
    s, A = se_system(n, sn2=1e-2, seed=20 + n)
    b = s.B[:, 0]
    x_or, it_or, rr_or = oracle.cg(A, b, 1e-10, 20000, R=R)
    Xd = gpchol.colmajor(n, 1)
    Xd.zero_()
    res = gpchol.cg_solve(dev(A), dev(b), Xd, rtol=1e-10, maxit=20000, replace_every=R, ctx=ctx)
    x = host(Xd)[:, 0]
    assert res.converged == 1 and res.relres_max <= 1e-10
    true_rel = np.linalg.norm(b - A @ x) / np.linalg.norm(b)
    assert true_rel <= 1e-9
    # iterates differ only by rounding order: same outcome, near-equal counts
    assert abs(res.iterations - it_or) <= max(3, 0.05 * it_or)
    ref = np.linalg.solve(A, b)
    assert oracle.forward_error(x, ref) <= max(1e-6, 10 * oracle.forward_error(x_or, ref))


def test_cg_closed_form_three_eigenvalues(ctx):
    A = np.diag([1.0, 2.0, 3.0])
    Xd = gpchol.colmajor(3, 1)
    Xd.zero_()
    res = gpchol.cg_solve(dev(A), dev(np.ones(3)), Xd, rtol=1e-12, maxit=100, ctx=ctx)
    assert res.iterations == 3
    np.testing.assert_allclose(host(Xd)[:, 0], [1.0, 0.5, 1.0 / 3.0], rtol=1e-14)


@pytest.mark.parametrize("nrhs", [2, 3, 8, 16, 20])
def test_cg_multi_rhs(ctx, nrhs):
    n = 300
    s, A = se_system(n, sn2=5e-2, nrhs=nrhs, seed=30 + nrhs)
    Xd = gpchol.colmajor(n, nrhs)
    Xd.zero_()
    res = gpchol.cg_solve(dev(A), dev(s.B), Xd, rtol=1e-10, maxit=5000, ctx=ctx)
    assert res.converged == nrhs
    X = host(Xd)
    for r in range(nrhs):
        x_or, it_or, _ = oracle.cg(A, s.B[:, r], 1e-10, 5000)
        rel = np.linalg.norm(s.B[:, r] - A @ X[:, r]) / np.linalg.norm(s.B[:, r])
        assert rel <= 1e-9
        assert oracle.forward_error(X[:, r], x_or) <= 1e-6


def test_cg_f32_matrix(ctx):
    n = 400
    s, A = se_system(n, sn2=1e-1, seed=41)
    A32 = A.astype(np.float32)
    A32u = A32.astype(np.float64)          # the stored operator, widened exactly
    b = s.B[:, 0]
    x_or, _, _ = oracle.cg(A32u, b, 1e-10, 5000)
    Xd = gpchol.colmajor(n, 1)
    Xd.zero_()
    res = gpchol.cg_solve(dev(A32, torch.float32), dev(b), Xd, rtol=1e-10, maxit=5000, ctx=ctx)
    x = host(Xd)[:, 0]
    assert res.converged == 1
    assert np.linalg.norm(b - A32u @ x) / np.linalg.norm(b) <= 1e-9
    assert oracle.forward_error(x, x_or) <= 1e-7


def test_cg_not_converged_and_start_vector(ctx):
    n = 200
    s, A = se_system(n, sn2=1e-3, seed=42)
    b = s.B[:, 0]
    Xd = gpchol.colmajor(n, 1)
    Xd.zero_()
    res = gpchol.cg_solve(dev(A), dev(b), Xd, rtol=1e-14, maxit=5, ctx=ctx, raise_on_not_converged=False)
    assert res.status == gpchol.GPCH_NOT_CONVERGED and res.iterations == 5
    x5, it, _ = oracle.cg(A, b, 1e-14, 5)
    assert oracle.forward_error(host(Xd)[:, 0], x5) <= 1e-10
    # exact start: zero residual, no iteration
    Xd2 = dev(np.ones(4))
    res = gpchol.cg_solve(dev(2 * np.eye(4)), dev(2 * np.ones(4)), Xd2, rtol=1e-10, maxit=10, ctx=ctx)
    assert res.iterations == 0 and np.array_equal(host(Xd2)[:, 0], np.ones(4))


def test_cg_config1_scale(ctx):
    s = inputs.config1()
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    b = s.B[:, 0]
    x_or, it_or, _ = oracle.cg(A, b, 1e-10, 100000)
    Xd = gpchol.colmajor(2048, 1)
    Xd.zero_()
    res = gpchol.cg_solve(dev(A), dev(b), Xd, rtol=1e-10, maxit=100000, ctx=ctx)
    x = host(Xd)[:, 0]
    assert res.converged == 1
    assert abs(res.iterations - it_or) <= max(5, 0.05 * it_or)
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-9
