"""GPU parity of the mixed-precision path (A4 tensor-core update, A8 factor,
A9 refined solve).  The tensor-core update is compared with the same
product computed in FP64 from the bfloat16-rounded operands (rounding done by
the oracle's bf16 routine); the factor with the oracle's emulation of it;
the refined solve by its FP64 backward error (<= 1e-12) and its forward
error against the oracle's FP64 Cholesky solution."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13209_b300 import gpchol, inputs
from gpu_helpers import ctx, dev, host  # noqa: F401

pytestmark = pytest.mark.gpu

_round_bf16 = np.vectorize(oracle.round_bf16)
_round_f16 = np.vectorize(oracle.round_f16)


def bf16_split(P32):
    hi = _round_bf16(P32.astype(np.float64))
    lo = _round_bf16((P32.astype(np.float64) - hi).astype(np.float32).astype(np.float64))
    return hi, lo


def f16_split(P32):
    """Scaled binary16 head and tail: 2^e P with the largest |entry| in
    [2^14, 2^15) (e clamped to [-60, 60]); returns (hi, lo, e)."""
    mx = float(np.abs(P32).max())
    e = 0
    if mx > 0:
        e = int(min(60, max(-60, 14 - (np.frexp(mx)[1] - 1))))
    Ps = P32.astype(np.float64) * 2.0 ** e
    hi = _round_f16(Ps)
    lo = _round_f16(Ps - hi)
    return hi, lo, e


@pytest.mark.parametrize("m,k", [(1, 64), (100, 64), (128, 64), (129, 128), (300, 512), (512, 256), (700, 200)])
@pytest.mark.parametrize("prec", ["bf16", "split_bf16", "split_f16"])
def test_syrk_lowprec_parity(ctx, m, k, prec):
    rng = np.random.default_rng(m * 7 + k)
    P = (rng.standard_normal((m, k)) * 10.0 ** rng.integers(-3, 3)).astype(np.float32)
    C0 = rng.standard_normal((m, m)).astype(np.float32)
    if prec == "split_f16":
        hi, lo, e = f16_split(P)
        prod = (hi @ hi.T + hi @ lo.T + lo @ hi.T) * 2.0 ** (-2 * e)
        hi = hi * 2.0 ** -e
    else:
        hi, lo = bf16_split(P)
    if prec == "bf16":
        prod = hi @ hi.T
    elif prec == "split_bf16":
        prod = hi @ hi.T + hi @ lo.T + lo @ hi.T
    ref = C0.astype(np.float64) - prod
    Cd = dev(C0, torch.float32)
    gpchol.syrk_lowprec(dev(P, torch.float32), Cd, prec, ctx=ctx)
    got = host(Cd)
    il = np.tril_indices(m)
    iu = np.triu_indices(m, 1)
    # FP32 accumulation of k exact products: |err| <= k * 2^-24 * sum|terms|
    bound = 4 * k * 2.0 ** -24 * (np.abs(hi) @ np.abs(hi).T * (1 if prec == "bf16" else 3) + np.abs(C0)) + 1e-30
    assert np.all(np.abs(got[il] - ref[il]) <= bound[il])
    assert np.array_equal(got[iu], C0.astype(np.float64)[iu])   # upper triangle untouched


@pytest.mark.parametrize("n,tile", [(64, 64), (200, 64), (513, 128), (1000, 256), (777, 192), (1100, 320)])
@pytest.mark.parametrize("prec", ["bf16", "split_bf16", "split_f16"])
def test_mixed_factor_vs_emulation(ctx, n, tile, prec):
    # tiles that are not multiples of the 128-column tensor-core tile (64,
    # 192, 320) exercise the column limit of the block-column updates
    s = inputs.gp_system(n, 8, 0.5, 1e-1, seed=n)
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    Lexact, _ = oracle.cholesky(A)
    Lemu, info = oracle.mixed_factor(A, tile, prec)
    assert info == 0
    L, info = gpchol.chol_factor_mixed(dev(A), prec, tile, ctx=ctx)
    assert info == 0
    Lg = np.tril(host(L))
    e_gpu = oracle.factor_error(Lg, Lexact)
    e_emu = oracle.factor_error(Lemu, Lexact)
    # same arithmetic up to rounding order: errors of the same size, plus the
    # FP32 accumulation of the tile-long sums on the tensor cores (the
    # emulation sums in FP64), at most about tile * 2^-24 relative
    slack = 4 * tile * 2.0 ** -24
    assert e_gpu <= 4 * e_emu + slack
    assert oracle.factor_error(Lg, Lemu) <= 4 * e_emu + slack
    assert np.all(np.diag(Lg) > 0)


def test_mixed_factor_exact_on_representable(ctx):
    """Sparse unit-diagonal {-1, 0, 1} factor: every operand (including the
    inverted 64 x 64 diagonal blocks) is a small integer, exact in bf16, and
    every sum is exact in FP32, so the low-precision factor is exact."""
    rng = np.random.default_rng(5)
    n = 256
    L0 = np.tril(rng.choice([-1.0, 0.0, 1.0], size=(n, n), p=[0.04, 0.92, 0.04]))
    np.fill_diagonal(L0, 1.0)
    for prec in ("bf16", "split_bf16", "split_f16"):
        L, info = gpchol.chol_factor_mixed(dev(L0 @ L0.T), prec, 64, ctx=ctx)
        assert info == 0
        assert np.array_equal(np.tril(host(L)), L0), prec


def test_mixed_factor_breakdown_reports_info(ctx):
    n = 300
    s = inputs.gp_system(n, 8, 0.5, 1e-1, seed=3)
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    A[150, 150] = -5.0
    _, info = gpchol.chol_factor_mixed(dev(A), "split_bf16", 128, ctx=ctx, raise_on_not_spd=False)
    _, info_ref = oracle.mixed_factor(A, 128, "split_bf16")
    assert info == info_ref == 151


@pytest.mark.parametrize("n,sn2,prec", [(300, 1e-2, "bf16"), (300, 1e-2, "split_bf16"), (1000, 1e-3, "bf16"),
                                        (1000, 1e-3, "split_bf16"), (2048, 1e-3, "split_bf16"),
                                        (300, 1e-2, "split_f16"), (2048, 1e-3, "split_f16")])
def test_refined_solve(ctx, n, sn2, prec):
    s = inputs.gp_system(n, 8, 0.5, sn2, nrhs=2, seed=50 + n)
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    L, _ = oracle.cholesky(A)
    Xref = oracle.chol_solve(L, s.B)
    Xd = gpchol.colmajor(n, 2)
    res = gpchol.solve_refined(dev(A), dev(s.B), Xd, prec=prec, tile=256, bwd_tol=1e-12, ctx=ctx)
    X = host(Xd)
    for r in range(2):
        be = oracle.backward_error(A, X[:, r], s.B[:, r])
        assert be <= 1e-12
        fe_gpu = oracle.forward_error(X[:, r], Xref[:, r])
        assert fe_gpu <= 1e-6
    assert res.backward_error_max <= 1e-12
    assert res.iterations >= 1


def test_refined_solve_zero_rhs_and_shift(ctx):
    n = 400
    s = inputs.gp_system(n, 8, 0.5, 1e-3, nrhs=1, seed=9)
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    B = np.zeros((n, 2))
    B[:, 1] = s.B[:, 0]
    Xd = gpchol.colmajor(n, 2)
    res = gpchol.solve_refined(dev(A), dev(B), Xd, prec="bf16", tile=128, ctx=ctx)
    X = host(Xd)
    assert np.all(X[:, 0] == 0.0)
    assert oracle.backward_error(A, X[:, 1], B[:, 1]) <= 1e-12
    assert res.shift > 0.0 and res.factor_attempts >= 1


@pytest.mark.parametrize("nrhs", [3, 17, 18])
def test_refined_solve_many_rhs(ctx, nrhs):
    """More than two right-hand sides: the products over all of A (groups of
    up to 16), and with 17 and 18 a last group of one or two columns that
    takes the lower-triangle products with a packed copy of its own."""
    n = 700
    s = inputs.gp_system(n, 8, 0.5, 1e-3, nrhs=nrhs, seed=60 + nrhs)
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    Xd = gpchol.colmajor(n, nrhs)
    res = gpchol.solve_refined(dev(A), dev(s.B), Xd, prec="split_f16", tile=256, bwd_tol=1e-12, ctx=ctx)
    X = host(Xd)
    for r in range(nrhs):
        assert oracle.backward_error(A, X[:, r], s.B[:, r]) <= 1e-12, r
    assert res.backward_error_max <= 1e-12


@pytest.mark.parametrize("nrhs", [1, 2])
def test_refined_solve_reads_lower_triangle_only(ctx, nrhs):
    """With one or two right-hand sides nothing of the refined solve reads
    above A's diagonal (the factor, the norm and the products take the
    lower triangle): NaN there leaves the result as accurate as before."""
    n = 900
    s = inputs.gp_system(n, 8, 0.5, 1e-3, nrhs=nrhs, seed=70 + nrhs)
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    Ad = dev(A)
    Ad.copy_(Ad + torch.triu(torch.full_like(Ad, float("nan")), 1))
    Xd = gpchol.colmajor(n, nrhs)
    res = gpchol.solve_refined(Ad, dev(s.B), Xd, prec="split_f16", tile=256, bwd_tol=1e-12, ctx=ctx)
    X = host(Xd)
    assert np.all(np.isfinite(X))
    for r in range(nrhs):
        assert oracle.backward_error(A, X[:, r], s.B[:, r]) <= 1e-12, r
    assert res.backward_error_max <= 1e-12
