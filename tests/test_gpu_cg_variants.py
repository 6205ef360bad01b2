"""GPU parity of the CG options of gpch_cg_solve_ex against the oracle:
the single-reduction (Chronopoulos-Gear) form of Algorithm 1 (left), the
double-float product arithmetic and the FP64-accurate tensor-core products
(8 digits per entry, 512-entry passes), on FP64- and FP32-stored matrices, one to
16 right-hand sides, ragged and unaligned shapes, and the CG-bound system's
shape (ell = 0.3, sn2 = 0.1, 16 right-hand sides) at n = 4096.

CG iterates differ from the oracle's only by rounding order, so parity is
on outcomes: convergence, the true residual against the stored operator,
the iteration count within 5 % of the oracle's, and the solution against
the oracle's solution.  Early iterates of well-conditioned systems are
compared directly (they agree to rounding level)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13209_b300 import gpchol, inputs
from gpu_helpers import ctx, dev, host  # noqa: F401

pytestmark = pytest.mark.gpu

FORMS = [("classic", "fp64"), ("single_reduction", "fp64"), ("classic", "double_float"),
         ("single_reduction", "double_float"), ("classic", "tensor"), ("single_reduction", "tensor")]


def se_system(n, ell=0.5, sn2=1e-2, nrhs=1, seed=0):
    s = inputs.gp_system(n, 8, ell, sn2, nrhs=nrhs, seed=seed)
    return s, oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)


def run(ctx, A, B, variant, products, rtol=1e-10, maxit=20000, R=50, dtype=torch.float64, x0=None, lda=None):
    n = A.shape[0]
    B = np.asarray(B, dtype=np.float64)
    B2 = B[:, None] if B.ndim == 1 else B
    if lda is None:
        Ad = dev(A, dtype)
    else:
        Ad = gpchol.colmajor(n, n, dtype=dtype, ld=lda)
        Ad.copy_(torch.from_numpy(np.asarray(A)).to(dtype))
    Xd = dev(np.zeros_like(B2) if x0 is None else x0)
    res = gpchol.cg_solve(Ad, dev(B2), Xd, rtol=rtol, maxit=maxit, replace_every=R, ctx=ctx,
                          raise_on_not_converged=False, variant=variant, products=products)
    return res, host(Xd)


@pytest.mark.parametrize("variant,products", FORMS)
@pytest.mark.parametrize("n,R", [(1, 50), (3, 50), (257, 50), (1000, 7), (2048, 50)])
def test_cg_forms_parity(ctx, variant, products, n, R):
    s, A = se_system(n, sn2=1e-2, seed=700 + n)
    b = s.B[:, 0]
    ref_fn = oracle.cg_single_reduction if variant == "single_reduction" else oracle.cg
    x_or, it_or, _ = ref_fn(A, b, 1e-10, 20000, R=R)
    res, X = run(ctx, A, b, variant, products, R=R)
    x = X[:, 0]
    assert res.status == gpchol.GPCH_OK and res.converged == 1 and res.relres_max <= 1e-10
    assert np.linalg.norm(b - A @ x) / np.linalg.norm(b) <= 1e-9
    assert abs(res.iterations - it_or) <= max(3, 0.05 * it_or)
    assert oracle.forward_error(x, x_or) <= 1e-6


@pytest.mark.parametrize("variant,products", FORMS)
def test_cg_forms_early_iterates(ctx, variant, products):
    """Well conditioned (sn2 = 0.5): after k iterations the iterate equals
    the oracle's to rounding level, so the product A s is right to about
    1e-14 (a wrong head/tail split, a dropped cross term or a wrong scale
    each show here)."""
    s, A = se_system(600, sn2=0.5, nrhs=2, seed=710)
    ref_fn = oracle.cg_single_reduction if variant == "single_reduction" else oracle.cg
    for k in (1, 2, 3, 6):
        res, X = run(ctx, A, s.B, variant, products, rtol=0.0, maxit=k, R=0)
        assert res.status == gpchol.GPCH_NOT_CONVERGED and res.iterations == k
        for r in range(2):
            xk, itk, _ = ref_fn(A, s.B[:, r], 0.0, k, R=0)
            assert itk == k
            assert oracle.forward_error(X[:, r], xk) <= 1e-12, (k, r)


@pytest.mark.parametrize("variant,products", FORMS)
@pytest.mark.parametrize("nrhs", [2, 5, 16])
def test_cg_forms_multi_rhs_f32(ctx, variant, products, nrhs):
    """FP32-stored A (exactly widened on both sides), several right-hand
    sides sharing one pass over A per iteration."""
    n = 700
    s, A = se_system(n, sn2=5e-2, nrhs=nrhs, seed=720 + nrhs)
    A32u = A.astype(np.float32).astype(np.float64)
    res, X = run(ctx, A32u.astype(np.float32), s.B, variant, products, dtype=torch.float32, maxit=5000)
    assert res.converged == nrhs
    for r in range(nrhs):
        b = s.B[:, r]
        x_or, it_or, _ = oracle.cg(A32u, b, 1e-10, 5000)
        assert np.linalg.norm(b - A32u @ X[:, r]) / np.linalg.norm(b) <= 1e-9
        assert oracle.forward_error(X[:, r], x_or) <= 1e-6


_CG_BOUND_REF = {}


def _cg_bound_ref(dtype):
    """The n = 4096 CG-bound system, its stored operator (widened) and the
    oracle's solutions of columns 0 and 15 (cached: the oracle takes a few
    seconds per column)."""
    if dtype not in _CG_BOUND_REF:
        s = inputs.config3(4096, 16)
        A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
        Aop = A if dtype == torch.float64 else A.astype(np.float32).astype(np.float64)
        refs = {r: oracle.cg(Aop, s.B[:, r], 1e-10, 20000) for r in (0, 15)}
        _CG_BOUND_REF[dtype] = (s, Aop, refs)
    return _CG_BOUND_REF[dtype]


@pytest.mark.parametrize("variant,products", FORMS)
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_cg_cg_bound_shape(ctx, variant, products, dtype):
    """The CG-bound workload's shape at n = 4096: ell = 0.3, sn2 = 0.1, 16
    right-hand sides, relative residual 1e-10, replacement every 50
    iterations; FP64- and FP32-stored A against the oracle on the stored
    (widened) operator."""
    s, Aop, refs = _cg_bound_ref(dtype)
    res, X = run(ctx, Aop if dtype == torch.float64 else Aop.astype(np.float32), s.B, variant, products,
                 dtype=dtype, maxit=20000)
    assert res.status == gpchol.GPCH_OK and res.converged == 16
    its = []
    for r in (0, 15):
        b = s.B[:, r]
        x_or, it_or, _ = refs[r]
        its.append(it_or)
        assert np.linalg.norm(b - Aop @ X[:, r]) / np.linalg.norm(b) <= 1e-9
        assert oracle.forward_error(X[:, r], x_or) <= 1e-7
    for r in range(16):
        assert np.linalg.norm(s.B[:, r] - Aop @ X[:, r]) / np.linalg.norm(s.B[:, r]) <= 1e-9
    assert res.iterations <= 1.05 * max(its) + 10


@pytest.mark.parametrize("products", ["fp64", "double_float"])
def test_cg_unaligned_lda_and_start_vector(ctx, products):
    """lda = n + 1 (rows no longer start on 16-byte boundaries, so the
    kernels take the element-wise loads) and a nonzero start vector."""
    n = 301
    s, A = se_system(n, sn2=1e-2, seed=730)
    b = s.B[:, 0]
    x0 = np.linspace(-1.0, 1.0, n)
    x_or, it_or, _ = oracle.cg(A, b, 1e-10, 5000, x0=x0)
    for variant in ("classic", "single_reduction"):
        res, X = run(ctx, A, b, variant, products, x0=x0, lda=n + 1, maxit=5000)
        assert res.converged == 1
        assert np.linalg.norm(b - A @ X[:, 0]) / np.linalg.norm(b) <= 1e-9
        assert abs(res.iterations - it_or) <= max(3, 0.05 * it_or)


def test_cg_double_float_scale_invariance(ctx):
    """Powers of two in b (2^-100, 2^+100) and in A (2^-60) leave the
    double-float path's iterates unchanged up to that power: the scales
    taken from max |b| and max A_ii are exact."""
    s, A = se_system(500, sn2=1e-2, seed=740)
    b = s.B[:, 0]
    base, Xb = run(ctx, A, b, "classic", "double_float", maxit=5000)
    for fa, fb in ((1.0, 2.0 ** -100), (1.0, 2.0 ** 100), (2.0 ** -60, 1.0)):
        res, X = run(ctx, A * fa, b * fb, "classic", "double_float", maxit=5000)
        assert res.iterations == base.iterations
        np.testing.assert_array_equal(X[:, 0], Xb[:, 0] * (fb / fa))


def test_cg_zero_rhs_column(ctx):
    s, A = se_system(200, sn2=1e-2, nrhs=3, seed=750)
    B = s.B.copy()
    B[:, 1] = 0.0
    for variant, products in FORMS:
        res, X = run(ctx, A, B, variant, products, maxit=5000)
        assert res.converged == 3
        assert np.all(X[:, 1] == 0.0)
