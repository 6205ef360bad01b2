"""GPU parity of gpch_symv_lower (the product of the refined solve's CG
iteration, Algorithm 1 (left)) against the oracle's long-double product.

Only A's lower triangle may affect the result, so the strict upper triangle
is filled with NaN.  The products are double-float products with a relative
error below about 2^-44 each, so y_i is compared against the oracle's
long-double y_i within 1e-12 of (|A| |x|)_i (observed about 1e-15); a
dropped or doubled diagonal, a lost strip or chunk partial or a row sum in
the wrong place is an error of order (|A| |x|)_i.  Shapes span one and
several 256-column strips and 512-row chunks with ragged tails, odd leading
dimensions (the scalar-load path) and one to three right-hand sides (pairs
and a single column)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13209_b300 import gpchol
from gpu_helpers import ctx, dev, host  # noqa: F401

pytestmark = pytest.mark.gpu


def _sym(n, seed, spd=True):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n))
    A = (M + M.T) / 2.0
    if spd:
        A += n * np.eye(n) if n else 0.0
    return A


def _check(ctx, A, X, lda=None):
    n, nrhs = X.shape
    ref = -oracle.gemm_update(np.zeros((n, nrhs)), A, X.T)
    Ad = gpchol.colmajor(n, n, ld=lda if lda is not None else n)
    # NaN above the diagonal: only the lower triangle may be used
    Ad.copy_(torch.from_numpy(np.tril(A) + np.triu(np.full((n, n), np.nan), 1)))
    Y = gpchol.symv_lower(Ad, dev(X), ctx=ctx)
    torch.cuda.synchronize()
    got = host(Y)
    scale = np.abs(A) @ np.abs(X)
    assert np.all(np.isfinite(got))
    err = np.abs(got - ref)
    assert np.all(err <= 1e-12 * scale + 1e-300), float(np.max(err / np.maximum(scale, 1e-300)))


@pytest.mark.parametrize("n", [1, 2, 3, 255, 256, 257, 511, 512, 513, 1000, 1537, 2600])
@pytest.mark.parametrize("nrhs", [1, 2, 3])
def test_symv_lower_parity(ctx, n, nrhs):
    A = _sym(n, 100 * n + nrhs)
    X = np.random.default_rng(n + 31 * nrhs).standard_normal((n, nrhs))
    _check(ctx, A, X)


@pytest.mark.parametrize("n,lda", [(300, 301), (777, 800), (1025, 1031)])
def test_symv_lower_leading_dimension(ctx, n, lda):
    """Odd or padded lda: the scalar-load path and the column stride."""
    A = _sym(n, 7 * n)
    X = np.random.default_rng(n).standard_normal((n, 2))
    _check(ctx, A, X, lda=lda)


def test_symv_lower_indefinite_and_scaled(ctx):
    """A symmetric indefinite matrix whose entries stay below its largest
    diagonal entry, and right-hand sides of very different magnitudes
    (each column has its own power-of-two scale)."""
    n = 700
    A = _sym(n, 5, spd=False)
    A[np.diag_indices(n)] = 4.0 * np.sign(np.random.default_rng(6).standard_normal(n))
    X = np.random.default_rng(8).standard_normal((n, 2))
    X[:, 1] *= 1e-200
    _check(ctx, A, X)


def test_symv_lower_se_matrix(ctx):
    """The refined solve's operator: an SE covariance matrix (entries from
    sf2 down to underflow) and a vector of mixed signs."""
    from paper_2605_13209_b300 import inputs
    s = inputs.gp_system(3000, 8, 0.5, 1e-3, nrhs=1, seed=44)
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    X = np.random.default_rng(45).standard_normal((3000, 1))
    _check(ctx, A, X)


def test_symv_lower_large_residual_property(ctx):
    """n = 20000 (79 strips, 40 chunks): y = A x against a torch FP64
    product of the symmetrized matrix; the difference stays within the
    products' error (a property that holds at any size)."""
    n = 20000
    g = torch.Generator(device="cuda").manual_seed(77)
    L = torch.tril(torch.randn(n, n, device="cuda", dtype=torch.float64, generator=g))
    L.diagonal().add_(float(n))
    A = gpchol.colmajor(n, n)
    A.copy_(L)
    x = torch.randn(n, 1, device="cuda", dtype=torch.float64, generator=g)
    X = gpchol.colmajor(n, 1)
    X.copy_(x)
    Y = gpchol.symv_lower(A, X, ctx=ctx)
    S = L + torch.tril(L, -1).T
    ref = S @ x
    scale = S.abs() @ x.abs()
    # observed about 1e-15 relative; FP64 GEMM reference adds n u
    assert float(((Y - ref).abs() / scale).max()) <= 1e-11
