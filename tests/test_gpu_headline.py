"""GPU parity of the exact mixed path the benchmark times, checked against
the oracle at growing sizes.

The path: split-f16 mixed factor with tile 512 (FP64 diagonal tiles, the
panel as a split-f16 tensor-core product with L_jj^-1, the left-looking
step-3 update on the second stream in long passes of up to 16 panels, the
look-ahead rectangle on the side stream), then FP64 PCG refinement to a
backward error of 1e-12 (Algorithm 1, right; Sec. 2.2's L L^T = A).  The
systems are the leading n x n blocks of the n = 32768 benchmark system
(same points, same hyper-parameters).

* n = 4096: the factor against the oracle's emulation, entry by entry
  (relative Frobenius error over the lower triangle), and the solve.
* n = 8192: backward error and forward error of the refined solve.
* n = 16384: the first size at which the long pass of a block column is
  split into more than one 16-panel launch; backward error.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13209_b300 import gpchol, inputs
from gpu_helpers import ctx, dev, host  # noqa: F401

pytestmark = pytest.mark.gpu

TILE = 512
PREC = "split_f16"


def bench_block(n):
    """Leading n x n block of the benchmark system, built by the oracle."""
    s = inputs.config2(n)
    return oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2), s.B[:, 0].copy()


def refined(ctx, A, b):
    n = A.shape[0]
    Xd = gpchol.colmajor(n, 1)
    res = gpchol.solve_refined(dev(A), dev(b), Xd, prec=PREC, tile=TILE, bwd_tol=1e-12, maxit=500, ctx=ctx)
    return host(Xd)[:, 0], res


def test_headline_factor_vs_emulation_n4096(ctx):
    A, b = bench_block(4096)
    Lexact, info = oracle.cholesky(A)
    assert info == 0
    Lemu, info = oracle.mixed_factor(A, TILE, PREC)
    assert info == 0
    L, info = gpchol.chol_factor_mixed(dev(A), PREC, TILE, ctx=ctx)
    assert info == 0
    Lg = np.tril(host(L))
    assert np.all(np.diag(Lg) > 0)
    assert np.all(np.isfinite(Lg))
    e_gpu = oracle.factor_error(Lg, Lexact)
    e_emu = oracle.factor_error(Lemu, Lexact)
    # same arithmetic up to rounding order (left-looking order, the panel
    # through L_jj^-1, FP32 sums of 256-product pieces): errors of the same
    # size, plus the FP32 accumulation bound tile * 2^-24
    slack = 4 * TILE * 2.0 ** -24
    assert e_gpu <= 4 * e_emu + slack
    assert oracle.factor_error(Lg, Lemu) <= 4 * e_emu + slack

    x, res = refined(ctx, A, b)
    assert res.status == gpchol.GPCH_OK
    assert oracle.backward_error(A, x, b) <= 1e-12
    x_ref = oracle.chol_solve(Lexact, b)
    assert oracle.forward_error(x, x_ref) <= 1e-6


def test_headline_refined_n8192(ctx):
    A, b = bench_block(8192)
    x, res = refined(ctx, A, b)
    assert res.status == gpchol.GPCH_OK and res.iterations >= 1
    be = oracle.backward_error(A, x, b)
    assert be <= 1e-12
    assert res.backward_error_max <= 1e-12
    x_ref = oracle.solve_spd(A, b)
    assert oracle.forward_error(x, x_ref) <= 1e-6


def test_headline_refined_n16384(ctx):
    A, b = bench_block(16384)
    x, res = refined(ctx, A, b)
    assert res.status == gpchol.GPCH_OK and res.iterations >= 1
    assert oracle.backward_error(A, x, b) <= 1e-12
    del A
    torch.cuda.empty_cache()
