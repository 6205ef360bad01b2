"""GPU parity of the substitution sweeps with an FP32 factor
(gpch_chol_solve_f32: Sec. 2.2's forward and back substitution with the
low-precision factor, the preconditioner application of the refined solve)
against the oracle's FP64 substitution on the same FP32 values.

With one or two right-hand sides the sweeps walk 128-row blocks through the
coupling blocks inv(L_II) L_{I,I-1} and L_{I+1,I} inv(L_II); with three or
more, 64-row blocks.  The factors are well conditioned (diagonal in [1, 2],
strictly lower entries of size 0.5 / sqrt(n)), so FP32 block products keep
the solution within about 1e-6 of the oracle's relative to its largest
entry; a wrong coupling block, a lost partial sum or a misplaced block row
is of order 1."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13209_b300 import gpchol, inputs
from gpu_helpers import ctx, dev, host  # noqa: F401

pytestmark = pytest.mark.gpu


def _factor(n, seed):
    rng = np.random.default_rng(seed)
    L = np.tril(rng.standard_normal((n, n)) * (0.5 / np.sqrt(max(n, 1))), -1)
    L[np.diag_indices(n)] = rng.uniform(1.0, 2.0, n)
    return L.astype(np.float32).astype(np.float64)


@pytest.mark.parametrize("n", [1, 64, 127, 128, 129, 300, 1000, 2600, 4100])
@pytest.mark.parametrize("nrhs", [1, 2, 3])
def test_sweep_f32_parity(ctx, n, nrhs):
    L = _factor(n, 10 * n + nrhs)
    rng = np.random.default_rng(n + 7 * nrhs)
    B = rng.standard_normal((n, nrhs))
    ref = oracle.chol_solve(L, B)
    Ld = dev(L, torch.float32)
    # junk above the diagonal must not be read
    Ld.copy_(Ld + torch.triu(torch.full_like(Ld, float("nan")), 1))
    Bd = dev(B)
    gpchol.chol_solve_f32(Ld, Bd, ctx=ctx)
    got = host(Bd)
    assert np.all(np.isfinite(got))
    # observed at most 2.9e-7
    assert np.max(np.abs(got - ref)) <= 2e-6 * np.max(np.abs(ref))


def test_sweep_f32_mixed_factor(ctx):
    """The factor the refined solve uses: L of gpch_chol_factor_mixed on an
    SE system; the result against the oracle on the same factor values."""
    s = inputs.gp_system(2000, 8, 0.5, 1e-1, nrhs=2, seed=2100)
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    L, info = gpchol.chol_factor_mixed(dev(A), "split_f16", 256, ctx=ctx)
    assert info == 0
    Lh = np.tril(host(L))
    ref = oracle.chol_solve(Lh, s.B)
    Bd = dev(s.B)
    gpchol.chol_solve_f32(L, Bd, ctx=ctx)
    got = host(Bd)
    # observed 4.3e-7
    assert np.max(np.abs(got - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("nrhs", [1, 2])
def test_sweep_f32_more_blocks_than_sms(ctx, nrhs):
    """n = 20000: 157 blocks of 128 rows, more than the grid's one CTA per
    SM, so CTAs own several blocks.  Checked by the residual of the two
    triangular systems in FP64 (a property that holds at any size)."""
    n = 20000
    g = torch.Generator(device="cuda").manual_seed(31 + nrhs)
    L = torch.randn(n, n, device="cuda", generator=g, dtype=torch.float32) * (0.5 / n ** 0.5)
    L = torch.tril(L, -1)
    L.diagonal().copy_(1.0 + torch.rand(n, device="cuda", generator=g, dtype=torch.float32))
    Lc = gpchol.colmajor(n, n, dtype=torch.float32)
    Lc.copy_(L)
    del L
    B = torch.randn(n, nrhs, device="cuda", generator=g, dtype=torch.float64)
    X = gpchol.colmajor(n, nrhs)
    X.copy_(B)
    gpchol.chol_solve_f32(Lc, X, ctx=ctx)
    L64 = Lc.double()
    R = L64 @ (L64.T @ X) - B
    scale = (L64.abs() @ (L64.T.abs() @ X.abs())).max()
    # observed 1.8e-9
    assert float(R.abs().max() / scale) <= 5e-8
