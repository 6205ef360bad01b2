"""GPU parity of the GP quantities computed on a solved system (the GP
behaviour prediction of Sec. 4.1): log det A from the FP64 factor and the
predictive mean K(Xs, X) alpha, against the oracle on the same inputs."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13209_b300 import gpchol, inputs
from gpu_helpers import ctx, dev, host  # noqa: F401

pytestmark = pytest.mark.gpu


def se_system(n, ell=0.5, sn2=1e-2, nrhs=1, seed=0, d=8):
    s = inputs.gp_system(n, d, ell, sn2, nrhs=nrhs, seed=seed)
    return s, oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)


@pytest.mark.parametrize("n,tile", [(1, 64), (65, 64), (700, 256), (2048, 512)])
def test_logdet_parity(ctx, n, tile):
    """The factor agrees with the oracle's to ~1e-13 relative per entry, so
    2 sum log L_ii agrees to about n * 1e-13 absolute."""
    _, A = se_system(n, seed=500 + n)
    ref, info = oracle.logdet(A)
    assert info == 0
    Ad = dev(A)
    assert gpchol.chol_factor(Ad, tile=tile, ctx=ctx) == 0
    got = gpchol.logdet(Ad, ctx=ctx)
    assert abs(got - ref) <= 1e-12 * max(1.0, abs(ref)) + n * 1e-13, (got, ref)


def test_logdet_reproducible_and_not_spd(ctx):
    _, A = se_system(300, seed=511)
    Ad = dev(A)
    gpchol.chol_factor(Ad, tile=128, ctx=ctx)
    v1 = gpchol.logdet(Ad, ctx=ctx)
    v2 = gpchol.logdet(Ad, ctx=ctx)
    assert v1 == v2
    Ad[7, 7] = -1.0
    with pytest.raises(gpchol.GpchError) as e:
        gpchol.logdet(Ad, ctx=ctx)
    assert e.value.status == gpchol.GPCH_NOT_SPD


def _mean_bound(Xs, X, sf2, ell, alpha):
    """sum_i |k(xs, x_i)| |alpha_i| per entry (numpy), the scale that the
    FP64 rounding of the sum is measured against."""
    d2 = ((Xs[:, None, :] - X[None, :, :]) ** 2).sum(-1)
    K = sf2 * np.exp(-d2 / (2 * ell * ell))
    return K @ np.abs(alpha)


@pytest.mark.parametrize("m,n,d,nrhs", [(1, 1, 1, 1), (17, 100, 8, 1), (16, 33, 3, 2), (300, 1000, 8, 3),
                                        (129, 777, 8, 16), (40, 5000, 8, 1), (5, 64, 64, 4), (3000, 257, 8, 5)])
def test_predict_mean_parity(ctx, m, n, d, nrhs):
    rng = np.random.default_rng(1000 * m + n)
    X = rng.uniform(0.0, 1.0, (n, d))
    Xs = rng.uniform(-0.2, 1.2, (m, d))
    alpha = rng.standard_normal((n, nrhs))
    sf2, ell = 1.3, 0.45
    ref = oracle.predict_mean(Xs, X, sf2, ell, alpha)
    got = host(gpchol.predict_mean(torch.from_numpy(Xs).cuda(), torch.from_numpy(X).cuda(), sf2, ell, dev(alpha),
                                   ctx=ctx))
    bound = _mean_bound(Xs, X, sf2, ell, alpha)
    assert got.shape == (m, nrhs)
    assert np.all(np.abs(got - ref) <= 1e-13 * bound + 1e-300), np.max(np.abs(got - ref) / (bound + 1e-300))


def test_predict_mean_reproducible_and_ld(ctx):
    rng = np.random.default_rng(77)
    X = rng.uniform(0.0, 1.0, (2000, 8))
    Xs = rng.uniform(0.0, 1.0, (50, 8))
    alpha = rng.standard_normal((2000, 2))
    Ad = gpchol.colmajor(2000, 2, ld=2048)
    Ad.copy_(torch.from_numpy(alpha))
    out = gpchol.colmajor(50, 2, ld=64)
    out.fill_(123.0)
    a = host(gpchol.predict_mean(torch.from_numpy(Xs).cuda(), torch.from_numpy(X).cuda(), 1.0, 0.5, Ad, mean=out,
                                 ctx=ctx)).copy()
    b = host(gpchol.predict_mean(torch.from_numpy(Xs).cuda(), torch.from_numpy(X).cuda(), 1.0, 0.5, Ad, mean=out,
                                 ctx=ctx))
    assert np.array_equal(a, b)
    np.testing.assert_allclose(a, oracle.predict_mean(Xs, X, 1.0, 0.5, alpha), rtol=1e-12, atol=1e-13)


def test_gp_pipeline_mean_at_training_points(ctx):
    """Factor, solve alpha = (K + sn2 I)^-1 y, then the mean at the training
    points must be y - sn2 alpha; log det agrees with the oracle."""
    s, A = se_system(2048, ell=0.5, sn2=1e-1, nrhs=2, seed=520)
    Ad = dev(A)
    assert gpchol.chol_factor(Ad, tile=256, ctx=ctx) == 0
    alpha = dev(s.B)
    gpchol.chol_solve(Ad, alpha, ctx=ctx)
    Xd = torch.from_numpy(s.X).cuda()
    mean = host(gpchol.predict_mean(Xd, Xd, s.sf2, s.ell, alpha, ctx=ctx))
    a = host(alpha)
    np.testing.assert_allclose(mean, s.B - s.sn2 * a, rtol=0, atol=1e-10 * np.abs(s.B).max())
    ref, _ = oracle.logdet(A)
    assert abs(gpchol.logdet(Ad, ctx=ctx) - ref) <= 1e-12 * abs(ref) + 2048 * 1e-13


def test_predict_mean_empty_and_bad_args(ctx):
    Xs = torch.zeros((0, 8), dtype=torch.float64, device="cuda")
    X = torch.rand((10, 8), dtype=torch.float64, device="cuda")
    alpha = gpchol.colmajor(10, 1)
    alpha.fill_(1.0)
    out = gpchol.predict_mean(Xs, X, 1.0, 0.5, alpha, ctx=ctx)
    assert out.shape == (0, 1)
    with pytest.raises(gpchol.GpchError):
        gpchol.predict_mean(torch.rand((3, 8), dtype=torch.float64, device="cuda"), X, 1.0, -0.5, alpha, ctx=ctx)
