"""GPU parity of the batched solve (A10) against the oracle: every system's
factor within 1e-12 of the oracle's, its solve within 1e-13 backward error;
a system's result is bit-identical alone and inside a batch; a non-SPD
member reports its own info while the others are solved; replaying the
captured graph reproduces the result."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13209_b300 import gpchol, inputs
from gpu_helpers import ctx, dev, host  # noqa: F401

pytestmark = pytest.mark.gpu


def make_batch(ns, nrhs=1, seed=0):
    sys_, As, Bs = [], [], []
    for i, n in enumerate(ns):
        s = inputs.gp_system(int(n), 8, 0.3 + 0.05 * (i % 10), 1e-3 + 1e-2 * (i % 7), nrhs=nrhs, seed=1000 + seed + i)
        A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
        sys_.append(s)
        As.append(A)
        Bs.append(s.B)
    return sys_, As, Bs


@pytest.mark.parametrize("ns", [[1, 63, 64, 65, 130, 200, 333, 70], [256, 300, 257, 511, 512, 640]])
def test_batched_parity(ctx, ns):
    _, As, Bs = make_batch(ns, nrhs=2)
    Ad = [dev(A) for A in As]
    Bd = [dev(B) for B in Bs]
    info = gpchol.batched_solve(Ad, Bd, ctx=ctx)
    assert info == [0] * len(ns)
    for A, B, a, b in zip(As, Bs, Ad, Bd):
        Lref, _ = oracle.cholesky(A)
        assert oracle.factor_error(np.tril(host(a)), Lref) <= 1e-12
        X = host(b)
        for r in range(B.shape[1]):
            assert oracle.backward_error(A, X[:, r], B[:, r]) <= 1e-13


def test_batched_invariance_and_replay(ctx):
    ns = [100, 257, 64, 190]
    _, As, Bs = make_batch(ns, seed=7)
    # alone
    solo = []
    for A, B in zip(As, Bs):
        a, b = dev(A), dev(B)
        assert gpchol.batched_solve([a], [b], ctx=ctx) == [0]
        solo.append((host(a), host(b)))
    # in the mix, twice (second call replays the captured graph)
    Ad = [dev(A) for A in As]
    Bd = [dev(B) for B in Bs]
    for rep in range(2):
        for a, b, A, B in zip(Ad, Bd, As, Bs):
            a.copy_(torch.from_numpy(A))
            b.copy_(torch.from_numpy(B))
        assert gpchol.batched_solve(Ad, Bd, ctx=ctx) == [0] * len(ns)
        for (La, Xa), a, b in zip(solo, Ad, Bd):
            assert np.array_equal(np.tril(host(a)), np.tril(La))
            assert np.array_equal(host(b), Xa)


def test_batched_not_spd_member(ctx):
    ns = [120, 150, 90]
    _, As, Bs = make_batch(ns, seed=3)
    As[1] = As[1].copy()
    As[1][70, 70] = -1.0
    _, info_ref = oracle.cholesky(As[1])
    Ad = [dev(A) for A in As]
    Bd = [dev(B) for B in Bs]
    info = gpchol.batched_solve(Ad, Bd, ctx=ctx, raise_on_not_spd=False)
    assert info[1] == info_ref == 71
    assert info[0] == 0 and info[2] == 0
    for i in (0, 2):
        x = host(Bd[i])[:, 0]
        assert oracle.backward_error(As[i], x, Bs[i][:, 0]) <= 1e-13


def test_batched_log_uniform_sizes(ctx):
    spec = inputs.batch_spec(count=24, nmin=256, nmax=1024, seed=4)
    As, Bs, Ad, Bd = [], [], [], []
    for k in range(24):
        s = spec.system(k)
        A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
        As.append(A)
        Bs.append(s.B)
        Ad.append(dev(A))
        Bd.append(dev(s.B))
    assert gpchol.batched_solve(Ad, Bd, ctx=ctx) == [0] * 24
    for A, B, b in zip(As, Bs, Bd):
        assert oracle.backward_error(A, host(b)[:, 0], B[:, 0]) <= 1e-13


# ------------------------------------------------------- mixed precision
def _mixed(ctx, As, Bs, tol=1e-12, maxit=30):
    Ad = [dev(A) for A in As]
    Bd = [dev(B) for B in Bs]
    Xd = [gpchol.colmajor(B.shape[0], B.shape[1]) for B in Bs]
    res = gpchol.batched_solve_mixed(Ad, Bd, Xd, bwd_tol=tol, maxit=maxit, ctx=ctx, raise_on_error=False)
    return res, Ad, Bd, Xd


@pytest.mark.parametrize("ns,nrhs", [([1, 63, 64, 65, 130, 200, 333, 70], 2), ([256, 300, 257, 511, 512, 640], 1),
                                     ([1000, 64, 1500, 129], 3)])
def test_batched_mixed_parity(ctx, ns, nrhs):
    """Every system to backward error <= 1e-12 by the oracle's long-double
    residual; forward error against the oracle's FP64 solve; A and B read
    only."""
    _, As, Bs = make_batch(ns, nrhs=nrhs, seed=50)
    res, Ad, Bd, Xd = _mixed(ctx, As, Bs)
    assert res.status == gpchol.GPCH_OK and res.info == [0] * len(ns)
    assert res.backward_error_max <= 1e-12
    for A, B, a, b, x in zip(As, Bs, Ad, Bd, Xd):
        assert np.array_equal(host(a), A) and np.array_equal(host(b), B)
        X = host(x)
        L, _ = oracle.cholesky(A)
        for r in range(B.shape[1]):
            assert oracle.backward_error(A, X[:, r], B[:, r]) <= 1e-12
            xo = oracle.chol_solve(L, B[:, r])
            cond = np.linalg.cond(A)
            assert oracle.forward_error(X[:, r], xo) <= max(1e-12 * cond, 1e-14)


def test_batched_mixed_invariance_and_replay(ctx):
    """A system's result is bit-identical alone and in the batch, and on a
    replay of the captured graph."""
    ns = [100, 257, 64, 190, 700]
    _, As, Bs = make_batch(ns, nrhs=2, seed=60)
    solo = []
    for A, B in zip(As, Bs):
        res, _, _, Xd = _mixed(ctx, [A], [B])
        assert res.info == [0]
        solo.append(host(Xd[0]))
    Ad = [dev(A) for A in As]
    Bd = [dev(B) for B in Bs]
    Xd = [gpchol.colmajor(B.shape[0], B.shape[1]) for B in Bs]
    for rep in range(2):
        for x in Xd:
            x.fill_(7.0)
        res = gpchol.batched_solve_mixed(Ad, Bd, Xd, ctx=ctx)
        assert res.info == [0] * len(ns)
        for xa, x in zip(solo, Xd):
            assert np.array_equal(host(x), xa)


def test_batched_mixed_not_spd_and_unreachable_tol(ctx):
    """An indefinite member reports its FP32 breakdown column while the others
    are solved; an unreachable tolerance reports -1 (not converged)."""
    _, As, Bs = make_batch([120, 90, 200], seed=70)
    bad = As[1].copy()
    bad[40, 40] = -5.0
    res, _, _, Xd = _mixed(ctx, [As[0], bad, As[2]], Bs)
    assert res.status == gpchol.GPCH_NOT_SPD
    assert res.info[0] == 0 and res.info[1] == 41 and res.info[2] == 0
    for A, B, x in ((As[0], Bs[0], Xd[0]), (As[2], Bs[2], Xd[2])):
        assert oracle.backward_error(A, host(x)[:, 0], B[:, 0]) <= 1e-12
    res, _, _, _ = _mixed(ctx, As, Bs, tol=1e-30, maxit=8)
    assert res.status == gpchol.GPCH_NOT_CONVERGED and set(res.info) == {-1}


def test_batched_mixed_config4_sample(ctx):
    """A 32-system sample of the batched workload (n log-uniform in
    [256, 4096], ell in [0.2, 1], sn2 in [1e-3, 1e-1]) to 1e-12."""
    spec = inputs.batch_spec(count=256, nmin=256, nmax=4096, seed=4)
    idx = list(range(0, 256, 8))
    syss = [spec.system(k, d=8) for k in idx]
    As = [oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2) for s in syss]
    Bs = [s.B for s in syss]
    res, _, _, Xd = _mixed(ctx, As, Bs)
    assert res.status == gpchol.GPCH_OK and res.backward_error_max <= 1e-12
    for A, B, x in zip(As, Bs, Xd):
        assert oracle.backward_error(A, host(x)[:, 0], B[:, 0]) <= 1e-12
