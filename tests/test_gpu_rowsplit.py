"""GPU parity of the row-split CG pieces (f4): the block product
gpch_block_matvec against the FP64 product of the same numbers, and the
row-split driver over the library's local steps, against the oracle's
single-reduction CG (Algorithm 1 left, Chronopoulos-Gear form).

This run has one GPU, so the ranks of a multi-rank solve are emulated as
host threads in one process, each with its own library context and CUDA
stream, exchanging through host-side barriers (no kernel waits on another
rank's kernel; the exchange stands in for NCCL's allgather / allreduce)."""
import threading

import numpy as np
import pytest
import torch

import oracle
from paper_2605_13209_b300 import gpchol, inputs, rowsplit
from gpu_helpers import ctx, dev, host  # noqa: F401

pytestmark = pytest.mark.gpu


def se_matrix(n, ell=0.5, sn2=1e-2, nrhs=1, seed=0):
    s = inputs.gp_system(n, 8, ell, sn2, nrhs=nrhs, seed=seed)
    return s, oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)


@pytest.mark.parametrize("products", ["fp64", "double_float"])
@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
@pytest.mark.parametrize("n,r0,m,nrhs", [(300, 0, 300, 1), (300, 100, 77, 3), (1025, 513, 512, 16),
                                         (64, 63, 1, 2), (2000, 1000, 1000, 5)])
def test_block_matvec_parity(ctx, products, dtype, n, r0, m, nrhs):
    _, A = se_matrix(n, seed=n + m)
    Aop = A.astype(np.float32).astype(np.float64) if dtype == torch.float32 else A
    rng = np.random.default_rng(n * 7 + r0)
    V = rng.standard_normal((n, nrhs))
    blk = Aop[:, r0:r0 + m]
    Ad = gpchol.colmajor(n, m, dtype=dtype)
    Ad.copy_(torch.from_numpy(np.asfortranarray(blk)).to(dtype))
    T = gpchol.colmajor(m, nrhs)
    gpchol.block_matvec(Ad, r0, dev(V), T, products, ctx=ctx)
    got = host(T)
    ref = blk.T @ V
    scale = np.abs(blk).T @ np.abs(V)
    tol = 1e-14 if products == "fp64" else 2e-13
    assert np.all(np.abs(got - ref) <= tol * scale + 1e-300), np.max(np.abs(got - ref) / scale)


class LocalComm:
    """World size 1: the exchanges are copies."""

    def allgather_rows(self, local, full):
        full[:local.shape[0]] = local

    def allreduce_sum(self, t):
        pass


class ThreadComm:
    """Ranks as host threads of one process: publish a copy, meet at a
    barrier, read every rank's copy in rank order (so every rank adds the
    same numbers in the same order), meet again."""

    def __init__(self, n, world):
        self.offs, self.sizes = rowsplit.partition(n, world)
        self.world = world
        self.bar = threading.Barrier(world, timeout=120)
        self.slots = [None] * world
        self.local = threading.local()

    def _exchange(self, rank, t):
        self.slots[rank] = t.clone()
        torch.cuda.current_stream().synchronize()
        self.bar.wait()
        got = list(self.slots)
        return got

    def allgather_rows(self, local, full):
        rank = self.local.rank
        got = self._exchange(rank, local)
        for k in range(self.world):
            o, m = self.offs[k], self.sizes[k]
            full[o:o + m] = got[k]
        torch.cuda.current_stream().synchronize()
        self.bar.wait()

    def allreduce_sum(self, t):
        rank = self.local.rank
        got = self._exchange(rank, t)
        acc = got[0].clone()
        for k in range(1, self.world):
            acc += got[k]
        t.copy_(acc)
        torch.cuda.current_stream().synchronize()
        self.bar.wait()


def _oracle_refs(A, B, R):
    return [oracle.cg_single_reduction(A, B[:, c], 1e-10, 20000, R=R) for c in range(B.shape[1])]


def _check(A, B, X, iters, rel, refs):
    for c, (x_or, it_or, _) in enumerate(refs):
        assert rel[c] <= 1e-10
        assert np.linalg.norm(B[:, c] - A @ X[:, c]) / np.linalg.norm(B[:, c]) <= 1e-9
        assert abs(iters[c] - it_or) <= max(3, 0.05 * it_or)
        assert oracle.forward_error(X[:, c], x_or) <= 1e-6


@pytest.mark.parametrize("products", ["fp64", "double_float"])
def test_rowsplit_one_rank(ctx, products):
    s, A = se_matrix(700, nrhs=2, seed=801)
    Xd = gpchol.colmajor(700, 2)
    Xd.zero_()
    ops = rowsplit.RankOps(dev(A), 0, dev(s.B), Xd, products=products, ctx=ctx)
    iters, rel, loops = rowsplit.rowsplit_cg(LocalComm(), ops, rtol=1e-10, maxit=20000, replace_every=50)
    _check(A, s.B, host(Xd), iters, rel, _oracle_refs(A, s.B, 50))


@pytest.mark.parametrize("world,n,nrhs,R,products,dtype", [(2, 1000, 1, 50, "fp64", torch.float64),
                                                           (3, 1001, 3, 7, "double_float", torch.float64),
                                                           (2, 777, 2, 50, "double_float", torch.float32)])
def test_rowsplit_threads(world, n, nrhs, R, products, dtype):
    s, A = se_matrix(n, nrhs=nrhs, seed=810 + n)
    Aop = A.astype(np.float32).astype(np.float64) if dtype == torch.float32 else A
    comm = ThreadComm(n, world)
    results = [None] * world
    errors = []
    xs = [None] * world

    def rank_main(rank):
        try:
            comm.local.rank = rank
            c = gpchol.Context(0)
            stream = torch.cuda.Stream()
            with torch.cuda.stream(stream):
                o, m = comm.offs[rank], comm.sizes[rank]
                Ablk = gpchol.colmajor(n, m, dtype=dtype)
                Ablk.copy_(torch.from_numpy(np.asfortranarray(Aop[:, o:o + m])).to(dtype))
                Bl = dev(s.B[o:o + m])
                Xl = gpchol.colmajor(m, nrhs)
                Xl.zero_()
                ops = rowsplit.RankOps(Ablk, o, Bl, Xl, products=products, ctx=c)
                results[rank] = rowsplit.rowsplit_cg(comm, ops, rtol=1e-10, maxit=20000, replace_every=R)
                xs[rank] = host(Xl)
                stream.synchronize()
            c.close()
        except Exception as e:  # surfaced below
            errors.append(e)
            comm.bar.abort()

    threads = [threading.Thread(target=rank_main, args=(k,)) for k in range(world)]
    for t in threads:
        t.start()
    for t in threads:
        t.join(timeout=600)
    assert not errors, errors
    for r in results[1:]:
        assert r == results[0]                       # identical scalars on every rank
    X = np.vstack(xs)
    iters, rel, _ = results[0]
    _check(Aop, s.B, X, iters, rel, _oracle_refs(Aop, s.B, R))
