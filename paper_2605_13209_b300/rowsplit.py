"""Row-split CG across ranks (one GPU per rank).

The paper splits the matrix of a CG solve by rows between the CPU and the
GPU (its horizontal split, Sec. 3.1).  Here the same split runs across GPUs:
rank k owns a contiguous block of rows r0 .. r0+m-1 of the symmetric A,
stored as the n x m column block A[:, r0:r0+m], and the same rows of x, b
and every CG vector.  The iteration is the single-reduction (Chronopoulos-
Gear) form of Algorithm 1 (left), so one iteration exchanges exactly

  * one allgather of the n x nrhs vector the product needs (r), and
  * one allreduce of 2 nrhs doubles (the rank's partial r^T r and w^T r),

plus, on replacement iterations (every R, Sec. 2.1), the allgathers of x
and p for the true residual b - A x and s = A p.

Every arithmetic step runs in the rank's `ops` (on a GPU: RankOps, the
library's kernels through the C ABI); this module only sequences the steps
and moves data through `comm` (TorchComm: torch.distributed, NCCL between
GPUs).  All ranks compute the same scalars from the same reduced sums, so
they stop at the same iteration.
"""
from __future__ import annotations

import torch

from . import gpchol


def partition(n: int, world: int):
    """Contiguous row blocks, sizes differing by at most one: (offsets, sizes)."""
    base, extra = divmod(n, world)
    sizes = [base + (1 if k < extra else 0) for k in range(world)]
    offs = [sum(sizes[:k]) for k in range(world)]
    return offs, sizes


class TorchComm:
    """The two exchanges of the row-split solve over torch.distributed.

    allgather_rows(local, full): every rank's m_k x nrhs block into the
    n x nrhs `full` (rank order = row order), through a padded staging
    buffer so that every rank sends the same number of entries.
    allreduce_sum(t): elementwise sum over ranks, in place."""

    def __init__(self, n: int, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.world = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        self.offs, self.sizes = partition(n, self.world)
        self.mmax = max(self.sizes)

    def allgather_rows(self, local: torch.Tensor, full: torch.Tensor):
        nrhs = local.shape[1]
        send = torch.zeros((nrhs, self.mmax), dtype=local.dtype, device=local.device)
        send[:, :local.shape[0]] = local.t()
        recv = torch.empty((self.world * nrhs, self.mmax), dtype=local.dtype, device=local.device)
        self.dist.all_gather_into_tensor(recv, send, group=self.group)
        for k in range(self.world):
            o, m = self.offs[k], self.sizes[k]
            full[o:o + m, :] = recv[k * nrhs:(k + 1) * nrhs, :m].t()

    def allreduce_sum(self, t: torch.Tensor):
        self.dist.all_reduce(t, op=self.dist.ReduceOp.SUM, group=self.group)


class RankOps:
    """One rank's arithmetic through the C ABI: the block product
    (gpch_block_matvec) and the single-reduction steps (gpch_cgsr_*).

    Ablk: n x m column block (column-major, float64 or float32) holding
    columns r0 .. r0+m-1 of A; B, X: m x nrhs column-major float64 (X holds
    the start vector and receives the solution)."""

    def __init__(self, Ablk: torch.Tensor, r0: int, B: torch.Tensor, X: torch.Tensor, products: str = "fp64",
                 ctx: gpchol.Context | None = None):
        self.ctx = ctx or gpchol.default_context()
        self.A, self.r0, self.B, self.X, self.products = Ablk, int(r0), B, X, products
        n, m = Ablk.shape
        nrhs = B.shape[1]
        if nrhs > 16:
            raise ValueError("at most 16 right-hand sides per solve")
        dev = B.device
        self.n, self.m, self.nrhs = n, m, nrhs
        self.V = gpchol.colmajor(n, nrhs, device=dev)
        self.R, self.W, self.P, self.S, self.T = (gpchol.colmajor(m, nrhs, device=dev) for _ in range(5))
        self.P.zero_()
        self.S.zero_()
        self.sums = torch.zeros(2 * nrhs, dtype=torch.float64, device=dev)
        self.state = torch.zeros(gpchol.CGSR_STATE_BYTES, dtype=torch.uint8, device=dev)

    def product(self, out: torch.Tensor, true_residual: bool = False):
        """out = Ablk^T V.  Products for a true residual b - A x take FP64
        products whatever the iteration's arithmetic, as gpch_cg_solve_ex
        does: they bound the accuracy the iteration can reach."""
        prod = "fp64" if true_residual else self.products
        gpchol.block_matvec(self.A, self.r0, self.V, out, prod, ctx=self.ctx)

    def residual(self, all_columns: bool):
        gpchol.cgsr_residual(self.state, self.B, self.T, self.R, all_columns, ctx=self.ctx)

    def partials(self):
        gpchol.cgsr_partials(self.R, self.W, self.sums, ctx=self.ctx)

    def scalars(self, first: bool, rtol: float, maxit: int):
        gpchol.cgsr_scalars(self.sums, self.state, self.nrhs, first, rtol, maxit, ctx=self.ctx)

    def vectors(self, replace: bool):
        gpchol.cgsr_vectors(self.state, self.X, self.R, self.W, self.P, self.S, replace, ctx=self.ctx)

    def _ints(self):
        return self.state[4 * 16 * 8:].view(torch.int32).cpu()

    def done(self) -> bool:
        return bool(self._ints()[32].item())

    def stats(self):
        """(iterations per column, sqrt(gamma / gamma_0) per column)."""
        d = self.state[:4 * 16 * 8].view(torch.float64).cpu()
        ints = self._ints()
        gam, gam0 = d[:16], d[16:32]
        rel = [float((gam[c] / gam0[c]).sqrt()) if gam0[c] > 0 else 0.0 for c in range(self.nrhs)]
        return [int(ints[16 + c]) for c in range(self.nrhs)], rel


def rowsplit_cg(comm, ops, rtol: float = 1e-10, maxit: int = 10000, replace_every: int = 50,
                check_every: int = 16):
    """Single-reduction CG on row-split ranks (see the module docstring).
    Every rank calls it with its own `ops`.  Returns (iterations per
    column, sqrt(gamma / gamma_0) per column, loop iterations run); the
    loop checks the common stop every `check_every` iterations, so it may
    run a few iterations past the last column's stop (they change
    nothing: retired columns are frozen)."""
    # r = b - A x0
    comm.allgather_rows(ops.X, ops.V)
    ops.product(ops.T, true_residual=True)
    ops.residual(True)
    # w = A r, gamma_0, delta_0, alpha_0
    comm.allgather_rows(ops.R, ops.V)
    ops.product(ops.W)
    ops.partials()
    comm.allreduce_sum(ops.sums)
    ops.scalars(True, rtol, maxit)
    it = 0
    while it < maxit and not ops.done():
        for _ in range(min(check_every, maxit - it)):
            it += 1
            replace = replace_every > 0 and it % replace_every == 0
            ops.vectors(replace)
            if replace:
                comm.allgather_rows(ops.X, ops.V)
                ops.product(ops.T, true_residual=True)
                ops.residual(False)
                comm.allgather_rows(ops.P, ops.V)
                ops.product(ops.S)
            comm.allgather_rows(ops.R, ops.V)
            ops.product(ops.W)
            ops.partials()
            comm.allreduce_sum(ops.sums)
            ops.scalars(False, rtol, maxit)
    iters, rel = ops.stats()
    return iters, rel, it
