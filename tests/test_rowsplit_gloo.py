"""The row-split CG driver (paper_2605_13209_b300/rowsplit.py) on the CPU:
2 or 3 ranks in a gloo process group, each owning a contiguous block of
rows of the SE system (the paper's horizontal split, Sec. 3.1, carried to
one GPU per rank).  The ranks' local arithmetic is a plain torch-CPU
restatement of the library's gpch_block_matvec / gpch_cgsr_* steps (test
infrastructure; on GPUs the same driver calls the library), so what is
checked here is the driver: the row partition, the allgather of the
product's vector, the allreduce of the two sums, the replacement schedule
and the common stop.  Results are compared with the oracle's
single-reduction CG (Algorithm 1 left, Chronopoulos-Gear form) on the whole
system."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

WORKER = r"""
import json, os, sys
sys.path.insert(0, os.environ["ROOT_DIR"])
import numpy as np
import torch
import torch.distributed as dist
dist.init_process_group("gloo")
import oracle
from paper_2605_13209_b300 import inputs, rowsplit

n, nrhs, R, seed = (int(os.environ[k]) for k in ("N", "NRHS", "R", "SEED"))
rank, world = dist.get_rank(), dist.get_world_size()
s = inputs.gp_system(n, 8, 0.5, 1e-2, nrhs=nrhs, seed=seed)
A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
offs, sizes = rowsplit.partition(n, world)
o, m = offs[rank], sizes[rank]


class CpuRankOps:
    # torch-CPU restatement of the library's local steps (see gpchol.h, f4)
    def __init__(self):
        self.A = torch.from_numpy(np.ascontiguousarray(A[:, o:o + m]))
        self.B = torch.from_numpy(np.ascontiguousarray(s.B[o:o + m, :]))
        self.X = torch.zeros((m, nrhs), dtype=torch.float64)
        self.V = torch.zeros((n, nrhs), dtype=torch.float64)
        self.R, self.W, self.P, self.S, self.T = (torch.zeros((m, nrhs), dtype=torch.float64) for _ in range(5))
        self.sums = torch.zeros(2 * nrhs, dtype=torch.float64)
        self.gamma = np.zeros(nrhs); self.gamma0 = np.zeros(nrhs)
        self.alpha = np.zeros(nrhs); self.beta = np.zeros(nrhs)
        self.active = np.zeros(nrhs, dtype=bool); self.iters = np.zeros(nrhs, dtype=int)
        self.is_done = False
        self.products = 0

    def product(self, out, true_residual=False):
        out[:] = self.A.t() @ self.V
        self.products += 1

    def residual(self, all_columns):
        for c in range(nrhs):
            if all_columns or (self.active[c] and not self.is_done):
                self.R[:, c] = self.B[:, c] - self.T[:, c]

    def partials(self):
        self.sums[:nrhs] = (self.R * self.R).sum(0)
        self.sums[nrhs:] = (self.W * self.R).sum(0)

    def scalars(self, first, rtol, maxit):
        g = self.sums[:nrhs].numpy().copy(); d = self.sums[nrhs:].numpy().copy()
        for c in range(nrhs):
            if first:
                self.gamma0[c] = self.gamma[c] = g[c]
                self.iters[c] = 0; self.beta[c] = 0.0
                self.alpha[c] = g[c] / d[c] if g[c] > 0 else 0.0
                self.active[c] = g[c] > 0
            elif self.active[c]:
                self.iters[c] += 1
                b = g[c] / self.gamma[c]
                self.alpha[c] = g[c] / (d[c] - b * g[c] / self.alpha[c])
                self.beta[c] = b; self.gamma[c] = g[c]
                if g[c] <= rtol * rtol * self.gamma0[c] or self.iters[c] >= maxit:
                    self.active[c] = False
        self.is_done = not self.active.any()

    def vectors(self, replace):
        if self.is_done:
            return
        for c in range(nrhs):
            if not self.active[c]:
                continue
            a, b = self.alpha[c], self.beta[c]
            self.P[:, c] = self.R[:, c] + b * self.P[:, c]
            self.S[:, c] = self.W[:, c] + b * self.S[:, c]
            self.X[:, c] += a * self.P[:, c]
            if not replace:
                self.R[:, c] -= a * self.S[:, c]

    def done(self):
        return self.is_done

    def stats(self):
        rel = [float(np.sqrt(self.gamma[c] / self.gamma0[c])) if self.gamma0[c] > 0 else 0.0 for c in range(nrhs)]
        return [int(i) for i in self.iters], rel


ops = CpuRankOps()
comm = rowsplit.TorchComm(n)
iters, rel, loops = rowsplit.rowsplit_cg(comm, ops, rtol=1e-10, maxit=5000, replace_every=R)
full = torch.zeros((n, nrhs), dtype=torch.float64)
comm.allgather_rows(ops.X, full)
dist.barrier()
dist.destroy_process_group()
out = {"rank": rank, "world": world, "rows": [o, m], "iters": iters, "relres": rel, "products": ops.products, "loops": loops}
if rank == 0:
    X = full.numpy()
    ref = []
    for c in range(nrhs):
        x_or, it_or, _ = oracle.cg_single_reduction(A, s.B[:, c], 1e-10, 5000, R=R)
        ref.append({"it": it_or, "fwd": oracle.forward_error(X[:, c], x_or),
                    "true": float(np.linalg.norm(s.B[:, c] - A @ X[:, c]) / np.linalg.norm(s.B[:, c]))})
    out["ref"] = ref
print(json.dumps(out))
"""


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _run(world, n, nrhs, R, seed):
    port = _free_port()
    procs = []
    for rank in range(world):
        env = dict(os.environ, ROOT_DIR=ROOT, MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                   WORLD_SIZE=str(world), LOCAL_RANK=str(rank), N=str(n), NRHS=str(nrhs), R=str(R),
                   SEED=str(seed), OMP_NUM_THREADS="1")
        procs.append(subprocess.Popen([sys.executable, "-c", WORKER], env=env, stdout=subprocess.PIPE,
                                      stderr=subprocess.PIPE, text=True))
    outs = []
    for p in procs:
        out, err = p.communicate(timeout=300)
        assert p.returncode == 0, err
        outs.append(json.loads(out.strip().splitlines()[-1]))
    return sorted(outs, key=lambda o: o["rank"])


def test_partition():
    from paper_2605_13209_b300.rowsplit import partition
    assert partition(10, 3) == ([0, 4, 7], [4, 3, 3])
    assert partition(8, 2) == ([0, 4], [4, 4])
    offs, sizes = partition(65536, 8)
    assert sizes == [8192] * 8 and offs[-1] == 7 * 8192
    offs, sizes = partition(5, 8)          # more ranks than rows: empty blocks at the end
    assert sum(sizes) == 5 and sizes[-1] == 0


@pytest.mark.parametrize("world,n,nrhs,R", [(2, 300, 1, 50), (3, 301, 3, 7), (2, 257, 2, 0)])
def test_rowsplit_cg_gloo_matches_oracle(world, n, nrhs, R):
    outs = _run(world, n, nrhs, R, seed=900 + n)
    # the partition covers the rows once, in rank order
    rows = [o["rows"] for o in outs]
    assert rows[0][0] == 0 and sum(m for _, m in rows) == n
    for a, b in zip(rows, rows[1:]):
        assert b[0] == a[0] + a[1]
    # every rank ran the same iterations and stopped together
    for o in outs[1:]:
        assert o["iters"] == outs[0]["iters"] and o["products"] == outs[0]["products"]
    for c, ref in enumerate(outs[0]["ref"]):
        assert outs[0]["relres"][c] <= 1e-10
        assert ref["true"] <= 1e-9
        assert abs(outs[0]["iters"][c] - ref["it"]) <= max(3, 0.05 * ref["it"])
        assert ref["fwd"] <= 1e-6
    # two set-up products, one per loop iteration, two more per replacement;
    # the loop stops at the first check after the last column retired
    it = outs[0]["loops"]
    assert max(outs[0]["iters"]) <= it < max(outs[0]["iters"]) + 16
    extra = 2 * (it // R) if R > 0 else 0
    assert outs[0]["products"] == 2 + it + extra
