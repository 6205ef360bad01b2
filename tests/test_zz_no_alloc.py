"""The allocation-free CG entry point (gpch_cg_solve_noalloc) against the
allocating one (gpch_cg_solve), through the C ABI, on two calls in a row.

Some callers cannot allocate device memory (a host framework that owns the
GPU memory budget, a real-time loop that cannot take the allocator's
synchronization, a caller without a library context); this entry point
serves them from a fixed library-owned scratch array, so the second call
also checks that what the first call left in that array does not leak into
the next result.  This file is collected last on purpose."""
import numpy as np
import pytest
import torch

import oracle
from paper_2605_13209_b300 import gpchol, inputs

pytestmark = pytest.mark.gpu


def _dev(a, dtype=torch.float64):
    a = np.asarray(a)
    if a.ndim == 1:
        a = a[:, None]
    t = gpchol.colmajor(a.shape[0], a.shape[1], dtype=dtype)
    t.copy_(torch.from_numpy(np.ascontiguousarray(a)).to(dtype))
    return t


def test_noalloc_cg_matches_allocating_cg_twice():
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    torch.cuda.set_device(0)
    ctx = gpchol.Context(0)
    cases = [(700, 3, 1e-2, 11), (1000, 1, 1e-1, 12)]   # two different systems, back to back
    for n, nrhs, sn2, seed in cases:
        s = inputs.gp_system(n, 8, 0.5, sn2, nrhs=nrhs, seed=seed)
        A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
        Ad, Bd = _dev(A), _dev(s.B)
        Xa = gpchol.colmajor(n, nrhs)
        Xa.zero_()
        ra = gpchol.cg_solve(Ad, Bd, Xa, rtol=1e-10, maxit=5000, replace_every=50, ctx=ctx)
        Xn = gpchol.colmajor(n, nrhs)
        Xn.zero_()
        rn = gpchol.cg_solve_noalloc(Ad, Bd, Xn, rtol=1e-10, maxit=5000, replace_every=50)
        torch.cuda.synchronize()
        assert rn.status == gpchol.GPCH_OK and rn.converged == nrhs
        assert rn.iterations == ra.iterations
        xa, xn = Xa.cpu().numpy(), Xn.cpu().numpy()
        # same kernels on the same inputs; held to the CG tests' tolerance
        for r in range(nrhs):
            assert oracle.forward_error(xn[:, r], xa[:, r]) <= 1e-12
            rel = np.linalg.norm(s.B[:, r] - A @ xn[:, r]) / np.linalg.norm(s.B[:, r])
            assert rel <= 1e-9
    ctx.close()


def test_noalloc_cg_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    n = 262145
    A = torch.empty(1, dtype=torch.float64, device="cuda")   # never read: the size check comes first
    lib = gpchol.lib()
    st = lib.gpch_cg_solve_noalloc(n, A.data_ptr(), gpchol.GPCH_F64, n, A.data_ptr(), n, A.data_ptr(), n, 1, 1e-10,
                                   10, 0, None, None)
    assert st == gpchol.GPCH_INVALID_ARG
