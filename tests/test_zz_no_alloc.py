"""The allocation-free CG entry point (gpch_cg_solve_noalloc) against the
allocating one (gpch_cg_solve), through the C ABI, on two calls in a row.

Some callers cannot allocate device memory (a host framework that owns the
GPU memory budget, a real-time loop that cannot take the allocator's
synchronization, a caller without a library context); this entry point
serves them from a fixed library-owned scratch array, so the second call
also checks that what the first call left in that array does not leak into
the next result.  This file is collected last on purpose."""
import os
import subprocess
import sys

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


def test_noalloc_cg_f32_storage_and_size_limit():
    """FP32-stored A (widened exactly, the same operator for both entry
    points), and the largest accepted problem: n * nrhs = 262144 with 16
    right-hand sides, the widest partial-sum layout."""
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    torch.cuda.set_device(0)
    ctx = gpchol.Context(0)
    for n, nrhs, dtype in [(900, 5, torch.float32), (16384, 16, torch.float64)]:
        assert n * nrhs <= 262144
        s = inputs.gp_system(n, 8, 0.3, 1e-1, nrhs=nrhs, seed=13)
        Xd = torch.from_numpy(s.X).cuda()
        Ad = gpchol.se_matrix(Xd, s.sf2, s.ell, s.sn2, ctx=ctx).to(dtype)
        Ad = gpchol.as_colmajor(Ad)
        Bd = _dev(s.B)
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
        for r in range(nrhs):
            assert oracle.forward_error(xn[:, r], xa[:, r]) <= 1e-12
        del Ad
    ctx.close()


_FIRST_CALL_CHILD = r"""
import numpy as np, torch
from paper_2605_13209_b300 import gpchol
torch.cuda.set_device(0)
n, nrhs = 600, 2
rng = np.random.default_rng(3)
Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
A = (Q * np.linspace(1.0, 50.0, n)) @ Q.T
A = 0.5 * (A + A.T)
B = rng.standard_normal((n, nrhs))
Ad = gpchol.as_colmajor(torch.from_numpy(A).cuda())
Bd = gpchol.as_colmajor(torch.from_numpy(B).cuda())
X1 = gpchol.colmajor(n, nrhs); X1.zero_()
X2 = gpchol.colmajor(n, nrhs); X2.zero_()
torch.cuda.synchronize()
lib = gpchol.lib()
# the set-up call is this process's first call into the library on the device
st = lib.gpch_cg_solve_noalloc(0, None, gpchol.GPCH_F64, 1, None, 1, None, 1, 0, 1e-10, 1, 0, None, None)
assert st == gpchol.GPCH_OK, st
torch.cuda.synchronize()
free0 = torch.cuda.mem_get_info()[0]
r1 = gpchol.cg_solve_noalloc(Ad, Bd, X1, rtol=1e-12, maxit=2000)
r2 = gpchol.cg_solve_noalloc(Ad, Bd, X2, rtol=1e-12, maxit=2000)
torch.cuda.synchronize()
free1 = torch.cuda.mem_get_info()[0]
assert r1.status == r2.status == gpchol.GPCH_OK
x_ref = np.linalg.solve(A, B)
x1, x2 = X1.cpu().numpy(), X2.cpu().numpy()
assert np.array_equal(x1, x2)
assert np.linalg.norm(x1 - x_ref) / np.linalg.norm(x_ref) <= 1e-9
print("FREE", free0, free1)
assert free1 == free0, (free0, free1)
print("CHILD_OK")
"""


def test_noalloc_cg_first_call_in_fresh_process():
    """In a process whose first library call on the device is the set-up
    call (n = 0), the solves after it leave the device's free memory
    unchanged, and two solves of the same system agree bit for bit."""
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = dict(os.environ, PYTHONPATH=root + os.pathsep + os.environ.get("PYTHONPATH", ""))
    r = subprocess.run([sys.executable, "-c", _FIRST_CALL_CHILD], cwd=root, env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0 and "CHILD_OK" in r.stdout, r.stdout + r.stderr


def test_noalloc_cg_rejects_oversize():
    if not torch.cuda.is_available():
        pytest.fail("GPU test run without a CUDA device")
    n = 262145
    A = torch.empty(1, dtype=torch.float64, device="cuda")   # never read: the size check comes first
    lib = gpchol.lib()
    st = lib.gpch_cg_solve_noalloc(n, A.data_ptr(), gpchol.GPCH_F64, n, A.data_ptr(), n, A.data_ptr(), n, 1, 1e-10,
                                   10, 0, None, None)
    assert st == gpchol.GPCH_INVALID_ARG
    # 16 right-hand sides: n * nrhs = 262160 > 262144 is rejected as well
    st = lib.gpch_cg_solve_noalloc(16385, A.data_ptr(), gpchol.GPCH_F64, 16385, A.data_ptr(), 16385, A.data_ptr(),
                                   16385, 16, 1e-10, 10, 0, None, None)
    assert st == gpchol.GPCH_INVALID_ARG
    # more than 16 right-hand sides is rejected whatever n
    st = lib.gpch_cg_solve_noalloc(10, A.data_ptr(), gpchol.GPCH_F64, 10, A.data_ptr(), 10, A.data_ptr(), 10, 17,
                                   1e-10, 10, 0, None, None)
    assert st == gpchol.GPCH_INVALID_ARG
