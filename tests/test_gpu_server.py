"""GPU tests of the serving loop (A11): results match the oracle; a request's
result is the same alone and inside a mix of concurrent requests; the HBM
budget bounds the memory of admitted requests; oversize requests are
refused at submission."""
import numpy as np
import pytest

import oracle
from paper_2605_13209_b300 import gpchol, inputs

pytestmark = pytest.mark.gpu


def req(n, nrhs, seed, ell=0.5, sn2=1e-2):
    s = inputs.gp_system(n, 8, ell, sn2, nrhs=nrhs, seed=5000 + seed)
    return s


def check(s, X, tol):
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    for r in range(s.nrhs):
        assert oracle.backward_error(A, X[:, r], s.B[:, r]) <= tol


def test_server_alone_vs_mix():
    srv = gpchol.Server(0, hbm_budget=8 << 30, lanes=3, batch_max_count=8, batch_max_n=512, solo_prec="split_bf16")
    probe_small = req(300, 2, 1)
    probe_large = req(1100, 1, 2, sn2=1e-3)
    # alone
    t = srv.submit(probe_small.X, probe_small.B, probe_small.sf2, probe_small.ell, probe_small.sn2)
    x_small_alone, r1 = srv.wait(t)
    assert r1["status"] == 0 and r1["path"] == 1
    t = srv.submit(probe_large.X, probe_large.B, probe_large.sf2, probe_large.ell, probe_large.sn2)
    x_large_alone, r2 = srv.wait(t)
    assert r2["status"] == 0 and r2["path"] == 2
    check(probe_small, x_small_alone, 1e-13)
    check(probe_large, x_large_alone, 1e-12)
    # the same two requests inside a mix of concurrent small and large ones
    rng = np.random.default_rng(0)
    mix = []
    for i in range(24):
        n = int(rng.choice([64, 100, 257, 400, 512, 700, 900]))
        mix.append(req(n, int(rng.integers(1, 4)), 100 + i))
    tickets = []
    for i, s in enumerate(mix):
        tickets.append((s, srv.submit(s.X, s.B, s.sf2, s.ell, s.sn2)))
        if i == 5:
            ts = srv.submit(probe_small.X, probe_small.B, probe_small.sf2, probe_small.ell, probe_small.sn2)
        if i == 9:
            tl = srv.submit(probe_large.X, probe_large.B, probe_large.sf2, probe_large.ell, probe_large.sn2)
    xs, _ = srv.wait(ts)
    xl, _ = srv.wait(tl)
    assert np.array_equal(xs, x_small_alone)
    assert np.array_equal(xl, x_large_alone)
    for s, t in tickets:
        x, r = srv.wait(t)
        assert r["status"] == 0
        check(s, x, 1e-13 if s.n <= 512 else 1e-12)
    st = srv.stats()
    assert st["completed"] == 2 + 24 + 2 and st["failed"] == 0
    assert st["batches"] >= 1 and st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
    srv.close()


def test_server_batches_queued_small_requests():
    """Continuous batching: three large requests occupy the three lanes,
    twelve small ones arrive meanwhile and queue; the first lane to free
    takes up to batch_max_count of them in one batched launch, so at least
    one batch holds several requests.  Each result still matches the
    oracle, and every small result is bit-identical to the same request
    solved alone."""
    srv = gpchol.Server(0, hbm_budget=16 << 30, lanes=3, batch_max_count=8, batch_max_n=512,
                        solo_prec="split_f16")
    smalls = [req(int(n), 1 + i % 3, 600 + i) for i, n in enumerate(np.linspace(100, 512, 12).astype(int))]
    alone = []
    for s in smalls:
        x, r = srv.wait(srv.submit(s.X, s.B, s.sf2, s.ell, s.sn2))
        assert r["status"] == 0 and r["path"] == 1
        alone.append(x)
    before = srv.stats()
    larges = [req(4096, 1, 700 + i, sn2=1e-3) for i in range(3)]
    tl = [srv.submit(s.X, s.B, s.sf2, s.ell, s.sn2) for s in larges]
    ts = [srv.submit(s.X, s.B, s.sf2, s.ell, s.sn2) for s in smalls]
    for s, t, xa in zip(smalls, ts, alone):
        x, r = srv.wait(t)
        assert r["status"] == 0 and r["path"] == 1
        assert np.array_equal(x, xa)
    for s, t in zip(larges, tl):
        x, r = srv.wait(t)
        assert r["status"] == 0 and r["path"] == 2
        assert r["backward_error"] <= 1e-12
    after = srv.stats()
    batches = after["batches"] - before["batches"]
    grouped = after["batched_requests"] - before["batched_requests"]
    assert grouped == 12
    assert batches < grouped          # some batch held two or more requests
    srv.close()


def test_server_budget_and_fp64_path():
    budget = 64 << 20
    srv = gpchol.Server(0, hbm_budget=budget, lanes=2, batch_max_count=4, batch_max_n=300, solo_prec="fp64")
    reqs = [req(n, 1, 300 + i) for i, n in enumerate([200, 280, 600, 800, 150, 1000, 250])]
    ts = [srv.submit(s.X, s.B, s.sf2, s.ell, s.sn2) for s in reqs]
    for s, t in zip(reqs, ts):
        x, r = srv.wait(t)
        assert r["status"] == 0 and r["path"] in (1, 3)
        check(s, x, 1e-13)
    st = srv.stats()
    assert 0 < st["peak_reserved_bytes"] <= budget
    with pytest.raises(gpchol.GpchError):
        big = req(4000, 1, 999)
        srv.submit(big.X, big.B, big.sf2, big.ell, big.sn2)   # 128 MB matrix > 64 MB budget
    srv.close()
