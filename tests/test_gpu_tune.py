"""GPU tests of the autotuner (gpch_autotune): a measured table holds only
valid choices and is cached as JSON under the GPU's name; a later call
loads it; the batched solves give bit-identical results whatever update
tile the table picks; the refined solve takes the tuned tile when asked
for tile 0.  The table is process-wide, so the last test puts the default
table back (by loading it) for the tests that follow."""
import json

import numpy as np
import pytest
import torch

import oracle
from paper_2605_13209_b300 import gpchol, inputs
from gpu_helpers import ctx, dev, host  # noqa: F401

pytestmark = pytest.mark.gpu

DEFAULT = {"refined_tile": [256, 256, 256, 256, 512, 512, 512, 512, 512],
           "batch_tile_fp64": [64] * 9, "batch_tile_mixed": [64] * 9}


def _write(path, gpu, table):
    with open(path, "w") as f:
        json.dump({gpu: table}, f)


def test_autotune_measures_caches_and_loads(ctx, tmp_path):
    before = gpchol.tune_get(ctx=ctx)
    assert before["source"] in ("defaults", "loaded", "measured")
    path = str(tmp_path / "tune.json")
    t = gpchol.autotune(path, force=True, nmax=2048, ctx=ctx)
    assert t["source"] == "measured"
    assert all(v in (256, 384, 512) for v in t["refined_tile"])
    assert all(v in (32, 64) for v in t["batch_tile_fp64"] + t["batch_tile_mixed"])
    cached = json.load(open(path))
    assert t["gpu"] in cached
    assert cached[t["gpu"]]["refined_tile"] == t["refined_tile"]
    again = gpchol.autotune(path, ctx=ctx)
    assert again["source"] == "loaded"
    for k in ("refined_tile", "batch_tile_fp64", "batch_tile_mixed"):
        assert again[k] == t[k]
    # another GPU's entry in the same file is kept on rewrite
    data = json.load(open(path))
    data["some other GPU"] = DEFAULT
    json.dump(data, open(path, "w"))
    gpchol.autotune(path, force=True, nmax=1024, ctx=ctx)
    assert set(json.load(open(path))) == {t["gpu"], "some other GPU"}


def test_batched_results_do_not_depend_on_the_update_tile(ctx, tmp_path):
    gpu = gpchol.tune_get(ctx=ctx)["gpu"]
    ns = [300, 700, 129, 1100]
    syss = [inputs.gp_system(n, 8, 0.5, 1e-2, nrhs=1, seed=1200 + n) for n in ns]
    As = [oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2) for s in syss]
    out = {}
    for bt in (32, 64):
        path = str(tmp_path / f"t{bt}.json")
        _write(path, gpu, {"refined_tile": DEFAULT["refined_tile"], "batch_tile_fp64": [bt] * 9,
                           "batch_tile_mixed": [bt] * 9})
        assert gpchol.autotune(path, ctx=ctx)["batch_tile_fp64"] == [bt] * 9
        Ad = [dev(A) for A in As]
        Bd = [dev(s.B) for s in syss]
        assert gpchol.batched_solve(Ad, Bd, ctx=ctx) == [0] * len(ns)
        Am = [dev(A) for A in As]
        Bm = [dev(s.B) for s in syss]
        Xm = [gpchol.colmajor(s.n, 1) for s in syss]
        res = gpchol.batched_solve_mixed(Am, Bm, Xm, ctx=ctx)
        assert res.info == [0] * len(ns)
        out[bt] = ([host(a) for a in Ad], [host(b) for b in Bd], [host(x) for x in Xm])
    for k in range(3):
        for u, v in zip(out[32][k], out[64][k]):
            assert np.array_equal(u, v)
    for A, s, x in zip(As, syss, out[32][2]):
        assert oracle.backward_error(A, x[:, 0], s.B[:, 0]) <= 1e-12


def test_refined_tile_zero_takes_the_table_then_restore(ctx, tmp_path):
    gpu = gpchol.tune_get(ctx=ctx)["gpu"]
    path = str(tmp_path / "t384.json")
    tiles = [384] * 9
    _write(path, gpu, {"refined_tile": tiles, "batch_tile_fp64": [64] * 9, "batch_tile_mixed": [64] * 9})
    assert gpchol.autotune(path, ctx=ctx)["refined_tile"] == tiles
    s = inputs.gp_system(1500, 8, 0.5, 1e-3, nrhs=1, seed=1300)
    A = oracle.se_matrix(s.X, s.sf2, s.ell, s.sn2)
    Ad = dev(A)
    X0, X384 = gpchol.colmajor(1500, 1), gpchol.colmajor(1500, 1)
    gpchol.solve_refined(Ad, dev(s.B), X0, prec="split_f16", tile=0, ctx=ctx)
    gpchol.solve_refined(Ad, dev(s.B), X384, prec="split_f16", tile=384, ctx=ctx)
    assert np.array_equal(host(X0), host(X384))
    assert oracle.backward_error(A, host(X0)[:, 0], s.B[:, 0]) <= 1e-12
    # put the default table back for the tests that follow
    path = str(tmp_path / "default.json")
    _write(path, gpu, DEFAULT)
    t = gpchol.autotune(path, ctx=ctx)
    assert t["refined_tile"] == DEFAULT["refined_tile"] and t["batch_tile_fp64"] == [64] * 9
