"""Seeded synthetic inputs shared by the CUDA path, the oracle and the bench.

This module holds none of the solvers' arithmetic: it only draws the random
numbers that define a workload (GP training points, right-hand sides,
hyper-parameters, batch sizes, request arrival times).  The squared-
exponential matrix itself is built from these points by each side on its
own (the oracle on the host, the A1 kernel on the device).

The paper's matrices are GP covariance matrices of a mass-spring-damper
dataset (Sec. 4.1) that is not available; squared-exponential kernels of
uniform points in [0,1]^d stand in for them.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

SEED_X = 0xC0F1   # + config index
SEED_B = 0xB0F1   # + config index
SEED_ARRIVALS = 0x5E7E


@dataclass
class GPSystem:
    """One GP system: points X (n x d, row-major), SE hyper-parameters and
    right-hand sides B (n x nrhs, column-major)."""
    X: np.ndarray
    B: np.ndarray
    sf2: float
    ell: float
    sn2: float

    @property
    def n(self) -> int:
        return self.X.shape[0]

    @property
    def d(self) -> int:
        return self.X.shape[1]

    @property
    def nrhs(self) -> int:
        return self.B.shape[1]


def points(n: int, d: int, seed: int) -> np.ndarray:
    """n points i.i.d. uniform on [0,1]^d, row-major float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.ascontiguousarray(rng.random((n, d)))


def rhs(n: int, nrhs: int, seed: int) -> np.ndarray:
    """n x nrhs standard-normal right-hand sides, column-major float64."""
    rng = np.random.Generator(np.random.PCG64(seed))
    return np.asfortranarray(rng.standard_normal((nrhs, n)).T)


def gp_system(n: int, d: int = 8, ell: float = 0.5, sn2: float = 1e-2, sf2: float = 1.0,
              nrhs: int = 1, seed: int = 0) -> GPSystem:
    return GPSystem(points(n, d, SEED_X + seed), rhs(n, nrhs, SEED_B + seed), sf2, ell, sn2)


# The five workloads (Sec. 4.1 GP systems, synthetic; sizes from the scope table).
def config1() -> GPSystem:
    """n=2048, d=8, ell=0.5, sn2=1e-2, one RHS (FP64, tile 256 / CG 1e-10)."""
    return gp_system(2048, 8, 0.5, 1e-2, 1.0, 1, seed=1)


def config2(n: int = 32768) -> GPSystem:
    """n=32768, d=8, ell=0.5, sn2=1e-3, one RHS (FP64 tile 512 vs mixed)."""
    return gp_system(n, 8, 0.5, 1e-3, 1.0, 1, seed=2)


def config3(n: int = 65536, nrhs: int = 16) -> GPSystem:
    """n=65536, d=8, ell=0.3, sn2=1e-1, 16 RHS (CG-bound)."""
    return gp_system(n, 8, 0.3, 1e-1, 1.0, nrhs, seed=3)


@dataclass
class BatchSpec:
    ns: np.ndarray
    ells: np.ndarray
    sn2s: np.ndarray
    seeds: np.ndarray

    def system(self, k: int, d: int = 8) -> GPSystem:
        n = int(self.ns[k])
        s = int(self.seeds[k])
        return GPSystem(points(n, d, s), rhs(n, 1, s + 1), 1.0, float(self.ells[k]),
                        float(self.sn2s[k]))


def batch_spec(count: int = 256, nmin: int = 256, nmax: int = 4096, seed: int = 4) -> BatchSpec:
    """Batched workload: n log-uniform in [nmin, nmax], ell ~ U[0.2, 1.0],
    sn2 ~ U[1e-3, 1e-1], one RHS each."""
    rng = np.random.Generator(np.random.PCG64(SEED_X + seed))
    ns = np.exp(rng.uniform(np.log(nmin), np.log(nmax), count)).astype(np.int64)
    ns = np.clip(ns, nmin, nmax)
    ells = rng.uniform(0.2, 1.0, count)
    sn2s = rng.uniform(1e-3, 1e-1, count)
    seeds = (SEED_X * 1000 + np.arange(count) * 2).astype(np.int64)
    return BatchSpec(ns, ells, sn2s, seeds)


@dataclass
class RequestStream:
    arrival_s: np.ndarray
    ns: np.ndarray
    nrhs: np.ndarray
    ells: np.ndarray
    sn2s: np.ndarray
    seeds: np.ndarray = field(default=None)


def request_stream(count: int = 10000, rate_per_s: float = 100.0, nmin: int = 512,
                   nmax: int = 16384, seed: int = SEED_ARRIVALS) -> RequestStream:
    """Serving workload: Poisson arrivals at rate_per_s, n log-uniform in
    [nmin, nmax], 1-8 RHS, ell ~ U[0.2, 1.0], sn2 ~ U[1e-3, 1e-1]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_per_s, count)
    ns = np.clip(np.exp(rng.uniform(np.log(nmin), np.log(nmax), count)).astype(np.int64), nmin, nmax)
    nrhs = rng.integers(1, 9, count)
    ells = rng.uniform(0.2, 1.0, count)
    sn2s = rng.uniform(1e-3, 1e-1, count)
    seeds = (seed * 100000 + np.arange(count) * 2).astype(np.int64)
    return RequestStream(np.cumsum(gaps), ns, nrhs, ells, sn2s, seeds)
