"""Seeded synthetic inputs shared by the tests, the benchmark and the oracle runs.

This module holds no arithmetic of the method (no sampling from the power law,
no fitting, no KS).  It only defines the workload configurations -- which
(alpha, xmin, n, replicates) cells to run, the batched-instance mix and the
serving request stream -- and the rounded-lognormal alternative data used to
check the power of the bootstrap test.  Power-law data sets themselves are
drawn by the method's own sampler with stream tag 2 (test data).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

# stream tags of the Philox counter's last word
PURPOSE_CUTOFFS = 0
PURPOSE_BOOTSTRAP = 1
PURPOSE_TESTDATA = 2

QUANTILES = (0.90, 0.95, 0.99)


@dataclass(frozen=True)
class Cell:
    alpha: float
    xmin: int
    n: int
    replicates: int
    cell_id: int


def cutoff_cell_small() -> list[Cell]:
    """Plain method, FP64: alpha = 2.5, xmin = 1, n = 100, 10,000 replicates."""
    return [Cell(2.5, 1, 100, 10_000, 0)]


SWEEP_ALPHAS = (1.5, 1.75, 2.0, 2.25, 2.5, 2.75, 3.0, 3.25, 3.5)
SWEEP_NS = (10, 20, 50, 100, 200, 500, 1000, 2000, 5000, 10000)


def cutoff_table_sweep(replicates: int = 100_000) -> list[Cell]:
    """Cutoff-table sweep: 9 exponents x 10 sample sizes, xmin = 1; cell id =
    10 * (exponent index) + (size index)."""
    return [Cell(a, 1, n, replicates, 10 * i + j)
            for i, a in enumerate(SWEEP_ALPHAS) for j, n in enumerate(SWEEP_NS)]


def large_n_cell(replicates: int = 10_000) -> list[Cell]:
    """Large-n heavy tail: alpha = 2.0, n = 1,000,000 per replicate."""
    return [Cell(2.0, 1, 1_000_000, replicates, 0)]


def batched_instances(count: int = 4096, replicates: int = 2000, seed: int = 2) -> list[Cell]:
    """Uneven batch: n log-uniform in [10, 1e5] (rounded), alpha uniform in
    [1.6, 3.2], xmin uniform over {1, 2, 5}; cell id = instance index."""
    rng = np.random.default_rng(seed)
    n = np.rint(np.exp(rng.uniform(np.log(10.0), np.log(1e5), count))).astype(np.int64)
    alpha = rng.uniform(1.6, 3.2, count)
    xmin = rng.choice(np.array([1, 2, 5]), count)
    return [Cell(float(alpha[i]), int(xmin[i]), int(n[i]), replicates, i) for i in range(count)]


@dataclass(frozen=True)
class Request:
    request_id: int
    arrival_s: float
    n: int
    alpha: float          # exponent of the power-law data (unused when lognormal)
    xmin: int
    lognormal: bool


def serving_requests(duration_s: float, rate_per_s: float = 200.0, seed: int = 4,
                     n_lo: float = 50, n_hi: float = 1e6, lognormal_frac: float = 0.1
                     ) -> list[Request]:
    """Open-loop Poisson arrivals of fit requests: n log-uniform in [n_lo, n_hi],
    alpha uniform in [1.5, 3.5], xmin = 1; a fraction carries rounded-lognormal
    data instead of power-law data."""
    rng = np.random.default_rng(seed)
    out = []
    t = 0.0
    i = 0
    while True:
        t += rng.exponential(1.0 / rate_per_s)
        if t > duration_s:
            break
        n = int(np.rint(np.exp(rng.uniform(np.log(n_lo), np.log(n_hi)))))
        out.append(Request(i, t, n, float(rng.uniform(1.5, 3.5)), 1,
                           bool(rng.random() < lognormal_frac)))
        i += 1
    return out


def rounded_lognormal(rng: np.random.Generator, n: int, mu: float = 2.0, sigma: float = 1.0,
                      xmin: int = 1) -> np.ndarray:
    """int32 data: exp(mu + sigma Z) rounded half to even; values below xmin redrawn."""
    out = np.empty(n, dtype=np.int64)
    filled = 0
    while filled < n:
        v = np.rint(np.exp(mu + sigma * rng.standard_normal(n - filled)))
        v = v[(v >= xmin) & (v < 2**31 - 1)]
        out[filled:filled + v.size] = v.astype(np.int64)
        filled += v.size
    return out.astype(np.int32)


INT32_MAX = 2**31 - 1


def as_request_data(values) -> np.ndarray:
    """Fit requests carry int32 data: sampled values above 2^31 - 1 (the far
    tail at exponents near 1.5, a few per million draws) are clamped to it."""
    v = np.asarray(values).view(np.uint64) if np.asarray(values).dtype == np.int64 else np.asarray(values)
    return np.minimum(v.astype(np.uint64), np.uint64(INT32_MAX)).astype(np.int32)


# Table 1 of the paper: 8 exponents x 15 sample sizes, xmin = 1, 50,000
# replicates per run, each cell the mean of 10 runs; quantiles 0.9 ... 0.999.
TABLE1_GAMMAS = (1.25, 1.5, 1.75, 2.0, 2.5, 3.0, 3.5, 4.0)
TABLE1_NS = (10, 20, 30, 40, 50, 100, 500, 1000, 2000, 3000, 4000, 5000, 10000, 20000, 50000)
TABLE1_QUANTILES = (0.9, 0.95, 0.99, 0.999)
TABLE1_RUNS = 10


def table1_cells(replicates: int = 50_000) -> list[Cell]:
    """One run of Table 1: every (gamma, N) cell; cell id = 100 * (gamma
    index) + (N index).  Runs differ by seed (run r uses seed r + 1)."""
    return [Cell(g, 1, n, replicates, 100 * i + j)
            for i, g in enumerate(TABLE1_GAMMAS) for j, n in enumerate(TABLE1_NS)]


# Tables 2-6 of the paper (truncated law on 1..K): K = 20, 50, 100, 500, 1000,
# 12 exponents x the 15 sample sizes of Table 1, 50,000 replicates per run,
# each cell the mean of 10 runs; the same quantiles.
TZ_KS = (20, 50, 100, 500, 1000)
TZ_GAMMAS = (0.25, 0.5, 0.75, 1.0, 1.25, 1.5, 1.75, 2.0, 2.5, 3.0, 3.5, 4.0)
TZ_NS = TABLE1_NS
TZ_QUANTILES = TABLE1_QUANTILES
TZ_RUNS = 10


@dataclass
class TzCell:
    gamma: float
    K: int
    n: int
    replicates: int
    cell_id: int


def tables2to6_cells(replicates: int = 50_000, Ks=TZ_KS) -> list[TzCell]:
    """One run of Tables 2-6: every (K, gamma, N) cell; cell id = 10000 * (K
    index) + 100 * (gamma index) + (N index).  Runs differ by seed (run r uses
    seed r + 1)."""
    return [TzCell(g, K, n, replicates, 10000 * TZ_KS.index(K) + 100 * i + j)
            for K in Ks for i, g in enumerate(TZ_GAMMAS) for j, n in enumerate(TZ_NS)]


@dataclass
class BespokeRequest:
    request_id: int
    truncated: bool
    exponent: float       # alpha (untruncated) or gamma (truncated) of the data's law
    xmin_or_K: int        # xmin (untruncated) or K (truncated)
    n: int


def bespoke_requests(count: int = 64, seed: int = 7) -> list[BespokeRequest]:
    """Data sets for the bespoke-cutoff workload: half from the untruncated law
    (alpha ~ U(1.6, 3.0), xmin = 1, n log-uniform in [100, 10^4]), half from
    the truncated law (K in {20, 100, 1000}, gamma ~ U(0.25, 3.0), n
    log-uniform in [10, 10^4]); the data themselves are drawn by the method's
    sampler with stream tag 2 (cell id = request id)."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        if i % 2 == 0:
            n = int(round(math.exp(rng.uniform(math.log(100), math.log(10_000)))))
            out.append(BespokeRequest(i, False, float(rng.uniform(1.6, 3.0)), 1, n))
        else:
            n = int(round(math.exp(rng.uniform(math.log(10), math.log(10_000)))))
            out.append(BespokeRequest(i, True, float(rng.uniform(0.25, 3.0)), int(rng.choice([20, 100, 1000])), n))
    return out
