"""Seeded synthetic inputs for Aggregate Risk Analysis (ARA) workloads.

Both the FP64 oracle and the CUDA engine are fed from here, so this module
holds no part of the method's arithmetic: it only draws random numbers and
lays them out as the arrays the method consumes.

* Year Event Table (Section III): trials T_i = {(E_ik, t_ik)} in ascending
  time-stamp order, stored as CSR -- ``offsets int64[N+1]``, ``ids int32[M]``
  and optional ``ts float32[M]``.
* Event Loss Tables (Section III): a pool of ELTs, each a set of distinct
  (event id, loss) pairs plus its financial terms FT1, read here as a
  deductible and a limit.
* Layers (Section III): an ordered list of ELTs from the pool plus the
  occurrence terms FT2 = (OccR, OccL) and aggregate terms FT3 = (AggR, AggL).

The paper's industry data (Section IV-C: one million trials of about one
thousand events, one layer over sixteen ELTs) is proprietary; the presets below
stand in for it with the distributions listed beside each one.

Randomness: each named stream gets its own 64-bit seed, derived from the
workload seed with SplitMix64 (Steele, Lea & Flood, OOPSLA 2014), and drives a
NumPy PCG64 generator.  Large streams are drawn in fixed-size chunks, each with
its own derived seed, so the arrays do not depend on the thread count.
"""
from __future__ import annotations

import concurrent.futures as _fut
import os
from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import numpy as np

DEFAULT_SEED = 0x14124556
_CHUNK = 1 << 24  # events per independently seeded chunk of the YET
_MASK64 = (1 << 64) - 1


def splitmix64(x: int) -> int:
    """One SplitMix64 output for state ``x`` (the published constants)."""
    z = (x + 0x9E3779B97F4A7C15) & _MASK64
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & _MASK64
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & _MASK64
    return z ^ (z >> 31)


def sub_seed(seed: int, *tags) -> int:
    """Derive a 64-bit stream seed from ``seed`` and a tuple of tags."""
    s = splitmix64(seed & _MASK64)
    for t in tags:
        if isinstance(t, str):
            for ch in t.encode():
                s = splitmix64(s ^ ch)
        else:
            s = splitmix64(s ^ (int(t) & _MASK64))
    return s


def rng_for(seed: int, *tags) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(sub_seed(seed, *tags)))


# --------------------------------------------------------------------------
# Containers
# --------------------------------------------------------------------------
@dataclass
class YET:
    """CSR Year Event Table: trial t owns ids[offsets[t]:offsets[t+1]]."""
    catalog_size: int
    offsets: np.ndarray          # int64[N+1], offsets[0] == 0, nondecreasing
    ids: np.ndarray              # int32[M], each in [0, catalog_size)
    ts: Optional[np.ndarray] = None   # float32[M], ascending within a trial

    @property
    def n_trials(self) -> int:
        return int(self.offsets.shape[0] - 1)

    @property
    def n_occurrences(self) -> int:
        return int(self.offsets[-1])


@dataclass
class ELTPool:
    """Pool of ELTs in CSR form: ELT j owns ids/losses[offsets[j]:offsets[j+1]]."""
    offsets: np.ndarray          # int64[n+1]
    ids: np.ndarray              # int32, distinct within one ELT
    losses: np.ndarray           # float64 >= 0
    deductibles: np.ndarray      # float64[n]
    limits: np.ndarray           # float64[n] (may hold +inf)

    @property
    def n_elts(self) -> int:
        return int(self.offsets.shape[0] - 1)

    def elt(self, j: int):
        a, b = int(self.offsets[j]), int(self.offsets[j + 1])
        return self.ids[a:b], self.losses[a:b]


@dataclass
class Layer:
    """A layer: ELTs (pool indices, in summation order) and FT2/FT3 terms."""
    elts: List[int]
    occ_ret: float
    occ_lim: float
    agg_ret: float
    agg_lim: float


@dataclass
class Workload:
    name: str
    yet: YET
    pool: ELTPool
    layers: List[Layer]
    return_periods: List[float] = field(default_factory=list)
    seed: int = DEFAULT_SEED


@dataclass
class Request:
    """One ad hoc pricing request: a layer priced over a prefix of the YET."""
    arrival_s: float
    layer: Layer
    n_trials: int


# --------------------------------------------------------------------------
# Year Event Table
# --------------------------------------------------------------------------
def _fill_ids(seed: int, catalog: int, out: np.ndarray, threads: int) -> None:
    n = out.shape[0]
    n_chunks = (n + _CHUNK - 1) // _CHUNK

    def work(c: int) -> None:
        a = c * _CHUNK
        b = min(n, a + _CHUNK)
        g = rng_for(seed, "yet-ids", c)
        out[a:b] = g.integers(0, catalog, size=b - a, dtype=np.int32)

    if n_chunks <= 1 or threads <= 1:
        for c in range(n_chunks):
            work(c)
    else:
        with _fut.ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(work, range(n_chunks)))


_TS_TRIALS = 1 << 14  # trials per independently seeded chunk of time-stamps


def _sorted_timestamps(seed: int, offsets: np.ndarray, days: float, threads: int = 1) -> np.ndarray:
    """Uniform [0, days) time-stamps, sorted ascending within each trial.

    The n order statistics of n uniforms on [0, 1) are distributed as the
    partial sums of n + 1 standard exponential gaps divided by their total
    (Devroye, Non-Uniform Random Variate Generation, 1986, V.2), so each
    trial's sorted time-stamps come from one cumulative sum, with no sort.
    Chunks of 2^14 trials draw from their own seeded streams."""
    n = offsets.shape[0] - 1
    m = int(offsets[-1])
    ts = np.empty(m, dtype=np.float32)
    n_chunks = (n + _TS_TRIALS - 1) // _TS_TRIALS

    def work(c: int) -> None:
        t0, t1 = c * _TS_TRIALS, min(n, (c + 1) * _TS_TRIALS)
        a, b = int(offsets[t0]), int(offsets[t1])
        counts = np.diff(offsets[t0:t1 + 1])
        g = rng_for(seed, "yet-ts", c)
        gaps = g.standard_exponential(b - a + (t1 - t0))
        cs = np.cumsum(gaps)
        # trial t's gaps sit at [start[t], start[t] + counts[t]], one extra gap
        # closing the trial; its time-stamps are the first counts[t] partial
        # sums, less the sum before the trial, over the trial's total
        start = (offsets[t0:t1] - a) + np.arange(t1 - t0)
        before = np.where(start > 0, cs[np.maximum(start - 1, 0)], 0.0)
        total = cs[start + counts] - before
        trial = np.repeat(np.arange(t1 - t0), counts)
        pos = np.arange(b - a) + trial  # index of each event's gap
        u = (cs[pos] - before[trial]) / total[trial]
        # float32 rounding is monotone, so each trial stays sorted
        ts[a:b] = np.minimum(u * days, np.nextafter(np.float32(days), np.float32(0))).astype(np.float32)

    if n_chunks <= 1 or threads <= 1:
        for c in range(n_chunks):
            work(c)
    else:
        with _fut.ThreadPoolExecutor(max_workers=threads) as ex:
            list(ex.map(work, range(n_chunks)))
    return ts


def make_yet(seed: int, catalog_size: int, n_trials: int, lam: float,
             with_timestamps: bool = True, days: float = 365.0,
             counts: Optional[np.ndarray] = None, threads: Optional[int] = None) -> YET:
    """A YET of ``n_trials`` trials with Poisson(lam) events each (or given counts).

    Event ids are uniform with replacement over the catalog.
    """
    if counts is None:
        counts = rng_for(seed, "yet-counts").poisson(lam, size=n_trials).astype(np.int64)
    counts = np.asarray(counts, dtype=np.int64)
    offsets = np.zeros(n_trials + 1, dtype=np.int64)
    np.cumsum(counts, out=offsets[1:])
    m = int(offsets[-1])
    ids = np.empty(m, dtype=np.int32)
    threads = threads or min(32, os.cpu_count() or 1)
    _fill_ids(seed, catalog_size, ids, threads)
    ts = _sorted_timestamps(seed, offsets, days, threads) if with_timestamps else None
    return YET(catalog_size, offsets, ids, ts)


# --------------------------------------------------------------------------
# ELT pool and layers
# --------------------------------------------------------------------------
def make_elt_pool(seed: int, catalog_size: int, sizes: Sequence[int],
                  deductibles: np.ndarray, limits: np.ndarray,
                  mu: float = 12.0, sigma: float = 1.5) -> ELTPool:
    """ELTs with distinct ids (uniform without replacement) and lognormal losses."""
    sizes = [int(s) for s in sizes]
    offsets = np.zeros(len(sizes) + 1, dtype=np.int64)
    np.cumsum(sizes, out=offsets[1:])
    ids = np.empty(int(offsets[-1]), dtype=np.int32)
    losses = np.empty(int(offsets[-1]), dtype=np.float64)
    for j, s in enumerate(sizes):
        g = rng_for(seed, "elt", j)
        a, b = int(offsets[j]), int(offsets[j + 1])
        ids[a:b] = g.choice(catalog_size, size=s, replace=False).astype(np.int32)
        losses[a:b] = g.lognormal(mu, sigma, size=s)
    return ELTPool(offsets, ids, losses,
                   np.asarray(deductibles, dtype=np.float64).copy(),
                   np.asarray(limits, dtype=np.float64).copy())


def _log_uniform(g: np.random.Generator, lo: float, hi: float) -> float:
    return float(np.exp(g.uniform(np.log(lo), np.log(hi))))


def random_layer(g: np.random.Generator, n_pool: int, k_lo: int, k_hi: int) -> Layer:
    """k ~ U{k_lo..k_hi} distinct pool ELTs; terms log-uniform over the batched-layer ranges."""
    k = min(int(g.integers(k_lo, k_hi + 1)), n_pool)
    elts = [int(x) for x in g.choice(n_pool, size=k, replace=False)]
    return Layer(elts,
                 occ_ret=_log_uniform(g, 1e4, 1e6), occ_lim=_log_uniform(g, 1e6, 1e8),
                 agg_ret=_log_uniform(g, 1e5, 1e7), agg_lim=_log_uniform(g, 1e7, 1e9))


# --------------------------------------------------------------------------
# Presets
# --------------------------------------------------------------------------
def tiny(seed: int = DEFAULT_SEED, n_trials: int = 1_000) -> Workload:
    """Tiny plain ARA: catalog 10,000; one layer over 4 ELTs x 1,000 events;
    deductible 1e4, limit 5e6; Poisson(100) events per trial; sorted uniform
    time-stamps in [0, 365); OccR=1e5, OccL=2e7, AggR=5e5, AggL=1e8; RP 100/250."""
    c = 10_000
    yet = make_yet(seed, c, n_trials, 100.0, with_timestamps=True)
    pool = make_elt_pool(seed, c, [1_000] * 4, np.full(4, 1e4), np.full(4, 5e6))
    layer = Layer([0, 1, 2, 3], 1e5, 2e7, 5e5, 1e8)
    return Workload("tiny", yet, pool, [layer], [100.0, 250.0], seed)


def paper_scale(seed: int = DEFAULT_SEED, n_trials: int = 1_000_000, lam: float = 1000.0,
                with_timestamps: bool = False, catalog_size: int = 2_000_000,
                threads: Optional[int] = None) -> Workload:
    """Paper-scale plain ARA (Section IV-C workload shape): catalog 2,000,000;
    one layer over 16 ELTs x 20,000 events; deductibles U[5e3, 5e4], limits
    U[1e6, 1e7]; Poisson(1000) events per trial over 1,000,000 trials; layer
    terms as in ``tiny``; RP 100/250/500.  The YET's time-stamps are drawn when
    with_timestamps is set (the YLT does not read them)."""
    yet = make_yet(seed, catalog_size, n_trials, lam, with_timestamps=with_timestamps, threads=threads)
    g = rng_for(seed, "elt-terms")
    ded = g.uniform(5e3, 5e4, size=16)
    lim = g.uniform(1e6, 1e7, size=16)
    pool = make_elt_pool(seed, catalog_size, [20_000] * 16, ded, lim)
    layer = Layer(list(range(16)), 1e5, 2e7, 5e5, 1e8)
    return Workload("paper", yet, pool, [layer], [100.0, 250.0, 500.0], seed)


def batched(seed: int = DEFAULT_SEED, n_layers: int = 64, n_trials: int = 1_000_000,
            lam: float = 1000.0, catalog_size: int = 2_000_000, n_pool: int = 256,
            with_timestamps: bool = False, yet: Optional[YET] = None) -> Workload:
    """Batched layers: the paper-scale YET shared by ``n_layers`` layers; each
    covers k ~ U{1..32} ELTs from a pool of 256 ELTs of U{10k..50k} events;
    per-layer OccR, OccL, AggR, AggL log-uniform over [1e4,1e6], [1e6,1e8],
    [1e5,1e7], [1e7,1e9].  ``yet``: an already drawn YET to share (the
    paper-scale YET of the same seed is this YET)."""
    if yet is None:
        yet = make_yet(seed, catalog_size, n_trials, lam, with_timestamps=with_timestamps)
    elif yet.catalog_size != catalog_size:
        raise ValueError("the shared YET has another catalog size")
    g = rng_for(seed, "pool-sizes")
    sizes = g.integers(10_000, 50_001, size=n_pool)
    gt = rng_for(seed, "pool-terms")
    ded = gt.uniform(5e3, 5e4, size=n_pool)
    lim = gt.uniform(1e6, 1e7, size=n_pool)
    pool = make_elt_pool(seed, catalog_size, sizes, ded, lim)
    gl = rng_for(seed, "layers")
    layers = [random_layer(gl, n_pool, 1, 32) for _ in range(n_layers)]
    return Workload("batched", yet, pool, layers, [100.0, 250.0, 500.0], seed)


def service_requests(seed: int = DEFAULT_SEED, n_requests: int = 2_000, rate_per_s: float = 50.0,
                     n_pool: int = 256, trial_choices: Sequence[int] = (100_000, 250_000, 1_000_000)
                     ) -> List[Request]:
    """Ad hoc pricing stream: Poisson arrivals at ``rate_per_s``; each request is
    a layer of 2-32 pool ELTs with batched-layer terms over a YET prefix of
    100k, 250k or 1M trials."""
    g = rng_for(seed, "requests")
    gaps = g.exponential(1.0 / rate_per_s, size=n_requests)
    arrivals = np.cumsum(gaps)
    out = []
    for i in range(n_requests):
        layer = random_layer(g, n_pool, 2, 32)
        nt = int(trial_choices[int(g.integers(0, len(trial_choices)))])
        out.append(Request(float(arrivals[i]), layer, nt))
    return out
