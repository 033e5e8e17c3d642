"""Seeded synthetic inputs shared by the tests, the benchmark and the CPU baseline.

This module only draws workload parameters (seeds, luxury levels, counts, skip
distances, request traces) with numpy's PCG64; it holds none of the generator's
arithmetic.  The paper's workloads are synthetic (Sec. 4.2: every thread seeds its own
state and draws doubles), so no dataset is stood in for.
"""
from __future__ import annotations

import numpy as np

LUXURY_MIX = (24, 223, 389, 2048)   # the four levels of the mixed batch
PAPER_LUXURY = 2048                  # Sec. 4.2


def consecutive_seeds(n, first=1):
    """Seeds first, first+1, ...: stream i of the 2^20-stream workload is the seed-1
    state skipped by i 2^96 advances, i.e. seed i + 1."""
    return np.arange(first, first + n, dtype=np.uint64)


def random_seeds(n, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    return rng.integers(1, np.iinfo(np.uint64).max, size=n, dtype=np.uint64, endpoint=True)


def log_uniform_counts(n, lo, hi, seed):
    """floor(exp(U[ln lo, ln hi])), clamped to [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    c = np.floor(np.exp(rng.uniform(np.log(lo), np.log(hi), size=n))).astype(np.int64)
    return np.clip(c, lo, hi)


def batch_mix(n_streams=65536, max_count=10**6, seed=3):
    """Mixed batch: luxury uniform over LUXURY_MIX, counts log-uniform in [1, max_count],
    output type u24 / f64 50/50.  Returns (levels, level_index, counts, is_f64)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    level_index = rng.integers(0, len(LUXURY_MIX), size=n_streams).astype(np.uint8)
    counts = log_uniform_counts(n_streams, 1, max_count, seed + 1000)
    is_f64 = rng.integers(0, 2, size=n_streams).astype(bool)
    return list(LUXURY_MIX), level_index, counts, is_f64


def skip_distances(n_streams, seed=4, bits=128):
    """Independent uniform distances in [0, 2^bits) as (n, 2) uint64, low word first."""
    rng = np.random.Generator(np.random.PCG64(seed))
    out = rng.integers(0, np.iinfo(np.uint64).max, size=(n_streams, 2), dtype=np.uint64, endpoint=True)
    if bits < 128:
        if bits <= 64:
            out[:, 1] = 0
            if bits < 64:
                out[:, 0] &= np.uint64((1 << bits) - 1)
        else:
            out[:, 1] &= np.uint64((1 << (bits - 64)) - 1)
    return out


def ragged_counts(n_streams, max_count, seed, zero_frac=0.1):
    """Uniform counts in [0, max_count] with a share of zeros, and exclusive-prefix
    offsets into one packed output in a shuffled stream order."""
    rng = np.random.Generator(np.random.PCG64(seed))
    counts = rng.integers(0, max_count + 1, size=n_streams).astype(np.int64)
    counts[rng.random(n_streams) < zero_frac] = 0
    order = rng.permutation(n_streams)
    offsets = np.zeros(n_streams, dtype=np.int64)
    offsets[order] = np.concatenate([[0], np.cumsum(counts[order])[:-1]])
    return counts, offsets


def serving_trace(n_requests, rate_hz, n_resident, lo=10**2, hi=10**7, seed=5):
    """Poisson arrivals at rate_hz: (arrival_s, stream, count, is_f64) arrays."""
    rng = np.random.Generator(np.random.PCG64(seed))
    gaps = rng.exponential(1.0 / rate_hz, size=n_requests)
    arrival = np.cumsum(gaps)
    stream = rng.integers(0, n_resident, size=n_requests).astype(np.int64)
    counts = log_uniform_counts(n_requests, lo, hi, seed + 1000)
    is_f64 = rng.integers(0, 2, size=n_requests).astype(bool)
    return arrival, stream, counts, is_f64


def rank_seeds(rank, world, n_per_rank):
    """Seeds of one rank when the stream workload is sharded over `world` GPUs (weak
    scaling): rank r owns seeds 1 + r n .. (r + 1) n, so the ranks together run the
    single-GPU workload's streams for world x n streams, without overlap."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    return consecutive_seeds(n_per_rank, first=1 + rank * n_per_rank)
