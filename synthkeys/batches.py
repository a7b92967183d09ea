"""Seeded layout of a batch of filters (sizes and key runs); no filter arithmetic.

Filter sizes are log-uniform between two byte sizes (rounded down to whole
blocks), drawn from numpy's PCG64 generator with a fixed seed; keys are given
to the filters in proportion to their sizes (largest remainders get the
leftover keys).  Keys themselves come from the SplitMix64 streams of
``synthkeys``.
"""
from __future__ import annotations

import numpy as np


def log_uniform_bytes(nfilters: int, min_bytes: int, max_bytes: int, seed: int = 5):
    """Filter sizes in whole bytes, log-uniform in [min_bytes, max_bytes)."""
    rng = np.random.default_rng(seed)
    u = rng.random(nfilters)
    sizes = np.exp(np.log(min_bytes) + u * (np.log(max_bytes) - np.log(min_bytes)))
    return np.floor(sizes).astype(np.int64)


def blocks_of(size_bytes: np.ndarray, block_bytes: int):
    """Whole blocks per filter (at least one)."""
    return np.maximum(1, size_bytes // block_bytes)


def log_uniform_sizes(nfilters: int, min_bytes: int, max_bytes: int, block_bytes: int, seed: int = 5):
    return blocks_of(log_uniform_bytes(nfilters, min_bytes, max_bytes, seed), block_bytes)


def proportional_counts(weights: np.ndarray, total: int) -> np.ndarray:
    w = np.asarray(weights, dtype=np.float64)
    exact = w / w.sum() * total
    base = np.floor(exact).astype(np.int64)
    left = int(total - base.sum())
    if left > 0:
        order = np.argsort(-(exact - base), kind="stable")
        base[order[:left]] += 1
    return base


def arena_offsets(blocks: np.ndarray, block_bytes: int, align: int = 256):
    """Byte offset of each filter in one arena (each start aligned to `align`)."""
    nbytes = blocks * block_bytes
    padded = (nbytes + align - 1) // align * align
    off = np.zeros(len(blocks), dtype=np.int64)
    off[1:] = np.cumsum(padded)[:-1]
    return off, int(padded.sum())
