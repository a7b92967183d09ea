"""Oracle work for the full-size parity test, split into chunks for a spawn
process pool (test infrastructure; imported by the pool's workers).

Each worker regenerates its share of the seeded key or query stream on the
CPU (synthkeys) and runs the oracle's block-range construction or lookup on
it; nothing here comes from the CUDA path.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import oracle  # noqa: E402
import synthkeys  # noqa: E402


def _in_range(blocks, a, b):
    return np.nonzero((blocks >= a) & (blocks < b))[0]


def add_ranges(args):
    """Bits of each block range contributed by insert keys [lo, hi).  The
    oracle's block index selects each range's keys first, so the range
    construction only sees keys that land in it."""
    geom_kw, ranges, lo, hi = args
    geom = oracle.Geometry(**geom_kw)
    keys = synthkeys.splitmix64(synthkeys.SEED_INSERT, lo, hi - lo)
    blocks = oracle.block_indices(keys, geom.num_blocks, geom.seed)
    return [oracle.add_block_range(geom, a, b, keys[_in_range(blocks, a, b)]) for a, b in ranges]


def lookup_ranges(args):
    """(query index, answer) of queries [lo, hi) whose block lies in one of
    the ranges, against those ranges' final bits."""
    geom_kw, ranges, slices, lo, hi, n_insert, ratio_den = args
    geom = oracle.Geometry(**geom_kw)
    q, _ = synthkeys.stream_queries(lo, hi - lo, n_insert, ratio_den)
    blocks = oracle.block_indices(q, geom.num_blocks, geom.seed)
    idx, ans = [], []
    for (a, b), words in zip(ranges, slices):
        sel = _in_range(blocks, a, b)
        r = oracle.contains_block_range(geom, words, a, b, q[sel])
        assert (r != 2).all()
        idx.append(sel + lo)
        ans.append(r)
    return np.concatenate(idx), np.concatenate(ans)
