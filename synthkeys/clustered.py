"""Seeded clustered-interval key sets for the learned prefilter; no filter arithmetic.

Members: `n_intervals` intervals of the uint64 line, their centres grouped in
`n_clusters` clusters (cluster centres uniform; interval centres normally
spread around them), widths log-normal; member keys are drawn uniformly
inside intervals chosen in proportion to their widths.  Non-members: half
uniform over uint64, half "near" keys lying outside every interval but within
twice an interval's width of it.  Everything comes from numpy's PCG64 with a
fixed seed; duplicates among members are removed.
"""
from __future__ import annotations

import numpy as np

U64 = np.uint64


def intervals(n_intervals: int = 10_000, n_clusters: int = 32, seed: int = 17,
              median_width: float = 2.0 ** 36, sigma_width: float = 1.0, spread: float = 2.0 ** 52):
    """(starts, widths) as uint64 arrays, sorted by start, non-overlapping."""
    rng = np.random.default_rng(seed)
    centres = rng.integers(0, 2**63, size=n_clusters, dtype=np.int64).astype(np.float64) * 2.0
    which = rng.integers(0, n_clusters, size=n_intervals)
    c = centres[which] + rng.normal(0.0, spread, size=n_intervals)
    c = np.clip(c, 2.0 ** 40, 2.0 ** 64 - 2.0 ** 40)
    w = np.exp(np.log(median_width) + sigma_width * rng.standard_normal(n_intervals))
    w = np.clip(w, 64.0, 2.0 ** 44)
    starts = (c - w / 2).astype(np.float64)
    order = np.argsort(starts)
    starts, w = starts[order], w[order]
    s = np.array([int(x) for x in starts], dtype=object)
    wi = np.array([int(x) for x in w], dtype=object)
    # remove overlaps: an interval starts no earlier than the previous one ends
    out_s, out_w = [], []
    end = -1
    for a, b in zip(s, wi):
        a = max(a, end + 1)
        if a + b >= 2**64:
            break
        out_s.append(a)
        out_w.append(b)
        end = a + b - 1
    return np.array(out_s, dtype=U64), np.array(out_w, dtype=U64)


def members(n: int, starts: np.ndarray, widths: np.ndarray, seed: int = 18) -> np.ndarray:
    rng = np.random.default_rng(seed)
    p = widths.astype(np.float64)
    p /= p.sum()
    idx = rng.choice(starts.size, size=n, p=p)
    off = (rng.random(n) * widths[idx].astype(np.float64)).astype(U64)
    off = np.minimum(off, widths[idx] - U64(1))
    keys = starts[idx] + off
    return np.unique(keys)


def non_members(n: int, starts: np.ndarray, widths: np.ndarray, seed: int = 19):
    """(keys, near_flag): n//2 uniform keys and n - n//2 near keys, all outside every interval."""
    rng = np.random.default_rng(seed)
    n_u = n // 2
    uni = rng.integers(0, 2**63, size=2 * n_u + 64, dtype=np.int64).view(U64) * U64(2) + \
        rng.integers(0, 2, size=2 * n_u + 64, dtype=np.int64).view(U64)
    uni = uni[~inside(uni, starts, widths)][:n_u]
    n_n = n - n_u
    near = []
    while sum(x.size for x in near) < n_n:
        m = 2 * (n_n + 64)
        idx = rng.integers(0, starts.size, size=m)
        w = widths[idx].astype(np.float64)
        side = rng.integers(0, 2, size=m)
        d = (rng.random(m) * 2.0 * w).astype(U64) + U64(1)
        with np.errstate(over="ignore"):
            k = np.where(side == 0, starts[idx] - d, starts[idx] + widths[idx] - U64(1) + d)
        ok = ~inside(k, starts, widths)
        near.append(k[ok])
    near = np.concatenate(near)[:n_n]
    keys = np.concatenate([uni, near])
    flag = np.concatenate([np.zeros(uni.size, np.uint8), np.ones(near.size, np.uint8)])
    return keys, flag


def inside(keys: np.ndarray, starts: np.ndarray, widths: np.ndarray) -> np.ndarray:
    """True where a key lies in one of the (sorted, disjoint) intervals."""
    i = np.searchsorted(starts, keys, side="right") - 1
    ok = i >= 0
    j = np.where(ok, i, 0)
    return ok & (keys - starts[j] < widths[j])
