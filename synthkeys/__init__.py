"""Seeded synthetic key streams for the Bloom-filter workloads.

This module feeds both the CPU oracle tests and the CUDA path (tests and
bench).  It holds none of the filter's arithmetic: no hashing of keys, no
block selection, no bit patterns.  It only produces 64-bit keys.

Generator: SplitMix64 (Steele, Lea and Flood, "Fast splittable pseudorandom
number generators", OOPSLA 2014), used counter-based.  A generator seeded with
state ``seed`` returns, as its i-th output (i = 0, 1, ...),

    mix64(seed + (i + 1) * GAMMA  mod 2^64)

with GAMMA = 0x9E3779B97F4A7C15 and

    mix64(z): z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9
              z = (z ^ (z >> 27)) * 0x94D049BB133111EB
              return z ^ (z >> 31)

(all arithmetic mod 2^64, ``>>`` logical).  Because the i-th output needs no
state but ``seed`` and ``i``, any slice of a stream can be generated on its
own, on the host (numpy) or on the device (torch int64 ops, two's-complement
wrap), and the two agree bit for bit.

The paper draws "unique, random 64-bit input keys" (Sec. V-A); these streams
stand in for them.  Stream seeds used by the workloads:

    1  keys inserted into the filter
    2  fresh (non-member) query keys
    3  selection of member queries among the inserted keys
    4  placement of member / fresh queries in the query stream
"""
from __future__ import annotations

import numpy as np

GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
MASK64 = (1 << 64) - 1

SEED_INSERT = 1
SEED_FRESH = 2
SEED_SELECT = 3
SEED_PLACE = 4


# --------------------------------------------------------------------------
# host (numpy, uint64 with wrap-around)
# --------------------------------------------------------------------------
def _mix64_np(z: np.ndarray) -> np.ndarray:
    z = (z ^ (z >> np.uint64(30))) * np.uint64(MIX1)
    z = (z ^ (z >> np.uint64(27))) * np.uint64(MIX2)
    return z ^ (z >> np.uint64(31))


def splitmix64(seed: int, start: int, count: int) -> np.ndarray:
    """Outputs ``start .. start+count-1`` of the SplitMix64 stream ``seed``."""
    idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + idx * np.uint64(GAMMA)
        return _mix64_np(z)


def splitmix64_at(seed: int, idx: np.ndarray) -> np.ndarray:
    """Outputs at the given indices of the SplitMix64 stream ``seed``."""
    idx = np.asarray(idx, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + (idx + np.uint64(1)) * np.uint64(GAMMA)
        return _mix64_np(z)


def splitmix64_scalar(seed: int, i: int) -> int:
    """The i-th output of stream ``seed`` in plain Python integers."""
    z = (seed + (i + 1) * GAMMA) & MASK64
    z = ((z ^ (z >> 30)) * MIX1) & MASK64
    z = ((z ^ (z >> 27)) * MIX2) & MASK64
    return z ^ (z >> 31)


# --------------------------------------------------------------------------
# device (torch int64; the bit pattern is the uint64 value)
# --------------------------------------------------------------------------
def _s64(x: int) -> int:
    x &= MASK64
    return x - (1 << 64) if x >> 63 else x


def _lsr_torch(z, r: int):
    import torch
    return torch.bitwise_and(torch.bitwise_right_shift(z, r), (1 << (64 - r)) - 1)


def _mix64_torch(z):
    z = (z ^ _lsr_torch(z, 30)) * _s64(MIX1)
    z = (z ^ _lsr_torch(z, 27)) * _s64(MIX2)
    return z ^ _lsr_torch(z, 31)


def splitmix64_torch(seed: int, start: int, count: int, device, out=None, chunk: int = 1 << 26):
    """Same stream as :func:`splitmix64`, produced on ``device`` as int64.

    Writes into ``out`` (int64, length ``count``) when given.  Works in chunks
    so that temporaries stay small for multi-billion-key streams.
    """
    import torch
    if out is None:
        out = torch.empty(count, dtype=torch.int64, device=device)
    for lo in range(0, count, chunk):
        c = min(chunk, count - lo)
        idx = torch.arange(start + lo + 1, start + lo + c + 1, dtype=torch.int64, device=device)
        z = idx * _s64(GAMMA) + _s64(seed)
        out[lo:lo + c] = _mix64_torch(z)
    return out


def as_uint64(t) -> np.ndarray:
    """A torch int64 tensor (any device) viewed as a numpy uint64 array."""
    return t.detach().cpu().numpy().view(np.uint64)


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
def insert_keys(n: int, seed: int = SEED_INSERT) -> np.ndarray:
    return splitmix64(seed, 0, n)


def mixed_queries(n_insert: int, n_members: int, n_fresh: int,
                  seed_insert: int = SEED_INSERT, seed_fresh: int = SEED_FRESH,
                  seed_select: int = SEED_SELECT, seed_place: int = SEED_PLACE):
    """Query keys with an exact member count (small workloads, host side).

    Members are ``n_members`` distinct inserted keys chosen by ranking the
    ``seed_select`` stream over the insert indices (selection without
    replacement).  Fresh keys are the first ``n_fresh`` outputs of the
    ``seed_fresh`` stream that are not inserted keys (exact set exclusion).
    The two groups are interleaved by ranking the ``seed_place`` stream.
    Returns ``(queries, is_member)``.
    """
    ins = insert_keys(n_insert, seed_insert)
    order = np.argsort(splitmix64(seed_select, 0, n_insert), kind="stable")
    members = ins[order[:n_members]]
    fresh = np.empty(0, dtype=np.uint64)
    start, want = 0, n_fresh
    ins_sorted = np.sort(ins)
    while fresh.size < n_fresh:
        cand = splitmix64(seed_fresh, start, want + 64)
        start += cand.size
        pos = np.searchsorted(ins_sorted, cand)
        pos[pos == ins_sorted.size] = 0
        keep = cand[ins_sorted[pos] != cand] if ins_sorted.size else cand
        fresh = np.concatenate([fresh, keep])[:n_fresh]
        want = n_fresh - fresh.size
    q = np.concatenate([members, fresh])
    flag = np.concatenate([np.ones(n_members, np.uint8), np.zeros(n_fresh, np.uint8)])
    perm = np.argsort(splitmix64(seed_place, 0, q.size), kind="stable")
    return q[perm], flag[perm]


# Counter-based query stream for large workloads: query i is a member with
# probability 1/ratio_den.  Position i is a member iff
# (stream_place[i] >> 11) % ratio_den == 0; a member query is the inserted
# key at index (stream_select[i] >> 11) % n_insert (with replacement); other
# queries are stream_fresh[i].  Any index can be produced on its own.
def stream_queries_at(idx: np.ndarray, n_insert: int, ratio_den: int = 10,
                      seed_insert: int = SEED_INSERT, seed_fresh: int = SEED_FRESH,
                      seed_select: int = SEED_SELECT, seed_place: int = SEED_PLACE):
    idx = np.asarray(idx, dtype=np.uint64)
    is_mem = (splitmix64_at(seed_place, idx) >> np.uint64(11)) % np.uint64(ratio_den) == 0
    ins_idx = (splitmix64_at(seed_select, idx) >> np.uint64(11)) % np.uint64(n_insert)
    member = splitmix64_at(seed_insert, ins_idx)
    fresh = splitmix64_at(seed_fresh, idx)
    return np.where(is_mem, member, fresh), is_mem.astype(np.uint8)


def stream_queries(start: int, count: int, n_insert: int, ratio_den: int = 10, **kw):
    return stream_queries_at(np.arange(start, start + count, dtype=np.uint64), n_insert, ratio_den, **kw)


def stream_queries_torch(count: int, n_insert: int, device, ratio_den: int = 10, out=None,
                         chunk: int = 1 << 25, seed_insert: int = SEED_INSERT,
                         seed_fresh: int = SEED_FRESH, seed_select: int = SEED_SELECT,
                         seed_place: int = SEED_PLACE, member_flags=None):
    """Device version of :func:`stream_queries` for indices ``0..count-1``.

    ``member_flags`` (uint8/bool tensor of length ``count``), when given, is
    filled with the member indicator.
    """
    import torch
    if out is None:
        out = torch.empty(count, dtype=torch.int64, device=device)
    for lo in range(0, count, chunk):
        c = min(chunk, count - lo)
        idx1 = torch.arange(lo + 1, lo + c + 1, dtype=torch.int64, device=device)
        place = _mix64_torch(idx1 * _s64(GAMMA) + _s64(seed_place))
        is_mem = torch.remainder(_lsr_torch(place, 11), ratio_den) == 0
        sel = _mix64_torch(idx1 * _s64(GAMMA) + _s64(seed_select))
        ins_idx = torch.remainder(_lsr_torch(sel, 11), n_insert)
        member = _mix64_torch((ins_idx + 1) * _s64(GAMMA) + _s64(seed_insert))
        fresh = _mix64_torch(idx1 * _s64(GAMMA) + _s64(seed_fresh))
        out[lo:lo + c] = torch.where(is_mem, member, fresh)
        if member_flags is not None:
            member_flags[lo:lo + c] = is_mem
        del place, sel, ins_idx, member, fresh, is_mem, idx1
    return out
