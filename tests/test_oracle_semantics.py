"""Pins of the oracle's construction and lookup (Sec. II-A, Sec. IV-B).

A second, set-based implementation on tiny filters (every key's pattern as an
explicit set of (block, word, bit) positions) must give the same bit array
and the same answers; and the invariants the definition fixes must hold:
no false negatives, union, order independence, idempotence.
"""
import itertools

import numpy as np
import pytest

import oracle
import synthkeys

BLOCKS = (64, 128, 256, 512, 1024)
WORDS = (32, 64)
KS = (1, 2, 4, 8, 16, 32)


def valid_geometries():
    for B, S, k in itertools.product(BLOCKS, WORDS, KS):
        if B < S:
            continue
        s = B // S
        if k >= s and k % s == 0:
            yield B, S, k


def positions_of(key, geom):
    """The key's pattern as a set of (block, word, bit), from the definition."""
    h = oracle.key_hash(key, geom.seed)
    j = oracle.block_index(h, geom.num_blocks)
    out = set()
    for w in range(geom.s):
        for t in range(geom.kp):
            out.add((j, w, oracle.bit_position(h, w + geom.s * t, geom.word_bits)))
    return out


@pytest.mark.parametrize("B,S,k", list(valid_geometries()))
@pytest.mark.parametrize("b", [1, 2, 3, 5])
def test_brute_force_sets(B, S, k, b):
    geom = oracle.Geometry(num_blocks=b, block_bits=B, word_bits=S, k=k, seed=7)
    keys = synthkeys.splitmix64(100 + b, 0, 48)
    f = oracle.SBF(geom)
    f.add(keys[:32])
    union = set()
    for key in keys[:32]:
        union |= positions_of(int(key), geom)
    expect = np.zeros(geom.num_words, dtype=geom.word_dtype)
    for j, w, bit in union:
        expect[j * geom.s + w] |= geom.word_dtype(1) << geom.word_dtype(bit)
    assert np.array_equal(f.words, expect)
    got = f.contains(keys)
    want = np.array([positions_of(int(x), geom) <= union for x in keys], dtype=np.uint8)
    assert np.array_equal(got, want)
    assert got[:32].all()


def test_invalid_geometries_rejected():
    # Sec. II-A: an SBF needs k >= s and s | k
    for B, S, k in [(256, 32, 4), (512, 32, 4), (512, 32, 8), (512, 64, 4), (256, 32, 12), (1024, 32, 16)]:
        assert not oracle.Geometry(num_blocks=4, block_bits=B, word_bits=S, k=k).valid()
    assert not oracle.Geometry(num_blocks=0).valid()
    for B, S, k in [(256, 32, 8), (512, 64, 8), (64, 64, 4), (1024, 64, 16)]:
        assert oracle.Geometry(num_blocks=4, block_bits=B, word_bits=S, k=k).valid()


def test_invariants_cfg1_shape():
    geom = oracle.Geometry(num_blocks=1 << 12, block_bits=256, word_bits=32, k=8, seed=0)
    keys = synthkeys.insert_keys(50_000)
    a, b, ab = oracle.SBF(geom), oracle.SBF(geom), oracle.SBF(geom)
    a.add(keys[:20_000])
    b.add(keys[20_000:])
    ab.add(keys)
    # union: filter(A u B) == filter(A) | filter(B)
    assert np.array_equal(ab.words, a.words | b.words)
    # no false negatives
    assert ab.contains(keys).all()
    # popcount <= k * n
    assert int(np.bitwise_count(ab.words).sum()) <= geom.k * keys.size
    # order independence and idempotence
    perm = oracle.SBF(geom)
    perm.add(keys[np.argsort(synthkeys.splitmix64(9, 0, keys.size))])
    perm.add(keys[:1000])
    assert np.array_equal(perm.words, ab.words)
    # an empty filter answers 0 for every key
    assert not oracle.SBF(geom).contains(keys).any()


def test_block_range_slices_match_full_filter():
    geom = oracle.Geometry(num_blocks=1000, block_bits=512, word_bits=64, k=16, seed=3)
    keys = synthkeys.insert_keys(20_000)
    f = oracle.SBF(geom)
    f.add(keys)
    lo, hi = 123, 456
    sl = oracle.add_block_range(geom, lo, hi, keys)
    assert np.array_equal(sl, f.words[lo * geom.s:hi * geom.s])
    q, _ = synthkeys.mixed_queries(20_000, 1000, 1000)
    r = oracle.contains_block_range(geom, sl, lo, hi, q)
    full = f.contains(q)
    j = oracle.block_indices(q, geom.num_blocks, geom.seed)
    inside = (j >= lo) & (j < hi)
    assert np.array_equal(r[inside], full[inside])
    assert (r[~inside] == 2).all()


def test_salt_tables():
    s64 = oracle.salts(64)
    s32 = oracle.salts(32)
    assert all(x & 1 for x in s64) and all(x & 1 for x in s32)
    assert len(set(s64)) == 64 and len(set(s32)) == 64
    assert all(s32[i] == ((s64[i] >> 32) | 1) for i in range(64))
    # salt i is the i-th SplitMix64 output from state 0x5A175EED, made odd
    assert s64[0] == synthkeys.splitmix64_scalar(0x5A175EED, 0) | 1
    assert s64[63] == synthkeys.splitmix64_scalar(0x5A175EED, 63) | 1


def test_block_index_rule():
    rng = np.random.default_rng(5)
    hs = [int(x) for x in rng.integers(0, 2**63, size=200, dtype=np.int64)] + [0, 2**64 - 1, 2**32, 2**63]
    for b in (1, 3, 1000, 2**20 + 7, 2**32):
        for h in hs:
            j = oracle.block_index(h, b)
            assert 0 <= j < b
            assert j == ((h >> 32) * b) >> 32
    for b in (2**32 + 1, 2**40 + 12345):
        for h in hs:
            assert oracle.block_index(h, b) == (h * b) >> 64


@pytest.mark.parametrize("B,S,k,z", [(256, 32, 8, 0), (512, 64, 16, 0), (64, 32, 4, 0), (1024, 64, 16, 2),
                                     (256, 64, 8, 2)])
def test_sparse_construction_equals_dense(B, S, k, z):
    """add_sparse (per-key block images ORed per block) against the dense
    construction: the same words in every touched block, zero elsewhere,
    with duplicates and shared blocks present."""
    geom = oracle.Geometry(num_blocks=97, block_bits=B, word_bits=S, k=k, seed=11, groups=z)
    keys = synthkeys.splitmix64(31, 0, 400)
    keys = np.concatenate([keys, keys[:50]])
    blocks, words = oracle.add_sparse(geom, keys)
    f = oracle.SBF(geom)
    f.add(keys)
    dense = f.as_bytes().view(geom.word_dtype).reshape(geom.num_blocks, geom.s)
    assert np.array_equal(np.unique(oracle.block_indices(keys, geom.num_blocks, geom.seed)), blocks)
    assert np.array_equal(dense[blocks.astype(np.int64)], words)
    rest = np.ones(geom.num_blocks, dtype=bool)
    rest[blocks.astype(np.int64)] = False
    assert not dense[rest].any()
    b0, w0 = oracle.add_sparse(geom, keys[:0])
    assert b0.size == 0 and w0.shape == (0, geom.s)
