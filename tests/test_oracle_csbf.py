"""Pins of the oracle's cache-sectorized filter (Sec. II-A, CSBF).

* the closed-form FPR against exhaustive enumeration of tiny ideal filters
  (exact fractions) and against Monte Carlo with an unrelated generator;
* with one word per group it reduces to the sectorized filter;
* the hash-based oracle filter: measured FPR inside the 3-sigma band of its
  realized array's FPR, next to the closed form; word selection uniform;
* a set-based brute force of the construction / lookup semantics.
"""
import itertools
import math
from collections import Counter
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synthkeys


def _key_outcomes(b, z, g, S, kp):
    """(block, {word: mask}) for every equally likely draw of one key."""
    out = []
    per_group = list(itertools.product(range(g), itertools.product(range(S), repeat=kp)))
    for j in range(b):
        for choice in itertools.product(per_group, repeat=z):
            masks = {}
            for q, (sel, pos) in enumerate(choice):
                m = 0
                for p in pos:
                    m |= 1 << p
                masks[q * g + sel] = m
            out.append((j, tuple(sorted(masks.items()))))
    return out


def _exact_fpr(b, z, g, S, kp, n):
    outcomes = _key_outcomes(b, z, g, S, kp)
    s = z * g
    filters = Counter()
    for keys in itertools.product(range(len(outcomes)), repeat=n):
        state = [[0] * s for _ in range(b)]
        for o in keys:
            j, masks = outcomes[o]
            for w, m in masks:
                state[j][w] |= m
        filters[tuple(tuple(x) for x in state)] += 1
    hits = 0
    for st, cnt in filters.items():
        for j, masks in outcomes:
            if all(st[j][w] & m == m for w, m in masks):
                hits += cnt
    return Fraction(hits, len(outcomes) ** (n + 1))


@pytest.mark.parametrize("b,z,g,S,kp,n", [(1, 1, 2, 4, 1, 3), (2, 1, 2, 3, 1, 2), (1, 2, 2, 2, 1, 2), (1, 1, 4, 2, 2, 2)])
def test_csbf_closed_form_equals_enumeration(b, z, g, S, kp, n):
    exact = _exact_fpr(b, z, g, S, kp, n)
    got = oracle.fpr_csbf_closed_form(b, n, z * g * S, S, z * kp, z)
    assert got == pytest.approx(float(exact), rel=1e-12, abs=1e-15)


def test_csbf_closed_form_reduces_to_sbf():
    for b, n, B, S, k in [(1 << 10, 30_000, 256, 32, 8), (64, 900, 512, 64, 16)]:
        s = B // S
        assert oracle.fpr_csbf_closed_form(b, n, B, S, k, s) == pytest.approx(
            oracle.fpr_sbf_closed_form(b, n, B, S, k), rel=1e-14)


@pytest.mark.parametrize("b,z,g,S,kp,n", [(64, 2, 4, 32, 2, 400), (32, 1, 8, 64, 4, 100)])
def test_csbf_closed_form_against_monte_carlo(b, z, g, S, kp, n):
    rng = np.random.default_rng(99)
    reps, queries = 200, 4000
    s = z * g
    hits = 0
    for _ in range(reps):
        blk = rng.integers(0, b, size=n)
        sel = rng.integers(0, g, size=(n, z))
        pos = rng.integers(0, S, size=(n, z, kp))
        state = np.zeros((b, s, S), dtype=bool)
        words = np.arange(z)[None, :] * g + sel
        for t in range(kp):
            state[blk[:, None], words, pos[:, :, t]] = True
        qb = rng.integers(0, b, size=queries)
        qw = np.arange(z)[None, :] * g + rng.integers(0, g, size=(queries, z))
        qp = rng.integers(0, S, size=(queries, z, kp))
        ok = np.ones(queries, dtype=bool)
        for t in range(kp):
            ok &= state[qb[:, None], qw, qp[:, :, t]].all(axis=1)
        hits += int(ok.sum())
    N = reps * queries
    p = oracle.fpr_csbf_closed_form(b, n, s * S, S, z * kp, z)
    assert abs(hits / N - p) < 4 * math.sqrt(p * (1 - p) / N) + 0.05 * p


@pytest.mark.parametrize("block_bits,word_bits,k,groups", [(512, 64, 16, 2), (1024, 64, 16, 4), (256, 32, 8, 2),
                                                           (512, 32, 4, 1)])
def test_csbf_measured_fpr_within_3_sigma(block_bits, word_bits, k, groups):
    b = 1 << 12
    n = b * block_bits // 10
    geom = oracle.Geometry(num_blocks=b, block_bits=block_bits, word_bits=word_bits, k=k, groups=groups)
    f = oracle.SBF(geom)
    f.add(synthkeys.insert_keys(n))
    q, _ = synthkeys.mixed_queries(n, 0, 400_000)
    measured = f.contains(q).mean()
    realized = oracle.fpr_given_filter(f.words, geom)
    assert abs(measured - realized) <= oracle.binomial_3sigma(realized, q.size)
    closed = oracle.fpr_csbf_closed_form(b, n, block_bits, word_bits, k, groups)
    assert realized == pytest.approx(closed, rel=0.03)


def test_csbf_word_selection_uniform():
    geom = oracle.Geometry(num_blocks=8, block_bits=1024, word_bits=64, k=16, groups=2)  # g = 8
    f = oracle.SBF(geom)
    h = oracle.hash_keys(synthkeys.insert_keys(40_000))
    for q in range(2):
        w = np.array([f.group_word(int(x), q) for x in h])
        assert w.min() >= q * 8 and w.max() < (q + 1) * 8
        c = np.bincount(w - q * 8, minlength=8)
        e = w.size / 8
        z = (float(((c - e) ** 2 / e).sum()) - 7) / math.sqrt(14)
        assert abs(z) < 5


@pytest.mark.parametrize("B,S,k,z", [(256, 32, 8, 2), (512, 64, 8, 4), (1024, 64, 16, 2), (512, 32, 4, 1)])
def test_csbf_brute_force_sets(B, S, k, z):
    geom = oracle.Geometry(num_blocks=5, block_bits=B, word_bits=S, k=k, seed=3, groups=z)
    f = oracle.SBF(geom)
    keys = synthkeys.splitmix64(77, 0, 64)
    f.add(keys[:40])
    g = geom.s // z

    def positions(key):
        h = oracle.key_hash(int(key), geom.seed)
        j = oracle.block_index(h, geom.num_blocks)
        out = set()
        for q in range(z):
            w = f.group_word(h, q)
            assert q * g <= w < (q + 1) * g
            for t in range(k // z):
                out.add((j, w, oracle.bit_position(h, q + z * t, S)))
        return out

    union = set()
    for key in keys[:40]:
        union |= positions(key)
    expect = np.zeros(geom.num_words, dtype=geom.word_dtype)
    for j, w, bit in union:
        expect[j * geom.s + w] |= geom.word_dtype(1) << geom.word_dtype(bit)
    assert np.array_equal(f.words, expect)
    want = np.array([positions(x) <= union for x in keys], dtype=np.uint8)
    assert np.array_equal(f.contains(keys), want)


def test_csbf_geometry_rules():
    ok = [(512, 64, 16, 2), (1024, 64, 16, 4), (256, 32, 4, 1), (1024, 32, 8, 8)]
    for B, S, k, z in ok:
        assert oracle.Geometry(num_blocks=4, block_bits=B, word_bits=S, k=k, groups=z).valid(), (B, S, k, z)
    bad = [(512, 64, 16, 3), (512, 64, 6, 4), (256, 32, 8, 16), (256, 32, 64, 4)]
    for B, S, k, z in bad:
        assert not oracle.Geometry(num_blocks=4, block_bits=B, word_bits=S, k=k, groups=z).valid(), (B, S, k, z)
    # one word per group is the sectorized filter
    keys = synthkeys.insert_keys(5000)
    a = oracle.SBF(oracle.Geometry(num_blocks=100, block_bits=256, word_bits=32, k=16, groups=8))
    b = oracle.SBF(oracle.Geometry(num_blocks=100, block_bits=256, word_bits=32, k=16))
    a.add(keys)
    b.add(keys)
    assert np.array_equal(a.words, b.words)
