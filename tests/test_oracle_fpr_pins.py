"""Pins of the oracle's false-positive-rate formulas and of its hash quality.

* exhaustive enumeration of tiny ideal-hashing filters (exact fractions);
* the large-word limit, which must reduce to the paper's Eq. (1);
* Monte Carlo with a random generator that is not the oracle's hash;
* the oracle's own hash-based filter, whose measured FPR must fall in the
  binomial 3-sigma band around the exact FPR of its realized bit array, and
  whose realized FPR must sit next to the closed form.
"""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synthkeys


# ---------------------------------------------------------------------------
# exhaustive enumeration (ideal hashing, exact)
# ---------------------------------------------------------------------------
def _key_outcomes(b, s, S, kp):
    """All (block, per-word bit masks) a key can produce, each equally likely."""
    out = []
    for j in range(b):
        for pos in itertools.product(range(S), repeat=s * kp):
            masks = [0] * s
            for idx, p in enumerate(pos):
                masks[idx // kp] |= 1 << p  # word of the idx-th throw; kp throws per word
            out.append((j, tuple(masks)))
    return out


def _exact_fpr(b, s, S, kp, n):
    outcomes = _key_outcomes(b, s, S, kp)
    from collections import Counter
    filters = Counter()
    for keys in itertools.product(range(len(outcomes)), repeat=n):
        state = [[0] * s for _ in range(b)]
        for o in keys:
            j, m = outcomes[o]
            for w in range(s):
                state[j][w] |= m[w]
        filters[tuple(tuple(x) for x in state)] += 1
    hits = 0
    for st, cnt in filters.items():
        for j, m in outcomes:
            if all(st[j][w] & m[w] == m[w] for w in range(s)):
                hits += cnt
    return Fraction(hits, len(outcomes) ** (n + 1))


@pytest.mark.parametrize("b,s,S,kp,n", [
    (2, 1, 4, 2, 2),
    (1, 2, 4, 1, 3),
    (3, 1, 3, 2, 2),
    (2, 2, 2, 2, 2),
    (1, 1, 4, 3, 2),
])
def test_closed_form_equals_exhaustive_enumeration(b, s, S, kp, n):
    exact = _exact_fpr(b, s, S, kp, n)
    got = oracle.fpr_sbf_closed_form(b, n, s * S, S, s * kp)
    assert got == pytest.approx(float(exact), rel=1e-12, abs=1e-15)


def test_distinct_pmf_sums_to_one_and_matches_enumeration():
    for throws, bins in [(1, 32), (2, 32), (3, 5), (4, 4), (16, 64)]:
        pmf = oracle.distinct_pmf(throws, bins)
        assert math.fsum(pmf) == pytest.approx(1.0, abs=1e-12)
    # enumeration for 3 throws into 5 bins
    from collections import Counter
    c = Counter(len(set(t)) for t in itertools.product(range(5), repeat=3))
    pmf = oracle.distinct_pmf(3, 5)
    for q in range(4):
        assert pmf[q] == pytest.approx(c.get(q, 0) / 125, abs=1e-15)


def test_fpr_given_filter_equals_enumeration():
    rng = np.random.default_rng(11)
    geom = oracle.Geometry(num_blocks=3, block_bits=8, word_bits=4, k=4)  # s=2, k'=2, S=4
    words = rng.integers(0, 16, size=6).astype(np.uint32)
    exact = Fraction(0)
    for j in range(3):
        for pos in itertools.product(range(4), repeat=4):
            m = [0, 0]
            for idx, p in enumerate(pos):
                m[idx // 2] |= 1 << p
            if all(int(words[j * 2 + w]) & m[w] == m[w] for w in range(2)):
                exact += Fraction(1, 3 * 4 ** 4)
    assert oracle.fpr_given_filter(words, geom) == pytest.approx(float(exact), rel=1e-12)


# ---------------------------------------------------------------------------
# the paper's Eq. (1)
# ---------------------------------------------------------------------------
def test_eq1_optimum_form():
    # Eq. (1), second form: at k* = c ln 2 the rate is (1/2)^(c ln 2)
    for c in (4.0, 8.0, 10.0, 16.0):
        kstar = oracle.eq1_kopt(c)
        assert oracle.eq1_cbf(c, kstar) == pytest.approx(0.5 ** (c * math.log(2)), rel=1e-12)
        # and k* minimises f(c, k) over real k
        assert oracle.eq1_cbf(c, kstar) <= oracle.eq1_cbf(c, kstar * 1.05)
        assert oracle.eq1_cbf(c, kstar) <= oracle.eq1_cbf(c, kstar * 0.95)


@pytest.mark.parametrize("c,k", [(10, 7), (8, 6), (16, 11), (10, 3)])
def test_closed_form_reduces_to_eq1_for_one_large_word(c, k):
    # one block, one word of S bits, n = S / c keys: a classical filter of
    # m = S bits, which Eq. (1) approximates to O(1/m)
    S = 1 << 22
    n = S // c
    got = oracle.fpr_sbf_closed_form(1, n, S, S, k)
    assert got == pytest.approx(oracle.eq1_cbf(c, k), rel=2e-3)


# ---------------------------------------------------------------------------
# Monte Carlo with an unrelated generator
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("b,s,S,kp,n", [(64, 4, 32, 2, 300), (16, 2, 64, 4, 60), (256, 8, 32, 1, 8000)])
def test_closed_form_against_monte_carlo(b, s, S, kp, n):
    rng = np.random.default_rng(1234)
    reps, queries = 200, 4000
    hits = 0
    for _ in range(reps):
        blocks = rng.integers(0, b, size=n)
        pos = rng.integers(0, S, size=(n, s, kp))
        state = np.zeros((b, s, S), dtype=bool)
        for t in range(kp):
            state[blocks[:, None], np.arange(s)[None, :], pos[:, :, t]] = True
        qb = rng.integers(0, b, size=queries)
        qp = rng.integers(0, S, size=(queries, s, kp))
        ok = np.ones(queries, dtype=bool)
        for t in range(kp):
            ok &= state[qb[:, None], np.arange(s)[None, :], qp[:, :, t]].all(axis=1)
        hits += int(ok.sum())
    N = reps * queries
    est = hits / N
    p = oracle.fpr_sbf_closed_form(b, n, s * S, S, s * kp)
    # queries within one filter are correlated; widen the band by the number
    # of filters' spread: use 4 sigma of the per-filter mean as a bound
    assert abs(est - p) < 4 * math.sqrt(p * (1 - p) / N) + 0.05 * p


# ---------------------------------------------------------------------------
# the oracle's hash-based filter behaves like ideal hashing
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("block_bits,word_bits,k", [(256, 32, 8), (256, 64, 8), (512, 64, 16), (128, 32, 16)])
def test_measured_fpr_within_3_sigma_of_realized_filter(block_bits, word_bits, k):
    b = 1 << 13
    n = b * block_bits // 10  # 10 bits per key
    geom = oracle.Geometry(num_blocks=b, block_bits=block_bits, word_bits=word_bits, k=k)
    f = oracle.SBF(geom)
    f.add(synthkeys.insert_keys(n))
    q, is_mem = synthkeys.mixed_queries(n, 0, 400_000)
    assert is_mem.sum() == 0
    measured = f.contains(q).mean()
    realized = oracle.fpr_given_filter(f.words, geom)
    assert abs(measured - realized) <= oracle.binomial_3sigma(realized, q.size)
    closed = oracle.fpr_sbf_closed_form(b, n, block_bits, word_bits, k)
    # the realized filter's FPR fluctuates around the closed form by a few
    # percent at this size
    assert realized == pytest.approx(closed, rel=0.03)


def test_blocked_filter_less_accurate_than_classical():
    # Sec. II-A: uneven block occupancy makes a blocked filter less accurate
    # than a classical filter of the same size and k (Eq. (1))
    for b, n, B, S, k in [(1 << 15, 10**6, 256, 32, 8), (1 << 12, 1 << 16, 512, 64, 16)]:
        c = b * B / n
        assert oracle.fpr_sbf_closed_form(b, n, B, S, k) > oracle.eq1_cbf(c, k)


def test_block_occupancy_is_binomial():
    b = 1 << 12
    keys = synthkeys.insert_keys(1 << 20)
    j = oracle.block_indices(keys, b).astype(np.int64)
    assert j.min() >= 0 and j.max() < b
    counts = np.bincount(j, minlength=b)
    e = keys.size / b
    chi2 = float(((counts - e) ** 2 / e).sum())
    z = (chi2 - (b - 1)) / math.sqrt(2 * (b - 1))
    assert abs(z) < 5


@pytest.mark.parametrize("word_bits", [32, 64])
def test_bit_positions_uniform_and_pairwise_independent(word_bits):
    keys = synthkeys.insert_keys(1 << 17)
    h = oracle.hash_keys(keys)
    S = word_bits
    lib = oracle.lib()
    sample = h[:60000]
    p0 = np.array([lib.orc_bit_position(int(x), 0, S) for x in sample])
    p1 = np.array([lib.orc_bit_position(int(x), 1, S) for x in sample])
    for p in (p0, p1):
        c = np.bincount(p, minlength=S)
        e = p.size / S
        z = (float(((c - e) ** 2 / e).sum()) - (S - 1)) / math.sqrt(2 * (S - 1))
        assert abs(z) < 5
    joint = np.bincount(p0 * S + p1, minlength=S * S)
    e = p0.size / (S * S)
    z = (float(((joint - e) ** 2 / e).sum()) - (S * S - 1)) / math.sqrt(2 * (S * S - 1))
    assert abs(z) < 5
