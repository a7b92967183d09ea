"""Pins of the oracle's hashing against a library outside this repository.

The Apache Parquet split-block Bloom filter, as written by pyarrow, hashes a
64-bit value with XXH64 (seed 0) over its 8 little-endian bytes, selects the
block with ((h >> 32) * num_blocks) >> 32 and sets, in each 32-bit word w of
the 256-bit block, the bit ((h_lo * m_w) mod 2^32) >> 27 for an odd
multiplier m_w.  The paper names this configuration (Sec. I and Sec. VI:
bitwise compatible with Arrow/Parquet split-block filters).  Its multipliers
are not in the paper and are not written here: the tests recover them from
pyarrow's output, so what is checked is that the oracle's XXH64 (both halves),
its block rule and its bit-position rule agree with an independent writer.

These tests need pyarrow and run on the CPU only.
"""
import io

import numpy as np
import pytest

import oracle

pa = pytest.importorskip("pyarrow")
pq = pytest.importorskip("pyarrow.parquet")

MASK32 = 0xFFFFFFFF


def parquet_bitset(values) -> np.ndarray:
    """The bloom-filter bitset pyarrow writes for an int64 column, as uint32 words."""
    t = pa.table({"k": pa.array(np.asarray(values, dtype=np.int64))})
    buf = io.BytesIO()
    pq.write_table(t, buf, bloom_filter_options={"k": {"ndv": max(len(values), 1), "fpp": 0.01}},
                   compression="none", use_dictionary=False)
    raw = buf.getvalue()
    col = pq.ParquetFile(io.BytesIO(raw)).metadata.row_group(0).column(0)
    off, ln = col.bloom_filter_offset, col.bloom_filter_length
    hdr = raw[off:off + ln]
    # Thrift compact header: field 1 (i32 numBytes) is 0x15 + zigzag varint
    assert hdr[0] == 0x15
    v, shift, i = 0, 0, 1
    while True:
        b = hdr[i]
        v |= (b & 0x7F) << shift
        shift += 7
        i += 1
        if not b & 0x80:
            break
    nbytes = (v >> 1) ^ -(v & 1)
    return np.frombuffer(hdr[ln - nbytes:], dtype="<u4").copy()


def consistent_multipliers(hlo, bits, chunk=1 << 23):
    """All odd 32-bit m with ((h * m) mod 2^32) >> 27 == bit for every pair.

    The first pair with odd h fixes m to inv(h) * y for y in one interval of
    2^27 values; the other pairs filter those candidates.
    """
    i0 = next(i for i, x in enumerate(hlo) if x & 1)
    inv = np.uint32(pow(hlo[i0], -1, 1 << 32))
    base = np.uint32(((bits[i0] << 27) * int(inv)) & MASK32)
    t = np.arange(chunk, dtype=np.uint32)
    found = []
    with np.errstate(over="ignore"):
        for lo in range(0, 1 << 27, chunk):
            cand = base + inv * (t + np.uint32(lo))
            for hv, b in zip(hlo, bits):
                cand = cand[(cand * np.uint32(hv)) >> np.uint32(27) == b]
                if cand.size == 0:
                    break
            found.extend(int(c) for c in cand if c & 1)
    return found


KEYS = [int(x) for x in (np.arange(30, dtype=np.int64) * 1000003 + 17)]


@pytest.fixture(scope="module")
def single_key_bits():
    obs = []
    for k in KEYS:
        w = parquet_bitset([k])
        assert w.size == 8
        assert all(bin(int(x)).count("1") == 1 for x in w)
        obs.append([int(x).bit_length() - 1 for x in w])
    return obs


@pytest.fixture(scope="module")
def recovered_multipliers(single_key_bits):
    hlo = [oracle.key_hash(k & (2**64 - 1), 0) & MASK32 for k in KEYS]
    return [consistent_multipliers(hlo, [ob[w] for ob in single_key_bits]) for w in range(8)]


def test_xxh64_low_half_consistent_with_parquet(recovered_multipliers):
    # 30 keys x 5 bits per word over-determine a 31-bit odd multiplier: with
    # the oracle's h_lo exactly one multiplier per word fits all keys.
    assert [len(m) for m in recovered_multipliers] == [1] * 8


def test_wrong_hash_has_no_consistent_multiplier(single_key_bits):
    # negative control: a different hash (seed 1) explains none of the words
    hlo = [oracle.key_hash(k & (2**64 - 1), 1) & MASK32 for k in KEYS]
    for w in range(2):
        assert consistent_multipliers(hlo, [ob[w] for ob in single_key_bits]) == []


def _predicted_block_ok(words, nb, h, mult, shift_block=0):
    j = (oracle.block_index(h, nb) + shift_block) % nb
    hlo = h & MASK32
    for w in range(8):
        bit = ((hlo * mult[w]) & MASK32) >> 27
        if not (int(words[j * 8 + w]) >> bit) & 1:
            return False
    return True


def test_xxh64_high_half_and_block_rule_consistent_with_parquet(recovered_multipliers):
    mult = [m[0] for m in recovered_multipliers]
    keys = [int(x) for x in (np.arange(3000, dtype=np.int64) * 7919 - 123456789)]
    words = parquet_bitset(keys)
    nb = words.size // 8
    assert nb >= 64
    hs = [oracle.key_hash(k & (2**64 - 1), 0) for k in keys]
    # every inserted key is found in the block the oracle's rule selects
    assert all(_predicted_block_ok(words, nb, h, mult) for h in hs)
    # negative control: the neighbouring block holds the pattern only rarely
    hits = sum(_predicted_block_ok(words, nb, h, mult, shift_block=1) for h in hs)
    assert hits < 0.2 * len(hs)


def test_oracle_parquet_salt_set_is_the_recovered_one(recovered_multipliers):
    # the oracle's salt set 1 equals what pyarrow's writer output determines
    assert oracle.parquet_salts() == [m[0] for m in recovered_multipliers]


@pytest.mark.parametrize("n", [1, 37, 3000, 20_000])
def test_oracle_parquet_mode_reproduces_pyarrow_bitsets(n):
    """With salt set 1 the oracle's whole bit array is the one pyarrow stores
    (same keys, same number of blocks): the filter is Parquet-compatible."""
    keys = np.arange(n, dtype=np.int64) * 2654435761 - 987654321
    words = parquet_bitset(keys)
    nb = words.size // 8
    geom = oracle.Geometry(num_blocks=nb, block_bits=256, word_bits=32, k=8, seed=0, salts=1)
    assert geom.valid()
    f = oracle.SBF(geom)
    f.add(keys.view(np.uint64))
    assert np.array_equal(f.words, words)
    # the default salt set does not reproduce it (negative control)
    g = oracle.SBF(oracle.Geometry(num_blocks=nb, block_bits=256, word_bits=32, k=8, seed=0))
    g.add(keys.view(np.uint64))
    assert not np.array_equal(g.words, words)


def test_parquet_salt_set_geometry_rules():
    ok = oracle.Geometry(num_blocks=10, block_bits=256, word_bits=32, k=8, salts=1)
    assert ok.valid()
    for kw in ({"k": 16}, {"block_bits": 512}, {"word_bits": 64, "block_bits": 512}, {"groups": 2}):
        args = dict(num_blocks=10, block_bits=256, word_bits=32, k=8, salts=1)
        args.update(kw)
        assert not oracle.Geometry(**args).valid(), kw
    assert not oracle.Geometry(num_blocks=10, salts=2).valid()
