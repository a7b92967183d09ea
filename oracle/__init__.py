"""CPU oracle for the sectorized blocked Bloom filter.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and
the CPU-baseline legs of ``bench.py`` may import this package.  The product
library never calls it, and it never calls the product library.

Two parts:

* ``sbf_oracle.c`` (built here with gcc into ``oracle/_build``): XXH64, salts,
  block selection, bit positions, construction and lookup, one key at a time.
* this module: ctypes marshalling for the C part, and the false-positive-rate
  formulas in fp64:
    - :func:`eq1_cbf` is the paper's Eq. (1) for the classical filter;
    - :func:`fpr_sbf_closed_form` extends it exactly to the blocked,
      sectorized filter (Sec. II-A: a block holds a binomial share of the
      keys, each of its s words receives k' = k/s independent bit positions);
    - :func:`fpr_given_filter` is the exact false-positive probability of a
      fresh key against a given bit array.

Pins against facts outside this code live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbf_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libsbf_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (idempotent)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra",
                           "-o", tmp, _SRC])
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Params(ctypes.Structure):
    _fields_ = [("num_blocks", ctypes.c_uint64), ("block_bits", ctypes.c_uint32),
                ("word_bits", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("groups", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("salts", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


def lib():
    global _lib
    if _lib is None:
        L = ctypes.CDLL(build())
        u64, u32, vp, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int
        P = ctypes.POINTER(_Params)
        sigs = {
            "orc_xxh64": (u64, [ctypes.c_char_p, u64, u64]),
            "orc_key_hash": (u64, [u64, u64]),
            "orc_salt64": (u64, [u32]),
            "orc_salt32": (u32, [u32]),
            "orc_parquet_salt32": (u32, [u32]),
            "orc_block_index": (u64, [u64, u64]),
            "orc_bit_position": (u32, [u64, u32, u32]),
            "orc_check": (i32, [P]),
            "orc_word_pattern": (u64, [P, u64, u32]),
            "orc_group_word": (u32, [P, u64, u32]),
            "orc_group_pattern": (u64, [P, u64, u32]),
            "orc_add": (i32, [P, vp, vp, u64]),
            "orc_add_block_range": (i32, [P, vp, u64, u64, vp, u64]),
            "orc_contains": (i32, [P, vp, vp, u64, vp]),
            "orc_contains_block_range": (i32, [P, vp, u64, u64, vp, u64, vp]),
            "orc_key_blocks": (i32, [P, vp, u64, vp, vp]),
            "orc_hash_keys": (None, [vp, u64, u64, vp]),
            "orc_block_indices": (None, [vp, u64, u64, u64, vp]),
        }
        for name, (res, args) in sigs.items():
            f = getattr(L, name)
            f.restype, f.argtypes = res, args
        _lib = L
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _keys(keys) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(keys).view(np.uint64) if np.asarray(keys).dtype == np.int64
                                else np.asarray(keys, dtype=np.uint64))


# ---------------------------------------------------------------------------
# hashing primitives
# ---------------------------------------------------------------------------
def xxh64(data: bytes, seed: int = 0) -> int:
    return lib().orc_xxh64(data, len(data), seed)


def key_hash(key: int, seed: int = 0) -> int:
    return lib().orc_key_hash(key, seed)


def hash_keys(keys, seed: int = 0) -> np.ndarray:
    k = _keys(keys)
    out = np.empty(k.size, dtype=np.uint64)
    lib().orc_hash_keys(_ptr(k), k.size, seed, _ptr(out))
    return out


def block_indices(keys, num_blocks: int, seed: int = 0) -> np.ndarray:
    k = _keys(keys)
    out = np.empty(k.size, dtype=np.uint64)
    lib().orc_block_indices(_ptr(k), k.size, seed, num_blocks, _ptr(out))
    return out


def parquet_salts() -> list[int]:
    """Salt set 1: the Parquet split-block filter's eight multipliers."""
    return [lib().orc_parquet_salt32(i) for i in range(8)]


def salts(word_bits: int, count: int = 64) -> list[int]:
    L = lib()
    return [L.orc_salt32(i) if word_bits == 32 else L.orc_salt64(i) for i in range(count)]


def block_index(h: int, num_blocks: int) -> int:
    return lib().orc_block_index(h, num_blocks)


def bit_position(h: int, salt_index: int, word_bits: int) -> int:
    return lib().orc_bit_position(h, salt_index, word_bits)


# ---------------------------------------------------------------------------
# the filter
# ---------------------------------------------------------------------------
@dataclass(frozen=True)
class Geometry:
    """Filter geometry.  groups = z: 0 (or s) = sectorized filter (SBF);
    0 < z < s = cache-sectorized filter (CSBF, Sec. II-A)."""
    num_blocks: int
    block_bits: int = 256
    word_bits: int = 32
    k: int = 8
    seed: int = 0
    groups: int = 0
    salts: int = 0  # 0: SplitMix64 salts; 1: the Parquet split-block salts (256/32/8 only)

    @property
    def s(self) -> int:
        return self.block_bits // self.word_bits

    @property
    def z(self) -> int:
        return self.groups or self.s

    @property
    def kp(self) -> int:
        """bits per touched word (k/s for the SBF, k/z for the CSBF)"""
        return self.k // self.z

    @property
    def num_words(self) -> int:
        return self.num_blocks * self.s

    @property
    def nbytes(self) -> int:
        return self.num_blocks * self.block_bits // 8

    @property
    def word_dtype(self):
        return np.uint32 if self.word_bits == 32 else np.uint64

    def cparams(self) -> _Params:
        return _Params(self.num_blocks, self.block_bits, self.word_bits, self.k, self.groups, self.seed, self.salts, 0)

    def valid(self) -> bool:
        p = self.cparams()
        return lib().orc_check(ctypes.byref(p)) == 0


class SBF:
    """The filter as plain host memory plus the C oracle's add / contains."""

    def __init__(self, geom: Geometry):
        if not geom.valid():
            raise ValueError(f"geometry not admitted by the SBF definition: {geom}")
        self.geom = geom
        self._p = geom.cparams()
        self.words = np.zeros(geom.num_words, dtype=geom.word_dtype)

    def add(self, keys) -> None:
        k = _keys(keys)
        rc = lib().orc_add(ctypes.byref(self._p), _ptr(self.words), _ptr(k), k.size)
        assert rc == 0

    def contains(self, keys) -> np.ndarray:
        k = _keys(keys)
        out = np.empty(k.size, dtype=np.uint8)
        rc = lib().orc_contains(ctypes.byref(self._p), _ptr(self.words), _ptr(k), k.size, _ptr(out))
        assert rc == 0
        return out

    def pattern(self, h: int, w: int) -> int:
        return lib().orc_word_pattern(ctypes.byref(self._p), h, w)

    def group_word(self, h: int, q: int) -> int:
        return lib().orc_group_word(ctypes.byref(self._p), h, q)

    def group_pattern(self, h: int, q: int) -> int:
        return lib().orc_group_pattern(ctypes.byref(self._p), h, q)

    def as_bytes(self) -> np.ndarray:
        return self.words.view(np.uint8)


def add_block_range(geom: Geometry, block_lo: int, block_hi: int, keys, words=None) -> np.ndarray:
    """Construction restricted to blocks [block_lo, block_hi) (a slice of the array)."""
    p = geom.cparams()
    if words is None:
        words = np.zeros((block_hi - block_lo) * geom.s, dtype=geom.word_dtype)
    k = _keys(keys)
    rc = lib().orc_add_block_range(ctypes.byref(p), _ptr(words), block_lo, block_hi, _ptr(k), k.size)
    assert rc == 0
    return words


def add_sparse(geom: Geometry, keys) -> tuple[np.ndarray, np.ndarray]:
    """Construction of a filter too large to hold, for few keys: the sorted
    indices of the blocks the keys touch and those blocks' words
    ([blocks, s]), every other block being zero.  Each key's block image
    comes from the oracle (its pattern in an empty block); the images of keys
    sharing a block are ORed (Sec. II-A: construction ORs every key's pattern
    into its block)."""
    p = geom.cparams()
    k = _keys(keys)
    blocks = np.empty(k.size, dtype=np.uint64)
    images = np.empty((k.size, geom.s), dtype=geom.word_dtype)
    rc = lib().orc_key_blocks(ctypes.byref(p), _ptr(k), k.size, _ptr(blocks), _ptr(images))
    assert rc == 0
    order = np.argsort(blocks, kind="stable")
    blocks, images = blocks[order], images[order]
    uniq, first = np.unique(blocks, return_index=True)
    words = np.bitwise_or.reduceat(images, first, axis=0) if k.size else images
    return uniq, words


def contains_block_range(geom: Geometry, words: np.ndarray, block_lo: int, block_hi: int, keys) -> np.ndarray:
    """Lookup against a slice; 2 marks keys whose block is outside the slice."""
    p = geom.cparams()
    k = _keys(keys)
    out = np.empty(k.size, dtype=np.uint8)
    rc = lib().orc_contains_block_range(ctypes.byref(p), _ptr(words), block_lo, block_hi,
                                        _ptr(k), k.size, _ptr(out))
    assert rc == 0
    return out


# ---------------------------------------------------------------------------
# false-positive rate
# ---------------------------------------------------------------------------
def eq1_cbf(c: float, k: int) -> float:
    """Eq. (1): f(c, k) ~ (1 - e^{-k/c})^k for a classical filter with c bits per key."""
    return (1.0 - math.exp(-k / c)) ** k


def eq1_kopt(c: float) -> float:
    """Eq. (1): the accuracy-optimal hash count k* = c ln 2."""
    return c * math.log(2.0)


def _stirling2(n: int, q: int) -> int:
    # S(n, q) by the recurrence S(n, q) = q S(n-1, q) + S(n-1, q-1)
    row = [1] + [0] * q
    for _ in range(n):
        new = [0] * (q + 1)
        for j in range(1, q + 1):
            new[j] = j * row[j] + row[j - 1]
        row = new
    return row[q]


def distinct_pmf(throws: int, bins: int) -> list[float]:
    """P(exactly q distinct bins hit) for ``throws`` uniform throws into ``bins`` bins."""
    total = bins ** throws
    return [math.comb(bins, q) * math.factorial(q) * _stirling2(throws, q) / total
            for q in range(throws + 1)]


def word_fpr(load: int, kp: int, S: int) -> float:
    """P(a fresh key's k' bits in one word are all set | the word got ``load`` bit throws).

    The fresh key's k' throws hit q distinct positions; each of those is set
    after ``load`` uniform throws, by inclusion-exclusion over the q positions.
    """
    pq = distinct_pmf(kp, S)
    total = 0.0
    for q in range(1, kp + 1):
        if pq[q] == 0.0:
            continue
        terms = [(-1) ** r * math.comb(q, r) * (1.0 - r / S) ** load for r in range(q + 1)]
        total += pq[q] * math.fsum(terms)
    return total


def _binom_pmf(i: int, n: int, p: float) -> float:
    if i > n:
        return 0.0
    log_falling = math.fsum(math.log(n - t) for t in range(i))
    return math.exp(log_falling - math.lgamma(i + 1) + i * math.log(p) + (n - i) * math.log1p(-p))


def fpr_sbf_closed_form(num_blocks: int, n: int, block_bits: int, word_bits: int, k: int) -> float:
    """Expected FPR of the SBF with ``n`` keys, ideal hashing (Sec. II-A + Eq. (1)).

    FPR = sum_i Binom(i; n, 1/b) * word_fpr(i * k', k', S) ** s.
    The sum runs until the binomial tail is below 1e-18.
    """
    s = block_bits // word_bits
    kp = k // s
    p = 1.0 / num_blocks
    mean = n * p
    sd = math.sqrt(max(mean * (1 - p), 1e-300))
    i_hi = min(n, int(mean + 40 * sd + 50))
    i_lo = max(0, int(mean - 40 * sd - 50))
    if num_blocks == 1:
        return word_fpr(n * kp, kp, word_bits) ** s
    acc = []
    for i in range(i_lo, i_hi + 1):
        w = _binom_pmf(i, n, p)
        if w == 0.0:
            continue
        acc.append(w * word_fpr(i * kp, kp, word_bits) ** s)
    return math.fsum(acc)


def fpr_csbf_closed_form(num_blocks: int, n: int, block_bits: int, word_bits: int, k: int, groups: int) -> float:
    """Expected FPR of the cache-sectorized filter (Sec. II-A, CSBF), ideal hashing.

    A block holds i ~ Binom(n, 1/b) keys; in each of its z groups a key selects
    one of g = s/z words, so the word a fresh query selects has received
    m ~ Binom(i, 1/g) keys' worth of k' = k/z throws:
        FPR = sum_i Binom(i; n, 1/b) * [sum_m Binom(m; i, 1/g) * word_fpr(m k', k', S)]^z.
    With z = s (g = 1) this is fpr_sbf_closed_form.
    """
    s = block_bits // word_bits
    z = groups or s
    g = s // z
    kp = k // z
    if g == 1:
        return fpr_sbf_closed_form(num_blocks, n, block_bits, word_bits, k)
    p = 1.0 / num_blocks
    mean = n * p
    sd = math.sqrt(max(mean * (1 - p), 1e-300))
    i_hi = min(n, int(mean + 40 * sd + 50))
    i_lo = max(0, int(mean - 40 * sd - 50))
    wf_cache = {}

    def wf(load):
        if load not in wf_cache:
            wf_cache[load] = word_fpr(load, kp, word_bits)
        return wf_cache[load]

    acc = []
    for i in range(i_lo, i_hi + 1):
        w = _binom_pmf(i, n, p) if num_blocks > 1 else (1.0 if i == n else 0.0)
        if w == 0.0:
            continue
        grp = math.fsum(_binom_pmf(m, i, 1.0 / g) * wf(m * kp) for m in range(i + 1))
        acc.append(w * grp ** z)
    return math.fsum(acc)


def fpr_given_filter(words: np.ndarray, geom: Geometry) -> float:
    """Exact FPR of a fresh key against this bit array (ideal hashing of the key).

    A fresh key picks a uniform block, then (SBF) k' independent uniform
    positions per word: P(all set) = (1/b) sum_blocks prod_w (popcount_w / S)^k';
    (CSBF) in each group a uniform word of its g, then k' positions in it:
    (1/b) sum_blocks prod_groups (1/g) sum_{w in group} (popcount_w / S)^k'.
    """
    pc = np.bitwise_count(words).astype(np.float64).reshape(geom.num_blocks, geom.z, geom.s // geom.z)
    per_group = np.mean((pc / geom.word_bits) ** geom.kp, axis=2)
    per_block = np.prod(per_group, axis=1)
    return float(math.fsum(per_block) / geom.num_blocks)


def binomial_3sigma(p: float, n: int) -> float:
    return 3.0 * math.sqrt(max(p * (1.0 - p), 0.0) / n)
