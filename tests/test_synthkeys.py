"""The seeded input generators (host logic, no GPU): SplitMix64 against its
published definition written out with Python integers, the numpy and torch
versions of every stream agreeing bit for bit (torch on the CPU here; the
same int64 code runs on the GPU), and the workload helpers' invariants."""
import numpy as np
import pytest

import synthkeys
from synthkeys import batches

M = (1 << 64) - 1


def splitmix64_ref(seed, i):
    """Output i of SplitMix64 seeded with `seed` (Steele, Lea and Flood 2014),
    counter-based: mix64(seed + (i + 1) * golden gamma)."""
    z = (seed + (i + 1) * 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def test_splitmix64_matches_definition():
    for seed in (0, 1, 2, 0xDEADBEEF, M):
        got = synthkeys.splitmix64(seed, 5, 40)
        assert [int(x) for x in got] == [splitmix64_ref(seed, i) for i in range(5, 45)]
    # the classic sequential generator started from state 0: its first output
    assert splitmix64_ref(0, 0) == 0xE220A8397B1DCDAF


def test_slices_and_indexed_outputs_agree():
    full = synthkeys.splitmix64(3, 0, 1000)
    assert np.array_equal(synthkeys.splitmix64(3, 400, 100), full[400:500])
    idx = np.array([0, 7, 999, 123], dtype=np.uint64)
    assert np.array_equal(synthkeys.splitmix64_at(3, idx), full[idx.astype(np.int64)])


def test_torch_streams_equal_numpy():
    torch = pytest.importorskip("torch")
    for seed, start, n in ((1, 0, 1000), (2, 12345, 777), (4, (1 << 40) + 3, 50)):
        t = synthkeys.splitmix64_torch(seed, start, n, "cpu", chunk=300)
        assert np.array_equal(synthkeys.as_uint64(t), synthkeys.splitmix64(seed, start, n))
    q = synthkeys.stream_queries_torch(5000, 777, "cpu", ratio_den=10, chunk=1234,
                                       member_flags=torch.empty(5000, dtype=torch.uint8))
    want, _ = synthkeys.stream_queries(0, 5000, 777, 10)
    assert np.array_equal(synthkeys.as_uint64(q), want)


def test_stream_queries_members_and_ratio():
    n_ins = 1000
    q, is_mem = synthkeys.stream_queries(0, 200_000, n_ins, ratio_den=10)
    ins = set(int(x) for x in synthkeys.insert_keys(n_ins))
    members = q[is_mem == 1]
    assert all(int(x) in ins for x in members[:2000])
    frac = is_mem.mean()
    assert abs(frac - 0.1) < 4 * np.sqrt(0.1 * 0.9 / is_mem.size)
    fresh = q[is_mem == 0][:5000]
    assert sum(int(x) in ins for x in fresh) == 0  # 2^-64-rare collisions


def test_mixed_queries_exact_counts():
    q, flag = synthkeys.mixed_queries(5000, 1200, 3000)
    ins = set(int(x) for x in synthkeys.insert_keys(5000))
    assert q.size == 4200 and int(flag.sum()) == 1200
    assert all(int(x) in ins for x in q[flag == 1])
    assert len(set(int(x) for x in q[flag == 1])) == 1200  # distinct members
    assert not any(int(x) in ins for x in q[flag == 0])


def test_batch_layout_helpers():
    sizes = batches.log_uniform_bytes(4096, 4 << 10, 16 << 20, seed=5)
    assert sizes.min() >= 4 << 10 and sizes.max() < 16 << 20
    # log-uniform: the median sits near the geometric mean of the bounds
    assert 0.8 < np.median(sizes) / np.sqrt((4 << 10) * (16 << 20)) < 1.25
    blocks = batches.blocks_of(sizes, 32)
    assert np.array_equal(blocks, np.maximum(1, sizes // 32))
    assert np.array_equal(batches.log_uniform_sizes(4096, 4 << 10, 16 << 20, 32, seed=5), blocks)
    counts = batches.proportional_counts(blocks, 1 << 20)
    assert counts.sum() == 1 << 20
    exact = blocks / blocks.sum() * (1 << 20)
    assert np.all(np.abs(counts - exact) < 1.0)
    off, total = batches.arena_offsets(blocks, 32)
    assert np.all(off % 256 == 0)
    ends = off + blocks * 32
    assert np.all(ends[:-1] <= off[1:]) and ends[-1] <= total < ends[-1] + 256
