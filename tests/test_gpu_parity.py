"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bit-exact on the filter's bit array and on every per-query result, for every
compiled geometry and every valid (Theta, Phi) layout with every keys-per-
thread value, on seeded synthetic keys, including ragged tails, single-block
filters, misaligned pointers and both residency regimes.
"""
import numpy as np
import pytest

import oracle
import synthkeys
from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

GEOMETRIES = [(64, 32), (128, 32), (256, 32), (512, 32), (64, 64), (128, 64), (256, 64), (512, 64), (1024, 64)]


def compiled_geometries():
    for B, S in GEOMETRIES:
        s = B // S
        for k in (4, 8, 16):
            if k >= s and k % s == 0:
                yield B, S, k


@pytest.fixture(scope="module")
def torch():
    import torch as t
    from paper_2512_15595_gb300 import build
    build.build()
    return t


def dev_keys(torch, keys_u64):
    return torch.from_numpy(np.ascontiguousarray(keys_u64).view(np.int64)).cuda()


def gpu_filter(geom, torch):
    from paper_2512_15595_gb300 import Filter
    return Filter(geom.num_blocks, geom.block_bits, geom.word_bits, geom.k, geom.seed)


def words_np(f):
    return f.words.cpu().numpy()


# ---------------------------------------------------------------------------
# the 1 MiB workload: 2^15 x 256-bit blocks, S = 32, k = 8, 10^6 keys
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def cfg1():
    geom = oracle.Geometry(num_blocks=1 << 15, block_bits=256, word_bits=32, k=8, seed=0)
    ins = synthkeys.insert_keys(10**6)
    q, is_mem = synthkeys.mixed_queries(10**6, 500_000, 500_000)
    ref = oracle.SBF(geom)
    ref.add(ins)
    return geom, ins, q, is_mem, ref, ref.contains(q)


@pytest.mark.parametrize("kpt", [1, 2, 4])
def test_cfg1_every_layout_bit_exact(torch, cfg1, kpt):
    from paper_2512_15595_gb300 import BF_OP_ADD, BF_OP_CONTAINS, valid_layouts
    geom, ins, q, is_mem, ref, ref_out = cfg1
    dk, dq = dev_keys(torch, ins), dev_keys(torch, q)
    for cg, phi in valid_layouts(256, 32):
        f = gpu_filter(geom, torch)
        f.set_layout(BF_OP_ADD, cg=cg, phi=phi, kpt=kpt)
        f.set_layout(BF_OP_CONTAINS, cg=cg, phi=phi, kpt=kpt)
        f.add(dk)
        out = f.contains(dq)
        torch.cuda.synchronize()
        assert np.array_equal(words_np(f), ref.as_bytes()), (cg, phi, kpt)
        got = out.cpu().numpy().astype(np.uint8)
        assert np.array_equal(got, ref_out), (cg, phi, kpt)
        assert got[is_mem == 1].all()  # no false negatives
        f.close()


def test_cfg1_fpr_in_band(torch, cfg1):
    geom, ins, q, is_mem, ref, ref_out = cfg1
    f = gpu_filter(geom, torch)
    f.add(dev_keys(torch, ins))
    out = f.contains(dev_keys(torch, q)).cpu().numpy()
    fresh = is_mem == 0
    measured = out[fresh].mean()
    realized = oracle.fpr_given_filter(ref.words, geom)
    assert abs(measured - realized) <= oracle.binomial_3sigma(realized, int(fresh.sum()))


# ---------------------------------------------------------------------------
# every compiled geometry x layout x keys-per-thread, ragged sizes
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("B,S,k", list(compiled_geometries()))
def test_every_geometry_layout_bit_exact(torch, B, S, k):
    from paper_2512_15595_gb300 import BF_OP_ADD, BF_OP_CONTAINS, valid_layouts
    geom = oracle.Geometry(num_blocks=1009, block_bits=B, word_bits=S, k=k, seed=0xABCDEF)
    n_ins = 1009 * B // 12 + 17
    ins = synthkeys.insert_keys(n_ins, seed=11)
    q, _ = synthkeys.mixed_queries(n_ins, 1500, 2505, seed_insert=11)
    ref = oracle.SBF(geom)
    ref.add(ins)
    ref_out = ref.contains(q)
    dk, dq = dev_keys(torch, ins), dev_keys(torch, q)
    for cg, phi in valid_layouts(B, S):
        for kpt in (1, 2, 4):
            f = gpu_filter(geom, torch)
            f.set_layout(BF_OP_ADD, cg=cg, phi=phi, kpt=kpt, block_threads=128)
            f.set_layout(BF_OP_CONTAINS, cg=cg, phi=phi, kpt=kpt, block_threads=128)
            f.add(dk)
            out = f.contains(dq)
            assert np.array_equal(words_np(f), ref.as_bytes()), (cg, phi, kpt)
            assert np.array_equal(out.cpu().numpy().astype(np.uint8), ref_out), (cg, phi, kpt)
            f.close()


# ---------------------------------------------------------------------------
# edge cases
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("n", [0, 1, 31, 32, 33, 127, 129, 1000])
@pytest.mark.parametrize("b", [1, 7])
def test_small_and_ragged(torch, n, b):
    from paper_2512_15595_gb300 import BF_OP_ADD, BF_OP_CONTAINS
    geom = oracle.Geometry(num_blocks=b, block_bits=256, word_bits=32, k=8, seed=5)
    ins = synthkeys.insert_keys(n, seed=21)
    q = synthkeys.splitmix64(22, 0, n + 3)
    q[: n // 2] = ins[: n // 2]
    ref = oracle.SBF(geom)
    ref.add(ins)
    for cg, kpt in [(1, 4), (8, 1), (2, 2)]:
        f = gpu_filter(geom, torch)
        f.set_layout(BF_OP_ADD, cg=cg, kpt=kpt)
        f.set_layout(BF_OP_CONTAINS, cg=cg, kpt=kpt)
        if n:
            f.add(dev_keys(torch, ins))
        else:
            f.add(torch.empty(0, dtype=torch.int64, device="cuda"))
        out = f.contains(dev_keys(torch, q))
        assert np.array_equal(words_np(f), ref.as_bytes())
        assert np.array_equal(out.cpu().numpy().astype(np.uint8), ref.contains(q))
        f.close()


def test_misaligned_pointers_and_launch_shapes(torch):
    from paper_2512_15595_gb300 import BF_OP_ADD, BF_OP_CONTAINS
    geom = oracle.Geometry(num_blocks=4099, block_bits=512, word_bits=64, k=16, seed=9)
    ins = synthkeys.insert_keys(40_001, seed=31)
    q, _ = synthkeys.mixed_queries(40_001, 7000, 9001, seed_insert=31)
    ref = oracle.SBF(geom)
    ref.add(ins)
    ref_out = ref.contains(q)
    # keys at an 8-byte (not 32-byte) offset, results at an odd byte offset
    dk = torch.empty(ins.size + 1, dtype=torch.int64, device="cuda")
    dk[1:] = dev_keys(torch, ins)
    dq = torch.empty(q.size + 1, dtype=torch.int64, device="cuda")
    dq[1:] = dev_keys(torch, q)
    out_buf = torch.zeros(q.size + 1, dtype=torch.uint8, device="cuda")
    for threads, grid in [(32, 1), (64, 3), (512, 0), (256, 1000)]:
        f = gpu_filter(geom, torch)
        f.set_layout(BF_OP_ADD, cg=8, phi=1, kpt=4, block_threads=threads, grid_ctas=grid)
        f.set_layout(BF_OP_CONTAINS, cg=2, phi=4, kpt=4, block_threads=threads, grid_ctas=grid)
        f.add(dk[1:])
        f.contains(dq[1:], out=out_buf[1:])
        assert np.array_equal(words_np(f), ref.as_bytes()), (threads, grid)
        assert np.array_equal(out_buf[1:].cpu().numpy(), ref_out), (threads, grid)
        f.close()


def test_duplicates_and_idempotence(torch):
    geom = oracle.Geometry(num_blocks=333, block_bits=128, word_bits=32, k=8, seed=1)
    ins = synthkeys.insert_keys(5000, seed=41)
    dup = np.concatenate([ins, ins[::-1], ins[:100]])
    ref = oracle.SBF(geom)
    ref.add(ins)
    f = gpu_filter(geom, torch)
    f.add(dev_keys(torch, dup))
    f.add(dev_keys(torch, ins))
    assert np.array_equal(words_np(f), ref.as_bytes())
    f.clear()
    assert not f.contains(dev_keys(torch, ins)).any().item()


def test_library_allocated_filter(torch):
    from paper_2512_15595_gb300 import _lib, bf_params, device_tensor
    geom = oracle.Geometry(num_blocks=2000, block_bits=256, word_bits=64, k=16, seed=77)
    ins = synthkeys.insert_keys(20_000, seed=51)
    ref = oracle.SBF(geom)
    ref.add(ins)
    h = _lib.bf_create(bf_params(2000, 256, 64, 16, 0, 77), None)
    try:
        ptr, nbytes = _lib.bf_words(h)
        assert nbytes == geom.nbytes
        words = device_tensor(ptr, nbytes, "cuda")
        assert not words.any().item()  # zeroed at creation
        dk = dev_keys(torch, ins)
        _lib.bf_add(h, dk.data_ptr(), dk.numel())
        torch.cuda.synchronize()
        assert np.array_equal(words.cpu().numpy(), ref.as_bytes())
    finally:
        _lib.bf_destroy(h)


@pytest.mark.parametrize("mode", ["direct_pinned", "direct_pageable", "staged"])
def test_host_pipeline(torch, mode):
    from paper_2512_15595_gb300 import _lib
    geom = oracle.Geometry(num_blocks=10007, block_bits=256, word_bits=32, k=8, seed=3)
    ins = synthkeys.insert_keys(300_001, seed=61)
    q, _ = synthkeys.mixed_queries(300_001, 50_000, 70_007, seed_insert=61)
    ref = oracle.SBF(geom)
    ref.add(ins)
    f = gpu_filter(geom, torch)
    # several chunks plus a ragged one when staged
    _lib.bf_set_staging(f.handle, 4096 * 7 + 3, _lib.BF_HOST_STAGED if mode == "staged" else _lib.BF_HOST_AUTO)
    if mode == "direct_pageable":
        h_ins, h_q = ins.copy(), q.copy()
        h_out = np.empty(q.size, dtype=np.uint8)
    else:
        h_ins = torch.from_numpy(ins.view(np.int64)).pin_memory().numpy()
        h_q = torch.from_numpy(q.view(np.int64)).pin_memory().numpy()
        h_out = torch.empty(q.size, dtype=torch.uint8).pin_memory().numpy()
    f.add_host(h_ins)
    f.contains_host(h_q, h_out)
    torch.cuda.current_stream().synchronize()
    if mode == "staged":
        assert f.last_launches() == -(-q.size // (4096 * 7 + 3))
    elif mode == "direct_pinned":
        assert f.last_launches() == 1
    assert np.array_equal(words_np(f), ref.as_bytes())
    assert np.array_equal(h_out, ref.contains(q))
    f.close()


# ---------------------------------------------------------------------------
# L2-blocked (partitioned) construction
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("B,S,k", [(256, 32, 8), (512, 64, 16), (64, 64, 4), (128, 32, 16), (1024, 64, 16)])
def test_partitioned_add_bit_exact(torch, B, S, k):
    from paper_2512_15595_gb300 import BF_OP_ADD, valid_layouts
    geom = oracle.Geometry(num_blocks=(1 << 14) + 77, block_bits=B, word_bits=S, k=k, seed=123)
    ins = synthkeys.insert_keys(150_001, seed=81)
    ref = oracle.SBF(geom)
    ref.add(ins)
    dk = dev_keys(torch, ins)
    cases = [dict(slice_log2=16), dict(slice_log2=17, chunk_keys=4096 * 5 + 1), dict(slice_log2=16, cap_override=128),
             dict(slice_log2=16, window_log2=17)]
    for cfg in cases:
        nparts = -(-geom.nbytes // (1 << cfg["slice_log2"]))
        per_launch = 1 << max(0, cfg.get("window_log2", 26) - cfg["slice_log2"])
        per_pass = 1 + -(-nparts // per_launch)
        for cg, phi in valid_layouts(B, S)[:: max(1, len(valid_layouts(B, S)) // 4)]:
            for kpt in (1, 4):
                f = gpu_filter(geom, torch)
                f.set_partition(mode=1, **cfg)
                f.set_layout(BF_OP_ADD, cg=cg, phi=phi, kpt=kpt)
                f.add(dk)
                launches = f.last_launches()
                assert np.array_equal(words_np(f), ref.as_bytes()), (cfg, cg, phi, kpt)
                passes = -(-ins.size // cfg.get("chunk_keys", 1 << 32))
                assert launches == per_pass * passes, (cfg, launches)
                assert f.device_status() == 0
                f.close()


def host_buffers(torch, buf, *arrays):
    """Host copies of `arrays`: page-locked, or plain (pageable) numpy."""
    if buf.startswith("pinned"):
        return [torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a).pin_memory().numpy()
                for a in arrays]
    return [a.copy() for a in arrays]


def host_plan(buf, n, cap, h_keys):
    """(keys per pass, launches per pass beyond the filter kernels) of a
    pass-wise host-buffer call: staged passes split n into 7.25 shares (a
    short last pass), rounded up to 256 keys;
    with keys the kernels can address (every buffer but the forced-staging
    one) the staging kernel runs once per pass, plus a one-thread launch for
    an odd last key of a 16-byte aligned pass; the copy engine counts none;
    in-place passes (BF_HOST_DIRECT) split n / 8 unrounded."""
    if buf == "pinned_direct":
        pk = min(cap, -(-n // 8))
        return pk, [0] * -(-n // pk)
    pk = min(cap, -(-(-(-4 * n // 29)) // 256) * 256)
    extra = []
    for lo in range(0, n, pk):
        cnt = min(pk, n - lo)
        if buf == "pageable_staged":
            extra.append(0)
        elif (h_keys.ctypes.data + 8 * lo) % 16 == 0:
            extra.append(int(cnt >= 2) + (cnt & 1))
        else:
            extra.append(1)
    return pk, extra


@pytest.mark.parametrize("buf", ["pinned", "pinned_direct", "pageable", "pageable_staged"])
def test_partitioned_add_from_host_keys(torch, buf):
    """Construction from host keys in passes: staged into two device slots
    (by the staging kernel from page-locked or pageable keys, by the copy
    engine when staging is forced) while the device partitions and inserts
    the previous pass; or, with BF_HOST_DIRECT, read in place over two
    alternating workspaces with the record inserts on a second stream.  Bits
    as the oracle's, launch counts as planned, and the workspace shared
    correctly with a following device-key construction and a host-key
    lookup."""
    geom = oracle.Geometry(num_blocks=(1 << 14) + 77, block_bits=256, word_bits=32, k=8, seed=5)
    ins = synthkeys.insert_keys(150_001, seed=87)
    more = synthkeys.insert_keys(40_000, seed=88)
    q, is_mem = synthkeys.mixed_queries(150_001, 30_000, 60_001, seed_insert=87)
    ref = oracle.SBF(geom)
    ref.add(ins)
    want_first = ref.as_bytes().copy()
    ref.add(more)
    h_ins, h_q, h_out = host_buffers(torch, buf, ins, q, np.zeros(q.size, dtype=np.uint8))
    cases = [dict(slice_log2=16), dict(slice_log2=16, chunk_keys=4096 * 5 + 1), dict(slice_log2=16, cap_override=128),
             dict(slice_log2=17, window_log2=17)]
    for cfg in cases:
        f = gpu_filter(geom, torch)
        f.set_partition(mode=1, **cfg)
        if buf in ("pageable_staged", "pinned_direct"):
            f.set_staging(mode="staged" if buf == "pageable_staged" else "direct")
        f.add_host(h_ins)
        torch.cuda.synchronize()
        nparts = -(-geom.nbytes // (1 << cfg["slice_log2"]))
        per_launch = 1 << max(0, cfg.get("window_log2", 26) - cfg["slice_log2"])
        _, extra = host_plan(buf, ins.size, cfg.get("chunk_keys", 1 << 32), h_ins)
        assert f.last_launches() == len(extra) * (1 + -(-nparts // per_launch)) + sum(extra), (cfg,
                                                                                                f.last_launches())
        assert np.array_equal(words_np(f), want_first), cfg
        f.add(dev_keys(torch, more))
        f.contains_host(h_q, h_out)
        torch.cuda.synchronize()
        assert np.array_equal(words_np(f), ref.as_bytes()), cfg
        assert np.array_equal(h_out, ref.contains(q)), cfg
        assert f.device_status() == 0
        f.close()


@pytest.mark.parametrize("B,S,k", [(256, 32, 8), (512, 64, 16)])
def test_partitioned_add_overlapped_passes(torch, B, S, k):
    """Device-key construction in passes over two workspaces, the record
    inserts of one pass on a second stream beside the next pass's partition
    (grid limited to part_ctas CTAs per SM): the oracle's bits for every pass
    count and CTA limit, keys at a 16-byte and at an 8-byte offset, and a
    following serial construction on the same filter."""
    geom = oracle.Geometry(num_blocks=(1 << 14) + 77, block_bits=B, word_bits=S, k=k, seed=77)
    ins = synthkeys.insert_keys(150_001, seed=85)
    more = synthkeys.insert_keys(30_000, seed=86)
    ref = oracle.SBF(geom)
    ref.add(ins)
    want_first = ref.as_bytes().copy()
    ref.add(more)
    buf = torch.zeros(ins.size + 1, dtype=torch.int64, device="cuda")
    nparts = -(-geom.nbytes // (1 << 16))
    windows = -(-nparts // (1 << (26 - 16)))
    for passes, part_ctas, offset, chunk in [(2, 0, 0, 1 << 32), (3, 1, 1, 1 << 32), (7, 2, 0, 1 << 32),
                                            (2, 1, 1, 4096 * 5 + 1)]:
        dk = buf[offset:offset + ins.size]
        dk.copy_(dev_keys(torch, ins))
        f = gpu_filter(geom, torch)
        f.set_partition(mode=1, slice_log2=16, passes=passes, part_ctas=part_ctas, chunk_keys=chunk)
        f.add(dk)
        pass_keys = min(chunk, -(-ins.size // passes))
        assert f.last_launches() == -(-ins.size // pass_keys) * (1 + windows), (passes, f.last_launches())
        assert np.array_equal(words_np(f), want_first), (passes, part_ctas, offset)
        f.set_partition(passes=0)
        f.add(dev_keys(torch, more))
        assert np.array_equal(words_np(f), ref.as_bytes()), (passes, part_ctas, offset)
        assert f.device_status() == 0
        f.close()


def test_partition_many_tiles_per_cta(torch):
    """Each partition CTA walks many tiles (grid limited to one CTA per SM for
    construction; lookup queries spanning several grid-strides): the
    prefetch of the next tile into the other key buffer, the alternating
    counter sets and the reuse of a tile's key buffer for its sorted records
    all run, with an odd key count (the last key copied alone) and keys at a
    16-byte and at an 8-byte offset."""
    from paper_2512_15595_gb300 import BF_OP_CONTAINS
    geom = oracle.Geometry(num_blocks=(1 << 15) + 5, block_bits=256, word_bits=32, k=8, seed=3)
    ins = synthkeys.insert_keys(2_000_007, seed=95)
    q, is_mem = synthkeys.mixed_queries(2_000_007, 1_000_000, 5_000_003, seed_insert=95)
    ref = oracle.SBF(geom)
    ref.add(ins)
    ref_out = ref.contains(q)
    kbuf = torch.zeros(ins.size + 1, dtype=torch.int64, device="cuda")
    qbuf = torch.zeros(q.size + 1, dtype=torch.int64, device="cuda")
    for offset in (0, 1):
        dk, dq = kbuf[offset:offset + ins.size], qbuf[offset:offset + q.size]
        dk.copy_(dev_keys(torch, ins))
        dq.copy_(dev_keys(torch, q))
        f = gpu_filter(geom, torch)
        f.set_partition(mode=1, slice_log2=16, part_ctas=1, lookup_mode=1)
        f.set_layout(BF_OP_CONTAINS, cg=1, phi=8, kpt=4)
        f.add(dk)
        assert np.array_equal(words_np(f), ref.as_bytes()), offset
        out = f.contains(dq)
        got = out.cpu().numpy().astype(np.uint8)
        assert np.array_equal(got, ref_out), offset
        assert got[is_mem == 1].all()
        assert f.device_status() == 0
        f.close()


@pytest.mark.parametrize("B,S,k", list(compiled_geometries()))
def test_warp_aggregated_add_bit_exact(torch, B, S, k):
    """BF_HINT_WARP_AGGREGATE: the direct and the record-insert construction
    set the oracle's bits for every layout, with distinct keys, with runs of
    repeated keys (many lanes of a warp on one block: the case the
    aggregation merges) and on a 3-block filter (distinct keys sharing
    blocks)."""
    from paper_2512_15595_gb300 import BF_HINT_WARP_AGGREGATE, BF_OP_ADD, valid_layouts
    distinct = synthkeys.insert_keys(20_011, seed=61)
    runs = np.repeat(synthkeys.insert_keys(700, seed=62), 37)
    for nb, keys in (((1 << 12) + 9, distinct), ((1 << 12) + 9, runs), (3, distinct[:3001])):
        geom = oracle.Geometry(num_blocks=nb, block_bits=B, word_bits=S, k=k, seed=44)
        ref = oracle.SBF(geom)
        ref.add(keys)
        dk = dev_keys(torch, keys)
        for cg, phi in valid_layouts(B, S):
            for kpt in (1, 4):
                for part in ((0,), (1,)) if nb > 3 else ((0,),):
                    f = gpu_filter(geom, torch)
                    f.set_layout(BF_OP_ADD, cg=cg, phi=phi, kpt=kpt, flags=BF_HINT_WARP_AGGREGATE)
                    if part[0]:
                        f.set_partition(mode=1, slice_log2=16)
                    f.add(dk)
                    assert np.array_equal(words_np(f), ref.as_bytes()), (nb, cg, phi, kpt, part)
                    assert f.device_status() == 0
                    f.close()


def test_phase_timing_counts_every_launch(torch):
    """bf_set_timing / bf_get_timing: every launch of a partitioned
    construction and lookup (and of the direct kernels) is counted in its
    phase, durations are positive, the sums restart after each read, and the
    results do not change."""
    geom = oracle.Geometry(num_blocks=(1 << 14) + 77, block_bits=256, word_bits=32, k=8, seed=12)
    ins = synthkeys.insert_keys(300_001, seed=97)
    q, _ = synthkeys.mixed_queries(300_001, 50_000, 50_001, seed_insert=97)
    ref = oracle.SBF(geom)
    ref.add(ins)
    f = gpu_filter(geom, torch)
    f.set_partition(mode=1, slice_log2=16, lookup_mode=1)
    f.set_timing(True)
    f.add(dev_keys(torch, ins))
    n_add = f.last_launches()
    out = f.contains(dev_keys(torch, q))
    n_con = f.last_launches()
    t = f.timing()
    assert set(t) == {"partition_add", "record_insert", "partition_lookup", "record_probe", "bitmap_expand"}
    assert t["partition_add"]["launches"] + t["record_insert"]["launches"] == n_add
    assert sum(t[k]["launches"] for k in ("partition_lookup", "record_probe", "bitmap_expand")) == n_con
    assert all(v["ms"] > 0 for v in t.values())
    assert f.timing() == {}
    f.set_partition(mode=0, lookup_mode=0)
    f.add(dev_keys(torch, ins))
    f.contains(dev_keys(torch, q), out=out)
    t = f.timing()
    assert t["add_direct"]["launches"] == 1 and t["contains_direct"]["launches"] == 1
    assert np.array_equal(words_np(f), ref.as_bytes())
    assert np.array_equal(out.cpu().numpy().astype(np.uint8), ref.contains(q))
    assert f.device_status() == 0
    f.set_timing(False)
    f.close()


@pytest.mark.parametrize("buf", ["pinned", "pageable_staged"])
def test_phase_timing_of_staged_host_passes(torch, buf):
    """The host_stage phase of staged host-buffer calls: with the staging
    kernel it counts exactly its launches (as planned per pass), with the
    copy engine (staging forced) none; either way it has a positive time,
    and every filter-kernel launch is counted in its own phase."""
    geom = oracle.Geometry(num_blocks=(1 << 14) + 77, block_bits=256, word_bits=32, k=8, seed=13)
    ins = synthkeys.insert_keys(150_001, seed=99)
    q, _ = synthkeys.mixed_queries(150_001, 30_000, 60_001, seed_insert=99)
    ref = oracle.SBF(geom)
    ref.add(ins)
    h_ins, h_q, h_out = host_buffers(torch, buf, ins, q, np.zeros(q.size, dtype=np.uint8))
    f = gpu_filter(geom, torch)
    f.set_partition(mode=1, slice_log2=16, lookup_mode=1)
    if buf == "pageable_staged":
        f.set_staging(mode="staged")
    f.set_timing(True)
    f.add_host(h_ins)
    n_add = f.last_launches()
    t = f.timing()
    _, extra = host_plan(buf, ins.size, 1 << 32, h_ins)
    assert t["host_stage"]["launches"] == sum(extra) and t["host_stage"]["ms"] > 0
    assert t["partition_add"]["launches"] + t["record_insert"]["launches"] + sum(extra) == n_add
    f.contains_host(h_q, h_out)
    n_con = f.last_launches()
    t = f.timing()
    _, extra = host_plan(buf, q.size, 1 << 28, h_q)
    assert t["host_stage"]["launches"] == sum(extra) and t["host_stage"]["ms"] > 0
    assert sum(t[k]["launches"] for k in ("partition_lookup", "record_probe", "bitmap_expand")) + sum(extra) == n_con
    torch.cuda.synchronize()
    assert np.array_equal(words_np(f), ref.as_bytes())
    assert np.array_equal(h_out, ref.contains(q))
    assert f.device_status() == 0
    f.set_timing(False)
    f.close()


@pytest.mark.parametrize("buf", ["pinned", "pinned_direct", "pageable", "pageable_staged"])
def test_partitioned_lookup_from_host_queries(torch, buf):
    """Slice-partitioned lookup of host queries in passes: through two
    device staging slots (queries in by the staging kernel, or by the copy
    engine when staging is forced; results out by the copy engine); or, with
    BF_HOST_DIRECT, read and written in place, the probes and the expansion
    of one pass on a second stream beside the next pass's partition.  Every
    answer is the oracle's, launch counts as planned, and a device lookup
    afterwards shares the workspace correctly."""
    geom = oracle.Geometry(num_blocks=(1 << 14) + 77, block_bits=256, word_bits=32, k=8, seed=15)
    ins = synthkeys.insert_keys(150_001, seed=93)
    q, is_mem = synthkeys.mixed_queries(150_001, 60_000, 140_003, seed_insert=93)
    ref = oracle.SBF(geom)
    ref.add(ins)
    want = ref.contains(q)
    h_q, h_out = host_buffers(torch, buf, q, np.zeros(q.size, dtype=np.uint8))
    for cfg in (dict(slice_log2=16), dict(slice_log2=16, lookup_chunk_keys=4096 * 3 + 1), dict(slice_log2=17,
                                                                                             window_log2=17)):
        f = gpu_filter(geom, torch)
        f.set_partition(mode=0, lookup_mode=1, **cfg)
        if buf in ("pageable_staged", "pinned_direct"):
            f.set_staging(mode="staged" if buf == "pageable_staged" else "direct")
        f.add(dev_keys(torch, ins))
        h_out[:] = 7
        f.contains_host(h_q, h_out)
        torch.cuda.synchronize()
        nparts = -(-geom.nbytes // (1 << cfg["slice_log2"]))
        windows = -(-nparts // (1 << max(0, cfg.get("window_log2", 26) - cfg["slice_log2"])))
        _, extra = host_plan(buf, q.size, cfg.get("lookup_chunk_keys", 1 << 28), h_q)
        assert f.last_launches() == len(extra) * (2 + windows) + sum(extra), (cfg, f.last_launches())
        assert np.array_equal(h_out, want), cfg
        assert h_out[is_mem == 1].all()
        out = f.contains(dev_keys(torch, q))
        assert np.array_equal(out.cpu().numpy().astype(np.uint8), want), cfg
        assert f.device_status() == 0
        f.close()


@pytest.mark.parametrize("buf", ["pinned", "pageable", "pageable_staged"])
def test_staged_host_passes_tiny_and_ragged(torch, buf):
    """Staged host passes at their edges: 1, 7, 255, 257 and 4099 keys on a
    slice-partitioned filter (a single short pass, the one-thread launch for
    an odd last key, several ragged passes), built up call by call; bits
    and answers as the oracle's after every call."""
    geom = oracle.Geometry(num_blocks=(1 << 14) + 77, block_bits=256, word_bits=32, k=8, seed=31)
    f = gpu_filter(geom, torch)
    f.set_partition(mode=1, slice_log2=16, lookup_mode=1)
    if buf == "pageable_staged":
        f.set_staging(mode="staged")
    ref = oracle.SBF(geom)
    for i, n in enumerate((1, 7, 255, 257, 4099)):
        ins = synthkeys.insert_keys(n, seed=200 + i)
        q, _ = synthkeys.mixed_queries(n, max(1, n // 3), n, seed_insert=200 + i)
        ref.add(ins)
        h_ins, h_q, h_out = host_buffers(torch, buf, ins, q, np.zeros(q.size, dtype=np.uint8))
        f.add_host(h_ins)
        f.contains_host(h_q, h_out)
        torch.cuda.synchronize()
        assert np.array_equal(words_np(f), ref.as_bytes()), n
        assert np.array_equal(h_out, ref.contains(q)), n
    assert f.device_status() == 0
    f.close()


@pytest.mark.parametrize("partitioned", [False, True])
def test_host_keys_at_an_odd_address(torch, partitioned):
    """Host keys 4 bytes off 8-byte alignment (no alignment is required of
    host buffers): the copy engine takes them, directly or in staged passes;
    bits and answers as the oracle's."""
    geom = oracle.Geometry(num_blocks=(1 << 14) + 77, block_bits=256, word_bits=32, k=8, seed=21)
    ins = synthkeys.insert_keys(100_003, seed=95)
    q, is_mem = synthkeys.mixed_queries(100_003, 30_000, 70_001, seed_insert=95)
    ref = oracle.SBF(geom)
    ref.add(ins)
    raw = torch.empty(8 * (ins.size + q.size) + 16, dtype=torch.uint8).pin_memory().numpy()
    base = (-raw.ctypes.data) % 8 + 4
    h_ins = np.frombuffer(raw, dtype=np.uint64, count=ins.size, offset=base)
    h_q = np.frombuffer(raw, dtype=np.uint64, count=q.size, offset=base + 8 * ins.size)
    assert h_ins.ctypes.data % 8 == 4 and h_q.ctypes.data % 8 == 4
    h_ins[:] = ins
    h_q[:] = q
    h_out = np.zeros(q.size + 1, dtype=np.uint8)[1:]
    f = gpu_filter(geom, torch)
    if partitioned:
        f.set_partition(mode=1, slice_log2=16, lookup_mode=1)
    f.add_host(h_ins)
    f.contains_host(h_q, h_out)
    torch.cuda.synchronize()
    assert np.array_equal(words_np(f), ref.as_bytes())
    assert np.array_equal(h_out, ref.contains(q))
    assert f.device_status() == 0
    f.close()


def test_partitioned_add_skewed_keys(torch):
    # every key lands in one slice (duplicates): the slice buffer overflows and
    # the overflow records take the direct path
    geom = oracle.Geometry(num_blocks=1 << 15, block_bits=256, word_bits=32, k=8, seed=0)
    base = synthkeys.insert_keys(64, seed=91)
    ins = np.concatenate([np.repeat(base[:1], 200_000), base, np.repeat(base[5:7], 30_000)])
    ref = oracle.SBF(geom)
    ref.add(ins)
    f = gpu_filter(geom, torch)
    f.set_partition(mode=1, slice_log2=16)
    f.add(dev_keys(torch, ins))
    assert np.array_equal(words_np(f), ref.as_bytes())
    assert f.device_status() == 0
    f.close()


@pytest.mark.parametrize("B,S,k", [(256, 32, 8), (512, 64, 16), (64, 64, 4), (128, 32, 16), (1024, 64, 16)])
def test_partitioned_lookup_bit_exact(torch, B, S, k):
    from paper_2512_15595_gb300 import BF_OP_CONTAINS, valid_layouts
    geom = oracle.Geometry(num_blocks=(1 << 14) + 77, block_bits=B, word_bits=S, k=k, seed=321)
    ins = synthkeys.insert_keys(150_001, seed=83)
    q, is_mem = synthkeys.mixed_queries(150_001, 30_000, 70_013, seed_insert=83)
    ref = oracle.SBF(geom)
    ref.add(ins)
    ref_out = ref.contains(q)
    dk, dq = dev_keys(torch, ins), dev_keys(torch, q)
    out_buf = torch.zeros(q.size + 1, dtype=torch.uint8, device="cuda")
    cases = [dict(slice_log2=16), dict(slice_log2=17, lookup_chunk_keys=4096 * 3 + 1),
             dict(slice_log2=16, cap_override=128), dict(slice_log2=16, window_log2=17)]
    f = gpu_filter(geom, torch)
    f.set_partition(mode=0)
    f.add(dk)
    assert np.array_equal(words_np(f), ref.as_bytes())
    for cfg in cases:
        nparts = -(-geom.nbytes // (1 << cfg["slice_log2"]))
        per_launch = 1 << max(0, cfg.get("window_log2", 26) - cfg["slice_log2"])
        per_pass = 2 + -(-nparts // per_launch)
        passes = -(-q.size // cfg.get("lookup_chunk_keys", 1 << 28))
        for cg, phi in valid_layouts(B, S)[:: max(1, len(valid_layouts(B, S)) // 4)]:
            for kpt, offset in ((1, 0), (4, 1)):
                f.set_partition(mode=0, lookup_mode=1, window_log2=26, cap_override=0, lookup_chunk_keys=1 << 28)
                f.set_partition(**cfg)
                f.set_layout(BF_OP_CONTAINS, cg=cg, phi=phi, kpt=kpt)
                out = out_buf[offset:offset + q.size]
                out.zero_()
                f.contains(dq, out=out)
                assert f.last_launches() == per_pass * passes, (cfg, f.last_launches())
                got = out.cpu().numpy()
                assert np.array_equal(got, ref_out), (cfg, cg, phi, kpt)
                assert got[is_mem == 1].all()
    assert f.device_status() == 0
    f.close()


def test_partition_auto_and_off(torch):
    from paper_2512_15595_gb300 import _lib
    geom = oracle.Geometry(num_blocks=1 << 12, block_bits=256, word_bits=32, k=8, seed=0)
    f = gpu_filter(geom, torch)
    assert f.partition()["mode"] == _lib.BF_PART_AUTO
    f.add(dev_keys(torch, synthkeys.insert_keys(10_000)))
    assert f.last_launches() == 1  # 128 KiB filter: fits L2, direct kernel
    f.set_partition(mode=0)
    f.add(dev_keys(torch, synthkeys.insert_keys(10_000)))
    assert f.last_launches() == 1
    with pytest.raises(Exception):
        f.set_partition(mode=1, slice_log2=8)
    with pytest.raises(Exception):
        f.set_partition(mode=1, cap_override=100)
    with pytest.raises(Exception):
        f.set_partition(passes=65)
    with pytest.raises(Exception):
        f.set_partition(part_ctas=9)
    assert _lib.lib().bf_set_staging(f.handle, 1 << 24, 3) == _lib.BF_EINVAL
    assert _lib.lib().bf_set_staging(f.handle, 1000, _lib.BF_HOST_DIRECT) == _lib.BF_EINVAL
    assert f.device_status() == 0
    f.close()


def test_rejects_misaligned_keys_before_launch(torch):
    from paper_2512_15595_gb300 import BloomError, _lib
    geom = oracle.Geometry(num_blocks=10, block_bits=256, word_bits=32, k=8)
    f = gpu_filter(geom, torch)
    buf = torch.zeros(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(BloomError):
        _lib.bf_add(f.handle, buf.data_ptr() + 4, 1)
    with pytest.raises(BloomError):
        f.set_layout(0, cg=16)
    assert f.device_status() == 0
    f.close()


# ---------------------------------------------------------------------------
# residency regimes
# ---------------------------------------------------------------------------
def test_l2_resident_32mib_with_and_without_persistence(torch):
    from paper_2512_15595_gb300 import BF_HINT_FILTER_EVICT_LAST, BF_OP_ADD, BF_OP_CONTAINS
    geom = oracle.Geometry(num_blocks=1 << 20, block_bits=256, word_bits=32, k=8, seed=0)
    n = (32 << 20) * 8 // 10
    ins = synthkeys.insert_keys(n)
    q, is_mem = synthkeys.stream_queries(0, 4_000_000, n)
    ref = oracle.SBF(geom)
    ref.add(ins)
    ref_out = ref.contains(q)
    dk, dq = dev_keys(torch, ins), dev_keys(torch, q)
    for persist, flags in [(0.0, 0), (1.0, BF_HINT_FILTER_EVICT_LAST)]:
        f = gpu_filter(geom, torch)
        f.set_layout(BF_OP_ADD, flags=flags)
        f.set_layout(BF_OP_CONTAINS, flags=flags)
        if persist:
            f.set_l2_persist(persist)
        f.add(dk)
        out = f.contains(dq)
        torch.cuda.synchronize()
        if persist:
            f.set_l2_persist(0.0)
        assert np.array_equal(words_np(f), ref.as_bytes())
        assert np.array_equal(out.cpu().numpy().astype(np.uint8), ref_out)
        assert f.device_status() == 0
        f.close()


def test_hbm_resident_256mib(torch):
    # 256 MiB is twice the GB300 L2, so most block accesses go to HBM; the
    # default (auto) construction partitions by slice, the direct kernel must agree
    geom = oracle.Geometry(num_blocks=1 << 23, block_bits=256, word_bits=64, k=8, seed=0)
    n = (256 << 20) * 8 // 10
    ins = synthkeys.insert_keys(n)
    q, _ = synthkeys.stream_queries(0, 2_000_000, n)
    ref = oracle.SBF(geom)
    ref.add(ins)
    ref_out = ref.contains(q)
    dk, dq = dev_keys(torch, ins), dev_keys(torch, q)
    # auto: 16 MiB slices, 64 MiB windows -> 1 partition + 4 record-insert launches
    for mode, launches in ((2, 5), (0, 1)):
        f = gpu_filter(geom, torch)
        f.set_partition(mode=mode)
        f.add(dk)
        assert f.last_launches() == launches
        out = f.contains(dq)
        assert np.array_equal(words_np(f), ref.as_bytes())
        assert np.array_equal(out.cpu().numpy().astype(np.uint8), ref_out)
        assert f.device_status() == 0
        f.close()


@pytest.mark.parametrize("nblocks", [1 << 32, (1 << 32) + 12345])
def test_block_index_beyond_32_bits(torch, nblocks):
    # B = 64 bits: 2^32 blocks are a 32 GiB filter; checks the b == 2^32 and
    # b > 2^32 block-selection paths.  The expected bits are composed from the
    # oracle's primitives for the touched words only.
    from paper_2512_15595_gb300 import BF_OP_ADD, BF_OP_CONTAINS
    geom = oracle.Geometry(num_blocks=nblocks, block_bits=64, word_bits=64, k=4, seed=99)
    ins = synthkeys.insert_keys(50_000, seed=71)
    expect = {}
    for key in ins:
        h = oracle.key_hash(int(key), geom.seed)
        j = oracle.block_index(h, nblocks)
        pat = 0
        for t in range(4):
            pat |= 1 << oracle.bit_position(h, t, 64)
        expect[j] = expect.get(j, 0) | pat
    f = gpu_filter(geom, torch)
    f.add(dev_keys(torch, ins))
    w = f.words.view(torch.int64)
    idx = torch.tensor(sorted(expect), dtype=torch.int64, device="cuda")
    got = w[idx].cpu().numpy().view(np.uint64)
    assert [int(x) for x in got] == [expect[j] for j in sorted(expect)]
    w[idx] = 0
    assert not w.any().item()  # no stray bits anywhere else
    w[idx] = torch.from_numpy(got.view(np.int64)).cuda()
    q = synthkeys.splitmix64(72, 0, 20_000)
    q[:5000] = ins[:5000]
    f.set_layout(BF_OP_CONTAINS, kpt=4)
    out = f.contains(dev_keys(torch, q)).cpu().numpy().astype(np.uint8)
    want = []
    for key in q:
        h = oracle.key_hash(int(key), geom.seed)
        j = oracle.block_index(h, nblocks)
        pat = 0
        for t in range(4):
            pat |= 1 << oracle.bit_position(h, t, 64)
        want.append(int((expect.get(j, 0) & pat) == pat))
    assert np.array_equal(out, np.array(want, dtype=np.uint8))
    f.close()
