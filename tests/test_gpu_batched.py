"""Batched filters against the oracle, filter by filter.

A batch of filters with log-uniform sizes and size-proportional key runs is
built and probed by one launch per operation; every filter's bit array and
every query's answer must equal the oracle's for that filter alone (and the
single-filter C-ABI calls).  Also: every layout, misaligned key runs, empty
filters, and replay from a captured CUDA graph.
"""
import numpy as np
import pytest

import oracle
import synthkeys
from conftest import gpu_available
from synthkeys import batches

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    from paper_2512_15595_gb300 import build
    build.build()
    return t


def make_batch(torch, B, S, k, nfilters=97, total_keys=300_000, seed=7, odd_offsets=False, zeros=(3, 50)):
    from paper_2512_15595_gb300 import Batch
    bb = B // 8
    blocks = batches.log_uniform_sizes(nfilters, 2 * bb, 4096 * bb, bb, seed=seed)
    counts = batches.proportional_counts(blocks, total_keys)
    for z in zeros:
        if z < nfilters:
            counts[z] = 0
    key_off = np.zeros(nfilters, dtype=np.int64)
    key_off[1:] = np.cumsum(counts)[:-1]
    if odd_offsets:
        key_off = key_off + np.arange(nfilters)  # runs start at odd offsets (gaps between runs)
    nkeys = int((key_off + counts).max())
    keys = synthkeys.splitmix64(seed + 100, 0, nkeys)
    off, arena_bytes = batches.arena_offsets(blocks, bb)
    arena = torch.zeros(arena_bytes, dtype=torch.uint8, device="cuda")
    views = [arena[int(o):int(o) + int(b) * bb] for o, b in zip(off, blocks)]
    filters = [(v, int(b), int(ko), int(c)) for v, b, ko, c in zip(views, blocks, key_off, counts)]
    batch = Batch(filters, B, S, k, seed=11)
    return batch, filters, keys, views


def oracle_for(filters, keys, B, S, k, i):
    _, b, ko, c = filters[i]
    geom = oracle.Geometry(num_blocks=b, block_bits=B, word_bits=S, k=k, seed=11)
    ref = oracle.SBF(geom)
    ref.add(keys[ko:ko + c])
    return ref


def queries_for(keys, filters, seed):
    """Half of each run replaced by fresh keys, the other half kept (members)."""
    q = keys.copy()
    fresh = synthkeys.splitmix64(seed, 0, q.size)
    q[1::2] = fresh[1::2]
    return q


@pytest.mark.parametrize("B,S,k", [(256, 32, 8), (512, 64, 16), (128, 32, 4)])
def test_batch_matches_oracle_per_filter(torch, B, S, k):
    from paper_2512_15595_gb300 import (BF_HINT_PREFETCH_L2, BF_HINT_WARP_AGGREGATE, BF_OP_ADD, BF_OP_CONTAINS,
                                        valid_layouts)
    batch, filters, keys, views = make_batch(torch, B, S, k)
    q = queries_for(keys, filters, 55)
    refs = [oracle_for(filters, keys, B, S, k, i) for i in range(len(filters))]
    want = np.zeros(q.size, dtype=np.uint8)
    for (_, b, ko, c), ref in zip(filters, refs):
        want[ko:ko + c] = ref.contains(q[ko:ko + c])
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dq = torch.from_numpy(q.view(np.int64)).cuda()
    it = 0
    for cg, phi in valid_layouts(B, S):
        for kpt in (1, 2, 4):
            for v in views:
                v.zero_()
            # the L2 prefetch hint on every other layout, the warp aggregation on every third
            flags = (BF_HINT_PREFETCH_L2 if it % 2 else 0) | (BF_HINT_WARP_AGGREGATE if it % 3 == 1 else 0)
            it += 1
            batch.set_layout(BF_OP_ADD, cg=cg, phi=phi, kpt=kpt, flags=flags)
            batch.set_layout(BF_OP_CONTAINS, cg=cg, phi=phi, kpt=kpt, flags=flags)
            batch.add(dk)
            out = batch.contains(dq)
            torch.cuda.synchronize()
            for i, (v, ref) in enumerate(zip(views, refs)):
                assert np.array_equal(v.cpu().numpy(), ref.as_bytes()), (i, cg, phi, kpt)
            got = out.cpu().numpy().astype(np.uint8)
            covered = np.zeros(q.size, dtype=bool)
            for _, b, ko, c in filters:
                covered[ko:ko + c] = True
            assert np.array_equal(got[covered], want[covered]), (cg, phi, kpt)
            assert not got[~covered].any()
    batch.close()


def test_batch_prefetch_tiny_and_ragged_filters(torch):
    """The L2 prefetch hint on 64-bit blocks: filters of 1-5 blocks (8-40
    bytes, below one 16-byte prefetch unit or with an 8-byte tail), odd
    block counts and many chunks per filter; bits and answers as the oracle's."""
    from paper_2512_15595_gb300 import BF_HINT_PREFETCH_L2, BF_OP_ADD, BF_OP_CONTAINS, Batch
    B, S, k = 64, 32, 8
    blocks = np.array([1, 2, 3, 5, 1, 4097, 3, 65537, 7, 1], dtype=np.int64)
    counts = np.array([50, 0, 300, 1000, 7, 40_000, 129, 150_001, 1, 128], dtype=np.int64)
    key_off = np.zeros(blocks.size, dtype=np.int64)
    key_off[1:] = np.cumsum(counts)[:-1]
    keys = synthkeys.splitmix64(301, 0, int(counts.sum()))
    q = queries_for(keys, None, 302)
    off, arena_bytes = batches.arena_offsets(blocks, B // 8)
    arena = torch.zeros(arena_bytes, dtype=torch.uint8, device="cuda")
    views = [arena[int(o):int(o) + int(b) * (B // 8)] for o, b in zip(off, blocks)]
    filters = [(v, int(b), int(ko), int(c)) for v, b, ko, c in zip(views, blocks, key_off, counts)]
    batch = Batch(filters, B, S, k, seed=11)
    for op in (BF_OP_ADD, BF_OP_CONTAINS):
        batch.set_layout(op, kpt=2, flags=BF_HINT_PREFETCH_L2)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dq = torch.from_numpy(q.view(np.int64)).cuda()
    batch.add(dk)
    got = batch.contains(dq).cpu().numpy().astype(np.uint8)
    for i, (v, b, ko, c) in enumerate(filters):
        ref = oracle_for(filters, keys, B, S, k, i)
        assert np.array_equal(v.cpu().numpy(), ref.as_bytes()), i
        assert np.array_equal(got[ko:ko + c], ref.contains(q[ko:ko + c])), i
    batch.close()


def test_batch_odd_key_offsets_and_single_filter_equivalence(torch):
    from paper_2512_15595_gb300 import Filter
    B, S, k = 256, 64, 8
    batch, filters, keys, views = make_batch(torch, B, S, k, nfilters=40, total_keys=120_000, seed=9,
                                             odd_offsets=True)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    batch.add(dk)
    torch.cuda.synchronize()
    for v, (_, b, ko, c) in zip(views, filters):
        f = Filter(b, B, S, k, seed=11)
        f.add(dk[ko:ko + c])
        assert torch.equal(f.words, v)
        f.close()
    batch.close()


def test_batch_cuda_graph_replay(torch):
    B, S, k = 256, 32, 8
    batch, filters, keys, views = make_batch(torch, B, S, k, nfilters=64, total_keys=200_000, seed=13)
    q = queries_for(keys, filters, 77)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dq = torch.from_numpy(q.view(np.int64)).cuda()
    out = torch.zeros(q.size, dtype=torch.uint8, device="cuda")
    # eager reference
    batch.add(dk)
    batch.contains(dq, out=out)
    torch.cuda.synchronize()
    ref_words = [v.clone() for v in views]
    ref_out = out.clone()
    for v in views:
        v.zero_()
    out.zero_()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        batch.add(dk, stream=s)
        batch.contains(dq, out=out, stream=s)
    for _ in range(2):
        g.replay()
    torch.cuda.synchronize()
    for v, r in zip(views, ref_words):
        assert torch.equal(v, r)
    assert torch.equal(out, ref_out)
    batch.close()


def test_empty_batch_and_errors(torch):
    from paper_2512_15595_gb300 import Batch, BloomError
    b = Batch([], 256, 32, 8)
    b.add(torch.zeros(1, dtype=torch.int64, device="cuda"))
    b.close()
    buf = torch.zeros(1024, dtype=torch.uint8, device="cuda")
    with pytest.raises(BloomError):
        Batch([(buf[4:36], 1, 0, 10)], 256, 32, 8)  # misaligned bit array
    with pytest.raises(BloomError):
        Batch([(buf, 0, 0, 10)], 256, 32, 8)  # no blocks
    with pytest.raises(BloomError):
        Batch([(buf, 32, 0, 10)], 256, 32, 4)  # k < s


def test_batch_autotune_sweep_keeps_parity(torch):
    """The batched autotuner times every layout, leaves the fastest set, and
    the batch built with it still equals the oracle filter by filter."""
    from paper_2512_15595_gb300 import BF_HINT_PREFETCH_L2, BF_OP_ADD, BF_OP_CONTAINS, autotune, valid_layouts
    B, S, k = 256, 32, 8
    batch, filters, keys, views = make_batch(torch, B, S, k, nfilters=41, total_keys=120_000, seed=9)
    q = queries_for(keys, filters, 56)
    dk = torch.from_numpy(keys.view(np.int64)).cuda()
    dq = torch.from_numpy(q.view(np.int64)).cuda()
    out = torch.zeros(q.size, dtype=torch.uint8, device="cuda")
    res = autotune.sweep_batch(torch, batch, dk, dq, out, kpts=(1, 4), reps=1, flag_sets=(0, BF_HINT_PREFETCH_L2),
                               grids=(0, 7))
    assert res["key"] == "batch_B256_S32_K8"
    assert len(res["rows"]) == 2 * 2 * 2 * 2 * len(valid_layouts(B, S))
    for op, name in ((BF_OP_ADD, "add"), (BF_OP_CONTAINS, "contains")):
        got = batch.layout(op)
        want = res["entry"][name]["layout"]
        assert (got["cg"], got["phi"], got["kpt"], got["flags"], got["grid_ctas"]) == \
            (want["cg"], want["phi"], want["kpt"], want["flags"], want["grid_ctas"])
        assert res["entry"][name]["ms"] == min(r["ms"] for r in res["rows"] if r["op"] == name)
    for v in views:
        v.zero_()
    batch.add(dk)
    got = batch.contains(dq, out=out).cpu().numpy()
    want = np.zeros(q.size, dtype=np.uint8)
    for i, (v, b, ko, c) in enumerate(filters):
        ref = oracle_for(filters, keys, B, S, k, i)
        assert np.array_equal(v.cpu().numpy(), ref.as_bytes()), f"filter {i}"
        want[ko:ko + c] = ref.contains(q[ko:ko + c])
    assert np.array_equal(got, want)
