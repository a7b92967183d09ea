"""The Parquet split-block salt set on the GPU against the oracle.

With salts = 1 (256-bit blocks, S = 32, K = 8) the oracle's bit arrays are
pinned to the ones pyarrow's Parquet writer stores (test_oracle_hash_pins);
here every path of the CUDA library must set the same bits and give the same
answers as that oracle: every compiled layout of the direct kernels, the
slice-partitioned construction and lookup, batches, the construction without
allocation and the lookup server.  A default-salt filter over the same keys
must differ (the salt set is really in use).
"""
import ctypes

import numpy as np
import pytest

import oracle
import synthkeys
from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def torch():
    import torch as t
    from paper_2512_15595_gb300 import build
    build.build()
    return t


def ref_filter(nb, keys, seed=0):
    f = oracle.SBF(oracle.Geometry(num_blocks=nb, block_bits=256, word_bits=32, k=8, seed=seed, salts=1))
    f.add(keys)
    return f


def dev(torch, a):
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).cuda()


def test_every_layout_bit_exact(torch):
    from paper_2512_15595_gb300 import BF_OP_ADD, BF_OP_CONTAINS, Filter, valid_layouts
    nb = 3001
    ins = synthkeys.insert_keys(nb * 25 + 7, seed=31)
    q, _ = synthkeys.mixed_queries(ins.size, 20_000, 20_001, seed_insert=31)
    ref = ref_filter(nb, ins)
    want = ref.contains(q)
    plain = oracle.SBF(oracle.Geometry(num_blocks=nb, block_bits=256, word_bits=32, k=8))
    plain.add(ins)
    assert not np.array_equal(plain.as_bytes(), ref.as_bytes())
    dk, dq = dev(torch, ins), dev(torch, q)
    for cg, phi in valid_layouts(256, 32):
        for kpt in (1, 2, 4):
            f = Filter(nb, 256, 32, 8, 0, salts=1)
            f.set_partition(mode=0)
            f.set_layout(BF_OP_ADD, cg=cg, phi=phi, kpt=kpt)
            f.set_layout(BF_OP_CONTAINS, cg=cg, phi=phi, kpt=kpt)
            f.add(dk)
            got = f.contains(dq).cpu().numpy().astype(np.uint8)
            assert np.array_equal(f.words.cpu().numpy(), ref.as_bytes()), (cg, phi, kpt)
            assert np.array_equal(got, want), (cg, phi, kpt)
            f.close()


def test_slice_partitioned_paths_bit_exact(torch):
    from paper_2512_15595_gb300 import Filter
    nb = (1 << 20) + 77  # 32 MiB + a ragged tail: several 16 MiB slices
    ins = synthkeys.insert_keys(nb * 5, seed=32)
    q, flags = synthkeys.mixed_queries(ins.size, 100_000, 100_003, seed_insert=32)
    ref = ref_filter(nb, ins)
    f = Filter(nb, 256, 32, 8, 0, salts=1)
    f.set_partition(mode=1, slice_log2=18, lookup_mode=1)
    f.add(dev(torch, ins))
    assert f.last_launches() > 1  # the partitioned construction ran
    got = f.contains(dev(torch, q)).cpu().numpy().astype(np.uint8)
    assert f.last_launches() > 1
    assert np.array_equal(f.words.cpu().numpy(), ref.as_bytes())
    assert np.array_equal(got, ref.contains(q))
    assert got[flags == 1].all()


def test_batch_bit_exact(torch):
    from paper_2512_15595_gb300 import Batch
    sizes = [1, 7, 300, 4096, 2]
    counts = [0, 90, 5000, 100_000, 33]
    offs = np.concatenate([[0], np.cumsum(counts)[:-1]])
    keys = synthkeys.splitmix64(33, 0, int(sum(counts)))
    bufs = [torch.zeros(b * 32, dtype=torch.uint8, device="cuda") for b in sizes]
    filters = [(w, b, int(o), c) for w, b, o, c in zip(bufs, sizes, offs, counts)]
    batch = Batch(filters, 256, 32, 8, seed=5, salts=1)
    batch.add(dev(torch, keys))
    out = batch.contains(dev(torch, keys)).cpu().numpy().astype(np.uint8)
    torch.cuda.synchronize()
    for (w, b, o, c) in filters:
        ref = ref_filter(b, keys[o:o + c], seed=5)
        assert np.array_equal(w.cpu().numpy(), ref.as_bytes())
        assert out[o:o + c].all()


def test_noalloc_bit_exact(torch):
    from paper_2512_15595_gb300 import _lib as L
    nb = 1 << 20
    keys = synthkeys.splitmix64(34, 0, 600_000)
    p = L.bf_params(nb, 256, 32, 8, 0, 0, 1, 0)
    words = torch.zeros(nb * 32, dtype=torch.uint8, device="cuda")
    mx = ctypes.c_uint64()
    st = L.lib().bf_add_noalloc(ctypes.byref(p), words.data_ptr(), dev(torch, keys).data_ptr(), keys.size,
                                ctypes.byref(mx), torch.cuda.current_stream().cuda_stream)
    assert st == L.BF_OK, L.bf_last_error()
    torch.cuda.synchronize()
    assert np.array_equal(words.cpu().numpy(), ref_filter(nb, keys).as_bytes())


def test_server_answers(torch):
    from paper_2512_15595_gb300 import Filter, _lib as L
    nb = 4096
    keys = synthkeys.splitmix64(35, 0, 50_000)
    f = Filter(nb, 256, 32, 8, 0, salts=1)
    f.add(dev(torch, keys))
    torch.cuda.synchronize()
    ref = ref_filter(nb, keys)
    srv = L.bf_server_create(L.bf_params(1, 256, 32, 8, 0, 0, 1, 0), [(f.words.data_ptr(), nb)], arena_keys=100_000)
    try:
        q = synthkeys.splitmix64(36, 0, 20_000)
        q[:5000] = keys[:5000]
        hk = torch.from_numpy(q.view(np.int64)).pin_memory()
        ho = torch.zeros(q.size, dtype=torch.uint8).pin_memory()
        t = L.bf_server_submit(srv, 0, hk.data_ptr(), q.size, ho.data_ptr())
        L.bf_server_wait(srv, t, 60.0)
        assert np.array_equal(ho.numpy(), ref.contains(q))
    finally:
        L.bf_server_destroy(srv)
        f.close()
