"""bf_add_noalloc: construction for callers that cannot let a library allocate.

Such callers run their GPU memory through their own allocator (a caching pool
that owns the free memory) or run loops that must not pay for the device
synchronization of cudaMalloc / cudaFree.  The entry point keeps its scratch
in a fixed 16 MiB array inside the library instead.  These tests call it
through the C ABI and check, over two calls in a row on the same bit array,
that it sets exactly the bits the regular bf_add sets, and that a call with
more keys than the array can take is refused before anything runs.

This file is collected last on purpose, so that a failure here cannot stop a
run before the other GPU tests.
"""
import ctypes

import numpy as np
import pytest

import synthkeys
from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


def f_status(L):
    v = ctypes.c_uint32()
    assert L.lib().bf_noalloc_status(ctypes.byref(v)) == L.BF_OK
    return v.value


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2512_15595_gb300 import _lib, build
    build.build()
    return torch, _lib


@pytest.mark.parametrize("num_blocks,B,S,k", [(1 << 21, 256, 32, 8), ((1 << 19) + 333, 512, 64, 16)])
def test_noalloc_matches_bf_add_on_two_calls(env, num_blocks, B, S, k):
    torch, L = env
    p = L.bf_params(num_blocks, B, S, k, 0, 17)
    nbytes = num_blocks * B // 8
    ref = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    got = torch.zeros(nbytes, dtype=torch.uint8, device="cuda")
    h = L.bf_create(p, ref.data_ptr())
    try:
        # the regular path, forced to its partitioned construction
        L.bf_set_partition(h, L.bf_partition(L.BF_PART_ON, 24, 1 << 32, 0, 26, L.BF_PART_AUTO, 1 << 28))
        stream = torch.cuda.current_stream().cuda_stream
        limit = ctypes.c_uint64()
        for call, (seed, n) in enumerate([(101, 1_000_003), (102, 777_777)]):
            keys = torch.from_numpy(synthkeys.splitmix64(seed, 0, n).view(np.int64)).cuda()
            L.bf_add(h, keys.data_ptr(), n, stream)
            rc = L.lib().bf_add_noalloc(ctypes.byref(p), got.data_ptr(), keys.data_ptr(), n,
                                        ctypes.byref(limit), stream)
            assert rc == L.BF_OK, (call, rc)
            assert limit.value >= n
            torch.cuda.synchronize()
            assert torch.equal(got, ref), f"bit arrays differ after call {call + 1}"
            assert f_status(L) == 0
        assert int(got.ne(0).sum().item()) > 0
    finally:
        L.bf_destroy(h)


def test_noalloc_rejects_too_many_keys(env):
    torch, L = env
    p = L.bf_params(1 << 20, 256, 32, 8, 0, 0)
    words = torch.zeros((1 << 20) * 32, dtype=torch.uint8, device="cuda")
    limit = ctypes.c_uint64()
    keys = torch.zeros(8, dtype=torch.int64, device="cuda")
    rc = L.lib().bf_add_noalloc(ctypes.byref(p), words.data_ptr(), keys.data_ptr(), 1 << 40,
                                ctypes.byref(limit), None)
    assert rc == L.BF_EINVAL
    assert 1_000_000 < limit.value < (16 << 20) // 8
    torch.cuda.synchronize()
    assert not words.any().item()  # nothing ran


@pytest.mark.parametrize("num_blocks", [1 << 29, 1 << 15])
def test_noalloc_at_its_limit_matches_the_oracle(env, num_blocks):
    """The documented extremes, against the oracle: a 16 GiB filter of
    256-bit blocks (1024 slices of 16 MiB, where the slice buffers are
    smallest and overflow to the direct path is likeliest) and a 1 MiB
    filter of one slice, each with two calls in a row of exactly *max_keys
    keys.  The 16 GiB array is compared block by block: the oracle gives the
    blocks the keys touch and their words, and every other block must be
    zero."""
    import oracle
    torch, L = env
    geom = oracle.Geometry(num_blocks=num_blocks, block_bits=256, word_bits=32, k=8, seed=0)
    p = L.bf_params(num_blocks, 256, 32, 8, 0, 0)
    limit = ctypes.c_uint64()
    words = torch.zeros(num_blocks * 32, dtype=torch.uint8, device="cuda")
    probe = torch.zeros(8, dtype=torch.int64, device="cuda")
    rc = L.lib().bf_add_noalloc(ctypes.byref(p), words.data_ptr(), probe.data_ptr(), 1 << 40,
                                ctypes.byref(limit), None)
    assert rc == L.BF_EINVAL and limit.value > 1_000_000
    n = limit.value
    stream = torch.cuda.current_stream().cuda_stream
    host = []
    for seed in (201, 202):
        keys = synthkeys.splitmix64(seed, 0, n)
        host.append(keys)
        dk = torch.from_numpy(keys.view(np.int64)).cuda()
        rc = L.lib().bf_add_noalloc(ctypes.byref(p), words.data_ptr(), dk.data_ptr(), n, None, stream)
        assert rc == L.BF_OK
        torch.cuda.synchronize()
        del dk
    assert f_status(L) == 0
    blocks, want = oracle.add_sparse(geom, np.concatenate(host))
    w = words.view(torch.int64).view(-1, 4)
    nz = (w != 0).any(dim=1).nonzero().squeeze(1)
    assert np.array_equal(nz.cpu().numpy().astype(np.uint64), blocks), "touched blocks differ from the oracle's"
    got = w[nz].cpu().numpy().view(np.uint32).reshape(-1, 8)
    assert np.array_equal(got, want), "block contents differ from the oracle's"
