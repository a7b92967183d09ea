"""The lookup server: requests across filters, admitted into a small device
arena (so the ring wraps and requests wait for room), batched per launch;
every request's answers must equal the oracle's for its filter."""
import numpy as np
import pytest

import oracle
import synthkeys
from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]


@pytest.fixture(scope="module")
def env():
    import torch
    from paper_2512_15595_gb300 import Filter, _lib, build
    build.build()
    return torch, Filter, _lib


def request_buffers(torch, q, kind):
    """Host key / result buffers of one request: 0 pinned, 1 pageable (the
    kernels address both in place: staging kernels), 2 pinned keys at an
    address 4 bytes off 8-byte alignment (the copy engine stages the whole
    launch).  Returns (key pointer, result array, objects to keep alive)."""
    n = q.size
    if kind == 1:
        keys, out = q.copy(), np.zeros(max(n, 1), dtype=np.uint8)
        return keys.ctypes.data, out, (keys,)
    out_t = torch.zeros(max(n, 1), dtype=torch.uint8).pin_memory()
    if kind == 2:
        raw = torch.empty(8 * n + 16, dtype=torch.uint8).pin_memory()
        base = (-raw.data_ptr()) % 8 + 4
        np.frombuffer(raw.numpy(), dtype=np.uint64, count=n, offset=base)[:] = q
        return raw.data_ptr() + base, out_t.numpy(), (raw, out_t)
    keys_t = torch.from_numpy(q.view(np.int64)).pin_memory()
    return keys_t.data_ptr(), out_t.numpy(), (keys_t, out_t)


def test_server_answers_match_oracle(env):
    """Requests of pinned, pageable and misaligned host buffers (staging
    kernels or copy-engine copies per launch), empty requests, ring wraps."""
    torch, Filter, L = env
    B, S, k = 256, 32, 8
    sizes = [1000, 333, 4097, 64, 2500]
    filters, refs = [], []
    for i, nb in enumerate(sizes):
        keys = synthkeys.splitmix64(200 + i, 0, nb * 20)
        f = Filter(nb, B, S, k, seed=21)
        f.add(torch.from_numpy(keys.view(np.int64)).cuda())
        ref = oracle.SBF(oracle.Geometry(num_blocks=nb, block_bits=B, word_bits=S, k=k, seed=21))
        ref.add(keys)
        filters.append(f)
        refs.append(ref)
    torch.cuda.synchronize()
    srv = L.bf_server_create(L.bf_params(1, B, S, k, 0, 21), [(f.words.data_ptr(), nb) for f, nb in zip(filters, sizes)],
                             arena_keys=50_000, max_requests_per_launch=7)
    try:
        rng = np.random.default_rng(3)
        reqs = []
        for r in range(300):
            fi = int(rng.integers(0, len(sizes)))
            n = int(rng.choice([0, 1, 31, int(rng.integers(1, 20_000)), 49_999]))
            q = synthkeys.splitmix64(1000 + r, 0, n)
            if n:
                own = synthkeys.splitmix64(200 + fi, 0, sizes[fi] * 20)
                q[::3] = own[rng.integers(0, own.size, size=q[::3].size)]
            kind = 2 if r % 23 == 5 else r % 2  # a misaligned request now and then
            kp, ho, keep = request_buffers(torch, q, kind)
            t = L.bf_server_submit(srv, fi, kp if n else 0, n, ho.ctypes.data if n else 0)
            reqs.append((t, fi, q, keep, ho, n))
        for t, fi, q, keep, ho, n in reqs:
            lat = L.bf_server_wait(srv, t, 60.0)
            assert lat >= 0
            if n:
                assert np.array_equal(ho[:n], refs[fi].contains(q)), (t, fi, n)
        st = L.bf_server_get_stats(srv)
        assert st["requests"] == 300 and st["keys"] == sum(r[5] for r in reqs)
        assert st["launches"] >= 300 // 7
        assert st["p50_s"] <= st["p99_s"] <= st["max_s"]
        assert st["stage_in_s"] > 0 and st["lookup_s"] > 0 and st["stage_out_s"] > 0
    finally:
        L.bf_server_destroy(srv)
        for f in filters:
            f.close()


def test_server_errors_and_poisson(env):
    torch, Filter, L = env
    f = Filter(4096, 256, 32, 8)
    f.add(torch.from_numpy(synthkeys.insert_keys(40_000).view(np.int64)).cuda())
    srv = L.bf_server_create(L.bf_params(1, 256, 32, 8, 0, 0), [(f.words.data_ptr(), 4096)], arena_keys=100_000)
    try:
        buf = torch.zeros(8, dtype=torch.int64).pin_memory()
        out = torch.zeros(8, dtype=torch.uint8).pin_memory()
        with pytest.raises(L.BloomError):
            L.bf_server_submit(srv, 1, buf.data_ptr(), 8, out.data_ptr())  # no filter 1
        with pytest.raises(L.BloomError):
            L.bf_server_submit(srv, 0, buf.data_ptr(), 100_001, out.data_ptr())  # larger than the arena
        with pytest.raises(L.BloomError):
            L.bf_server_wait(srv, 12345, 0.1)  # unknown ticket
        pool = torch.from_numpy(synthkeys.splitmix64(5, 0, 1 << 20).view(np.int64)).pin_memory()
        pout = torch.zeros(1 << 20, dtype=torch.uint8).pin_memory()
        st = L.bf_server_run_poisson(srv, 2000.0, 0.3, 1, 5000, pool.data_ptr(), pool.numel(), pout.data_ptr(), 7)
        assert st["requests"] > 300 and st["keys"] > 0
        assert 0 < st["p50_s"] <= st["p99_s"] <= st["max_s"] < 5.0
        # the pool's answers are the filter's answers (every request used filter 0)
        want = f.contains(pool.cuda()).cpu().numpy().astype(np.uint8)
        touched = pout.numpy() != 0
        assert np.array_equal(pout.numpy()[touched], want[touched])
    finally:
        L.bf_server_destroy(srv)
        f.close()
