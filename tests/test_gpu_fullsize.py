"""The 4 GiB workload at full size, in the launch configuration bench.py
times (tuned layouts, slice-partitioned construction of 3,435,973,836 keys,
slice-partitioned lookup of 10^9 queries in passes of 2^29), against the
oracle on sampled outputs: the bit array of five 4096-block ranges --
the first and the last blocks, two ranges across the boundary between two
record-insert windows (the 16th and the 48th window boundary) and one
across a slice boundary inside a window (the 32nd window's first slice
boundary), slice and window sizes taken from the tuned setting -- recomputed by the
oracle from every insert key, and the answer of every query whose block
lies in those ranges (about 150,000 of them); plus the property that holds
at any size: every member query is found.

The oracle's share runs in a spawn process pool over the host's cores
(spawned workers start fresh interpreters: none inherits a CUDA context).
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle
import synthkeys
from conftest import gpu_available

pytestmark = [pytest.mark.gpu, pytest.mark.slow,
              pytest.mark.skipif(not gpu_available(), reason="needs a CUDA GPU")]

B, S, K = 256, 32, 8
NBYTES = 4 << 30
NBLOCKS = NBYTES // (B // 8)
N_INSERT = NBYTES * 8 // 10
N_LOOKUP = 10**9
RATIO_DEN = 10
SPAN = 4096
CHUNK = 1 << 23


def tuned_slice_window():
    """Blocks per slice and per record-insert window of the tuned setting."""
    from paper_2512_15595_gb300 import autotune
    part = autotune.tuned_layout(B, S, K, "hbm", 0)["partition"]
    return (1 << part["slice_log2"]) // (B // 8), (1 << part["window_log2"]) // (B // 8)


def test_4gib_workload_sampled_parity():
    import torch
    from paper_2512_15595_gb300 import Filter, autotune, build
    import fullsize_oracle as FO

    geom_kw = dict(num_blocks=NBLOCKS, block_bits=B, word_bits=S, k=K, seed=0)
    oracle.build()  # compiled once here, before the pool's workers load it
    SLICE, WINDOW = tuned_slice_window()
    assert WINDOW > SLICE and NBLOCKS // WINDOW >= 64
    half = SPAN // 2
    ranges = [(0, SPAN), (WINDOW * 16 - half, WINDOW * 16 + half),
              (WINDOW * 32 + SLICE - half, WINDOW * 32 + SLICE + half),
              (WINDOW * 48 - half, WINDOW * 48 + half), (NBLOCKS - SPAN, NBLOCKS)]
    ctx = mp.get_context("spawn")
    workers = max(1, min(32, os.cpu_count() or 1))
    with ctx.Pool(workers) as pool:
        # oracle: the two block ranges' bits from every insert key
        add_jobs = [(geom_kw, ranges, lo, min(N_INSERT, lo + CHUNK)) for lo in range(0, N_INSERT, CHUNK)]
        add_async = pool.map_async(FO.add_ranges, add_jobs, chunksize=1)

        # GPU: the bench's step with its tuned layouts
        build.build()
        dev = torch.device("cuda", 0)
        ins = synthkeys.splitmix64_torch(synthkeys.SEED_INSERT, 0, N_INSERT, dev)
        qd = torch.empty(N_LOOKUP, dtype=torch.int64, device=dev)
        flags = torch.empty(N_LOOKUP, dtype=torch.uint8, device=dev)
        synthkeys.stream_queries_torch(N_LOOKUP, N_INSERT, dev, ratio_den=RATIO_DEN, out=qd, member_flags=flags)
        f = Filter(NBLOCKS, B, S, K, 0)
        autotune.apply_tuned(f, "hbm")
        f.add(ins)
        launches_add = f.last_launches()
        out = torch.empty(N_LOOKUP, dtype=torch.uint8, device=dev)
        f.contains(qd, out=out)
        launches_con = f.last_launches()
        torch.cuda.synchronize()
        assert f.device_status() == 0  # no index check failed in the partitioned kernels
        assert launches_add > 1 and launches_con > 1  # the slice-partitioned paths ran
        members = flags == 1
        assert int(members.sum().item()) > 0
        assert bool((out[members] == 1).all().item()), "a member query was not found"
        bb = B // 8
        got_slices = [f.words[a * bb:b * bb].cpu().numpy() for a, b in ranges]
        got_out = out.cpu().numpy()
        f.close()
        del ins, qd, flags, out
        torch.cuda.empty_cache()

        # oracle slices: OR of every chunk's contribution
        parts = add_async.get()
        want = [np.bitwise_or.reduce(np.stack([p[i] for p in parts]), axis=0) for i in range(len(ranges))]
        for (a, b), g, w in zip(ranges, got_slices, want):
            assert np.array_equal(g, w.view(np.uint8)), f"bit array differs in blocks [{a}, {b})"

        # oracle answers of every query that lands in the ranges
        look_jobs = [(geom_kw, ranges, want, lo, min(N_LOOKUP, lo + CHUNK), N_INSERT, RATIO_DEN)
                     for lo in range(0, N_LOOKUP, CHUNK)]
        res = pool.map(FO.lookup_ranges, look_jobs, chunksize=1)
    idx = np.concatenate([r[0] for r in res])
    ans = np.concatenate([r[1] for r in res])
    expect = SPAN * len(ranges) / NBLOCKS * N_LOOKUP
    assert 0.9 * expect < idx.size < 1.1 * expect, idx.size
    mism = np.nonzero(got_out[idx] != ans)[0]
    assert mism.size == 0, f"{mism.size} sampled answers differ, e.g. query {idx[mism[0]]}"
