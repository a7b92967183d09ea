#!/usr/bin/env python
"""Benchmark of bulk construction + bulk lookup of the sectorized blocked
Bloom filter on GB300, measured against the random-access bound.

One step = construction of the whole insert set + lookup of the whole query
set (every row of the hot path: key load, XXH64, block selection, pattern,
atomic OR / wide-load test, result store).  The default workload is the
HBM-resident filter of the "filter at scale" configuration:

    4 GiB filter: 2^27 blocks x 256 bits, S = 32-bit words, K = 8, seed 0;
    insert 3,435,973,836 keys (10 bits/key; SplitMix64 stream 1);
    look up 10^9 keys, 10% members (counter-based query stream).

Inputs are generated on the device before timing (inputs larger than L2, so
no flush is needed).  Prints one JSON line (rank 0).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload 4GiB|32MiB|1MiB] [--sweep] [--no-e2e] [--no-cpu-baseline]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "4GiB": dict(nbytes=4 << 30, block_bits=256, word_bits=32, k=8, n_lookup=10**9, member_den=10,
                 desc="4 GiB HBM-resident SBF, 2^27 x 256-bit blocks, S=32, K=8; insert 10 bits/key "
                      "(3,435,973,836 keys), look up 1e9 keys at 10% members"),
    "32MiB": dict(nbytes=32 << 20, block_bits=256, word_bits=32, k=8, n_lookup=10**9, member_den=10,
                  desc="32 MiB L2-resident SBF, 2^20 x 256-bit blocks, S=32, K=8; insert 10 bits/key "
                       "(26,843,545 keys), look up 1e9 keys at 10% members"),
    "256MiB": dict(nbytes=256 << 20, block_bits=256, word_bits=32, k=8, n_lookup=10**8, member_den=10,
                   desc="256 MiB HBM-resident SBF (2x L2), 2^23 x 256-bit blocks, S=32, K=8; insert 10 bits/key "
                        "(214,748,364 keys), look up 1e8 keys at 10% members (profiling size)"),
    "32MiB-S64k16": dict(nbytes=32 << 20, block_bits=256, word_bits=64, k=16, n_insert=11_626_502, n_lookup=10**9,
                         member_den=10,
                         desc="the paper's own configuration, L2-resident: 32 MiB SBF, 2^20 x 256-bit blocks, S=64, "
                              "K=16; insert the Eq. (1)-optimal load for k=16 (c = 16/ln 2 = 23.08 bits/key: "
                              "11,626,502 keys), look up 1e9 keys at 10% members"),
    "1MiB": dict(nbytes=1 << 20, block_bits=256, word_bits=32, k=8, n_insert=10**6, n_lookup=10**6,
                 member_den=2,
                 desc="1 MiB SBF, 2^15 x 256-bit blocks, S=32, K=8; insert 1e6 keys, look up 1e6 keys"),
}
METRIC = "G lookups/s & G inserts/s vs measured random-access bound; FPR at bits/key"


def wl_sizes(w):
    b = w["nbytes"] * 8 // w["block_bits"]
    n_ins = w.get("n_insert", w["nbytes"] * 8 // 10)
    return b, n_ins, w["n_lookup"]


# ---------------------------------------------------------------------------
# distributed plumbing (one process per GPU; replicas, no data-path collective)
# ---------------------------------------------------------------------------
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def max_over_ranks(value: float, world: int, device=None) -> float:
    """Max of a per-rank float over all ranks (a timing reduction, not data)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world: int, keys_per_step: int, steps: int, total_ms: float) -> float:
    """G keys/s of the whole job: every rank processes keys_per_step per step;
    total_ms is the slowest rank's time for all timed steps."""
    return world * keys_per_step * steps / (total_ms * 1e-3) / 1e9


def barrier(world: int):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int, uuid: str | None):
        self.sel = str(device_index)
        if uuid:
            try:
                listing = subprocess.run(["nvidia-smi", "-L"], capture_output=True, text=True, timeout=10).stdout
                if uuid in listing:
                    self.sel = uuid
            except Exception:
                pass
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", self.sel, f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "50"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out = ""
        sm, smax, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax = max(smax, float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        loaded = [x for x in sm if x > 0.5 * max(sm)] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# CPU oracle timing (bounded sample; rank 0 only)
# ---------------------------------------------------------------------------
def cpu_oracle_rate(w, budget_s: float):
    """Oracle insert+lookup throughput on a bounded sample of the workload.

    Inserts the first keys of the insert stream into a full-size host filter
    and looks up the first queries of the query stream, in chunks, until the
    budget is spent (about half the budget per operation).
    """
    import numpy as np
    import oracle
    import synthkeys
    b, n_ins, n_q = wl_sizes(w)
    geom = oracle.Geometry(num_blocks=b, block_bits=w["block_bits"], word_bits=w["word_bits"], k=w["k"], seed=0,
                           salts=w.get("salts", 0))
    f = oracle.SBF(geom)
    chunk = 1 << 20
    done_i, t_i = 0, 0.0
    while t_i < budget_s / 2 and done_i < n_ins:
        c = min(chunk, n_ins - done_i)
        keys = synthkeys.splitmix64(synthkeys.SEED_INSERT, done_i, c)
        t0 = time.perf_counter()
        f.add(keys)
        t_i += time.perf_counter() - t0
        done_i += c
    done_q, t_q = 0, 0.0
    mixed = synthkeys.mixed_queries(n_ins, n_q // 2, n_q - n_q // 2)[0] if w["member_den"] == 2 else None
    while t_q < budget_s / 2 and done_q < n_q:
        c = min(chunk, n_q - done_q)
        if mixed is not None:
            q = mixed[done_q:done_q + c]
        else:
            q, _ = synthkeys.stream_queries(done_q, c, n_ins, w["member_den"])
        t0 = time.perf_counter()
        f.contains(q)
        t_q += time.perf_counter() - t0
        done_q += c
    return {"insert_keys": done_i, "insert_s": t_i, "lookup_keys": done_q, "lookup_s": t_q,
            "gkeys_s": (done_i + done_q) / (t_i + t_q) / 1e9,
            "insert_gkeys_s": done_i / t_i / 1e9, "lookup_gkeys_s": done_q / t_q / 1e9}


def _oracle_range_worker(job):
    """One process of the all-core oracle timing: the unchanged oracle over
    one block range of the full-size filter.  Every worker hashes the whole
    sample (the oracle's block index) and inserts / looks up only the keys
    whose block is in its range, so the ranges' bits are exactly the
    oracle's; returns (insert seconds, lookup seconds)."""
    import numpy as np
    import oracle
    import synthkeys
    geom_kw, lo, hi, n_ins, n_q, n_insert_total, member_den, chunk = job
    geom = oracle.Geometry(**geom_kw)
    words = np.zeros((hi - lo) * geom.s, dtype=geom.word_dtype)
    ti = tq = 0.0  # oracle time only (the input generation is not timed)
    for c0 in range(0, n_ins, chunk):
        keys = synthkeys.splitmix64(synthkeys.SEED_INSERT, c0, min(chunk, n_ins - c0))
        t0 = time.perf_counter()
        j = oracle.block_indices(keys, geom.num_blocks, geom.seed)
        oracle.add_block_range(geom, lo, hi, keys[(j >= lo) & (j < hi)], words)
        ti += time.perf_counter() - t0
    for c0 in range(0, n_q, chunk):
        q, _ = synthkeys.stream_queries(c0, min(chunk, n_q - c0), n_insert_total, member_den)
        t0 = time.perf_counter()
        j = oracle.block_indices(q, geom.num_blocks, geom.seed)
        oracle.contains_block_range(geom, words, lo, hi, q[(j >= lo) & (j < hi)])
        tq += time.perf_counter() - t0
    return ti, tq


def cpu_oracle_rate_all_cores(w, n_sample: int = 1 << 24):
    """The oracle on every host core: a spawn pool with one worker per core,
    each owning one block range of the full-size filter (the oracle's
    construction ORs without atomics, so workers split the filter, not the
    keys).  Throughput = sample keys / the slowest worker's time."""
    import multiprocessing as mp
    b, n_ins, n_q = wl_sizes(w)
    cores = os.cpu_count() or 1
    if w["member_den"] == 2:
        return None  # the small workload's mixed query set is built on one host only
    geom_kw = dict(num_blocks=b, block_bits=w["block_bits"], word_bits=w["word_bits"], k=w["k"], seed=0,
                   salts=w.get("salts", 0))
    ni, nq = min(n_sample, n_ins), min(n_sample, n_q)
    step = -(-b // cores)
    jobs = [(geom_kw, lo, min(b, lo + step), ni, nq, n_ins, w["member_den"], 1 << 22) for lo in range(0, b, step)]
    import oracle
    oracle.build()
    with mp.get_context("spawn").Pool(len(jobs)) as pool:
        res = pool.map(_oracle_range_worker, jobs, chunksize=1)
    ti = max(r[0] for r in res)
    tq = max(r[1] for r in res)
    return {"value": (ni + nq) / (ti + tq) / 1e9, "unit": "G keys/s", "cores": len(jobs),
            "insert_gkeys_s": ni / ti / 1e9, "lookup_gkeys_s": nq / tq / 1e9,
            "sample": f"first {ni:,} inserts and first {nq:,} queries, the full-size filter split into "
                      f"{len(jobs)} block ranges, one spawn worker per range (every worker hashes the whole sample)"}


def run_reference(args, w, wname):
    """The reference arm: the CPU oracle as it stands, on the host cores."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    steps, warm = args.steps, args.warmup
    per_step = max(1.0, min(20.0, 150.0 / max(1, steps + warm)))
    for _ in range(warm):
        cpu_oracle_rate(w, per_step * 0.25)
    vals = []
    t0 = time.perf_counter()
    for _ in range(steps):
        vals.append(cpu_oracle_rate(w, per_step))
    wall = time.perf_counter() - t0
    v = statistics.median(x["gkeys_s"] for x in vals)
    r = vals[len(vals) // 2]
    sample = (f"per step: first {r['insert_keys']:,} insert keys into the full-size host filter, then first "
              f"{r['lookup_keys']:,} queries of the query stream (~{per_step:.0f} s of single-thread CPU work)")
    line = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": "G keys/s", "n_gpus": world,
        "steps": steps, "warmup": warm, "ms_per_step": wall / steps * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64/u32 integer", "data": "synthetic",
        "config": {"workload": wname, "desc": w["desc"]},
        "cpu_baseline": {"value": v, "unit": "G keys/s", "cores": 1, "kind": "oracle", "sample": sample,
                         "insert_gkeys_s": r["insert_gkeys_s"], "lookup_gkeys_s": r["lookup_gkeys_s"]},
        "e2e": {"value": v, "unit": "G keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm
# ---------------------------------------------------------------------------
KERNEL_SOURCES = ("sbf_kernels.cuh", "sbf_device.cuh", "salts.cuh", "sbf_partition.cuh", "sbf_expand.cu",
                  "registry.h")


def kernel_source_hash(sources=KERNEL_SOURCES) -> str:
    h = hashlib.sha256()
    for f in sources:
        with open(os.path.join(ROOT, "paper_2512_15595_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(op: str, wname: str, sources=KERNEL_SOURCES):
    """DRAM bytes of one call of `op` from the committed ncu summary, if the
    kernel sources have not changed since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        t = json.load(f)
    e = t.get(f"{op}/{wname}")
    if not e or e.get("kernel_source_hash") != kernel_source_hash(sources):
        return None
    return e.get("dram_bytes_per_launch")


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def gen_inputs(torch, w, device):
    import synthkeys
    b, n_ins, n_q = wl_sizes(w)
    ins = torch.empty(n_ins, dtype=torch.int64, device=device)
    synthkeys.splitmix64_torch(synthkeys.SEED_INSERT, 0, n_ins, device, out=ins)
    flags = torch.empty(n_q, dtype=torch.uint8, device=device)
    if w["member_den"] == 2:
        import numpy as np
        q, fl = synthkeys.mixed_queries(n_ins, n_q // 2, n_q - n_q // 2)
        qd = torch.from_numpy(q.view(np.int64)).to(device)
        flags.copy_(torch.from_numpy(fl))
    else:
        qd = torch.empty(n_q, dtype=torch.int64, device=device)
        synthkeys.stream_queries_torch(n_q, n_ins, device, ratio_den=w["member_den"], out=qd, member_flags=flags)
    torch.cuda.synchronize()
    return ins, qd, flags


def gups_bounds(torch, w, ins, q, device, reps=3, window_bytes=None):
    """Random-access bound on the filter's footprint with the same key
    streams; with window_bytes, also the full-sector OR rate (the record-insert
    kernel's traffic) on a table of one record-insert window."""
    from paper_2512_15595_gb300 import BF_GUPS_LOAD, BF_GUPS_RED_OR, BF_GUPS_RED_OR_SECTOR, _lib, bf_layout
    unit = max(32, w["block_bits"] // 8)
    table = torch.zeros(w["nbytes"], dtype=torch.uint8, device=device)
    gout = torch.empty(q.numel(), dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream()
    best = {}
    runs = [(BF_GUPS_LOAD, "load", q, w["nbytes"]), (BF_GUPS_RED_OR, "red_or", ins, w["nbytes"])]
    if window_bytes:
        runs.append((BF_GUPS_RED_OR_SECTOR, "red_sector_window", ins, min(window_bytes, w["nbytes"])))
    for mode, name, keys, tbytes in runs:
        for kpt in (1, 2, 4):
            lay = bf_layout(0, 0, kpt, 256, 0, 0)
            ts = []
            for i in range(reps + 1):
                s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s.record(stream)
                _lib.bf_gups(mode, table.data_ptr(), tbytes, unit, keys.data_ptr(), keys.numel(),
                             gout.data_ptr() if mode == BF_GUPS_LOAD else None, lay, stream)
                e.record(stream)
                e.synchronize()
                if i:
                    ts.append(s.elapsed_time(e))
            g = keys.numel() / (min(ts) * 1e-3) / 1e9
            if name not in best or g > best[name]["gkeys_s"]:
                best[name] = {"gkeys_s": g, "kpt": kpt, "unit_bytes": unit, "table_bytes": tbytes}
    del table, gout
    torch.cuda.empty_cache()
    return best


def popcount_fpr(torch, words, w):
    """E[FPR | this bit array] for ideal query hashing: mean over blocks of
    prod_w (popcount_w / S)^k' (computed on the device from the array)."""
    lut = torch.tensor([bin(i).count("1") for i in range(256)], dtype=torch.float32, device=words.device)
    s = w["block_bits"] // w["word_bits"]
    kp = w["k"] // s
    bpw = w["word_bits"] // 8
    block_bytes = w["block_bits"] // 8
    nblocks = words.numel() // block_bytes
    total = 0.0
    step = 1 << 22
    for lo in range(0, nblocks, step):
        hi = min(nblocks, lo + step)
        blk = words[lo * block_bytes:hi * block_bytes].view(hi - lo, s, bpw).long()
        pc = lut[blk].sum(-1)
        total += float(torch.prod((pc / w["word_bits"]) ** kp, dim=-1).double().sum().item())
    return total / nblocks


PHASE_KERNELS = {
    "add_direct": "sbf_add_kernel", "contains_direct": "sbf_contains_kernel",
    "partition_add": "sbf_partition_kernel (construction)", "record_insert": "sbf_add_records_kernel",
    "partition_lookup": "sbf_partition_kernel (lookup)", "record_probe": "sbf_probe_records_kernel",
    "bitmap_expand": "bitmap_expand_kernel", "host_stage": "host_stage16_kernel (host keys to device staging)",
}


def phase_bytes(phase, w, n_ins, n_q, part):
    """Algorithmic DRAM bytes of one call's launches of one kernel: 8-byte
    keys and records, 4-byte query indexes, 1-byte results, and the filter's
    blocks -- for the direct kernels one random sector access per key (read
    and written back for construction), for the windowed kernels every
    window's blocks read (and written back) once per pass."""
    fb = w["nbytes"]
    sectors = max(1, w["block_bits"] // 256)
    add_passes = -(-n_ins // max(1, part["chunk_keys"]))
    look_passes = -(-n_q // max(1, part["lookup_chunk_keys"]))
    return {
        "add_direct": n_ins * (8 + 64 * sectors),
        "contains_direct": n_q * (8 + 32 * sectors + 1),
        "partition_add": n_ins * (8 + 8),
        "record_insert": n_ins * 8 + 2 * fb * add_passes,
        "partition_lookup": n_q * (8 + 12),
        "record_probe": n_q * 12 + fb * look_passes,
        "bitmap_expand": n_q // 8 + n_q,
        "host_stage": 8 * (n_ins + n_q),  # host keys over the link into device staging slots
    }[phase]


def run_ours(args, w, wname):
    import torch
    world, rank, local = dist_env()
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=device)
    from paper_2512_15595_gb300 import Filter, _lib, autotune
    b, n_ins, n_q = wl_sizes(w)
    props = torch.cuda.get_device_properties(device)
    regime = autotune.regime_of(w["nbytes"], props.L2_cache_size)

    ins, qd, flags = gen_inputs(torch, w, device)
    if args.key_runs > 1:
        # an insert stream of runs of equal keys (same length; every run's key
        # is an insert key, so the member queries stay members)
        ins = ins[: -(-n_ins // args.key_runs)].repeat_interleave(args.key_runs)[:n_ins].contiguous()
        torch.cuda.synchronize()
    f = Filter(b, w["block_bits"], w["word_bits"], w["k"], 0, device=device, salts=w.get("salts", 0))
    layouts = autotune.apply_tuned(f, regime)
    if args.add_flags:
        from paper_2512_15595_gb300 import BF_HINT_WARP_AGGREGATE, BF_OP_ADD
        lay = f.layout(BF_OP_ADD)
        lay["flags"] |= {"aggregate": BF_HINT_WARP_AGGREGATE}[args.add_flags]
        f.set_layout(BF_OP_ADD, **lay)
        layouts = {"add": f.layout(BF_OP_ADD), "contains": f.layout(1)}
    out = torch.empty(n_q, dtype=torch.uint8, device=device)
    stream = torch.cuda.current_stream()

    part0 = f.partition()
    bounds = (gups_bounds(torch, w, ins, qd, device,
                          window_bytes=(1 << part0["window_log2"]) if regime == "hbm" else None)
              if not args.no_gups else None)
    if args.l2_persist > 0:
        f.set_l2_persist(args.l2_persist)

    launches = []
    launches_add, launches_con = [], []

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        f.add(ins)
        launches_add.append(f.last_launches())
        if ev:
            ev[1].record(stream)
        f.contains(qd, out=out)
        launches_con.append(f.last_launches())
        launches.append(launches_add[-1] + launches_con[-1])
        if ev:
            ev[2].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches.clear()
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    sampler = ClockSampler(local, getattr(props, "uuid", None) and f"GPU-{props.uuid}")
    barrier(world)
    torch.cuda.synchronize()
    sampler.start()
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    f.set_timing(True)  # per-kernel CUDA events on the launching streams, read after the region
    t_start.record(stream)
    for i in range(args.steps):
        step(evs[i])
    t_end.record(stream)
    torch.cuda.synchronize()
    barrier(world)
    clocks = sampler.stop()
    phase_tm = f.timing()
    f.set_timing(False)
    if args.l2_persist > 0:
        f.set_l2_persist(0.0)
    local_ms = t_start.elapsed_time(t_end)
    total_ms = max_over_ranks(local_ms, world, device)
    add_ms = statistics.median(e[0].elapsed_time(e[1]) for e in evs)
    con_ms = statistics.median(e[1].elapsed_time(e[2]) for e in evs)
    keys_per_step = n_ins + n_q
    value = whole_job_rate(world, keys_per_step, args.steps, total_ms)
    ins_g = n_ins / (add_ms * 1e-3) / 1e9
    look_g = n_q / (con_ms * 1e-3) / 1e9

    # accuracy of the constructed filter: FPR of the fresh queries at 10 bits/key
    fresh = flags == 0
    n_fresh = int(fresh.sum().item())
    measured_fpr = float(out[fresh].float().sum().item()) / max(1, n_fresh)
    # member queries are insert-stream keys; with --key-runs the insert set is
    # smaller, so the no-false-negative count only applies to the plain stream
    missed = int((out[flags == 1] == 0).sum().item()) if args.key_runs == 1 else None
    realized_fpr = popcount_fpr(torch, f.words, w)

    # per-kernel device time of the timed steps (events around each group of
    # launches, on the stream it runs on)
    peak, peak_kind = peaks()
    part = f.partition()
    steps = args.steps
    kern_ms = sum(v["ms"] for v in phase_tm.values()) or 1.0
    kernels = {}
    for ph, v in phase_tm.items():
        nb = phase_bytes(ph, w, n_ins, n_q, part)
        lpc = v["launches"] / steps
        avg = v["ms"] / max(1, v["launches"])
        kernels[ph] = {"kernel": PHASE_KERNELS[ph], "ms_per_step": v["ms"] / steps, "launches_per_step": lpc,
                       "share": v["ms"] / kern_ms, "avg_launch_ms": avg,
                       "algorithmic_bytes_per_launch": nb / lpc,
                       "achieved_gbs": nb / lpc / (avg * 1e-3) / 1e9}
    # roofline of the dominant kernel (largest share of the step)
    dom = max(kernels, key=lambda k: kernels[k]["ms_per_step"])
    kd = kernels[dom]
    roof = {"bound": "hbm", "kernel": kd["kernel"], "achieved": kd["achieved_gbs"], "peak": peak, "unit": "GB/s",
            "frac": kd["achieved_gbs"] / peak,
            "traffic": measured_traffic(dom, wname), "per": "one launch",
            "algorithmic_bytes_per_launch": kd["algorithmic_bytes_per_launch"], "avg_launch_ms": kd["avg_launch_ms"],
            "launches_per_step": kd["launches_per_step"], "share_of_kernel_time": kd["share"],
            "peak_source": f"{peak_kind} HBM copy bandwidth (MEASURED_PEAKS.json)",
            "algorithmic_bytes": {
                "record_insert": "8 B per record + the window's blocks read and written back once",
                "partition_add": "8 B key read + 8 B record written per key",
                "add_direct": "8 B key + one random 32 B sector read and written back per key",
            }.get(dom, "see phase_bytes() in bench.py")}
    if roof["traffic"]:
        roof["traffic_over_algorithmic"] = roof["traffic"] / kd["algorithmic_bytes_per_launch"]
    if regime == "l2" and bounds and dom in ("add_direct", "contains_direct"):
        # an L2-resident filter: the bound is the random-access rate on the
        # same footprint with the same key stream (Sec. V-B), not HBM
        gb = bounds["red_or" if dom == "add_direct" else "load"]["gkeys_s"]
        rate = (n_ins if dom == "add_direct" else n_q) / (kd["ms_per_step"] * 1e-3) / 1e9
        roof.update({"bound": "l2", "achieved": rate, "peak": gb, "unit": "G keys/s", "frac": rate / gb,
                     "peak_source": "bf_gups on the filter's footprint with the same key stream "
                                    "(random 32-byte loads / red.or), best kpt",
                     "hbm_equivalent_gbs": kd["achieved_gbs"]})
    if dom == "record_insert" and bounds and "red_sector_window" in bounds:
        rb = bounds["red_sector_window"]
        rec_s = n_ins / (kd["ms_per_step"] * 1e-3) / 1e9
        roof["limit"] = {"what": "SM-to-L2 red path: one full 32-byte sector OR per record",
                         "achieved_grecords_s": rec_s, "bound_grecords_s": rb["gkeys_s"],
                         "frac": rec_s / rb["gkeys_s"],
                         "how": f"bf_gups full-sector red.or (4 lanes x 64 bit) on a {rb['table_bytes'] >> 20} MiB "
                                f"table (one window) with the insert key stream, best kpt"}
    # whole operations: the random-access formulation (key + sector access per
    # key; the slice-partitioned path replaces it by streaming, so this is an
    # equivalent rate) next to the measured DRAM traffic of one call
    sectors = max(1, w["block_bits"] // 256)
    ops = {}
    for op, ms_, n_, bpk in (("add", add_ms, n_ins, 8 + 64 * sectors), ("contains", con_ms, n_q, 9 + 32 * sectors)):
        t = measured_traffic(op, wname)
        ops[op] = {"ms_per_call": ms_, "random_access_bytes_per_key": bpk,
                   "random_access_equivalent_frac": bpk * n_ / (ms_ * 1e-3) / 1e9 / peak,
                   "traffic_per_call": t,
                   "achieved_traffic_frac": (t / (ms_ * 1e-3) / 1e9 / peak) if t else None}
    roof["operations"] = ops
    ra = None
    if bounds:
        ra = {"lookup_bound_gkeys_s": bounds["load"]["gkeys_s"], "insert_bound_gkeys_s": bounds["red_or"]["gkeys_s"],
              "lookup_frac": look_g / bounds["load"]["gkeys_s"], "insert_frac": ins_g / bounds["red_or"]["gkeys_s"],
              "unit_bytes": bounds["load"]["unit_bytes"], "how": "bf_gups: same key streams, same footprint, "
              "random unit loads (lookup) / red.or (insert), best kpt"}
        if "red_sector_window" in bounds:
            ra["window_full_sector_red_gkeys_s"] = bounds["red_sector_window"]["gkeys_s"]
    status = f.device_status()

    e2e = None
    if not args.no_e2e:
        e2e = run_e2e(torch, f, ins, qd, args, world, device)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # the oracle: a forked process pool is never used, and the oracle
        # runs in this process only after all GPU work above is done
        r = cpu_oracle_rate(w, args.cpu_budget)
        cpu = {"value": r["gkeys_s"], "unit": "G keys/s", "cores": 1, "kind": "oracle",
               "sample": f"first {r['insert_keys']:,} inserts into the full-size host filter and first "
                         f"{r['lookup_keys']:,} queries ({r['insert_s'] + r['lookup_s']:.1f} s single-thread)",
               "insert_gkeys_s": r["insert_gkeys_s"], "lookup_gkeys_s": r["lookup_gkeys_s"],
               "host_cores": os.cpu_count()}
        if not args.no_cpu_all_cores:
            cpu["all_cores"] = cpu_oracle_rate_all_cores(w)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "G keys/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64 keys / u32 words (integer)",
            "data": "synthetic (SplitMix64 key streams generated on the device)",
            "config": {"workload": wname, "desc": w["desc"], "num_blocks": b, "block_bits": w["block_bits"],
                       "word_bits": w["word_bits"], "k": w["k"], "n_insert": n_ins, "n_lookup": n_q,
                       "salts": "parquet split-block" if w.get("salts") else "splitmix64",
                       "regime": regime, "layouts": layouts, "partition": f.partition(),
                       "key_runs": args.key_runs,
                       "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (no flush)" if n_ins * 8 > props.L2_cache_size
                             else "warm L2 (cache-resident regime)"},
            "insert_gkeys_s": ins_g, "lookup_gkeys_s": look_g, "insert_ms": add_ms, "lookup_ms": con_ms,
            "random_access_bound": ra,
            "fpr": {"bits_per_key": w["nbytes"] * 8 / n_ins, "measured": measured_fpr,
                    "realized_filter": realized_fpr, "fresh_queries": n_fresh, "false_negatives": missed},
            "roofline": roof, "kernels": kernels, "cpu_baseline": cpu, "e2e": e2e,
            "gpu_launches": sum(launches), "clocks": clocks, "device_status": status,
            "l2_persist": args.l2_persist if args.l2_persist > 0 else None,
        }
        print(json.dumps(line), flush=True)
    f.close()
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def link_rates(torch, regions, stream, nbytes=2 << 30, reps=3):
    """Host-link rates: the best of `reps` copy-engine copies of `nbytes`
    from and back to each pinned region in `regions` (tensors of 8-byte
    elements) through one device buffer -- the link itself, not a slow patch
    of host memory.  The step's ceiling is its host-to-device bytes at the
    host-to-device rate."""
    out = {"h2d_gbs": 0.0, "d2h_gbs": 0.0}
    for r in regions:
        n = min(r.numel(), nbytes // 8)
        d = torch.empty(n, dtype=r.dtype, device=stream.device)
        for name, fn in (("h2d_gbs", lambda: d.copy_(r[:n], non_blocking=True)),
                         ("d2h_gbs", lambda: r[:n].copy_(d, non_blocking=True))):
            for _ in range(reps):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                fn()
                b.record(stream)
                b.synchronize()
                out[name] = max(out[name], 8 * n / (a.elapsed_time(b) * 1e-3) / 1e9)
        del d  # the region's first n elements went there and back unchanged
    return out


def run_e2e(torch, f, ins, qd, args, world, device):
    """Same step through the host-buffer entry points: keys start in pinned
    host memory, results end there; the copies are inside the timed region."""
    h_ins = torch.empty(ins.numel(), dtype=torch.int64, pin_memory=True)
    h_q = torch.empty(qd.numel(), dtype=torch.int64, pin_memory=True)
    h_out = torch.empty(qd.numel(), dtype=torch.uint8, pin_memory=True)
    h_ins.copy_(ins)
    h_q.copy_(qd)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    a_ins, a_q, a_out = h_ins.numpy(), h_q.numpy(), h_out.numpy()
    link = link_rates(torch, [h_q, h_ins[h_ins.numel() // 2:]], stream)
    f.set_staging(mode=args.host_mode)

    def step(ev=None):
        if ev:
            ev[0].record(stream)
        f.add_host(a_ins)
        if ev:
            ev[1].record(stream)
        f.contains_host(a_q, a_out)
        if ev:
            ev[2].record(stream)

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize()
    barrier(world)
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s.record(stream)
    for i in range(args.steps):
        step(evs[i])
    e.record(stream)
    e.synchronize()
    ms = max_over_ranks(s.elapsed_time(e), world, device)
    add_ms = statistics.median(x[0].elapsed_time(x[1]) for x in evs)
    con_ms = statistics.median(x[1].elapsed_time(x[2]) for x in evs)
    n = ins.numel() + qd.numel()
    # per-phase device time of one more (untimed) step: where the schedule spends it
    f.set_timing(True)
    step()
    phases = {k: {"ms": round(v["ms"], 3), "launches": v["launches"]} for k, v in f.timing().items()}
    f.set_timing(False)
    f.set_staging(mode="auto")
    del h_ins, h_q, h_out
    return {"value": world * n * args.steps / (ms * 1e-3) / 1e9, "unit": "G keys/s",
            "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": qd.numel(), "ms_per_step": ms / args.steps,
            "add_host_ms": add_ms, "contains_host_ms": con_ms,
            "add_host_link_gbs": 8 * ins.numel() / (add_ms * 1e-3) / 1e9,
            "contains_host_link_gbs": 9 * qd.numel() / (con_ms * 1e-3) / 1e9,
            "api": "bf_add_host + bf_contains_host (pinned host buffers)", "host_mode": args.host_mode,
            # every key and query crosses host-to-device once (8 bytes); results go the other way
            "link": dict(link, ceiling_gkeys_s=link["h2d_gbs"] / 8,
                         frac_of_ceiling=n * args.steps / (ms * 1e-3) / 1e9 / (link["h2d_gbs"] / 8)),
            "phases_one_step": phases}


def run_sweep(args, w, wname):
    """Autotune every layout of this workload's geometry and store the best."""
    import torch
    from paper_2512_15595_gb300 import Filter, autotune
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    props = torch.cuda.get_device_properties(device)
    b, n_ins, n_q = wl_sizes(w)
    regime = autotune.regime_of(w["nbytes"], props.L2_cache_size)
    ins, qd, flags = gen_inputs(torch, w, device)
    # construction is swept at the full insert count: the partitioned path's
    # benefit depends on how many keys share an L2 window
    n_add = n_ins
    n_con = min(n_q, args.sweep_keys)
    f = Filter(b, w["block_bits"], w["word_bits"], w["k"], 0, device=device)
    f.add(ins)  # occupancy of the real workload
    out = torch.empty(n_con, dtype=torch.uint8, device=device)
    parts = [dict(mode=0)]
    if regime == "hbm":
        parts += [dict(mode=1, slice_log2=sl, window_log2=wl)
                  for sl, wl in ((24, 25), (24, 26), (25, 25), (25, 26), (26, 26))]
    lparts = [dict(lookup_mode=0)] + ([dict(lookup_mode=1, lookup_chunk_keys=c) for c in (1 << 27, 1 << 28, 1 << 29)]
                                      if regime == "hbm" else [])
    res = autotune.sweep(torch, f, ins[:n_add], qd[:n_con], out, regime, partitions=parts, kpts=(1, 4), reps=3,
                         lookup_partitions=lparts,
                         log=lambda r: print(json.dumps(r), file=sys.stderr, flush=True))
    table = autotune.load_tuned()
    table[res["key"]] = res["entry"]
    autotune.save_tuned(table)
    print(json.dumps({"sweep": wname, "key": res["key"], "best": res["entry"]}), flush=True)


BATCH_GEOMETRIES = [(64, 32), (128, 32), (256, 32), (64, 64), (128, 64), (256, 64), (512, 64)]  # K = 8 valid


class _BatchRun:
    """One geometry's batch over the batched workload's filters: an arena of
    the filters' bit arrays (same bytes per filter for every geometry, whole
    blocks), the Batch handle, and its captured build + probe graph."""

    def __init__(self, torch, B, S, K, size_bytes, key_off, counts, ins, qd, out, device):
        from synthkeys import batches
        from paper_2512_15595_gb300 import Batch
        self.B, self.S, self.K = B, S, K
        bb = B // 8
        self.blocks = batches.blocks_of(size_bytes, bb)
        off, self.arena_bytes = batches.arena_offsets(self.blocks, bb)
        self.arena = torch.zeros(self.arena_bytes, dtype=torch.uint8, device=device)
        self.views = [self.arena[int(o):int(o) + int(b) * bb] for o, b in zip(off, self.blocks)]
        self.batch = Batch([(v, int(b), int(ko), int(c))
                            for v, b, ko, c in zip(self.views, self.blocks, key_off, counts)], B, S, K)
        self.ins, self.qd, self.out = ins, qd, out
        self.graph = None

    def capture(self, torch):
        stream = torch.cuda.Stream()
        stream.wait_stream(torch.cuda.current_stream())
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, stream=stream):
            self.batch.add(self.ins, stream=stream)
            self.batch.contains(self.qd, out=self.out, stream=stream)

    def false_positives(self, torch) -> int:
        """Positives among the fresh (odd-indexed) queries after a full step."""
        self.batch.add(self.ins)
        self.batch.contains(self.qd, out=self.out)
        return int(self.out[1::2].sum().item())

    def close(self):
        self.batch.close()
        self.arena = None
        self.views = None


def _batched_inputs(torch, device, nfilters=4096, total=1 << 28, B=256):
    """The batched workload: 4096 filter sizes log-uniform 4 KiB-16 MiB (PCG64
    seed 5), 2^28 insert keys split in proportion to the 256-bit-block counts,
    queries = the insert stream with every second key replaced by a fresh one
    (fewer filters and keys for profiling-sized cases)."""
    import numpy as np
    import synthkeys
    from synthkeys import batches
    size_bytes = batches.log_uniform_bytes(nfilters, 4 << 10, 16 << 20, seed=5)
    counts = batches.proportional_counts(batches.blocks_of(size_bytes, B // 8), total)
    key_off = np.zeros(nfilters, dtype=np.int64)
    key_off[1:] = np.cumsum(counts)[:-1]
    ins = synthkeys.splitmix64_torch(synthkeys.SEED_INSERT, 0, total, device)
    fresh = synthkeys.splitmix64_torch(synthkeys.SEED_FRESH, 0, total, device)
    qd = ins.clone()
    qd[1::2] = fresh[1::2]
    del fresh
    out = torch.zeros(total, dtype=torch.uint8, device=device)
    return size_bytes, counts, key_off, ins, qd, out


def _timed(torch, fn, steps, warm):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    s_, e_ = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s_.record()
    for _ in range(steps):
        fn()
    e_.record()
    e_.synchronize()
    return s_.elapsed_time(e_) / steps


def run_batched_sweep(args):
    """Autotune the batched workload: every compiled layout of the batched add
    and contains launches (with and without the L2 prefetch hint, at four grid
    sizes) for every geometry with K = 8, then the block width
    (and word size) of the fastest step whose false positives on the fresh
    queries stay within the 3-sigma band of the 256-bit / 32-bit geometry's.
    Stores the layouts per geometry and the choice in tuned_layouts.json."""
    import torch
    from paper_2512_15595_gb300 import BF_HINT_PREFETCH_L2, autotune
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    K = 8
    size_bytes, counts, key_off, ins, qd, out = _batched_inputs(torch, device, args.batch_filters, args.batch_keys)
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    grids = (0, sms, 2 * sms, 4 * sms)
    table = autotune.load_tuned()
    results = []
    for B, S in BATCH_GEOMETRIES:
        run = _BatchRun(torch, B, S, K, size_bytes, key_off, counts, ins, qd, out, device)
        res = autotune.sweep_batch(torch, run.batch, ins, qd, out, reps=3, flag_sets=(0, BF_HINT_PREFETCH_L2),
                                   grids=grids)
        run.arena.zero_()
        fp = run.false_positives(torch)
        entry = dict(res["entry"], fp=fp, queries=int(counts.sum()) // 2, filter_bytes=int(run.arena_bytes))
        table[res["key"]] = entry
        results.append(dict(block_bits=B, word_bits=S, k=K, step_ms=entry["step_ms"], fp=fp,
                            queries=entry["queries"]))
        print(json.dumps({"sweep": "batched", "key": res["key"], "best": entry}), flush=True)
        run.close()
        del run
        torch.cuda.empty_cache()
    choice = autotune.choose_batch_geometry(results, (256, 32))
    table[f"batch_K{K}_geometry"] = choice
    autotune.save_tuned(table)
    print(json.dumps({"sweep": "batched", "geometry": choice}), flush=True)


def run_batched(args):
    """Batched filters: 4096 filters, log-uniform 4 KiB-16 MiB (256-bit blocks,
    S=32, K=8), 2^28 keys split in proportion to size; one step = build all
    filters + probe all of them (half of each run replaced by fresh keys), as
    one captured CUDA graph of two launches, against one launch per filter per
    operation.  Layouts come from the autotuner's table when it holds this
    geometry; the geometry the autotuner picked (block width at the same FPR
    band) is timed beside it when it differs."""
    import numpy as np
    import torch
    import synthkeys
    from paper_2512_15595_gb300 import BF_OP_ADD, BF_OP_CONTAINS, Filter, autotune
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    B, S, K = 256, 32, 8
    size_bytes, counts, key_off, ins, qd, out = _batched_inputs(torch, device, args.batch_filters, args.batch_keys)
    nfilters, total = len(counts), int(counts.sum())
    default_layouts = {BF_OP_ADD: dict(cg=4, phi=2, kpt=4), BF_OP_CONTAINS: dict(cg=1, phi=8, kpt=4)}

    def layouts_for(b, s_):
        tuned = {op: autotune.tuned_batch_layout(b, s_, K, op) for op in (BF_OP_ADD, BF_OP_CONTAINS)}
        if all(tuned.values()):
            return tuned, True
        return default_layouts, False

    run = _BatchRun(torch, B, S, K, size_bytes, key_off, counts, ins, qd, out, device)
    lays, autotuned = layouts_for(B, S)
    for op, lay in lays.items():
        run.batch.set_layout(op, **lay)
    run.capture(torch)
    ms_graph = _timed(torch, run.graph.replay, args.steps, args.warmup)
    # eager batched calls (same two launches, not captured), and each operation alone
    ms_eager = _timed(torch, lambda: (run.batch.add(ins), run.batch.contains(qd, out=out)), args.steps, args.warmup)
    ms_add = _timed(torch, lambda: run.batch.add(ins), args.steps, 1)
    ms_con = _timed(torch, lambda: run.batch.contains(qd, out=out), args.steps, 1)
    # one launch per filter per operation, on the same buffers
    fs = [] if args.no_per_filter else [Filter(int(b), B, S, K, 0, words=v) for v, b in zip(run.views, run.blocks)]
    for f in fs:
        f.set_partition(mode=0, lookup_mode=0)
        for op, lay in lays.items():
            # the same thread layout; each launch sized for its own filter
            f.set_layout(op, cg=lay["cg"], phi=lay["phi"], kpt=lay["kpt"])
    runs = [(f, ins[ko:ko + c], qd[ko:ko + c], out[ko:ko + c]) for f, ko, c in zip(fs, key_off, counts) if c]

    def per_filter():
        for f, k_, q_, o_ in runs:
            f.add(k_)
        for f, k_, q_, o_ in runs:
            f.contains(q_, out=o_)
    ms_per_filter = _timed(torch, per_filter, max(1, args.steps // 2), 1) if runs else None
    for f in fs:
        f.close()
    per_filter_launches = 2 * len(runs)
    del fs, runs
    # properties: no false negatives; FPR of the fresh half
    run.graph.replay()
    torch.cuda.synchronize()
    fn = int((out[0::2] == 0).sum().item())
    fp = int(out[1::2].sum().item())
    # spot parity of a few filters against the oracle
    import oracle
    sample = [0, 1, nfilters // 2, nfilters - 1]
    mismatches = 0
    for i in sample:
        geom = oracle.Geometry(num_blocks=int(run.blocks[i]), block_bits=B, word_bits=S, k=K, seed=0)
        ref = oracle.SBF(geom)
        ref.add(synthkeys.splitmix64(synthkeys.SEED_INSERT, int(key_off[i]), int(counts[i])))
        mismatches += int(not np.array_equal(run.views[i].cpu().numpy(), ref.as_bytes()))
    layouts = {"add": run.batch.layout(BF_OP_ADD), "contains": run.batch.layout(BF_OP_CONTAINS)}
    arena_bytes = run.arena_bytes
    run.close()
    del run
    torch.cuda.empty_cache()
    keys_per_step = 2 * total
    line = {
        "metric": f"batched build+probe, G keys/s ({nfilters} filters, one CUDA-graph launch per step)",
        "value": keys_per_step / (ms_graph * 1e-3) / 1e9, "unit": "G keys/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_graph, "higher_is_better": True,
        "dtype": "u64 keys / u32 words (integer)", "data": "synthetic",
        "config": {"workload": "batched" if (nfilters, total) == (4096, 1 << 28) else "batched (reduced)",
                   "filters": nfilters, "sizes": "log-uniform 4 KiB-16 MiB (seed 5)",
                   "filter_bytes": int(arena_bytes), "keys": total, "queries": total,
                   "layouts": layouts, "layouts_autotuned": autotuned},
        "eager_batched_ms_per_step": ms_eager,
        "add_gkeys_s": total / (ms_add * 1e-3) / 1e9, "contains_gkeys_s": total / (ms_con * 1e-3) / 1e9,
        "per_filter_launches": None if ms_per_filter is None else {
            "ms_per_step": ms_per_filter, "launches_per_step": per_filter_launches,
            "value": keys_per_step / (ms_per_filter * 1e-3) / 1e9},
        "speedup_vs_per_filter": None if ms_per_filter is None else ms_per_filter / ms_graph,
        "gpu_launches": 2 * args.steps,
        "checks": {"false_negatives": fn, "false_positives": fp, "fresh_queries": total // 2,
                   "fpr_fresh_half": fp / (total // 2), "oracle_filters_checked": len(sample),
                   "oracle_mismatches": mismatches},
    }
    choice = None if args.no_per_filter else autotune.load_tuned().get(f"batch_K{K}_geometry")
    if choice and (choice["block_bits"], choice["word_bits"]) != (B, S):
        Bt, St = choice["block_bits"], choice["word_bits"]
        trun = _BatchRun(torch, Bt, St, K, size_bytes, key_off, counts, ins, qd, out, device)
        tl, _ = layouts_for(Bt, St)
        for op, lay in tl.items():
            trun.batch.set_layout(op, **lay)
        tfp = trun.false_positives(torch)
        tfn = int((out[0::2] == 0).sum().item())
        trun.capture(torch)
        tms = _timed(torch, trun.graph.replay, args.steps, args.warmup)
        line["tuned_geometry"] = {"block_bits": Bt, "word_bits": St, "k": K, "ms_per_step": tms,
                                  "value": keys_per_step / (tms * 1e-3) / 1e9, "false_positives": tfp,
                                  "false_negatives": tfn, "fp_limit": choice["fp_limit"],
                                  "layouts": {"add": trun.batch.layout(BF_OP_ADD),
                                              "contains": trun.batch.layout(BF_OP_CONTAINS)},
                                  "filter_bytes": int(trun.arena_bytes), "gpu_launches": 2 * args.steps}
        trun.close()
    elif choice:
        line["tuned_geometry"] = {"block_bits": B, "word_bits": S, "k": K, "same_as_workload": True}
    print(json.dumps(line), flush=True)


def run_frontier(args):
    """Throughput vs FPR of the sectorized (SBF) and cache-sectorized (CSBF)
    variants, as the paper's frontier (Sec. V-A, V-B, V-C): S = 64, k = 16,
    block sizes 256/512/1024, every compiled group count, on a 32 MiB
    (L2-resident) and a 1 GiB (HBM-resident) filter.  The filter holds the
    Eq. (1)-optimal number of keys for k = 16 (c = k / ln 2 bits per key);
    throughput = best layout for inserting them and for looking them all up
    (true positives), FPR = fraction of 10^8 fresh keys reported present.
    One JSON line per configuration, then a summary line."""
    import torch
    import synthkeys
    from paper_2512_15595_gb300 import BF_OP_ADD, BF_OP_CONTAINS, Filter
    from paper_2512_15595_gb300.autotune import time_op
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    S, K = 64, 16
    c_opt = K / math.log(2.0)
    fresh_n = 10**8
    fresh = synthkeys.splitmix64_torch(synthkeys.SEED_FRESH + 100, 0, fresh_n, device)
    rows = []
    for size_name, nbytes in (("32MiB", 32 << 20), ("1GiB", 1 << 30)):
        for B in (256, 512, 1024):
            s_ = B // S
            nb = nbytes * 8 // B
            n = int(nbytes * 8 / c_opt)
            keys = synthkeys.splitmix64_torch(synthkeys.SEED_INSERT, 0, n, device)
            out = torch.empty(max(n, fresh_n), dtype=torch.uint8, device=device)
            variants = [0] + [z for z in (1, 2, 4, 8) if z < s_ and K % z == 0]
            for z in variants:
                f = Filter(nb, B, S, K, 0, device=device, groups=z)
                if z:
                    layouts = [(cg, 1) for cg in (1, 2, 4, 8) if z % cg == 0]
                else:
                    layouts = [(cg, s_ // cg) for cg in (1, 2, 4, 8, 16) if cg <= s_]  # max phi per cg (tables)
                best = {}
                for part in ((0,) if z else (0, 1)):
                    f.set_partition(mode=part, lookup_mode=part)
                    for cg, phi in layouts:
                        for kpt in (1, 4):
                            for op, name, ks in ((BF_OP_ADD, "add", keys), (BF_OP_CONTAINS, "contains", keys)):
                                f.set_layout(op, cg=cg, phi=phi, kpt=kpt)
                                if op == BF_OP_CONTAINS:
                                    f.clear()
                                    f.add(keys)
                                ms = time_op(torch, f, op, ks, out[:n], reps=3, warmup=1)
                                g = n / (ms * 1e-3) / 1e9
                                if g > best.get(name, (0,))[0]:
                                    best[name] = (g, dict(cg=cg, phi=phi, kpt=kpt, partitioned=bool(part)))
                f.set_partition(mode=0, lookup_mode=0)
                f.clear()
                f.add(keys)
                hits = f.contains(fresh, out=out[:fresh_n])
                fpr = float(hits.float().mean().item())
                row = {"size": size_name, "block_bits": B, "word_bits": S, "k": K, "groups": z or s_,
                       "variant": "SBF" if not z else f"CSBF z={z}", "keys": n, "bits_per_key": nbytes * 8 / n,
                       "insert_gkeys_s": best["add"][0], "insert_layout": best["add"][1],
                       "lookup_gkeys_s": best["contains"][0], "lookup_layout": best["contains"][1],
                       "fpr": fpr}
                rows.append(row)
                print(json.dumps(row), flush=True)
                f.close()
            del keys, out
            torch.cuda.empty_cache()
    print(json.dumps({"frontier": len(rows), "note": "S=64, k=16, Eq. (1)-optimal load; best layout per op"}))


def run_serving(args):
    """Serving loop: 64 device-resident filters with sizes log-uniform 1 MiB-2 GiB
    (256-bit blocks, S=32, K=8; each holds 10 bits/key of its own key stream);
    lookup requests arrive as a Poisson process, each for one filter (uniform)
    with log-uniform 1K-16M keys from a pinned host pool; the server admits
    them into a 2^28-key device arena and batches them across filters per
    launch.  Reports p50/p99 latency and sustained G lookups/s at several
    offered loads."""
    import numpy as np
    import torch
    import synthkeys
    from synthkeys import batches
    from paper_2512_15595_gb300 import Filter, _lib
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    B, S, K, nf = 256, 32, 8, 64
    bb = B // 8
    blocks = batches.log_uniform_sizes(nf, 1 << 20, 2 << 30, bb, seed=6)
    filters = []
    for i, nb in enumerate(blocks):
        f = Filter(int(nb), B, S, K, 0, device=device)
        f.set_partition(mode=0)  # set-up only: the direct kernel needs no workspace
        n = int(nb) * B // 10
        for lo in range(0, n, 1 << 28):
            c = min(1 << 28, n - lo)
            f.add(synthkeys.splitmix64_torch(1000 + i, lo, c, device))
        filters.append(f)
    torch.cuda.synchronize()
    pool_n = 1 << 28
    pool = torch.empty(pool_n, dtype=torch.int64, pin_memory=True)
    pool.copy_(synthkeys.splitmix64_torch(synthkeys.SEED_FRESH, 0, pool_n, device))
    pout = torch.zeros(pool_n, dtype=torch.uint8, pin_memory=True)
    srv = _lib.bf_server_create(_lib.bf_params(1, B, S, K, 0, 0),
                                [(f.words.data_ptr(), int(nb)) for f, nb in zip(filters, blocks)],
                                arena_keys=1 << 28, max_requests_per_launch=4096)
    min_k, max_k = 1 << 10, 1 << 24
    mean_keys = (max_k - min_k) / math.log(max_k / min_k)
    results = []
    try:
        # warm-up
        _lib.bf_server_run_poisson(srv, 200.0, 0.2, min_k, max_k, pool.data_ptr(), pool_n, pout.data_ptr(), 1)
        for load_gkeys in (5.0, 10.0, 15.0, 20.0, 25.0):
            rate = load_gkeys * 1e9 / mean_keys
            st = _lib.bf_server_run_poisson(srv, rate, args.serve_seconds, min_k, max_k, pool.data_ptr(), pool_n,
                                            pout.data_ptr(), 11)
            results.append({"offered_gkeys_s": load_gkeys, "requests_per_s": rate,
                            "sustained_gkeys_s": st["keys"] / st["span_s"] / 1e9 if st["span_s"] else 0.0,
                            "p50_ms": st["p50_s"] * 1e3, "p99_ms": st["p99_s"] * 1e3, "max_ms": st["max_s"] * 1e3,
                            "requests": st["requests"], "launches": st["launches"],
                            # device time of each stage over the served span: how busy each stream was
                            "busy": {k: st[k + "_s"] / st["span_s"] if st["span_s"] else 0.0
                                     for k in ("stage_in", "lookup", "stage_out")},
                            "stage_in_gbs": 8 * st["keys"] / st["stage_in_s"] / 1e9 if st["stage_in_s"] else 0.0})
            print(json.dumps(results[-1]), file=sys.stderr, flush=True)
    finally:
        _lib.bf_server_destroy(srv)
        for f in filters:
            f.close()
    best = max(results, key=lambda r: r["sustained_gkeys_s"])
    line = {
        "metric": "serving: sustained G lookups/s and p50/p99 latency (64 filters, Poisson requests)",
        "value": best["sustained_gkeys_s"], "unit": "G keys/s", "n_gpus": 1, "higher_is_better": True,
        "data": "synthetic", "dtype": "u64 keys / u32 words (integer)",
        "config": {"workload": "serving", "filters": nf, "sizes": "log-uniform 1 MiB-2 GiB (seed 6)",
                   "filter_bytes": int(blocks.sum()) * bb, "request_keys": "log-uniform 1K-16M",
                   "arena_keys": 1 << 28, "seconds_per_load": args.serve_seconds,
                   "path": "pinned host keys -> device arena -> one batched launch per admission round -> host"},
        "loads": results,
    }
    print(json.dumps(line), flush=True)


LEARNED_DESC = ("learned prefilter: 64M member keys from 10k clustered intervals (32 clusters, log-normal widths); "
                "network 64->128->64->1 over the key bits, int8 weights, trained on 2M members + 2M non-members "
                "(half uniform, half within 2x an interval's width of one); backup SBF 256-bit blocks, S=32, K=8; "
                "10 bits/key for learned (model + backup) and plain SBF alike; lookups: 64M members + 64M non-members")


def learned_data(n_members=1 << 26, n_train=1 << 21, n_query_non=1 << 26, n_val=1 << 21, seed=17):
    """Host arrays of the learned-prefilter workload (seeded; see synthkeys.clustered)."""
    import numpy as np
    from synthkeys import clustered
    s, w = clustered.intervals(n_intervals=10_000, n_clusters=32, seed=seed)
    mem = clustered.members(n_members + n_members // 50, s, w, seed=seed + 1)
    rng = np.random.default_rng(seed + 2)
    mem = rng.permutation(mem)[:n_members]
    tr_non, _ = clustered.non_members(n_train, s, w, seed=seed + 3)
    val_non, val_near = clustered.non_members(n_val, s, w, seed=seed + 4)
    q_non, q_near = clustered.non_members(n_query_non, s, w, seed=seed + 5)
    return {"members": mem, "train_non": tr_non, "val_non": val_non, "val_near": val_near,
            "query_non": q_non, "query_near": q_near, "n_intervals": int(s.size)}


def run_learned(args):
    """Learned prefilter vs the plain filter at equal bits/key: train, export,
    pick tau on a validation set, build, then time lookups (model + backup)."""
    import numpy as np
    import torch
    from paper_2512_15595_gb300 import Filter, learned as LB
    from synthkeys.mlp_params import flatten, init_params
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    t_gen = time.perf_counter()
    d = learned_data(n_members=args.learned_members, n_query_non=args.learned_members)
    t_gen = time.perf_counter() - t_gen
    n_mem = d["members"].size
    to_dev = lambda a: torch.from_numpy(np.ascontiguousarray(a).view(np.int64)).to(device)
    members = to_dev(d["members"])
    n_tr = d["train_non"].size
    train_keys = to_dev(np.concatenate([d["members"][:n_tr], d["train_non"]]))
    train_labels = torch.cat([torch.ones(n_tr), torch.zeros(n_tr)]).to(device)
    # training
    batch, steps = 4096, args.train_steps
    tr = LB.Trainer(flatten(init_params(1, scale=1.0)), batch=batch, device=device)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    losses = tr.train(train_keys, train_labels, steps, lr=2e-3)
    e1.record()
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)
    model = LB.IntModel(tr.export(train_keys), device=device)
    bits = 10 * n_mem
    B, S, K = 256, 32, 8
    plain_blocks = bits // B
    backup_blocks = (bits - LB.model_bits()) // B
    # tau on the validation set: candidates at quantiles of the non-member scores
    val = to_dev(d["val_non"])
    val_scores = model.scores(val).cpu().numpy()
    cands = sorted(set(int(x) for x in np.quantile(val_scores, [0.5, 0.8, 0.9, 0.95, 0.99, 0.999])) |
                   {int(val_scores.max()) + 1})

    def pick_tau(backup_blocks):
        curve, best = [], None
        for t in cands:
            f_ = LB.LearnedFilter(model, t, members, backup_blocks, B, S, K, 0)
            fp = f_.contains(val).float().mean().item()
            curve.append({"tau": t, "backup_keys": f_.n_backup, "val_fpr": fp})
            if best is None or fp < best[1]:
                best = (t, fp)
            f_.backup.close()
        return best[0], curve

    tau, curve = pick_tau(backup_blocks)
    lf = LB.LearnedFilter(model, tau, members, backup_blocks, B, S, K, 0)
    plain = Filter(plain_blocks, B, S, K, 0, device=device)
    plain.add(members)
    # query set: all members, then the non-member query set
    qn = to_dev(d["query_non"])
    queries = torch.cat([members, qn])
    near = torch.from_numpy(d["query_near"]).to(device).bool()
    out = torch.empty(queries.numel(), dtype=torch.bool, device=device)
    pout = torch.empty_like(out)
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts), ts

    scores = torch.empty(queries.numel(), dtype=torch.int32, device=device)
    score_ms, _ = timed(lambda: model.scores(queries, scores), max(3, args.steps))
    plain_ms, _ = timed(lambda: plain.contains(queries, out=pout), max(3, args.steps))
    props = torch.cuda.get_device_properties(device)
    sampler = ClockSampler(0, getattr(props, "uuid", None) and f"GPU-{props.uuid}")
    torch.cuda.synchronize()
    sampler.start()
    look_ms, all_ms = timed(lambda: lf.contains(queries, out=out), args.steps)
    clocks = sampler.stop()
    launches_per_lookup = lf.backup.last_launches() + 1  # backup filter lookup + the model kernel
    model.check()
    nq = queries.numel()
    o = out.cpu().numpy()
    po = pout.cpu().numpy()
    nr = d["query_near"].astype(bool)
    fn_learned = int((~o[:n_mem]).sum())
    fn_plain = int((~po[:n_mem]).sum())
    ln, pn = o[n_mem:], po[n_mem:]
    fpr = {"bits_per_key": 10.0, "model_bits": LB.model_bits(), "tau": tau, "backup_keys": lf.n_backup,
           "learned": {"all": float(ln.mean()), "uniform": float(ln[~nr].mean()), "near": float(ln[nr].mean())},
           "plain": {"all": float(pn.mean()), "uniform": float(pn[~nr].mean()), "near": float(pn[nr].mean())},
           "false_negatives": {"learned": fn_learned, "plain": fn_plain}, "tau_curve": curve,
           "non_member_queries": int(ln.size)}
    # the same comparison at other budgets (tau re-chosen on the validation set for each)
    by_bits = []
    qn_near = torch.from_numpy(nr).to(device)
    for bpk in [int(x) for x in args.learned_bits.split(",") if x]:
        tb = bpk * n_mem
        pb, bb = tb // B, max(1, (tb - LB.model_bits()) // B)
        t_b, _ = pick_tau(bb)
        lb = LB.LearnedFilter(model, t_b, members, bb, B, S, K, 0)
        pf = Filter(pb, B, S, K, 0, device=device)
        pf.add(members)
        lo_ = lb.contains(qn)
        po_ = pf.contains(qn)
        by_bits.append({"bits_per_key": bpk, "tau": t_b, "backup_keys": lb.n_backup,
                        "learned": {"all": lo_.float().mean().item(), "uniform": lo_[~qn_near].float().mean().item(),
                                    "near": lo_[qn_near].float().mean().item()},
                        "plain": {"all": po_.float().mean().item(), "uniform": po_[~qn_near].float().mean().item(),
                                  "near": po_[qn_near].float().mean().item()}})
        print(json.dumps(by_bits[-1]), file=sys.stderr, flush=True)
        lb.backup.close()
        pf.close()
    fpr["by_bits_per_key"] = by_bits
    # roofline of the model kernel: 2 * (64*128 + 128*64 + 64) algorithmic flops per key (tensor engine)
    flops_key = 2 * (64 * 128 + 128 * 64 + 64)
    pk_path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    with open(pk_path) as f:
        pk = json.load(f)
    tf = flops_key * nq / (score_ms * 1e-3) / 1e12
    engine = "tensor (tcgen05 kind::f16, bf16 operands, fp32 accumulate; exact)" \
        if model.engine == LB.BF_MLP_ENGINE_TENSOR else "dp4a (CUDA cores)"
    traffic = measured_traffic("scores", "learned", ("lbf_tc.cu", "lbf.h")) if nq == 1 << 27 else None
    roof = {"bound": "tensor", "achieved": tf, "peak": pk["bf16_tflops"], "unit": "TFLOP/s",
            "frac": tf / pk["bf16_tflops"], "traffic": traffic, "kernel": f"bf_mlp_scores: {engine}",
            "per": "one call", "peak_source": "measured bf16 dense burst (MEASURED_PEAKS.json)",
            "algorithmic_flops_per_key": flops_key, "keys_per_call": nq, "ms_per_call": score_ms}
    # the tensor-instruction bound: one tile of 128 keys is 4 MMAs (N = 128, A
    # in shared memory) + 8 MMAs (N = 64, A in tensor memory); their measured
    # per-instruction cost at the sampled SM clock
    from paper_2512_15595_gb300 import _lib as LL
    c128, c64 = LL.bf_mma_cost(128, False), LL.bf_mma_cost(64, True)
    tile_cycles = 4 * c128 + 8 * c64
    f_hz = (clocks or {}).get("sm_mhz") or 2070.0
    sms = torch.cuda.get_device_properties(device).multi_processor_count
    bound = 128 * sms * f_hz * 1e6 / tile_cycles / 1e9
    tib = {"cycles_per_mma_n128_smem": c128, "cycles_per_mma_n64_tmem": c64, "cycles_per_tile": tile_cycles,
           "sm_mhz": f_hz, "gkeys_s": bound, "model_frac": (nq / (score_ms * 1e-3) / 1e9) / bound,
           "how": "bf_mma_cost: back-to-back tcgen05.mma kind::f16, M=128, K=16, one issuing thread per SM"}
    e2e = None
    if not args.no_e2e:
        e2e = learned_e2e(torch, lf, queries, args)
    line = {
        "metric": "learned prefilter: G lookups/s (model + backup) and FPR vs plain SBF at equal bits/key",
        "value": nq / (look_ms * 1e-3) / 1e9, "unit": "G keys/s", "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": look_ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int8 model (exact, bf16 MMA) / u32 words", "data": "synthetic",
        "config": {"workload": "learned", "desc": LEARNED_DESC, "members": n_mem, "queries": nq,
                   "intervals": d["n_intervals"], "plain_blocks": plain_blocks, "backup_blocks": backup_blocks,
                   "l2": "inputs larger than L2 (no flush)", "host_data_s": t_gen},
        "plain_lookup_gkeys_s": nq / (plain_ms * 1e-3) / 1e9, "model_scores_gkeys_s": nq / (score_ms * 1e-3) / 1e9,
        "training": {"steps": steps, "batch": batch, "ms": train_ms, "ms_per_step": train_ms / steps,
                     "first_loss": float(losses[:10].mean().item()), "last_loss": float(losses[-50:].mean().item())},
        "engine": engine, "fpr": fpr, "roofline": roof, "tensor_instruction_bound": tib, "e2e": e2e,
        "clocks": clocks,
        "gpu_launches": launches_per_lookup * args.steps,
    }
    print(json.dumps(line), flush=True)
    lf.backup.close()
    plain.close()
    model.close()


def learned_e2e(torch, lf, queries, args):
    """Learned lookups from pinned host keys to a pinned host result through
    bf_mlp_contains_host (staged copies overlapped with the lookups)."""
    n = queries.numel()
    hk = torch.empty(n, dtype=torch.int64, pin_memory=True)
    hk.copy_(queries)
    ho = torch.empty(n, dtype=torch.bool, pin_memory=True)

    def go():
        lf.contains_host(hk, ho)
        torch.cuda.synchronize()

    go()
    ts = []
    for _ in range(max(1, args.steps // 2)):
        t0 = time.perf_counter()
        go()
        ts.append(time.perf_counter() - t0)
    t = statistics.median(ts)
    return {"value": n / t / 1e9, "unit": "G keys/s", "h2d_bytes_per_step": 8 * n, "d2h_bytes_per_step": n,
            "path": "bf_mlp_contains_host: pinned host keys -> device staging (2^24-key chunks, 3 streams) -> "
                    "backup lookup + model -> pinned host bytes"}


def run_learned_reference(args):
    """The oracle's integer model + backup lookups on a bounded sample (host cores)."""
    import numpy as np
    import oracle
    from oracle import learned as OL
    from synthkeys.mlp_params import init_params
    world, rank, _ = dist_env()
    if rank != 0:
        return
    d = learned_data(n_members=1 << 20, n_train=1 << 10, n_query_non=1 << 18, n_val=1 << 10)
    m = OL.quantize(init_params(1, scale=1.0), d["members"][:4096])
    sm = OL.int_scores(m, d["members"])
    tau = int(np.quantile(sm, 0.5))
    geom = oracle.Geometry(num_blocks=(10 * (1 << 26)) // 256, block_bits=256, word_bits=32, k=8, seed=0)
    f = oracle.SBF(geom)
    f.add(d["members"][sm < tau])
    q = np.concatenate([d["members"][: 1 << 18], d["query_non"]])
    vals = []
    t_all = time.perf_counter()
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        got = (OL.int_scores(m, q) >= tau) | (f.contains(q) != 0)
        dt = time.perf_counter() - t0
        if i >= args.warmup:
            vals.append(q.size / dt / 1e9)
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": "learned prefilter: G lookups/s (model + backup) and FPR vs plain SBF "
            "at equal bits/key", "value": v, "unit": "G keys/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": q.size / v / 1e6, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "int64 numpy (integer model) / u32 words", "data": "synthetic",
            "config": {"workload": "learned", "desc": LEARNED_DESC},
            "cpu_baseline": {"value": v, "unit": "G keys/s", "cores": 1, "kind": "oracle",
                             "sample": f"{q.size:,} queries (2^18 members + 2^18 non-members) through the oracle's "
                                       "integer model and its backup filter (full-size geometry), per step"},
            "e2e": {"value": v, "unit": "G keys/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "positives": int(got.sum())}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="4GiB", choices=sorted(WORKLOADS) + ["batched", "serving", "learned"])
    ap.add_argument("--train-steps", type=int, default=3000)
    ap.add_argument("--learned-bits", default="2,4,6,8", help="other bits/key budgets for the FPR comparison")
    ap.add_argument("--salts", default="default", choices=["default", "parquet"],
                    help="salt set of the filter (parquet: the Parquet split-block multipliers; 256/32/8 only)")
    ap.add_argument("--learned-members", type=int, default=1 << 26,
                    help="member keys of the learned workload (queries: as many non-members again)")
    ap.add_argument("--serve-seconds", type=float, default=3.0)
    ap.add_argument("--n-lookup", type=int, default=0,
                    help="filter workloads: lookups per step instead of the workload's (profiling-sized runs)")
    ap.add_argument("--batch-filters", type=int, default=4096, help="batched workload: number of filters")
    ap.add_argument("--batch-keys", type=int, default=1 << 28, help="batched workload: keys (and queries)")
    ap.add_argument("--no-per-filter", action="store_true",
                    help="batched workload: skip the per-filter-launch comparison and the tuned-geometry run")
    ap.add_argument("--sweep", action="store_true")
    ap.add_argument("--frontier", action="store_true")
    ap.add_argument("--sweep-keys", type=int, default=1 << 28)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-gups", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-all-cores", action="store_true", help="skip the all-core oracle timing")
    ap.add_argument("--add-flags", default="", choices=["", "aggregate"],
                    help="construction hint: aggregate = BF_HINT_WARP_AGGREGATE")
    ap.add_argument("--key-runs", type=int, default=1,
                    help="insert stream as runs of this many equal keys (same length)")
    ap.add_argument("--l2-persist", type=float, default=0.0,
                    help="L2 persistence window over the filter with this hit ratio during the timed steps")
    ap.add_argument("--host-mode", default="auto", choices=["auto", "direct", "staged"],
                    help="host-buffer schedule of the e2e leg (bf_set_staging): auto = passes staged "
                         "through device memory, direct = kernels read host memory in place, "
                         "staged = copy-engine staging")
    ap.add_argument("--cpu-budget", type=float, default=20.0)
    args = ap.parse_args()
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.frontier:
        run_frontier(args)
        return
    if args.workload == "serving":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "no CPU arm for the serving workload"}))
        else:
            run_serving(args)
        return
    if args.workload == "learned":
        if args.impl == "reference":
            run_learned_reference(args)
        else:
            run_learned(args)
        return
    if args.workload == "batched":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "no CPU arm for the batched workload"}))
        elif args.sweep:
            run_batched_sweep(args)
        else:
            run_batched(args)
        return
    w = dict(WORKLOADS[args.workload])
    if args.n_lookup:
        w["n_lookup"] = args.n_lookup
        w["desc"] = w["desc"] + f"; reduced to {args.n_lookup} lookups per step"
    if args.salts == "parquet":
        if (w["block_bits"], w["word_bits"], w["k"]) != (256, 32, 8):
            ap.error("the Parquet salt set exists for 256-bit blocks, S = 32, K = 8 only")
        w["salts"] = 1
        w["desc"] = w["desc"] + "; Parquet split-block salt set (bit-compatible with Parquet/Arrow filters)"
    if args.impl == "reference":
        run_reference(args, w, args.workload)
    elif args.sweep:
        run_sweep(args, w, args.workload)
    else:
        run_ours(args, w, args.workload)


if __name__ == "__main__":
    main()
