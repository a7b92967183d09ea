"""Autotuner for the execution layout of construction and lookup.

The paper tunes the layout offline per block size, memory regime and GPU
(Sec. V-A: best over all valid (Theta, Phi); Sec. V-D: the optimum differs
across architectures).  This module times every compiled layout (Theta, Phi,
keys per thread) of one geometry through the C ABI with CUDA events, keeps
the fastest per operation, and stores the choice in ``tuned_layouts.json``
next to this file, keyed by geometry and residency regime.  Filters built
through :func:`apply_tuned` start from that choice.  For batches of filters
(one launch per operation over all of them) it tunes the batched launches'
layouts per geometry and picks the block width and word size at a
false-positive band (:func:`sweep_batch`, :func:`choose_batch_geometry`).
"""
from __future__ import annotations

import json
import os

from . import BF_OP_ADD, BF_OP_CONTAINS, Filter, valid_layouts

TUNED_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuned_layouts.json")


def regime_of(nbytes: int, l2_bytes: int) -> str:
    """'l2' if the bit array fits in half the L2, else 'hbm'."""
    return "l2" if nbytes * 2 <= l2_bytes else "hbm"


def key_of(block_bits: int, word_bits: int, k: int, regime: str) -> str:
    return f"B{block_bits}_S{word_bits}_K{k}_{regime}"


def load_tuned() -> dict:
    if os.path.exists(TUNED_PATH):
        with open(TUNED_PATH) as f:
            return json.load(f)
    return {}


def save_tuned(table: dict) -> None:
    tmp = TUNED_PATH + ".tmp"
    with open(tmp, "w") as f:
        json.dump(table, f, indent=1, sort_keys=True)
    os.replace(tmp, TUNED_PATH)


def tuned_layout(block_bits: int, word_bits: int, k: int, regime: str, op: int) -> dict | None:
    entry = load_tuned().get(key_of(block_bits, word_bits, k, regime))
    if not entry:
        return None
    return entry.get("add" if op == BF_OP_ADD else "contains", {}).get("layout")


def apply_tuned(f: Filter, regime: str) -> dict:
    """Set the filter's layouts (and construction partitioning) from the tuned table."""
    p = f.params
    used = {}
    for op, name in ((BF_OP_ADD, "add"), (BF_OP_CONTAINS, "contains")):
        lay = tuned_layout(p.block_bits, p.word_bits, p.k, regime, op)
        if lay:
            lay = dict(lay)
            part = lay.pop("partition", None)
            f.set_layout(op, **lay)
            if part is not None:
                f.set_partition(**part)
        used[name] = f.layout(op)
    return used


def time_op(torch, f: Filter, op: int, keys, out, reps: int = 5, warmup: int = 2, flush=None) -> float:
    """Median device time (ms) of one bulk call with the filter's current layout."""
    stream = torch.cuda.current_stream()
    times = []
    for i in range(warmup + reps):
        if flush is not None:
            flush()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        if op == BF_OP_ADD:
            f.add(keys)
        else:
            f.contains(keys, out=out)
        e.record(stream)
        e.synchronize()
        if i >= warmup:
            times.append(s.elapsed_time(e))
    times.sort()
    return times[len(times) // 2]


def sweep(torch, f: Filter, keys_add, keys_q, out, regime: str, kpts=(1, 2, 4), block_threads=(256,),
          flags=0, reps: int = 5, flush=None, log=None, partitions=None, lookup_partitions=None) -> dict:
    """Time every layout of both operations; returns the table entry (and rows).

    ``partitions`` / ``lookup_partitions``: lists of slice-partitioning
    settings (dicts for ``Filter.set_partition``) to sweep for construction /
    lookup, or None to keep the filter's setting.  The lookup sweep runs with
    the best construction setting applied (they share the slice geometry).
    """
    p = f.params
    rows = []
    best = {}
    for op, name, keys in ((BF_OP_ADD, "add", keys_add), (BF_OP_CONTAINS, "contains", keys_q)):
        parts = partitions if op == BF_OP_ADD else lookup_partitions
        if op == BF_OP_CONTAINS and best.get("add", {}).get("layout", {}).get("partition"):
            f.set_partition(**best["add"]["layout"]["partition"])
        for part in ([None] if parts is None else parts):
            if part is not None:
                f.set_partition(**part)
            for cg, phi in valid_layouts(p.block_bits, p.word_bits):
                for kpt in kpts:
                    for bt in block_threads:
                        lay = dict(cg=cg, phi=phi, kpt=kpt, block_threads=bt, flags=flags)
                        f.set_layout(op, **lay)
                        ms = time_op(torch, f, op, keys, out, reps=reps, flush=flush)
                        g = keys.numel() / (ms * 1e-3) / 1e9
                        if part is not None:
                            lay = dict(lay, partition=part)
                        row = dict(op=name, gkeys_s=g, ms=ms, **lay)
                        rows.append(row)
                        if log:
                            log(row)
                        if name not in best or g > best[name]["gkeys_s"]:
                            best[name] = dict(gkeys_s=g, layout=lay)
    entry = {"add": best["add"], "contains": best["contains"],
             "n_add": keys_add.numel(), "n_contains": keys_q.numel(), "filter_bytes": f.nbytes}
    return {"key": key_of(p.block_bits, p.word_bits, p.k, regime), "entry": entry, "rows": rows}


# --- batched filters ---------------------------------------------------------
#
# A batch fixes one geometry for all its filters; the autotuner times every
# compiled layout (Theta, Phi, keys per thread) of the batched add and
# contains launches, and, across geometries with the same K at the same bytes
# per filter, picks the block width (and word size) of the fastest build +
# probe step whose measured false-positive count stays within the binomial
# 3-sigma band of a reference geometry's.


def batch_key(block_bits: int, word_bits: int, k: int) -> str:
    return f"batch_B{block_bits}_S{word_bits}_K{k}"


def tuned_batch_layout(block_bits: int, word_bits: int, k: int, op: int) -> dict | None:
    entry = load_tuned().get(batch_key(block_bits, word_bits, k))
    if not entry:
        return None
    return entry.get("add" if op == BF_OP_ADD else "contains", {}).get("layout")


def time_call(torch, fn, reps: int = 5, warmup: int = 2) -> float:
    """Median device time (ms) of fn() on the current stream."""
    stream = torch.cuda.current_stream()
    times = []
    for i in range(warmup + reps):
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        fn()
        e.record(stream)
        e.synchronize()
        if i >= warmup:
            times.append(s.elapsed_time(e))
    times.sort()
    return times[len(times) // 2]


def sweep_batch(torch, batch, keys_add, keys_q, out, kpts=(1, 2, 4), reps: int = 5, log=None,
                flag_sets=(0,), grids=(0,)) -> dict:
    """Time every layout of the batched add and contains; returns the table entry.

    ``batch``: a :class:`Batch`; its layouts are left at the best found.
    ``flag_sets``: layout flag values to try with every layout (e.g. with and
    without the L2 prefetch hint); ``grids``: CTA counts to try (0 = SMs x
    resident CTAs per SM).  A smaller grid narrows the run of filters the
    warps work on at a time, which decides how much of it stays in L2.
    """
    p = batch.params
    rows, best = [], {}
    for op, name in ((BF_OP_ADD, "add"), (BF_OP_CONTAINS, "contains")):
        if op == BF_OP_ADD:
            fn = lambda: batch.add(keys_add)  # noqa: E731
        else:
            fn = lambda: batch.contains(keys_q, out=out)  # noqa: E731
        for cg, phi in valid_layouts(p.block_bits, p.word_bits):
            for kpt in kpts:
                for flags in flag_sets:
                    for grid in grids:
                        lay = dict(cg=cg, phi=phi, kpt=kpt, flags=flags, grid_ctas=grid)
                        batch.set_layout(op, **lay)
                        ms = time_call(torch, fn, reps=reps)
                        g = batch.total_keys / (ms * 1e-3) / 1e9
                        row = dict(op=name, gkeys_s=g, ms=ms, **lay)
                        rows.append(row)
                        if log:
                            log(row)
                        if name not in best or ms < best[name]["ms"]:
                            best[name] = dict(gkeys_s=g, ms=ms, layout=lay)
        batch.set_layout(op, **best[name]["layout"])
    entry = {"add": best["add"], "contains": best["contains"], "step_ms": best["add"]["ms"] + best["contains"]["ms"],
             "filters": batch.nfilters, "keys": batch.total_keys}
    return {"key": batch_key(p.block_bits, p.word_bits, p.k), "entry": entry, "rows": rows}


def fp_count_limit(reference_count: int) -> float:
    """Upper end of the 3-sigma band of a false-positive count (Poisson
    approximation of the binomial, at least one count of width)."""
    return reference_count + 3.0 * max(1.0, reference_count) ** 0.5


def choose_batch_geometry(results: list, reference: tuple, min_gain: float = 0.03) -> dict:
    """Pick the fastest geometry whose false positives stay within the band.

    ``results``: dicts with block_bits, word_bits, k, step_ms, fp (false
    positives among ``queries`` non-member queries), queries.  ``reference``:
    (block_bits, word_bits) of the geometry whose count sets the band.  Another
    geometry replaces the reference only if its step is at least ``min_gain``
    (a fraction) faster, so that timing noise does not trade FPR for nothing.
    """
    ref = [r for r in results if (r["block_bits"], r["word_bits"]) == tuple(reference)]
    if not ref:
        raise ValueError("reference geometry not among the results")
    limit = fp_count_limit(ref[0]["fp"])
    ok = [r for r in results if r["fp"] <= limit]
    best = min(ok, key=lambda r: r["step_ms"])
    if best["step_ms"] > ref[0]["step_ms"] * (1.0 - min_gain):
        best = ref[0]
    return {"block_bits": best["block_bits"], "word_bits": best["word_bits"], "k": best["k"],
            "step_ms": best["step_ms"], "fp": best["fp"], "fp_limit": limit,
            "reference": {"block_bits": reference[0], "word_bits": reference[1], "fp": ref[0]["fp"],
                          "step_ms": ref[0]["step_ms"]},
            "min_gain": min_gain, "queries": best["queries"]}
