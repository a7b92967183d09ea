"""ctypes binding of libbloomgb.so (include/bloomgb.h).

Argument marshalling only: every step of construction and lookup runs in the
library's CUDA kernels.  The functions keep the C names; a non-OK status
raises :class:`BloomError`.  If the library is missing this module raises on
first use: there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "_build", "libbloomgb.so")

BF_OK, BF_EINVAL, BF_ENOMEM, BF_ECUDA, BF_EUNSUPPORTED, BF_ETIMEDOUT = range(6)
BF_OP_ADD, BF_OP_CONTAINS = 0, 1
BF_HINT_FILTER_EVICT_LAST = 1 << 0
BF_HINT_KEYS_EVICT_NORMAL = 1 << 1
BF_HINT_PREFETCH_L2 = 1 << 2
BF_HINT_WARP_AGGREGATE = 1 << 3
BF_GUPS_LOAD, BF_GUPS_RED_OR, BF_GUPS_RED_OR_SECTOR = 0, 1, 2
BF_HOST_AUTO, BF_HOST_STAGED, BF_HOST_DIRECT = 0, 1, 2

# every symbol include/bloomgb.h declares
EXPORTED = (
    "bf_params_check", "bf_layout_check", "bf_create", "bf_destroy", "bf_clear", "bf_add",
    "bf_contains", "bf_add_host", "bf_contains_host", "bf_set_staging", "bf_words",
    "bf_get_params", "bf_set_layout", "bf_get_layout", "bf_set_l2_persist", "bf_gups",
    "bf_set_partition", "bf_get_partition", "bf_last_launches", "bf_set_timing", "bf_get_timing",
    "bf_device_status", "bf_add_noalloc", "bf_noalloc_status", "bf_batch_create",
    "bf_batch_destroy", "bf_batch_set_layout", "bf_batch_get_layout", "bf_batch_add", "bf_batch_contains",
    "bf_batch_info", "bf_server_create", "bf_server_destroy", "bf_server_submit", "bf_server_wait",
    "bf_server_get_stats", "bf_server_run_poisson", "bf_mlp_workspace_bytes", "bf_mlp_grad", "bf_mlp_adam",
    "bf_mlp_train", "bf_mlp_export", "bf_mlp_load", "bf_mlp_free", "bf_mlp_scores", "bf_mlp_select_below",
    "bf_mlp_contains", "bf_mlp_contains_host", "bf_mlp_set_engine", "bf_mlp_get_engine", "bf_mlp_check", "bf_mma_cost", "bf_status_str", "bf_last_error", "bf_version",
)

BF_MLP_PARAMS = 16641
BF_MLP_ENGINE_AUTO, BF_MLP_ENGINE_TENSOR, BF_MLP_ENGINE_DP4A = 0, 1, 2


class BloomError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: {_STATUS.get(status, status)}: {msg}")
        self.status = status


_STATUS = {0: "BF_OK", 1: "BF_EINVAL", 2: "BF_ENOMEM", 3: "BF_ECUDA", 4: "BF_EUNSUPPORTED", 5: "BF_ETIMEDOUT"}


BF_SALTS_DEFAULT, BF_SALTS_PARQUET = 0, 1


class bf_params(ctypes.Structure):
    _fields_ = [("num_blocks", ctypes.c_uint64), ("block_bits", ctypes.c_uint32),
                ("word_bits", ctypes.c_uint32), ("k", ctypes.c_uint32),
                ("groups", ctypes.c_uint32), ("seed", ctypes.c_uint64),
                ("salts", ctypes.c_uint32), ("reserved", ctypes.c_uint32)]


BF_PART_OFF, BF_PART_ON, BF_PART_AUTO = 0, 1, 2


class bf_partition(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_uint32), ("slice_log2", ctypes.c_uint32),
                ("chunk_keys", ctypes.c_uint64), ("cap_override", ctypes.c_uint64),
                ("window_log2", ctypes.c_uint32), ("lookup_mode", ctypes.c_uint32),
                ("lookup_chunk_keys", ctypes.c_uint64), ("passes", ctypes.c_uint32),
                ("part_ctas", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


BF_PHASES = 8
PHASE_NAMES = ("add_direct", "contains_direct", "partition_add", "record_insert", "partition_lookup",
               "record_probe", "bitmap_expand", "host_stage")


class bf_timing(ctypes.Structure):
    _fields_ = [("ms", ctypes.c_float * BF_PHASES), ("launches", ctypes.c_uint32 * BF_PHASES)]

    def as_dict(self):
        return {name: {"ms": self.ms[i], "launches": self.launches[i]}
                for i, name in enumerate(PHASE_NAMES) if self.launches[i] or self.ms[i] > 0}


class bf_batch_filter(ctypes.Structure):
    _fields_ = [("d_words", ctypes.c_void_p), ("num_blocks", ctypes.c_uint64),
                ("key_offset", ctypes.c_uint64), ("key_count", ctypes.c_uint64)]


class bf_server_stats_t(ctypes.Structure):
    _fields_ = [("requests", ctypes.c_uint64), ("keys", ctypes.c_uint64), ("launches", ctypes.c_uint64),
                ("p50_s", ctypes.c_double), ("p99_s", ctypes.c_double), ("mean_s", ctypes.c_double),
                ("max_s", ctypes.c_double), ("span_s", ctypes.c_double), ("offered_s", ctypes.c_double),
                ("stage_in_s", ctypes.c_double), ("lookup_s", ctypes.c_double), ("stage_out_s", ctypes.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class bf_layout(ctypes.Structure):
    _fields_ = [("cg", ctypes.c_uint32), ("phi", ctypes.c_uint32), ("kpt", ctypes.c_uint32),
                ("block_threads", ctypes.c_uint32), ("grid_ctas", ctypes.c_uint32),
                ("flags", ctypes.c_uint32)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class bf_mlp_int8(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_int8 * (64 * 128)), ("w2", ctypes.c_int8 * (128 * 64)), ("w3", ctypes.c_int8 * 64),
                ("b1", ctypes.c_int32 * 128), ("b2", ctypes.c_int32 * 64), ("b3", ctypes.c_int32),
                ("sh1", ctypes.c_int32), ("sh2", ctypes.c_int32), ("unit", ctypes.c_double)]


_lib = None


def lib():
    """Load the library (built by ``paper_2512_15595_gb300.build``)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libbloomgb.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    u64, u32, vp, i32 = ctypes.c_uint64, ctypes.c_uint32, ctypes.c_void_p, ctypes.c_int
    P, LY = ctypes.POINTER(bf_params), ctypes.POINTER(bf_layout)
    sigs = {
        "bf_params_check": (i32, [P]),
        "bf_layout_check": (i32, [P, i32, LY]),
        "bf_create": (i32, [P, vp, ctypes.POINTER(vp)]),
        "bf_destroy": (i32, [vp]),
        "bf_clear": (i32, [vp, vp]),
        "bf_add": (i32, [vp, vp, u64, vp]),
        "bf_contains": (i32, [vp, vp, u64, vp, vp]),
        "bf_add_host": (i32, [vp, vp, u64, vp]),
        "bf_contains_host": (i32, [vp, vp, u64, vp, vp]),
        "bf_set_staging": (i32, [vp, u64, i32]),
        "bf_words": (i32, [vp, ctypes.POINTER(vp), ctypes.POINTER(u64)]),
        "bf_get_params": (i32, [vp, P]),
        "bf_set_layout": (i32, [vp, i32, LY]),
        "bf_get_layout": (i32, [vp, i32, LY]),
        "bf_set_l2_persist": (i32, [vp, vp, ctypes.c_float]),
        "bf_gups": (i32, [i32, vp, u64, u32, vp, u64, vp, LY, vp]),
        "bf_set_partition": (i32, [vp, ctypes.POINTER(bf_partition)]),
        "bf_device_status": (i32, [vp, vp, ctypes.POINTER(ctypes.c_uint32)]),
        "bf_set_timing": (i32, [vp, ctypes.c_int]),
        "bf_get_timing": (i32, [vp, ctypes.POINTER(bf_timing)]),
        "bf_noalloc_status": (i32, [ctypes.POINTER(ctypes.c_uint32)]),
        "bf_get_partition": (i32, [vp, ctypes.POINTER(bf_partition)]),
        "bf_last_launches": (i32, [vp, ctypes.POINTER(u32)]),
        "bf_add_noalloc": (i32, [P, vp, vp, u64, ctypes.POINTER(u64), vp]),
        "bf_batch_create": (i32, [P, ctypes.POINTER(bf_batch_filter), u32, ctypes.POINTER(vp)]),
        "bf_batch_destroy": (i32, [vp]),
        "bf_batch_set_layout": (i32, [vp, i32, LY]),
        "bf_batch_get_layout": (i32, [vp, i32, LY]),
        "bf_batch_add": (i32, [vp, vp, vp]),
        "bf_batch_contains": (i32, [vp, vp, vp, vp]),
        "bf_batch_info": (i32, [vp, ctypes.POINTER(u32), ctypes.POINTER(u64)]),
        "bf_server_create": (i32, [P, ctypes.POINTER(bf_batch_filter), u32, u64, u32, ctypes.POINTER(vp)]),
        "bf_server_destroy": (i32, [vp]),
        "bf_server_submit": (i32, [vp, u32, vp, u64, vp, ctypes.POINTER(u64)]),
        "bf_server_wait": (i32, [vp, u64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
        "bf_server_get_stats": (i32, [vp, i32, ctypes.POINTER(bf_server_stats_t)]),
        "bf_server_run_poisson": (i32, [vp, ctypes.c_double, ctypes.c_double, u64, u64, vp, u64, vp, u64,
                                        ctypes.POINTER(bf_server_stats_t)]),
        "bf_mlp_workspace_bytes": (u64, [u32]),
        "bf_mlp_grad": (i32, [vp, vp, vp, u64, u64, u64, u32, vp, vp, vp, u64, vp]),
        "bf_mlp_adam": (i32, [vp, vp, vp, vp, u32, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                              ctypes.c_float, vp]),
        "bf_mlp_train": (i32, [vp, vp, vp, vp, vp, u64, u64, u32, u32, u32, ctypes.c_float, ctypes.c_float,
                               ctypes.c_float, ctypes.c_float, vp, vp, u64, vp]),
        "bf_mlp_export": (i32, [vp, vp, u64, ctypes.POINTER(bf_mlp_int8), vp]),
        "bf_mlp_load": (i32, [ctypes.POINTER(bf_mlp_int8), ctypes.POINTER(vp)]),
        "bf_mlp_free": (i32, [vp]),
        "bf_mlp_scores": (i32, [vp, vp, u64, vp, vp]),
        "bf_mlp_select_below": (i32, [vp, i32, vp, u64, vp, vp, vp]),
        "bf_mlp_contains": (i32, [vp, i32, vp, vp, u64, vp, vp]),
        "bf_mlp_contains_host": (i32, [vp, i32, vp, vp, u64, vp, vp]),
        "bf_mlp_set_engine": (i32, [vp, i32]),
        "bf_mlp_get_engine": (i32, [vp, ctypes.POINTER(i32)]),
        "bf_mlp_check": (i32, [vp]),
        "bf_mma_cost": (i32, [u32, i32, u32, ctypes.POINTER(ctypes.c_double)]),
        "bf_status_str": (ctypes.c_char_p, [i32]),
        "bf_last_error": (ctypes.c_char_p, []),
        "bf_version": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype, f.argtypes = res, args
    _lib = L
    return L


def _check(status: int, where: str):
    if status != BF_OK:
        raise BloomError(status, where, lib().bf_last_error().decode())


def _stream(stream) -> int | None:
    """A torch.cuda.Stream, a raw handle (int) or None (torch's current stream)."""
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ---------------------------------------------------------------------------
# C entry points, same names
# ---------------------------------------------------------------------------
def bf_params_check(p: bf_params) -> int:
    return lib().bf_params_check(ctypes.byref(p))


def bf_layout_check(p: bf_params, op: int, layout: bf_layout | None) -> int:
    return lib().bf_layout_check(ctypes.byref(p), op, ctypes.byref(layout) if layout else None)


def bf_create(p: bf_params, d_words: int | None = None) -> int:
    h = ctypes.c_void_p()
    _check(lib().bf_create(ctypes.byref(p), d_words, ctypes.byref(h)), "bf_create")
    return h.value


def bf_destroy(f: int) -> None:
    _check(lib().bf_destroy(f), "bf_destroy")


def bf_clear(f: int, stream=None) -> None:
    _check(lib().bf_clear(f, _stream(stream)), "bf_clear")


def bf_add(f: int, d_keys: int, n: int, stream=None) -> None:
    _check(lib().bf_add(f, d_keys, n, _stream(stream)), "bf_add")


def bf_contains(f: int, d_keys: int, n: int, d_out: int, stream=None) -> None:
    _check(lib().bf_contains(f, d_keys, n, d_out, _stream(stream)), "bf_contains")


def bf_add_host(f: int, h_keys: int, n: int, stream=None) -> None:
    _check(lib().bf_add_host(f, h_keys, n, _stream(stream)), "bf_add_host")


def bf_contains_host(f: int, h_keys: int, n: int, h_out: int, stream=None) -> None:
    _check(lib().bf_contains_host(f, h_keys, n, h_out, _stream(stream)), "bf_contains_host")


def bf_set_staging(f: int, chunk_keys: int, mode: int = 0) -> None:
    _check(lib().bf_set_staging(f, chunk_keys, mode), "bf_set_staging")


def bf_words(f: int) -> tuple[int, int]:
    p, n = ctypes.c_void_p(), ctypes.c_uint64()
    _check(lib().bf_words(f, ctypes.byref(p), ctypes.byref(n)), "bf_words")
    return p.value, n.value


def bf_get_params(f: int) -> bf_params:
    p = bf_params()
    _check(lib().bf_get_params(f, ctypes.byref(p)), "bf_get_params")
    return p


def bf_set_layout(f: int, op: int, layout: bf_layout) -> None:
    _check(lib().bf_set_layout(f, op, ctypes.byref(layout)), "bf_set_layout")


def bf_get_layout(f: int, op: int) -> bf_layout:
    out = bf_layout()
    _check(lib().bf_get_layout(f, op, ctypes.byref(out)), "bf_get_layout")
    return out


def bf_set_l2_persist(f: int, hit_ratio: float, stream=None) -> None:
    _check(lib().bf_set_l2_persist(f, _stream(stream), hit_ratio), "bf_set_l2_persist")


def bf_gups(mode: int, d_table: int, table_bytes: int, unit_bytes: int, d_keys: int, n: int,
            d_out: int | None, layout: bf_layout | None = None, stream=None) -> None:
    _check(lib().bf_gups(mode, d_table, table_bytes, unit_bytes, d_keys, n, d_out,
                         ctypes.byref(layout) if layout else None, _stream(stream)), "bf_gups")


def bf_set_partition(f: int, cfg: bf_partition) -> None:
    _check(lib().bf_set_partition(f, ctypes.byref(cfg)), "bf_set_partition")


def bf_device_status(f: int, stream=None) -> int:
    """Index-check bits of the filter's slice-partitioned kernels since the
    last call (0 = none); waits for the stream."""
    v = ctypes.c_uint32()
    _check(lib().bf_device_status(f, _stream(stream), ctypes.byref(v)), "bf_device_status")
    return v.value


def bf_set_timing(f: int, enable: bool) -> None:
    _check(lib().bf_set_timing(f, int(bool(enable))), "bf_set_timing")


def bf_get_timing(f: int) -> dict:
    """Per-phase device time (ms) and launch count since the last read."""
    out = bf_timing()
    _check(lib().bf_get_timing(f, ctypes.byref(out)), "bf_get_timing")
    return out.as_dict()


def bf_get_partition(f: int) -> bf_partition:
    out = bf_partition()
    _check(lib().bf_get_partition(f, ctypes.byref(out)), "bf_get_partition")
    return out


def bf_last_launches(f: int) -> int:
    n = ctypes.c_uint32()
    _check(lib().bf_last_launches(f, ctypes.byref(n)), "bf_last_launches")
    return n.value


def bf_status_str(s: int) -> str:
    return lib().bf_status_str(s).decode()


def bf_last_error() -> str:
    return lib().bf_last_error().decode()


def bf_version() -> str:
    return lib().bf_version().decode()


def bf_batch_create(p: bf_params, filters) -> int:
    """filters: sequence of bf_batch_filter (or (d_words, num_blocks, key_offset, key_count))."""
    arr = (bf_batch_filter * len(filters))(*[f if isinstance(f, bf_batch_filter) else bf_batch_filter(*f)
                                              for f in filters])
    h = ctypes.c_void_p()
    _check(lib().bf_batch_create(ctypes.byref(p), arr, len(filters), ctypes.byref(h)), "bf_batch_create")
    return h.value


def bf_batch_destroy(b: int) -> None:
    _check(lib().bf_batch_destroy(b), "bf_batch_destroy")


def bf_batch_set_layout(b: int, op: int, layout: bf_layout) -> None:
    _check(lib().bf_batch_set_layout(b, op, ctypes.byref(layout)), "bf_batch_set_layout")


def bf_batch_get_layout(b: int, op: int) -> bf_layout:
    out = bf_layout()
    _check(lib().bf_batch_get_layout(b, op, ctypes.byref(out)), "bf_batch_get_layout")
    return out


def bf_batch_add(b: int, d_keys: int, stream=None) -> None:
    _check(lib().bf_batch_add(b, d_keys, _stream(stream)), "bf_batch_add")


def bf_batch_contains(b: int, d_keys: int, d_out: int, stream=None) -> None:
    _check(lib().bf_batch_contains(b, d_keys, d_out, _stream(stream)), "bf_batch_contains")


def bf_batch_info(b: int) -> tuple[int, int]:
    n, k = ctypes.c_uint32(), ctypes.c_uint64()
    _check(lib().bf_batch_info(b, ctypes.byref(n), ctypes.byref(k)), "bf_batch_info")
    return n.value, k.value


def bf_server_create(p: bf_params, filters, arena_keys: int, max_requests_per_launch: int = 4096) -> int:
    """filters: sequence of (d_words, num_blocks)."""
    arr = (bf_batch_filter * len(filters))(*[bf_batch_filter(w, nb, 0, 0) for w, nb in filters])
    h = ctypes.c_void_p()
    _check(lib().bf_server_create(ctypes.byref(p), arr, len(filters), arena_keys, max_requests_per_launch,
                                  ctypes.byref(h)), "bf_server_create")
    return h.value


def bf_server_destroy(s: int) -> None:
    _check(lib().bf_server_destroy(s), "bf_server_destroy")


def bf_server_submit(s: int, filt: int, h_keys: int, n: int, h_out: int) -> int:
    t = ctypes.c_uint64()
    _check(lib().bf_server_submit(s, filt, h_keys, n, h_out, ctypes.byref(t)), "bf_server_submit")
    return t.value


def bf_server_wait(s: int, ticket: int, timeout_s: float = 60.0) -> float:
    lat = ctypes.c_double()
    _check(lib().bf_server_wait(s, ticket, timeout_s, ctypes.byref(lat)), "bf_server_wait")
    return lat.value


def bf_server_get_stats(s: int, reset: bool = False) -> dict:
    out = bf_server_stats_t()
    _check(lib().bf_server_get_stats(s, int(reset), ctypes.byref(out)), "bf_server_get_stats")
    return out.as_dict()


def bf_server_run_poisson(s: int, rate_per_s: float, duration_s: float, min_keys: int, max_keys: int,
                          h_key_pool: int, pool_keys: int, h_out_pool: int, seed: int = 1) -> dict:
    out = bf_server_stats_t()
    _check(lib().bf_server_run_poisson(s, rate_per_s, duration_s, min_keys, max_keys, h_key_pool, pool_keys,
                                       h_out_pool, seed, ctypes.byref(out)), "bf_server_run_poisson")
    return out.as_dict()


def bf_mlp_workspace_bytes(batch: int) -> int:
    return lib().bf_mlp_workspace_bytes(batch)


def bf_mlp_grad(d_params: int, d_keys: int, d_labels: int, n: int, first: int, mult: int, batch: int,
                d_grads: int, d_loss: int | None, d_ws: int, ws_bytes: int, stream=None) -> None:
    _check(lib().bf_mlp_grad(d_params, d_keys, d_labels, n, first, mult, batch, d_grads, d_loss, d_ws, ws_bytes,
                             _stream(stream)), "bf_mlp_grad")


def bf_mlp_adam(d_params: int, d_grads: int, d_m: int, d_v: int, step: int, lr: float, beta1: float = 0.9,
                beta2: float = 0.999, eps: float = 1e-8, stream=None) -> None:
    _check(lib().bf_mlp_adam(d_params, d_grads, d_m, d_v, step, lr, beta1, beta2, eps, _stream(stream)),
           "bf_mlp_adam")


def bf_mlp_train(d_params: int, d_m: int, d_v: int, d_keys: int, d_labels: int, n: int, mult: int, batch: int,
                 first_step: int, steps: int, lr: float, beta1: float, beta2: float, eps: float,
                 d_loss: int | None, d_ws: int, ws_bytes: int, stream=None) -> None:
    _check(lib().bf_mlp_train(d_params, d_m, d_v, d_keys, d_labels, n, mult, batch, first_step, steps, lr, beta1,
                              beta2, eps, d_loss, d_ws, ws_bytes, _stream(stream)), "bf_mlp_train")


def bf_mlp_export(h_params: int, d_calib: int, n_calib: int, stream=None) -> bf_mlp_int8:
    out = bf_mlp_int8()
    _check(lib().bf_mlp_export(h_params, d_calib, n_calib, ctypes.byref(out), _stream(stream)), "bf_mlp_export")
    return out


def bf_mlp_load(m: bf_mlp_int8) -> int:
    h = ctypes.c_void_p()
    _check(lib().bf_mlp_load(ctypes.byref(m), ctypes.byref(h)), "bf_mlp_load")
    return h.value


def bf_mlp_free(m: int) -> None:
    _check(lib().bf_mlp_free(m), "bf_mlp_free")


def bf_mlp_scores(m: int, d_keys: int, n: int, d_scores: int, stream=None) -> None:
    _check(lib().bf_mlp_scores(m, d_keys, n, d_scores, _stream(stream)), "bf_mlp_scores")


def bf_mlp_select_below(m: int, tau: int, d_keys: int, n: int, d_out_keys: int, d_count: int, stream=None) -> None:
    _check(lib().bf_mlp_select_below(m, tau, d_keys, n, d_out_keys, d_count, _stream(stream)),
           "bf_mlp_select_below")


def bf_mlp_contains(m: int, tau: int, backup: int, d_keys: int, n: int, d_out: int, stream=None) -> None:
    _check(lib().bf_mlp_contains(m, tau, backup, d_keys, n, d_out, _stream(stream)), "bf_mlp_contains")


def bf_mlp_set_engine(m: int, engine: int) -> None:
    _check(lib().bf_mlp_set_engine(m, engine), "bf_mlp_set_engine")


def bf_mlp_get_engine(m: int) -> int:
    e = ctypes.c_int()
    _check(lib().bf_mlp_get_engine(m, ctypes.byref(e)), "bf_mlp_get_engine")
    return e.value


def bf_mlp_check(m: int) -> None:
    _check(lib().bf_mlp_check(m), "bf_mlp_check")


def bf_mlp_contains_host(m: int, tau: int, backup: int, h_keys: int, n: int, h_out: int, stream=None) -> None:
    _check(lib().bf_mlp_contains_host(m, tau, backup, h_keys, n, h_out, _stream(stream)), "bf_mlp_contains_host")


def bf_mma_cost(n: int, a_tmem: bool, reps: int = 4096) -> float:
    c = ctypes.c_double()
    _check(lib().bf_mma_cost(n, int(a_tmem), reps, ctypes.byref(c)), "bf_mma_cost")
    return c.value
