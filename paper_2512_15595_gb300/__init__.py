"""Sectorized blocked Bloom filter on one GB300 (sm_103a).

The compute path is the CUDA library ``_build/libbloomgb.so`` (C ABI in
``include/bloomgb.h``); this package is its thin Python binding.  PyTorch
supplies device memory and streams.  :class:`Filter` is a convenience
wrapper over the ``bf_*`` functions for torch tensors.
"""
from __future__ import annotations

from . import _lib
from ._lib import (BF_GUPS_LOAD, BF_GUPS_RED_OR, BF_GUPS_RED_OR_SECTOR, BF_HINT_FILTER_EVICT_LAST, BF_HINT_KEYS_EVICT_NORMAL,
                   BF_HINT_PREFETCH_L2, BF_HINT_WARP_AGGREGATE, BF_OP_ADD, BF_OP_CONTAINS, BloomError, bf_layout,
                   bf_params)

__all__ = ["Filter", "BloomError", "bf_params", "bf_layout", "BF_OP_ADD", "BF_OP_CONTAINS",
           "BF_HINT_FILTER_EVICT_LAST", "BF_HINT_KEYS_EVICT_NORMAL", "BF_HINT_PREFETCH_L2", "BF_HINT_WARP_AGGREGATE",
           "BF_GUPS_LOAD",
           "BF_GUPS_RED_OR", "BF_GUPS_RED_OR_SECTOR",
           "valid_layouts", "device_tensor", "Batch"]


def valid_layouts(block_bits: int, word_bits: int):
    """All (cg, phi) pairs of Sec. IV-A: powers of two with 1 <= cg*phi <= s."""
    s = block_bits // word_bits
    out = []
    cg = 1
    while cg <= s:
        phi = 1
        while cg * phi <= s:
            out.append((cg, phi))
            phi *= 2
        cg *= 2
    return out


class _DevBuf:
    def __init__(self, ptr: int, nbytes: int):
        self.__cuda_array_interface__ = {"shape": (nbytes,), "typestr": "|u1", "data": (ptr, False),
                                         "version": 3, "strides": None}


def device_tensor(ptr: int, nbytes: int, device):
    """A torch uint8 view of device memory the library owns (no copy)."""
    import torch
    return torch.as_tensor(_DevBuf(ptr, nbytes), device=device)


def _key_ptr(keys):
    import torch
    if not keys.is_cuda:
        raise ValueError("keys must be a CUDA tensor")
    if keys.dtype not in (torch.int64, getattr(torch, "uint64", torch.int64)):
        raise ValueError("keys must be int64 or uint64 (the 64-bit key bit pattern)")
    if not keys.is_contiguous():
        raise ValueError("keys must be contiguous")
    return keys.data_ptr(), keys.numel()


class Filter:
    """A filter whose bit array is a torch tensor (adopted by the library)."""

    def __init__(self, num_blocks: int, block_bits: int = 256, word_bits: int = 32, k: int = 8,
                 seed: int = 0, device=None, words=None, groups: int = 0, salts: int = 0):
        """salts = 1: the Parquet split-block salt set (256/32/8 only; with seed
        0 the bit array is the one a Parquet writer stores)."""
        import torch
        self.params = bf_params(num_blocks, block_bits, word_bits, k, groups, seed, salts, 0)
        self.nbytes = num_blocks * block_bits // 8
        if words is None:
            device = torch.device(device or "cuda")
            words = torch.zeros(self.nbytes, dtype=torch.uint8, device=device)
        if not words.is_cuda or words.numel() * words.element_size() != self.nbytes or not words.is_contiguous():
            raise ValueError("words must be a contiguous CUDA tensor of num_blocks*block_bits/8 bytes")
        self.words = words
        self.device = words.device
        with torch.cuda.device(self.device):
            self.handle = _lib.bf_create(self.params, words.data_ptr())

    # -- operations ------------------------------------------------------
    def add(self, keys, stream=None) -> None:
        ptr, n = _key_ptr(keys)
        _lib.bf_add(self.handle, ptr, n, stream)

    def contains(self, keys, out=None, stream=None):
        import torch
        ptr, n = _key_ptr(keys)
        if out is None:
            out = torch.empty(n, dtype=torch.bool, device=keys.device)
        if out.numel() != n or out.element_size() != 1 or not out.is_contiguous():
            raise ValueError("out must be a contiguous 1-byte tensor with one element per key")
        _lib.bf_contains(self.handle, ptr, n, out.data_ptr(), stream)
        return out

    def add_host(self, keys_np, stream=None) -> None:
        """Construction from a host numpy uint64/int64 array (bf_add_host)."""
        _lib.bf_add_host(self.handle, keys_np.ctypes.data, keys_np.size, stream)

    def contains_host(self, keys_np, out_np, stream=None) -> None:
        """Lookup of host queries into a host uint8 array (bf_contains_host)."""
        _lib.bf_contains_host(self.handle, keys_np.ctypes.data, keys_np.size, out_np.ctypes.data, stream)

    def set_staging(self, chunk_keys: int = 1 << 24, mode: str = "auto") -> None:
        """Host-variant settings (bf_set_staging): chunk size of the chunked
        way, and mode "auto", "staged" (the kernels never read host memory)
        or "direct" (they read it in place whenever they can address it)."""
        modes = {"auto": _lib.BF_HOST_AUTO, "staged": _lib.BF_HOST_STAGED, "direct": _lib.BF_HOST_DIRECT}
        _lib.bf_set_staging(self.handle, chunk_keys, modes[mode])

    def clear(self, stream=None) -> None:
        _lib.bf_clear(self.handle, stream)

    def set_layout(self, op: int, cg: int = 0, phi: int = 0, kpt: int = 0, block_threads: int = 0,
                   grid_ctas: int = 0, flags: int = 0) -> None:
        _lib.bf_set_layout(self.handle, op, bf_layout(cg, phi, kpt, block_threads, grid_ctas, flags))

    def layout(self, op: int) -> dict:
        return _lib.bf_get_layout(self.handle, op).as_dict()

    def set_partition(self, mode: int | None = None, slice_log2: int | None = None, chunk_keys: int | None = None,
                      cap_override: int | None = None, window_log2: int | None = None,
                      lookup_mode: int | None = None, lookup_chunk_keys: int | None = None,
                      passes: int | None = None, part_ctas: int | None = None) -> None:
        """Slice-partitioned construction / lookup settings (modes: 0 off, 1 on,
        2 auto); arguments left as None keep their current value."""
        cur = _lib.bf_get_partition(self.handle)
        for name, val in (("mode", mode), ("slice_log2", slice_log2), ("chunk_keys", chunk_keys),
                          ("cap_override", cap_override), ("window_log2", window_log2),
                          ("lookup_mode", lookup_mode), ("lookup_chunk_keys", lookup_chunk_keys),
                          ("passes", passes), ("part_ctas", part_ctas)):
            if val is not None:
                setattr(cur, name, val)
        _lib.bf_set_partition(self.handle, cur)

    def partition(self) -> dict:
        return _lib.bf_get_partition(self.handle).as_dict()

    def set_timing(self, enable: bool = True) -> None:
        """Record per-phase device times of every call (bf_set_timing)."""
        _lib.bf_set_timing(self.handle, enable)

    def timing(self) -> dict:
        """Per-phase device time (ms) and launches since the last read."""
        return _lib.bf_get_timing(self.handle)

    def device_status(self, stream=None) -> int:
        """Bits of failed index checks in the slice-partitioned kernels since
        the last call (0 = none; waits for the stream)."""
        return _lib.bf_device_status(self.handle, stream)

    def last_launches(self) -> int:
        return _lib.bf_last_launches(self.handle)

    def set_l2_persist(self, hit_ratio: float, stream=None) -> None:
        _lib.bf_set_l2_persist(self.handle, hit_ratio, stream)

    def close(self) -> None:
        if getattr(self, "handle", None):
            _lib.bf_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many filters of one geometry built / probed by one launch per operation.

    ``filters``: list of (words_tensor, num_blocks, key_offset, key_count);
    every words tensor is a contiguous CUDA byte buffer of num_blocks*B/8
    bytes (slices of one arena are fine).  Keys and results are single arrays
    indexed by each filter's key run.
    """

    def __init__(self, filters, block_bits: int = 256, word_bits: int = 32, k: int = 8, seed: int = 0,
                 salts: int = 0):
        self.params = bf_params(1, block_bits, word_bits, k, 0, seed, salts, 0)
        self._keep = [f[0] for f in filters]
        descs = [(f[0].data_ptr(), f[1], f[2], f[3]) for f in filters]
        self.handle = _lib.bf_batch_create(self.params, descs)
        self.nfilters, self.total_keys = _lib.bf_batch_info(self.handle)

    def add(self, keys, stream=None) -> None:
        ptr, n = _key_ptr(keys)
        if n < self.total_keys:
            raise ValueError("key array shorter than the batch's key runs")
        _lib.bf_batch_add(self.handle, ptr, stream)

    def contains(self, keys, out=None, stream=None):
        import torch
        ptr, n = _key_ptr(keys)
        if n < self.total_keys:
            raise ValueError("key array shorter than the batch's key runs")
        if out is None:
            out = torch.zeros(n, dtype=torch.bool, device=keys.device)
        _lib.bf_batch_contains(self.handle, ptr, out.data_ptr(), stream)
        return out

    def set_layout(self, op: int, cg: int = 0, phi: int = 0, kpt: int = 0, block_threads: int = 0,
                   grid_ctas: int = 0, flags: int = 0) -> None:
        _lib.bf_batch_set_layout(self.handle, op, bf_layout(cg, phi, kpt, block_threads, grid_ctas, flags))

    def layout(self, op: int) -> dict:
        return _lib.bf_batch_get_layout(self.handle, op).as_dict()

    def close(self) -> None:
        if getattr(self, "handle", None):
            _lib.bf_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
