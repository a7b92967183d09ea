"""Learned prefilter: the ``bf_mlp_*`` entry points wrapped for torch tensors.

A network over the 64 key bits scores each key; keys scoring at least ``tau``
are reported present, and a backup blocked filter holds the members scored
below ``tau``, so no member is ever rejected.  Training, export calibration,
scoring, compaction of the false negatives and the combined lookup all run in
the library's kernels; this module allocates tensors and passes pointers.
"""
from __future__ import annotations

import math

import numpy as np

from . import _lib
from ._lib import BF_MLP_ENGINE_AUTO, BF_MLP_ENGINE_DP4A, BF_MLP_ENGINE_TENSOR, BF_MLP_PARAMS, bf_mlp_int8

__all__ = ["Trainer", "IntModel", "LearnedFilter", "BF_MLP_PARAMS", "coprime_multiplier", "BF_MLP_ENGINE_AUTO",
           "BF_MLP_ENGINE_TENSOR", "BF_MLP_ENGINE_DP4A"]


def coprime_multiplier(n: int, start: int = 0x9E3779B1) -> int:
    """A multiplier below 2^32 coprime to n (for the training-set permutation)."""
    m = start % (1 << 32) or 1
    while n > 1 and math.gcd(m, n) != 1:
        m = (m + 2) % (1 << 32) or 1
    return m


class Trainer:
    """fp32 parameters, Adam moments and the workspace of one training run."""

    def __init__(self, init_params: np.ndarray, batch: int = 4096, device=None):
        import torch
        if init_params.size != BF_MLP_PARAMS:
            raise ValueError(f"expected {BF_MLP_PARAMS} parameters")
        self.device = torch.device(device or "cuda")
        self.batch = batch
        self.params = torch.from_numpy(np.ascontiguousarray(init_params, dtype=np.float32)).to(self.device)
        self.m = torch.zeros_like(self.params)
        self.v = torch.zeros_like(self.params)
        self.ws_bytes = _lib.bf_mlp_workspace_bytes(batch)
        self.ws = torch.empty(self.ws_bytes, dtype=torch.uint8, device=self.device)
        self.step = 0

    def grad(self, keys, labels, first: int = 0, mult: int = 1, stream=None):
        """(gradient vector, loss) of one batch; both device tensors."""
        import torch
        g = torch.empty_like(self.params)
        loss = torch.empty(1, dtype=torch.float32, device=self.device)
        _lib.bf_mlp_grad(self.params.data_ptr(), keys.data_ptr(), labels.data_ptr(), keys.numel(), first, mult,
                         self.batch, g.data_ptr(), loss.data_ptr(), self.ws.data_ptr(), self.ws_bytes, stream)
        return g, loss

    def train(self, keys, labels, steps: int, lr: float = 1e-3, beta1: float = 0.9, beta2: float = 0.999,
              eps: float = 1e-8, mult: int | None = None, stream=None):
        """`steps` Adam steps over the (device) training set; returns the per-step losses (device)."""
        import torch
        n = keys.numel()
        if labels.numel() != n or labels.dtype != torch.float32:
            raise ValueError("labels: one float32 per key")
        mult = coprime_multiplier(n) if mult is None else mult
        losses = torch.empty(steps, dtype=torch.float32, device=self.device)
        _lib.bf_mlp_train(self.params.data_ptr(), self.m.data_ptr(), self.v.data_ptr(), keys.data_ptr(),
                          labels.data_ptr(), n, mult, self.batch, self.step + 1, steps, lr, beta1, beta2, eps,
                          losses.data_ptr(), self.ws.data_ptr(), self.ws_bytes, stream)
        self.step += steps
        return losses

    def export(self, calib_keys, stream=None) -> bf_mlp_int8:
        host = self.params.cpu().numpy()
        return _lib.bf_mlp_export(host.ctypes.data, calib_keys.data_ptr(), calib_keys.numel(), stream)


def int_model_arrays(m: bf_mlp_int8) -> dict:
    """The integer model as numpy arrays (W1q [64][128], W2q [128][64], ...)."""
    return {"W1q": np.ctypeslib.as_array(m.w1).reshape(64, 128).astype(np.int64),
            "b1q": np.ctypeslib.as_array(m.b1).astype(np.int64), "sh1": int(m.sh1),
            "W2q": np.ctypeslib.as_array(m.w2).reshape(128, 64).astype(np.int64),
            "b2q": np.ctypeslib.as_array(m.b2).astype(np.int64), "sh2": int(m.sh2),
            "W3q": np.ctypeslib.as_array(m.w3).astype(np.int64), "b3q": int(m.b3), "unit": float(m.unit)}


def model_bits() -> int:
    """Storage of the integer model: int8 weights, int32 biases, two shifts and tau."""
    return 8 * (64 * 128 + 128 * 64 + 64) + 32 * (128 + 64 + 1) + 32 * 3


class IntModel:
    """An exported integer model resident on the device."""

    def __init__(self, m: bf_mlp_int8, device=None):
        import torch
        self.int8 = m
        self.device = torch.device(device or "cuda")
        with torch.cuda.device(self.device):
            self.handle = _lib.bf_mlp_load(m)

    def set_engine(self, engine: int) -> None:
        _lib.bf_mlp_set_engine(self.handle, engine)

    @property
    def engine(self) -> int:
        return _lib.bf_mlp_get_engine(self.handle)

    def check(self) -> None:
        """Synchronize; raise if a bounded wait of a tensor-core launch ran out."""
        _lib.bf_mlp_check(self.handle)

    def scores(self, keys, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(keys.numel(), dtype=torch.int32, device=keys.device)
        _lib.bf_mlp_scores(self.handle, keys.data_ptr(), keys.numel(), out.data_ptr(), stream)
        return out

    def select_below(self, tau: int, keys, out=None, stream=None):
        """(device buffer, count): the keys scoring below tau, compacted (count read back: synchronizes)."""
        import torch
        if out is None:
            out = torch.empty(keys.numel(), dtype=keys.dtype, device=keys.device)
        cnt = torch.zeros(1, dtype=torch.int64, device=keys.device)
        _lib.bf_mlp_select_below(self.handle, int(tau), keys.data_ptr(), keys.numel(), out.data_ptr(),
                                 cnt.data_ptr(), stream)
        return out, int(cnt.item())

    def close(self):
        if getattr(self, "handle", None):
            _lib.bf_mlp_free(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class LearnedFilter:
    """Model + threshold + backup filter over a member set (no false negatives)."""

    def __init__(self, model: IntModel, tau: int, members, backup_blocks: int, block_bits: int = 256,
                 word_bits: int = 32, k: int = 8, seed: int = 0, stream=None):
        from . import Filter
        self.model, self.tau = model, int(tau)
        fn, self.n_backup = model.select_below(self.tau, members, stream=stream)
        self.backup = Filter(max(1, backup_blocks), block_bits, word_bits, k, seed, device=members.device)
        if self.n_backup:
            self.backup.add(fn[:self.n_backup], stream=stream)
        self.bits = self.backup.nbytes * 8 + model_bits()

    def contains(self, keys, out=None, stream=None):
        import torch
        if out is None:
            out = torch.empty(keys.numel(), dtype=torch.bool, device=keys.device)
        _lib.bf_mlp_contains(self.model.handle, self.tau, self.backup.handle, keys.data_ptr(), keys.numel(),
                             out.data_ptr(), stream)
        return out

    def contains_host(self, keys, out, stream=None) -> None:
        """Lookups from a host tensor (pinned for overlap) into a host bool/uint8 tensor."""
        if keys.is_cuda or out.is_cuda or out.numel() != keys.numel() or out.element_size() != 1:
            raise ValueError("host keys and a host 1-byte output of the same length")
        _lib.bf_mlp_contains_host(self.model.handle, self.tau, self.backup.handle, keys.data_ptr(), keys.numel(),
                                  out.data_ptr(), stream)
