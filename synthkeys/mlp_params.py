"""Seeded random float32 parameters of the prefilter network (64 -> 128 -> 64 -> 1),
for parity tests; no network arithmetic.  Layout of the flat vector (also the
CUDA path's): W1 [64][128], b1 [128], W2 [128][64], b2 [64], W3 [64], b3 [1]."""
from __future__ import annotations

import numpy as np

SHAPES = (("W1", (64, 128)), ("b1", (128,)), ("W2", (128, 64)), ("b2", (64,)), ("W3", (64,)), ("b3", (1,)))
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def init_params(seed: int = 0, scale: float = 0.2) -> dict:
    rng = np.random.default_rng(seed)
    f = np.float32
    return {"W1": (rng.standard_normal((64, 128)) * scale / 8).astype(f),
            "b1": (rng.standard_normal(128) * scale).astype(f),
            "W2": (rng.standard_normal((128, 64)) * scale / 11).astype(f),
            "b2": (rng.standard_normal(64) * scale).astype(f),
            "W3": (rng.standard_normal(64) * scale / 8).astype(f),
            "b3": np.array([rng.standard_normal() * scale], dtype=f)}


def flatten(p: dict) -> np.ndarray:
    return np.concatenate([p[k].reshape(-1) for k, _ in SHAPES]).astype(np.float32)


def unflatten(v: np.ndarray) -> dict:
    out, o = {}, 0
    for k, s in SHAPES:
        n = int(np.prod(s))
        out[k] = np.asarray(v[o:o + n], dtype=np.float32).reshape(s)
        o += n
    return out
