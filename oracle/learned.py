"""CPU oracle of the learned prefilter (test infrastructure only).

Network: the 64 bits of a key (bit i = (key >> i) & 1, as 0/1 features) ->
128 ReLU units -> 64 ReLU units -> 1 logit.  Parameters: W1 [64][128],
b1 [128], W2 [128][64], b2 [64], W3 [64], b3 (scalar).

Training (fp64 here; Adam updates): weights are fake-quantized per layer, W_q = s * round(W / s)
with s = max|W| / 127 (round half away from zero, clamp to +-127), and the
gradient passes straight through the rounding (w.r.t. the float weights it
equals the gradient w.r.t. W_q).  Loss: mean binary cross-entropy with logits.

Integer inference (the exported model, reproduced exactly by the CUDA path):
    W1q = clamp(round(W1 / s1)), b1q = round(b1 / s1)              (x in {0,1})
    a1  = x . W1q + b1q ;            h1 = min(relu(a1) >> sh1, 127)
    W2q = clamp(round(W2 / s2)), b2q = round(b2 / (s1 2^sh1 s2))
    a2  = h1 . W2q + b2q ;           h2 = min(relu(a2) >> sh2, 127)
    W3q = clamp(round(W3 / s3)), b3q = round(b3 / (s1 2^sh1 s2 2^sh2 s3))
    score = clamp(h2 . W3q + b3q)     (saturated to int32; present iff score >= tau)
sh1 / sh2 are the smallest shifts that bring the largest relu(a1) / relu(a2)
over the calibration keys to <= 127.  Scales and quotients are computed in
fp64 from the fp32 parameters; biases saturate to the int32 range.
"""
from __future__ import annotations

import numpy as np

N_IN, N_H1, N_H2 = 64, 128, 64
INT32_MIN, INT32_MAX = -(2**31), 2**31 - 1


def features(keys) -> np.ndarray:
    k = np.asarray(keys, dtype=np.uint64)
    bits = (k[:, None] >> np.arange(64, dtype=np.uint64)[None, :]) & np.uint64(1)
    return bits.astype(np.float64)


def _round_half_away(x):
    return np.sign(x) * np.floor(np.abs(x) + 0.5)


def quant_scale(w: np.ndarray) -> float:
    m = float(np.max(np.abs(w.astype(np.float64)))) if w.size else 0.0
    return m / 127.0 if m > 0 else 1.0


def fake_quant(w: np.ndarray) -> np.ndarray:
    s = quant_scale(w)
    return np.clip(_round_half_away(w.astype(np.float64) / s), -127, 127) * s


def forward_backward(params: dict, keys, labels, quant: bool = True):
    """Mean BCE loss and its gradients w.r.t. every parameter (fp64)."""
    X = features(keys)
    y = np.asarray(labels, dtype=np.float64)
    n = X.shape[0]
    Wq = {k: (fake_quant(params[k]) if quant else params[k].astype(np.float64)) for k in ("W1", "W2", "W3")}
    b1, b2, b3 = (params[k].astype(np.float64) for k in ("b1", "b2", "b3"))
    Z1 = X @ Wq["W1"] + b1
    H1 = np.maximum(Z1, 0.0)
    Z2 = H1 @ Wq["W2"] + b2
    H2 = np.maximum(Z2, 0.0)
    Z3 = H2 @ Wq["W3"] + b3[0]
    loss = float(np.mean(np.maximum(Z3, 0) - Z3 * y + np.log1p(np.exp(-np.abs(Z3)))))
    dZ3 = (1.0 / (1.0 + np.exp(-Z3)) - y) / n
    g = {"W3": H2.T @ dZ3, "b3": np.array([dZ3.sum()])}
    dH2 = np.outer(dZ3, Wq["W3"])
    dZ2 = dH2 * (Z2 > 0)
    g["W2"] = H1.T @ dZ2
    g["b2"] = dZ2.sum(axis=0)
    dH1 = dZ2 @ Wq["W2"].T
    dZ1 = dH1 * (Z1 > 0)
    g["W1"] = X.T @ dZ1
    g["b1"] = dZ1.sum(axis=0)
    return loss, g


def adam_step(p, g, m, v, t: int, lr: float, beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (Kingma and Ba, 2015, Algorithm 1) in fp64: returns (p, m, v).

    m and v are exponential moving averages of the gradient and its square;
    they are divided by (1 - beta^t) to undo their bias toward zero."""
    p, g, m, v = (np.asarray(a, dtype=np.float64) for a in (p, g, m, v))
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    m_hat = m / (1.0 - beta1 ** t)
    v_hat = v / (1.0 - beta2 ** t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


# ---------------------------------------------------------------------------
# exact integer model
# ---------------------------------------------------------------------------
def _qweights(w):
    s = quant_scale(w)
    q = np.clip(_round_half_away(w.astype(np.float64) / s), -127, 127).astype(np.int64)
    return q, s


def _qbias(b, unit):
    return np.clip(_round_half_away(b.astype(np.float64) / unit), INT32_MIN, INT32_MAX).astype(np.int64)


def _shift_for(r: int) -> int:
    sh = 0
    while (r >> sh) > 127:
        sh += 1
    return sh


def quantize(params: dict, calib_keys) -> dict:
    """The integer model of the float parameters (see the module docstring)."""
    X = features(calib_keys).astype(np.int64)
    W1q, s1 = _qweights(params["W1"])
    b1q = _qbias(params["b1"], s1)
    a1 = X @ W1q + b1q
    sh1 = _shift_for(int(np.maximum(a1, 0).max()) if a1.size else 0)
    h1 = np.minimum(np.maximum(a1, 0) >> sh1, 127)
    W2q, s2 = _qweights(params["W2"])
    u2 = s1 * (2.0 ** sh1) * s2
    b2q = _qbias(params["b2"], u2)
    a2 = h1 @ W2q + b2q
    sh2 = _shift_for(int(np.maximum(a2, 0).max()) if a2.size else 0)
    W3q, s3 = _qweights(params["W3"])
    u3 = u2 * (2.0 ** sh2) * s3
    b3q = _qbias(params["b3"], u3)
    return {"W1q": W1q, "b1q": b1q, "sh1": sh1, "W2q": W2q, "b2q": b2q, "sh2": sh2, "W3q": W3q,
            "b3q": int(b3q[0]), "unit": u3}


def int_scores(model: dict, keys) -> np.ndarray:
    X = features(keys).astype(np.int64)
    a1 = X @ model["W1q"] + model["b1q"]
    h1 = np.minimum(np.maximum(a1, 0) >> model["sh1"], 127)
    a2 = h1 @ model["W2q"] + model["b2q"]
    h2 = np.minimum(np.maximum(a2, 0) >> model["sh2"], 127)
    return np.clip(h2 @ model["W3q"] + model["b3q"], INT32_MIN, INT32_MAX).astype(np.int64)


def float_logits(params: dict, keys) -> np.ndarray:
    X = features(keys)
    H1 = np.maximum(X @ params["W1"].astype(np.float64) + params["b1"], 0)
    H2 = np.maximum(H1 @ params["W2"].astype(np.float64) + params["b2"], 0)
    return H2 @ params["W3"].astype(np.float64) + params["b3"][0]


def model_bits(model: dict) -> int:
    """Storage of the integer model: int8 weights, int32 biases, two shifts and tau."""
    w = model["W1q"].size + model["W2q"].size + model["W3q"].size
    b = model["b1q"].size + model["b2q"].size + 1
    return 8 * w + 32 * b + 32 * 3
