"""Pins of the learned-prefilter oracle (integer inference and training gradients).

* backward pass against central finite differences (fp64, no quantization);
* the straight-through reading: the gradient with fake-quantized weights is
  the unquantized gradient evaluated at the quantized weights;
* the mean BCE loss in closed form for a network with zero weights;
* quantization error bounds (|W - s Wq| <= s/2) and saturation ranges;
* integer inference against an element-by-element brute-force loop, and
  against the float network (within the quantization error it allows);
* the clustered key generator: members inside intervals, non-members outside.
"""
import numpy as np
import pytest

import synthkeys
from oracle import learned as L
from synthkeys import clustered
from synthkeys.mlp_params import init_params


def test_backward_matches_finite_differences():
    p = init_params(3, scale=0.5)
    keys = synthkeys.splitmix64(5, 0, 48)
    y = (np.arange(48) % 3 == 0).astype(np.float64)
    _, g = L.forward_backward(p, keys, y, quant=False)
    rng = np.random.default_rng(0)
    eps = 1e-6
    for name in ("W1", "b1", "W2", "b2", "W3", "b3"):
        flat = p[name].reshape(-1)
        for idx in rng.choice(flat.size, size=min(6, flat.size), replace=False):
            pp = {k: v.astype(np.float64).copy() for k, v in p.items()}
            pm = {k: v.astype(np.float64).copy() for k, v in p.items()}
            pp[name].reshape(-1)[idx] += eps
            pm[name].reshape(-1)[idx] -= eps
            fd = (L.forward_backward(pp, keys, y, quant=False)[0] - L.forward_backward(pm, keys, y, quant=False)[0]) / (2 * eps)
            assert g[name].reshape(-1)[idx] == pytest.approx(fd, rel=1e-5, abs=1e-9), (name, idx)


def test_straight_through_gradient():
    p = init_params(4)
    keys = synthkeys.splitmix64(6, 0, 64)
    y = (np.arange(64) % 2).astype(np.float64)
    loss_q, gq = L.forward_backward(p, keys, y, quant=True)
    pq = dict(p)
    for k in ("W1", "W2", "W3"):
        pq[k] = L.fake_quant(p[k])
    loss_f, gf = L.forward_backward(pq, keys, y, quant=False)
    assert loss_q == pytest.approx(loss_f, rel=1e-12)
    for k in gq:
        assert np.allclose(gq[k], gf[k], rtol=1e-12, atol=1e-15)


def test_zero_network_loss_closed_form():
    p = {k: np.zeros_like(v) for k, v in init_params(0).items()}
    p["b3"] = np.array([0.7], dtype=np.float32)
    keys = synthkeys.splitmix64(7, 0, 10)
    y = np.array([1, 0, 1, 1, 0, 0, 0, 1, 0, 1], dtype=np.float64)
    loss, g = L.forward_backward(p, keys, y)
    b = float(np.float32(0.7))
    sig = 1 / (1 + np.exp(-b))
    want = -np.mean(y * np.log(sig) + (1 - y) * np.log(1 - sig))
    assert loss == pytest.approx(want, rel=1e-12)
    assert g["b3"][0] == pytest.approx(np.mean(sig - y), rel=1e-12)


def test_quantization_bounds():
    p = init_params(8)
    for k in ("W1", "W2", "W3"):
        q, s = L._qweights(p[k])
        assert np.abs(q).max() <= 127 and np.abs(q).max() == 127
        assert np.all(np.abs(p[k].astype(np.float64) - s * q) <= s / 2 + 1e-12)
    m = L.quantize(p, synthkeys.splitmix64(9, 0, 2000))
    X = L.features(synthkeys.splitmix64(9, 0, 2000)).astype(np.int64)
    a1 = X @ m["W1q"] + m["b1q"]
    assert (np.maximum(a1, 0) >> m["sh1"]).max() <= 127
    if m["sh1"] > 0:
        assert (np.maximum(a1, 0) >> (m["sh1"] - 1)).max() > 127  # smallest such shift


def test_integer_inference_brute_force():
    p = init_params(10)
    calib = synthkeys.splitmix64(11, 0, 500)
    m = L.quantize(p, calib)
    keys = synthkeys.splitmix64(12, 0, 20)
    fast = L.int_scores(m, keys)
    for key, sc in zip(keys, fast):
        x = [(int(key) >> i) & 1 for i in range(64)]
        h1 = []
        for j in range(128):
            a = int(m["b1q"][j]) + sum(x[i] * int(m["W1q"][i][j]) for i in range(64))
            h1.append(min(max(a, 0) >> m["sh1"], 127))
        h2 = []
        for j in range(64):
            a = int(m["b2q"][j]) + sum(h1[i] * int(m["W2q"][i][j]) for i in range(128))
            h2.append(min(max(a, 0) >> m["sh2"], 127))
        s = m["b3q"] + sum(h2[i] * int(m["W3q"][i]) for i in range(64))
        assert s == int(sc)


def test_integer_scores_track_the_float_network():
    p = init_params(13, scale=0.4)
    calib = synthkeys.splitmix64(14, 0, 4000)
    m = L.quantize(p, calib)
    keys = calib[:1000]
    approx = L.int_scores(m, keys) * m["unit"]
    exact = L.float_logits(p, keys)
    # 8-bit weights and activations: the logits agree to a few percent of their range
    span = exact.max() - exact.min()
    assert np.corrcoef(approx, exact)[0, 1] > 0.97
    assert np.median(np.abs(approx - exact)) < 0.1 * span


def test_clustered_generator():
    s, w = clustered.intervals(n_intervals=500, n_clusters=8, seed=3)
    assert np.all(s[1:] > s[:-1]) and np.all(s[:-1] + w[:-1] <= s[1:])
    m = clustered.members(20_000, s, w, seed=4)
    assert clustered.inside(m, s, w).all()
    k, f = clustered.non_members(10_000, s, w, seed=5)
    assert not clustered.inside(k, s, w).any()
    assert f.sum() == 5000


def test_adam_first_step_is_a_signed_step():
    # after one step m_hat = g and v_hat = g^2, so every parameter moves by lr * g / (|g| + eps)
    rng = np.random.default_rng(1)
    p, g = rng.standard_normal(50), rng.standard_normal(50) * 1e-3
    q, m, v = L.adam_step(p, g, np.zeros(50), np.zeros(50), 1, lr=0.01)
    assert np.allclose(p - q, 0.01 * g / (np.abs(g) + 1e-8), rtol=1e-12, atol=0)
    assert np.allclose(m, 0.1 * g) and np.allclose(v, 0.001 * g * g)


def test_adam_constant_gradient_bias_correction():
    # with a constant gradient the bias-corrected moments equal g and g^2 at every step t
    g = np.array([0.3, -2.0, 1e-4])
    p = np.zeros(3)
    m = v = np.zeros(3)
    for t in range(1, 8):
        q, m, v = L.adam_step(p, g, m, v, t, lr=0.05, beta1=0.8, beta2=0.95, eps=0.0)
        assert np.allclose(p - q, 0.05 * np.sign(g), rtol=1e-12, atol=0), t
        p = q
