"""Pins of the oracle's MLP (the learned initial-state proposal): gradients
against central finite differences of its own loss, the forward pass against
numpy matrix products, and Adam against its closed-form first step."""
import numpy as np

import oracle


def _params(rng, Din=12, H=16, Dout=5):
    return {"W1": rng.normal(0, 0.5, (H, Din)), "b1": rng.normal(0, 0.1, H),
            "W2": rng.normal(0, 0.3, (H, H)), "b2": rng.normal(0, 0.1, H),
            "W3": rng.normal(0, 0.3, (Dout, H)), "b3": rng.normal(0, 0.1, Dout)}


def test_forward_matches_numpy():
    rng = np.random.default_rng(0)
    p = _params(rng)
    x = rng.normal(size=(7, 12))
    _, _, z = oracle.mlp_forward(p, x)
    h1 = np.maximum(x @ p["W1"].T + p["b1"], 0)
    h2 = np.maximum(h1 @ p["W2"].T + p["b2"], 0)
    assert np.allclose(z, np.tanh(h2 @ p["W3"].T + p["b3"]), rtol=1e-13, atol=1e-13)


def test_gradients_match_finite_differences():
    rng = np.random.default_rng(1)
    p = _params(rng)
    x = rng.normal(size=(9, 12))
    t = np.tanh(rng.normal(size=(9, 5)))
    mask = np.array([1, 1, 0, 1, 1.0])
    loss, g, _ = oracle.mlp_backward(p, x, t, mask)
    h = 1e-6
    for k in p:
        flat = p[k].ravel()
        for idx in rng.choice(flat.size, min(12, flat.size), replace=False):
            old = flat[idx]
            flat[idx] = old + h
            lp, _, _ = oracle.mlp_backward(p, x, t, mask)
            flat[idx] = old - h
            lm, _, _ = oracle.mlp_backward(p, x, t, mask)
            flat[idx] = old
            fd = (lp - lm) / (2 * h)
            assert abs(g[k].ravel()[idx] - fd) <= 1e-7 * max(abs(fd), 1e-3), (k, idx)


def test_adam_first_step_moves_by_lr():
    w = np.array([1.0, -2.0, 3.0])
    g = np.array([0.5, -4.0, 1e-3])
    m, v = np.zeros(3), np.zeros(3)
    oracle.adam(w, g, m, v, 1, 0.01)
    # bias-corrected first step is lr * sign(g) (up to eps)
    assert np.allclose(w, [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01], atol=1e-7)
