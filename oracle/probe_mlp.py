"""fp64 oracle of the learned probe-count model (test infrastructure).

Not part of the paper: a small MLP that predicts, per query, how many
partitions to probe.  Input z = [q (d values) || the query's top-64 centroid
scores in descending order]; two hidden layers of width H with ReLU; one
output y, trained by mean squared error against log t*(q), where t*(q) is the
smallest probe count that reaches the recall target for that query (see
``soar_oracle.probe_labels``).  Optimiser: Adam with bias correction.

Only ``tests/`` and ``bench.py`` may import this module.

Parameter layout (shared with the GPU kernels as a plain contract, row-major):
W1 [H, D_in], b1 [H], W2 [H, H], b2 [H], W3 [1, H], b3 [1].
"""
from __future__ import annotations

import numpy as np

F64 = np.float64
PARAM_NAMES = ("W1", "b1", "W2", "b2", "W3", "b3")


def features(Q: np.ndarray, C: np.ndarray, top: int = 64) -> np.ndarray:
    """[q || top-``top`` centroid scores <q, C_i>, descending] in fp64."""
    Q = np.asarray(Q, dtype=F64)
    S = Q @ np.asarray(C, dtype=F64).T
    S = -np.sort(-S, axis=1)[:, :top]
    return np.concatenate([Q, S], axis=1)


def forward(p: dict, Z: np.ndarray):
    """Returns (y [B], cache) for inputs Z [B, D_in]."""
    Z = np.asarray(Z, dtype=F64)
    a1 = Z @ p["W1"].T + p["b1"]
    h1 = np.maximum(a1, 0.0)
    a2 = h1 @ p["W2"].T + p["b2"]
    h2 = np.maximum(a2, 0.0)
    y = (h2 @ p["W3"].T)[:, 0] + p["b3"][0]
    return y, (Z, a1, h1, a2, h2)


def loss(p: dict, Z: np.ndarray, target: np.ndarray) -> float:
    y, _ = forward(p, Z)
    return float(np.mean((y - target) ** 2))


def backward(p: dict, Z: np.ndarray, target: np.ndarray):
    """Gradients of mean((y - target)^2) with respect to every parameter."""
    y, (Z, a1, h1, a2, h2) = forward(p, Z)
    B = Z.shape[0]
    gy = 2.0 * (y - np.asarray(target, dtype=F64)) / B          # [B]
    g = {}
    g["W3"] = gy[None, :] @ h2                                   # [1, H]
    g["b3"] = np.array([gy.sum()])
    gh2 = gy[:, None] * p["W3"]                                  # [B, H]
    ga2 = gh2 * (a2 > 0)
    g["W2"] = ga2.T @ h1
    g["b2"] = ga2.sum(axis=0)
    gh1 = ga2 @ p["W2"]
    ga1 = gh1 * (a1 > 0)
    g["W1"] = ga1.T @ Z
    g["b1"] = ga1.sum(axis=0)
    return g


def init_params(d_in: int, hidden: int, seed: int) -> dict:
    """He-uniform weights, zero biases, from a seeded generator."""
    rng = np.random.default_rng(seed)

    def he(fan_out, fan_in):
        lim = np.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, size=(fan_out, fan_in))

    return {"W1": he(hidden, d_in), "b1": np.zeros(hidden),
            "W2": he(hidden, hidden), "b2": np.zeros(hidden),
            "W3": he(1, hidden), "b3": np.zeros(1)}


def adam_step(p: dict, g: dict, m: dict, v: dict, step: int, lr: float,
              beta1: float = 0.9, beta2: float = 0.999, eps: float = 1e-8):
    """One Adam update (in place); ``step`` counts from 1."""
    for name in PARAM_NAMES:
        m[name] = beta1 * m[name] + (1 - beta1) * g[name]
        v[name] = beta2 * v[name] + (1 - beta2) * g[name] ** 2
        mh = m[name] / (1 - beta1 ** step)
        vh = v[name] / (1 - beta2 ** step)
        p[name] = p[name] - lr * mh / (np.sqrt(vh) + eps)
    return p, m, v


def predict_probes(p: dict, Z: np.ndarray, alpha: float, c: int) -> np.ndarray:
    """t(q) = clamp(ceil(alpha * exp(y)), 1, c)."""
    y, _ = forward(p, Z)
    return np.clip(np.ceil(alpha * np.exp(y)), 1, c).astype(np.int32)
