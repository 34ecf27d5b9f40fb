"""Training and calibration of the learned probe-count model (an extension
the paper does not have), sequencing the library's C-ABI calls.

All arithmetic runs in libsoar.so: features, labels, forward, backward and
Adam are kernels; this module only batches the calls and picks alpha by
bisection over the recall the search itself reports.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import binding as sb


def he_uniform_params(d_in: int, hidden: int, seed: int) -> np.ndarray:
    """Initial parameters (W1 | b1 | W2 | b2 | W3 | b3), He-uniform weights and
    zero biases drawn from a seeded generator (the random draws are inputs)."""
    rng = np.random.default_rng(seed)

    def he(fan_out, fan_in):
        lim = math.sqrt(6.0 / fan_in)
        return rng.uniform(-lim, lim, size=(fan_out, fan_in))

    parts = [he(hidden, d_in), np.zeros(hidden), he(hidden, hidden), np.zeros(hidden), he(1, hidden), np.zeros(1)]
    flat = np.concatenate([p.reshape(-1) for p in parts]).astype(np.float32)
    assert flat.size == sb.soar_mlp_param_count(d_in, hidden)
    return flat


def train(index: "sb.Index", Z: torch.Tensor, labels: torch.Tensor, hidden: int = 256, steps: int = 2000,
          batch: int = 4096, lr: float = 1e-3, bf16: bool = True, seed: int = 7, shuffle_seed: int = 8):
    """Adam on mean squared error against log(label); returns (params, losses)."""
    n, d_in = Z.shape
    params = torch.from_numpy(he_uniform_params(d_in, hidden, seed)).to(Z.device)
    m1 = torch.zeros_like(params)
    m2 = torch.zeros_like(params)
    grads = torch.empty_like(params)
    loss = torch.empty((1,), dtype=torch.float32, device=Z.device)
    target = torch.log(labels.to(torch.float32))
    order = np.random.default_rng(shuffle_seed).permutation(n)
    losses = []
    pos = 0
    for step in range(1, steps + 1):
        if pos + batch > n:
            order = np.random.default_rng(shuffle_seed + step).permutation(n)
            pos = 0
        idx = torch.from_numpy(order[pos:pos + batch]).to(Z.device)
        pos += batch
        zb = Z.index_select(0, idx).contiguous()
        tb = target.index_select(0, idx).contiguous()
        sb.soar_mlp_backward(params, d_in, hidden, zb, tb, bf16, grads, loss)
        sb.soar_mlp_adam(params, grads, m1, m2, step, lr)
        if step % 50 == 0 or step == steps:
            losses.append(float(loss))
    return params, losses


def recall(ids: torch.Tensor, truth: torch.Tensor) -> float:
    return float((ids[:, :, None] == truth[:, None, :]).any(dim=2).float().mean())


def calibrate_alpha(index, params, hidden, Z, Q, truth, k, c, target=0.9, bf16=True, lo=0.05, hi=64.0, iters=20):
    """Smallest alpha (by bisection on a log scale) whose predicted probe
    counts reach mean recall@k >= target on (Q, truth)."""
    d_in = Z.shape[1]

    def rec(alpha):
        t = sb.soar_mlp_predict_probes(params, d_in, hidden, Z, alpha, c, bf16)
        ids, _ = sb.soar_search(index, Q, k, int(t.max()), t_per_query=t)
        return recall(ids, truth), t

    if rec(hi)[0] < target:
        return hi
    for _ in range(iters):
        mid = math.sqrt(lo * hi)
        if rec(mid)[0] >= target:
            hi = mid
        else:
            lo = mid
    return hi
