"""Seeded synthetic inputs shared by the CPU oracle and the GPU path.

This module holds no arithmetic of the indexing or search method: it only
draws datapoints, queries and the random choices the method consumes
(k-means seed rows) from fixed seeds.  Both sides of every parity test take
their inputs from here, so neither side can drift from the other's data.

Workload shapes (the paper's datasets are not available, these stand in):

* ``tiny``     n=20 000, d=64, 16-component isotropic mixture, sigma=0.3.
* ``glove``    n=1 183 514, d=100, 500-component anisotropic mixture
               (covariance U diag(e) U^T, U Haar-random, e log-uniform in
               [0.01, 1]); the shape of Glove-1M (Section 5.1, Appendix A.2).
* ``precision`` n=10^7, d=96, 1 000-component isotropic mixture, bf16 storage.
* ``serving``  n=10^8, d=128, 4 000-component isotropic mixture, bf16.

Means are drawn from N(0, s^2 I_d) (s = 1, except s = 0.2 for ``glove``:
with s = 1 the components barely overlap and 2 of 2000 partitions already
reach recall@10 = 0.9; at s = 0.2 it takes t = 16-32, about 1.6% of the
data, the order of the paper's Glove-1M figures in Appendix A.2),
components have equal weight,
every vector is unit-normalised (Section 3.2 takes ||q|| = 1 without loss of
generality), and queries come from the same mixture as the data with a
different draw seed.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    n: int
    d: int
    components: int
    kind: str            # "isotropic" | "anisotropic"
    sigma: float         # isotropic standard deviation (unused for anisotropic)
    c: int               # number of partitions
    nq: int
    k: int
    lam: float
    spills: int
    data_seed: int
    query_seed: int
    init_seed: int
    param_seed: int
    kmeans_iters: int = 10
    mean_scale: float = 1.0   # component means ~ N(0, mean_scale^2 I_d)


WORKLOADS = {
    "tiny": Workload("tiny", 20_000, 64, 16, "isotropic", 0.3, 64, 100, 10,
                     1.0, 1, 101, 102, 103, 100),
    "glove": Workload("glove", 1_183_514, 100, 500, "anisotropic", 0.0, 2000,
                      10_000, 10, 1.0, 1, 201, 202, 203, 200, mean_scale=0.2),
    "precision": Workload("precision", 10_000_000, 96, 1000, "isotropic", 0.3,
                          10_000, 10_000, 10, 1.0, 1, 301, 302, 303, 300),
    "serving": Workload("serving", 100_000_000, 128, 4000, "isotropic", 0.3,
                        40_000, 10_000, 10, 1.0, 1, 501, 502, 503, 500),
    # many partitions of ~100 rows, for the two-level (coarse over fine
    # centroids) selection; 10 partitions per mixture component as above
    "multilevel": Workload("multilevel", 10_000_000, 96, 10_000, "isotropic", 0.3,
                           100_000, 10_000, 10, 1.0, 1, 601, 602, 603, 600, kmeans_iters=4),
}


class Mixture:
    """A Gaussian mixture whose parameters are fixed by ``param_seed``.

    ``sample(n, seed)`` draws ``n`` unit-normalised float32 vectors; the
    component of each draw is uniform over the components.
    """

    def __init__(self, d: int, components: int, kind: str = "isotropic",
                 sigma: float = 0.3, param_seed: int = 0, mean_scale: float = 1.0):
        if kind not in ("isotropic", "anisotropic"):
            raise ValueError(f"unknown mixture kind {kind!r}")
        self.d, self.m, self.kind, self.sigma = d, components, kind, sigma
        rng = np.random.default_rng(param_seed)
        self.means = mean_scale * rng.standard_normal((components, d))
        if kind == "anisotropic":
            # Per-component covariance U diag(e) U^T with U Haar-distributed
            # (QR of a Gaussian matrix with the sign of R's diagonal fixed)
            # and eigenvalues e log-uniform in [0.01, 1].
            self.factors = np.empty((components, d, d))
            for j in range(components):
                g = rng.standard_normal((d, d))
                qm, rm = np.linalg.qr(g)
                qm *= np.sign(np.diag(rm))[None, :]
                e = np.exp(rng.uniform(np.log(0.01), np.log(1.0), size=d))
                self.factors[j] = qm * np.sqrt(e)[None, :]

    def sample(self, n: int, seed: int, chunk: int = 1 << 18) -> np.ndarray:
        rng = np.random.default_rng(seed)
        out = np.empty((n, self.d), dtype=np.float32)
        for lo in range(0, n, chunk):
            hi = min(n, lo + chunk)
            comp = rng.integers(0, self.m, size=hi - lo)
            z = rng.standard_normal((hi - lo, self.d))
            if self.kind == "isotropic":
                v = self.means[comp] + self.sigma * z
            else:
                v = self.means[comp].copy()
                for j in np.unique(comp):
                    sel = comp == j
                    v[sel] += z[sel] @ self.factors[j].T
            v /= np.linalg.norm(v, axis=1, keepdims=True)
            out[lo:hi] = v
        return out


def sample_on_device(mix: Mixture, n: int, seed: int, device, dtype=None, chunk: int = 1 << 22):
    """``n`` unit-normalised draws of an isotropic mixture made on a CUDA
    device with torch's counter-based (Philox) generator, for workloads too
    large to draw on the host (the serving workload's 10^8 points).  Same
    mixture parameters as ``Mixture.sample``, a different random stream:
    component uniform over the components, then mean + sigma * N(0, I),
    normalised in fp32, cast to ``dtype`` (default fp32).  Deterministic for a
    given seed, device type and chunk size."""
    import torch
    if mix.kind != "isotropic":
        raise ValueError("device sampling covers isotropic mixtures")
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    means = torch.as_tensor(mix.means, dtype=torch.float32, device=device)
    out = torch.empty((n, mix.d), dtype=dtype or torch.float32, device=device)
    for lo in range(0, n, chunk):
        m = min(chunk, n - lo)
        comp = torch.randint(0, mix.m, (m,), generator=g, device=device)
        v = means[comp] + mix.sigma * torch.randn((m, mix.d), generator=g, device=device)
        v /= v.norm(dim=1, keepdim=True)
        out[lo:lo + m] = v.to(out.dtype)
    return out


def mixture_for(w: Workload) -> Mixture:
    return Mixture(w.d, w.components, w.kind, w.sigma, w.param_seed, w.mean_scale)


def init_indices(n: int, c: int, seed: int) -> np.ndarray:
    """c distinct row indices, drawn uniformly: the k-means seed rows."""
    if c > n:
        raise ValueError("cannot draw more distinct seed rows than datapoints")
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=c, replace=False)).astype(np.int32)


def workload_arrays(name: str, n: int | None = None, nq: int | None = None):
    """(X, Q, init_idx) for a named workload, optionally with fewer points
    (n) or queries (nq).

    A smaller count draws from the same seeded stream in the same 2^18-row
    chunks, so it is a prefix of the full draw only when it is a multiple of
    the chunk; otherwise it is another draw from the same mixture.
    """
    w = WORKLOADS[name]
    n = w.n if n is None else n
    nq = w.nq if nq is None else nq
    mix = mixture_for(w)
    X = mix.sample(n, w.data_seed)
    Q = mix.sample(nq, w.query_seed)
    init = init_indices(n, w.c, w.init_seed)
    return X, Q, init


def probe_train_queries(name: str, nq: int, seed: int = 304) -> np.ndarray:
    """Training queries for the learned probe-count model (fresh seed)."""
    return mixture_for(WORKLOADS[name]).sample(nq, seed)


def poisson_arrivals(rate_qps: float, count: int, seed: int = 504) -> np.ndarray:
    """Arrival times (seconds) of a Poisson process with the given rate."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_qps, size=count))


def request_mix(count: int, seed: int = 505, ks=(10, 100), t_lo=32, t_hi=512):
    """Per-request (k, t) for the serving workload: k in {10, 100}, t in [t_lo, t_hi]."""
    rng = np.random.default_rng(seed)
    k = rng.choice(np.asarray(ks, dtype=np.int32), size=count)
    t = rng.integers(t_lo, t_hi + 1, size=count).astype(np.int32)
    return k, t
