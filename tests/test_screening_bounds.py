"""The error bounds the tensor-core screens rely on, checked by emulation.

The scan screens rows on approximate scores s~ and rescores the survivors
exactly; its exactness rests on |s~ - s| staying inside the band it keeps
(s: the exact fp32 dot product the finishing kernel computes).  This CPU
test restates that arithmetic and checks the stated bounds on random and
on adversarial vectors (q proportional to x with all entries positive, so
Cauchy-Schwarz is tight, and every bit a tf32 truncation drops set):

* tf32 screen (fp32 rows): both operands rounded to tf32 (truncation or
  round-to-nearest, either way under 2^-10 of the value), exact products,
  fp32 accumulation in either order; with delta = 2^-8 ||q|| ||x|| the
  error stays below 0.504 delta for K <= 104 (2^-9 from the inputs plus
  the fp32 accumulation of both sums).  The screen's uses need less: a
  dropped row lies under a_k - 2 delta, L_k = a_k - delta, and a
  candidate's upper bound is s~ + delta.
* bf16 split screen (bf16 rows): the query enters as hi = bf16(q) and
  lo = bf16(q - hi); the error stays below (2^-18 + 2.5 K 2^-23) ||q|| ||x||,
  a quarter of the band delta = max(2^-12, 4 (2^-18 + 2.5 K 2^-23)) ||q|| ||x||.

No GPU: this pins the derivation, the GPU parity tests pin the kernels.
"""
import numpy as np
import pytest


def _tf32(v, mode):
    b = np.asarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    if mode == "rn":
        b = b + 0x0FFF + ((b >> 13) & 1)
    return (b & 0xFFFFE000).astype(np.uint32).view(np.float32)


def _bf16(v):
    b = np.asarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


def _fp32_sum(products, reverse=False):
    """fp32 accumulation of per-trial product rows, one add at a time."""
    acc = np.zeros(products.shape[0], dtype=np.float32)
    cols = range(products.shape[1] - 1, -1, -1) if reverse else range(products.shape[1])
    for k in cols:
        acc = (acc.astype(np.float64) + products[:, k].astype(np.float64)).astype(np.float32)
    return acc


def _fp32_fma_dot(q, x):
    """The exact kernel's dot product: an fp32 fused multiply-add chain."""
    acc = np.zeros(q.shape[0], dtype=np.float32)
    for k in range(q.shape[1]):
        acc = (q[:, k].astype(np.float64) * x[:, k].astype(np.float64) + acc.astype(np.float64)).astype(np.float32)
    return acc


def _cases(K, trials, seed):
    rng = np.random.default_rng(seed)
    out = []
    q = rng.standard_normal((trials, K)).astype(np.float32)
    x = rng.standard_normal((trials, K)).astype(np.float32)
    out.append((q, x))
    # q proportional to x (a power-of-two factor keeps the mantissas), all
    # positive, every value just above a power of two with all the bits a
    # tf32 truncation drops set: each operand loses almost 2^-10 of itself
    # and sum |q_k x_k| = ||q|| ||x||
    m = 1.0 + (0.99 + 0.009 * rng.random((trials, K))) * 2.0 ** -10
    e = 2.0 ** rng.integers(-3, 3, size=(trials, K))
    x2 = (m * e).astype(np.float32)
    out.append((x2 * np.float32(0.5), x2))
    out.append((x2, x2))
    return out


@pytest.mark.parametrize("K", [8, 64, 104])
@pytest.mark.parametrize("mode", ["trunc", "rn"])
def test_tf32_screen_error_below_half_the_band(K, mode):
    worst = 0.0
    for q, x in _cases(K, 2000, K):
        s = _fp32_fma_dot(q, x)
        prod = _tf32(q, mode).astype(np.float64) * _tf32(x, mode).astype(np.float64)   # exact products
        delta = 2.0 ** -8 * np.linalg.norm(q.astype(np.float64), axis=1) * np.linalg.norm(x.astype(np.float64), axis=1)
        for rev in (False, True):
            st = _fp32_sum(prod.astype(np.float32), rev)       # 11-bit x 11-bit products are exact in fp32
            err = np.abs(st.astype(np.float64) - s.astype(np.float64)) / delta
            worst = max(worst, float(err.max()))
    assert worst < 0.504, worst
    # the adversarial cases come close to the input part of the bound
    if mode == "trunc":
        assert worst > 0.45, worst


@pytest.mark.parametrize("K", [16, 96, 128])
def test_bf16_split_screen_error_below_a_quarter_of_the_band(K):
    worst = 0.0
    for q, x in _cases(K, 2000, 100 + K):
        xb = _bf16(x)                                          # bf16 rows enter exactly
        hi = _bf16(q)
        lo = _bf16((q.astype(np.float64) - hi.astype(np.float64)).astype(np.float32))
        s = _fp32_fma_dot(q, xb)
        prod = np.concatenate([hi.astype(np.float64) * xb, lo.astype(np.float64) * xb], axis=1)
        nq = np.linalg.norm(q.astype(np.float64), axis=1)
        nx = np.linalg.norm(xb.astype(np.float64), axis=1)
        err_bound = (2.0 ** -18 + 2.5 * K * 2.0 ** -23) * nq * nx
        delta = np.maximum(2.0 ** -12, 4 * (2.0 ** -18 + 2.5 * K * 2.0 ** -23)) * nq * nx
        for rev in (False, True):
            st = _fp32_sum(prod.astype(np.float32), rev)       # 8-bit x 8-bit products are exact in fp32
            err = np.abs(st.astype(np.float64) - s.astype(np.float64))
            worst = max(worst, float((err / err_bound).max()))
            assert np.all(err < delta / 4)
    assert worst < 1.0, worst


def test_the_screen_keeps_every_row_of_the_exact_top_k():
    # the three uses of the band with errors up to 0.504 delta: a row below
    # a_k - 2 delta is beaten by k rows, L_k = a_k - delta bounds the k-th
    # best from below, and s~ + delta bounds a row's exact score from above
    rng = np.random.default_rng(7)
    delta, e = 1.0, 0.504
    for _ in range(2000):
        n, k = 60, 10
        s = rng.standard_normal(n) * 3.0                       # exact scores
        st = s + rng.uniform(-e, e, n) * delta                 # screened scores
        a_k = np.sort(st)[::-1][k - 1]
        kth = np.sort(s)[::-1][k - 1]
        assert np.all(s[st < a_k - 2 * delta] < kth)           # dropped rows are not in the top k
        assert kth >= a_k - delta                              # L_k is a lower bound
        assert np.all(st + delta >= s)                         # upper bounds hold
