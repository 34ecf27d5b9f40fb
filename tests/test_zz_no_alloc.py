"""soar_select_partitions_static: the allocation-free variant of partition
selection, for callers that must not allocate device memory during a call
(a host framework that owns the device memory budget, or a serving thread
that must stay out of the CUDA allocator).  Its scratch is a fixed device
array inside the library, shared by every call on a device.

Checked through the C ABI against soar_select_partitions (which allocates
its scratch from the stream-ordered pool) and against the oracle's top-t
partitions, on two calls in a row so that the second call runs over the
first one's leftovers in the shared array; the tensor-core selection (t <= 32
on an fp32 index), the score-matrix path that uses the static array (t > 32,
and every FP8 index) are all exercised, and the device's stream-ordered pool
is checked to see no allocation during a call.  This file is collected last
and builds its own inputs, so it passes alone or after the rest of the suite.
"""
import ctypes as ct

import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import topk_mismatches

_POOL_USED_CURRENT, _POOL_USED_HIGH = 0x7, 0x8     # cudaMemPoolAttrUsedMem{Current,High}


class _PoolWatch:
    """Used bytes of the current device's default stream-ordered pool (the
    pool the allocating entry points draw their scratch from), and device
    memory in use, around a call."""

    def __init__(self):
        self.rt = ct.CDLL("libcudart.so.13")
        dev = ct.c_int()
        assert self.rt.cudaGetDevice(ct.byref(dev)) == 0
        self.pool = ct.c_void_p()
        assert self.rt.cudaDeviceGetDefaultMemPool(ct.byref(self.pool), dev) == 0

    def attr(self, which):
        v = ct.c_uint64()
        assert self.rt.cudaMemPoolGetAttribute(self.pool, which, ct.byref(v)) == 0
        return v.value

    def __enter__(self):
        torch.cuda.synchronize()
        zero = ct.c_uint64(0)
        assert self.rt.cudaMemPoolSetAttribute(self.pool, _POOL_USED_HIGH, ct.byref(zero)) == 0  # high := current
        self.used0 = self.attr(_POOL_USED_CURRENT)
        self.free0 = torch.cuda.mem_get_info()[0]
        return self

    def __exit__(self, *exc):
        torch.cuda.synchronize()
        self.high = self.attr(_POOL_USED_HIGH)
        self.used1 = self.attr(_POOL_USED_CURRENT)
        self.free1 = torch.cuda.mem_get_info()[0]
        return False

    def allocated_nothing(self):
        return self.high == self.used0 and self.used1 == self.used0 and self.free1 == self.free0

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def index(soar):
    mix = synth.Mixture(48, 12, "isotropic", 0.3, param_seed=7)
    X = torch.from_numpy(mix.sample(6000, seed=8)).cuda()
    init = torch.from_numpy(synth.init_indices(6000, 96, seed=9)).cuda()
    C = soar.soar_train_centroids(X, 96, 3, init)
    A = soar.soar_assign(X, C, 1.0, 1)
    ix = soar.soar_index_build(X, C, A)
    # the first call on a device looks up the static array's device address
    # (and the CUDA runtime may load the library's device code then); later
    # calls are the ones checked for allocations
    soar.soar_select_partitions_static(ix, X[:4], 3, torch.empty((4, 3), dtype=torch.int32, device="cuda"))
    torch.cuda.synchronize()
    yield ix, C.cpu().numpy().astype(np.float64), mix
    ix.close()


def _check_same(top_s, sc_s, top_r, sc_r, C, Q, fp8=False):
    exact = lambda q, p: C[np.asarray(p, np.int64)] @ Q[q].astype(np.float64)
    assert topk_mismatches(top_s, top_r, sc_r.astype(np.float64), exact) == []
    np.testing.assert_allclose(sc_s, sc_r, rtol=1e-6, atol=1e-7)
    # and against the oracle's top-t partitions of the same queries
    t = top_s.shape[1]
    if fp8:
        want, wsc = oracle.select_partitions_fp8(Q, C, t)
        q8, qs = oracle.quantize_rows_fp8(Q)
        c8, cs = oracle.quantize_rows_fp8(C.astype(np.float32))
        exact = lambda q, p: (c8[np.asarray(p, np.int64)].astype(np.float64) @ q8[q].astype(np.float64)
                              ) * cs[np.asarray(p, np.int64)] * qs[q]
    else:
        want, wsc = oracle.select_partitions(Q, C, t)
    assert topk_mismatches(top_s, want, wsc, exact) == []
    np.testing.assert_allclose(sc_s, wsc, rtol=1e-5, atol=1e-6)


def _static_then_allocating(soar, ix, Q, t):
    nq = Q.shape[0]
    Qd = torch.from_numpy(Q).cuda()
    top_s = torch.full((nq, t), -7, dtype=torch.int32, device="cuda")
    sc_s = torch.full((nq, t), float("nan"), dtype=torch.float32, device="cuda")
    with _PoolWatch() as watch:
        soar.soar_select_partitions_static(ix, Qd, t, top_s, sc_s)
    assert watch.allocated_nothing(), (watch.used0, watch.high, watch.used1, watch.free0, watch.free1)
    top_r, sc_r = soar.soar_select_partitions(ix, Qd, t, with_scores=True)
    torch.cuda.synchronize()
    return top_s.cpu().numpy(), sc_s.cpu().numpy(), top_r.cpu().numpy(), sc_r.cpu().numpy()


def test_static_variant_matches_allocating_variant_twice(soar, index):
    ix, C, mix = index
    # t = 24 and 7: tensor-core selection; t = 40: score matrix in the static array
    for call, (nq, t, seed) in enumerate([(700, 24, 11), (333, 7, 12), (517, 40, 14), (129, 40, 15)]):
        Q = mix.sample(nq, seed=seed)
        _check_same(*_static_then_allocating(soar, ix, Q, t), C, Q)


def test_static_variant_on_an_fp8_index_twice(soar, index):
    ix, C, mix = index
    X = torch.from_numpy(mix.sample(6000, seed=8)).cuda()
    A = soar.soar_assign(X, torch.from_numpy(C.astype(np.float32)).cuda(), 1.0, 1)
    ix8 = soar.soar_index_build(X.to(torch.bfloat16), torch.from_numpy(C.astype(np.float32)).cuda(), A,
                                mode=soar.SOAR_SCORE_FP8)
    try:
        for nq, t, seed in [(300, 9, 16), (41, 33, 17)]:
            Q = mix.sample(nq, seed=seed)
            _check_same(*_static_then_allocating(soar, ix8, Q, t), C, Q, fp8=True)
    finally:
        ix8.close()


def test_static_variant_bf16_queries_without_scores(soar, index):
    ix, C, mix = index
    Q = mix.sample(257, seed=13)
    Qb = torch.from_numpy(Q).cuda().to(torch.bfloat16)
    top_s = torch.empty((257, 5), dtype=torch.int32, device="cuda")
    soar.soar_select_partitions_static(ix, Qb, 5, top_s)
    top_r = soar.soar_select_partitions(ix, Qb, 5)
    assert torch.equal(top_s, top_r)


def test_static_variant_rejects_batches_beyond_its_buffer(soar, index):
    ix, C, mix = index
    limit = soar.load().soar_select_partitions_static  # noqa: F841 (symbol must exist)
    nq = (32 << 20) // (4 * 96) + 1            # the score matrix alone exceeds 32 MiB
    Qd = torch.zeros((nq, 48), dtype=torch.float32, device="cuda")
    top = torch.empty((nq, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(soar.SoarError) as e:
        soar.soar_select_partitions_static(ix, Qd, 4, top)
    assert e.value.status == soar.SOAR_EINVAL
    assert "static buffer" in str(e.value)
