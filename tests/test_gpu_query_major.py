"""The query-major exact scan (a warp per query over its probed partitions),
taken when a batch probes few (query, partition) pairs per partition
(nq * t <= 2c), against the oracle and against the tensor-core scan.

c = 400 partitions of a 40 000-point index (SOAR, one spill), fp32 and bf16
rows; batches of up to 100 queries with t <= 8 take the query-major path,
the same queries replicated into a batch of 4 000 take the tensor-core path.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import topk_mismatches

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _t(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    return t.to(dtype) if dtype is not None else t


@pytest.fixture(scope="module")
def qm_index(soar):
    mix = synth.Mixture(100, 80, "isotropic", 0.3, param_seed=81)
    X = mix.sample(40_000, seed=82)
    X[30_000:30_050] = X[123]            # 51 identical rows: exact ties, lower ids first
    Q = mix.sample(100, seed=83)
    Q[5] = X[123] / np.linalg.norm(X[123])
    u = np.random.default_rng(86).standard_normal(100).astype(np.float32)
    u /= np.linalg.norm(u)
    X[35_000:35_005] = u                 # a partition of five copies of a far-off point
    C = oracle.kmeans(X, synth.init_indices(40_000, 400, seed=84), 2)
    C[399] = u
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, 400)
    Xb = oracle.bf16_round(X)
    ix = soar.soar_index_build(_t(X), _t(C), _t(A))
    ixb = soar.soar_index_build(_t(X, torch.bfloat16), _t(C), _t(A))
    yield dict(X=X, Xb=Xb, Q=Q, C=C, off=off, ids=ids, ix=ix, ixb=ixb, u=u)
    ixb.close()
    ix.close()


def _exact(X, Q):
    Xd, Qd = np.asarray(X, np.float64), np.asarray(Q, np.float64)
    return lambda q, ids: Xd[np.asarray(ids, np.int64)] @ Qd[q]


@pytest.mark.parametrize("bf16", [False, True])
@pytest.mark.parametrize("k,t", [(10, 8), (1, 1), (32, 4), (10, 3)])
def test_query_major_matches_oracle(soar, qm_index, bf16, k, t):
    L = qm_index
    assert 100 * t <= 2 * 400                       # the query-major path
    X = L["Xb"] if bf16 else L["X"]
    gi, gs = soar.soar_search(L["ixb"] if bf16 else L["ix"], _t(L["Q"]), k, t)
    wi, ws = oracle.ivf_search(L["Q"], X, L["C"], L["off"], L["ids"], k, t)
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    assert topk_mismatches(gi, wi, ws, _exact(X, L["Q"])) == []
    valid = wi >= 0
    np.testing.assert_allclose(gs[valid], ws[valid], rtol=1e-5, atol=1e-5)
    for row in gi:                                  # spilled copies removed
        v = row[row >= 0]
        assert len(v) == len(set(v.tolist()))
    if k >= 10:                                     # 51 tied copies of X[123]: the lowest ids first
        tied = np.sort(np.r_[[123], np.arange(30_000, 30_050)])[:k]
        np.testing.assert_array_equal(gi[5], tied)


@pytest.mark.parametrize("bf16", [False, True])
def test_query_major_equals_tensor_core_scan(soar, qm_index, bf16):
    # the same 100 queries alone (query-major) and inside a batch of 4 000
    # (tensor-core scan): both rescore in fp32 with the elements in ascending
    # order, so ids and scores agree bit for bit
    L = qm_index
    ix = L["ixb"] if bf16 else L["ix"]
    k, t = 10, 8
    small = _t(L["Q"])
    big = _t(np.tile(L["Q"], (40, 1)))
    assert 4000 * t > 2 * 400
    gi, gs = soar.soar_search(ix, small, k, t)
    bi, bs = soar.soar_search(ix, big, k, t)
    np.testing.assert_array_equal(gi.cpu().numpy(), bi[:100].cpu().numpy())
    np.testing.assert_array_equal(gs.cpu().numpy(), bs[:100].cpu().numpy())


def test_query_major_per_query_counts(soar, qm_index):
    L = qm_index
    tpq = np.random.default_rng(85).integers(0, 9, size=100).astype(np.int32)
    tpq[:4] = [0, 1, 8, 0]
    gi, gs = soar.soar_search(L["ix"], _t(L["Q"]), 10, 8, t_per_query=_t(tpq))
    wi, ws = oracle.ivf_search(L["Q"], L["X"], L["C"], L["off"], L["ids"], 10, 8, t_per_query=tpq)
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    assert topk_mismatches(gi, wi, ws, _exact(L["X"], L["Q"])) == []
    assert np.all(gi[tpq == 0] == -1) and np.all(np.isneginf(gs[tpq == 0]))


def test_query_major_fewer_rows_than_k(soar, qm_index):
    # the query u probes only the planted partition 399 (its five copies of
    # u plus whatever was spilled there): k = 32 exceeds its distinct points,
    # so the tail is padding
    L = qm_index
    Q = L["u"][None, :]
    top, _ = oracle.select_partitions(Q, L["C"], 1)
    assert top[0, 0] == 399
    gi, gs = soar.soar_search(L["ix"], _t(Q), 32, 1)
    wi, ws = oracle.ivf_search(Q, L["X"], L["C"], L["off"], L["ids"], 32, 1)
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    members = np.unique(L["ids"][L["off"][399]:L["off"][400]])
    assert 5 <= len(members) < 32
    assert topk_mismatches(gi, wi, ws, _exact(L["X"], Q)) == []
    assert (gi[0] >= 0).sum() == len(members)
    assert np.all(np.isneginf(gs[0][len(members):]))
    np.testing.assert_array_equal(np.sort(gi[0][:5]), np.arange(35_000, 35_005))
