"""4-bit PQ layout (Section 3.5, App. A.3) on the GPU against the oracle:
codebook training on residuals, the code of every copy, and the search that
shortlists each query's probed union by PQ score and rescores exactly.

Sizes: 12 000 points, d = 40 (20 subspaces, 10 code bytes padded to 16),
c = 60 partitions, one spill; 150 queries.
"""
import os
import tempfile

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


def _unpack(codes_bytes, m):
    lo, hi = codes_bytes & 0xF, codes_bytes >> 4
    out = np.empty((codes_bytes.shape[0], 2 * codes_bytes.shape[1]), np.uint8)
    out[:, 0::2], out[:, 1::2] = lo, hi
    return out[:, :m]


@pytest.fixture(scope="module")
def pq_setup(soar):
    mix = synth.Mixture(40, 30, "isotropic", 0.3, param_seed=111)
    X = mix.sample(12_000, seed=112)
    Q = mix.sample(150, seed=113)
    C = oracle.kmeans(X, synth.init_indices(12_000, 60, seed=114), 2)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, 60)
    init = synth.init_indices(12_000, 16, seed=115)
    B = oracle.pq_train(oracle.pq_residuals(X, C, A[:, 0]), 4, init)
    codes = oracle.pq_index_codes(X, C, off, ids, B)
    ix = soar.soar_index_build_pq(_t(X), _t(C), _t(A), _t(B))
    yield dict(X=X, Q=Q, C=C, A=A, off=off, ids=ids, B=B, codes=codes, init=init, ix=ix)
    ix.close()


def test_pq_train_matches_oracle(soar, pq_setup):
    L = pq_setup
    B = soar.soar_pq_train(_t(L["X"]), _t(L["C"]), _t(L["A"][:, 0].copy()), 4, _t(L["init"]))
    np.testing.assert_allclose(B.cpu().numpy(), L["B"], rtol=1e-5, atol=1e-6)


def test_pq_train_on_lattice_residuals_is_exact(soar):
    # entries in {0, 1}: residual subvectors take 9 values, every sum is an
    # integer, so the GPU and the oracle reach the same centres bit for bit
    rng = np.random.default_rng(116)
    C = rng.integers(0, 2, size=(6, 8)).astype(np.float32)
    X = rng.integers(0, 2, size=(3000, 8)).astype(np.float32)
    part = oracle.primary_assign(X, C)[0].astype(np.int32)
    init = synth.init_indices(3000, 16, seed=117)
    want = oracle.pq_train(oracle.pq_residuals(X, C, part), 6, init)
    got = soar.soar_pq_train(_t(X), _t(C), _t(part), 6, _t(init)).cpu().numpy()
    np.testing.assert_array_equal(got, want)


def test_pq_codes_of_every_copy(soar, pq_setup):
    L = pq_setup
    m = L["X"].shape[1] // 2
    got = _unpack(L["ix"].vectors().cpu().numpy(), m)
    want = L["codes"]
    diff = np.argwhere(got != want)
    # a code may differ only where two centres are a near-tie for the residual
    part = np.repeat(np.arange(60), np.diff(L["off"]))
    R = oracle.pq_residuals(L["X"][L["ids"]], L["C"], part).astype(np.float64)
    for r, s in diff:
        dist = ((R[r, 2 * s:2 * s + 2][None, :] - L["B"][s].astype(np.float64)) ** 2).sum(axis=1)
        assert abs(dist[got[r, s]] - dist[want[r, s]]) <= 1e-6 * max(dist[want[r, s]], 1e-12), (r, s)
    assert len(diff) <= 2


def _approx_sorted(L, q, t):
    """The oracle's approximate scores of query q's probed union (earliest-probed copy), descending."""
    top, _ = oracle.select_partitions(L["Q"], L["C"], t)
    lut = np.einsum("sjd,sd->sj", L["B"].astype(np.float64), L["Q"][q].astype(np.float64).reshape(-1, 2))
    seen = {}
    for p in top[q]:
        base = float(L["C"][p].astype(np.float64) @ L["Q"][q].astype(np.float64))
        for r in range(L["off"][p], L["off"][p + 1]):
            i = int(L["ids"][r])
            if i not in seen:
                seen[i] = base + lut[np.arange(lut.shape[0]), L["codes"][r]].sum()
    return np.sort(np.fromiter(seen.values(), float))[::-1]


@pytest.mark.parametrize("k,t,R", [(10, 4, 100), (10, 1, 10), (32, 8, 500), (5, 3, 37)])
def test_pq_search_matches_oracle(soar, pq_setup, k, t, R):
    L = pq_setup
    gi, gs = soar.soar_search(L["ix"], _t(L["Q"]), k, t, rescore=R)
    wi, ws = oracle.pq_search(L["Q"], L["X"], L["C"], L["off"], L["ids"], L["B"], L["codes"], k, t, R)
    Xd, Qd = L["X"].astype(np.float64), L["Q"].astype(np.float64)
    bad = topk_mismatches(gi.cpu().numpy(), wi, ws, lambda q, i: Xd[np.asarray(i, np.int64)] @ Qd[q])
    for q in bad:
        a = _approx_sorted(L, q, t)
        assert a.size > R and (a[R - 1] - a[R]) <= 1e-5 * abs(a[R - 1]), f"query {q} differs without a near-tie"
    valid = wi >= 0
    np.testing.assert_allclose(gs.cpu().numpy()[valid], ws[valid], rtol=1e-5, atol=1e-5)


def test_pq_search_with_exact_codes_is_ivf_search(soar):
    # lattice data: the codes reconstruct every residual exactly, so the
    # shortlist by PQ score holds the exact best points
    rng = np.random.default_rng(118)
    C = rng.integers(0, 2, size=(6, 8)).astype(np.float32)
    X = rng.integers(0, 2, size=(600, 8)).astype(np.float32)
    Q = rng.standard_normal((40, 8)).astype(np.float32)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, 6)
    pts = np.array([[a, b] for a in (-1.0, 0.0, 1.0) for b in (-1.0, 0.0, 1.0)], np.float32)
    B = np.stack([np.vstack([pts, np.full((7, 2), 50.0, np.float32)]) for _ in range(4)])
    ix = soar.soar_index_build_pq(_t(X), _t(C), _t(A), _t(B))
    try:
        gi, gs = soar.soar_search(ix, _t(Q), 10, 3, rescore=40)
        wi, ws = oracle.ivf_search(Q, X, C, off, ids, 10, 3)
        np.testing.assert_array_equal(gi.cpu().numpy(), wi)
        np.testing.assert_allclose(gs.cpu().numpy(), ws, rtol=1e-5, atol=1e-5)
    finally:
        ix.close()


def test_pq_index_save_load(soar, pq_setup):
    L = pq_setup
    with tempfile.TemporaryDirectory() as d:
        path = os.path.join(d, "pq.idx")
        soar.soar_index_save(L["ix"], path)
        ix2 = soar.soar_index_load(path)
        try:
            a = soar.soar_search(L["ix"], _t(L["Q"]), 10, 4, rescore=100)
            b = soar.soar_search(ix2, _t(L["Q"]), 10, 4, rescore=100)
            np.testing.assert_array_equal(a[0].cpu().numpy(), b[0].cpu().numpy())
            np.testing.assert_array_equal(a[1].cpu().numpy(), b[1].cpu().numpy())
        finally:
            ix2.close()


def test_pq_rejects_bad_arguments(soar, pq_setup):
    L = pq_setup
    with pytest.raises(soar.SoarError):     # PQ4 needs its codebooks
        soar.soar_index_build(_t(L["X"]), _t(L["C"]), _t(L["A"]), mode=soar.SOAR_SCORE_PQ4)
    with pytest.raises(soar.SoarError):     # odd d
        soar.soar_pq_train(_t(L["X"][:, :39].copy()), _t(L["C"][:, :39].copy()), _t(L["A"][:, 0].copy()), 1,
                           _t(L["init"]))
    with pytest.raises(soar.SoarError):     # rescore below k
        soar.soar_search(L["ix"], _t(L["Q"]), 10, 4, rescore=5)
