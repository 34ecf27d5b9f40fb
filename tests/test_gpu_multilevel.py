"""Two-level partition selection (multi-level VQ) on the GPU against the oracle.

The fine centroids are quantized again into coarse partitions (SOAR at that
level too); selection is an IVF search over the centroids.  Sizes: 600 fine
centroids (ten 64-row tiles of the coarse scan and a ragged one), 24 coarse
partitions, 300 queries (two full 128-query blocks and a ragged one).
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
def two_level(soar):
    mix = synth.Mixture(40, 60, "isotropic", 0.3, param_seed=71)
    X = mix.sample(30_000, seed=72)
    Q = mix.sample(300, seed=73)
    C = oracle.kmeans(X, synth.init_indices(30_000, 600, seed=74), 2)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, 600)
    C2 = oracle.kmeans(C, synth.init_indices(600, 24, seed=75), 3)
    A2 = oracle.soar_assign(C, C2, 1.0, 1)
    off2, ids2 = oracle.build_ivf(A2, 24)
    fine = soar.soar_index_build(_t(X), _t(C), _t(A))
    coarse = soar.soar_index_build(_t(C.astype(np.float32)), _t(C2), _t(A2))
    yield dict(X=X, Q=Q, C=C, off=off, ids=ids, C2=C2, A2=A2, off2=off2, ids2=ids2, fine=fine, coarse=coarse)
    coarse.close()
    fine.close()


def _cdot(C, Q):
    Cd, Qd = np.asarray(C, np.float64), np.asarray(Q, np.float64)
    return lambda q, p: Cd[np.asarray(p, np.int64)] @ Qd[q]


@pytest.mark.parametrize("t,t1", [(1, 1), (10, 3), (64, 5), (200, 2), (600, 24)])
def test_multilevel_select_matches_oracle(soar, two_level, t, t1):
    L = two_level
    top, sc, cnt = soar.soar_select_partitions_multilevel(L["coarse"], _t(L["Q"]), t, t1)
    want, wsc = oracle.multilevel_select(L["Q"], L["C"], L["C2"], L["off2"], L["ids2"], t, t1)
    top, sc, cnt = top.cpu().numpy(), sc.cpu().numpy(), cnt.cpu().numpy()
    assert topk_mismatches(top, want, wsc, _cdot(L["C"], L["Q"])) == []
    np.testing.assert_array_equal(cnt, (want >= 0).sum(axis=1))
    valid = want >= 0
    np.testing.assert_allclose(sc[valid], wsc[valid], rtol=1e-5, atol=1e-6)
    assert np.all(np.isneginf(sc[~valid])) and np.all(top[~valid] == -1)
    if t == 200:
        assert cnt.min() < 200        # two coarse probes cannot always supply 200


def test_multilevel_select_with_every_coarse_partition_is_flat(soar, two_level):
    L = two_level
    top, _, cnt = soar.soar_select_partitions_multilevel(L["coarse"], _t(L["Q"]), 17, 24)
    flat = soar.soar_select_partitions(L["fine"], _t(L["Q"]), 17)
    want, wsc = oracle.select_partitions(L["Q"], L["C"], 17)
    assert topk_mismatches(top.cpu().numpy(), want, wsc, _cdot(L["C"], L["Q"])) == []
    assert topk_mismatches(flat.cpu().numpy(), want, wsc, _cdot(L["C"], L["Q"])) == []
    assert int(cnt.min()) == 17


@pytest.mark.parametrize("k,t,t1", [(10, 8, 2), (32, 20, 4), (1, 1, 1), (10, 600, 24), (64, 40, 3)])
def test_multilevel_search_matches_oracle(soar, two_level, k, t, t1):
    L = two_level
    gi, gs = soar.soar_search_multilevel(L["fine"], L["coarse"], _t(L["Q"]), k, t, t1)
    wi, ws = oracle.multilevel_search(L["Q"], L["X"], L["C"], L["off"], L["ids"], L["C2"], L["off2"], L["ids2"],
                                      k, t, t1)
    Xd, Qd = L["X"].astype(np.float64), L["Q"].astype(np.float64)
    exact = lambda q, ids: Xd[np.asarray(ids, np.int64)] @ Qd[q]
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    assert topk_mismatches(gi, wi, ws, exact) == []
    valid = wi >= 0
    np.testing.assert_allclose(gs[valid], ws[valid], rtol=1e-5, atol=1e-5)


def test_empty_coarse_partition_probes_nothing(soar, two_level):
    # a coarse centroid far out along u holds no fine centroid; the query u
    # ranks it first, so with t1 = 1 it finds no fine partition and gets only
    # padding, in the selection and in the search
    L = two_level
    d = L["C"].shape[1]
    u = np.zeros(d, np.float32)
    u[0] = 1.0
    C2e = np.vstack([L["C2"], 100.0 * u]).astype(np.float32)
    A2e = oracle.soar_assign(L["C"], C2e, 1.0, 1)
    assert not np.any(A2e == C2e.shape[0] - 1)
    off2e, ids2e = oracle.build_ivf(A2e, C2e.shape[0])
    Qe = np.vstack([u, L["Q"][L["Q"][:, 0] < -0.05][:40]]).astype(np.float32)
    coarse = soar.soar_index_build(_t(L["C"].astype(np.float32)), _t(C2e), _t(A2e))
    try:
        top, sc, cnt = soar.soar_select_partitions_multilevel(coarse, _t(Qe), 5, 1)
        assert int(cnt[0]) == 0 and bool((top[0] == -1).all())
        gi, gs = soar.soar_search_multilevel(L["fine"], coarse, _t(Qe), 10, 5, 1)
        wi, ws = oracle.multilevel_search(Qe, L["X"], L["C"], L["off"], L["ids"], C2e, off2e, ids2e, 10, 5, 1)
        gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
        assert np.all(gi[0] == -1) and np.all(np.isneginf(gs[0]))
        Xd, Qd = L["X"].astype(np.float64), Qe.astype(np.float64)
        assert topk_mismatches(gi, wi, ws, lambda q, ids: Xd[np.asarray(ids, np.int64)] @ Qd[q]) == []
    finally:
        coarse.close()


def test_per_query_zero_probes_give_padding(soar, two_level):
    L = two_level
    tpq = np.random.default_rng(76).integers(0, 7, size=L["Q"].shape[0]).astype(np.int32)
    tpq[:3] = 0
    gi, gs = soar.soar_search(L["fine"], _t(L["Q"]), 10, 6, t_per_query=_t(tpq))
    wi, ws = oracle.ivf_search(L["Q"], L["X"], L["C"], L["off"], L["ids"], 10, 6, t_per_query=tpq)
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    assert np.all(gi[tpq == 0] == -1) and np.all(np.isneginf(gs[tpq == 0]))
    Xd, Qd = L["X"].astype(np.float64), L["Q"].astype(np.float64)
    assert topk_mismatches(gi, wi, ws, lambda q, ids: Xd[np.asarray(ids, np.int64)] @ Qd[q]) == []


def test_build_coarse_matches_oracle_kmeans_and_assignment(soar, two_level):
    # the library's coarse build (k-means over the fine centroids, SOAR
    # assignment, index build) against the oracle's steps from the same init
    L = two_level
    init = synth.init_indices(600, 24, seed=75)
    coarse = soar.soar_index_build_coarse(L["fine"], 24, 3, _t(init.astype(np.int32)), 1.0, 1)
    try:
        C2g = coarse.centroids().cpu().numpy()
        np.testing.assert_allclose(C2g, L["C2"], rtol=1e-5, atol=1e-6)
        assert coarse.info.n == 600 and coarse.info.c == 24 and coarse.info.rows == 1200
        off2g, ids2g = coarse.offsets().cpu().numpy(), coarse.ids().cpu().numpy()
        np.testing.assert_array_equal(off2g, L["off2"])
        np.testing.assert_array_equal(ids2g, L["ids2"])
        gi, _ = soar.soar_search_multilevel(L["fine"], coarse, _t(L["Q"]), 10, 8, 2)
        ref, _ = soar.soar_search_multilevel(L["fine"], L["coarse"], _t(L["Q"]), 10, 8, 2)
        np.testing.assert_array_equal(gi.cpu().numpy(), ref.cpu().numpy())
    finally:
        coarse.close()


def test_multilevel_rejects_a_mismatched_coarse_index(soar, two_level):
    L = two_level
    with pytest.raises(soar.SoarError):
        soar.soar_search_multilevel(L["coarse"], L["coarse"], _t(L["Q"]), 10, 4, 2)
