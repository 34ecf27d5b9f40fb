"""GPU path vs CPU oracle at the sizes the benchmark runs.

* Assignment with c = 2 000 centroids at d = 100 (the Glove-shaped shape):
  the primary pass spans eight 256-centroid tiles and the spill pass sixteen
  128-centroid tiles, so the merge of candidates across tiles is exercised
  (Section 2.2 for the primary assignment, Eq. 2 and Theorem 3.1 for the
  spill).
* Search where every partition is probed by more than 128 queries, so each
  partition is split into several 128-query work items whose per-item lists
  are merged per query (Section 2.2, Section 3.5).
* A 500-query sample of the full Glove-shaped benchmark index (n = 1 183 514,
  c = 2 000, lambda = 1, one spill, t = 14), searched in the benchmark's own
  launch configuration (the whole 10 000-query batch in one call) and
  compared with the oracle's search over the same codebook and inverted lists.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import assign_mismatches, score_errors, topk_mismatches

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _t(a, dtype=None):
    t = torch.from_numpy(np.ascontiguousarray(a)).to(DEV)
    return t.to(dtype) if dtype is not None else t


def _exact_rows(X, Q):
    """exact(q, ids): fp64 <Q[q], X[ids]> without an fp64 copy of all of X."""
    Qd = Q.astype(np.float64)
    return lambda q, ids: X[np.asarray(ids, dtype=np.int64)].astype(np.float64) @ Qd[q]


@pytest.fixture(scope="module")
def glove_slice():
    w = synth.WORKLOADS["glove"]
    X = synth.mixture_for(w).sample(40_000, seed=211)
    init = synth.init_indices(40_000, 2000, seed=212)
    C = oracle.kmeans(X, init, 2)
    return X, init, C


@pytest.mark.parametrize("lam,spills", [(1.0, 1), (0.0, 1), (0.5, 0)])
def test_assign_2000_centroids_matches_oracle(soar, glove_slice, lam, spills):
    X, _, C = glove_slice
    got = soar.soar_assign(_t(X), _t(C), lam, spills).cpu().numpy()
    want, gaps, best = oracle.soar_assign(X, C, lam, spills, return_gaps=True)
    bad, exempt = assign_mismatches(got, want, gaps, best)
    assert len(bad) == 0, f"{len(bad)} rows differ beyond near-ties (e.g. {bad[:5]}), {exempt} exempt"
    # the candidates of a point do come from different centroid tiles
    assert len(np.unique(got[:, 0] // 256)) == 8


def test_kmeans_step_2000_centroids_matches_oracle(soar, glove_slice):
    X, init, _ = glove_slice
    C_gpu = soar.soar_train_centroids(_t(X), 2000, 1, _t(init)).cpu().numpy()
    C_ref = oracle.kmeans(X, init, 1)
    # clusters touched by a near-tie point may differ; the rest are the same
    # fp64 means rounded to fp32 (at most 1 ulp apart)
    a, gaps, best = oracle.soar_assign(X, X[init], 0.0, 1, return_gaps=True)
    near = gaps[:, 0] <= 1e-5 * best[:, 0]
    touched = np.zeros(2000, dtype=bool)
    touched[a[near, 0]] = True
    touched[a[near, 1]] = True
    assert touched.sum() <= 40
    np.testing.assert_array_max_ulp(C_gpu[~touched], C_ref[~touched], maxulp=1)
    np.testing.assert_allclose(C_gpu[touched], C_ref[touched], atol=1e-3)


@pytest.fixture(scope="module")
def crowded_index(soar):
    """c = 32 partitions probed by 1 000 queries at t = 8: about 250 queries per
    partition, so every partition is split into two or three work items."""
    mix = synth.Mixture(40, 10, "isotropic", 0.3, param_seed=61)
    X = mix.sample(20_000, seed=62)
    C = oracle.kmeans(X, synth.init_indices(20_000, 32, seed=63), 4)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, 32)
    ix = soar.soar_index_build(_t(X), _t(C), _t(A))
    Q = mix.sample(1000, seed=64)
    yield X, Q, C, off, ids, ix
    ix.close()


@pytest.mark.parametrize("k,t", [(10, 8), (32, 8), (64, 8), (1, 12)])
def test_search_with_several_work_items_per_partition(soar, crowded_index, k, t):
    X, Q, C, off, ids, ix = crowded_index
    top, _ = oracle.select_partitions(Q, C, t)
    per_part = np.bincount(top.reshape(-1), minlength=C.shape[0])
    assert per_part.max() > 256 and (per_part > 128).sum() >= 8
    gi, gs = soar.soar_search(ix, _t(Q), k, t)
    wi, ws = oracle.ivf_search(Q, X, C, off, ids, k, t)
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    ex = _exact_rows(X, Q)
    assert topk_mismatches(gi, wi, ws, ex) == []
    mx, _ = score_errors(gi, gs, ex)
    assert mx < 1e-5


def test_search_several_work_items_per_query_counts(soar, crowded_index):
    X, Q, C, off, ids, ix = crowded_index
    tpq = np.random.default_rng(65).integers(1, 13, size=Q.shape[0]).astype(np.int32)
    gi, _ = soar.soar_search(ix, _t(Q), 10, 12, t_per_query=_t(tpq))
    wi, ws = oracle.ivf_search(Q, X, C, off, ids, 10, 12, t_per_query=tpq)
    assert topk_mismatches(gi.cpu().numpy(), wi, ws, _exact_rows(X, Q)) == []


@pytest.mark.slow
def test_full_glove_index_sample_matches_oracle(soar):
    w = synth.WORKLOADS["glove"]
    X, Q, init = synth.workload_arrays("glove")
    Xd = _t(X)
    C = soar.soar_train_centroids(Xd, w.c, w.kmeans_iters, _t(init))
    A = soar.soar_assign(Xd, C, w.lam, w.spills)
    ix = soar.soar_index_build(Xd, C, A)
    Cn, An = C.cpu().numpy(), A.cpu().numpy()
    # a sample of the assignments against the oracle on the same codebook
    rows = np.random.default_rng(213).choice(w.n, 20_000, replace=False)
    want, gaps, best = oracle.soar_assign(X[rows], Cn, w.lam, w.spills, return_gaps=True)
    bad, _ = assign_mismatches(An[rows], want, gaps, best)
    assert len(bad) == 0, bad[:5]
    # the whole query batch in one call, as the benchmark times it
    t = 14
    gi, gs = soar.soar_search(ix, _t(Q), w.k, t)
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    off, ids = oracle.build_ivf(An, w.c)
    np.testing.assert_array_equal(ix.offsets().cpu().numpy(), off)
    sample = np.random.default_rng(214).choice(Q.shape[0], 500, replace=False)
    wi, ws = oracle.ivf_search(Q[sample], X, Cn, off, ids, w.k, t)
    ex = _exact_rows(X, Q[sample])
    assert topk_mismatches(gi[sample], wi, ws, ex) == []
    mx, _ = score_errors(gi[sample], gs[sample], ex)
    assert mx < 1e-5
    ix.close()
