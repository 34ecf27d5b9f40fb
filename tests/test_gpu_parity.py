"""GPU path vs CPU oracle, element by element, through the C ABI.

Sizes span several tiles with ragged tails (n, nq not multiples of 64; d not
a multiple of 4) and the degenerate cases of the method (lambda = 0, a zero
residual, more neighbours requested than candidates, t = c).  Each stage is
tested in isolation: the GPU stage receives the oracle's inputs.
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


@pytest.fixture(scope="module")
def tiny():
    X, Q, init = synth.workload_arrays("tiny")
    C = oracle.kmeans(X, init, 10)
    return X, Q, init, C


def _exact(X, Q):
    Xd, Qd = X.astype(np.float64), Q.astype(np.float64)
    return lambda q, ids: Xd[np.asarray(ids, dtype=np.int64)] @ Qd[q]


# ------------------------------------------------------------------ k-means

def test_kmeans_one_step_matches(soar, tiny):
    X, Q, init, _ = tiny
    C_gpu = soar.soar_train_centroids(_t(X), 64, 1, _t(init)).cpu().numpy()
    C_ref = oracle.kmeans(X, init, 1)
    # A point whose two nearest seed rows are a near-tie may join either
    # cluster; every other centroid is the same fp64 mean rounded to fp32, so
    # at most 1 ulp apart.
    C0 = X[init]
    a, gaps, best = oracle.soar_assign(X, C0, 0.0, 1, return_gaps=True)
    near = gaps[:, 0] <= 1e-5 * best[:, 0]
    touched = np.zeros(64, dtype=bool)
    touched[a[near, 0]] = True
    touched[a[near, 1]] = True
    assert touched.sum() <= 4
    np.testing.assert_array_max_ulp(C_gpu[~touched], C_ref[~touched], maxulp=1)
    np.testing.assert_allclose(C_gpu[touched], C_ref[touched], atol=1e-4)


def test_kmeans_ten_iterations_objective(soar, tiny):
    X, Q, init, C_ref = tiny
    C_gpu = soar.soar_train_centroids(_t(X), 64, 10, _t(init)).cpu().numpy()
    obj_gpu = oracle.kmeans_objective(X, C_gpu)
    obj_ref = oracle.kmeans_objective(X, C_ref)
    assert obj_gpu == pytest.approx(obj_ref, rel=1e-4)
    assert np.abs(C_gpu - C_ref).max() < 1e-3


def test_kmeans_zero_iterations_returns_seed_rows(soar, tiny):
    X, Q, init, _ = tiny
    C_gpu = soar.soar_train_centroids(_t(X), 64, 0, _t(init)).cpu().numpy()
    np.testing.assert_array_equal(C_gpu, X[init])


# --------------------------------------------------------------- assignment

@pytest.mark.parametrize("lam", [0.0, 0.5, 1.0, 2.0])
@pytest.mark.parametrize("spills", [0, 1, 2])
def test_soar_assign_matches_oracle(soar, tiny, lam, spills):
    X, Q, init, C = tiny
    got = soar.soar_assign(_t(X), _t(C), lam, spills).cpu().numpy()
    want, gaps, best = oracle.soar_assign(X, C, lam, spills, return_gaps=True)
    bad, exempt = assign_mismatches(got, want, gaps, best)
    assert len(bad) == 0, f"{len(bad)} rows differ beyond near-ties (e.g. {bad[:5]}), {exempt} exempt"


def test_soar_assign_bf16_inputs(soar, tiny):
    X, Q, init, C = tiny
    Xb = oracle.bf16_round(X)
    got = soar.soar_assign(_t(X, torch.bfloat16), _t(C), 1.0, 1).cpu().numpy()
    want, gaps, best = oracle.soar_assign(Xb, C, 1.0, 1, return_gaps=True)
    bad, _ = assign_mismatches(got, want, gaps, best)
    assert len(bad) == 0


def test_soar_assign_ragged_and_degenerate(soar):
    rng = np.random.default_rng(21)
    n, d, c = 1037, 37, 70          # ragged n and d, c not a tile multiple
    X = rng.standard_normal((n, d)).astype(np.float32)
    C = rng.standard_normal((c, d)).astype(np.float32)
    X[:5] = C[3]                    # zero residual: the penalty vanishes
    C[50] = C[10]                   # duplicate centroid: lower index wins
    for lam, s in [(0.0, 1), (1.0, 1), (3.0, 4)]:
        got = soar.soar_assign(_t(X), _t(C), lam, s).cpu().numpy()
        want, gaps, best = oracle.soar_assign(X, C, lam, s, return_gaps=True)
        bad, _ = assign_mismatches(got, want, gaps, best)
        assert len(bad) == 0, (lam, s, bad[:5])
    # c == 1 + spills: the spill takes the only centroid left
    got = soar.soar_assign(_t(X[:100]), _t(C[:2]), 1.0, 1).cpu().numpy()
    assert np.all(np.sort(got, axis=1) == [0, 1])


def test_soar_assign_many_tied_centroids(soar):
    # 21 identical centroids tie exactly for the points around them: more
    # candidates than the tensor-core screen keeps, so those points are
    # decided by scoring every centroid, and the lowest index must win
    rng = np.random.default_rng(41)
    n, d, c = 700, 24, 90
    X = rng.standard_normal((n, d)).astype(np.float32)
    C = rng.standard_normal((c, d)).astype(np.float32)
    C[20:40] = C[5]
    X[:200] = C[5] + 0.05 * rng.standard_normal((200, d)).astype(np.float32)
    for lam, s in [(0.0, 0), (1.0, 1), (0.0, 1)]:
        got = soar.soar_assign(_t(X), _t(C), lam, s).cpu().numpy()
        want, gaps, best = oracle.soar_assign(X, C, lam, s, return_gaps=True)
        bad, _ = assign_mismatches(got, want, gaps, best)
        assert len(bad) == 0, (lam, s, bad[:5])
        assert np.all(got[:200, 0] == 5)
        if s:
            assert np.all(got[:200, 1] == 20)


def test_soar_assign_glove_shaped_slice(soar):
    # d = 100 (the Glove shape): many 128-point tiles; c = 256 is one
    # primary-pass tile of 256 centroids and two spill-pass tiles of 128 (the
    # primary pass across several tiles runs at c = 2 000 in test_gpu_at_size.py)
    w = synth.WORKLOADS["glove"]
    mix = synth.mixture_for(w)
    X = mix.sample(12_000, 7)
    C = X[synth.init_indices(12_000, 256, 8)].copy()
    for lam, s in [(1.0, 1), (0.0, 0)]:
        got = soar.soar_assign(_t(X), _t(C), lam, s).cpu().numpy()
        want, gaps, best = oracle.soar_assign(X, C, lam, s, return_gaps=True)
        bad, _ = assign_mismatches(got, want, gaps, best)
        assert len(bad) == 0, (lam, s, bad[:5])


def test_soar_assign_unaligned_rows(soar):
    # a row pointer 4 bytes past a 16-byte boundary takes the element-wise
    # staging path; the result must not change
    rng = np.random.default_rng(43)
    n, d, c = 900, 32, 40
    X = rng.standard_normal((n, d)).astype(np.float32)
    C = rng.standard_normal((c, d)).astype(np.float32)
    flat = torch.zeros(n * d + 1, dtype=torch.float32, device=DEV)
    flat[1:] = _t(X).reshape(-1)
    Xu = flat[1:].view(n, d)
    assert Xu.data_ptr() % 16 == 4
    for lam, s in [(1.0, 1), (0.0, 0)]:
        got = soar.soar_assign(Xu, _t(C), lam, s).cpu().numpy()
        np.testing.assert_array_equal(got, soar.soar_assign(_t(X), _t(C), lam, s).cpu().numpy())
        want, gaps, best = oracle.soar_assign(X, C, lam, s, return_gaps=True)
        bad, _ = assign_mismatches(got, want, gaps, best)
        assert len(bad) == 0


def test_fig3_worked_example_on_gpu(soar):
    x = np.array([[2.8, 1.9]], dtype=np.float32)
    C = np.array([[2.0, 2.5], [1.68, 2.74], [3.01, 0.24]], dtype=np.float32)
    for lam, want in [(0.0, 1), (1.0, 1), (1.3, 1), (1.5, 2), (2.0, 2)]:
        a = soar.soar_assign(_t(x), _t(C), lam, 1).cpu().numpy()
        assert a[0, 0] == 0 and a[0, 1] == want


# --------------------------------------------------------------- index build

@pytest.mark.parametrize("spills", [0, 1, 2])
def test_index_build_is_bit_exact(soar, tiny, spills):
    X, Q, init, C = tiny
    A = oracle.soar_assign(X, C, 1.0, spills)
    ix = soar.soar_index_build(_t(X), _t(C), _t(A))
    off, ids = oracle.build_ivf(A, C.shape[0])
    np.testing.assert_array_equal(ix.offsets().cpu().numpy(), off)
    np.testing.assert_array_equal(ix.ids().cpu().numpy(), ids)
    np.testing.assert_array_equal(ix.vectors().cpu().numpy()[:, :X.shape[1]], X[ids])
    assert ix.info.max_partition == np.diff(off).max()
    ix.close()


def test_index_build_rejects_bad_assignments(soar, tiny):
    X, Q, init, C = tiny
    A = oracle.soar_assign(X, C, 1.0, 1)
    bad = A.copy()
    bad[7, 1] = 64                  # outside [0, c)
    with pytest.raises(soar.SoarError) as e:
        soar.soar_index_build(_t(X), _t(C), _t(bad))
    assert e.value.status == soar.SOAR_EINVAL
    bad = A.copy()
    bad[9, 1] = bad[9, 0]           # same partition twice
    with pytest.raises(soar.SoarError):
        soar.soar_index_build(_t(X), _t(C), _t(bad))


# --------------------------------------------------------------- search

@pytest.fixture(scope="module")
def tiny_index(soar, tiny):
    X, Q, init, C = tiny
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, C.shape[0])
    ix = soar.soar_index_build(_t(X), _t(C), _t(A))
    yield X, Q, C, A, off, ids, ix
    ix.close()


@pytest.mark.parametrize("t", [1, 4, 17, 64])
def test_select_partitions_matches(soar, tiny_index, t):
    X, Q, C, A, off, ids, ix = tiny_index
    top, sc = soar.soar_select_partitions(ix, _t(Q), t, with_scores=True)
    want, wsc = oracle.select_partitions(Q, C, t)
    exact = lambda q, p: np.asarray(C, np.float64)[np.asarray(p, np.int64)] @ Q[q].astype(np.float64)
    assert topk_mismatches(top.cpu().numpy(), want, wsc, exact) == []
    np.testing.assert_allclose(sc.cpu().numpy(), wsc, rtol=1e-5, atol=1e-6)


@pytest.fixture(scope="module")
def select_index(soar):
    """c = 200 centroids (three full 64-centroid tiles and a ragged one of 8),
    d = 100 (query rows padded to 104 columns), centroids 3 and 150 and 199
    identical (exact ties), built from the oracle's codebook."""
    mix = synth.Mixture(100, 40, "isotropic", 0.3, param_seed=21)
    X = mix.sample(4000, seed=22)
    C = oracle.kmeans(X, synth.init_indices(4000, 200, seed=23), 2)
    C[150] = C[3]
    C[199] = C[3]
    A = oracle.soar_assign(X, C, 1.0, 0)
    ix = soar.soar_index_build(_t(X), _t(C), _t(A))
    yield mix, C, ix
    ix.close()


@pytest.mark.parametrize("t", [1, 13, 16, 17, 32, 33])
def test_select_partitions_tiles_and_tails(soar, select_index, t):
    # 300 queries: two full 128-query blocks and a ragged one of 44
    mix, C, ix = select_index
    Q = mix.sample(300, seed=24 + t)
    Q[7] = C[3] / np.linalg.norm(C[3])          # ranks the tied centroids first
    top, sc = soar.soar_select_partitions(ix, _t(Q), t, with_scores=True)
    want, wsc = oracle.select_partitions(Q, C, t)
    exact = lambda q, p: np.asarray(C, np.float64)[np.asarray(p, np.int64)] @ Q[q].astype(np.float64)
    top, sc = top.cpu().numpy(), sc.cpu().numpy()
    assert topk_mismatches(top, want, wsc, exact) == []
    np.testing.assert_allclose(sc, wsc, rtol=1e-5, atol=1e-6)
    # equal scores keep the lower id first
    assert list(top[7][: min(t, 3)]) == [3, 150, 199][: min(t, 3)]
    assert sc[7][0] == sc[7][min(t, 3) - 1]


@pytest.mark.parametrize("k,t", [(10, 4), (1, 1), (100, 8), (10, 64)])
def test_search_matches_oracle(soar, tiny_index, k, t):
    X, Q, C, A, off, ids, ix = tiny_index
    gi, gs = soar.soar_search(ix, _t(Q), k, t)
    wi, ws = oracle.ivf_search(Q, X, C, off, ids, k, t)
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    ex = _exact(X, Q)
    assert topk_mismatches(gi, wi, ws, ex) == []
    mx, mean = score_errors(gi, gs, ex)
    assert mx < 1e-5, (mx, mean)


@pytest.fixture(scope="module")
def wide_index(soar):
    """c = 1 500 centroids: the kernel that lays out the grouped (query,
    probe) pairs then gives each of its threads a run of two partitions
    (c + 2 > 1 024); built from the oracle's codebook and assignment."""
    mix = synth.Mixture(32, 60, "isotropic", 0.3, param_seed=31)
    X = mix.sample(30000, seed=32)
    C = oracle.kmeans(X, synth.init_indices(30000, 1500, seed=33), 2)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, C.shape[0])
    ix = soar.soar_index_build(_t(X), _t(C), _t(A))
    yield mix, X, C, off, ids, ix
    ix.close()


@pytest.mark.parametrize("k,t", [(10, 8), (10, 40)])
def test_search_many_partitions_matches_oracle(soar, wide_index, k, t):
    mix, X, C, off, ids, ix = wide_index
    Q = mix.sample(150, seed=34)
    gi, gs = soar.soar_search(ix, _t(Q), k, t)
    wi, ws = oracle.ivf_search(Q, X, C, off, ids, k, t)
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    ex = _exact(X, Q)
    assert topk_mismatches(gi, wi, ws, ex) == []
    mx, mean = score_errors(gi, gs, ex)
    assert mx < 1e-5, (mx, mean)


def test_search_all_partitions_is_brute_force(soar, tiny_index):
    X, Q, C, A, off, ids, ix = tiny_index
    gi, gs = soar.soar_search(ix, _t(Q), 10, C.shape[0])
    wi, ws = oracle.mips_topk(Q, X, 10)
    assert topk_mismatches(gi.cpu().numpy(), wi, ws, _exact(X, Q)) == []


def test_search_per_query_probe_counts(soar, tiny_index):
    X, Q, C, A, off, ids, ix = tiny_index
    tpq = np.random.default_rng(3).integers(1, 9, size=Q.shape[0]).astype(np.int32)
    gi, gs = soar.soar_search(ix, _t(Q), 10, 8, t_per_query=_t(tpq))
    wi, ws = oracle.ivf_search(Q, X, C, off, ids, 10, 8, t_per_query=tpq)
    assert topk_mismatches(gi.cpu().numpy(), wi, ws, _exact(X, Q)) == []


def test_search_pads_when_candidates_run_out(soar):
    rng = np.random.default_rng(5)
    X = rng.standard_normal((90, 37)).astype(np.float32)
    Q = rng.standard_normal((3, 37)).astype(np.float32)
    C = oracle.kmeans(X, np.arange(5), 3)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, 5)
    ix = soar.soar_index_build(_t(X), _t(C), _t(A))
    gi, gs = soar.soar_search(ix, _t(Q), 100, 1)
    wi, ws = oracle.ivf_search(Q, X, C, off, ids, 100, 1)
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    np.testing.assert_array_equal(gi < 0, wi < 0)
    assert np.all(np.isneginf(gs[gi < 0]))
    assert topk_mismatches(gi, wi, ws, _exact(X, Q)) == []
    ix.close()


@pytest.mark.parametrize("k,t", [(5, 1), (10, 1), (16, 1), (16, 2)])
def test_search_short_partitions_few_probes(soar, k, t):
    # Partitions of about 60 rows (one short tile each), probed by one or two
    # partitions per query: a query's first partition starts without a bound
    # from the others, and at k = 16 a tile of fewer than 61 rows has fewer
    # than k groups of four, so the screening cut stays at -inf for the whole
    # partition.  Rows past a partition's end (the tile's padding) must still
    # never become candidates: they would be rescored as rows of the next
    # partition.
    mix = synth.Mixture(24, 12, "isotropic", 0.3, param_seed=41)
    X = mix.sample(1500, seed=42)
    Q = mix.sample(400, seed=43)
    C = oracle.kmeans(X, synth.init_indices(1500, 50, seed=44), 3)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, 50)
    assert np.median(np.diff(off)) < 64
    ix = soar.soar_index_build(_t(X), _t(C), _t(A))
    try:
        gi, gs = soar.soar_search(ix, _t(Q), k, t)
        wi, ws = oracle.ivf_search(Q, X, C, off, ids, k, t)
        gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
        np.testing.assert_array_equal(gi < 0, wi < 0)
        assert topk_mismatches(gi, wi, ws, _exact(X, Q)) == []
        mx, mean = score_errors(gi, gs, _exact(X, Q))
        assert mx < 1e-5, (mx, mean)
    finally:
        ix.close()


def test_search_equal_rows_overflow_candidate_lists(soar):
    # 200 identical rows in one partition tie exactly for queries sitting on
    # them: more candidates than a screened list holds (160 entries for
    # k <= 16, 32 for k <= 32), so the exact rescan of that partition
    # decides, and ties must still go to the lower ids
    rng = np.random.default_rng(31)
    X = rng.standard_normal((3000, 40)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    X[100:300] = X[100]
    Q = rng.standard_normal((20, 40)).astype(np.float32)
    Q[:6] = X[100] + 0.01 * rng.standard_normal((6, 40)).astype(np.float32)
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    C = oracle.kmeans(X, rng.choice(3000, 16, replace=False), 3)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, 16)
    ix = soar.soar_index_build(_t(X), _t(C), _t(A))
    for k, t in [(10, 2), (16, 3), (32, 3), (1, 1)]:
        gi, gs = soar.soar_search(ix, _t(Q), k, t)
        wi, ws = oracle.ivf_search(Q, X, C, off, ids, k, t)
        gi = gi.cpu().numpy()
        assert topk_mismatches(gi, wi, ws, _exact(X, Q)) == [], (k, t)
        np.testing.assert_array_equal(gi[:6, :min(k, 10)], wi[:6, :min(k, 10)])
    soar.soar_check_device()
    ix.close()


@pytest.mark.parametrize("k", [10, 16])
def test_search_fp32_rows_past_the_group_maxima_scan(soar, k):
    # d = 130 (136 fp32 columns): two A buffers of the group-maxima scan no
    # longer fit in shared memory, so k <= 16 runs on the single-buffer scan
    # (register top-k); ragged sizes, parity with the oracle
    mix = synth.Mixture(130, 20, "isotropic", 0.3, param_seed=61)
    X = mix.sample(6001, seed=62)
    Q = mix.sample(301, seed=63)
    C = oracle.kmeans(X, synth.init_indices(6001, 24, seed=64), 3)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, 24)
    ix = soar.soar_index_build(_t(X), _t(C), _t(A))
    try:
        gi, gs = soar.soar_search(ix, _t(Q), k, 4)
        wi, ws = oracle.ivf_search(Q, X, C, off, ids, k, 4)
        gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
        assert topk_mismatches(gi, wi, ws, _exact(X, Q)) == []
        mx, mean = score_errors(gi, gs, _exact(X, Q))
        assert mx < 1e-5, (mx, mean)
    finally:
        ix.close()


@pytest.mark.parametrize("k,t", [(33, 4), (64, 17), (128, 6)])
def test_search_wide_k_matches_oracle(soar, tiny_index, k, t):
    # k above 32: per-query heaps of screened scores, global candidate lists
    X, Q, C, A, off, ids, ix = tiny_index
    tpq = np.random.default_rng(k).integers(1, t + 1, size=Q.shape[0]).astype(np.int32)
    for per_query in (None, tpq):
        gi, gs = soar.soar_search(ix, _t(Q), k, t, t_per_query=None if per_query is None else _t(per_query))
        wi, ws = oracle.ivf_search(Q, X, C, off, ids, k, t, t_per_query=per_query)
        gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
        ex = _exact(X, Q)
        assert topk_mismatches(gi, wi, ws, ex) == [], k
        np.testing.assert_array_equal(gi < 0, wi < 0)
        mx, _ = score_errors(gi, gs, ex)
        assert mx < 1e-5


def test_search_wide_k_overflow_rescans_partition(soar):
    # 400 identical rows tie exactly: more candidates than a 224-entry list
    # holds for k = 100, so the exact rescan of the partition decides
    rng = np.random.default_rng(37)
    X = rng.standard_normal((4000, 24)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    X[500:900] = X[500]
    Q = rng.standard_normal((12, 24)).astype(np.float32)
    Q[:5] = X[500] + 0.02 * rng.standard_normal((5, 24)).astype(np.float32)
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    C = oracle.kmeans(X, rng.choice(4000, 8, replace=False), 3)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, 8)
    ix = soar.soar_index_build(_t(X), _t(C), _t(A))
    for k, t in [(100, 1), (100, 3), (128, 2)]:
        gi, gs = soar.soar_search(ix, _t(Q), k, t)
        wi, ws = oracle.ivf_search(Q, X, C, off, ids, k, t)
        gi = gi.cpu().numpy()
        assert topk_mismatches(gi, wi, ws, _exact(X, Q)) == [], (k, t)
        np.testing.assert_array_equal(gi[:5], wi[:5])     # ties go to the lower ids
    soar.soar_check_device()
    ix.close()


def test_search_bf16_index(soar, tiny):
    X, Q, init, C = tiny
    Xb = oracle.bf16_round(X)
    A = oracle.soar_assign(Xb, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, C.shape[0])
    ix = soar.soar_index_build(_t(X, torch.bfloat16), _t(C), _t(A))
    gi, gs = soar.soar_search(ix, _t(Q), 10, 4)
    wi, ws = oracle.ivf_search(Q, Xb, C, off, ids, 10, 4)
    assert topk_mismatches(gi.cpu().numpy(), wi, ws, _exact(Xb, Q)) == []
    ix.close()


# --------------------------------------------------------------- brute force

@pytest.mark.parametrize("dtype", [torch.float32, torch.bfloat16])
def test_exact_mips_matches(soar, tiny, dtype):
    X, Q, init, C = tiny
    Xr = X if dtype == torch.float32 else oracle.bf16_round(X)
    gi, gs = soar.soar_exact_mips(_t(X, dtype), _t(Q), 10)
    wi, ws = oracle.mips_topk(Q, Xr, 10)
    gi = gi.cpu().numpy()
    assert topk_mismatches(gi, wi, ws, _exact(Xr, Q)) == []
    mx, _ = score_errors(gi, gs.cpu().numpy(), _exact(Xr, Q))
    assert mx < 1e-5


def test_exact_mips_ragged(soar):
    rng = np.random.default_rng(8)
    X = rng.standard_normal((5003, 37)).astype(np.float32)
    Q = rng.standard_normal((65, 37)).astype(np.float32)
    gi, gs = soar.soar_exact_mips(_t(X), _t(Q), 7)
    wi, ws = oracle.mips_topk(Q, X, 7)
    assert topk_mismatches(gi.cpu().numpy(), wi, ws, _exact(X, Q)) == []


# --------------------------------------------------------------- FP8 path

def test_fp8_codes_bit_exact(soar, tiny):
    X, Q, init, C = tiny
    codes, scales = soar.soar_quantize_fp8(_t(X))
    want_codes, want_scales = oracle.quantize_rows_fp8(X)
    got_vals = codes.cpu().view(torch.float8_e4m3fn).to(torch.float32).numpy()
    np.testing.assert_array_equal(scales.cpu().numpy(), want_scales)
    np.testing.assert_array_equal(got_vals, want_codes)


def test_fp8_index_search_with_rescoring(soar, tiny):
    X, Q, init, C = tiny
    Xb, Qb = oracle.bf16_round(X), oracle.bf16_round(Q)
    A = oracle.soar_assign(Xb, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, C.shape[0])
    ix = soar.soar_index_build(_t(X, torch.bfloat16), _t(C), _t(A), mode=soar.SOAR_SCORE_FP8)
    gi, gs = soar.soar_search(ix, _t(Q, torch.bfloat16), 10, 4, rescore=200)
    wi, ws = oracle.precision_search(Qb, Xb, C, off, ids, 10, 4, 200)
    gi = gi.cpu().numpy()
    bad = topk_mismatches(gi, wi, ws, _exact(Xb, Qb))
    # a query may differ only where the oracle's own decision is a near-tie
    # in approximate (FP8) score: the 4th / 5th partition, or the 200th /
    # 201st candidate of the probed union (the GPU sums the FP8 products in
    # fp32, the oracle in fp64)
    top_c, sc_c = oracle.select_partitions_fp8(Qb, C, 5)
    q8, qs = oracle.quantize_rows_fp8(Qb)
    for q in bad:
        near = abs(sc_c[q, 3] - sc_c[q, 4]) <= 1e-5 * abs(sc_c[q, 3])
        mem = np.unique(np.concatenate([ids[off[p]:off[p + 1]] for p in top_c[q, :4]]))
        x8, xs = oracle.quantize_rows_fp8(Xb[mem])
        approx = np.sort((x8.astype(np.float64) @ q8[q].astype(np.float64)) * xs * qs[q])[::-1]
        if approx.size > 200:
            near = near or (approx[199] - approx[200]) <= 1e-5 * abs(approx[199])
        assert near, f"query {q} differs without a near-tie in the oracle's approximate scores"
    ix.close()


# --------------------------------------------------------------- errors

def test_search_rejects_bad_t_and_k(soar, tiny_index):
    X, Q, C, A, off, ids, ix = tiny_index
    with pytest.raises(soar.SoarError):
        soar.soar_search(ix, _t(Q), 10, 65)
    with pytest.raises(soar.SoarError):
        soar.soar_search(ix, _t(Q), 0, 4)


@pytest.fixture(scope="module")
def bf16_index(soar):
    """A bf16 index at d = 100 (K padded to 112 for the bf16 tensor-core
    scan), 48 partitions probed by 700 queries (several 128-query work items
    per partition), built from the oracle's codebook over the bf16-rounded
    data."""
    mix = synth.Mixture(100, 30, "isotropic", 0.3, param_seed=71)
    X = oracle.bf16_round(mix.sample(12_000, seed=72))
    C = oracle.kmeans(X, synth.init_indices(12_000, 48, seed=73), 3)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, C.shape[0])
    ix = soar.soar_index_build(_t(X, torch.bfloat16), _t(C), _t(A))
    Q = mix.sample(700, seed=74)
    yield X, Q, C, off, ids, ix
    ix.close()


@pytest.mark.parametrize("k,t", [(10, 6), (16, 3), (32, 9), (64, 5), (1, 1)])
def test_bf16_index_tensor_core_scan_matches_oracle(soar, bf16_index, k, t):
    # exact results over the bf16 rows (each widened to fp32), whatever the
    # bf16 rounding of the queries inside the screen
    X, Q, C, off, ids, ix = bf16_index
    for qd in (torch.float32, torch.bfloat16):
        Qin = Q if qd == torch.float32 else oracle.bf16_round(Q)
        gi, gs = soar.soar_search(ix, _t(Qin, qd), k, t)
        wi, ws = oracle.ivf_search(Qin, X, C, off, ids, k, t)
        gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
        ex = _exact(X, Qin)
        assert topk_mismatches(gi, wi, ws, ex) == [], (k, t, qd)
        mx, _ = score_errors(gi, gs, ex)
        assert mx < 1e-5, (mx, k, t)


@pytest.mark.parametrize("dtype,k", [(torch.float32, 10), (torch.bfloat16, 10), (torch.float32, 64),
                                     (torch.bfloat16, 33), (torch.float32, 1)])
def test_exact_mips_several_chunks(soar, dtype, k):
    # 200 003 rows: three full 65 536-row chunks of the tensor-core brute
    # force and a ragged fourth; 300 queries (a ragged 128-query work item)
    rng = np.random.default_rng(81)
    X = rng.standard_normal((200_003, 24)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    X[150_000:150_040] = X[7]            # exact ties across chunks: lower ids first
    Q = rng.standard_normal((300, 24)).astype(np.float32)
    Q[:3] = X[7]
    Xr = X if dtype == torch.float32 else oracle.bf16_round(X)
    gi, gs = soar.soar_exact_mips(_t(X, dtype), _t(Q), k)
    wi, ws = oracle.mips_topk(Q, Xr, k)
    gi, gs = gi.cpu().numpy(), gs.cpu().numpy()
    ex = _exact(Xr, Q)
    assert topk_mismatches(gi, wi, ws, ex) == []
    mx, _ = score_errors(gi, gs, ex)
    assert mx < 1e-5
    np.testing.assert_array_equal(gi[:3, :min(k, 41)], wi[:3, :min(k, 41)])
