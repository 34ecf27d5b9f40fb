"""Pins of the CPU oracle against facts fixed by the paper or by mathematics.

Each test ties one oracle function to something other than itself: the
worked example of Figure 3, the closed form of Theorem 3.1 (and the
recursion in its proof, Appendix A.1), Corollaries 3.1.1 and 3.1.2,
Lemma 3.2, the end points of the KMR curve (Eq. 1), exhaustive search,
library routines (scipy distances, torch dtype conversions) and pure-Python
brute force on tiny inputs.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial.distance import cdist

import oracle
from oracle import probe_mlp

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_fig3():
    xs, cs, prim, spills = None, [], None, []
    with open(os.path.join(GOLDEN, "fig3_worked_example.txt")) as f:
        for line in f:
            line = line.split("#")[0].split()
            if not line:
                continue
            tag, vals = line[0], line[1:]
            if tag == "x":
                xs = np.array([float(v) for v in vals])
            elif tag == "c":
                cs.append([float(v) for v in vals])
            elif tag == "primary":
                prim = int(vals[0])
            elif tag == "spill":
                spills.append((float(vals[0]), int(vals[1]), float(vals[2]), float(vals[3])))
    return xs, np.array(cs), prim, spills


# ---------------------------------------------------------------- Figure 3

def test_fig3_primary_and_spill_by_lambda():
    x, C, prim, spills = _read_fig3()
    pi, best, _ = oracle.primary_assign(x[None, :], C)
    assert int(pi[0]) == prim
    assert best[0] == pytest.approx(1.0, abs=1e-12)
    r = x - C[prim]
    for lam, want, l2, l3 in spills:
        a = oracle.soar_assign(x[None, :], C, lam, 1)
        assert a[0, 0] == prim
        assert a[0, 1] == want, f"lambda={lam}"
        assert oracle.soar_loss(x, C[1], r, lam) == pytest.approx(l2, abs=1e-9)
        assert oracle.soar_loss(x, C[2], r, lam) == pytest.approx(l3, abs=1e-9)


def test_fig3_crossover_lambda():
    x, C, prim, _ = _read_fig3()
    lam_star = 0.8397 / 0.605104
    assert oracle.soar_assign(x[None, :], C, lam_star - 1e-6, 1)[0, 1] == 1
    assert oracle.soar_assign(x[None, :], C, lam_star + 1e-6, 1)[0, 1] == 2


# ------------------------------------------------ Theorem 3.1 and corollaries

def _unit_sphere(n, d, seed):
    g = np.random.default_rng(seed).standard_normal((n, d))
    return g / np.linalg.norm(g, axis=1, keepdims=True)


def _J(d, lam):
    """integral over [0, pi] of |cos theta|^lambda sin^d theta (I_d without A)."""
    return integrate.quad(lambda th: abs(math.cos(th)) ** lam * math.sin(th) ** d, 0, math.pi)[0]


def _I(d, lam):
    """I_d of Appendix A.1, A normalising the density of theta (prop. to sin^(d-2))."""
    return _J(d, lam) / _J(d - 2, 0.0)


@pytest.mark.parametrize("d", [8, 16, 64])
@pytest.mark.parametrize("lam", [0.0, 1.0, 2.0])
def test_recursion_of_I_d(d, lam):
    # (d + lambda) I_d = (d - 1) I_{d-2}, derived by parts in Appendix A.1
    assert (d + lam) * _J(d, lam) == pytest.approx((d - 1) * _J(d - 2, lam), rel=1e-7)


@pytest.mark.parametrize("d", [8, 16])
@pytest.mark.parametrize("lam", [0.0, 1.0, 2.0])
def test_theorem_closed_form_monte_carlo(d, lam):
    # E_q[|cos theta|^lambda <q, r'>^2] over uniform unit q equals
    # I_d / (d-1) * (||r'||^2 + lambda ||proj_r r'||^2): the oracle's loss
    # times that constant must match a Monte Carlo estimate for many r'.
    q = _unit_sphere(400_000, d, 7)
    rng = np.random.default_rng(11)
    r = rng.standard_normal(d)
    cos = q @ (r / np.linalg.norm(r))
    w = np.abs(cos) ** lam
    const = _I(d, lam) / (d - 1)
    x = rng.standard_normal(d)
    for _ in range(6):
        rp = rng.standard_normal(d) * rng.uniform(0.2, 2.0)
        # a component along r makes the penalty matter
        rp += rng.uniform(-1.5, 1.5) * r / np.linalg.norm(r) * np.linalg.norm(rp)
        mc = np.mean(w * (q @ rp) ** 2)
        loss = oracle.soar_loss(x, x - rp, r, lam)
        assert mc == pytest.approx(const * loss, rel=0.03)


def test_lambda_zero_constant_is_one_over_d():
    # with w = 1, E[<q, r'>^2] = ||r'||^2 / d, since E[q q^T] = I/d (Lemma 3.2's proof)
    for d in (4, 10, 100):
        assert _I(d, 0.0) / (d - 1) == pytest.approx(1.0 / d, rel=1e-9)


def test_corollary_lambda_zero_is_second_nearest():
    rng = np.random.default_rng(5)
    X = rng.standard_normal((300, 12))
    C = rng.standard_normal((40, 12))
    a = oracle.soar_assign(X, C, 0.0, 1)
    D = cdist(X, C, "sqeuclidean")
    order = np.argsort(D, axis=1, kind="stable")
    np.testing.assert_array_equal(a[:, 0], order[:, 0])
    np.testing.assert_array_equal(a[:, 1], order[:, 1])


def test_corollary_orthogonal_residual():
    rng = np.random.default_rng(6)
    for _ in range(20):
        d = int(rng.integers(2, 40))
        r = rng.standard_normal(d)
        rp = rng.standard_normal(d)
        rp -= (rp @ r) / (r @ r) * r          # r' orthogonal to r
        x = rng.standard_normal(d)
        for lam in (0.0, 0.7, 3.0):
            assert oracle.soar_loss(x, x - rp, r, lam) == pytest.approx(rp @ rp, rel=1e-12)
        # for fixed ||r'||, any parallel component raises the loss when lambda > 0
        tilt = rp + 0.3 * r
        tilt *= np.linalg.norm(rp) / np.linalg.norm(tilt)
        assert oracle.soar_loss(x, x - tilt, r, 1.0) > oracle.soar_loss(x, x - rp, r, 1.0)


def test_lemma_pearson_equals_cosine():
    d = 12
    q = _unit_sphere(300_000, d, 3)
    rng = np.random.default_rng(4)
    for _ in range(4):
        r, rp = rng.standard_normal(d), rng.standard_normal(d)
        rho = np.corrcoef(q @ r, q @ rp)[0, 1]
        cos = r @ rp / np.linalg.norm(r) / np.linalg.norm(rp)
        assert rho == pytest.approx(cos, abs=0.01)
        # ||proj_r r'|| = ||r'|| rho
        proj = abs(r @ rp) / np.linalg.norm(r)
        assert proj == pytest.approx(np.linalg.norm(rp) * abs(cos), rel=1e-12)


def test_zero_residual_drops_penalty():
    C = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 2.0]])
    x = np.array([[0.0, 0.0]])                  # x sits on C_0: r = 0
    for lam in (0.0, 1.0, 5.0):
        a = oracle.soar_assign(x, C, lam, 1)
        assert a[0, 0] == 0 and a[0, 1] == 1     # plain second-nearest


# ---------------------------------------------------- brute force, tiny data

def test_soar_assign_matches_pure_python_loops():
    rng = np.random.default_rng(8)
    n, c, d = 60, 9, 5
    X = rng.standard_normal((n, d))
    C = rng.standard_normal((c, d))
    for lam in (0.0, 1.0, 2.5):
        got = oracle.soar_assign(X, C, lam, 3)
        for i in range(n):
            x = X[i]
            dist = [sum((x[j] - C[m][j]) ** 2 for j in range(d)) for m in range(c)]
            a = [min(range(c), key=lambda m: (dist[m], m))]
            dirs = []
            for _ in range(3):
                r = [x[j] - C[a[-1]][j] for j in range(d)]
                nr = math.sqrt(sum(v * v for v in r))
                dirs.append([v / nr for v in r] if nr > 0 else [0.0] * d)

                def L(m):
                    rp = [x[j] - C[m][j] for j in range(d)]
                    return sum(v * v for v in rp) + lam * sum(
                        sum(rp[j] * u[j] for j in range(d)) ** 2 for u in dirs)

                cands = [m for m in range(c) if m not in a]
                a.append(min(cands, key=lambda m: (L(m), m)))
            assert list(got[i]) == a, (lam, i)


def test_primary_assign_matches_cdist_and_ties():
    rng = np.random.default_rng(9)
    X = rng.standard_normal((500, 7))
    C = rng.standard_normal((33, 7))
    C[20] = C[3]                                 # exact duplicate centroid
    X[:5] = C[3]                                 # points sitting on it
    pi, best, gap = oracle.primary_assign(X, C)
    D = cdist(X, C, "sqeuclidean")
    np.testing.assert_array_equal(pi, np.argmin(D, axis=1))
    assert np.all(pi[:5] == 3)                   # tie goes to the lower index
    assert np.all(gap[:5] == 0)
    np.testing.assert_allclose(best, D.min(axis=1), atol=1e-10)
    Ds = np.sort(D, axis=1)                      # gap: runner-up minus best
    np.testing.assert_allclose(gap, Ds[:, 1] - Ds[:, 0], atol=1e-10)


def test_mips_topk_matches_pure_python_with_ties():
    rng = np.random.default_rng(10)
    X = rng.integers(-3, 4, size=(80, 4)).astype(float)   # many exact ties
    Q = rng.integers(-2, 3, size=(12, 4)).astype(float)
    ids, sc = oracle.mips_topk(Q, X, 7)
    for i in range(Q.shape[0]):
        s = [sum(Q[i][j] * X[m][j] for j in range(4)) for m in range(80)]
        want = sorted(range(80), key=lambda m: (-s[m], m))[:7]
        assert list(ids[i]) == want
        assert list(sc[i]) == [s[m] for m in want]


def test_topk_pads_short_lists():
    ids, sc = oracle.topk_desc(np.array([0.5, 2.0]), 4, np.array([7, 3]))
    assert list(ids) == [3, 7, -1, -1]
    assert sc[0] == 2.0 and np.isneginf(sc[2])


def test_rank_definition():
    X = np.array([[1.0, 0.0], [0.0, 1.0], [0.5, 0.5], [1.0, 0.0]])
    q = np.array([1.0, 0.2])
    # scores 1.0, 0.2, 0.6, 1.0 -> Rank of X[0] counts both 1.0 entries
    assert oracle.rank(q, X[0], X) == 2
    assert oracle.rank(q, X[1], X) == 4
    assert oracle.rank(q, X[2], X) == 3


# ---------------------------------------------------- inverted index, search

def _small_index(seed=12, n=3000, d=16, c=24, lam=1.0, s=1):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((n, d)).astype(np.float32)
    X /= np.linalg.norm(X, axis=1, keepdims=True)
    Q = rng.standard_normal((25, d)).astype(np.float32)
    Q /= np.linalg.norm(Q, axis=1, keepdims=True)
    C = oracle.kmeans(X, rng.choice(n, c, replace=False), 5)
    A = oracle.soar_assign(X, C, lam, s)
    off, ids = oracle.build_ivf(A, c)
    return X, Q, C, A, off, ids


def test_build_ivf_invariants():
    X, Q, C, A, off, ids = _small_index(s=2)
    n, c = X.shape[0], C.shape[0]
    assert off[0] == 0 and off[-1] == n * 3
    assert np.all(np.diff(off) >= 0)
    seen = np.zeros((n, c), dtype=int)
    for p in range(c):
        mem = ids[off[p]:off[p + 1]]
        assert np.all(np.diff(mem) > 0)          # ascending, no repeats
        seen[mem, p] += 1
    assert np.all(seen.sum(axis=1) == 3)         # exactly 1 + s partitions ...
    assert np.all(seen.max(axis=1) == 1)         # ... all distinct
    for i in range(n):
        assert set(np.nonzero(seen[i])[0]) == set(A[i])


def test_search_with_all_partitions_is_brute_force():
    X, Q, C, A, off, ids = _small_index()
    got_i, got_s = oracle.ivf_search(Q, X, C, off, ids, 10, C.shape[0])
    want_i, want_s = oracle.mips_topk(Q, X, 10)
    np.testing.assert_array_equal(got_i, want_i)
    np.testing.assert_allclose(got_s, want_s, rtol=1e-12)


def test_search_dedups_spilled_copies():
    X, Q, C, A, off, ids = _small_index()
    got_i, _ = oracle.ivf_search(Q, X, C, off, ids, 50, 8)
    for row in got_i:
        v = row[row >= 0]
        assert len(v) == len(set(v.tolist()))


def test_search_is_topk_of_probed_union():
    X, Q, C, A, off, ids = _small_index(s=1)
    t = 5
    got_i, _ = oracle.ivf_search(Q, X, C, off, ids, 10, t)
    S = Q.astype(float) @ C.astype(float).T
    for i in range(Q.shape[0]):
        parts = sorted(range(C.shape[0]), key=lambda p: (-S[i, p], p))[:t]
        allowed = [j for j in range(X.shape[0]) if set(A[j]) & set(parts)]
        s = X[allowed].astype(float) @ Q[i].astype(float)
        want = [allowed[j] for j in sorted(range(len(allowed)), key=lambda j: (-s[j], allowed[j]))[:10]]
        assert list(got_i[i]) == want


def test_kmr_end_points_and_monotone():
    X, Q, C, A, off, ids = _small_index()
    truth, _ = oracle.mips_topk(Q, X, 10)
    ts = np.arange(0, C.shape[0] + 1)
    kmr = oracle.kmr_curve(Q, C, A, truth, ts)
    assert kmr[0] == 0.0 and kmr[-1] == 1.0
    assert np.all(np.diff(kmr) >= 0)
    # Eq. 1 written out with the Rank function for one t
    t = 4
    hits = 0
    for i in range(Q.shape[0]):
        for v in truth[i]:
            hits += min(oracle.rank(Q[i], C[p], C) for p in A[v]) <= t
    assert kmr[t] == pytest.approx(hits / (10 * Q.shape[0]))


def test_probe_labels_equal_direct_sweep():
    X, Q, C, A, off, ids = _small_index()
    truth, _ = oracle.mips_topk(Q, X, 10)
    lab = oracle.probe_labels(Q, C, A, truth, 0.9)
    c = C.shape[0]
    rec = np.stack([oracle.recall_at_k(oracle.ivf_search(Q, X, C, off, ids, 10, t)[0], truth)
                    for t in range(1, c + 1)])
    for i in range(Q.shape[0]):
        first = 1 + int(np.argmax(rec[:, i] >= 0.9 - 1e-12))
        assert lab[i] == first


def test_datapoints_searched_counts_partition_sizes():
    X, Q, C, A, off, ids = _small_index()
    ds = oracle.datapoints_searched(Q, C, off, C.shape[0])
    assert np.all(ds == 2 * X.shape[0])          # every row of a 1-spill index
    ds1 = oracle.datapoints_searched(Q, C, off, 1)
    top, _ = oracle.select_partitions(Q, C, 1)
    np.testing.assert_array_equal(ds1, np.diff(off)[top[:, 0]])


def test_recall_helpers():
    truth = np.array([[1, 2, 3, 4]])
    found = np.array([[4, 9, 1, -1]])
    assert oracle.recall_at_k(found, truth)[0] == 0.5
    X = np.array([[1.0], [0.9], [0.8], [0.7], [0.6], [0.7]])
    Q = np.array([[1.0]])
    ids, sc = oracle.mips_topk(Q, X, 4)
    # id 5 ties id 3 exactly: it counts as a hit under the tie rule
    assert oracle.recall_at_k_tol(np.array([[0, 1, 2, 5]]), Q, X, sc)[0] == 1.0
    assert oracle.recall_at_k(np.array([[0, 1, 2, 5]]), ids)[0] == 0.75


# ---------------------------------------------------------------- k-means

def test_kmeans_one_step_by_hand():
    X = np.array([[0.0], [1.0], [2.0], [10.0], [11.0]], dtype=np.float32)
    C = oracle.kmeans(X, np.array([0, 3]), 1)
    np.testing.assert_allclose(C[:, 0], [1.0, 10.5])
    C2 = oracle.kmeans(X, np.array([0, 1]), 2)
    # step 1: {0} {1,2,10,11} -> 0, 6 ; step 2: {0,1,2} {10,11} -> 1, 10.5
    np.testing.assert_allclose(C2[:, 0], [1.0, 10.5])


def test_kmeans_empty_cluster_keeps_centroid():
    X = np.array([[0.0], [0.1], [0.2]], dtype=np.float32)
    init = np.array([0, 1])
    X2 = np.concatenate([X, np.array([[50.0]], dtype=np.float32)])
    C = oracle.kmeans(X2, np.array([0, 3]), 1)
    assert C[1, 0] == 50.0
    # a centroid that attracts nothing stays where it is
    X3 = np.array([[0.0], [0.0], [0.1]], dtype=np.float32)
    C3 = oracle.kmeans(X3, np.array([0, 1]), 1)   # both seeds at 0: tie -> all to index 0
    assert C3[1, 0] == 0.0
    assert C3[0, 0] == pytest.approx(np.float32(0.1 / 3))
    del init


def test_kmeans_objective_non_increasing():
    rng = np.random.default_rng(13)
    X = rng.standard_normal((2000, 8)).astype(np.float32)
    _, hist = oracle.kmeans(X, rng.choice(2000, 30, replace=False), 8, return_history=True)
    assert all(b <= a + 1e-9 for a, b in zip(hist, hist[1:]))


# --------------------------------------------- low precision and the MLP

def test_fp8_round_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(14)
    v = np.concatenate([rng.uniform(-448, 448, 20000), rng.uniform(-1, 1, 20000) * 2.0 ** -6,
                        np.array([0.0, 448.0, -448.0, 2.0 ** -9, 2.0 ** -10, 1.0625, 1.1875])])
    v = v.astype(np.float32)
    want = torch.from_numpy(v).to(torch.float8_e4m3fn).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle.fp8_e4m3_round(v), want)


def test_fp8_saturates_and_scales():
    assert oracle.fp8_e4m3_round(np.array([470.0, -1e6]))[0] == 448.0
    codes, scale = oracle.quantize_rows_fp8(np.array([[0.5, -2.0, 1.0], [0, 0, 0]], dtype=np.float32))
    assert scale[0] == np.float32(2.0) / np.float32(448.0) and scale[1] == 1.0
    assert codes[0, 1] == -448.0


def test_bf16_round_matches_torch():
    torch = pytest.importorskip("torch")
    v = np.random.default_rng(15).standard_normal(50000).astype(np.float32)
    want = torch.from_numpy(v).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle.bf16_round(v), want)


def test_precision_search_exhaustive_rescore_is_exact():
    X, Q, C, A, off, ids = _small_index()
    Xb, Qb = oracle.bf16_round(X), oracle.bf16_round(Q)
    got_i, _ = oracle.precision_search(Qb, Xb, C, off, ids, 10, C.shape[0], X.shape[0])
    want_i, _ = oracle.mips_topk(Qb, Xb, 10)
    np.testing.assert_array_equal(got_i, want_i)


def test_mlp_gradients_match_finite_differences():
    rng = np.random.default_rng(16)
    p = probe_mlp.init_params(9, 6, 1)
    for name in ("b1", "b2", "b3"):
        p[name] = rng.standard_normal(p[name].shape) * 0.1
    Z = rng.standard_normal((13, 9))
    y = rng.standard_normal(13)
    g = probe_mlp.backward(p, Z, y)
    eps = 1e-6
    for name in probe_mlp.PARAM_NAMES:
        flat = p[name].reshape(-1)
        for j in range(0, flat.size, max(1, flat.size // 7)):
            old = flat[j]
            flat[j] = old + eps
            lp = probe_mlp.loss(p, Z, y)
            flat[j] = old - eps
            lm = probe_mlp.loss(p, Z, y)
            flat[j] = old
            assert g[name].reshape(-1)[j] == pytest.approx((lp - lm) / (2 * eps), rel=1e-5, abs=1e-8)


def test_mlp_adam_matches_hand_update():
    p = {"W1": np.array([[1.0]]), "b1": np.zeros(1), "W2": np.array([[1.0]]), "b2": np.zeros(1),
         "W3": np.array([[1.0]]), "b3": np.zeros(1)}
    g = {k: np.ones_like(v) for k, v in p.items()}
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(v) for k, v in p.items()}
    probe_mlp.adam_step(p, g, m, v, 1, 0.1)
    # first Adam step moves each parameter by lr * sign(g) (bias corrected)
    assert p["W1"][0, 0] == pytest.approx(1.0 - 0.1, rel=1e-6)


# ------------------------------------- FP8 shortlist on exactly encodable rows

def _fp8_exact_rows(rng, m, d, big):
    """Rows s_i * c_i with integer c_i in [-13, 13] plus one entry of +-14 and
    a power-of-two s_i: max|row| = 14 s_i, so the per-row scale is s_i / 32,
    the codes are 32 c_i (integers times 32 below 16 * 32 are E4M3 values) and
    the FP8 form of every row is exact.  ``big`` sets the spread of s_i."""
    c = rng.integers(-13, 14, size=(m, d)).astype(np.float64)
    c[np.arange(m), rng.integers(0, d, size=m)] = 14.0 * rng.choice([-1.0, 1.0], size=m)
    s = 2.0 ** rng.integers(-big, 1, size=m).astype(np.float64)
    return (c * s[:, None]).astype(np.float32)


def test_fp8_exact_rows_are_fixed_points():
    rng = np.random.default_rng(40)
    R = _fp8_exact_rows(rng, 50, 9, 3)
    codes, scale = oracle.quantize_rows_fp8(R)
    np.testing.assert_array_equal(codes.astype(np.float64) * scale[:, None].astype(np.float64),
                                  R.astype(np.float64))


@pytest.mark.parametrize("rescore", [10, 25])
def test_precision_search_equals_exact_search_when_fp8_is_exact(rescore):
    # With every query, centroid and row exactly representable in the scaled
    # FP8 form, the approximate scores are the exact ones: the FP8 partition
    # choice and the FP8 shortlist (even one of k entries) rank exactly as the
    # fp64 search does, so precision_search must return ivf_search's top k id
    # for id.  Row scales spread over 2^-4..1, so a score that left out a
    # per-row or per-centroid scale would rank differently and fail.
    rng = np.random.default_rng(41)
    n, d, c = 1500, 12, 20
    X = _fp8_exact_rows(rng, n, d, 4)
    Q = _fp8_exact_rows(rng, 30, d, 2)
    C = _fp8_exact_rows(rng, c, d, 4)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, c)
    for t in (3, 7):
        got_i, got_s = oracle.precision_search(Q, X, C, off, ids, 10, t, rescore)
        want_i, want_s = oracle.ivf_search(Q, X, C, off, ids, 10, t)
        np.testing.assert_array_equal(got_i, want_i)
        np.testing.assert_allclose(got_s, want_s, rtol=1e-12)
    # the pin has teeth: dropping the per-row scales changes the answer
    codes, _ = oracle.quantize_rows_fp8(X)
    unscaled = np.asarray(codes, np.float64) @ np.asarray(Q[0], np.float64)
    scaled = X.astype(np.float64) @ Q[0].astype(np.float64)
    assert not np.array_equal(np.argsort(-unscaled, kind="stable")[:10], np.argsort(-scaled, kind="stable")[:10])


def test_precision_search_shortlist_is_the_fp8_top_r():
    # rows that FP8 cannot represent: with rescore = k the answer is the top k
    # of the FP8 ranking over the probed union (then ordered by exact score),
    # worked out here from per-row products of the decoded codes
    X = np.array([[1.0, 0.0], [0.0, 1.0], [0.97, 0.26], [0.9, 0.5], [0.3, 0.95]], dtype=np.float32)
    Q = np.array([[0.8, 0.6]], dtype=np.float32)
    C = np.array([[1.0, 0.0], [0.0, 1.0]], dtype=np.float32)
    A = np.array([[0, 1], [1, 0], [0, 1], [0, 1], [1, 0]])
    off, ids = oracle.build_ivf(A, 2)
    q8, qs = oracle.quantize_rows_fp8(Q)
    x8, xs = oracle.quantize_rows_fp8(X)
    approx = (x8.astype(np.float64) @ q8[0].astype(np.float64)) * xs * qs[0]
    top2 = sorted(range(5), key=lambda i: (-approx[i], i))[:2]
    got_i, _ = oracle.precision_search(Q, X, C, off, ids, 2, 2, 2)
    exact = X.astype(np.float64) @ Q[0].astype(np.float64)
    assert sorted(got_i[0].tolist()) == sorted(top2)
    assert list(got_i[0]) == sorted(top2, key=lambda i: (-exact[i], i))


# ------------------------------------------- learned-probe helpers by hand

def test_probe_features_by_hand():
    Q = np.array([[1.0, 0.0], [0.0, 2.0]])
    C = np.array([[0.0, 1.0], [2.0, 0.0], [-1.0, 0.5]])
    # query 0 scores (0, 2, -1) -> descending (2, 0, -1); query 1 scores (2, 0, 1) -> (2, 1, 0)
    np.testing.assert_array_equal(probe_mlp.features(Q, C, 3), [[1, 0, 2, 0, -1], [0, 2, 2, 1, 0]])
    np.testing.assert_array_equal(probe_mlp.features(Q, C, 2), [[1, 0, 2, 0], [0, 2, 2, 1]])


def test_predict_probes_ceil_and_clamp_by_hand():
    H = 3
    p = {"W1": np.zeros((H, 2)), "b1": np.zeros(H), "W2": np.zeros((H, H)), "b2": np.zeros(H),
         "W3": np.zeros((1, H)), "b3": np.array([np.log(5.2)])}       # y = log 5.2 for every input
    Z = np.zeros((1, 2))
    assert probe_mlp.predict_probes(p, Z, 1.0, 100)[0] == 6            # ceil(5.2)
    assert probe_mlp.predict_probes(p, Z, 0.1, 100)[0] == 1            # ceil(0.52)
    assert probe_mlp.predict_probes(p, Z, 0.01, 100)[0] == 1           # ceil(0.052)
    assert probe_mlp.predict_probes(p, Z, 10.0, 20)[0] == 20           # 52 clamped to c
    # the hidden layers feed through: a ReLU unit with input 1 and weight 1
    p["W1"][0, 0], p["W2"][0, 0], p["W3"][0, 0], p["b3"][0] = 1.0, 1.0, np.log(3.0), 0.0
    # y = log(3) * relu(relu(z0)) -> exp(y) = 3^z0: 3^1.5 = 5.196 -> 6; z0 < 0 -> y = 0 -> 1
    assert probe_mlp.predict_probes(p, np.array([[1.5, 0.0]]), 1.0, 100)[0] == 6
    assert probe_mlp.predict_probes(p, np.array([[-4.0, 7.0]]), 1.0, 100)[0] == 1


def test_mlp_adam_three_steps_by_hand():
    # gradients +1, -1, +1 on a single weight, lr 0.1, beta1 0.9, beta2 0.999:
    #   m: 0.1, -0.01, 0.091     v: 0.001, 0.001999, 0.002997001
    #   bias-corrected m: 1, -0.01/0.19, 0.091/0.271; bias-corrected v: 1 each step
    # so the weight moves by -0.1, +0.1 * 0.0526316, -0.1 * 0.3357934.
    # Moments restarted at every step would move it by -0.1, +0.1, -0.1.
    names = probe_mlp.PARAM_NAMES
    p = {k: np.zeros((1, 1)) if k.startswith("W") else np.zeros(1) for k in names}
    p["W2"][0, 0] = 1.0
    m = {k: np.zeros_like(v) for k, v in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    want = [0.9, 0.9 + 0.1 * 0.01 / 0.19, 0.9 + 0.1 * 0.01 / 0.19 - 0.1 * 0.091 / 0.271]
    for step, (g, w) in enumerate(zip((1.0, -1.0, 1.0), want), start=1):
        grads = {k: np.full_like(x, g) for k, x in p.items()}
        probe_mlp.adam_step(p, grads, m, v, step, 0.1, eps=0.0)
        assert p["W2"][0, 0] == pytest.approx(w, rel=1e-12)
        assert p["b1"][0] == pytest.approx(w - 1.0, rel=1e-12)
    assert m["W2"][0, 0] == pytest.approx(0.091, rel=1e-12)
    assert v["W2"][0, 0] == pytest.approx(0.002997001, rel=1e-12)


# ---------------------------------------------------------------- multi-level VQ

def _two_level(seed=31, c=40, c2=5, s2=1):
    """The small index above with c = 40 fine partitions whose centroids are
    quantized again into c2 coarse partitions (SOAR, lambda = 1, s2 spills)."""
    X, Q, C, A, off, ids = _small_index(seed=seed, c=c)
    rng = np.random.default_rng(seed + 1)
    C2 = oracle.kmeans(C, rng.choice(c, c2, replace=False), 4)
    A2 = oracle.soar_assign(C, C2, 1.0, s2)
    off2, ids2 = oracle.build_ivf(A2, c2)
    return X, Q, C, A, off, ids, C2, A2, off2, ids2


@pytest.mark.parametrize("t", [1, 7, 40])
def test_multilevel_with_every_coarse_partition_is_flat(t):
    # every fine centroid sits in at least one coarse partition, so probing
    # all of them ranks all of C: the flat top-t selection and flat search
    X, Q, C, A, off, ids, C2, A2, off2, ids2 = _two_level()
    top, sc = oracle.multilevel_select(Q, C, C2, off2, ids2, t, C2.shape[0])
    want, wsc = oracle.select_partitions(Q, C, t)
    np.testing.assert_array_equal(top, want)
    np.testing.assert_allclose(sc, wsc, rtol=1e-12)
    gi, gs = oracle.multilevel_search(Q, X, C, off, ids, C2, off2, ids2, 10, t, C2.shape[0])
    wi, ws = oracle.ivf_search(Q, X, C, off, ids, 10, t)
    np.testing.assert_array_equal(gi, wi)
    np.testing.assert_allclose(gs, ws, rtol=1e-12)


def _select_by_loops(q, C, C2, A2, t, t1):
    """Pure-Python two-level selection: coarse dot products by loops, the top
    t1 coarse partitions, the fine centroids assigned to any of them, their
    dot products by loops, the top t (score desc, lower id first), padded."""
    dot = lambda u, v: sum(float(a) * float(b) for a, b in zip(u, v))
    cs = [dot(q, C2[j]) for j in range(len(C2))]
    probed = set(sorted(range(len(C2)), key=lambda j: (-cs[j], j))[:t1])
    fine = [i for i in range(len(C)) if probed & set(int(a) for a in A2[i])]
    fs = {i: dot(q, C[i]) for i in fine}
    best = sorted(fine, key=lambda i: (-fs[i], i))[:t]
    return best + [-1] * (t - len(best)), [fs[i] for i in best] + [-math.inf] * (t - len(best))


@pytest.mark.parametrize("t,t1", [(1, 1), (4, 1), (30, 1), (6, 2), (12, 3)])
def test_multilevel_select_by_loops(t, t1):
    X, Q, C, A, off, ids, C2, A2, off2, ids2 = _two_level()
    top, sc = oracle.multilevel_select(Q[:8], C, C2, off2, ids2, t, t1)
    for i in range(8):
        want_i, want_s = _select_by_loops(Q[i], C, C2, A2, t, t1)
        assert list(top[i]) == want_i
        np.testing.assert_allclose(sc[i], want_s, rtol=1e-12)


def test_multilevel_search_is_topk_of_selected_partitions():
    X, Q, C, A, off, ids, C2, A2, off2, ids2 = _two_level()
    t, t1 = 6, 2
    got_i, _ = oracle.multilevel_search(Q[:6], X, C, off, ids, C2, off2, ids2, 10, t, t1)
    for i in range(6):
        parts, _ = _select_by_loops(Q[i], C, C2, A2, t, t1)
        parts = set(p for p in parts if p >= 0)
        allowed = [j for j in range(X.shape[0]) if set(int(a) for a in A[j]) & parts]
        s = X[allowed].astype(float) @ Q[i].astype(float)
        want = [allowed[j] for j in sorted(range(len(allowed)), key=lambda j: (-s[j], allowed[j]))[:10]]
        assert list(got_i[i]) == want


def test_multilevel_empty_coarse_partition_gives_padding():
    # a coarse centroid far out along u holds no fine centroid (every fine
    # centroid lies within the unit ball); the query u ranks it first, so
    # with t1 = 1 it probes nothing and gets only padding
    X, Q, C, A, off, ids, C2, A2, off2, ids2 = _two_level(s2=1)
    u = np.zeros(C.shape[1])
    u[0] = 1.0
    C2e = np.vstack([C2, 100.0 * u])
    A2e = oracle.soar_assign(C, C2e, 1.0, 1)
    assert not np.any(A2e == C2e.shape[0] - 1)
    off2e, ids2e = oracle.build_ivf(A2e, C2e.shape[0])
    neg = Q[Q[:, 0] < -0.05][:3]                 # queries that rank the far centroid last
    Qe = np.vstack([u, neg]).astype(np.float32)
    top, sc = oracle.multilevel_select(Qe, C, C2e, off2e, ids2e, 5, 1)
    assert np.all(top[0] == -1) and np.all(np.isneginf(sc[0]))
    gi, gs = oracle.multilevel_search(Qe, X, C, off, ids, C2e, off2e, ids2e, 10, 5, 1)
    assert np.all(gi[0] == -1) and np.all(np.isneginf(gs[0]))
    assert np.all(gi[1:] >= 0)
    # with two coarse probes the query reaches the next coarse partition
    top2, _ = oracle.multilevel_select(Qe[:1], C, C2e, off2e, ids2e, 5, 2)
    assert np.all(top2[0] >= 0)


# ---------------------------------------------------------------- product quantization

def _lattice_index(seed=41, n=600, d=8, c=6, s=1):
    """Centroids and points with entries in {0, 1}: every residual x - C_p of
    every copy has entries in {-1, 0, 1}, so each 2-D residual subvector is
    one of 9 lattice points, which 16 PQ centres represent exactly."""
    rng = np.random.default_rng(seed)
    C = rng.integers(0, 2, size=(c, d)).astype(np.float32)
    X = rng.integers(0, 2, size=(n, d)).astype(np.float32)
    Q = rng.standard_normal((12, d)).astype(np.float32)
    A = oracle.soar_assign(X, C, 1.0, s)
    off, ids = oracle.build_ivf(A, c)
    return X, Q, C, A, off, ids


def _lattice_codebook(d):
    pts = np.array([[a, b] for a in (-1.0, 0.0, 1.0) for b in (-1.0, 0.0, 1.0)], dtype=np.float32)
    far = np.array([[50.0 + j, -50.0] for j in range(7)], dtype=np.float32)
    return np.stack([np.vstack([pts, far]) for _ in range(d // 2)])


def test_pq_train_recovers_lattice_centres_and_codes_reconstruct():
    # residuals whose subvectors take 9 values: started from rows holding all
    # 9 (plus 7 repeats), k-means ends with the 9 values among its centres,
    # and every residual is reconstructed exactly by its code
    X, Q, C, A, off, ids = _lattice_index()
    part = np.repeat(np.arange(C.shape[0]), np.diff(off))
    R = oracle.pq_residuals(X[ids], C, part)
    rng = np.random.default_rng(42)
    R = np.vstack([np.tile(_lattice_codebook(8)[0][:9].reshape(9, 2), (1, 4)), R])   # rows 0..8: the 9 values
    init = np.r_[np.arange(9), rng.choice(np.arange(9, R.shape[0]), 7, replace=False)]
    B = oracle.pq_train(R, 5, init)
    codes = oracle.pq_encode(R, B)
    rec = np.stack([B[s][codes[:, s]] for s in range(4)], axis=1).reshape(R.shape)
    np.testing.assert_array_equal(rec, R)


def test_pq_encode_by_loops_with_ties():
    rng = np.random.default_rng(43)
    R = rng.standard_normal((30, 6)).astype(np.float32)
    B = rng.standard_normal((3, 16, 2)).astype(np.float32)
    B[1, 9] = B[1, 4]                                  # a tied pair of centres: the lower index wins
    R[5, 2:4] = B[1, 4]
    codes = oracle.pq_encode(R, B)
    for i in range(30):
        for s in range(3):
            dist = [sum((float(R[i, 2 * s + e]) - float(B[s, j, e])) ** 2 for e in range(2)) for j in range(16)]
            assert codes[i, s] == min(range(16), key=lambda j: (dist[j], j))
    assert codes[5, 1] == 4


@pytest.mark.parametrize("t", [1, 3, 6])
def test_pq_search_with_exact_codes_is_ivf_search(t):
    # exact reconstruction: <q, C_p> + sum <q_s, B[code_s]> = <q, x> for
    # every copy, so the best k approximate scores are the best k exact ones
    X, Q, C, A, off, ids = _lattice_index(s=1)
    B = _lattice_codebook(X.shape[1])
    codes = oracle.pq_index_codes(X, C, off, ids, B)
    gi, gs = oracle.pq_search(Q, X, C, off, ids, B, codes, 10, t, 10)
    wi, ws = oracle.ivf_search(Q, X, C, off, ids, 10, t)
    np.testing.assert_allclose(gs, ws, rtol=1e-12)
    exact = X.astype(np.float64) @ Q.astype(np.float64).T
    for q in range(Q.shape[0]):                        # equal ids up to exact ties on the lattice
        for a, b in zip(gi[q], wi[q]):
            assert a == b or exact[a, q] == exact[b, q]


def _pq_search_by_loops(q, X, C, off, ids, B, codes, k, t, R):
    dot = lambda u, v: sum(float(a) * float(b) for a, b in zip(u, v))
    cs = [dot(q, C[p]) for p in range(len(C))]
    probes = sorted(range(len(C)), key=lambda p: (-cs[p], p))[:t]
    approx = {}
    for p in probes:                                   # earliest probe first
        for r in range(off[p], off[p + 1]):
            pid = int(ids[r])
            if pid in approx:
                continue
            approx[pid] = cs[p] + sum(dot(q[2 * s:2 * s + 2], B[s, codes[r, s]]) for s in range(B.shape[0]))
    short = sorted(approx, key=lambda i: (-approx[i], i))[:R]
    ex = {i: dot(q, X[i]) for i in short}
    best = sorted(short, key=lambda i: (-ex[i], i))[:k]
    return best + [-1] * (k - len(best))


@pytest.mark.parametrize("k,t,R", [(5, 2, 12), (3, 3, 3), (10, 1, 40)])
def test_pq_search_by_loops(k, t, R):
    # trained (lossy) codes: the shortlist, the earliest-probe rule for a
    # spilled point's two codes and the exact rescoring, written out by loops
    rng = np.random.default_rng(44)
    X = rng.standard_normal((200, 6)).astype(np.float32)
    Q = rng.standard_normal((5, 6)).astype(np.float32)
    C = oracle.kmeans(X, rng.choice(200, 8, replace=False), 3)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, 8)
    part = np.repeat(np.arange(8), np.diff(off))
    Rres = oracle.pq_residuals(X[ids], C, part)
    B = oracle.pq_train(Rres, 3, rng.choice(Rres.shape[0], 16, replace=False))
    codes = oracle.pq_index_codes(X, C, off, ids, B)
    gi, _ = oracle.pq_search(Q, X, C, off, ids, B, codes, k, t, R)
    for q in range(5):
        assert list(gi[q]) == _pq_search_by_loops(Q[q], X, C, off, ids, B, codes, k, t, R)


def test_pq_search_rescoring_everything_is_brute_force():
    X, Q, C, A, off, ids = _small_index()
    part = np.repeat(np.arange(C.shape[0]), np.diff(off))
    Rres = oracle.pq_residuals(X[ids], C, part)
    B = oracle.pq_train(Rres, 2, np.arange(16))
    codes = oracle.pq_index_codes(X, C, off, ids, B)
    gi, gs = oracle.pq_search(Q, X, C, off, ids, B, codes, 10, C.shape[0], X.shape[0])
    wi, ws = oracle.mips_topk(Q, X, 10)
    np.testing.assert_array_equal(gi, wi)
    np.testing.assert_allclose(gs, ws, rtol=1e-12)


# ------------------------------- FP8 selection, probe positions, MLP forward

def test_select_partitions_fp8_on_exact_rows_is_the_exact_selection():
    # every query and centroid exactly representable in its scaled FP8 form,
    # the centroid scales spread over 2^-4..1: the FP8 selection must equal
    # the fp64 one id for id and score for score (a score without the
    # per-centroid scale would rank the centroids differently)
    rng = np.random.default_rng(43)
    Q = _fp8_exact_rows(rng, 25, 10, 2)
    C = _fp8_exact_rows(rng, 40, 10, 4)
    for t in (1, 6, 40):
        got_i, got_s = oracle.select_partitions_fp8(Q, C, t)
        want_i, want_s = oracle.select_partitions(Q, C, t)
        np.testing.assert_array_equal(got_i, want_i)
        np.testing.assert_array_equal(got_s, want_s)
    c8, _ = oracle.quantize_rows_fp8(C)
    q8, _ = oracle.quantize_rows_fp8(Q)
    unscaled = q8.astype(np.float64) @ c8.astype(np.float64).T
    exact = Q.astype(np.float64) @ C.astype(np.float64).T
    assert not np.array_equal(np.argsort(-unscaled, axis=1, kind="stable")[:, :6],
                              np.argsort(-exact, axis=1, kind="stable")[:, :6])


def test_select_partitions_fp8_rounding_by_hand():
    # every row's largest entry is 1.75, so its scale 1.75 / 448 = 2^-8 is
    # exact in fp32.  q = (1.75, 0) encodes exactly (code 448).  Centroid 0 =
    # (0.97 * 1.75, 1.75): 0.97 * 448 = 434.56 lies above the midpoint 432 of
    # the E4M3 neighbours 416 and 448, so its first code is 448 and its FP8
    # score 448 * 448 * 2^-16 = 3.0625 ties with centroid 1 = (1.75, 0)
    # (exact score 3.0625); the tie goes to the lower id, so FP8 ranks 0
    # first where the exact scores (2.97 against 3.06) rank 1 first
    Q = np.array([[1.75, 0.0]], dtype=np.float32)
    C = np.array([[0.97 * 1.75, 1.75], [1.75, 0.0]], dtype=np.float32)
    ids, sc = oracle.select_partitions_fp8(Q, C, 2)
    assert ids.tolist() == [[0, 1]]
    np.testing.assert_array_equal(sc, [[3.0625, 3.0625]])
    assert oracle.select_partitions(Q, C, 2)[0].tolist() == [[1, 0]]


def test_partition_positions_by_hand_with_ties():
    # scores of query 0: (0.5, 1, 0.5, -1) -> probe order 1, 0, 2, 3 (the tie
    # of partitions 0 and 2 goes to the lower id); query 1 scores (0, 0, 2, 1)
    # -> order 2, 3, 0, 1
    Q = np.array([[1.0, 0.0], [0.0, 1.0]])
    C = np.array([[0.5, 0.0], [1.0, 0.0], [0.5, 2.0], [-1.0, 1.0]])
    pos = oracle.partition_positions(Q, C)
    assert pos.tolist() == [[2, 1, 3, 4], [3, 4, 1, 2]]


def test_partition_positions_without_ties_are_ranks():
    # without ties the position of partition p is 1 + the number of
    # centroids that score strictly higher (Rank(q, C_p, C) of Section 2.1),
    # and reading the positions back gives the full probe order
    rng = np.random.default_rng(44)
    Q, C = rng.standard_normal((7, 5)), rng.standard_normal((30, 5))
    pos = oracle.partition_positions(Q, C)
    S = Q @ C.T
    for i in range(7):
        for p in range(30):
            assert pos[i, p] == 1 + sum(1 for j in range(30) if S[i, j] > S[i, p])
    order, _ = oracle.select_partitions(Q, C, 30)
    for i in range(7):
        assert [int(np.nonzero(pos[i] == r)[0][0]) for r in range(1, 31)] == order[i].tolist()


def test_mlp_forward_by_hand():
    # W1 [H, D_in] row-major, ReLU after both hidden layers, none after the
    # output: row 0 = (3, 1): a1 = (2, 5), h1 = (2, 5), a2 = (7.5, -2),
    # h2 = (7.5, 0), y = 15 + 0.25; row 1 = (-1, 2): a1 = (-3, -3), h1 = 0,
    # a2 = (0.5, 0), y = 1 + 0.25
    p = {"W1": np.array([[1.0, -1.0], [2.0, 0.0]]), "b1": np.array([0.0, -1.0]),
         "W2": np.array([[1.0, 1.0], [-1.0, 0.0]]), "b2": np.array([0.5, 0.0]),
         "W3": np.array([[2.0, -3.0]]), "b3": np.array([0.25])}
    y, (Z, a1, h1, a2, h2) = probe_mlp.forward(p, np.array([[3.0, 1.0], [-1.0, 2.0]]))
    np.testing.assert_array_equal(y, [15.25, 1.25])
    np.testing.assert_array_equal(a1, [[2.0, 5.0], [-3.0, -3.0]])
    np.testing.assert_array_equal(h2, [[7.5, 0.0], [0.5, 0.0]])
    assert probe_mlp.loss(p, np.array([[3.0, 1.0], [-1.0, 2.0]]), np.array([15.0, 2.25])) == pytest.approx(
        (0.25 ** 2 + 1.0) / 2)


# ------------------------------ ties, gaps and edge values (mutation checks)

def test_soar_assign_ties_and_gaps_by_loops():
    # integer points and centroids, two centroids duplicated: squared
    # distances are exact, a duplicate's loss equals its twin's bit for bit,
    # so ties are exact and must go to the lower index, for the primary and
    # for every spill; each decision's gap (runner-up minus best among the
    # centroids still allowed) and best loss match loops over the direct form
    rng = np.random.default_rng(45)
    n, c, d = 80, 10, 4
    X = rng.integers(-3, 4, size=(n, d)).astype(np.float64)
    C = rng.integers(-3, 4, size=(c, d)).astype(np.float64)
    C[6], C[8] = C[2], C[4]
    X[:10] = C[2]                                     # zero residuals on a duplicated centroid
    for lam in (0.0, 1.5):
        got, gaps, best = oracle.soar_assign(X, C, lam, 2, return_gaps=True)
        for i in range(n):
            x = X[i]
            a, dirs = [], []
            for j in range(3):
                def L(m):
                    rp = x - C[m]
                    return float(rp @ rp) + lam * sum(float(rp @ u) ** 2 for u in dirs)
                losses = sorted((L(m), m) for m in range(c) if m not in a)
                a.append(losses[0][1])
                assert got[i, j] == losses[0][1], (lam, i, j)
                assert best[i, j] == pytest.approx(losses[0][0], rel=1e-9, abs=1e-9)
                assert gaps[i, j] == pytest.approx(losses[1][0] - losses[0][0], rel=1e-9, abs=1e-9)
                r = x - C[a[-1]]
                nr = math.sqrt(float(r @ r))
                dirs.append(r / nr if nr > 0 else np.zeros(d))
        assert np.all(got[:10, 0] == 2) and np.all(got[:10, 1] == 6)   # the exact twin, lower index first


@pytest.mark.parametrize("target", [0.75, 0.85])
def test_probe_labels_with_a_fractional_rank_equal_direct_sweep(target):
    # target * k = 7.5 and 8.5: the label needs ceil(target * k) neighbours
    X, Q, C, A, off, ids = _small_index()
    truth, _ = oracle.mips_topk(Q, X, 10)
    lab = oracle.probe_labels(Q, C, A, truth, target)
    rec = np.stack([oracle.recall_at_k(oracle.ivf_search(Q, X, C, off, ids, 10, t)[0], truth)
                    for t in range(1, C.shape[0] + 1)])
    for i in range(Q.shape[0]):
        assert lab[i] == 1 + int(np.argmax(rec[:, i] >= target - 1e-12))


def test_bf16_round_ties_to_even():
    torch = pytest.importorskip("torch")
    # 1 + 2^-8 lies halfway between 1 and 1 + 2^-7: even mantissa -> 1;
    # 1 + 3 * 2^-8 lies halfway between 1 + 2^-7 (odd) and 1 + 2^-6 (even)
    v = np.array([1 + 2 ** -8, 1 + 3 * 2 ** -8, -(1 + 2 ** -8), -(1 + 3 * 2 ** -8)], dtype=np.float32)
    np.testing.assert_array_equal(oracle.bf16_round(v), [1.0, 1 + 2 ** -6, -1.0, -(1 + 2 ** -6)])
    # every exact tie pattern (low 16 bits 0x8000) against torch's conversion
    rng = np.random.default_rng(46)
    bits = (rng.integers(0x0080, 0x7F00, size=4000, dtype=np.uint32) << 16) | 0x8000
    bits[::2] |= 0x80000000
    t = bits.view(np.float32)
    want = torch.from_numpy(t.copy()).to(torch.bfloat16).to(torch.float32).numpy()
    np.testing.assert_array_equal(oracle.bf16_round(t), want)


def test_precision_search_probes_the_fp8_selection():
    # the centroids of the FP8 hand case: with t = 1 the FP8 scores probe
    # partition 0, the exact scores would probe partition 1; each partition
    # holds one point, so the answer shows which partition was probed
    Q = np.array([[1.75, 0.0]], dtype=np.float32)
    C = np.array([[0.97 * 1.75, 1.75], [1.75, 0.0]], dtype=np.float32)
    X = np.array([[0.0, 1.0], [1.0, 0.0]], dtype=np.float32)
    off, ids = oracle.build_ivf(np.array([[0], [1]]), 2)
    got_i, got_s = oracle.precision_search(Q, X, C, off, ids, 1, 1, 1)
    assert got_i.tolist() == [[0]] and got_s.tolist() == [[0.0]]
    assert oracle.ivf_search(Q, X, C, off, ids, 1, 1)[0].tolist() == [[1]]


def test_mlp_adam_first_step_with_small_and_non_unit_gradients():
    # first step: m = 0.1 g, v = 0.001 g^2, bias-corrected m = g and v = g^2,
    # update = lr * g / (|g| + eps): for g = 0.5 that is lr * 0.5 / (0.5 + 1e-8),
    # for g = 1e-6 it is lr / 1.01 (eps added to the root, not under it)
    names = probe_mlp.PARAM_NAMES
    p = {k: np.zeros((1, 1)) if k.startswith("W") else np.zeros(1) for k in names}
    m = {k: np.zeros_like(x) for k, x in p.items()}
    v = {k: np.zeros_like(x) for k, x in p.items()}
    gv = {"W1": 0.5, "b1": 1e-6, "W2": -3.0, "b2": 0.0, "W3": 1.0, "b3": -1e-6}
    g = {k: np.full_like(p[k], gv[k]) for k in names}
    probe_mlp.adam_step(p, g, m, v, 1, 0.1)
    assert p["W1"][0, 0] == pytest.approx(-0.1 * 0.5 / (0.5 + 1e-8), rel=1e-12)
    assert p["b1"][0] == pytest.approx(-0.1 * 1e-6 / (1e-6 + 1e-8), rel=1e-12)
    assert p["W2"][0, 0] == pytest.approx(0.1 * 3.0 / (3.0 + 1e-8), rel=1e-12)
    assert p["b2"][0] == 0.0
    assert p["b3"][0] == pytest.approx(0.1 / 1.01, rel=1e-12)
    assert v["W2"][0, 0] == pytest.approx(0.001 * 9.0, rel=1e-12)


def test_predict_probes_clamps_an_underflowed_count_to_one():
    H = 2
    p = {"W1": np.zeros((H, 2)), "b1": np.zeros(H), "W2": np.zeros((H, H)), "b2": np.zeros(H),
         "W3": np.zeros((1, H)), "b3": np.array([-1000.0])}    # exp(y) underflows to 0
    assert probe_mlp.predict_probes(p, np.zeros((3, 2)), 1.0, 50).tolist() == [1, 1, 1]


def test_init_params_he_uniform_bounds():
    # He-uniform: U(-sqrt(6 / fan_in), sqrt(6 / fan_in)) per weight matrix,
    # zero biases; with 1 600 draws the extremes come close to the bound
    d_in, hidden = 4, 400
    p = probe_mlp.init_params(d_in, hidden, 7)
    for name, fan_in, shape in (("W1", d_in, (hidden, d_in)), ("W2", hidden, (hidden, hidden)),
                                ("W3", hidden, (1, hidden))):
        lim = math.sqrt(6.0 / fan_in)
        assert p[name].shape == shape
        assert np.abs(p[name]).max() <= lim
        assert np.abs(p[name]).max() >= 0.95 * lim
    for name in ("b1", "b2", "b3"):
        assert not np.any(p[name])


def test_kmeans_update_sums_in_fp64():
    # one Lloyd step with one cluster: the new centroid is the mean of the
    # 20 000 fp32 points summed in fp64 (exactly: math.fsum) and rounded to
    # fp32; an fp32 running sum of values near 1 000 drifts by about 0.1
    rng = np.random.default_rng(47)
    n = 20_000
    X = (1000.0 + rng.random((n, 2))).astype(np.float32)
    C = oracle.kmeans(X, np.array([0]), 1)
    want = np.array([math.fsum(X[:, j].astype(np.float64)) / n for j in range(2)]).astype(np.float32)
    np.testing.assert_array_equal(C[0], want)


# ------------------------------------------- IVF search by loops, edge cases

def _ivf_by_loops(Q, X, C, offsets, ids, k, tq):
    """One query's IVF search written out: partitions ranked by (-<q, c>, id),
    the first tq probed, their members as a set (a spilled point once), exact
    scores ranked by (-score, id), the first k kept, padded with (-1, -inf)."""
    q = [float(v) for v in Q]
    score = lambda v: sum(a * float(b) for a, b in zip(q, v))
    order = sorted(range(len(C)), key=lambda p: (-score(C[p]), p))
    members = set()
    for p in order[:tq]:
        members.update(int(i) for i in ids[offsets[p]:offsets[p + 1]])
    ranked = sorted(((-score(X[i]), i) for i in members))[:k]
    out = [(i, -s) for s, i in ranked]
    return out + [(-1, -math.inf)] * (k - len(out))


def test_ivf_search_by_loops_with_per_query_counts_padding_and_spills():
    # two spills, so a point met in up to three probed partitions must count
    # once; per-query probe counts 0 .. c, and k larger than a small union
    rng = np.random.default_rng(48)
    n, d, c = 90, 6, 9
    X = rng.standard_normal((n, d))
    Q = rng.standard_normal((12, d))
    C = oracle.kmeans(X, rng.choice(n, c, replace=False), 3).astype(np.float64)
    A = oracle.soar_assign(X, C, 1.0, 2)
    off, ids = oracle.build_ivf(A, c)
    tpq = np.array([0, 1, 2, 3, 9, 5, 1, 0, 4, 9, 2, 7])
    for k in (5, 60):
        got_i, got_s = oracle.ivf_search(Q, X, C, off, ids, k, 9, t_per_query=tpq)
        for i in range(12):
            want = _ivf_by_loops(Q[i], X, C, off, ids, k, int(tpq[i]))
            assert got_i[i].tolist() == [w[0] for w in want], (k, i)
            np.testing.assert_allclose(got_s[i], [w[1] for w in want], rtol=1e-12)
            real = got_i[i][got_i[i] >= 0]
            assert len(set(real.tolist())) == len(real)          # no point twice
        assert np.all(got_i[[0, 7]] == -1) and np.all(np.isneginf(got_s[[0, 7]]))
    # with t for every query the per-query form equals the plain one
    np.testing.assert_array_equal(oracle.ivf_search(Q, X, C, off, ids, 5, 4, t_per_query=np.full(12, 4))[0],
                                  oracle.ivf_search(Q, X, C, off, ids, 5, 4)[0])


def test_pq_search_per_query_counts_by_loops():
    # per-query probe counts (0 probes nothing): each row equals the loops
    # at that query's own count
    rng = np.random.default_rng(49)
    X = rng.standard_normal((200, 6)).astype(np.float32)
    Q = rng.standard_normal((6, 6)).astype(np.float32)
    C = oracle.kmeans(X, rng.choice(200, 8, replace=False), 3)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, 8)
    part = np.repeat(np.arange(8), np.diff(off))
    Rres = oracle.pq_residuals(X[ids], C, part)
    B = oracle.pq_train(Rres, 3, rng.choice(Rres.shape[0], 16, replace=False))
    codes = oracle.pq_index_codes(X, C, off, ids, B)
    tpq = np.array([3, 0, 1, 8, 2, 5])
    gi, _ = oracle.pq_search(Q, X, C, off, ids, B, codes, 4, 8, 12, t_per_query=tpq)
    for q in range(6):
        assert list(gi[q]) == _pq_search_by_loops(Q[q], X, C, off, ids, B, codes, 4, int(tpq[q]), 12)
    assert list(gi[1]) == [-1] * 4
