"""fp64 oracle for SOAR indexing and IVF search (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py`` (CPU baseline
and ``--impl reference``) may import this module.  It is independent of the
CUDA path.  All arithmetic is fp64 (numpy); integer results use explicit
tie rules:

* argmin over centroids: the lower centroid index wins a tie;
* top-t partitions and top-k neighbours: higher score first, the lower id
  wins a tie.

Notation follows the paper: X (datapoints, n x d), C (codebook, c x d),
pi (primary assignment), r = x - C[pi] (partitioning residual), r_hat =
r / ||r||, lambda (SOAR weight), t (partitions probed), k (neighbours).

Readings taken where the paper is silent (each one is listed with the others
in the design notes):

* spilled candidates exclude the centroids the point is already assigned to;
* r = 0 makes the penalty term vanish (r_hat := 0);
* a third or later assignment penalises the projection on every earlier
  residual direction: ||r'||^2 + lambda * sum_i <r', r_hat_i>^2;
* empty k-means clusters keep their previous centroid;
* Rank for a spilled point is the best rank over its partitions.
"""
from __future__ import annotations

import numpy as np

F64 = np.float64

__all__ = [
    "topk_desc", "mips_topk", "recall_at_k", "recall_at_k_tol", "rank",
    "primary_assign", "soar_loss", "soar_assign", "kmeans", "kmeans_objective",
    "build_ivf", "select_partitions", "ivf_search", "partition_positions",
    "kmr_curve", "datapoints_searched", "probe_labels", "fp8_e4m3_round",
    "quantize_rows_fp8", "select_partitions_fp8", "precision_search", "bf16_round",
    "multilevel_select", "multilevel_search", "pq_residuals", "pq_train", "pq_encode",
    "pq_index_codes", "pq_search",
]


# --------------------------------------------------------------------------
# Section 2.1: maximum inner product search, recall@k, Rank
# --------------------------------------------------------------------------

def topk_desc(scores: np.ndarray, k: int, ids: np.ndarray | None = None):
    """Top-k of a 1-D score vector: score descending, lower id first on ties.

    Returns (ids int64[k], scores f64[k]); when fewer than k entries exist the
    tail is padded with id -1 and score -inf.
    """
    scores = np.asarray(scores, dtype=F64)
    n = scores.shape[0]
    if ids is None:
        ids = np.arange(n, dtype=np.int64)
    ids = np.asarray(ids, dtype=np.int64)
    out_i = np.full(k, -1, dtype=np.int64)
    out_s = np.full(k, -np.inf, dtype=F64)
    if n == 0 or k == 0:
        return out_i, out_s
    if n > k:
        # every entry whose score reaches the k-th largest value is a
        # candidate; the exact order among them is settled by the sort below
        kth = np.partition(scores, n - k)[n - k]
        cand = np.nonzero(scores >= kth)[0]
    else:
        cand = np.arange(n)
    order = np.lexsort((ids[cand], -scores[cand]))[:k]
    m = order.shape[0]
    out_i[:m] = ids[cand[order]]
    out_s[:m] = scores[cand[order]]
    return out_i, out_s


def mips_topk(Q: np.ndarray, X: np.ndarray, k: int, chunk: int = 64):
    """MIPS_k(q, X): the k datapoints of largest <q, x> (Section 2.1), exact.

    Returns ids int64 [nq, k] and fp64 scores [nq, k].
    """
    Q = np.asarray(Q, dtype=F64)
    nq = Q.shape[0]
    ids = np.empty((nq, k), dtype=np.int64)
    sc = np.empty((nq, k), dtype=F64)
    Xd = np.asarray(X, dtype=F64)
    for lo in range(0, nq, chunk):
        S = Q[lo:lo + chunk] @ Xd.T
        for i in range(S.shape[0]):
            ids[lo + i], sc[lo + i] = topk_desc(S[i], k)
    return ids, sc


def recall_at_k(found: np.ndarray, truth: np.ndarray) -> np.ndarray:
    """recall@k = |MIPS_k(q, X) intersect S| / k per query (Section 2.1)."""
    k = truth.shape[1]
    out = np.empty(truth.shape[0], dtype=F64)
    for i in range(truth.shape[0]):
        f = set(int(v) for v in found[i] if v >= 0)
        out[i] = len(f.intersection(int(v) for v in truth[i])) / k
    return out


def recall_at_k_tol(found: np.ndarray, Q: np.ndarray, X: np.ndarray,
                    true_scores: np.ndarray, rel: float = 1e-4) -> np.ndarray:
    """recall@k where exact ties count as hits.

    The paper's recall assumes no ties.  Here a returned id is a hit when its
    exact fp64 score reaches the k-th true score minus ``rel`` relative; the
    count is capped at k.  Without ties this equals ``recall_at_k``.
    """
    k = true_scores.shape[1]
    out = np.empty(found.shape[0], dtype=F64)
    for i in range(found.shape[0]):
        f = np.unique(found[i][found[i] >= 0])
        if f.size == 0:
            out[i] = 0.0
            continue
        s = np.asarray(X[f], dtype=F64) @ np.asarray(Q[i], dtype=F64)
        kth = true_scores[i, k - 1]
        out[i] = min(k, int(np.sum(s >= kth - rel * abs(kth)))) / k
    return out


def rank(q: np.ndarray, v: np.ndarray, X: np.ndarray) -> int:
    """Rank(q, v, X) = sum over x in X of 1[<q,v> <= <q,x>] (Section 2.1)."""
    q = np.asarray(q, dtype=F64)
    sv = float(np.asarray(v, dtype=F64) @ q)
    return int(np.sum(np.asarray(X, dtype=F64) @ q >= sv))


# --------------------------------------------------------------------------
# Section 2.2: vector quantisation, primary assignment, inverted index
# --------------------------------------------------------------------------

def _sqdist(Xc: np.ndarray, C: np.ndarray, c2: np.ndarray) -> np.ndarray:
    """||x - C_i||^2 for a chunk of rows, all centroids, in fp64.

    Uses ||x||^2 - 2<x, C_i> + ||C_i||^2, the same quantity; in fp64 its
    rounding error (~1e-15 of ||x||^2) is far below every tolerance used.
    """
    x2 = np.einsum("ij,ij->i", Xc, Xc)
    D = x2[:, None] - 2.0 * (Xc @ C.T) + c2[None, :]
    return np.maximum(D, 0.0)


def primary_assign(X: np.ndarray, C: np.ndarray, chunk: int = 8192):
    """pi(x) = argmin_i ||x - C_i||^2 (Section 2.2), lower index on ties.

    Returns (pi int32 [n], best loss f64 [n], gap f64 [n]) where gap is the
    runner-up loss minus the best loss (inf when c == 1).
    """
    C = np.asarray(C, dtype=F64)
    n = X.shape[0]
    c2 = np.einsum("ij,ij->i", C, C)
    pi = np.empty(n, dtype=np.int32)
    best = np.empty(n, dtype=F64)
    gap = np.full(n, np.inf, dtype=F64)
    for lo in range(0, n, chunk):
        Xc = np.asarray(X[lo:lo + chunk], dtype=F64)
        D = _sqdist(Xc, C, c2)
        a = np.argmin(D, axis=1)
        rows = np.arange(D.shape[0])
        pi[lo:lo + chunk] = a
        best[lo:lo + chunk] = D[rows, a]
        if C.shape[0] > 1:
            D[rows, a] = np.inf
            gap[lo:lo + chunk] = D.min(axis=1) - best[lo:lo + chunk]
    return pi, best, gap


def soar_loss(x: np.ndarray, c_prime: np.ndarray, r: np.ndarray, lam: float) -> float:
    """SOAR assignment loss for one candidate, direct form (Theorem 3.1).

    L(r', r) = ||r'||^2 + lambda * ||proj_r r'||^2 with r' = x - c'.
    ||proj_r r'|| = |<r', r_hat>|; r = 0 makes the penalty vanish.
    """
    x = np.asarray(x, dtype=F64)
    rp = x - np.asarray(c_prime, dtype=F64)
    r = np.asarray(r, dtype=F64)
    nr = np.sqrt(r @ r)
    pen = 0.0 if nr == 0.0 else float((rp @ r) / nr) ** 2
    return float(rp @ rp) + lam * pen


def soar_assign(X: np.ndarray, C: np.ndarray, lam: float, spills: int,
                chunk: int = 4096, return_gaps: bool = False):
    """Primary plus SOAR spilled assignments (Section 3.4, Theorem 3.1).

    Row i of the result is [pi(x), pi'_1(x), ..., pi'_s(x)].  Spill j picks
    argmin over the centroids not yet assigned to x of
        ||x - c'||^2 + lambda * sum_{i<j} <x - c', r_hat_i>^2,
    where r_hat_i is the unit residual of the i-th earlier assignment (for
    j = 1 only the primary residual, which is the paper's loss).  The primary
    assignment comes first, as the indexing pipeline of Section 3.5 orders it.
    With ``return_gaps`` the result is (assign, gaps, best): gaps [n, 1+s]
    is runner-up minus best loss per decision, best [n, 1+s] the best loss;
    a decision is a near-tie when gap <= 1e-5 * best.
    """
    C = np.asarray(C, dtype=F64)
    n, c = X.shape[0], C.shape[0]
    if spills < 0 or c < 1 + spills:
        raise ValueError("need c >= 1 + spills")
    c2 = np.einsum("ij,ij->i", C, C)
    out = np.empty((n, 1 + spills), dtype=np.int32)
    gaps = np.full((n, 1 + spills), np.inf, dtype=F64)
    bests = np.zeros((n, 1 + spills), dtype=F64)
    for lo in range(0, n, chunk):
        Xc = np.asarray(X[lo:lo + chunk], dtype=F64)
        m = Xc.shape[0]
        rows = np.arange(m)
        D = _sqdist(Xc, C, c2)                       # ||x - c'||^2
        a0 = np.argmin(D, axis=1)
        out[lo:lo + m, 0] = a0
        bests[lo:lo + m, 0] = D[rows, a0]
        if c > 1:
            Dm = D.copy()
            Dm[rows, a0] = np.inf
            gaps[lo:lo + m, 0] = Dm.min(axis=1) - D[rows, a0]
        taken = np.zeros((m, c), dtype=bool)
        taken[rows, a0] = True
        pen = np.zeros((m, c), dtype=F64)
        prev = a0
        for j in range(1, 1 + spills):
            r = Xc - C[prev]
            nr = np.sqrt(np.einsum("ij,ij->i", r, r))
            rhat = np.where(nr[:, None] > 0, r / np.where(nr > 0, nr, 1.0)[:, None], 0.0)
            # <x - c', r_hat> = <x, r_hat> - <c', r_hat>
            proj = np.einsum("ij,ij->i", Xc, rhat)[:, None] - rhat @ C.T
            pen += proj * proj
            L = D + lam * pen
            L[taken] = np.inf
            aj = np.argmin(L, axis=1)
            out[lo:lo + m, j] = aj
            best = L[rows, aj]
            bests[lo:lo + m, j] = best
            L[rows, aj] = np.inf
            nxt = L.min(axis=1)
            gaps[lo:lo + m, j] = nxt - best
            taken[rows, aj] = True
            prev = aj
    if return_gaps:
        return out, gaps, bests
    return out


def kmeans_objective(X: np.ndarray, C: np.ndarray) -> float:
    """sum_x min_i ||x - C_i||^2, the quantity Lloyd's iteration lowers."""
    _, best, _ = primary_assign(X, C)
    return float(best.sum())


def kmeans(X: np.ndarray, init_idx: np.ndarray, iters: int, return_history: bool = False):
    """Lloyd's k-means producing the codebook C (Section 2.2).

    C starts as the rows X[init_idx].  Each iteration assigns every point to
    its nearest centroid (``primary_assign``), then sets each non-empty
    centroid to the fp64 mean of its points rounded to fp32; an empty cluster
    keeps its previous centroid.  Returns float32 C [c, d].
    """
    C = np.asarray(X[np.asarray(init_idx)], dtype=np.float32).copy()
    c, d = C.shape
    hist = []
    for _ in range(iters):
        pi, best, _ = primary_assign(X, C)
        hist.append(float(best.sum()))
        sums = np.zeros((c, d), dtype=F64)
        np.add.at(sums, pi, np.asarray(X, dtype=F64))
        cnt = np.bincount(pi, minlength=c)
        nz = cnt > 0
        C[nz] = (sums[nz] / cnt[nz, None]).astype(np.float32)
    if return_history:
        return C, hist
    return C


def build_ivf(assign: np.ndarray, c: int):
    """Inverted index {j | x_j assigned to partition i} per partition (Section 2.2).

    ``assign`` is [n, 1+s]; a spilled point appears in each of its
    partitions (Section 3.5).  Members of a partition are listed in
    ascending id.  Returns (offsets int64 [c+1], ids int32 [n(1+s)]).
    """
    assign = np.asarray(assign).reshape(assign.shape[0], -1)
    n, a = assign.shape
    part = assign.reshape(-1).astype(np.int64)
    pid = np.repeat(np.arange(n, dtype=np.int64), a)
    order = np.lexsort((pid, part))
    cnt = np.bincount(part, minlength=c)
    offsets = np.zeros(c + 1, dtype=np.int64)
    offsets[1:] = np.cumsum(cnt)
    return offsets, pid[order].astype(np.int32)


# --------------------------------------------------------------------------
# Section 2.2 (IVF search) and Section 3.5 (deduplication of spilled copies)
# --------------------------------------------------------------------------

def select_partitions(Q: np.ndarray, C: np.ndarray, t: int):
    """MIPS_t(q, C): the t partitions of largest <q, C_i>, ties to lower id.

    Returns (ids int32 [nq, t], scores f64 [nq, t]) in rank order.
    """
    S = np.asarray(Q, dtype=F64) @ np.asarray(C, dtype=F64).T
    nq = S.shape[0]
    ids = np.empty((nq, t), dtype=np.int32)
    sc = np.empty((nq, t), dtype=F64)
    for i in range(nq):
        a, b = topk_desc(S[i], t)
        ids[i], sc[i] = a, b
    return ids, sc


def ivf_search(Q, X, C, offsets, ids, k: int, t: int, t_per_query=None):
    """IVF search with deduplication (Section 2.2, Section 3.5).

    For each query: rank partitions by <q, C_i>, keep the top t (or the
    query's own t), take the union of their members with spilled copies
    removed, and return the exact top-k by <q, x> (fp64).  Returns ids int64
    [nq, k] (-1 padded) and scores f64 [nq, k] (-inf padded).
    """
    Q = np.asarray(Q, dtype=F64)
    nq = Q.shape[0]
    tmax = t if t_per_query is None else int(np.max(t_per_query))
    top, _ = select_partitions(Q, C, tmax)
    out_i = np.empty((nq, k), dtype=np.int64)
    out_s = np.empty((nq, k), dtype=F64)
    for i in range(nq):
        tq = t if t_per_query is None else int(t_per_query[i])
        parts = top[i, :tq]
        mem = np.concatenate([ids[offsets[p]:offsets[p + 1]] for p in parts]) if tq else np.empty(0, np.int32)
        mem = np.unique(mem).astype(np.int64)
        s = np.asarray(X[mem], dtype=F64) @ Q[i]
        out_i[i], out_s[i] = topk_desc(s, k, mem)
    return out_i, out_s


# --------------------------------------------------------------------------
# Product quantization of the partitioning residuals (Section 3.5, App. A.3)
# --------------------------------------------------------------------------

PQ_DIMS = 2        # dimensions per subspace
PQ_CENTRES = 16    # centres per subspace: 4-bit codes


def pq_residuals(X, C, part):
    """r = x - C[part] for every row, formed in fp32 (the stored precision of x and C)."""
    return (np.asarray(X, dtype=np.float32) - np.asarray(C, dtype=np.float32)[np.asarray(part)]).astype(np.float32)


def pq_train(R, iters: int, init_idx):
    """PQ codebooks of residuals R [n, d] (d even): for each subspace s (dims
    2s, 2s+1), Lloyd's k-means (``kmeans``) with 16 centres started from the
    rows ``init_idx`` (16 distinct rows, the same for every subspace).
    Returns B float32 [d/2, 16, 2]."""
    R = np.asarray(R, dtype=np.float32)
    n, d = R.shape
    assert d % PQ_DIMS == 0 and len(init_idx) == PQ_CENTRES
    return np.stack([kmeans(np.ascontiguousarray(R[:, PQ_DIMS * s:PQ_DIMS * (s + 1)]), init_idx, iters)
                     for s in range(d // PQ_DIMS)])


def pq_encode(R, B):
    """code[i, s] = argmin_j ||R[i, 2s:2s+2] - B[s, j]||^2, lower j on ties
    (``primary_assign`` per subspace).  Returns uint8 [n, d/2] (values < 16)."""
    R = np.asarray(R, dtype=np.float32)
    return np.stack([primary_assign(np.ascontiguousarray(R[:, PQ_DIMS * s:PQ_DIMS * (s + 1)]), B[s])[0]
                     for s in range(B.shape[0])], axis=1).astype(np.uint8)


def pq_index_codes(X, C, offsets, ids, B):
    """The PQ code of every index row: row r is the copy of point ids[r] in
    its partition p (offsets[p] <= r < offsets[p+1]), encoded from the
    residual x - C_p, so a spilled point has one code per copy (Section 3.5:
    the compressed form is duplicated, the full-precision row is not)."""
    part = np.repeat(np.arange(len(offsets) - 1), np.diff(offsets))
    return pq_encode(pq_residuals(np.asarray(X)[ids], C, part), B)


def pq_search(Q, X, C, offsets, ids, B, codes, k: int, t: int, rescore: int, t_per_query=None):
    """IVF search scoring the probed copies by their PQ codes, then exact rescoring.

    approx(q, copy in p) = <q, C_p> + sum_s <q_s, B[s, code_s]> (fp64).
    The top t partitions by <q, C> are probed in that order; a point met in
    several of them is scored by its copy in the first (earliest-probed)
    one.  The best ``rescore`` points by approximate score (higher first,
    lower id on ties) are rescored exactly as <q, x> (fp64) and the top k of
    those returned.  Returns (ids int64 [nq,k], exact scores f64 [nq,k]).
    """
    Q = np.asarray(Q, dtype=F64)
    nq = Q.shape[0]
    tmax = t if t_per_query is None else int(np.max(t_per_query))
    top, _ = select_partitions(Q, C, tmax)
    Cd, Bd = np.asarray(C, dtype=F64), np.asarray(B, dtype=F64)
    out_i = np.empty((nq, k), dtype=np.int64)
    out_s = np.empty((nq, k), dtype=F64)
    m = Bd.shape[0]
    for i in range(nq):
        tq = t if t_per_query is None else int(t_per_query[i])
        lut = np.einsum("sjd,sd->sj", Bd, Q[i].reshape(m, PQ_DIMS))       # <q_s, B[s, j]>
        seen = {}
        for p in top[i, :tq]:
            base = float(Cd[p] @ Q[i])
            for r in range(offsets[p], offsets[p + 1]):
                pid = int(ids[r])
                if pid not in seen:
                    seen[pid] = base + float(lut[np.arange(m), codes[r]].sum())
        mem = np.fromiter(seen.keys(), dtype=np.int64, count=len(seen))
        approx = np.fromiter(seen.values(), dtype=F64, count=len(seen))
        cand, _ = topk_desc(approx, rescore, mem)
        cand = cand[cand >= 0]
        exact = np.asarray(X[cand], dtype=F64) @ Q[i]
        out_i[i], out_s[i] = topk_desc(exact, k, cand)
    return out_i, out_s


# --------------------------------------------------------------------------
# Multi-level VQ (App. A.4, general index setup; Section 4)
# --------------------------------------------------------------------------

def multilevel_select(Q, C, C2, offsets2, ids2, t: int, t1: int):
    """Partition selection through a second VQ level.

    The fine centroids C (c x d) are themselves vector-quantized by a coarse
    codebook C2 into an IVF index over the rows of C (``offsets2``, ``ids2``
    from ``build_ivf``; a fine centroid may be spilled to several coarse
    partitions, since SOAR assigns at each level of the tree, Section 4).  A
    query ranks the coarse partitions by <q, C2_j>, probes the top t1, takes
    the union of their fine centroids (a spilled one counts once) and keeps
    the t with the largest <q, C_i>, higher score first, lower id on ties.
    That is an IVF search over the centroids (``ivf_search`` with C as the
    datapoints and k = t).  When the probed coarse partitions hold fewer than
    t fine centroids the rest of the row is padding (id -1, score -inf).
    Returns ids int64 [nq, t] and scores f64 [nq, t].
    """
    return ivf_search(Q, C, C2, offsets2, ids2, t, t1)


def multilevel_search(Q, X, C, offsets, ids, C2, offsets2, ids2, k: int, t: int, t1: int):
    """IVF search whose probed partitions come from ``multilevel_select``.

    Per query: the fine partitions it returns (padding dropped), the union of
    their members with spilled copies removed, and the exact top-k by
    <q, x> (fp64).  A query whose coarse probes hold no fine centroid probes
    nothing and gets only padding.  Returns ids int64 [nq, k] (-1 padded) and
    scores f64 [nq, k] (-inf padded).
    """
    Q = np.asarray(Q, dtype=F64)
    top, _ = multilevel_select(Q, C, C2, offsets2, ids2, t, t1)
    nq = Q.shape[0]
    out_i = np.empty((nq, k), dtype=np.int64)
    out_s = np.empty((nq, k), dtype=F64)
    for i in range(nq):
        parts = top[i][top[i] >= 0]
        if parts.size:
            mem = np.concatenate([ids[offsets[p]:offsets[p + 1]] for p in parts])
        else:
            mem = np.empty(0, np.int32)
        mem = np.unique(mem).astype(np.int64)
        s = np.asarray(X[mem], dtype=F64) @ Q[i]
        out_i[i], out_s[i] = topk_desc(s, k, mem)
    return out_i, out_s


# --------------------------------------------------------------------------
# Eq. 1 (KMR curve), Section 5.1 (datapoints searched), probe-count labels
# --------------------------------------------------------------------------

def partition_positions(Q: np.ndarray, C: np.ndarray) -> np.ndarray:
    """1-based position of every partition in each query's probe order.

    The order is the one ``select_partitions`` uses (score descending, lower
    id first on ties); without ties the position equals Rank(q, C_p, C).
    """
    S = np.asarray(Q, dtype=F64) @ np.asarray(C, dtype=F64).T
    nq, c = S.shape
    pos = np.empty((nq, c), dtype=np.int64)
    for i in range(nq):
        order = np.lexsort((np.arange(c), -S[i]))
        pos[i, order] = np.arange(1, c + 1)
    return pos


def kmr_curve(Q, C, assign, truth, ts) -> np.ndarray:
    """KMR(t) of Eq. 1 for each t in ``ts``.

    KMR(t) = (1 / (k |Q|)) sum_q sum_{v in MIPS_k(q)} 1[Rank(q, C_pi(v), C) <= t].
    For a spilled index a neighbour counts as found when any of its
    partitions is within the top t (its best rank over its assignments).
    Rank counts every centroid scoring at least as high, as Section 2.1
    defines it.
    """
    S = np.asarray(Q, dtype=F64) @ np.asarray(C, dtype=F64).T
    assign = np.asarray(assign).reshape(assign.shape[0], -1)
    ts = np.asarray(ts)
    k = truth.shape[1]
    hits = np.zeros(ts.shape[0], dtype=F64)
    for i in range(S.shape[0]):
        best = np.full(k, np.iinfo(np.int64).max, dtype=np.int64)
        for j in range(assign.shape[1]):
            p = assign[truth[i], j]
            r = np.sum(S[i][None, :] >= S[i, p][:, None], axis=1)
            best = np.minimum(best, r)
        hits += np.sum(best[None, :] <= ts[:, None], axis=1)
    return hits / (k * S.shape[0])


def datapoints_searched(Q, C, offsets, t: int) -> np.ndarray:
    """Sum of the sizes of each query's top-t partitions (Section 5.1).

    Spilled copies count once per partition they sit in, as the paper's
    partition-size weighting does.
    """
    top, _ = select_partitions(Q, C, t)
    sizes = np.diff(np.asarray(offsets))
    return sizes[top].sum(axis=1)


def probe_labels(Q, C, assign, truth, target: float = 0.9) -> np.ndarray:
    """Smallest t at which a query's recall@k reaches ``target``.

    A true neighbour v is found at probe count t exactly when one of its
    partitions has position <= t in the query's probe order, so recall(t)
    = #{v : pos_v <= t} / k and the smallest sufficient t is the
    ceil(target k)-th smallest pos_v.
    """
    pos = partition_positions(Q, C)
    assign = np.asarray(assign).reshape(assign.shape[0], -1)
    k = truth.shape[1]
    need = int(np.ceil(target * k - 1e-9))
    out = np.empty(truth.shape[0], dtype=np.int32)
    for i in range(truth.shape[0]):
        pv = pos[i][assign[truth[i]]].min(axis=1)
        out[i] = np.sort(pv)[need - 1]
    return out


# --------------------------------------------------------------------------
# Low-precision scoring with exact rescoring (the FP8/BF16 extension)
# --------------------------------------------------------------------------

def bf16_round(v: np.ndarray) -> np.ndarray:
    """Round fp32 values to the nearest bfloat16 (ties to even), as fp32."""
    u = np.asarray(v, dtype=np.float32).view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    u = (u + 0x7FFF + lsb) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32)


def fp8_e4m3_round(v: np.ndarray) -> np.ndarray:
    """Nearest FP8 E4M3 value (ties to even, saturating at +-448), as fp32.

    E4M3: 1 sign, 4 exponent bits (bias 7), 3 mantissa bits; normal values
    2^(e-7) (1 + m/8) for e in 1..15 (the all-ones pattern is NaN, so 448 is
    the largest finite value); subnormals m/8 * 2^-6.
    """
    v = np.asarray(v, dtype=np.float64)
    a = np.abs(v)
    e = np.floor(np.log2(np.where(a > 0, a, 1.0)))
    e = np.maximum(e, -6.0)                 # subnormal spacing below 2^-6
    step = np.exp2(e - 3.0)                 # 3 mantissa bits
    q = np.round(a / step) * step           # numpy rounds half to even
    q = np.minimum(q, 448.0)
    return (np.sign(v) * q).astype(np.float32)


def quantize_rows_fp8(R: np.ndarray):
    """Per-row scaled FP8: scale = max|row| / 448, codes = e4m3(row / scale).

    The division is done in fp32, as the codes are an fp32 decision.
    Returns (codes as fp32 values [m, d], scales fp32 [m]); an all-zero row
    gets scale 1.
    """
    R = np.asarray(R, dtype=np.float32)
    amax = np.max(np.abs(R), axis=1)
    scale = np.where(amax > 0, amax / np.float32(448.0), np.float32(1.0)).astype(np.float32)
    codes = fp8_e4m3_round((R / scale[:, None]).astype(np.float32))
    return codes, scale


def select_partitions_fp8(Q, C, t: int):
    """MIPS_t(q, C) on the scaled FP8 forms of queries and centroids.

    score(q, C_i) = s_q * s_c * sum_j q8_j c8_j (fp64 sum of the decoded
    codes); ties to the lower id.  Returns (ids int32 [nq, t], scores f64).
    """
    q8, qs = quantize_rows_fp8(np.asarray(Q, dtype=np.float32))
    c8, cs = quantize_rows_fp8(np.asarray(C, dtype=np.float32))
    Sc = (q8.astype(F64) @ c8.astype(F64).T) * qs[:, None].astype(F64) * cs[None, :].astype(F64)
    nq = Sc.shape[0]
    ids = np.empty((nq, t), dtype=np.int32)
    sc = np.empty((nq, t), dtype=F64)
    for i in range(nq):
        ids[i], sc[i] = topk_desc(Sc[i], t)
    return ids, sc


def precision_search(Q, X, C, offsets, ids, k: int, t: int, rescore: int):
    """Low-precision IVF search followed by exact rescoring.

    Queries, centroids and datapoints are scored from their per-row scaled
    FP8 forms (score = s_q * s_x * sum q8_i x8_i, summed in fp64 here); the
    top t partitions are probed, spilled copies removed, the best
    ``rescore`` candidates kept, and those are rescored exactly as
    <q, x> over the stored (bf16) values; the top-k of the rescored list is
    returned.  Returns (ids int64 [nq,k], exact scores f64 [nq,k]).
    """
    Qf = np.asarray(Q, dtype=np.float32)
    q8, qs = quantize_rows_fp8(Qf)
    top, _ = select_partitions_fp8(Qf, C, t)
    nq = Qf.shape[0]
    out_i = np.empty((nq, k), dtype=np.int64)
    out_s = np.empty((nq, k), dtype=F64)
    for i in range(nq):
        parts = top[i]
        mem = np.unique(np.concatenate([ids[offsets[p]:offsets[p + 1]] for p in parts])).astype(np.int64)
        x8, xs = quantize_rows_fp8(np.asarray(X[mem], dtype=np.float32))
        approx = (x8.astype(F64) @ q8[i].astype(F64)) * xs.astype(F64) * F64(qs[i])
        cand, _ = topk_desc(approx, rescore, mem)
        cand = cand[cand >= 0]
        exact = np.asarray(X[cand], dtype=F64) @ Qf[i].astype(F64)
        out_i[i], out_s[i] = topk_desc(exact, k, cand)
    return out_i, out_s
