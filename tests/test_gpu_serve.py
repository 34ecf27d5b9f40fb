"""Continuous-batching serving loop (soar_server_*) on the GPU.

A request's result must not depend on what else shares its batch: every
request of a concurrent, mixed-k / mixed-t stream is compared with the same
query searched alone through soar_search.
"""
import threading

import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import topk_mismatches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def served(soar):
    X, Q, init = synth.workload_arrays("tiny", nq=400)
    C = oracle.kmeans(X, init, 10)
    A = oracle.soar_assign(X, C, 1.0, 1)
    ix = soar.soar_index_build(torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(), torch.from_numpy(A).cuda())
    ix.centroids_host = C
    ix.ivf_host = oracle.build_ivf(A, C.shape[0])
    yield X, Q, ix
    ix.close()


def _alone(soar, ix, q, k, t):
    ids, sc = soar.soar_search(ix, torch.from_numpy(q[None, :]).cuda(), k, t)
    return ids.cpu().numpy()[0], sc.cpu().numpy()[0]


def test_results_equal_alone_and_in_a_concurrent_mix(soar, served):
    X, Q, ix = served
    rng = np.random.default_rng(9)
    ks = rng.choice([10, 100], size=len(Q))
    ts = rng.integers(1, 17, size=len(Q))
    srv = soar.Server(ix, max_batch=48, streams=3, memory_budget=1 << 28, max_k=100)
    rids = [None] * len(Q)

    def producer(lo, hi):
        for i in range(lo, hi):
            rids[i] = srv.submit(Q[i], int(ks[i]), int(ts[i]))

    threads = [threading.Thread(target=producer, args=(j * 100, (j + 1) * 100)) for j in range(4)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    Xd, Qd = X.astype(np.float64), Q.astype(np.float64)
    for i in range(len(Q)):
        ids, sc, lat = srv.wait(rids[i], int(ks[i]))
        want_ids, want_sc = _alone(soar, ix, Q[i], int(ks[i]), int(ts[i]))
        ex = lambda q, v: Xd[np.asarray(v, np.int64)] @ Qd[i]
        assert topk_mismatches(ids[None], want_ids[None], want_sc[None].astype(np.float64), ex) == [], i
        np.testing.assert_allclose(sc, want_sc, rtol=1e-6, atol=1e-7)
        assert lat > 0
    st = srv.stats()
    assert st["completed"] == len(Q) and st["pending"] == 0
    assert st["queries_in_batches"] == len(Q)
    assert st["batches"] < len(Q)                  # requests were batched
    srv.close()


def test_served_results_match_the_oracle(soar, served):
    # each request of a replayed mixed stream against the oracle's search of
    # that one query with its own k and t over the same index
    X, Q, ix = served
    n = 160
    rng = np.random.default_rng(23)
    ks = rng.choice([10, 40, 100], size=n).astype(np.int32)
    ts = rng.integers(1, 17, size=n).astype(np.int32)
    arrivals = np.sort(rng.uniform(0.0, 0.02, size=n))
    srv = soar.Server(ix, max_batch=32, streams=3, memory_budget=1 << 28, max_k=100)
    rids = srv.submit_many(Q[:n], ks, ts, arrival_s=arrivals)
    ids, sc, _ = srv.wait_many(rids, 100)
    srv.close()
    C = ix.centroids_host
    off, iv = ix.ivf_host
    Xd, Qd = X.astype(np.float64), Q.astype(np.float64)
    for i in range(n):
        k, t = int(ks[i]), int(ts[i])
        wi, ws = oracle.ivf_search(Q[i:i + 1], X, C, off, iv, k, t)
        ex = lambda q, v: Xd[np.asarray(v, np.int64)] @ Qd[i]
        assert topk_mismatches(ids[i:i + 1, :k], wi, ws, ex) == [], i
        ok = wi[0] >= 0
        np.testing.assert_allclose(sc[i, :k][ok], ws[0][ok], rtol=1e-5, atol=1e-6)


def test_replayed_arrivals_match_alone_results(soar, served):
    X, Q, ix = served
    n = len(Q)
    rng = np.random.default_rng(21)
    ks = rng.choice([10, 40, 100], size=n).astype(np.int32)
    ts = rng.integers(1, 17, size=n).astype(np.int32)
    arrivals = np.sort(rng.uniform(0.0, 0.05, size=n))       # a 50 ms trace
    srv = soar.Server(ix, max_batch=64, streams=3, memory_budget=1 << 28, max_k=100)
    rids = srv.submit_many(Q, ks, ts, arrival_s=arrivals)
    ids, sc, lat = srv.wait_many(rids, 100)
    Xd, Qd = X.astype(np.float64), Q.astype(np.float64)
    for i in range(n):
        want_ids, want_sc = _alone(soar, ix, Q[i], int(ks[i]), int(ts[i]))
        ex = lambda q, v: Xd[np.asarray(v, np.int64)] @ Qd[i]
        got = ids[i, :ks[i]]
        assert topk_mismatches(got[None], want_ids[None], want_sc[None].astype(np.float64), ex) == [], i
        assert np.all(ids[i, ks[i]:] == -1) and np.all(np.isneginf(sc[i, ks[i]:]))
    assert np.all(lat > 0)
    st = srv.stats()
    assert st["completed"] == n and st["pending"] == 0
    with pytest.raises(soar.SoarError):
        srv.submit_many(Q[:2], [10, 101], [4, 4])          # one bad k rejects the call
    srv.close()


def test_batches_overlap_on_the_gpu(soar, served):
    X, Q, ix = served
    srv = soar.Server(ix, max_batch=16, streams=4, memory_budget=1 << 30, max_k=10)
    rids = [srv.submit(Q[i % len(Q)], 10, 16) for i in range(2000)]
    for r in rids:
        srv.wait(r, 10)
    st = srv.stats()
    assert st["max_in_flight"] >= 2, st
    assert st["p99_ms"] >= st["p50_ms"] > 0
    srv.close()


def test_memory_budget_limits_admission(soar, served):
    X, Q, ix = served
    # a budget below one request: only a lone request runs at a time
    srv = soar.Server(ix, max_batch=64, streams=4, memory_budget=1, max_k=10)
    rids = [srv.submit(Q[i], 10, 4) for i in range(50)]
    for i, r in enumerate(rids):
        ids, sc, _ = srv.wait(r, 10)
        want_ids, _ = _alone(soar, ix, Q[i], 10, 4)
        np.testing.assert_array_equal(ids, want_ids)
    st = srv.stats()
    assert st["max_in_flight"] == 1 and st["batches"] == 50
    srv.close()


def test_invalid_requests_are_rejected(soar, served):
    X, Q, ix = served
    srv = soar.Server(ix, max_batch=8, streams=1, memory_budget=1 << 20, max_k=10)
    with pytest.raises(soar.SoarError):
        srv.submit(Q[0], 11, 4)                     # k above max_k
    with pytest.raises(soar.SoarError):
        srv.submit(Q[0], 10, 0)                     # t below 1
    with pytest.raises(soar.SoarError):
        srv.wait(12345, 10, timeout_ms=10)          # never issued
    srv.close()
