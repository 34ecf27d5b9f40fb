"""Row-sharded search (paper_2404_00774_gb300.sharded): every rank indexes one
contiguous block of the rows under the same codebook, searches it, and the
per-shard top-k lists are all-gathered and merged (Section 2.2 for the
probe, Section 3.5 for counting a point once).

CPU test: two gloo ranks run the module's sharding, gathering and id
offsets with the oracle's search and a merge written from the definition in
place of the library's kernels; the merged result must equal the oracle's
search over all rows.  GPU test: the library's own search and merge over two
shards on one device against the oracle.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle
import synth
from paper_2404_00774_gb300 import sharded


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _data():
    mix = synth.Mixture(16, 8, "isotropic", 0.3, param_seed=91)
    X = mix.sample(3001, seed=92)
    Q = mix.sample(40, seed=93)
    C = oracle.kmeans(X, synth.init_indices(3001, 20, seed=94), 4)
    return X, Q, C


def _oracle_search(shard):
    """soar_search's contract on a shard, computed by the oracle (local ids)."""
    X, C, off, ids = shard

    def search(_ix, Q, k, t):
        i, s = oracle.ivf_search(Q.numpy(), X, C, off, ids, k, t)
        return torch.from_numpy(i), torch.from_numpy(s.astype(np.float32))
    return search


def _merge_by_definition(gi, gs, k, offsets):
    """Top k of the union of the lists: score desc, lower id on ties."""
    nq, m, _ = gi.shape
    out_i = torch.full((nq, k), -1, dtype=torch.int64)
    out_s = torch.full((nq, k), -np.inf, dtype=torch.float32)
    for q in range(nq):
        cand = {}
        for j in range(m):
            for i, s in zip(gi[q, j].tolist(), gs[q, j].tolist()):
                if i >= 0:
                    cand[i + int(offsets[j])] = s
        best = sorted(cand.items(), key=lambda e: (-e[1], e[0]))[:k]
        for r, (i, s) in enumerate(best):
            out_i[q, r], out_s[q, r] = i, s
    return out_i, out_s


def _rank_main(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        X, Q, C = _data()
        lo, hi = sharded.shard_bounds(X.shape[0], rank, world)
        A = oracle.soar_assign(X[lo:hi], C, 1.0, 1)
        off, ids = oracle.build_ivf(A, C.shape[0])
        ids_g, sc_g = sharded.sharded_search(None, torch.from_numpy(Q), 10, 5, X.shape[0],
                                             search=_oracle_search((X[lo:hi], C, off, ids)),
                                             merge=_merge_by_definition)
        out[rank] = (ids_g.numpy(), sc_g.numpy(), (lo, hi))
    finally:
        dist.destroy_process_group()


def test_shard_bounds_cover_the_rows():
    for n, w in [(10, 3), (3001, 2), (7, 7), (5, 8)]:
        spans = [sharded.shard_bounds(n, r, w) for r in range(w)]
        assert spans[0][0] == 0 and spans[-1][1] == n
        assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
        sizes = [h - l for l, h in spans]
        assert max(sizes) - min(sizes) <= 1


def test_two_gloo_ranks_equal_the_unsharded_search():
    world, port = 2, _free_port()
    with mp.get_context("spawn").Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    X, Q, C = _data()
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, C.shape[0])
    want_i, want_s = oracle.ivf_search(Q, X, C, off, ids, 10, 5)
    for r in range(world):
        got_i, got_s, _ = res[r]
        np.testing.assert_array_equal(got_i, want_i)
        np.testing.assert_allclose(got_s, want_s, rtol=1e-6)
    assert res[0][2][1] == res[1][2][0]


@pytest.mark.gpu
def test_merge_of_two_shards_on_one_gpu_matches_oracle(soar):
    # the library's search of each shard and its merge kernel (with the
    # shards' id offsets) against the oracle's search of all rows
    X, Q, C = _data()
    dev = "cuda"
    lists_i, lists_s, offs = [], [], []
    for r in range(2):
        lo, hi = sharded.shard_bounds(X.shape[0], r, 2)
        A = oracle.soar_assign(X[lo:hi], C, 1.0, 1)
        ix = soar.soar_index_build(torch.from_numpy(X[lo:hi]).to(dev), torch.from_numpy(C).to(dev),
                                   torch.from_numpy(A).to(dev))
        i, s = soar.soar_search(ix, torch.from_numpy(Q).to(dev), 10, 5)
        lists_i.append(i)
        lists_s.append(s)
        offs.append(lo)
        ix.close()
    gi = torch.stack(lists_i, dim=1).contiguous()
    gs = torch.stack(lists_s, dim=1).contiguous()
    mi, ms = soar.soar_merge_topk(gi, gs, 10, torch.tensor(offs, dtype=torch.int64, device=dev))
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, C.shape[0])
    want_i, want_s = oracle.ivf_search(Q, X, C, off, ids, 10, 5)
    np.testing.assert_array_equal(mi.cpu().numpy(), want_i)
    np.testing.assert_allclose(ms.cpu().numpy(), want_s, rtol=1e-5, atol=1e-6)
