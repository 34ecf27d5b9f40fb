"""soar_select_partitions_static: the allocation-free variant of partition
selection, for callers that must not allocate device memory during a call
(a host framework that owns the device memory budget, or a serving thread
that must stay out of the CUDA allocator).  Its scratch is a fixed device
array inside the library, shared by every call on a device.

Checked through the C ABI against soar_select_partitions (which allocates
its scratch from the stream-ordered pool), on two calls in a row so that the
second call runs over the first one's leftovers in the shared array.  This
file is collected last and builds its own inputs, so it passes alone or after
the rest of the suite.
"""
import numpy as np
import pytest
import torch

import synth
from parity_util import topk_mismatches

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def index(soar):
    mix = synth.Mixture(48, 12, "isotropic", 0.3, param_seed=7)
    X = torch.from_numpy(mix.sample(6000, seed=8)).cuda()
    init = torch.from_numpy(synth.init_indices(6000, 96, seed=9)).cuda()
    C = soar.soar_train_centroids(X, 96, 3, init)
    A = soar.soar_assign(X, C, 1.0, 1)
    ix = soar.soar_index_build(X, C, A)
    yield ix, C.cpu().numpy().astype(np.float64), mix
    ix.close()


def _check_same(top_s, sc_s, top_r, sc_r, C, Q):
    exact = lambda q, p: C[np.asarray(p, np.int64)] @ Q[q].astype(np.float64)
    assert topk_mismatches(top_s, top_r, sc_r.astype(np.float64), exact) == []
    np.testing.assert_allclose(sc_s, sc_r, rtol=1e-6, atol=1e-7)


def test_static_variant_matches_allocating_variant_twice(soar, index):
    ix, C, mix = index
    for call, (nq, t, seed) in enumerate([(700, 24, 11), (333, 7, 12)]):
        Q = mix.sample(nq, seed=seed)
        Qd = torch.from_numpy(Q).cuda()
        top_s = torch.full((nq, t), -7, dtype=torch.int32, device="cuda")
        sc_s = torch.full((nq, t), float("nan"), dtype=torch.float32, device="cuda")
        soar.soar_select_partitions_static(ix, Qd, t, top_s, sc_s)
        top_r, sc_r = soar.soar_select_partitions(ix, Qd, t, with_scores=True)
        torch.cuda.synchronize()
        _check_same(top_s.cpu().numpy(), sc_s.cpu().numpy(), top_r.cpu().numpy(), sc_r.cpu().numpy(), C, Q)


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
