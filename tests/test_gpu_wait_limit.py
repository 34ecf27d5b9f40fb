"""The partition scan's bounded waits give up cleanly.

Every mbarrier wait of the scan has a limit; a CTA whose wait runs out
records the failure, stops, lets its copies and MMAs in flight land, frees
its tensor memory and returns (the waits are bounded so that a fault in the
pipeline can never hang the GPU).  Here the limit is set to one SM cycle for
one search, so that the first wait for a copy runs out: the search must
return, soar_check_device must report SOAR_ETIMEOUT, and the next search with
the default limit must be correct again.
"""
import numpy as np
import pytest
import torch

import oracle
import synth
from parity_util import topk_mismatches

pytestmark = pytest.mark.gpu


def test_a_wait_that_runs_out_is_reported_and_the_next_search_is_clean(soar):
    X, Q, init = synth.workload_arrays("tiny", nq=200)
    C = oracle.kmeans(X, init, 3)
    A = oracle.soar_assign(X, C, 1.0, 1)
    off, ids = oracle.build_ivf(A, C.shape[0])
    ix = soar.soar_index_build(torch.from_numpy(X).cuda(), torch.from_numpy(C).cuda(), torch.from_numpy(A).cuda())
    Qd = torch.from_numpy(Q).cuda()
    soar.soar_check_device()                     # nothing pending from earlier calls
    try:
        soar.soar_set_wait_limit(1)
        soar.soar_search(ix, Qd, 10, 4)
    finally:
        soar.soar_set_wait_limit(0)
    with pytest.raises(soar.SoarError) as e:
        soar.soar_check_device()
    assert e.value.status == soar.SOAR_ETIMEOUT
    soar.soar_check_device()                     # the failure was cleared
    gi, _ = soar.soar_search(ix, Qd, 10, 4)
    soar.soar_check_device()
    wi, ws = oracle.ivf_search(Q, X, C, off, ids, 10, 4)
    Xd, Qf = X.astype(np.float64), Q.astype(np.float64)
    assert topk_mismatches(gi.cpu().numpy(), wi, ws, lambda q, v: Xd[np.asarray(v)] @ Qf[q]) == []
    ix.close()
