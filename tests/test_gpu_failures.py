"""Failure handling on the GPU without a fault: a device wait that runs out.

Every wait in the library's kernels is bounded.  rkm_debug_wait_timeout runs the product
kernels' own bounded mbarrier wait, with a short limit, on a barrier that nothing completes;
the wait must give up, the kernel must return, the call must report RKM_ETIMEOUT, and the
same context must then compute a correct top N.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rkm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_13445_gb300 as m
    return m


def test_bounded_wait_times_out_and_context_survives(rkm):
    W = workloads.plain(n=500, m=300, d=32, k=5, N=8, seed=4)
    tau_o, tid_o, topk_o = oracle.kmips(W.U, W.P, W.k)
    ids_o, tops_o = oracle.topn(oracle.scores_histogram(topk_o, W.m), W.N)
    U = torch.from_numpy(W.U).cuda()
    P = torch.from_numpy(W.P).cuda()
    with rkm.Context("bf16") as ctx:
        for limit in (1, 2_000_000):  # about a millisecond at most
            with pytest.raises(rkm.RkmError) as e:
                rkm.rkm_debug_wait_timeout(ctx.handle, limit)
            assert e.value.status == 5  # RKM_ETIMEOUT
        ids, tops = ctx.topn(U, P, W.k, W.N)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy(), ids_o)
        np.testing.assert_array_equal(tops.cpu().numpy(), tops_o)
        with pytest.raises(rkm.RkmError):
            rkm.rkm_debug_wait_timeout(ctx.handle, 0)  # argument check, no launch
