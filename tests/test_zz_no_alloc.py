"""The top-N entry point that allocates no device memory.

It exists for callers that cannot call cudaMalloc (a process that reserves all device memory
up front, or code inside another library's memory manager).  Its result must equal the top N
returned by rkm_topn for the same problem, on two calls in a row (the second call reuses the
library's fixed scratch array and must clear what it needs).  This file is collected last so
that a run stopping at the first failure has run every other test before it.
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


def test_noalloc_topn_matches_rkm_topn_twice(rkm):
    W = workloads.mf(20_000, 6_000, 64, 25, 50, seed=41)
    U = torch.from_numpy(W.U).cuda()
    P = torch.from_numpy(W.P).cuda()
    with rkm.Context("bf16", filter=False) as ctx:
        ids_ref, sc_ref, tau, tid = ctx.topn(U, P, W.k, W.N, return_thresholds=True)
        scores = ctx.scores(U, P, tau, tid)
    torch.cuda.synchronize()
    for _ in range(2):
        ids, sc = rkm.rkm_topn_scores_noalloc(scores, W.N)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(ids.cpu().numpy(), ids_ref.cpu().numpy())
        np.testing.assert_array_equal(sc.cpu().numpy(), sc_ref.cpu().numpy())
    # and against the oracle's Definition 3 on the same scores
    ids_o, sc_o = oracle.topn(scores.cpu().numpy().astype(np.int64), W.N)
    np.testing.assert_array_equal(ids.cpu().numpy(), ids_o)


def test_noalloc_rejects_n_beyond_the_scratch(rkm):
    scores = torch.zeros(10_000, dtype=torch.int32, device="cuda")
    with pytest.raises(rkm.RkmError, match="4096"):
        rkm.rkm_topn_scores_noalloc(scores, 5000)


def _check_against_oracle(rkm, scores_np, N):
    scores = torch.from_numpy(scores_np.astype(np.int32)).cuda()
    ids, sc = rkm.rkm_topn_scores_noalloc(scores, N)
    torch.cuda.synchronize()
    ids_o, sc_o = oracle.topn(scores_np.astype(np.int64), N)
    np.testing.assert_array_equal(ids.cpu().numpy(), ids_o)
    np.testing.assert_array_equal(sc.cpu().numpy(), sc_o)


def test_noalloc_capacity_edge_and_ties(rkm):
    """N at the scratch capacity (4096) and N = m, on arrays whose many equal scores straddle
    the N-th key; then N = 4096 followed by N = 7, so that keys left in the shared array by a
    larger call are never read by a smaller one."""
    rng = np.random.default_rng(5)
    tied = rng.integers(0, 6, size=9_000)           # ~1500 items per score value
    _check_against_oracle(rkm, tied, 4096)
    small = rng.integers(0, 3, size=4096)
    _check_against_oracle(rkm, small, 4096)         # N = m at the capacity
    _check_against_oracle(rkm, small[:777], 777)    # N = m below it
    _check_against_oracle(rkm, tied, 4096)
    _check_against_oracle(rkm, tied, 7)


def test_noalloc_signed_scores(rkm):
    """Signed int32 scores (negative values, INT32_MIN and INT32_MAX) order as integers."""
    rng = np.random.default_rng(6)
    s = rng.integers(-50, 50, size=5_000)
    s[[3, 10, 4000]] = [np.iinfo(np.int32).min, np.iinfo(np.int32).max, -1]
    for N in (1, 33, 4096):
        _check_against_oracle(rkm, s, N)
