"""Parity at the benchmark's full sizes, in the launch configuration bench.py times.

On the 500,000 x 100,000 workload (5e10 pairs) the oracle runs in full on every host core:
tau_u, t_u and S_k(u) of every user, every item's score and the top N are compared with
the oracle's own, element by element.  The oracle cannot score the 1e12 pairs of the
2,000,000 x 500,000 workloads in a test, so there:
* tau_u, t_u and S_k(u) are compared bit for bit on a seeded sample of 4,096 users that the
  oracle rescores one by one against every item;
* the scores satisfy sum(score) = n*k, and the two Section 2.2 formulations agree on the
  GPU (histogram of S_k(u) from rkm_thresholds vs per-item counting from rkm_scores);
* the filtered top-N of rkm_topn equals the top-N of the full score vector (the Eq. 2
  filter never changes the answer), and the Eq. 2 bound dominates every score (Theorem 2);
* rkm_topn with scores as the histogram of S_k(u) (no counting pass) gives the same top N;
* the BF16 tensor-core path and the FP32 CUDA-core path return identical integers, and so
  do the FP8 and BF16 tensor-core paths on the 2M x 500K precision workload.
"""
import os

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


def sample_users(n, count, seed):
    rng = np.random.default_rng(seed)
    return np.unique(np.r_[0, n - 1, rng.integers(0, n, size=count)])


def check_full(rkm, W, prec, sample, check_fp32=False, check_bf16=False, full_oracle=False):
    U = torch.from_numpy(W.U).cuda()
    P = torch.from_numpy(W.P).cuda()
    with rkm.Context(prec) as ctx:
        ids, tops, tau, tid = ctx.topn(U, P, W.k, W.N, return_thresholds=True)
        tau2, tid2, topk = ctx.thresholds(U, P, W.k, want_topk=True)
        scores = ctx.scores(U, P, tau2, tid2)
        us = ctx.item_bounds(U, P, tau2)
    tau, tid, tau2, tid2 = (x.cpu().numpy() for x in (tau, tid, tau2, tid2))
    topk = topk.cpu().numpy()
    scores = scores.cpu().numpy().astype(np.int64)
    us = us.cpu().numpy().astype(np.int64)
    # the same thresholds from both entry points
    np.testing.assert_array_equal(tau.view(np.uint64), tau2.view(np.uint64))
    np.testing.assert_array_equal(tid, tid2)
    threads = os.cpu_count() or 1
    if full_oracle:
        # every user, every item: the oracle's Definition 1, the first Section 2.2 baseline
        # and Definition 3, on all host cores
        t_o, i_o, k_o = oracle.kmips(W.U, W.P, W.k, block=64, threads=threads)
        sc_o = oracle.scores_histogram(k_o, W.m)
        np.testing.assert_array_equal(tau.view(np.uint64), t_o.view(np.uint64))
        np.testing.assert_array_equal(tid, i_o)
        np.testing.assert_array_equal(topk, k_o)
        np.testing.assert_array_equal(scores, sc_o)
        ids_o, tops_o = oracle.topn(sc_o, W.N)
    else:
        # sampled users against the oracle
        t_o, i_o, k_o = oracle.kmips(W.U[sample], W.P, W.k, block=64, threads=threads)
        np.testing.assert_array_equal(tau[sample].view(np.uint64), t_o.view(np.uint64))
        np.testing.assert_array_equal(tid[sample], i_o)
        np.testing.assert_array_equal(topk[sample], k_o)
        ids_o, tops_o = oracle.topn(scores, W.N)
    # invariants of the scores
    assert int(scores.sum()) == W.n * W.k
    np.testing.assert_array_equal(scores, np.bincount(topk.ravel(), minlength=W.m))
    assert np.all(us >= scores)
    np.testing.assert_array_equal(ids.cpu().numpy(), ids_o)
    np.testing.assert_array_equal(tops.cpu().numpy(), tops_o)
    with rkm.Context(prec, scores_from_topk=True) as ch:
        ih, sh = ch.topn(U, P, W.k, W.N)
    np.testing.assert_array_equal(ih.cpu().numpy(), ids_o)
    np.testing.assert_array_equal(sh.cpu().numpy(), tops_o)
    if check_bf16:
        with rkm.Context("bf16") as c16:
            i16, s16, t16, d16 = c16.topn(U, P, W.k, W.N, return_thresholds=True)
        np.testing.assert_array_equal(t16.cpu().numpy().view(np.uint64), tau.view(np.uint64))
        np.testing.assert_array_equal(d16.cpu().numpy(), tid)
        np.testing.assert_array_equal(i16.cpu().numpy(), ids_o)
        np.testing.assert_array_equal(s16.cpu().numpy(), tops_o)
    if check_fp32:
        with rkm.Context("fp32") as c32:
            i32, s32, t32, d32 = c32.topn(U, P, W.k, W.N, return_thresholds=True)
        np.testing.assert_array_equal(t32.cpu().numpy().view(np.uint64), tau.view(np.uint64))
        np.testing.assert_array_equal(d32.cpu().numpy(), tid)
        np.testing.assert_array_equal(i32.cpu().numpy(), ids_o)
        np.testing.assert_array_equal(s32.cpu().numpy(), tops_o)


def test_mf_500k_full_size_bf16_and_fp32_identical(rkm):
    """Every threshold, S_k(u) list and score of the 500,000 x 100,000 workload against the
    full oracle (about four minutes on 16 host cores)."""
    W = workloads.make("mf-500k")
    check_full(rkm, W, "bf16", None, check_fp32=True, full_oracle=True)


def test_mf_2m_k50_full_size(rkm):
    W = workloads.make("mf-2m-k50")
    check_full(rkm, W, "bf16", sample_users(W.n, 4096, 2))


def test_mf_2m_k10_full_size_fp8_and_bf16_identical(rkm):
    """The precision workload (2,000,000 x 500,000, d = 128, k = 10, N = 100): FP8 e4m3
    products with per-row / per-tile power-of-two scales, checked against the oracle on
    sampled users and for identity with the BF16 path."""
    W = workloads.make("mf-2m-k10")
    check_full(rkm, W, "fp8", sample_users(W.n, 4096, 3), check_bf16=True)
