"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Every test runs on the three product paths (FP32 CUDA cores, BF16 and FP8 e4m3 tensor
cores); the guard band and exact rescoring make their integer results identical.
Integer results (t_u, S_k(u), scores, top-N ids and scores, new-item counts) must be
identical.  tau_u must be bit-identical on grid inputs (where FP64 is exact); on
off-grid inputs it must agree with the oracle to 1e-12 relative (the two FP64 sums
may round differently), and the integer results must still agree.
"""
from __future__ import annotations

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

PRECISIONS = ["fp32", "bf16", "fp8"]


@pytest.fixture(scope="module")
def rkm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_13445_gb300 as m
    return m


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def check_thresholds(ctx, U, P, k, exact=True):
    tau_o, tid_o, topk_o = oracle.kmips(U, P, k)
    tau, tid, topk = ctx.thresholds(dev(U), dev(P), k, want_topk=True)
    tau, tid, topk = tau.cpu().numpy(), tid.cpu().numpy(), topk.cpu().numpy()
    if exact:
        assert np.array_equal(tau.view(np.uint64), tau_o.view(np.uint64)), "tau not bit-identical"
    else:
        np.testing.assert_allclose(tau, tau_o, rtol=1e-12, atol=1e-300)
    np.testing.assert_array_equal(tid, tid_o)
    np.testing.assert_array_equal(topk, topk_o)
    return tau_o, tid_o, topk_o


def full_check(ctx, U, P, k, N, exact=True):
    tau_o, tid_o, topk_o = check_thresholds(ctx, U, P, k, exact)
    sc_o = oracle.scores_histogram(topk_o, P.shape[0])
    sc = ctx.scores(dev(U), dev(P), dev(tau_o), dev(tid_o.astype(np.int32))).cpu().numpy()
    np.testing.assert_array_equal(sc, sc_o)
    ids_o, tops_o = oracle.topn(sc_o, N)
    ids, tops = ctx.topn(dev(U), dev(P), k, N)
    np.testing.assert_array_equal(ids.cpu().numpy(), ids_o)
    np.testing.assert_array_equal(tops.cpu().numpy(), tops_o)
    return tau_o, tid_o, sc_o


@pytest.mark.parametrize("prec", PRECISIONS)
def test_plain_workload(rkm, prec):
    W = workloads.make("plain-2k")
    with rkm.Context(prec) as ctx:
        full_check(ctx, W.U, W.P, W.k, W.N)
        st = ctx.stats()
        assert st["exact_integer_path"] == 1


@pytest.mark.parametrize("prec", PRECISIONS)
@pytest.mark.parametrize("shape", [(257, 300, 3, 5, 7), (1, 40, 1, 1, 40), (130, 517, 100, 25, 50),
                                   (300, 64, 128, 64, 64), (77, 1000, 256, 10, 17)])
def test_ragged_shapes(rkm, prec, shape):
    n, m, d, k, N = shape
    W = workloads.mf(n, m, d, k, N, seed=n + m + d)
    with rkm.Context(prec) as ctx:
        full_check(ctx, W.U, W.P, k, N)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_mid_size_mf_spans_many_tiles(rkm, prec):
    W = workloads.mf(20_000, 5_000, 64, 25, 50, seed=1)
    with rkm.Context(prec) as ctx:
        full_check(ctx, W.U, W.P, W.k, W.N)
        st = ctx.stats()
        assert st["items_counted"] <= W.m


@pytest.mark.parametrize("prec", ["bf16"])
def test_threshold_seed_order_and_stop(rkm, prec):
    """The tensor-core threshold pass with and without the seed order (a first pass over the
    highest-norm items, users grouped by bound / ||u||): identical thresholds and S_k(u), equal
    to the oracle's, and the Cauchy-Schwarz stop computes fewer than n*m products."""
    W = workloads.mf(24_000, 12_000, 128, 10, 20, seed=9)  # BF16 d = 128: two K-blocks per tile
    tau_o, tid_o, topk_o = oracle.kmips(W.U, W.P, W.k)
    out = []
    for order in (True, False):
        with rkm.Context(prec, seed_order=order) as ctx:
            tau, tid, topk = ctx.thresholds(dev(W.U), dev(W.P), W.k, want_topk=True)
            st = ctx.stats()
            out.append((tau.cpu().numpy(), tid.cpu().numpy(), topk.cpu().numpy()))
            assert st["threshold_launches"] == (2 if order else 1)
            # the seed pass computes n x 2048 products of its own
            assert 0 < st["threshold_pairs"] < W.n * W.m + (W.n * 2048 if order else 0)
    for tau, tid, topk in out:
        np.testing.assert_array_equal(tau.view(np.uint64), tau_o.view(np.uint64))
        np.testing.assert_array_equal(tid, tid_o)
        np.testing.assert_array_equal(topk, topk_o)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_filter_on_and_off_agree(rkm, prec):
    W = workloads.mf(30_000, 20_000, 32, 10, 20, seed=5)
    with rkm.Context(prec, filter=True) as a, rkm.Context(prec, filter=False) as b:
        ia, sa = a.topn(dev(W.U), dev(W.P), W.k, W.N)
        counted = a.stats()["items_counted"]
        ib, sb = b.topn(dev(W.U), dev(W.P), W.k, W.N)
    np.testing.assert_array_equal(ia.cpu().numpy(), ib.cpu().numpy())
    np.testing.assert_array_equal(sa.cpu().numpy(), sb.cpu().numpy())
    tau_o, tid_o, topk_o = oracle.kmips(W.U, W.P, W.k)
    ids_o, tops_o = oracle.topn(oracle.scores_histogram(topk_o, W.m), W.N)
    np.testing.assert_array_equal(ia.cpu().numpy(), ids_o)
    assert counted < W.m, "the Eq. 2 filter skipped no item on an MF-like workload"


@pytest.mark.parametrize("prec", PRECISIONS)
def test_ties_identical_items_and_duplicates(rkm, prec):
    rng = np.random.default_rng(7)
    U = (rng.integers(-64, 65, size=(300, 8)) / 64).astype(np.float32)
    P = np.tile((rng.integers(-64, 65, size=(1, 8)) / 64).astype(np.float32), (90, 1))
    P[40:50] = (rng.integers(-64, 65, size=(10, 8)) / 64).astype(np.float32)
    P[60] = P[41]
    with rkm.Context(prec) as ctx:
        full_check(ctx, U, P, 12, 15)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_zero_users_negative_thresholds_k_equals_m(rkm, prec):
    rng = np.random.default_rng(8)
    P = (rng.integers(1, 64, size=(50, 4)) / 64).astype(np.float32)
    U = -(rng.integers(1, 64, size=(200, 4)) / 64).astype(np.float32)
    U[::7] = 0.0
    with rkm.Context(prec) as ctx:
        full_check(ctx, U, P, 5, 9)
        full_check(ctx, U, P, 50, 50)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_off_grid_inputs_use_fp64_path(rkm, prec):
    rng = np.random.default_rng(9)
    U = rng.standard_normal((500, 24)).astype(np.float32)
    P = rng.standard_normal((700, 24)).astype(np.float32)
    assert not oracle.on_grid(U)
    with rkm.Context(prec) as ctx:
        full_check(ctx, U, P, 10, 20, exact=False)
        assert ctx.stats()["exact_integer_path"] == 0


@pytest.mark.parametrize("prec", PRECISIONS)
def test_new_item_queries(rkm, prec):
    W = workloads.mf(5_000, 2_000, 100, 20, 10, seed=3)
    tau_o, tid_o, _ = oracle.kmips(W.U, W.P, W.k)
    Q = workloads.queries(777, W.d, seed=4)
    Q[5] = W.P[17]  # a candidate equal to a catalogue item: ties at tau lose
    with rkm.Context(prec) as ctx:
        ctx.resident_set(dev(W.U), dev(tau_o), dev(tid_o.astype(np.int32)))
        for sl in (slice(0, 1), slice(0, 777), slice(100, 613)):
            got = ctx.query_new_items(dev(Q[sl])).cpu().numpy()
            np.testing.assert_array_equal(got, oracle.query_new_items(W.U, tau_o, Q[sl]))


@pytest.mark.parametrize("prec", PRECISIONS)
def test_item_bounds_theorem2(rkm, prec):
    W = workloads.mf(400, 300, 16, 5, 5, seed=12)
    tau_o, tid_o, topk_o = oracle.kmips(W.U, W.P, W.k)
    sc_o = oracle.scores_histogram(topk_o, W.m)
    exact = oracle.uscore(W.U, W.P, tau_o)
    with rkm.Context(prec) as ctx:
        us = ctx.item_bounds(dev(W.U), dev(W.P), dev(tau_o)).cpu().numpy()
    assert np.all(us >= exact)
    assert np.all(exact >= sc_o)
    assert np.mean(us - exact) < 0.05 * W.n  # bucketing loosens the count only slightly


@pytest.mark.parametrize("prec", PRECISIONS)
def test_deterministic_repeat(rkm, prec):
    W = workloads.mf(10_000, 3_000, 64, 10, 30, seed=21)
    with rkm.Context(prec) as ctx:
        a = [t.cpu().numpy() for t in ctx.topn(dev(W.U), dev(W.P), W.k, W.N, return_thresholds=True)]
        b = [t.cpu().numpy() for t in ctx.topn(dev(W.U), dev(W.P), W.k, W.N, return_thresholds=True)]
    for x, y in zip(a, b):
        np.testing.assert_array_equal(x, y)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_small_capacity_retries(rkm, prec):
    W = workloads.mf(3_000, 2_000, 32, 25, 10, seed=31)
    with rkm.Context(prec, cand_capacity=32, band_capacity=64) as ctx:
        full_check(ctx, W.U, W.P, W.k, W.N)


def test_grown_band_queue_holds_on_repeat_calls(rkm):
    # The first call overflows a 64-pair band queue and grows it; repeated calls on the same
    # inputs push a slightly different band (the order of users within a ratio bucket is not
    # fixed), and the grown queue keeps a margin for that: no further retries, same results.
    W = workloads.mf(20_000, 8_000, 64, 10, 20, seed=33)
    with rkm.Context("bf16", band_capacity=64) as ctx:
        first = [t.cpu().numpy() for t in ctx.topn(dev(W.U), dev(W.P), W.k, W.N, return_thresholds=True)]
        assert ctx.stats()["retries"] > 0
        for _ in range(3):
            again = [t.cpu().numpy() for t in ctx.topn(dev(W.U), dev(W.P), W.k, W.N, return_thresholds=True)]
            assert ctx.stats()["retries"] == 0
            for x, y in zip(first, again):
                np.testing.assert_array_equal(x, y)


def test_host_buffers_entry_point(rkm):
    W = workloads.make("plain-2k")
    tau_o, tid_o, topk_o = oracle.kmips(W.U, W.P, W.k)
    ids_o, tops_o = oracle.topn(oracle.scores_histogram(topk_o, W.m), W.N)
    with rkm.Context("fp32") as ctx:
        ids, tops = ctx.topn_host(W.U, W.P, W.k, W.N)
    np.testing.assert_array_equal(ids, ids_o)
    np.testing.assert_array_equal(tops, tops_o)


def test_invalid_arguments(rkm):
    W = workloads.plain(n=10, m=5, d=4, k=2, N=2, seed=1)
    with rkm.Context("fp32") as ctx:
        with pytest.raises(rkm.RkmError):
            ctx.thresholds(dev(W.U), dev(W.P), 6)       # k > m
        with pytest.raises(rkm.RkmError):
            ctx.topn(dev(W.U), dev(W.P), 2, 0)          # N < 1
        with pytest.raises(rkm.RkmError):
            ctx.query_new_items(dev(W.P))               # no resident users


@pytest.mark.parametrize("prec", PRECISIONS)
def test_adversarial_cancellation_rows(rkm, prec):
    """Rows whose products cancel almost completely: u . p is tiny next to ||u|| ||p||, the
    regime where BF16 rounding of the operands is largest relative to the scores, with many
    near-ties around tau_u.  The guard band must still give exact results."""
    rng = np.random.default_rng(77)
    d, n, m = 64, 600, 900
    base = rng.integers(1000, 4096, size=(1, d)).astype(np.float64)
    signs = np.where(np.arange(d) % 2 == 0, 1.0, -1.0)
    U = (base + rng.integers(-3, 4, size=(n, d))) / 4096
    P = (base * signs + rng.integers(-3, 4, size=(m, d))) / 4096
    P *= np.ldexp(1.0, rng.integers(-2, 2, size=(m, 1)))
    U = np.clip(U, -1, 1).astype(np.float32)
    P = np.clip(P, -2, 2).astype(np.float32)
    assert oracle.on_grid(U) and oracle.on_grid(P)
    with rkm.Context(prec) as ctx:
        full_check(ctx, U, P, 20, 30)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_extreme_row_magnitudes(rkm, prec):
    """Rows scaled by 2^70 and 2^-80: the FP8 operand exponent is clamped to [-60, 60], so
    these rows saturate or underflow in e4m3; the norms of the actual rounding error put
    their pairs in the guard band, and exact rescoring keeps every result exact."""
    W = workloads.mf(400, 300, 40, 7, 9, seed=61)
    U = W.U.copy()
    U[::5] *= np.float32(2.0 ** 70)
    U[1::5] *= np.float32(2.0 ** -80)
    P = W.P.copy()
    P[::7] *= np.float32(2.0 ** 20)
    assert oracle.on_grid(U) and oracle.on_grid(P)
    with rkm.Context(prec) as ctx:
        full_check(ctx, U, P, W.k, W.N)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_scores_from_topk_option(rkm, prec):
    """rkm_topn with scores taken as the histogram of the exact S_k(u) lists (no counting
    pass) gives the same top N as the oracle, with ties at tau_u and at the N-th score."""
    W = workloads.mf(20_000, 5_000, 64, 25, 50, seed=1)
    rng = np.random.default_rng(7)
    Ut = (rng.integers(-64, 65, size=(300, 8)) / 64).astype(np.float32)
    Pt = np.tile((rng.integers(-64, 65, size=(1, 8)) / 64).astype(np.float32), (90, 1))
    Pt[40:50] = (rng.integers(-64, 65, size=(10, 8)) / 64).astype(np.float32)
    for U, P, k, N in ((W.U, W.P, W.k, W.N), (Ut, Pt, 12, 15)):
        _, _, topk_o = oracle.kmips(U, P, k)
        ids_o, tops_o = oracle.topn(oracle.scores_histogram(topk_o, P.shape[0]), N)
        with rkm.Context(prec, scores_from_topk=True) as ctx:
            ids, tops, tau, tid = ctx.topn(dev(U), dev(P), k, N, return_thresholds=True)
        np.testing.assert_array_equal(ids.cpu().numpy(), ids_o)
        np.testing.assert_array_equal(tops.cpu().numpy(), tops_o)


@pytest.mark.parametrize("prec", PRECISIONS)
def test_topn_for_every_k_from_one_pass(rkm, prec):
    """One threshold pass at k_max = 50 keeps S_kmax(u); the top N for k = 1, 7, 25, 50 then
    follow from its prefixes (Section 4's offline/online split) and equal the oracle's."""
    W = workloads.mf(8_000, 3_000, 48, 50, 40, seed=17)
    kmax = 50
    with rkm.Context(prec) as ctx:
        _, _, lists = ctx.thresholds(dev(W.U), dev(W.P), kmax, want_topk=True)
        for k in (1, 7, 25, 50):
            _, _, topk_o = oracle.kmips(W.U, W.P, k)
            ids_o, tops_o = oracle.topn(oracle.scores_histogram(topk_o, W.m), W.N)
            ids, tops = ctx.topn_from_topk(lists, W.m, k, W.N)
            np.testing.assert_array_equal(ids.cpu().numpy(), ids_o)
            np.testing.assert_array_equal(tops.cpu().numpy(), tops_o)
        with pytest.raises(rkm.RkmError):
            ctx.topn_from_topk(lists, W.m, kmax + 1, W.N)
