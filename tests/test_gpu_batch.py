"""Batches of independent problems (one persistent threshold launch, a captured graph) give the
same top-N as the single-problem entry point and as the oracle, also when the graph is
replayed and when the counting tiles are autotuned."""
import os

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SHAPES = [(3000, 800, 32, 5, 20), (40_000, 7000, 64, 10, 20), (1500, 5000, 128, 25, 20),
          (700, 300, 100, 25, 7), (12_000, 2500, 64, 5, 20), (129, 257, 32, 10, 9)]


@pytest.fixture(scope="module")
def rkm():
    import __graft_entry__
    __graft_entry__.build()
    import paper_2504_13445_gb300 as m
    return m


@pytest.fixture(scope="module")
def problems():
    ws = [workloads.mf(n, m, d, k, N, seed=500 + j) for j, (n, m, d, k, N) in enumerate(SHAPES)]
    return ws, [(torch.from_numpy(W.U).cuda(), torch.from_numpy(W.P).cuda(), W.k, W.N) for W in ws]


def expected(W):
    _, _, topk = oracle.kmips(W.U, W.P, W.k)
    return oracle.topn(oracle.scores_histogram(topk, W.m), W.N)


@pytest.mark.parametrize("prec", ["bf16", "fp32", "fp8"])
def test_batch_matches_oracle_and_replays(rkm, problems, prec):
    ws, probs = problems
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream), rkm.Context(prec) as ctx:
        outs = ctx.topn_batch(probs)
        first = [(i.cpu().numpy(), s.cpu().numpy()) for i, s in outs]
        for _ in range(2):  # same layout: the captured graph is replayed
            outs = ctx.topn_batch(probs, outs)
            torch.cuda.synchronize()
            for (i, s), (i0, s0) in zip(outs, first):
                np.testing.assert_array_equal(i.cpu().numpy(), i0)
                np.testing.assert_array_equal(s.cpu().numpy(), s0)
        st = ctx.stats()
        assert st["kernel_launches"] > 0
    for W, (ids, sc) in zip(ws, first):
        ids_o, sc_o = expected(W)
        np.testing.assert_array_equal(ids, ids_o)
        np.testing.assert_array_equal(sc, sc_o)


def test_batch_on_default_stream_and_with_autotune(rkm, problems, tmp_path):
    ws, probs = problems
    cache = str(tmp_path / "tune.txt")
    with rkm.Context("bf16", autotune=True, tune_cache=cache) as ctx:
        outs = ctx.topn_batch(probs)
        outs = ctx.topn_batch(probs, outs)
        torch.cuda.synchronize()
        got = [(i.cpu().numpy(), s.cpu().numpy()) for i, s in outs]
    assert os.path.exists(cache) and open(cache).read().strip()
    for line in open(cache).read().split("\n"):
        if line.strip():  # bucket, work-unit size, first-stage items
            key, g, s1 = line.split()
            assert int(g) in (8, 16, 32) and int(s1) in (4096, 16384)
    for W, (ids, sc) in zip(ws, got):
        ids_o, sc_o = expected(W)
        np.testing.assert_array_equal(ids, ids_o)
        np.testing.assert_array_equal(sc, sc_o)
    # a second context reads the cached choices instead of tuning again
    with rkm.Context("bf16", autotune=True, tune_cache=cache) as ctx:
        outs = ctx.topn_batch(probs)
        torch.cuda.synchronize()
    for W, (ids, sc) in zip(ws, outs):
        np.testing.assert_array_equal(ids.cpu().numpy(), expected(W)[0])


def test_batch_overflow_falls_back_exactly(rkm, problems):
    ws, probs = problems
    with rkm.Context("bf16", cand_capacity=32, band_capacity=64) as ctx:
        outs = ctx.topn_batch(probs)
        torch.cuda.synchronize()
        assert ctx.stats()["retries"] > 0
    for W, (ids, sc) in zip(ws, outs):
        ids_o, sc_o = expected(W)
        np.testing.assert_array_equal(ids.cpu().numpy(), ids_o)
        np.testing.assert_array_equal(sc.cpu().numpy(), sc_o)
