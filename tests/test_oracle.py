"""Pins for the FP64 oracle: it is checked against things other than itself.

* brute force in exact rational arithmetic (Python Fractions, full sorts) on tiny
  inputs, plus the independent rank-count formulation of Definition 1;
* the invariant sum_i score(i) = n*k (each user contributes exactly k members);
* the two baselines of Section 2.2 (histogram of S_k(u) vs per-item counting);
* Theorem 2 (uscore >= score) for the Eq. 2 bound;
* closed-form tie cases and hand-derived golden fixtures (tests/golden/);
* planted mistakes: mutated copies of oracle functions must fail a pin.
"""
from __future__ import annotations

import types
from fractions import Fraction

import numpy as np
import pytest

import oracle
import workloads
from tests import golden_io


# ---------------------------------------------------------------- helpers

def tiny_grid(n, m, d, seed, levels=3, scale_rows=False):
    """Tiny grid inputs with many exact ties: entries in {-levels..levels}/4 * 2^e."""
    rng = np.random.default_rng(seed)
    U = rng.integers(-levels, levels + 1, size=(n, d)).astype(np.float64) / 4
    P = rng.integers(-levels, levels + 1, size=(m, d)).astype(np.float64) / 4
    if scale_rows:
        U *= np.ldexp(1.0, rng.integers(-3, 2, size=(n, 1)))
        P *= np.ldexp(1.0, rng.integers(-3, 2, size=(m, 1)))
    if m >= 3:
        P[m - 1] = P[0]            # a duplicate item row
    return U.astype(np.float32), P.astype(np.float32)


def brute_force(U, P, k):
    """Definition 1 by exact rational inner products and a full sort per user."""
    n, m = len(U), len(P)
    Uf = [[Fraction(float(v)) for v in row] for row in U]
    Pf = [[Fraction(float(v)) for v in row] for row in P]
    tau, tid, topk = [], [], []
    for u in range(n):
        s = [sum((a * b for a, b in zip(Uf[u], Pf[i])), Fraction(0)) for i in range(m)]
        order = sorted(range(m), key=lambda i: (-s[i], i))
        topk.append(order[:k])
        tid.append(order[k - 1])
        tau.append(s[order[k - 1]])
    return tau, tid, topk


def rank_count(U, P, k):
    """Definition 1 by ranks: rank_u(i) = #{j : s_j > s_i or (s_j = s_i and j < i)};
    i is in S_k(u) iff rank_u(i) < k, and t_u has rank k-1."""
    Uf = [[Fraction(float(v)) for v in row] for row in U]
    Pf = [[Fraction(float(v)) for v in row] for row in P]
    m = len(P)
    members, tids = [], []
    for urow in Uf:
        s = [sum((a * b for a, b in zip(urow, prow)), Fraction(0)) for prow in Pf]
        rank = [sum(1 for j in range(m) if s[j] > s[i] or (s[j] == s[i] and j < i)) for i in range(m)]
        members.append({i for i in range(m) if rank[i] < k})
        tids.append(next(i for i in range(m) if rank[i] == k - 1))
    return members, tids


def check_pins(orc, cases) -> list[str]:
    """Run the oracle `orc` (module-like) through the pins; return failures."""
    fails = []
    for (U, P, k, N) in cases:
        n, m = len(U), len(P)
        tau, tid, topk = orc.kmips(U, P, k)
        btau, btid, btopk = brute_force(U, P, k)
        if [Fraction(float(t)) for t in tau] != btau:
            fails.append("tau vs brute force")
        if list(tid) != btid:
            fails.append("tid vs brute force")
        if [list(r) for r in topk] != btopk:
            fails.append("topk vs brute force")
        members, rtids = rank_count(U, P, k)
        if [set(r) for r in topk] != members or list(tid) != rtids:
            fails.append("rank-count formulation")
        sc = orc.scores_histogram(topk, m)
        if int(sc.sum()) != n * k:
            fails.append("sum(score) != n*k")
        sc2 = orc.scores_counting(U, P, tau, tid)
        if not np.array_equal(sc, sc2):
            fails.append("Section 2.2 baselines disagree")
        ids, tops = orc.topn(sc, N)
        border = sorted(range(m), key=lambda i: (-int(sc[i]), i))[:N]
        if list(ids) != border or list(tops) != [int(sc[i]) for i in border]:
            fails.append("top-N vs sorted")
    for name in golden_io.names():
        g = golden_io.load(name)
        tau, tid, topk = orc.kmips(g["U"], g["P"], g["k"])
        if not (np.array_equal(tau, g["tau"]) and np.array_equal(tid, g["tid"])
                and np.array_equal(topk, g["topk"])):
            fails.append(f"golden {name}: thresholds")
        sc = orc.scores_histogram(topk, g["m"])
        if not np.array_equal(sc, g["scores"]):
            fails.append(f"golden {name}: scores")
        ids, tops = orc.topn(sc, g["N"])
        if not (np.array_equal(ids, g["topn_ids"]) and np.array_equal(tops, g["topn_scores"])):
            fails.append(f"golden {name}: top-N")
        if not np.array_equal(orc.query_new_items(g["U"], tau, g["Q"]), g["counts"]):
            fails.append(f"golden {name}: new-item counts")
        if not np.array_equal(orc.uscore(g["U"], g["P"], tau), g["uscore"]):
            fails.append(f"golden {name}: uscore")
    return fails


def pin_cases():
    cases = []
    for seed, (n, m, d, k, N) in enumerate([(6, 7, 2, 3, 4), (9, 8, 3, 1, 8), (5, 6, 4, 6, 2),
                                             (8, 9, 3, 4, 5), (7, 10, 1, 5, 3)]):
        U, P = tiny_grid(n, m, d, seed, scale_rows=bool(seed % 2))
        cases.append((U, P, k, N))
    return cases


# ---------------------------------------------------------------- pins

def test_oracle_passes_all_pins():
    assert check_pins(oracle, pin_cases()) == []


@pytest.mark.parametrize("name", golden_io.names())
def test_golden_fixture(name):
    g = golden_io.load(name)
    tau, tid, topk = oracle.kmips(g["U"], g["P"], g["k"])
    np.testing.assert_array_equal(tau, g["tau"])
    np.testing.assert_array_equal(tid, g["tid"])
    np.testing.assert_array_equal(topk, g["topk"])
    sc = oracle.scores_histogram(topk, g["m"])
    np.testing.assert_array_equal(sc, g["scores"])
    assert int(sc.sum()) == g["n"] * g["k"]
    np.testing.assert_array_equal(oracle.uscore(g["U"], g["P"], tau), g["uscore"])
    np.testing.assert_array_equal(oracle.query_new_items(g["U"], tau, g["Q"]), g["counts"])


def test_sum_of_scores_and_baselines_agree_plain_workload():
    W = workloads.make("plain-2k")
    assert oracle.on_grid(W.U) and oracle.on_grid(W.P)
    tau, tid, topk = oracle.kmips(W.U, W.P, W.k)
    sc = oracle.scores_histogram(topk, W.m)
    assert int(sc.sum()) == W.n * W.k
    np.testing.assert_array_equal(sc, oracle.scores_counting(W.U, W.P, tau, tid))
    ids, tops = oracle.topn(sc, W.N)
    assert np.all(np.diff(tops) <= 0)
    # exactness: integer recomputation of a sample of thresholds
    Uq = np.rint(W.U.astype(np.float64) * 4096).astype(np.int64)
    Pq = np.rint(W.P.astype(np.float64) * 4096).astype(np.int64)
    for u in range(0, W.n, 97):
        assert tau[u] == float(Uq[u] @ Pq[tid[u]]) / 2**24


def test_mf_workload_exact_in_fp64():
    W = workloads.mf(300, 400, 64, 25, 10, seed=1)
    assert oracle.on_grid(W.U) and oracle.on_grid(W.P)
    e_u = workloads.row_exponents(W.U)
    e_p = workloads.row_exponents(W.P)
    Uq = np.rint(np.ldexp(W.U.astype(np.float64), 12 - e_u[:, None])).astype(np.int64)
    Pq = np.rint(np.ldexp(W.P.astype(np.float64), 12 - e_p[:, None])).astype(np.int64)
    S = oracle.inner_products(W.U, W.P)
    Sq = np.ldexp((Uq @ Pq.T).astype(np.float64), (e_u[:, None] + e_p[None, :] - 24))
    np.testing.assert_array_equal(S, Sq)


def test_closed_form_identical_items():
    rng = np.random.default_rng(3)
    U = (rng.integers(-8, 9, size=(20, 4)) / 16).astype(np.float32)
    P = np.tile(np.array([[0.25, -0.5, 0.125, 0.75]], np.float32), (12, 1))
    k, N = 5, 7
    tau, tid, topk = oracle.kmips(U, P, k)
    assert np.all(tid == k - 1)
    assert np.all(topk == np.arange(k))
    sc = oracle.scores_histogram(topk, 12)
    np.testing.assert_array_equal(sc, np.r_[np.full(k, 20), np.zeros(12 - k)])
    ids, _ = oracle.topn(sc, N)
    np.testing.assert_array_equal(ids, np.arange(N))


def test_closed_form_zero_user_and_k_equals_m():
    rng = np.random.default_rng(4)
    U = (rng.integers(-8, 9, size=(10, 3)) / 16).astype(np.float32)
    U[3] = 0
    P = (rng.integers(-8, 9, size=(9, 3)) / 16).astype(np.float32)
    tau, tid, topk = oracle.kmips(U, P, 4)
    assert tau[3] == 0.0 and np.signbit(tau[3]) == False  # noqa: E712
    np.testing.assert_array_equal(topk[3], np.arange(4))
    tau, tid, topk = oracle.kmips(U, P, 9)
    np.testing.assert_array_equal(oracle.scores_histogram(topk, 9), np.full(9, 10))


def test_k1_is_max():
    W = workloads.plain(n=64, m=50, d=8, k=1, N=3, seed=9)
    tau, tid, _ = oracle.kmips(W.U, W.P, 1)
    S = oracle.inner_products(W.U, W.P)
    np.testing.assert_array_equal(tau, S.max(axis=1))
    np.testing.assert_array_equal(tid, np.argmax(S, axis=1))  # argmax returns the first max


def test_negative_thresholds():
    rng = np.random.default_rng(5)
    P = (rng.integers(1, 8, size=(12, 3)) / 8).astype(np.float32)
    U = -(rng.integers(1, 8, size=(6, 3)) / 8).astype(np.float32)
    tau, tid, topk = oracle.kmips(U, P, 3)
    assert np.all(tau < 0)
    btau, btid, _ = brute_force(U, P, 3)
    assert [Fraction(float(t)) for t in tau] == btau and list(tid) == btid


def test_topn_ties_at_boundary():
    sc = np.array([5, 7, 5, 7, 1, 5])
    ids, tops = oracle.topn(sc, 4)
    np.testing.assert_array_equal(ids, [1, 3, 0, 2])
    np.testing.assert_array_equal(tops, [7, 7, 5, 5])


def test_theorem2_uscore_bounds_score():
    for seed in range(3):
        U, P = tiny_grid(12, 15, 3, 100 + seed, scale_rows=True)
        tau, tid, topk = oracle.kmips(U, P, 4)
        sc = oracle.scores_histogram(topk, 15)
        us = oracle.uscore(U, P, tau)
        assert np.all(us >= sc)
        # exactness claim: restricting the ranking to items whose uscore can reach
        # the N-th score leaves the top-N unchanged
        ids, tops = oracle.topn(sc, 5)
        keep = us >= tops[-1]
        sc_f = np.where(keep, sc, -1)
        ids_f, tops_f = oracle.topn(sc_f, 5)
        np.testing.assert_array_equal(ids, ids_f)


def test_query_candidate_equal_to_item():
    W = workloads.plain(n=200, m=60, d=6, k=5, N=3, seed=11)
    tau, tid, topk = oracle.kmips(W.U, W.P, W.k)
    sc = oracle.scores_histogram(topk, W.m)
    S = oracle.inner_products(W.U, W.P)
    for i in (0, 7, 59):
        c = oracle.query_new_items(W.U, tau, W.P[i:i + 1])[0]
        ties = int(np.sum((S[:, i] == tau) & (tid >= i)))
        assert c == sc[i] - ties


# ---------------------------------------------------------------- planted mistakes

def _mutant(**overrides):
    ns = types.SimpleNamespace(**{k: getattr(oracle, k) for k in oracle.__all__}) \
        if hasattr(oracle, "__all__") else types.SimpleNamespace(
            kmips=oracle.kmips, scores_histogram=oracle.scores_histogram,
            scores_counting=oracle.scores_counting, topn=oracle.topn,
            uscore=oracle.uscore, query_new_items=oracle.query_new_items)
    for k, v in overrides.items():
        setattr(ns, k, v)
    return ns


def _kmips_variant(order_fn, pick=lambda k: k - 1):
    def kmips(U, P, k):
        S = np.asarray(U, np.float64) @ np.asarray(P, np.float64).T
        order = order_fn(S)[:, :k]
        tid = order[:, pick(k)]
        return S[np.arange(len(S)), tid] + 0.0, tid, order
    return kmips


MUTANTS = {
    "ties by larger id": dict(kmips=_kmips_variant(
        lambda S: S.shape[1] - 1 - np.argsort(-S[:, ::-1], axis=1, kind="stable"))),
    "ascending order (sign flip)": dict(kmips=_kmips_variant(
        lambda S: np.argsort(S, axis=1, kind="stable"))),
    "unstable sort": dict(kmips=_kmips_variant(
        lambda S: np.argsort(-S + 0.0, axis=1, kind="heapsort"))),
    "k-th off by one": dict(kmips=_kmips_variant(
        lambda S: np.argsort(-S, axis=1, kind="stable"), pick=lambda k: max(0, k - 2))),
    "dropped last dimension": dict(kmips=lambda U, P, k: oracle.kmips(
        np.asarray(U)[:, :-1], np.asarray(P)[:, :-1], k)),
    "counting uses >= tau only": dict(scores_counting=lambda U, P, tau, tid: (
        (oracle.inner_products(U, P) >= tau[:, None]).sum(axis=0))),
    "top-N ties by larger id": dict(topn=lambda sc, N: (
        (len(sc) - 1 - np.argsort(-np.asarray(sc)[::-1], kind="stable"))[:N],
        np.asarray(sc)[(len(sc) - 1 - np.argsort(-np.asarray(sc)[::-1], kind="stable"))[:N]])),
    "query counts ties": dict(query_new_items=lambda U, tau, Q: (
        (oracle.inner_products(U, Q) >= tau[:, None]).sum(axis=0))),
    "uscore strict bound": dict(uscore=lambda U, P, tau: np.array([
        sum(1 for u in range(len(U)) if tau[u] < 0 or
            float(np.linalg.norm(U[u].astype(np.float64)) * np.linalg.norm(P[i].astype(np.float64))) > tau[u])
        for i in range(len(P))])),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_is_caught(name):
    fails = check_pins(_mutant(**MUTANTS[name]), pin_cases())
    assert fails, f"planted mistake '{name}' passed every pin"
