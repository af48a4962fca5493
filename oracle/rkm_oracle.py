"""Plain FP64 statement of the reverse k-MIPS top-N problem (oracle; test infrastructure only).

Notation follows the paper (Section 2.1, Table 2): U holds n user vectors,
P holds m item vectors, both d-dimensional; the item id of P[i] is i.

Tie rule.  Definitions 1 and 3 break ties "arbitrarily".  Here both are
fixed to the smaller item id: for user u, item i precedes item j iff
u.p_i > u.p_j, or u.p_i == u.p_j and i < j.  Under that order S_k(u) is the
first k items, t_u is the k-th one and tau_u = u.p_{t_u}, so that

    i in S_k(u)  <=>  u.p_i > tau_u  or  (u.p_i == tau_u and i <= t_u).

Exactness.  For inputs on the grid 2^e * q / 4096 (|q| <= 4096, one exponent
per row, d <= 128) every inner product is an integer multiple of a power of
two below 2^31 units, so FP64 computes it exactly in any summation order and
the outputs below are exact.  ``on_grid`` checks that condition.

Signed zero.  A sum of products can be -0.0; tau_u is returned as
``tau_u + 0.0`` so that a zero threshold is always +0.0.
"""
from __future__ import annotations

import os
from concurrent.futures import ThreadPoolExecutor
from fractions import Fraction

import numpy as np


def on_grid(X: np.ndarray, bits: int = 12, qmax: int = 4096) -> bool:
    """True iff every row is 2^(e - bits) * q with integer |q| <= qmax, e chosen per row
    as the smallest integer with max|x| <= 2^e."""
    X = np.asarray(X, dtype=np.float64)
    if X.size == 0:
        return True
    mx = np.max(np.abs(X), axis=1)
    f, e = np.frexp(mx)
    e = np.where(f == 0.5, e - 1, e)
    e = np.where(mx == 0.0, 0, e)
    q = np.ldexp(X, bits - e[:, None])
    return bool(np.all(q == np.rint(q)) and np.all(np.abs(q) <= qmax))


def inner_products(U: np.ndarray, P: np.ndarray) -> np.ndarray:
    """All u.p in FP64 (Definition 1's relevance measure), shape [n, m]."""
    return np.asarray(U, dtype=np.float64) @ np.asarray(P, dtype=np.float64).T


def _kmips_block(U64: np.ndarray, P64: np.ndarray, k: int):
    S = U64 @ P64.T
    # A stable ascending sort of -s keeps equal scores in increasing id order,
    # which is the order "s descending, then id ascending" of Definition 1.
    order = np.argsort(-S, axis=1, kind="stable")[:, :k]
    rows = np.arange(S.shape[0])
    tid = order[:, k - 1]
    tau = S[rows, tid] + 0.0
    return tau, tid.astype(np.int64), order.astype(np.int64)


def kmips(U: np.ndarray, P: np.ndarray, k: int, block: int = 256, threads: int = 1):
    """Definition 1 for every user: returns (tau [n] f64, tid [n] i64, topk [n, k] i64).

    topk[u] lists S_k(u) in the order above; tid = topk[:, k-1]; tau = u.p_tid.
    """
    U64 = np.asarray(U, dtype=np.float64)
    P64 = np.asarray(P, dtype=np.float64)
    n, m = U64.shape[0], P64.shape[0]
    if not 1 <= k <= m:
        raise ValueError("Definition 1 needs 1 <= k <= m")
    tau = np.empty(n, dtype=np.float64)
    tid = np.empty(n, dtype=np.int64)
    topk = np.empty((n, k), dtype=np.int64)

    def work(u0):
        u1 = min(n, u0 + block)
        tau[u0:u1], tid[u0:u1], topk[u0:u1] = _kmips_block(U64[u0:u1], P64, k)

    starts = range(0, n, block)
    if threads > 1:
        with ThreadPoolExecutor(threads) as ex:
            list(ex.map(work, starts))
    else:
        for u0 in starts:
            work(u0)
    return tau, tid, topk


def scores_histogram(topk: np.ndarray, m: int) -> np.ndarray:
    """First baseline of Section 2.2: score(p) += 1 for every p in S_k(u), over all u."""
    return np.bincount(np.asarray(topk).ravel(), minlength=m).astype(np.int64)


def scores_counting(U: np.ndarray, P: np.ndarray, tau: np.ndarray, tid: np.ndarray,
                    block: int = 256) -> np.ndarray:
    """Second baseline of Section 2.2 via Eq. 1: score(p_i) = |T_k(p_i)| counted per item,
    with membership decided against (tau_u, t_u) under the tie rule."""
    U64 = np.asarray(U, dtype=np.float64)
    P64 = np.asarray(P, dtype=np.float64)
    m = P64.shape[0]
    ids = np.arange(m)
    out = np.zeros(m, dtype=np.int64)
    for u0 in range(0, U64.shape[0], block):
        u1 = min(U64.shape[0], u0 + block)
        S = U64[u0:u1] @ P64.T
        t = tau[u0:u1, None]
        member = (S > t) | ((S == t) & (ids[None, :] <= tid[u0:u1, None]))
        out += member.sum(axis=0)
    return out


def topn(scores: np.ndarray, N: int) -> tuple[np.ndarray, np.ndarray]:
    """Definition 3: the N items with the largest score, ties by smaller id.
    Returns (ids [N], scores [N]) in that order."""
    scores = np.asarray(scores)
    if not 1 <= N <= scores.shape[0]:
        raise ValueError("Definition 3 needs 1 <= N <= m")
    order = np.argsort(-scores, kind="stable")[:N]
    return order.astype(np.int64), scores[order].astype(np.int64)


def reverse_kmips_topn(U: np.ndarray, P: np.ndarray, k: int, N: int, threads: int = 1):
    """The whole problem of Definition 3: (tau, tid, scores, top ids, top scores)."""
    tau, tid, topk = kmips(U, P, k, threads=threads)
    sc = scores_histogram(topk, P.shape[0])
    ids, tops = topn(sc, N)
    return tau, tid, sc, ids, tops


def _exact_sq_norm(x: np.ndarray) -> Fraction:
    return sum((Fraction(float(v)) ** 2 for v in x), Fraction(0))


def uscore(U: np.ndarray, P: np.ndarray, tau: np.ndarray) -> np.ndarray:
    """Eq. 2 (Section 4.1) with the exact thresholds A_i^k = tau_u:
    uscore(p) = #{u : ||u|| ||p|| >= tau_u}, evaluated in exact rational arithmetic
    (as ||u||^2 ||p||^2 >= tau_u^2 when tau_u > 0; always true when tau_u <= 0).
    Pure Python: for small inputs only."""
    un2 = [_exact_sq_norm(u) for u in np.asarray(U)]
    pn2 = [_exact_sq_norm(p) for p in np.asarray(P)]
    out = np.zeros(len(pn2), dtype=np.int64)
    for u, t in enumerate(np.asarray(tau, dtype=np.float64)):
        tf = Fraction(float(t))
        for i, p2 in enumerate(pn2):
            if tf <= 0 or un2[u] * p2 >= tf * tf:
                out[i] += 1
    return out


def query_new_items(U: np.ndarray, tau: np.ndarray, Q: np.ndarray, block: int = 4096) -> np.ndarray:
    """Definition 2 for new candidate items: count(q) = #{u : u.q > tau_u}.  A new item
    takes an id larger than every catalogue id, so a tie at tau_u does not enter S_k(u);
    the catalogue and tau are left unchanged (each candidate is scored on its own)."""
    U64 = np.asarray(U, dtype=np.float64)
    Q64 = np.asarray(Q, dtype=np.float64)
    out = np.zeros(Q64.shape[0], dtype=np.int64)
    for u0 in range(0, U64.shape[0], block):
        u1 = min(U64.shape[0], u0 + block)
        S = U64[u0:u1] @ Q64.T
        out += (S > tau[u0:u1, None]).sum(axis=0)
    return out


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)
