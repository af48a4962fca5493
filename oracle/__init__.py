"""FP64 CPU oracle for reverse k-MIPS top-N (test infrastructure only).

This package is the checker, not the product: only the tests, the smoke check
and the CPU-baseline leg of the benchmark import it.  The CUDA library never
calls it and shares no code with it.

Every function restates a definition of "How to Mine Potentially Popular
Items? A Reverse MIPS-based Approach" (Amagata et al., arXiv 2504.13445) in
plain numpy FP64, with the tie rule fixed to "smaller item id first":

* ``kmips``              -- Definition 1 (k-MIPS), per user, ties by smaller id.
* ``scores_histogram``   -- Section 2.2, first baseline (increment per S_k(u)).
* ``scores_counting``    -- Definition 2 / Eq. 1 and the second baseline of
                            Section 2.2 (per-item reverse k-MIPS size).
* ``topn``               -- Definition 3, ties by smaller id.
* ``uscore``             -- Section 4.1, Eq. 2 (Cauchy-Schwarz) upper-bound count.
* ``query_new_items``    -- Definition 2 applied to a new item whose id is larger
                            than every catalogue id, so ties at tau_u lose.

Pins (tests/test_oracle.py): brute force in exact rational arithmetic on tiny
inputs, the rank-count formulation, sum(score) = n*k, the two Section-2.2
baselines agreeing, Theorem 2 (uscore >= score), closed-form tie cases and
hand-derived golden fixtures under tests/golden/.  No function here is
"parity unpinned".
"""
from .rkm_oracle import (  # noqa: F401
    inner_products, kmips, scores_histogram, scores_counting, topn, uscore,
    query_new_items, reverse_kmips_topn, on_grid,
)
