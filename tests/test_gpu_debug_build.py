"""The RKM_DEBUG build of the library (device index checks on the gathers whose index comes from
device data) gives the oracle's results and trips no check, on every precision path, in a
process of its own (RKM_LIBRARY selects the debug library)."""
import os
import subprocess
import sys

import pytest

pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import sys
sys.path.insert(0, ROOT)
import numpy as np, torch
import oracle, workloads
import paper_2504_13445_gb300 as rkm
assert rkm.LIB_PATH.endswith("librkm_debug.so")
W = workloads.mf(12_000, 9_000, 64, 10, 20, seed=13)
tau_o, tid_o, topk_o = oracle.kmips(W.U, W.P, W.k)
ids_o, tops_o = oracle.topn(oracle.scores_histogram(topk_o, W.m), W.N)
Q = workloads.queries(300, W.d, seed=13)
cnt_o = oracle.query_new_items(W.U, tau_o, Q)
U, P = torch.from_numpy(W.U).cuda(), torch.from_numpy(W.P).cuda()
for prec in ("bf16", "fp8", "fp32"):
    with rkm.Context(prec) as ctx:
        ids, tops, tau, tid = ctx.topn(U, P, W.k, W.N, return_thresholds=True)
        assert np.array_equal(tau.cpu().numpy().view(np.uint64), tau_o.view(np.uint64)), prec
        assert np.array_equal(tid.cpu().numpy(), tid_o), prec
        assert np.array_equal(ids.cpu().numpy(), ids_o) and np.array_equal(tops.cpu().numpy(), tops_o), prec
        ctx.resident_set(U, tau, tid)
        cnt = ctx.query_new_items(torch.from_numpy(Q).cuda())
        assert np.array_equal(cnt.cpu().numpy(), cnt_o), prec
print("debug build ok")
"""


def test_debug_library_matches_oracle():
    from paper_2504_13445_gb300 import build as b
    lib = b.build(debug=True)
    env = dict(os.environ, RKM_LIBRARY=lib)
    r = subprocess.run([sys.executable, "-c", f"ROOT = {ROOT!r}\n" + CHILD], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0 and "debug build ok" in r.stdout, r.stdout[-2000:] + r.stderr[-4000:]
