"""The serving loop: each request's counts are the same alone and in the mix.

Users and their oracle thresholds are made resident once.  A stream of what-if requests of
log-uniform sizes is scored three ways, and the integer counts must be identical:
  * by the oracle (Definition 2 for a new item, ties at tau_u lose);
  * alone, one rkm_query_new_items call per request;
  * in the mix: submitted to the serving loop from several host threads with Poisson gaps,
    so that requests are batched together, admitted by arena memory (the arena is sized to
    hold about two batches) and run on several slots at once.
"""
import threading
import time

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


def batch_bytes(items, d):
    """Arena bytes of a batch: FP32 rows and int32 counts, each rounded up to 256 bytes."""
    r = lambda b: (b + 255) // 256 * 256
    return r(items * d * 4) + r(items * 4)


@pytest.fixture(scope="module")
def resident():
    W = workloads.mf(20_000, 4_000, 100, 20, 1, seed=3)
    tau, tid, _ = oracle.kmips(W.U, W.P, W.k)
    arrivals, sizes, offsets = workloads.serving_stream(48, 2000.0, seed=4, max_q=2048)
    Qall = workloads.queries(int(sizes.sum()), W.d, seed=4)
    reqs = [np.ascontiguousarray(Qall[o:o + q]) for o, q in zip(offsets, sizes)]
    expect = [oracle.query_new_items(W.U, tau, Q) for Q in reqs]
    return W, tau, tid, arrivals, reqs, expect


@pytest.mark.parametrize("prec", ["bf16", "fp32", "fp8"])
def test_each_request_same_alone_and_in_the_mix(rkm, resident, prec):
    W, tau, tid, arrivals, reqs, expect = resident
    with rkm.Context(prec) as ctx:
        ctx.resident_set(torch.from_numpy(W.U).cuda(), torch.from_numpy(tau).cuda(),
                         torch.from_numpy(tid.astype(np.int32)).cuda())
        for Q, e in zip(reqs, expect):  # alone
            got = ctx.query_new_items(torch.from_numpy(Q).cuda()).cpu().numpy()
            np.testing.assert_array_equal(got, e)
        budget = 2 * batch_bytes(2048, W.d) + 4096
        with rkm.Server(ctx, slots=3, max_batch_items=2048, memory_bytes=budget) as srv:
            tickets = [None] * len(reqs)
            t0 = time.perf_counter()

            def producer(idx):
                for j in idx:
                    delay = arrivals[j] - (time.perf_counter() - t0)
                    if delay > 0:
                        time.sleep(delay)
                    tickets[j] = srv.submit(reqs[j])

            threads = [threading.Thread(target=producer, args=(range(r, len(reqs), 2),)) for r in range(2)]
            for t in threads:
                t.start()
            for t in threads:
                t.join()
            lat = []
            for j in range(len(reqs)):
                counts, ms = srv.wait(tickets[j])
                np.testing.assert_array_equal(counts, expect[j], err_msg=f"request {j} differs in the mix")
                lat.append(ms)
            st = srv.stats()
        assert st["completed"] == len(reqs) and st["failed"] == 0
        assert st["items"] == sum(Q.shape[0] for Q in reqs)
        assert st["batches"] <= len(reqs)
        assert st["arena_peak_bytes"] <= budget
        assert 0 < st["p50_ms"] <= st["p99_ms"] <= st["max_ms"]
        assert st["kernel_launches"] > 0


def test_all_at_once_is_batched_and_overlapped(rkm, resident):
    """Every request queued before the first is admitted: later batches hold many requests,
    and more than one batch is in flight at once."""
    W, tau, tid, _, reqs, expect = resident
    with rkm.Context("bf16") as ctx:
        ctx.resident_set(torch.from_numpy(W.U).cuda(), torch.from_numpy(tau).cuda(),
                         torch.from_numpy(tid.astype(np.int32)).cuda())
        with rkm.Server(ctx, slots=2, max_batch_items=4096, memory_bytes=64 << 20) as srv:
            tickets = [srv.submit(Q) for Q in reqs]
            srv.drain()
            for t, e in zip(tickets, expect):
                np.testing.assert_array_equal(srv.wait(t)[0], e)
            st = srv.stats()
    assert st["batches"] < len(reqs) // 2
    assert st["max_in_flight"] == 2


def test_serving_rejections(rkm, resident):
    W, tau, tid, _, reqs, _ = resident
    with rkm.Context("bf16") as ctx:
        with pytest.raises(rkm.RkmError, match="before rkm_resident_set"):
            rkm.Server(ctx)
        ctx.resident_set(torch.from_numpy(W.U).cuda(), torch.from_numpy(tau).cuda(),
                         torch.from_numpy(tid.astype(np.int32)).cuda())
        with rkm.Server(ctx, slots=1, max_batch_items=1024, memory_bytes=1 << 20) as srv:
            big = np.zeros((1025, W.d), dtype=np.float32)
            with pytest.raises(rkm.RkmError, match="max_batch_items"):
                srv.submit(big)
            # the resident set is borrowed while the server exists
            with pytest.raises(rkm.RkmError, match="serving loop"):
                ctx.resident_set(torch.from_numpy(W.U).cuda(), torch.from_numpy(tau).cuda(),
                                 torch.from_numpy(tid.astype(np.int32)).cuda())
            counts, _ = srv.wait(srv.submit(reqs[0]))
            assert counts.shape == (reqs[0].shape[0],)
        with rkm.Server(ctx, slots=1, max_batch_items=4096, memory_bytes=300_000) as srv:
            with pytest.raises(rkm.RkmError, match="arena"):
                srv.submit(np.zeros((4000, W.d), dtype=np.float32))


def test_state_save_and_load_round_trip(rkm, resident, tmp_path):
    """A saved serving state restores the resident set in a fresh context (no threshold
    pass): every request's counts equal the oracle's; a corrupted file is refused with
    RKM_EIO and leaves the loaded state in place."""
    W, tau, tid, arrivals, reqs, expect = resident
    path = str(tmp_path / "resident.rkmstate")
    with rkm.Context("bf16") as ctx:
        with pytest.raises(rkm.RkmError):
            ctx.state_save(path)  # no resident set yet
        ctx.resident_set(torch.from_numpy(W.U).cuda(), torch.from_numpy(tau).cuda(),
                         torch.from_numpy(tid.astype(np.int32)).cuda())
        ctx.state_save(path)
    with rkm.Context("bf16") as fresh:
        fresh.state_load(path)
        for Q, e in zip(reqs[:12], expect[:12]):
            np.testing.assert_array_equal(fresh.query_new_items(torch.from_numpy(Q).cuda()).cpu().numpy(), e)
        blob = bytearray(open(path, "rb").read())
        blob[100] ^= 1
        bad = str(tmp_path / "corrupt.rkmstate")
        open(bad, "wb").write(bytes(blob))
        with pytest.raises(rkm.RkmError) as err:
            fresh.state_load(bad)
        assert err.value.status == 9  # RKM_EIO
        Q, e = reqs[0], expect[0]
        np.testing.assert_array_equal(fresh.query_new_items(torch.from_numpy(Q).cuda()).cpu().numpy(), e)
