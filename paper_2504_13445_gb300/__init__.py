"""GB300 reverse k-MIPS top-N (arXiv 2504.13445): thin Python binding of librkm.so.

Every function here marshals arguments into the C ABI declared in include/rkm.h and
calls it; all computation runs in the library's CUDA kernels.  PyTorch supplies
device memory and the current CUDA stream only.  There is no fallback: if the
library is missing the import of a binding function raises.

Low-level names match the C ABI (``rkm_thresholds`` ...); ``Context`` wraps them.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
# RKM_LIBRARY selects another build of the library (e.g. lib/librkm_debug.so).
LIB_PATH = os.environ.get("RKM_LIBRARY") or os.path.join(HERE, "lib", "librkm.so")

RKM_FP32, RKM_BF16, RKM_FP8 = 0, 1, 2
PRECISIONS = {"fp32": RKM_FP32, "bf16": RKM_BF16, "fp8": RKM_FP8}
STATUS = {0: "RKM_OK", 1: "RKM_EINVAL", 2: "RKM_ENOMEM", 3: "RKM_ECUDA", 4: "RKM_EOVERFLOW",
          5: "RKM_ETIMEOUT", 6: "RKM_ESTATE", 7: "RKM_EINTERNAL", 8: "RKM_EBUSY", 9: "RKM_EIO"}

EXPORTED = ["rkm_default_opts", "rkm_create", "rkm_destroy", "rkm_last_error", "rkm_version",
            "rkm_thresholds", "rkm_scores", "rkm_topn", "rkm_topn_host", "rkm_item_bounds",
            "rkm_resident_set", "rkm_query_new_items", "rkm_get_stats", "rkm_topn_scores_noalloc",
            "rkm_topn_batch", "rkm_topn_from_topk", "rkm_debug_products", "rkm_debug_wait_timeout",
            "rkm_state_save", "rkm_state_load", "rkm_serve_default_opts", "rkm_serve_create", "rkm_serve_submit",
            "rkm_serve_wait", "rkm_serve_drain", "rkm_serve_get_stats", "rkm_serve_reset_stats",
            "rkm_serve_destroy"]


class RkmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("k_max", ctypes.c_int), ("cand_capacity", ctypes.c_int),
                ("band_capacity", ctypes.c_int64), ("filter", ctypes.c_int), ("profile", ctypes.c_int),
                ("autotune", ctypes.c_int), ("tune_cache", ctypes.c_char_p), ("scores_from_topk", ctypes.c_int),
                ("epilogue_groups", ctypes.c_int), ("seed_order", ctypes.c_int)]


class Instance(ctypes.Structure):
    _fields_ = [("U", ctypes.c_void_p), ("n", ctypes.c_int64), ("ldu", ctypes.c_int64),
                ("P", ctypes.c_void_p), ("m", ctypes.c_int64), ("ldp", ctypes.c_int64),
                ("d", ctypes.c_int), ("k", ctypes.c_int), ("N", ctypes.c_int),
                ("ids", ctypes.c_void_p), ("top_scores", ctypes.c_void_p)]


class Stats(ctypes.Structure):
    _fields_ = [("pairs_total", ctypes.c_uint64), ("pairs_evaluated", ctypes.c_uint64),
                ("candidates", ctypes.c_uint64), ("band_pairs", ctypes.c_uint64),
                ("items_counted", ctypes.c_uint64), ("retries", ctypes.c_int32),
                ("exact_integer_path", ctypes.c_int32), ("last_ms", ctypes.c_double),
                ("kernel_launches", ctypes.c_uint64), ("threshold_launches", ctypes.c_uint64),
                ("phase_ms", ctypes.c_double * 8), ("threshold_pairs", ctypes.c_uint64)]

    PHASES = ("prep", "threshold", "exact", "bounds", "count", "band", "topn", "transfer")

    def as_dict(self) -> dict:
        out = {f: getattr(self, f) for f, _ in self._fields_ if f != "phase_ms"}
        out["phase_ms"] = {name: self.phase_ms[i] for i, name in enumerate(self.PHASES)}
        return out


class ServeOpts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int), ("max_batch_items", ctypes.c_int64), ("memory_bytes", ctypes.c_int64),
                ("max_pending", ctypes.c_int64)]


class ServeStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                ("items", ctypes.c_uint64), ("batches", ctypes.c_uint64), ("mean_batch_items", ctypes.c_double),
                ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double), ("mean_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("mean_queue_ms", ctypes.c_double), ("window_ms", ctypes.c_double),
                ("items_per_s", ctypes.c_double), ("pairs_per_s", ctypes.c_double),
                ("arena_peak_bytes", ctypes.c_int64), ("max_in_flight", ctypes.c_int32),
                ("slots", ctypes.c_int32), ("kernel_launches", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {f: getattr(self, f) for f, _ in self._fields_}


_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load librkm.so (built by build.py); raises if it is missing."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"librkm.so not found at {path}; run __graft_entry__.build() first")
    lib = ctypes.CDLL(path)
    P, I64, I, V = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, None
    sig = {
        "rkm_default_opts": (V, [ctypes.POINTER(Opts)]),
        "rkm_create": (I, [ctypes.POINTER(P), ctypes.POINTER(Opts), I]),
        "rkm_destroy": (V, [P]),
        "rkm_last_error": (ctypes.c_char_p, []),
        "rkm_version": (ctypes.c_char_p, []),
        "rkm_thresholds": (I, [P, P, I64, I64, P, I64, I64, I, I, P, P, P, P]),
        "rkm_scores": (I, [P, P, I64, I64, P, I64, I64, I, P, P, P, P]),
        "rkm_topn": (I, [P, P, I64, I64, P, I64, I64, I, I, I, P, P, P, P, P]),
        "rkm_topn_host": (I, [P, P, I64, I64, P, I64, I64, I, I, I, P, P, P]),
        "rkm_item_bounds": (I, [P, P, I64, I64, P, I64, I64, I, P, P, P]),
        "rkm_resident_set": (I, [P, P, I64, I64, I, P, P, P]),
        "rkm_query_new_items": (I, [P, P, I64, I64, P, P]),
        "rkm_get_stats": (I, [P, ctypes.POINTER(Stats)]),
        "rkm_topn_scores_noalloc": (I, [P, I64, I, P, P, P]),
        "rkm_topn_batch": (I, [P, ctypes.POINTER(Instance), I, P]),
        "rkm_topn_from_topk": (I, [P, P, I64, I, I, I64, I, P, P, P]),
        "rkm_debug_products": (I, [P, P, I64, I64, P, I64, I64, I, P, P, I64, P]),
        "rkm_debug_wait_timeout": (I, [P, I64, P]),
        "rkm_state_save": (I, [P, ctypes.c_char_p]),
        "rkm_state_load": (I, [P, ctypes.c_char_p, P]),
        "rkm_serve_default_opts": (V, [ctypes.POINTER(ServeOpts)]),
        "rkm_serve_create": (I, [ctypes.POINTER(P), P, ctypes.POINTER(ServeOpts)]),
        "rkm_serve_submit": (I, [P, P, I64, I64, P, ctypes.POINTER(ctypes.c_uint64)]),
        "rkm_serve_wait": (I, [P, ctypes.c_uint64, ctypes.c_double, ctypes.POINTER(ctypes.c_double)]),
        "rkm_serve_drain": (I, [P]),
        "rkm_serve_get_stats": (I, [P, ctypes.POINTER(ServeStats)]),
        "rkm_serve_reset_stats": (I, [P]),
        "rkm_serve_destroy": (V, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _check(status: int) -> None:
    if status != 0:
        raise RkmError(status, load_library().rkm_last_error().decode())


def _stream():
    import torch
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr() if t is not None else 0)


def _mat(X):
    """A row-major float32 CUDA matrix with unit column stride: (tensor, rows, ld)."""
    import torch
    if not (isinstance(X, torch.Tensor) and X.is_cuda and X.dtype == torch.float32 and X.dim() == 2):
        raise TypeError("expected a 2-D float32 CUDA tensor")
    if X.stride(1) != 1:
        X = X.contiguous()
    return X, X.shape[0], X.stride(0) if X.shape[0] > 0 else X.shape[1]


# ---------------------------------------------------------------- C-ABI names

def rkm_create(precision: str = "bf16", device: int = 0, k_max: int = 64, cand_capacity: int = 0,
               band_capacity: int = 0, filter: bool = True, profile: bool = False, autotune: bool = False,
               tune_cache: str | None = None, scores_from_topk: bool = False,
               epilogue_groups: int = 0, seed_order: bool = True) -> ctypes.c_void_p:
    lib = load_library()
    o = Opts()
    lib.rkm_default_opts(ctypes.byref(o))
    o.precision = PRECISIONS[precision]
    o.k_max = k_max
    o.cand_capacity = cand_capacity
    o.band_capacity = band_capacity
    o.filter = 1 if filter else 0
    o.profile = 1 if profile else 0
    o.autotune = 1 if autotune else 0
    o.tune_cache = tune_cache.encode() if tune_cache else None
    o.scores_from_topk = 1 if scores_from_topk else 0
    o.epilogue_groups = epilogue_groups
    o.seed_order = 1 if seed_order else 0
    h = ctypes.c_void_p()
    _check(lib.rkm_create(ctypes.byref(h), ctypes.byref(o), device))
    return h


def rkm_destroy(ctx) -> None:
    load_library().rkm_destroy(ctx)


def rkm_thresholds(ctx, U, P, k: int, want_topk: bool = False):
    import torch
    U, n, ldu = _mat(U)
    P, m, ldp = _mat(P)
    d = U.shape[1]
    tau = torch.empty(n, dtype=torch.float64, device=U.device)
    tid = torch.empty(n, dtype=torch.int32, device=U.device)
    topk = torch.empty((n, k), dtype=torch.int32, device=U.device) if want_topk else None
    _check(load_library().rkm_thresholds(ctx, _ptr(U), n, ldu, _ptr(P), m, ldp, d, k, _ptr(tau), _ptr(tid),
                                         _ptr(topk), _stream()))
    return tau, tid, topk


def rkm_scores(ctx, U, P, tau, tid):
    import torch
    U, n, ldu = _mat(U)
    P, m, ldp = _mat(P)
    scores = torch.empty(m, dtype=torch.int32, device=U.device)
    _check(load_library().rkm_scores(ctx, _ptr(U), n, ldu, _ptr(P), m, ldp, U.shape[1],
                                     _ptr(tau.contiguous()), _ptr(tid.contiguous()), _ptr(scores), _stream()))
    return scores


def rkm_topn(ctx, U, P, k: int, N: int, return_thresholds: bool = False):
    import torch
    U, n, ldu = _mat(U)
    P, m, ldp = _mat(P)
    ids = torch.empty(N, dtype=torch.int32, device=U.device)
    sc = torch.empty(N, dtype=torch.int32, device=U.device)
    tau = torch.empty(n, dtype=torch.float64, device=U.device) if return_thresholds else None
    tid = torch.empty(n, dtype=torch.int32, device=U.device) if return_thresholds else None
    _check(load_library().rkm_topn(ctx, _ptr(U), n, ldu, _ptr(P), m, ldp, U.shape[1], k, N, _ptr(ids), _ptr(sc),
                                   _ptr(tau), _ptr(tid), _stream()))
    return (ids, sc, tau, tid) if return_thresholds else (ids, sc)


def rkm_topn_host(ctx, U, P, k: int, N: int):
    """Host numpy float32 inputs and outputs; the copies happen inside the library call."""
    import numpy as np
    U = np.ascontiguousarray(U, dtype=np.float32)
    P = np.ascontiguousarray(P, dtype=np.float32)
    ids = np.empty(N, dtype=np.int32)
    sc = np.empty(N, dtype=np.int32)
    _check(load_library().rkm_topn_host(ctx, U.ctypes.data_as(ctypes.c_void_p), U.shape[0], U.shape[1],
                                        P.ctypes.data_as(ctypes.c_void_p), P.shape[0], P.shape[1], U.shape[1],
                                        k, N, ids.ctypes.data_as(ctypes.c_void_p),
                                        sc.ctypes.data_as(ctypes.c_void_p), _stream()))
    return ids, sc


def rkm_item_bounds(ctx, U, P, tau):
    import torch
    U, n, ldu = _mat(U)
    P, m, ldp = _mat(P)
    us = torch.empty(m, dtype=torch.int32, device=U.device)
    _check(load_library().rkm_item_bounds(ctx, _ptr(U), n, ldu, _ptr(P), m, ldp, U.shape[1],
                                          _ptr(tau.contiguous()), _ptr(us), _stream()))
    return us


def rkm_resident_set(ctx, U, tau, tid) -> None:
    U, n, ldu = _mat(U)
    _check(load_library().rkm_resident_set(ctx, _ptr(U), n, ldu, U.shape[1], _ptr(tau.contiguous()),
                                           _ptr(tid.contiguous()), _stream()))


def rkm_query_new_items(ctx, Q):
    import torch
    Q, q, ldq = _mat(Q)
    counts = torch.empty(q, dtype=torch.int32, device=Q.device)
    _check(load_library().rkm_query_new_items(ctx, _ptr(Q), q, ldq, _ptr(counts), _stream()))
    return counts


def rkm_state_save(ctx, path: str) -> None:
    _check(load_library().rkm_state_save(ctx, os.fsencode(path)))


def rkm_state_load(ctx, path: str) -> None:
    _check(load_library().rkm_state_load(ctx, os.fsencode(path), _stream()))


def rkm_get_stats(ctx) -> dict:
    s = Stats()
    _check(load_library().rkm_get_stats(ctx, ctypes.byref(s)))
    return s.as_dict()


def rkm_topn_batch(ctx, problems, outs=None):
    """problems: list of (U, P, k, N) with float32 CUDA matrices.  Returns [(ids, scores)].
    Pass the previous result as `outs` to reuse the output buffers (a batch with the same
    inputs and outputs replays the library's captured graph)."""
    import torch
    arr = (Instance * len(problems))()
    new_outs, keep = [], []
    for j, (U, P, k, N) in enumerate(problems):
        U, n, ldu = _mat(U)
        P, m, ldp = _mat(P)
        if outs is not None:
            ids, sc = outs[j]
        else:
            ids = torch.empty(N, dtype=torch.int32, device=U.device)
            sc = torch.empty(N, dtype=torch.int32, device=U.device)
        keep += [U, P]
        new_outs.append((ids, sc))
        arr[j] = Instance(U.data_ptr(), n, ldu, P.data_ptr(), m, ldp, U.shape[1], k, N, ids.data_ptr(),
                          sc.data_ptr())
    _check(load_library().rkm_topn_batch(ctx, arr, len(problems), _stream()))
    return new_outs


def rkm_topn_from_topk(ctx, lists, m: int, k: int, N: int):
    """Top N for k <= kmax from the S_kmax(u) lists of rkm_thresholds (device int32 [n, kmax])."""
    import torch
    lists = lists.contiguous()
    n, kmax = lists.shape
    ids = torch.empty(N, dtype=torch.int32, device=lists.device)
    sc = torch.empty(N, dtype=torch.int32, device=lists.device)
    _check(load_library().rkm_topn_from_topk(ctx, _ptr(lists), n, kmax, k, m, N, _ptr(ids), _ptr(sc), _stream()))
    return ids, sc


def rkm_debug_products(ctx, U, P):
    """Approximate products of the context's tensor-core path and their error bounds:
    returns (v [n, m] float32, E [n, m] float32) with |v - u.p| <= E required for every pair."""
    import torch
    U, n, ldu = _mat(U)
    P, m, ldp = _mat(P)
    v = torch.empty((n, m), dtype=torch.float32, device=U.device)
    E = torch.empty((n, m), dtype=torch.float32, device=U.device)
    _check(load_library().rkm_debug_products(ctx, _ptr(U), n, ldu, _ptr(P), m, ldp, U.shape[1], _ptr(v), _ptr(E),
                                             m, _stream()))
    return v, E


def rkm_debug_wait_timeout(ctx, wait_cycles: int) -> None:
    """Run the kernels' bounded wait on a barrier nothing completes; raises RkmError
    (RKM_ETIMEOUT) when the wait gives up as it must."""
    _check(load_library().rkm_debug_wait_timeout(ctx, wait_cycles, _stream()))


def rkm_topn_scores_noalloc(scores, N: int):
    """Top N of a device int32 score array through the entry point that allocates no device
    memory (for callers that cannot call cudaMalloc); the output tensors are allocated here,
    by the caller's side, as the C ABI expects."""
    import torch
    scores = scores.contiguous()
    ids = torch.empty(N, dtype=torch.int32, device=scores.device)
    top = torch.empty(N, dtype=torch.int32, device=scores.device)
    _check(load_library().rkm_topn_scores_noalloc(_ptr(scores), scores.numel(), N, _ptr(ids), _ptr(top),
                                                  _stream()))
    return ids, top


def rkm_serve_default_opts() -> ServeOpts:
    o = ServeOpts()
    load_library().rkm_serve_default_opts(ctypes.byref(o))
    return o


def rkm_serve_create(ctx, slots: int | None = None, max_batch_items: int | None = None,
                     memory_bytes: int | None = None, max_pending: int | None = None) -> ctypes.c_void_p:
    o = rkm_serve_default_opts()
    for name, v in (("slots", slots), ("max_batch_items", max_batch_items), ("memory_bytes", memory_bytes),
                    ("max_pending", max_pending)):
        if v is not None:
            setattr(o, name, v)
    h = ctypes.c_void_p()
    _check(load_library().rkm_serve_create(ctypes.byref(h), ctx, ctypes.byref(o)))
    return h


def rkm_serve_submit(srv, Q, counts) -> int:
    """Q: host float32 [q, d] (numpy, unit column stride); counts: host int32 [q].  Both must
    stay alive until rkm_serve_wait returns for the ticket."""
    import numpy as np
    if not (isinstance(Q, np.ndarray) and Q.dtype == np.float32 and Q.ndim == 2 and Q.strides[1] == 4):
        raise TypeError("Q must be a 2-D float32 numpy array with unit column stride")
    if not (isinstance(counts, np.ndarray) and counts.dtype == np.int32 and counts.flags.c_contiguous
            and counts.size >= Q.shape[0]):
        raise TypeError("counts must be a contiguous int32 numpy array of q entries")
    t = ctypes.c_uint64()
    _check(load_library().rkm_serve_submit(srv, Q.ctypes.data, Q.shape[0], Q.strides[0] // 4,
                                           counts.ctypes.data, ctypes.byref(t)))
    return t.value


def rkm_serve_wait(srv, ticket: int, timeout_ms: float = -1.0) -> float:
    """Returns the request's latency in ms; raises RkmError with the request's status."""
    lat = ctypes.c_double()
    _check(load_library().rkm_serve_wait(srv, ticket, timeout_ms, ctypes.byref(lat)))
    return lat.value


def rkm_serve_drain(srv) -> None:
    _check(load_library().rkm_serve_drain(srv))


def rkm_serve_get_stats(srv) -> dict:
    s = ServeStats()
    _check(load_library().rkm_serve_get_stats(srv, ctypes.byref(s)))
    return s.as_dict()


def rkm_serve_reset_stats(srv) -> None:
    _check(load_library().rkm_serve_reset_stats(srv))


def rkm_serve_destroy(srv) -> None:
    load_library().rkm_serve_destroy(srv)


def rkm_version() -> str:
    return load_library().rkm_version().decode()


class Context:
    """Owns one rkm_ctx (device workspace, resident serving state)."""

    def __init__(self, precision: str = "bf16", device: int = 0, **opts):
        self.precision = precision
        self.handle = rkm_create(precision, device, **opts)

    def close(self) -> None:
        if self.handle:
            rkm_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def thresholds(self, U, P, k, want_topk=False):
        return rkm_thresholds(self.handle, U, P, k, want_topk)

    def scores(self, U, P, tau, tid):
        return rkm_scores(self.handle, U, P, tau, tid)

    def topn(self, U, P, k, N, return_thresholds=False):
        return rkm_topn(self.handle, U, P, k, N, return_thresholds)

    def topn_batch(self, problems, outs=None):
        return rkm_topn_batch(self.handle, problems, outs)

    def topn_from_topk(self, lists, m, k, N):
        return rkm_topn_from_topk(self.handle, lists, m, k, N)

    def topn_host(self, U, P, k, N):
        return rkm_topn_host(self.handle, U, P, k, N)

    def item_bounds(self, U, P, tau):
        return rkm_item_bounds(self.handle, U, P, tau)

    def resident_set(self, U, tau, tid):
        rkm_resident_set(self.handle, U, tau, tid)

    def query_new_items(self, Q):
        return rkm_query_new_items(self.handle, Q)

    def state_save(self, path):
        rkm_state_save(self.handle, path)

    def state_load(self, path):
        rkm_state_load(self.handle, path)

    def debug_products(self, U, P):
        return rkm_debug_products(self.handle, U, P)

    def stats(self) -> dict:
        return rkm_get_stats(self.handle)


class Server:
    """Serving loop over a Context's resident set (rkm_serve_*).  Requests are host numpy
    arrays; submit returns a ticket, wait returns (counts, latency_ms)."""

    def __init__(self, ctx: Context, **opts):
        self.ctx = ctx
        self.handle = rkm_serve_create(ctx.handle, **opts)
        self._held = {}

    def submit(self, Q) -> int:
        import numpy as np
        counts = np.empty(Q.shape[0], dtype=np.int32)
        t = rkm_serve_submit(self.handle, Q, counts)
        self._held[t] = (Q, counts)
        return t

    def wait(self, ticket: int, timeout_ms: float = -1.0):
        try:
            lat = rkm_serve_wait(self.handle, ticket, timeout_ms)
        except RkmError as e:
            if e.status != 5:  # the library released the ticket unless the wait timed out
                self._held.pop(ticket, None)
            raise
        return self._held.pop(ticket)[1], lat

    def drain(self) -> None:
        rkm_serve_drain(self.handle)

    def stats(self) -> dict:
        return rkm_serve_get_stats(self.handle)

    def reset_stats(self) -> None:
        rkm_serve_reset_stats(self.handle)

    def close(self) -> None:
        if self.handle:
            rkm_serve_destroy(self.handle)
            self.handle = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
