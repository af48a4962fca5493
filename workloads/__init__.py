"""Seeded synthetic inputs for the reverse k-MIPS top-N workloads.

This module holds only random-number generation and the quantisation of the
generated vectors to the 2^-12 grid.  It contains none of the method's
arithmetic (no inner products, no selection, no counting), so that the FP64
oracle and the CUDA path can both read the same bytes without sharing code.

Every value a generator returns is a float32 of the form ``2^e * q / 4096``
with an integer ``|q| <= 4096`` and a per-row integer exponent ``e``.  For such
inputs every inner product of two rows (d <= 128) is an integer multiple of a
power of two below 2^53 in magnitude, hence exact in FP64 whatever the
summation order.

Random numbers come from SplitMix64 (Steele, Lea & Flood, "Fast splittable
pseudorandom number generators", OOPSLA 2014) run as a counter-based stream:
output ``i`` of stream ``key`` is ``mix64(key + (i + 1) * 0x9E3779B97F4A7C15)``.
Uniforms take the top 53 bits; normals use the Box-Muller transform.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
GRID_BITS = 12          # values are multiples of 2^(e - 12)
GRID = 1 << GRID_BITS   # 4096


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def stream_key(seed: int, tag: int) -> int:
    """Key of the stream for (seed, tag); tags separate users, items, queries."""
    with np.errstate(over="ignore"):
        base = np.array([(seed * 1_000_003 + tag * 7_919 + 1) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64)
        return int(_mix64(base * _GAMMA)[0])


def uniform53(key: int, start: int, count: int) -> np.ndarray:
    """Outputs start..start+count-1 of the stream as float64 in (0, 1)."""
    with np.errstate(over="ignore"):
        idx = np.arange(start + 1, start + count + 1, dtype=np.uint64)
        z = _mix64(np.uint64(key) + idx * _GAMMA)
    return ((z >> np.uint64(11)).astype(np.float64) + 0.5) * (1.0 / 9007199254740992.0)


def normal(key: int, start: int, count: int) -> np.ndarray:
    """Normals start..start+count-1 of the stream: normals 2j and 2j+1 come from
    uniforms 2j and 2j+1 by the Box-Muller transform."""
    p0 = start // 2
    pairs = (start + count + 1) // 2 - p0
    u = uniform53(key, 2 * p0, 2 * pairs)
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log(u1))
    t = 2.0 * math.pi * u2
    out = np.empty(2 * pairs, dtype=np.float64)
    out[0::2] = r * np.cos(t)
    out[1::2] = r * np.sin(t)
    off = start - 2 * p0
    return out[off:off + count]


def row_exponents(x: np.ndarray) -> np.ndarray:
    """Smallest integer e per row with max|x_row| <= 2^e (0 for an all-zero row)."""
    mx = np.max(np.abs(x), axis=1)
    f, e = np.frexp(mx)             # mx = f * 2^e, f in [0.5, 1)
    e = e.astype(np.int64)
    e = np.where(f == 0.5, e - 1, e)
    return np.where(mx == 0.0, 0, e)


def quantise_rows(x: np.ndarray) -> np.ndarray:
    """Round each row to the grid 2^(e-12) (half to even), e = row_exponents(x)."""
    e = row_exponents(x)[:, None]
    q = np.rint(np.ldexp(x, GRID_BITS - e))
    return np.ldexp(q, e - GRID_BITS).astype(np.float32)


def gaussian_clipped(n: int, d: int, seed: int, tag: int, sigma: float = 0.5,
                     block: int = 1 << 16) -> np.ndarray:
    """Entries N(0, sigma^2) clipped to [-1, 1] and rounded to the 2^-12 grid (e = 0)."""
    key = stream_key(seed, tag)
    out = np.empty((n, d), dtype=np.float32)
    for r0 in range(0, n, block):
        r1 = min(n, r0 + block)
        g = normal(key, r0 * d, (r1 - r0) * d).reshape(r1 - r0, d) * sigma
        g = np.clip(g, -1.0, 1.0)
        out[r0:r1] = (np.rint(g * GRID) / GRID).astype(np.float32)
    return out


def mf_like(n: int, d: int, seed: int, tag: int, norm_sigma: float,
            row0: int = 0, block: int = 1 << 15) -> np.ndarray:
    """Matrix-factorisation-like rows row0..row0+n-1 of a stream: Gaussian direction
    times a log-normal(0, norm_sigma) norm, rounded per row to the grid 2^(e-12) with
    the row's own power-of-two exponent."""
    key = stream_key(seed, tag)
    nkey = stream_key(seed, tag + 101)
    out = np.empty((n, d), dtype=np.float32)
    for b0 in range(0, n, block):
        b1 = min(n, b0 + block)
        r0, r1 = row0 + b0, row0 + b1
        g = normal(key, r0 * d, (r1 - r0) * d).reshape(r1 - r0, d)
        gn = np.sqrt(np.sum(g * g, axis=1, keepdims=True))
        gn = np.where(gn == 0.0, 1.0, gn)
        r = np.exp(norm_sigma * normal(nkey, r0, r1 - r0))[:, None]
        out[b0:b1] = quantise_rows(r * g / gn)
    return out


TAG_USERS, TAG_ITEMS, TAG_QUERIES, TAG_SERVING = 1, 2, 3, 4


@dataclass
class Workload:
    """One reverse k-MIPS top-N instance: users U [n, d], items P [m, d], k, N."""
    name: str
    U: np.ndarray
    P: np.ndarray
    k: int
    N: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.U.shape[0]

    @property
    def m(self) -> int:
        return self.P.shape[0]

    @property
    def d(self) -> int:
        return self.U.shape[1]


def plain(n: int = 2000, m: int = 1000, d: int = 32, k: int = 10, N: int = 10,
          seed: int = 0) -> Workload:
    """Plain exact workload: i.i.d. N(0, 0.25) entries, clipped, on the 2^-12 grid."""
    U = gaussian_clipped(n, d, seed, TAG_USERS)
    P = gaussian_clipped(m, d, seed, TAG_ITEMS)
    return Workload(f"plain n={n} m={m} d={d} k={k} N={N} seed={seed}", U, P, k, N,
                    {"generator": "gaussian_clipped", "seed": seed})


def mf(n: int, m: int, d: int, k: int, N: int, seed: int,
       user_sigma: float = 0.3, item_sigma: float = 0.5) -> Workload:
    """MF-like workload: log-normal norms (users 0.3, items 0.5), Gaussian directions."""
    U = mf_like(n, d, seed, TAG_USERS, user_sigma)
    P = mf_like(m, d, seed, TAG_ITEMS, item_sigma)
    return Workload(f"mf n={n} m={m} d={d} k={k} N={N} seed={seed}", U, P, k, N,
                    {"generator": "mf_like", "seed": seed})


def queries(q: int, d: int, seed: int, item_sigma: float = 0.5, start_row: int = 0) -> np.ndarray:
    """New candidate item vectors drawn like catalogue items: rows start_row..start_row+q-1
    of the query stream (TAG_QUERIES) of this seed."""
    return mf_like(q, d, seed, TAG_QUERIES, item_sigma, row0=start_row)


# The workloads the benchmarks and parity tests use, by name.
CONFIGS = {
    "plain-2k": dict(kind="plain", n=2000, m=1000, d=32, k=10, N=10, seed=0),
    "mf-500k": dict(kind="mf", n=500_000, m=100_000, d=64, k=25, N=50, seed=1),
    "mf-2m-k10": dict(kind="mf", n=2_000_000, m=500_000, d=128, k=10, N=100, seed=2),
    "mf-2m-k50": dict(kind="mf", n=2_000_000, m=500_000, d=128, k=50, N=100, seed=2),
}


def make(name: str, **override) -> Workload:
    cfg = dict(CONFIGS[name])
    cfg.update(override)
    kind = cfg.pop("kind")
    if kind == "plain":
        return plain(**cfg)
    return mf(**cfg)


def rows(name: str, which: str, row0: int = 0, count: int | None = None, **override) -> np.ndarray:
    """Rows row0 .. row0+count-1 of the users ("U") or items ("P") of a named workload,
    generated on their own (the same bytes as slicing make(name)); for the MF-like
    workloads only those rows are drawn."""
    cfg = dict(CONFIGS[name])
    cfg.update(override)
    total = cfg["n"] if which == "U" else cfg["m"]
    count = total - row0 if count is None else min(count, total - row0)
    if cfg["kind"] == "plain":
        W = make(name, **override)
        return (W.U if which == "U" else W.P)[row0:row0 + count]
    tag, sigma = (TAG_USERS, 0.3) if which == "U" else (TAG_ITEMS, 0.5)
    return mf_like(count, cfg["d"], cfg["seed"], tag, sigma, row0=row0)


def batching_instances(count: int = 64, base_seed: int = 1000) -> list[dict]:
    """Sizes of the multi-instance batch: users log-uniform in [1e4, 1e6], items
    log-uniform in [5e3, 2e5], d in {32, 64, 128}, k in {5, 10, 25}, N = 20."""
    out = []
    for j in range(count):
        key = stream_key(base_seed + j, 77)
        u = uniform53(key, 0, 4)
        n = int(round(math.exp(math.log(1e4) + u[0] * (math.log(1e6) - math.log(1e4)))))
        m = int(round(math.exp(math.log(5e3) + u[1] * (math.log(2e5) - math.log(5e3)))))
        d = (32, 64, 128)[min(2, int(u[2] * 3))]
        k = (5, 10, 25)[min(2, int(u[3] * 3))]
        out.append(dict(n=n, m=m, d=d, k=k, N=20, seed=base_seed + j))
    return out


# The serving workload: resident users and the catalogue their thresholds come from, then a
# stream of what-if requests whose candidate rows come from the query stream of query_seed.
SERVING = dict(n=1_000_000, m=300_000, d=100, k=20, catalog_seed=3, query_seed=4)


def serving_stream(count: int, rate_per_s: float, seed: int = 4, max_q: int = 4096):
    """Poisson arrivals of `count` requests at `rate_per_s` (exponential gaps; rate <= 0 puts
    every arrival at time 0) with sizes log-uniform over [1, max_q]:
    q = min(max_q, floor(exp(U * ln(max_q + 1)))) for U uniform in (0, 1).  Request j's
    candidates are rows offsets[j] .. offsets[j] + sizes[j] - 1 of queries(.., seed).
    Returns (arrival times in seconds, sizes, offsets) as numpy arrays."""
    key = stream_key(seed, TAG_SERVING)
    u = uniform53(key, 0, 2 * count).reshape(count, 2)
    sizes = np.minimum(max_q, np.floor(np.exp(u[:, 0] * math.log(max_q + 1.0)))).astype(np.int64)
    sizes = np.maximum(sizes, 1)
    if rate_per_s > 0:
        arrivals = np.cumsum(-np.log(u[:, 1]) / rate_per_s)
    else:
        arrivals = np.zeros(count)
    offsets = np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64)
    return arrivals, sizes, offsets
