"""Direct check of the guard band: every approximate product of the tensor-core paths lies
within its error bound E of the exact inner product.

The library's guarded paths are exact only if |v - u.p| <= E holds for every pair the
threshold and counting kernels see.  E is a rigorous Cauchy-Schwarz bound on the operand
rounding plus an accumulation term c_acc ||u^|| ||p^||, whose constant is an assumption
about the tensor cores' internal FP32 (BF16) and FP8 accumulation (the PTX ISA does not
specify either).  rkm_debug_products returns the products exactly as those kernels compute
them (same operand packs, TMA boxes, swizzle, MMA shape and FP8 descale) together with E;
the exact u.p comes from the oracle (FP64 is exact for grid inputs).  The largest ratio
|v - u.p| / E seen per path is printed, so that a run with -s records the margin.
"""
import json

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


def cancellation_rows():
    """Products that cancel almost completely (u.p tiny next to ||u|| ||p||)."""
    rng = np.random.default_rng(77)
    d, n, m = 64, 600, 900
    base = rng.integers(1000, 4096, size=(1, d)).astype(np.float64)
    signs = np.where(np.arange(d) % 2 == 0, 1.0, -1.0)
    U = (base + rng.integers(-3, 4, size=(n, d))) / 4096
    P = (base * signs + rng.integers(-3, 4, size=(m, d))) / 4096
    P *= np.ldexp(1.0, rng.integers(-2, 2, size=(m, 1)))
    return np.clip(U, -1, 1).astype(np.float32), np.clip(P, -2, 2).astype(np.float32)


def extreme_rows():
    """Rows scaled by 2^70 and 2^-80 (FP8 exponents clamp: saturation and underflow)."""
    W = workloads.mf(400, 300, 40, 7, 9, seed=61)
    U = W.U.copy()
    U[::5] *= np.float32(2.0 ** 70)
    U[1::5] *= np.float32(2.0 ** -80)
    P = W.P.copy()
    P[::7] *= np.float32(2.0 ** 20)
    return U, P


def full_mantissa_rows(d, n, m, seed):
    """Every entry a random 12-bit grid value (no rescaling): operand rounding of BF16/FP8
    hits every mantissa pattern, products of mixed signs."""
    rng = np.random.default_rng(seed)
    U = rng.integers(-4096, 4097, size=(n, d)) / 4096
    P = rng.integers(-4096, 4097, size=(m, d)) / 4096
    return U.astype(np.float32), P.astype(np.float32)


def exact_operand_rows(prec, d, n, m, seed):
    """Rows whose operands the path represents exactly, so that E reduces to the accumulation
    term c_acc ||u|| ||p|| (+ the underflow term) and |v - u.p| / E measures the tensor core's
    accumulation error against the assumed constant.  Entries are q / 4096 with q = mantissa x
    2^shift (BF16: 8-bit mantissas, shifts 0..4; FP8 e4m3 after the library's scale 2^8: 4-bit
    mantissas, shifts 0..8), so partial sums span far more than FP32's 24 bits.  Column 0
    holds +-3840 in every row, which fixes each row's exponent (and each item tile's) at 0."""
    rng = np.random.default_rng(seed)

    def rows(r):
        if prec == "fp8":
            q = rng.integers(1, 16, size=(r, d)) << rng.integers(0, 9, size=(r, d))
        else:
            q = rng.integers(1, 256, size=(r, d)) << rng.integers(0, 5, size=(r, d))
        q = q * rng.choice([-1, 1], size=(r, d))
        q[:, 0] = 3840 * rng.choice([-1, 1], size=r)
        return (q / 4096).astype(np.float32)
    return rows(n), rows(m)


CASES = {
    "mf-d128": lambda: (lambda W: (W.U, W.P))(workloads.mf(1024, 2048, 128, 10, 10, seed=5)),
    "mf-d64": lambda: (lambda W: (W.U, W.P))(workloads.mf(1024, 2048, 64, 10, 10, seed=6)),
    "mf-d100-ragged": lambda: (lambda W: (W.U, W.P))(workloads.mf(333, 1001, 100, 10, 10, seed=7)),
    "plain-d32": lambda: (lambda W: (W.U, W.P))(workloads.plain(700, 900, 32, 10, 10, seed=3)),
    "uniform-d256": lambda: full_mantissa_rows(256, 256, 768, 11),
    "cancellation-d64": cancellation_rows,
    "extreme-magnitudes-d40": extreme_rows,
}


@pytest.mark.parametrize("prec", ["bf16", "fp8"])
def test_products_within_guard_band(rkm, prec):
    worst = {}
    cases = dict(CASES)
    cases["exact-operands-d128"] = lambda: exact_operand_rows(prec, 128, 512, 1024, 21)
    cases["exact-operands-d256"] = lambda: exact_operand_rows(prec, 256, 256, 512, 22)
    for name, make in cases.items():
        U, P = make()
        assert oracle.on_grid(U) and oracle.on_grid(P)
        exact = oracle.inner_products(U, P)
        with rkm.Context(prec) as ctx:
            v, E = ctx.debug_products(torch.from_numpy(np.ascontiguousarray(U)).cuda(),
                                      torch.from_numpy(np.ascontiguousarray(P)).cuda())
            torch.cuda.synchronize()
        v = v.cpu().numpy().astype(np.float64)
        E = E.cpu().numpy().astype(np.float64)
        assert np.all(np.isfinite(v)) and np.all(E >= 0)
        err = np.abs(v - exact)
        bad = err > E
        assert not bad.any(), (f"{prec} {name}: {int(bad.sum())} products outside the guard band, "
                               f"worst excess {float((err - E).max()):.3e}")
        pos = E > 0
        assert np.all(err[~pos] == 0)
        ratio = float((err[pos] / E[pos]).max()) if pos.any() else 0.0
        # the accumulation term alone, for the margin of the c_acc assumption
        worst[name] = {"max_err_over_E": ratio, "max_abs_err": float(err.max()), "pairs": int(err.size)}
    print("GUARD_BAND " + json.dumps({"precision": prec, "cases": worst}))
