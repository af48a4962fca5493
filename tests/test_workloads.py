"""The seeded generators: grid property, determinism by row range, and the serving stream
(Poisson arrivals, log-uniform request sizes)."""
import numpy as np

import oracle
import workloads


def test_rows_are_generated_independently_of_the_range():
    a = workloads.mf_like(50, 16, seed=9, tag=workloads.TAG_ITEMS, norm_sigma=0.5)
    b = workloads.mf_like(20, 16, seed=9, tag=workloads.TAG_ITEMS, norm_sigma=0.5, row0=30)
    np.testing.assert_array_equal(a[30:], b)
    assert oracle.on_grid(a)


def test_serving_stream_sizes_and_offsets():
    arr, sizes, offs = workloads.serving_stream(5000, 100.0, seed=4)
    assert sizes.min() >= 1 and sizes.max() <= 4096
    np.testing.assert_array_equal(offs[1:], np.cumsum(sizes)[:-1])
    assert offs[0] == 0
    # log-uniform over [1, 4097): the median of exp(U ln 4097) is sqrt(4097) ~ 64
    assert 45 <= np.median(sizes) <= 90
    # Poisson arrivals at 100/s: exponential gaps with mean 10 ms, increasing times
    gaps = np.diff(np.r_[0.0, arr])
    assert np.all(gaps > 0)
    assert abs(gaps.mean() - 0.01) < 0.001
    assert abs(gaps.std() / gaps.mean() - 1.0) < 0.1  # exponential: std = mean
    # deterministic and rate-free sizes
    arr2, sizes2, _ = workloads.serving_stream(5000, 1.0, seed=4)
    np.testing.assert_array_equal(sizes, sizes2)
    np.testing.assert_allclose(arr2, arr * 100.0, rtol=1e-12)


def test_serving_stream_all_at_once():
    arr, sizes, _ = workloads.serving_stream(10, 0.0, seed=4)
    assert np.all(arr == 0.0) and len(sizes) == 10


def test_queries_on_grid_with_mf_norms():
    Q = workloads.queries(2000, 100, seed=4)
    assert Q.dtype == np.float32 and oracle.on_grid(Q)
    ln = np.log(np.linalg.norm(Q.astype(np.float64), axis=1))
    assert abs(ln.mean()) < 0.05 and abs(ln.std() - 0.5) < 0.05
