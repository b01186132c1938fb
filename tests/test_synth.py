"""The seeded input generator: exact nnz, distinct in-range coordinates, determinism."""

import numpy as np
import pytest

from paper_2003_03572_gb300 import synth


@pytest.mark.parametrize("dims,nnz,dist,s", [((100, 100, 100), 10_000, "uniform", 0.0),
                                             ((5000, 2000, 50), 200_000, "zipf", 1.1),
                                             ((2000, 1000, 100, 20), 100_000, "zipf", 1.2),
                                             ((70_000, 90_000, 80_000, 60_000), 50_000, "zipf", 1.1)])
def test_sparse_tensor_distinct_exact(dims, nnz, dist, s):
    idx, vals = synth.sparse_tensor(dims, nnz, dist=dist, zipf_s=s, seed=3)
    assert idx.shape == (len(dims), nnz) and idx.dtype == np.int32
    assert vals.shape == (nnz,) and vals.dtype == np.float32
    for k, d in enumerate(dims):
        assert idx[k].min() >= 0 and idx[k].max() < d
    assert np.unique(idx.T, axis=0).shape[0] == nnz
    assert set(np.unique(vals)) <= {1.0, 2.0, 3.0, 4.0, 5.0}
    idx2, vals2 = synth.sparse_tensor(dims, nnz, dist=dist, zipf_s=s, seed=3)
    np.testing.assert_array_equal(idx, idx2)
    np.testing.assert_array_equal(vals, vals2)


def test_zipf_is_skewed():
    rng = np.random.default_rng(0)
    k = synth.zipf_indices(rng, 1000, 1.1, 200_000)
    counts = np.sort(np.bincount(k, minlength=1000))[::-1]
    # P(rank 1) / P(rank 10) = 10^1.1
    assert counts[0] / counts[9] == pytest.approx(10**1.1, rel=0.15)


def test_init_factors_exact_in_fp32():
    F = synth.init_factors((7, 9), 5, 1)
    for A in F:
        assert A.dtype == np.float32 and (A >= 0).all() and (A < 1).all()
        np.testing.assert_array_equal(A.astype(np.float64) * 2**24, np.round(A.astype(np.float64) * 2**24))


def test_serving_workloads_distribution():
    tensors, jobs = synth.serving_workloads(400, pool=40)
    assert len(tensors) == 40 and len(jobs) == 400
    for w in tensors:
        assert w.nmodes in (3, 4)
        assert all(500 <= d <= 100_000 for d in w.dims)
        assert 1 <= w.nnz <= 5_000_000
    assert {r for _, r, _ in jobs} == {16, 32, 64}


def test_poisson_arrivals_rate():
    from paper_2003_03572_gb300 import serve

    a = serve.poisson_arrivals(200.0, 20000, 1)
    assert (np.diff(a) > 0).all()
    assert a[-1] / 20000 == pytest.approx(1 / 200.0, rel=0.03)
