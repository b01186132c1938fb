"""Batches of independent jobs: every job's result is bit-identical alone and in the mix, and
the batched fits match the FP64 oracle (FP32 jobs within 1e-4, as for single contexts)."""

import numpy as np
import pytest

from oracle import sacd_oracle as O
from paper_2003_03572_gb300 import sacd as S
from paper_2003_03572_gb300 import synth

pytestmark = pytest.mark.gpu


def job_specs(seed=21):
    rng = np.random.default_rng(seed)
    specs = []
    shapes = [((200, 150, 40), 5), ((300, 120, 30), 8), ((150, 160, 20), 16), ((400, 250, 50), 32),
              ((80, 70, 60, 10), 16), ((120, 90, 30, 12), 64), ((50, 40, 30), 1), ((500, 300, 20), 24)]
    for j in range(20):
        dims, R = shapes[j % len(shapes)]
        nnz = int(rng.integers(2000, 12000))
        idx, vals = synth.sparse_tensor(dims, nnz, dist="zipf", zipf_s=1.1, seed=seed * 100 + j)
        init = synth.init_factors(dims, R, seed * 100 + j)
        prec = S.SACD_BF16_GATHER if j % 5 == 4 else S.SACD_FP32
        specs.append(dict(dims=dims, idx=idx, vals=vals, rank=R, init=init, precision=prec))
    # a job with no nonzeros
    specs.append(dict(dims=(30, 20, 10), idx=np.zeros((3, 0), np.int32), vals=np.zeros(0, np.float32), rank=4,
                      init=synth.init_factors((30, 20, 10), 4, 1)))
    return specs


def test_batch_bit_identical_to_alone():
    specs = job_specs()
    K = 4
    with S.SaCDBatch(specs) as b:
        b.iterate(K)
        obj, fit = b.fit()
        for j, sp in enumerate(specs):
            with S.SaCD(sp["dims"], sp["idx"], sp["vals"], sp["rank"], sp["init"], precision=sp["precision"]
                        if "precision" in sp else 0) as a:
                a.iterate(K)
                for n in range(len(sp["dims"])):
                    np.testing.assert_array_equal(b.factor(j, n), a.factor(n))
                oa, fa = a.fit()
                assert obj[j] == oa and fit[j] == fa


def test_batch_fits_match_oracle():
    specs = [s for s in job_specs(33) if s.get("precision", 0) == 0][:6]
    K = 10
    with S.SaCDBatch(specs) as b:
        b.iterate(K)
        obj, fit = b.fit()
    for j, sp in enumerate(specs):
        o = O.SaCDOracle(sp["dims"], sp["idx"], sp["vals"], sp["init"])
        o.iterate(K)
        assert abs(fit[j] - o.fit()[1]) <= 1e-4


def test_batch_of_small_ranks_only():
    """A batch whose jobs have padded ranks 16 and 8 only. The fused select/update kernel's shared
    memory need is not monotonic in the rank (rank 8 takes 1024-row chunks and more memory than
    rank 16), so one launch for both must be sized by the larger need, not by the larger rank.
    Results bit-identical to the jobs run alone."""
    specs = []
    for j, (dims, R) in enumerate([((300, 200, 50), 16), ((200, 220, 60), 8), ((1500, 90, 30), 8)]):
        idx, vals = synth.sparse_tensor(dims, 5000 + 2000 * j, dist="zipf", zipf_s=1.1, seed=40 + j)
        specs.append(dict(dims=dims, idx=idx, vals=vals, rank=R, init=synth.init_factors(dims, R, 40 + j)))
    with S.SaCDBatch(specs) as b:
        b.iterate(3)
        obj, fit = b.fit()
        for j, sp in enumerate(specs):
            with S.SaCD(sp["dims"], sp["idx"], sp["vals"], sp["rank"], sp["init"]) as a:
                a.iterate(3)
                for n in range(3):
                    np.testing.assert_array_equal(b.factor(j, n), a.factor(n))
                assert (obj[j], fit[j]) == a.fit()


def test_batch_mixes_tensor_core_and_fp32_grams():
    """Jobs of one padded rank whose mode-0 factors are tall (Gram on the tensor cores, I Rp >=
    2^20) or short (FP32-pipe Gram) run in one batch: the launch splits them by Gram kind, every
    result stays bit-identical to the job alone, and each Gram of the final factors matches the
    FP64 oracle within 1e-10."""
    specs = []
    shapes = [((40000, 300, 50), 32), ((3000, 200, 40), 32), ((20000, 500, 30), 64), ((5000, 400, 20), 64)]
    for j, (dims, R) in enumerate(shapes):
        idx, vals = synth.sparse_tensor(dims, 20000 + 5000 * j, dist="zipf", zipf_s=1.1, seed=60 + j)
        specs.append(dict(dims=dims, idx=idx, vals=vals, rank=R, init=synth.init_factors(dims, R, 60 + j)))
    with S.SaCDBatch(specs) as b:
        b.iterate(3)
        obj, fit = b.fit()
        for j, sp in enumerate(specs):
            with S.SaCD(sp["dims"], sp["idx"], sp["vals"], sp["rank"], sp["init"]) as a:
                a.iterate(3)
                for n in range(3):
                    F = a.factor(n)
                    np.testing.assert_array_equal(b.factor(j, n), F)
                    ref = O.gram(F)
                    assert np.linalg.norm(a.tap("GRAM", n) - ref) <= 1e-10 * np.linalg.norm(ref)
                assert (obj[j], fit[j]) == a.fit()
