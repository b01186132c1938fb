"""Evaluation (RMSE of Eq. 30 on held-out entries, pattern distinctiveness of Eq. pd) against the
oracle, and checkpoint/resume of the full SaCD state (resumed runs are bit-identical)."""

import numpy as np
import pytest

from oracle import sacd_oracle as O
from paper_2003_03572_gb300 import sacd as S
from paper_2003_03572_gb300 import synth

pytestmark = pytest.mark.gpu


def split_case(dims=(400, 300, 60), nnz=30_000, R=16, seed=4):
    idx, vals = synth.sparse_tensor(dims, nnz, dist="zipf", zipf_s=1.1, seed=seed)
    rng = np.random.default_rng(seed)
    test = rng.random(nnz) < 0.2  # 80 / 20 split as in the paper's evaluation
    return dims, R, idx[:, ~test], vals[~test], idx[:, test], vals[test], synth.init_factors(dims, R, seed)


def test_rmse_and_pd_match_oracle():
    dims, R, tr_i, tr_v, te_i, te_v, init = split_case()
    with S.SaCD(dims, tr_i, tr_v, R, init) as g:
        g.iterate(5)
        F = g.factors()
        got = g.rmse([te_i[k] for k in range(3)], te_v)
        assert got == pytest.approx(O.rmse(te_i, te_v, F), rel=1e-9)
        assert g.rmse([te_i[k][:0] for k in range(3)], te_v[:0]) == 0.0
        for n in range(3):
            assert g.pattern_distinctiveness(n) == pytest.approx(O.pattern_distinctiveness(F[n]), rel=1e-8, abs=1e-12)
        bad = te_i.copy()
        bad[1, 0] = dims[1]
        with pytest.raises(S.SacdError):
            g.rmse([bad[k] for k in range(3)], te_v)


@pytest.mark.parametrize("prec", [S.SACD_FP32, S.SACD_BF16_GATHER])
def test_checkpoint_resume_is_bit_identical(prec):
    dims, R, tr_i, tr_v, _, _, init = split_case(R=32)
    with S.SaCD(dims, tr_i, tr_v, R, init, precision=prec) as a, S.SaCD(dims, tr_i, tr_v, R, init, precision=prec) as b:
        a.iterate(3)
        state = a.save()
        a.iterate(4)
        b.load(state)
        b.iterate(4)
        for n in range(3):
            np.testing.assert_array_equal(a.factor(n), b.factor(n))
            np.testing.assert_array_equal(a.tap("ZPREV", n), b.tap("ZPREV", n))
        assert a.fit() == b.fit()
    with S.SaCD(dims, tr_i, tr_v, R + 1, seed=1) as c:
        with pytest.raises(S.SacdError):
            c.load(state)  # another rank


def test_rejected_state_leaves_the_context_unchanged():
    """A state buffer whose last factor holds a negative value is rejected before anything is
    copied: every factor of the context stays as it was, and the context then runs on exactly like
    a twin that never saw the buffer."""
    dims, R, tr_i, tr_v, _, _, init = split_case(R=16)
    N = len(dims)
    with S.SaCD(dims, tr_i, tr_v, R, init) as a, S.SaCD(dims, tr_i, tr_v, R, init) as b:
        a.iterate(2)
        b.iterate(2)
        state = a.save()
        saved_last = a.factor(N - 1).copy()
        a.iterate(1)
        b.iterate(1)
        # layout: magic, N, R, nnz, dims; per mode ti^{k-1} and the first-visit flag, then the
        # factor and z^{k-1}, I_n x R FP32 each
        off = 24 + 8 * N + sum(16 + 8 * dims[n] * R for n in range(N - 1)) + 16
        stored = np.frombuffer(state, np.float32, count=dims[N - 1] * R, offset=off).reshape(dims[N - 1], R)
        np.testing.assert_array_equal(stored, saved_last)  # the offset points at the last factor
        bad = bytearray(state)
        bad[off:off + 4] = np.float32(-1.0).tobytes()
        before = [a.factor(n).copy() for n in range(N)]
        with pytest.raises(S.SacdError):
            a.load(bytes(bad))
        for n in range(N):
            np.testing.assert_array_equal(a.factor(n), before[n])
        a.iterate(2)
        b.iterate(2)
        for n in range(N):
            np.testing.assert_array_equal(a.factor(n), b.factor(n))
        assert a.fit() == b.fit()
