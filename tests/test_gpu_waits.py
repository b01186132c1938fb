"""Bounded waits of the fused select/update kernel. Its blocks meet at a grid barrier between the
sum of z (ti, Eq. 25) and the selection (Eq. 24/27); every wait there is bounded by a cycle budget.
Here the budget is set to one cycle, so the blocks that arrive first give up at once: the kernel
must return (not hang), the next waiting call must report SACD_ETIMEOUT, the context is then
poisoned, and the GPU stays usable (a new context runs normally)."""

import numpy as np
import pytest

from oracle import sacd_oracle as O
from paper_2003_03572_gb300 import sacd as S
from paper_2003_03572_gb300 import synth

pytestmark = pytest.mark.gpu


def test_wait_budget_runs_out_and_reports_timeout():
    dims, R = (50_000, 300, 40), 32  # mode 0: 196 row chunks, so many blocks wait at the barrier
    idx, vals = synth.sparse_tensor(dims, 200_000, dist="zipf", zipf_s=1.1, seed=4)
    init = synth.init_factors(dims, R, 4)
    with S.SaCD(dims, idx, vals, R, init) as g:
        with pytest.raises(S.SacdError):
            S.sacd_set_wait_budget(g.ctx, 0)
        S.sacd_set_wait_budget(g.ctx, 1)
        with pytest.raises(S.SacdError) as e:
            g.mode_step(0)  # waits for the step: the error word is read
        assert e.value.status == 4 and "gave up" in str(e.value)
        with pytest.raises(S.SacdError) as e:
            g.fit()
        assert e.value.status == 5  # poisoned
    # the GPU is fine: a fresh context steps and matches the oracle
    with S.SaCD(dims, idx, vals, R, init) as g:
        g.set_debug(True)
        o = O.SaCDOracle(dims, idx, vals, init)
        g.mode_step(0)
        o.mode_step(0, mask=g.tap("MASK", 0, last_mode=0).astype(bool))
        A = g.factor(0)
        assert np.linalg.norm(A - o.A[0]) <= 1e-5 * np.linalg.norm(o.A[0])


def test_default_budget_never_runs_out_on_a_full_iteration():
    dims, R = (50_000, 300, 40), 32
    idx, vals = synth.sparse_tensor(dims, 200_000, dist="zipf", zipf_s=1.1, seed=4)
    with S.SaCD(dims, idx, vals, R, seed=4) as g:
        g.iterate(3)
        S.sacd_sync(g.ctx)
        assert np.isfinite(g.fit()[0])
