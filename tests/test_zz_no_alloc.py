"""The allocation-free MTTKRP entry point (sacd_mttkrp_noalloc), for callers that cannot call
cudaMalloc. It is checked through the C ABI against the MTTKRP that a regular context's mode
step computes from the same factors, within the MTTKRP tolerance of the other tests (1e-5
relative Frobenius), on two calls in a row (the static scratch keeps the previous call's
contents, which must not leak into the next result). This file is collected last on purpose.
"""

import numpy as np
import pytest

from paper_2003_03572_gb300 import sacd as S
from paper_2003_03572_gb300 import synth


def relerr(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0))


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    # checked on the host before any GPU work: 2^31-1 nonzeros need far more than 16 MiB of partials
    dims = (1000, 1000, 1000)
    with pytest.raises(S.SacdError) as e:
        S.sacd_mttkrp_noalloc(dims, 0, 2**31 - 1, 16, 16, 16, [16, 16, 16], 256, 256, 16)
    assert e.value.status == 1 and "static scratch" in str(e.value)
    with pytest.raises(S.SacdError) as e:
        S.sacd_mttkrp_noalloc(dims, 0, 100, 16, 16, 16, [16, 16, 16], 32, 40, 16)  # ld not the padded rank
    assert e.value.status == 1


@pytest.mark.gpu
@pytest.mark.parametrize("dims,nnz,R", [((600, 400, 50), 30_000, 32), ((300, 200, 40, 20), 20_000, 16),
                                         ((100, 100, 100), 10_000, 5)])
def test_noalloc_mttkrp_matches_mode_step(dims, nnz, R):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    idx, vals = synth.sparse_tensor(dims, nnz, dist="zipf", zipf_s=1.1, seed=5)
    init = synth.init_factors(dims, R, 5)
    with S.SaCD(dims, idx, vals, R, init) as g:
        Rp = g.info["rank_padded"]
        nz = g.info["nnz"]
        for n in range(len(dims)):
            F = g.factors()                 # factors the step's MTTKRP uses
            g.mode_step(n, want_count=False)
            M_ref = g.tap("M", n)
            rowid = torch.from_numpy(g.tap("CSF_ROW", n)).to(dev)
            cidx = torch.from_numpy(np.ascontiguousarray(g.tap("CSF_IDX", n))).to(dev)
            v = torch.from_numpy(g.tap("CSF_VAL", n)).to(dev)
            fac = []
            for k, A in enumerate(F):
                P = torch.zeros((A.shape[0], Rp), dtype=torch.float32)
                P[:, :R] = torch.from_numpy(A)
                fac.append(P.to(dev))
            M = torch.empty((dims[n], Rp), dtype=torch.float32, device=dev)
            for call in range(2):
                M.fill_(float("nan"))
                torch.cuda.synchronize()
                S.sacd_mttkrp_noalloc(dims, n, nz, rowid, cidx, v, fac, R, Rp, M)
                torch.cuda.synchronize()
                got = M[:, :R].cpu().numpy()
                assert np.isfinite(got).all()
                assert relerr(got, M_ref) <= 1e-5
