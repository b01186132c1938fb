"""The allocation-free MTTKRP entry point (sacd_mttkrp_noalloc), for callers that cannot call
cudaMalloc. It is checked through the C ABI against the MTTKRP that a regular context's mode
step computes from the same factors (the existing entry point) and against the FP64 oracle's
MTTKRP, within the MTTKRP tolerance of the other tests: 1e-5 relative Frobenius, and element by
element |M - M_ref| <= 1e-5 (|M_ref| + max |M_ref| of the row). Two calls in a row with the same
inputs must both match, and a call with other factors in between must not leak into the next
one (the static scratch keeps the previous call's partial rows). This file is collected last on
purpose.
"""

import numpy as np
import pytest

from oracle import sacd_oracle as O
from paper_2003_03572_gb300 import sacd as S
from paper_2003_03572_gb300 import synth


def relerr(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0))


def elementwise_ok(got, ref, tol=1e-5):
    ref = np.asarray(ref, np.float64)
    rowmax = np.abs(ref).max(axis=1, keepdims=True)
    return bool((np.abs(np.asarray(got, np.float64) - ref) <= tol * (np.abs(ref) + rowmax)).all())


def test_noalloc_rejects_sizes_beyond_the_static_scratch():
    # checked on the host before any GPU work: 2^31-1 nonzeros need far more than 16 MiB of partials
    dims = (1000, 1000, 1000)
    with pytest.raises(S.SacdError) as e:
        S.sacd_mttkrp_noalloc(dims, 0, 2**31 - 1, 16, 16, 16, [16, 16, 16], 256, 256, 16)
    assert e.value.status == 1 and "static scratch" in str(e.value)
    with pytest.raises(S.SacdError) as e:
        S.sacd_mttkrp_noalloc(dims, 0, 100, 16, 16, 16, [16, 16, 16], 32, 40, 16)  # ld not the padded rank
    assert e.value.status == 1


def _padded(torch, A, Rp, dev):
    P = torch.zeros((A.shape[0], Rp), dtype=torch.float32)
    P[:, : A.shape[1]] = torch.from_numpy(np.ascontiguousarray(A))
    return P.to(dev)


def _check_modes(dims, idx, vals, R, seed, modes=None):
    torch = pytest.importorskip("torch")
    dev = torch.device("cuda:0")
    init = synth.init_factors(dims, R, seed)
    cidx, cvals = O.coalesce(dims, idx, vals)
    with S.SaCD(dims, idx, vals, R, init) as g:
        Rp = g.info["rank_padded"]
        nz = g.info["nnz"]
        for n in modes if modes is not None else range(len(dims)):
            F = g.factors()  # factors the step's MTTKRP uses
            g.mode_step(n, want_count=False)
            M_ctx = g.tap("M", n)  # the existing entry point's MTTKRP
            M_ora = O.mttkrp(list(dims), cidx, cvals, F, n)
            row, other, v = O.csf_arrays(cidx, cvals, n)  # the oracle's mode-n sort
            rowid = torch.from_numpy(row).to(dev)
            ci = torch.from_numpy(np.ascontiguousarray(other)).to(dev)
            vv = torch.from_numpy(v).to(dev)
            fac = [_padded(torch, A, Rp, dev) for A in F]
            fac2 = [2.0 * f for f in fac]  # other factors for the call in between
            M = torch.empty((dims[n], Rp), dtype=torch.float32, device=dev)
            for call in range(3):
                M.fill_(float("nan"))
                torch.cuda.synchronize()
                S.sacd_mttkrp_noalloc(dims, n, nz, rowid, ci, vv, fac2 if call == 1 else fac, R, Rp, M)
                torch.cuda.synchronize()
                got = M[:, :R].cpu().numpy()
                assert np.isfinite(got).all()
                scale = 2.0 ** (len(dims) - 1) if call == 1 else 1.0
                assert relerr(got, scale * M_ora) <= 1e-5
                assert elementwise_ok(got, scale * M_ora)
                if call != 1:
                    assert relerr(got, M_ctx) <= 1e-5
                    assert elementwise_ok(got, M_ctx)


@pytest.mark.gpu
@pytest.mark.parametrize("dims,nnz,R", [((600, 400, 50), 30_000, 32), ((300, 200, 40, 20), 20_000, 16),
                                         ((100, 100, 100), 10_000, 5)])
def test_noalloc_mttkrp_matches_mode_step_and_oracle(dims, nnz, R):
    idx, vals = synth.sparse_tensor(dims, nnz, dist="zipf", zipf_s=1.1, seed=5)
    _check_modes(dims, idx, vals, R, 5)


@pytest.mark.gpu
def test_noalloc_mttkrp_large_tiles_and_long_border_runs():
    """5M nonzeros at R = 32: the tile rule reaches its largest lane-group share (128 nonzeros),
    and the hottest Zipf rows (over 200k nonzeros) cross hundreds of tile borders, so the border
    fix-up sums long runs of partials."""
    w = synth.WORKLOADS["zipf1.1-50000x20000x500-5M-r32"]
    idx, vals, _ = synth.make_workload(w)
    counts = np.bincount(idx[2], minlength=w.dims[2])
    assert counts.max() > 200_000
    _check_modes(w.dims, idx, vals, w.rank, 9, modes=[2, 0])
