"""The FP32 evaluation bound of z (Eq. 11-12, 20) used by the parity tests, checked on the CPU.

The kernels evaluate s = max(0, a - g * (1/h)) - a and z = -g s - (L/2) s^2 in FP32 with
round-to-nearest and no fused operations, from g rounded to FP32 and 1/h, L/2 computed in FP64
and rounded once. numpy's float32 arithmetic is IEEE round-to-nearest, so the same operation
sequence here reproduces that evaluation; the bound must hold for it, also where the two terms of
Eq. 20 cancel, and must not be so loose that a dropped term passes.
"""

import numpy as np

from fp32_bounds import z_fp32_bound
from oracle import sacd_oracle as O

f32 = np.float32


def z_fp32(a, g, h, L):
    """Eq. 11-12 and Eq. 20 in the kernels' FP32 operation order."""
    g32 = g.astype(f32)
    ih = np.where(h > 0, 1.0 / np.where(h > 0, h, 1.0), 0.0).astype(f32)
    lh = (0.5 * np.broadcast_to(L, g.shape)).astype(f32)
    a32 = a.astype(f32)
    t = (a32 - (g32 * ih).astype(f32)).astype(f32)
    s = (np.maximum(t, f32(0)) - a32).astype(f32)
    return ((-g32 * s).astype(f32) - (lh * (s * s).astype(f32)).astype(f32)).astype(f32), s


def case(seed, I=400, R=16):
    rng = np.random.default_rng(seed)
    a = (rng.integers(0, 2**24, size=(I, R)) * 2.0**-24).astype(f32).astype(np.float64)
    h = rng.uniform(0.5, 4.0, size=R)
    H = np.diag(h)
    L = float(np.sqrt(np.sum(h * h)) * rng.uniform(2.0, 6.0))  # L > 2 h_rr as with dense Grams
    g = rng.standard_normal((I, R)) * rng.uniform(0.1, 5.0)
    # cancelling elements: clamped (s = -a) with g = L a / 2, unclamped with L = 2 h (per column
    # via a GCD-like L vector in the second half of the cases)
    q = I // 4
    g[:q] = 0.5 * L * a[:q] * (1 + 1e-6 * rng.standard_normal((q, R)))
    return a, dict(G=g, H=H, L=L)


def test_bound_holds_for_the_fp32_evaluation():
    worst = 0.0
    for seed in range(20):
        a, t = case(seed)
        h = np.diag(t["H"])
        if seed % 2:
            t["L"] = 2 * h * (1 + 1e-7)  # L = 2 h: the unclamped z cancels
        z32, _ = z_fp32(a, t["G"], h, t["L"])
        z = O.importance(t["G"], O.projected_delta(a, t["G"], h), t["L"])
        err = np.abs(z32.astype(np.float64) - z)
        b = z_fp32_bound(a, t)
        assert (err <= b).all()
        worst = max(worst, float((err / np.maximum(b, 1e-300)).max()))
    assert worst > 0.05  # the bound is within a small factor of what FP32 actually does


def test_bound_is_tight_where_nothing_cancels_and_catches_a_dropped_term():
    a, t = case(7)
    h = np.diag(t["H"])
    s = O.projected_delta(a, t["G"], h)
    z = O.importance(t["G"], s, t["L"])
    b = z_fp32_bound(a, t)
    rest = slice(len(a) // 4, None)  # elements built without cancellation
    assert np.median(b[rest] / np.maximum(np.abs(z[rest]), 1e-300)) < 1e-5
    # a planted mistake: z without the (L/2) s^2 term
    wrong = -t["G"] * s
    assert (np.abs(wrong - z) > b).mean() > 0.5


def _fma_order_ah_f32(A, H):
    """A H in FP32, one rounding per product-accumulate, j ascending (the kernel's FMA chain)."""
    A32 = A.astype(f32)
    H32 = H.astype(f32)
    acc = np.zeros((A.shape[0], H.shape[1]), np.float64)
    for j in range(A.shape[1]):
        acc = (acc + A32[:, j:j + 1].astype(np.float64) * H32[j:j + 1, :].astype(np.float64)).astype(f32)
        acc = acc.astype(np.float64)
    return acc


def _worst_step_error(dims, nnz, R, lnorm, iters=2):
    from paper_2003_03572_gb300 import synth

    idx, vals = synth.sparse_tensor(dims, nnz, dist="zipf", zipf_s=1.1, seed=11)
    o = O.SaCDOracle(dims, idx, vals, synth.init_factors(dims, R, 11), lnorm=lnorm)
    worst = 0.0
    for _ in range(iters):
        for n in range(len(dims)):
            A0 = o.A[n].copy()
            o.mode_step(n)
            t = o.last
            g32 = (_fma_order_ah_f32(A0, t["H"]) - t["M"].astype(f32)).astype(f32).astype(np.float64)
            A1, _ = O.update_rows(A0.copy(), g32, t["H"], t["sel"], "column_gs")
            worst = max(worst, float(np.linalg.norm(A1 - o.A[n]) / np.linalg.norm(o.A[n])))
    return worst


def test_plain_fp32_gradient_meets_the_step_bound_except_for_gcd():
    """The gradient G = A H - M summed in plain FP32 (fused multiply-adds, then one rounded
    subtraction of M), with the oracle's selection replayed, keeps a mode step well inside the
    1e-5 bound with the Frobenius or spectral L, but not with h_rr in place of L (Eq. 18), whose
    larger and more numerous steps amplify the gradient error: that variant needs compensated
    products."""
    shapes = [((257, 129, 65), 7777, 64), ((300, 200, 40, 20), 20_000, 16)]
    for dims, nnz, R in shapes:
        assert _worst_step_error(dims, nnz, R, "fro") < 2e-6
        assert _worst_step_error(dims, nnz, R, "spectral") < 2e-6
    assert max(_worst_step_error(d, z, R, "gcd") for d, z, R in shapes) > 1e-5
