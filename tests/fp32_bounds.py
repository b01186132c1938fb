"""FP32 evaluation bounds used by the parity tests (test infrastructure)."""

import numpy as np

from oracle import sacd_oracle as O

U32 = 2.0**-24  # unit roundoff of FP32


def z_fp32_bound(a, t):
    """Per-element bound on |z_fp32 - z| for z = -g s - (L/2) s^2 (Eq. 20) with
    s = max(0, a - g/h) - a (Eq. 11-12) evaluated in FP32 from the FP32-rounded g.

    With u the FP32 roundoff: the rounded g, 1/h, their product and the two subtractions give
    |ds| <= 3u (|g|/h + |a| + |s|), which z scales by |g| + L|s|; the rounded g times s, the
    products s*s and (L/2)*s^2 (with L/2 rounded) and the difference add at most 4u of each
    term. The bound is twice the first-order sum. When the two terms of Eq. 20 cancel it
    exceeds any fixed fraction of max |z|."""
    a = np.asarray(a, np.float64)
    g = t["G"]
    h = O.curvatures(t["H"])
    L = np.broadcast_to(np.asarray(t["L"], np.float64), g.shape)
    s = O.projected_delta(a, g, h)
    inv = np.where(h > 0, 1.0 / np.where(h > 0, h, 1.0), 0.0)
    ds = 3 * U32 * (np.abs(g) * inv + np.abs(a) + np.abs(s))
    return 2 * ((np.abs(g) + L * np.abs(s)) * ds + 4 * U32 * (np.abs(g * s) + 0.5 * L * s * s))
