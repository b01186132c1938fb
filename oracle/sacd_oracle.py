"""FP64 CPU oracle for Saturating Coordinate Descent (SaCD) on sparse N-mode tensors.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
and reference legs may import or run this module. The product path (the CUDA library and its
Python binding) never calls it, and it shares no code with that path: it takes plain numpy
arrays and computes everything itself in FP64, one definition at a time, in the order of the
paper (Balasubramaniam, Nayak, Yuen, "Efficient Nonnegative Tensor Factorization via Saturating
Coordinate Descent", Algorithm 1, Sections 4.1-4.3).

Notation: N modes, factor ``A[n]`` of shape (I_n, R) (the paper's U, V, W for N = 3), tensor
nonzeros ``idx`` (N, nnz) int and ``vals`` (nnz,). Functions cite the equation they follow.

Readings where the paper is silent or garbled (each one is also listed with its reason in the
design notes of the repository):

* The delta in the importance (Eq. 20) is the projected delta of Eq. 12,
  s = max(0, u - g/h) - u, not the raw ratio of Eq. 11.
* L is the Frobenius norm of H (symbol table; proof of Lemma 1); the spectral norm is a flag,
  and "gcd" replaces L by h_rr per column (the GCD importance of Eq. 18).
* Selection uses z from the gradient at the start of the mode step, for every element; the ti
  comparison is strict (ti^k > ti^{k-1} takes Eq. 27) and an element is updated only if sp > 0
  (strict); z^{k-1} is refreshed for every element, selected or not.
* "k == 1" of Algorithm 1 is read per factor: the first time a factor is visited, z > 0 selects.
* Gradient fix-up (default "column_gs"): after u_qr moves by s, the rest of row q's gradient
  moves by s * H[r, :], so every later coordinate step in the row is an exact 1-D minimiser.
  "lemma2" is the literal reading of Lemma 2 (only g_qr changes; the row is updated from the
  start-of-step gradient).
* N modes generalise the 3-mode text with Khatri-Rao / Hadamard products over all k != n and
  modes visited 0..N-1 in order (Gauss-Seidel across modes, as Algorithm 1 does U, V, W).
* h_rr <= 0 (a zero column elsewhere), or h_rr numerically negligible, h_rr <= max(2^-40 max_j h_jj,
  2^-126) (a rank-one component whose other-mode factors have collapsed: its exact step g/h_rr
  grows without bound and leaves the FP32 range of the factors): s = 0 and z = 0.
* G of Eq. 9 is half the derivative of f in Eq. 6; the factor cancels in g/h.
* The objective sums over all cells (Eq. 7), so f = ||X||^2 - 2<X, M> + ||M||^2 with M the
  CP model; "fit" (not defined by the paper) is 1 - sqrt(max(f, 0)) / ||X||.
* Duplicate coordinates are summed (in FP32, in their input order) before anything else.
* The BF16-gather variant (not in the paper) is defined here as: each gathered factor value is
  the FP32 factor rounded to the nearest BF16 (ties to even); everything else is unchanged.
* FSaCD (Algorithm 2, ``FSaCDOracle``): the column gradient of Eq. colgrad carries Eq. 9's sign,
  g_r = (U H)_r - m_r; the column update of Eq. upur is Eq. 12's projected step,
  u_qr <- max(0, u_qr - g_qr/h_rr), taken on the selected elements only; "z_r > 0" of the first
  visit is elementwise; the choice between Eq. 24 and Eq. 27 compares ti = sum of z over all
  columns, so every column's z is formed before any element moves; the parallel columns all use
  the factor at the start of the mode step.

Pins (tests/test_oracle_pins.py) tie each function here to something other than itself:
explicit unfoldings and Khatri-Rao products, finite differences, the exact 1-D decrease, a HALS
sweep written separately, monotone objective, hand-computed selection tables.
"""

from __future__ import annotations

import numpy as np

__all__ = [
    "round_bf16",
    "coalesce",
    "csf_order",
    "csf_arrays",
    "mttkrp",
    "gram",
    "hadamard_of_grams",
    "curvatures",
    "lipschitz",
    "gradient",
    "projected_delta",
    "importance",
    "total_importance",
    "select",
    "update_rows",
    "norm_x_sq",
    "inner_x_model",
    "model_norm_sq",
    "objective",
    "fit_from_objective",
    "predict",
    "rmse",
    "pattern_distinctiveness",
    "SaCDOracle",
    "sttvp",
    "FSaCDOracle",
]


def round_bf16(a):
    """FP32 values rounded to the nearest BF16 (8-bit significand), ties to even; as FP64.

    BF16 keeps the upper 16 bits of the FP32 encoding: add 0x7FFF plus the lowest kept bit,
    then clear the low 16 bits (finite inputs only)."""
    x = np.ascontiguousarray(a, dtype=np.float32).view(np.uint32).astype(np.uint64)
    x = (x + 0x7FFF + ((x >> 16) & 1)) & 0xFFFF0000
    return x.astype(np.uint32).view(np.float32).astype(np.float64)


# ----------------------------------------------------------------------------------------
# Data structure: observed set Omega (symbol table) and its per-mode slices Omega^U_q etc.
# ----------------------------------------------------------------------------------------


def coalesce(dims, idx, vals):
    """Sort the nonzeros lexicographically by (i_0, ..., i_{N-1}) and sum repeated coordinates.

    Repeats are summed in FP32 in their input order (the paper has no repeated entries; the
    library accepts them and sums them). Returns (idx int64 (N, nnz'), vals float32 (nnz',)).
    """
    idx = np.asarray(idx, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float32)
    for n, d in enumerate(dims):
        if idx.shape[1] and (idx[n].min() < 0 or idx[n].max() >= d):
            raise ValueError(f"index out of range in mode {n}")
    # np.lexsort sorts by the LAST key first; it is stable, so repeats stay in input order.
    order = np.lexsort(tuple(idx[k] for k in range(len(dims) - 1, -1, -1)))
    sidx = idx[:, order]
    svals = vals[order]
    if sidx.shape[1] == 0:
        return sidx, svals
    new = np.ones(sidx.shape[1], dtype=bool)
    new[1:] = np.any(sidx[:, 1:] != sidx[:, :-1], axis=0)
    if new.all():
        return sidx, svals
    out_idx = sidx[:, new]
    heads = np.flatnonzero(new)
    ends = np.append(heads[1:], sidx.shape[1])
    out_vals = np.empty(heads.shape[0], dtype=np.float32)
    for t, (a, b) in enumerate(zip(heads, ends)):
        acc = np.float32(svals[a])
        for e in range(a + 1, b):  # sequential FP32 sum in input order
            acc = np.float32(acc + svals[e])
        out_vals[t] = acc
    return out_idx, out_vals


def csf_order(idx, n):
    """Order of the nonzeros for a mode-n slice structure: by i_n, then the other modes in
    ascending mode order (realises the slices Omega^{(n)}_q of the symbol table)."""
    idx = np.asarray(idx, dtype=np.int64)
    N = idx.shape[0]
    keys = [n] + [k for k in range(N) if k != n]
    return np.lexsort(tuple(idx[k] for k in reversed(keys)))


def csf_arrays(idx, vals, n):
    """The mode-n sorted arrays: row index per nonzero, the other modes' indices, values."""
    order = csf_order(idx, n)
    idx = np.asarray(idx, dtype=np.int64)
    others = [k for k in range(idx.shape[0]) if k != n]
    return (
        idx[n, order].astype(np.int32),
        idx[others][:, order].astype(np.int32),
        np.asarray(vals, dtype=np.float32)[order],
    )


# ----------------------------------------------------------------------------------------
# Per-mode primitives (Section 4.1)
# ----------------------------------------------------------------------------------------


def mttkrp(dims, idx, vals, factors, n):
    """M = X_(n) (Khatri-Rao of A_k, k != n), computed over the nonzeros (Eq. 9, first term;
    the column-wise form m_r = sum over the mode-n slice of x * prod_k a_k[i_k, r] in Sec. 4.4).

    Every nonzero adds x * (elementwise product of the other factors' rows) to row i_n of M.
    """
    idx = np.asarray(idx, dtype=np.int64)
    x = np.asarray(vals, dtype=np.float64)
    R = factors[0].shape[1]
    contrib = np.repeat(x[:, None], R, axis=1)
    for k in range(len(dims)):
        if k != n:
            contrib = contrib * np.asarray(factors[k], dtype=np.float64)[idx[k]]
    M = np.zeros((dims[n], R), dtype=np.float64)
    np.add.at(M, idx[n], contrib)
    return M


def gram(A):
    """A^T A in FP64 (the V^T V, W^T W terms of Eq. 10)."""
    A = np.asarray(A, dtype=np.float64)
    return A.T @ A


def hadamard_of_grams(factors, n):
    """H = Hadamard product of A_k^T A_k over k != n (Eq. 10; Eqs. for V and W in Sec. 4.3)."""
    R = factors[0].shape[1]
    H = np.ones((R, R), dtype=np.float64)
    for k, A in enumerate(factors):
        if k != n:
            H = H * gram(A)
    return H


H_REL_MIN = 2.0**-40  # h_rr below this share of the largest h_jj counts as zero
H_ABS_MIN = 2.0**-126  # ... and so does any h_rr without a normal FP32 reciprocal


def curvatures(H):
    """The h_rr that the coordinate steps use (Eq. 11-13, 15): the diagonal of H, with every entry
    <= max(H_REL_MIN * max_j h_jj, H_ABS_MIN) set to 0, so that such a column takes no step."""
    h = np.array(np.diag(np.asarray(H, dtype=np.float64)), copy=True)
    if h.size == 0:
        return h
    thr = max(H_REL_MIN * float(np.max(h)), H_ABS_MIN)
    h[h <= thr] = 0.0
    return h


def lipschitz(H, norm="fro"):
    """L = ||H|| (Algorithm 1; proof of Lemma 1). Frobenius by the symbol table's ||.||."""
    if norm == "fro":
        return float(np.sqrt(np.sum(H * H)))
    if norm == "spectral":
        return float(np.linalg.norm(H, 2))
    raise ValueError(norm)


def gradient(A, H, M):
    """G = A H - M (Eq. 9 with M the MTTKRP term; element form Eq. 14)."""
    return np.asarray(A, dtype=np.float64) @ H - M


def projected_delta(a, g, h):
    """Eq. 11 then Eq. 12: u_hat = g / h; s = max(0, u - u_hat) - u. s = 0 where h <= 0."""
    a = np.asarray(a, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    h = np.broadcast_to(np.asarray(h, dtype=np.float64), a.shape)
    s = np.zeros_like(a)
    ok = h > 0
    s[ok] = np.maximum(0.0, a[ok] - g[ok] / h[ok]) - a[ok]
    return s


def importance(g, s, L):
    """Lipschitz element importance z = -g s - (L/2) s^2 (Eq. 20)."""
    return -g * s - 0.5 * L * s * s


def total_importance(Z):
    """ti = sum over all elements of z (Eq. 25 / 26)."""
    return float(np.sum(Z))


def select(Z, Zprev, ti, tiprev, first):
    """Selection of Algorithm 1.

    First visit of the factor: z > 0. Later: sp = z^k - z^{k-1} (Eq. 24), or, if ti^k > ti^{k-1},
    sp = z^{k-1} - z^k (Eq. 27); the element is updated iff sp > 0.
    """
    if first:
        return Z > 0
    sp = (Zprev - Z) if ti > tiprev else (Z - Zprev)
    return sp > 0


def update_rows(A, G, H, sel, fixup="column_gs", h=None):
    """Nonnegative coordinate update of the selected elements (Eq. 11-13), columns in order.

    For r = 0..R-1 (Algorithm 1's column loop), every selected u_qr with h_rr > 0 moves by
    s = max(0, u_qr - g_qr/h_rr) - u_qr (Eq. 12) and u_qr += s (Eq. 13). ``h`` (default: the
    diagonal of H) gives the h_rr of the steps (``curvatures``); the fix-up uses H itself.
    Gradient fix-up: "column_gs" adds s * H[r, :] to row q's gradient (the exact change of
    g_q = a_q H - m_q), "lemma2" changes g_qr alone (Lemma 2).
    Returns (new A, number of elements that were selected).
    """
    A = np.array(A, dtype=np.float64, copy=True)
    g = np.array(G, dtype=np.float64, copy=True)
    R = A.shape[1]
    hd = np.diag(H) if h is None else np.asarray(h, dtype=np.float64)
    for r in range(R):
        hr = hd[r]
        if not hr > 0:
            continue
        rows = sel[:, r]
        s = np.zeros(A.shape[0])
        s[rows] = np.maximum(0.0, A[rows, r] - g[rows, r] / hr) - A[rows, r]
        A[:, r] += s
        if fixup == "column_gs":
            g += s[:, None] * H[r, :][None, :]
        elif fixup == "lemma2":
            g[:, r] += s * hr
        else:
            raise ValueError(fixup)
    return A, int(np.count_nonzero(sel))


# ----------------------------------------------------------------------------------------
# Objective (Eq. 6-8)
# ----------------------------------------------------------------------------------------


def norm_x_sq(vals):
    v = np.asarray(vals, dtype=np.float64)
    return float(np.sum(v * v))


def inner_x_model(idx, vals, factors):
    """<X, [[A]]> = sum over nonzeros of x * sum_r prod_k a_k[i_k, r] (Eq. 8 at observed cells)."""
    idx = np.asarray(idx, dtype=np.int64)
    R = factors[0].shape[1]
    p = np.ones((idx.shape[1], R), dtype=np.float64)
    for k, A in enumerate(factors):
        p = p * np.asarray(A, dtype=np.float64)[idx[k]]
    return float(np.sum(np.asarray(vals, dtype=np.float64) * p.sum(axis=1)))


def model_norm_sq(factors):
    """||[[A]]||^2 over all cells = sum_{r,s} prod_k (A_k^T A_k)[r, s]."""
    R = factors[0].shape[1]
    P = np.ones((R, R), dtype=np.float64)
    for A in factors:
        P = P * gram(A)
    return float(np.sum(P))


def objective(idx, vals, factors):
    """f = ||X - [[A]]||^2 summed over all cells (Eq. 6-7)."""
    return norm_x_sq(vals) - 2.0 * inner_x_model(idx, vals, factors) + model_norm_sq(factors)


def fit_from_objective(f, nx_sq):
    return 1.0 - np.sqrt(max(f, 0.0)) / np.sqrt(nx_sq) if nx_sq > 0 else 0.0


# ----------------------------------------------------------------------------------------
# Evaluation (Sec. 6.2)
# ----------------------------------------------------------------------------------------


def predict(idx, factors):
    """x_hat at the given coordinates: sum_r prod_k a_k[i_k, r] (Eq. 8)."""
    idx = np.asarray(idx, dtype=np.int64)
    R = factors[0].shape[1]
    p = np.ones((idx.shape[1], R), dtype=np.float64)
    for k, A in enumerate(factors):
        p = p * np.asarray(A, dtype=np.float64)[idx[k]]
    return p.sum(axis=1)


def rmse(idx, vals, factors):
    """RMSE over test entries, sqrt(sum (x - x_hat)^2 / n) (Eq. 30)."""
    v = np.asarray(vals, dtype=np.float64)
    if v.size == 0:
        return 0.0
    d = v - predict(idx, factors)
    return float(np.sqrt(np.sum(d * d) / v.size))


def pattern_distinctiveness(W):
    """PD of a factor (Eq. pd): the cosine similarity of columns i < r, averaged over the pairs
    (the paper reports one number per factor; the mean is the reading taken here). Columns of
    zero norm have no direction and are left out."""
    W = np.asarray(W, dtype=np.float64)
    R = W.shape[1]
    norms = np.sqrt(np.sum(W * W, axis=0))
    vals = []
    for i in range(R):
        for r in range(i + 1, R):
            if norms[i] > 0 and norms[r] > 0:
                vals.append(float(W[:, i] @ W[:, r]) / (norms[i] * norms[r]))
    return float(np.mean(vals)) if vals else 0.0


# ----------------------------------------------------------------------------------------
# Algorithm 1
# ----------------------------------------------------------------------------------------


class SaCDOracle:
    """SaCD state and steps (Algorithm 1), generalised to N modes.

    State per factor n: A[n] (FP64, from the FP32 initial values), z^{k-1} (Zprev[n]),
    ti^{k-1} (tiprev[n]) and whether the factor has been visited yet (first[n]).
    """

    def __init__(self, dims, idx, vals, init, *, lnorm="fro", fixup="column_gs", gather="fp32"):
        self.dims = [int(d) for d in dims]
        self.N = len(self.dims)
        self.idx, self.vals = coalesce(self.dims, idx, vals)
        self.A = [np.asarray(a, dtype=np.float64).copy() for a in init]
        self.R = self.A[0].shape[1]
        self.lnorm = lnorm
        self.fixup = fixup
        self.gather = gather  # "fp32": gathered factors as they are; "bf16": rounded to BF16
        self.Zprev = [np.zeros((d, self.R)) for d in self.dims]
        self.tiprev = [0.0] * self.N
        self.first = [True] * self.N
        self.nx_sq = norm_x_sq(self.vals)
        self.last = None  # taps of the last mode step

    def mode_step(self, n, mask=None):
        """One mode step of Algorithm 1 for factor n.

        ``mask`` (bool (I_n, R)), if given, replaces the selection (used to replay a selection
        taken elsewhere, so that the arithmetic alone can be compared).
        """
        A = self.A[n]
        if self.gather == "bf16":
            gathered = [round_bf16(F.astype(np.float32)) if k != n else F for k, F in enumerate(self.A)]
        else:
            gathered = self.A
        M = mttkrp(self.dims, self.idx, self.vals, gathered, n)  # Eq. 9, X_(n)(KRP)
        H = hadamard_of_grams(self.A, n)  # Eq. 10
        G = gradient(A, H, M)  # Eq. 9 / 14
        hd = curvatures(H)  # h_rr of the steps (negligible ones count as 0)
        h = hd[None, :]
        if self.lnorm == "gcd":
            L = h  # Eq. 18: h_rr in place of L
        else:
            L = lipschitz(H, self.lnorm)  # Algorithm 1: L = ||H||
        S = projected_delta(A, G, h)  # Eq. 11-12
        Z = importance(G, S, L)  # Eq. 20 (Eq. 18 with "gcd")
        ti = total_importance(Z)  # Eq. 25
        branch = None
        if mask is None:
            sel = select(Z, self.Zprev[n], ti, self.tiprev[n], self.first[n])
            branch = "first" if self.first[n] else ("eq27" if ti > self.tiprev[n] else "eq24")
        else:
            sel = np.asarray(mask, dtype=bool)
        Anew, nsel = update_rows(A, G, H, sel, self.fixup, hd)  # Eq. 13 (+ fix-up)
        self.last = dict(M=M, H=H, L=L, G=G, Z=Z, ti=ti, tiprev=self.tiprev[n], sel=sel, branch=branch,
                         first=self.first[n], Zprev=self.Zprev[n].copy(), Aold=A.copy())
        self.A[n] = Anew
        self.Zprev[n] = Z  # z^{k-1} <- z for every element
        self.tiprev[n] = ti
        self.first[n] = False
        return nsel

    def iterate(self, iters=1):
        for _ in range(iters):
            for n in range(self.N):
                self.mode_step(n)

    def objective(self):
        return objective(self.idx, self.vals, self.A)

    def fit(self):
        f = self.objective()
        return f, fit_from_objective(f, self.nx_sq)


# ----------------------------------------------------------------------------------------
# FSaCD (Section 4.4, Algorithm 2)
# ----------------------------------------------------------------------------------------


def sttvp(dims, idx, vals, factors, n, r):
    """Column r of the mode-n MTTKRP as a sparse tensor times vectors product (the column-wise
    m_r of FSaCD): m_r[q] = sum over the nonzeros with i_n = q of x times the product of the other
    factors' r-th entries at the nonzero's coordinates."""
    w = np.asarray(vals, dtype=np.float64).copy()
    for k in range(len(dims)):
        if k != n:
            w = w * np.asarray(factors[k], dtype=np.float64)[np.asarray(idx[k]), r]
    m = np.zeros(int(dims[n]))
    np.add.at(m, np.asarray(idx[n]), w)
    return m


class FSaCDOracle:
    """FSaCD (Algorithm 2), generalised to N modes, with the readings listed in the module header.

    Per mode step: H and L (Eq. 10, L = ||H||_F); for every column r, from the factor at the start
    of the step, m_r by sttvp, the column gradient, the column's projected deltas and importance
    (Eq. colgrad, Eq. 11-12, Eq. coleq); then ti (Eq. 25), the saturation test of every element
    (first visit: z > 0; else Eq. 24 or Eq. 27) and the update of the selected ones (Eq. 13).
    """

    def __init__(self, dims, idx, vals, init):
        self.dims = [int(d) for d in dims]
        self.N = len(self.dims)
        self.idx, self.vals = coalesce(self.dims, idx, vals)
        self.A = [np.asarray(a, dtype=np.float64).copy() for a in init]
        self.R = self.A[0].shape[1]
        self.Zprev = [np.zeros((d, self.R)) for d in self.dims]
        self.tiprev = [0.0] * self.N
        self.first = [True] * self.N

    def mode_step(self, n, mask=None):
        U = self.A[n]
        H = hadamard_of_grams(self.A, n)
        L = float(np.linalg.norm(H))
        h = curvatures(H)
        Z = np.zeros_like(U)
        S = np.zeros_like(U)
        for r in range(self.R):  # Algorithm 2's parallel loop over columns
            m_r = sttvp(self.dims, self.idx, self.vals, self.A, n, r)
            g_r = U @ H[:, r] - m_r
            if h[r] > 0:
                S[:, r] = np.maximum(0.0, U[:, r] - g_r / h[r]) - U[:, r]
            Z[:, r] = -g_r * S[:, r] - 0.5 * L * S[:, r] ** 2
        ti = float(Z.sum())
        if mask is not None:
            sel = np.asarray(mask, dtype=bool)
        elif self.first[n]:
            sel = Z > 0
        else:
            sp = self.Zprev[n] - Z if ti > self.tiprev[n] else Z - self.Zprev[n]
            sel = sp > 0
        self.A[n] = np.where(sel, U + S, U)
        self.Zprev[n] = Z
        self.tiprev[n] = ti
        self.first[n] = False
        return int(np.count_nonzero(sel))

    def iterate(self, iters=1):
        for _ in range(iters):
            for n in range(self.N):
                self.mode_step(n)
