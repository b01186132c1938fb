"""Pins for the FP64 oracle: each oracle function checked against something other than itself.

* MTTKRP: explicit mode-n unfolding times an explicit Khatri-Rao product (Eq. 3), dense.
* H: Hadamard of Grams equals (KRP)^T (KRP) (Eq. 10 against Eq. 3).
* G: central finite differences of f/2 evaluated on the dense reconstruction (Eq. 6-9).
* s: the exact constrained 1-D minimiser of the dense f along one coordinate (Eq. 11-12).
* z: with L replaced by h_rr, 2z is the exact decrease of the dense f (Eq. 16-18); with L, the
  closed-form shift -(L-h)/2 s^2 on top of it (Eq. 20).
* update: all elements selected with the Gauss-Seidel fix-up is one HALS sweep, written here
  separately from a dense MTTKRP.
* Algorithm 1: nonnegativity and monotone objective over many steps; a hand-worked 2x1x1
  rank-2 case (tests/golden) pins the selection branches.
* objective: against the dense sum of squared residuals (Eq. 7).
* CSF order / duplicate summation: against Python's sorted() and a dict.
"""

import itertools
import json
import os

import numpy as np
import pytest

from oracle import sacd_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")

# ---------------------------------------------------------------- independent brute force


def dense_from_coo(dims, idx, vals):
    X = np.zeros(dims)
    for e in range(len(vals)):
        X[tuple(int(idx[k][e]) for k in range(len(dims)))] += float(vals[e])
    return X


def unfold(X, n):
    """Mode-n matricization with the lower remaining modes varying fastest."""
    dims = X.shape
    others = [k for k in range(len(dims)) if k != n]
    ncols = int(np.prod([dims[k] for k in others]))
    Xn = np.zeros((dims[n], ncols))
    for cell in itertools.product(*[range(d) for d in dims]):
        col, stride = 0, 1
        for k in others:
            col += cell[k] * stride
            stride *= dims[k]
        Xn[cell[n], col] = X[cell]
    return Xn


def khatri_rao(mats):
    """Eq. 3: column r is the Kronecker product of the columns r, mats[0] the slowest."""
    R = mats[0].shape[1]
    cols = []
    for r in range(R):
        c = np.array([1.0])
        for A in mats:
            c = np.kron(c, A[:, r])
        cols.append(c)
    return np.stack(cols, axis=1)


def krp_for_mode(factors, n):
    # X_(n) pairs with A_{N-1} kr ... kr A_{n+1} kr A_{n-1} kr ... kr A_0 (A_0 fastest)
    return khatri_rao([factors[k] for k in range(len(factors) - 1, -1, -1) if k != n])


def reconstruct(factors):
    dims = [A.shape[0] for A in factors]
    R = factors[0].shape[1]
    Xh = np.zeros(dims)
    for r in range(R):
        t = np.array(1.0)
        for A in factors:
            t = np.multiply.outer(t, A[:, r])
        Xh += t
    return Xh


def dense_f(X, factors):
    return float(np.sum((X - reconstruct(factors)) ** 2))


def random_case(dims, R, nnz, seed):
    rng = np.random.default_rng(seed)
    cells = list(itertools.product(*[range(d) for d in dims]))
    pick = rng.choice(len(cells), size=nnz, replace=False)
    idx = np.array([cells[p] for p in pick], dtype=np.int64).T
    vals = rng.integers(1, 6, size=nnz).astype(np.float32)
    factors = [rng.random((d, R)) for d in dims]
    return idx, vals, factors


CASES = [((4, 5, 3), 3, 25, 1), ((3, 4, 2, 5), 4, 40, 2), ((6, 3, 4), 2, 30, 3)]

# ---------------------------------------------------------------- MTTKRP, H


@pytest.mark.parametrize("dims,R,nnz,seed", CASES)
def test_mttkrp_equals_unfolding_times_khatri_rao(dims, R, nnz, seed):
    idx, vals, F = random_case(dims, R, nnz, seed)
    X = dense_from_coo(dims, idx, vals)
    for n in range(len(dims)):
        ref = unfold(X, n) @ krp_for_mode(F, n)
        got = O.mttkrp(list(dims), idx, vals, F, n)
        np.testing.assert_allclose(got, ref, rtol=1e-13, atol=1e-12)


@pytest.mark.parametrize("dims,R,nnz,seed", CASES)
def test_hadamard_of_grams_equals_krp_gram(dims, R, nnz, seed):
    _, _, F = random_case(dims, R, nnz, seed)
    for n in range(len(dims)):
        K = krp_for_mode(F, n)
        np.testing.assert_allclose(O.hadamard_of_grams(F, n), K.T @ K, rtol=1e-13, atol=1e-12)


def test_lipschitz_norms():
    H = np.array([[3.0, 1.0], [1.0, 3.0]])
    assert O.lipschitz(H, "fro") == pytest.approx(np.sqrt(20.0), rel=1e-15)
    assert O.lipschitz(H, "spectral") == pytest.approx(4.0, rel=1e-14)  # eigenvalues 2 and 4


# ---------------------------------------------------------------- G, s, z


@pytest.mark.parametrize("dims,R,nnz,seed", CASES)
def test_gradient_is_half_derivative_of_dense_objective(dims, R, nnz, seed):
    idx, vals, F = random_case(dims, R, nnz, seed)
    X = dense_from_coo(dims, idx, vals)
    for n in range(len(dims)):
        M = O.mttkrp(list(dims), idx, vals, F, n)
        G = O.gradient(F[n], O.hadamard_of_grams(F, n), M)
        fd = np.zeros_like(G)
        d = 1e-3  # f is quadratic in A_n: central differences are exact up to rounding
        for q in range(dims[n]):
            for r in range(R):
                Fp = [A.copy() for A in F]
                Fm = [A.copy() for A in F]
                Fp[n][q, r] += d
                Fm[n][q, r] -= d
                fd[q, r] = (dense_f(X, Fp) - dense_f(X, Fm)) / (2 * d) / 2.0
        np.testing.assert_allclose(G, fd, rtol=1e-8, atol=1e-8 * np.abs(fd).max())


def _coordinate_quadratic(X, F, n, q, r):
    """Coefficients of t -> f(A + t e_qr) = c0 + c1 t + c2 t^2 from three dense evaluations."""
    vals = []
    for t in (-1.0, 0.0, 1.0):
        Ft = [A.copy() for A in F]
        Ft[n][q, r] += t
        vals.append(dense_f(X, Ft))
    fm, f0, fp = vals
    return f0, (fp - fm) / 2.0, (fp + fm) / 2.0 - f0


@pytest.mark.parametrize("dims,R,nnz,seed", CASES[:2])
def test_projected_delta_is_exact_constrained_minimiser(dims, R, nnz, seed):
    idx, vals, F = random_case(dims, R, nnz, seed)
    # make some rows overshoot (large other columns) so that the clamp at zero is exercised
    F[0][::2, 1:] = 30.0
    F[0][::2, 0] = 0.01
    F[0][1::3, 0] = 0.0
    X = dense_from_coo(dims, idx, vals)
    n = 0
    H = O.hadamard_of_grams(F, n)
    G = O.gradient(F[n], H, O.mttkrp(list(dims), idx, vals, F, n))
    S = O.projected_delta(F[n], G, np.diag(H)[None, :])
    clamped = 0
    for q in range(dims[n]):
        for r in range(R):
            c0, c1, c2 = _coordinate_quadratic(X, F, n, q, r)
            t_star = max(-F[n][q, r], -c1 / (2 * c2))  # minimiser of the parabola on u + t >= 0
            clamped += t_star == -F[n][q, r]
            assert S[q, r] == pytest.approx(t_star, rel=1e-9, abs=1e-10)
    assert clamped > 0


@pytest.mark.parametrize("dims,R,nnz,seed", CASES)
def test_importance_is_exact_decrease(dims, R, nnz, seed):
    idx, vals, F = random_case(dims, R, nnz, seed)
    X = dense_from_coo(dims, idx, vals)
    f0 = dense_f(X, F)
    for n in range(len(dims)):
        H = O.hadamard_of_grams(F, n)
        h = np.diag(H)
        L = O.lipschitz(H)
        G = O.gradient(F[n], H, O.mttkrp(list(dims), idx, vals, F, n))
        S = O.projected_delta(F[n], G, h[None, :])
        Zh = O.importance(G, S, h[None, :])  # GCD importance, Eq. 18
        ZL = O.importance(G, S, L)  # Lipschitz importance, Eq. 20
        for q in range(dims[n]):
            for r in range(R):
                Ft = [A.copy() for A in F]
                Ft[n][q, r] += S[q, r]
                dec = f0 - dense_f(X, Ft)
                assert 2 * Zh[q, r] == pytest.approx(dec, rel=1e-9, abs=1e-9 * f0)
                assert ZL[q, r] == pytest.approx(dec / 2 - (L - h[r]) / 2 * S[q, r] ** 2, rel=1e-9, abs=1e-9 * f0)


# ---------------------------------------------------------------- update = HALS when all selected


def hals_sweep(A, Mdense, H):
    """One HALS sweep (Cichocki-Phan): a_r <- max(0, a_r + (m_r - A h_r) / h_rr), r in order."""
    A = A.copy()
    for r in range(A.shape[1]):
        A[:, r] = np.maximum(0.0, A[:, r] + (Mdense[:, r] - A @ H[:, r]) / H[r, r])
    return A


@pytest.mark.parametrize("dims,R,nnz,seed", CASES)
def test_all_selected_gauss_seidel_equals_hals(dims, R, nnz, seed):
    idx, vals, F = random_case(dims, R, nnz, seed)
    X = dense_from_coo(dims, idx, vals)
    for n in range(len(dims)):
        Md = unfold(X, n) @ krp_for_mode(F, n)
        H = krp_for_mode(F, n).T @ krp_for_mode(F, n)
        G = O.gradient(F[n], O.hadamard_of_grams(F, n), O.mttkrp(list(dims), idx, vals, F, n))
        got, nsel = O.update_rows(F[n], G, O.hadamard_of_grams(F, n), np.ones_like(G, dtype=bool), "column_gs")
        np.testing.assert_allclose(got, hals_sweep(F[n], Md, H), rtol=1e-11, atol=1e-12)
        assert nsel == G.size


# ---------------------------------------------------------------- Algorithm 1 invariants


def sparse_case(dims, R, nnz, seed):
    rng = np.random.default_rng(seed)
    flat = rng.choice(int(np.prod(dims)), size=nnz, replace=False)
    idx = np.array(np.unravel_index(flat, dims), dtype=np.int64)
    vals = rng.integers(1, 6, size=nnz).astype(np.float32)
    init = [(rng.integers(0, 2**24, size=(d, R)) * 2.0**-24).astype(np.float32) for d in dims]
    return idx, vals, init


@pytest.mark.parametrize("dims,R", [((30, 20, 10), 5), ((12, 9, 7, 5), 4)])
def test_nonnegative_and_monotone_objective(dims, R):
    idx, vals, init = sparse_case(dims, R, 300, 7)
    o = O.SaCDOracle(dims, idx, vals, init)
    f_prev = o.objective()
    total_sel = 0
    branches = set()
    for k in range(8):
        for n in range(len(dims)):
            total_sel += o.mode_step(n)
            branches.add(o.last["branch"])
            assert all((A >= 0).all() for A in o.A)
            f = o.objective()
            assert f <= f_prev + 1e-12 * abs(f_prev)
            f_prev = f
    assert total_sel > 0
    assert "first" in branches and len(branches) >= 2


def test_objective_matches_dense():
    for dims, R, nnz, seed in CASES:
        idx, vals, F = random_case(dims, R, nnz, seed)
        X = dense_from_coo(dims, idx, vals)
        Xh = reconstruct(F)
        assert O.inner_x_model(idx, vals, F) == pytest.approx(float(np.sum(X * Xh)), rel=1e-13)
        assert O.model_norm_sq(F) == pytest.approx(float(np.sum(Xh * Xh)), rel=1e-13)
        assert O.objective(idx, vals, F) == pytest.approx(dense_f(X, F), rel=1e-11)


def test_hand_worked_selection_table():
    g = json.load(open(os.path.join(GOLDEN, "selection_2x1x1_r2.json")))
    init = [np.array(a, dtype=np.float32) for a in g["init"]]
    for fixup in ("column_gs", "lemma2"):
        o = O.SaCDOracle(g["dims"], np.array(g["idx"]), np.array(g["vals"], dtype=np.float32), init, fixup=fixup)
        assert o.objective() == pytest.approx(g["step1"]["f_before"], abs=1e-14)
        o.mode_step(0)
        t = o.last
        np.testing.assert_allclose(t["H"], g["H"], atol=0)
        assert t["L"] == pytest.approx(g["L"], abs=1e-15)
        np.testing.assert_allclose(t["M"], g["M"], atol=0)
        np.testing.assert_allclose(t["G"], g["step1"]["G"], atol=1e-15)
        np.testing.assert_allclose(t["Z"], g["step1"]["Z"], atol=1e-15)
        assert t["ti"] == pytest.approx(g["step1"]["ti"], abs=1e-15)
        assert t["branch"] == g["step1"]["branch"]
        np.testing.assert_array_equal(t["sel"], np.array(g["step1"]["sel"]))
        np.testing.assert_allclose(o.A[0], g["step1"]["U_" + fixup], atol=1e-15)
        assert o.objective() == pytest.approx(g["step1"]["f_" + fixup], abs=1e-14)
        o.mode_step(0)
        t = o.last
        s2 = g["step2_" + fixup]
        np.testing.assert_allclose(t["Z"], s2["Z"], atol=1e-15)
        assert t["ti"] == pytest.approx(s2["ti"], abs=1e-15)
        assert t["branch"] == s2["branch"]
        np.testing.assert_array_equal(t["sel"], np.array(s2["sel"]))
        np.testing.assert_allclose(o.A[0], s2["U"], atol=1e-15)


# ---------------------------------------------------------------- sort and duplicates


def test_csf_order_matches_python_sorted():
    idx, vals, _ = sparse_case((9, 7, 5, 4), 2, 200, 11)
    for n in range(4):
        keys = [n] + [k for k in range(4) if k != n]
        ref = sorted(range(idx.shape[1]), key=lambda e: tuple(int(idx[k][e]) for k in keys))
        np.testing.assert_array_equal(O.csf_order(idx, n), np.array(ref))


def test_coalesce_sums_repeats_in_input_order():
    rng = np.random.default_rng(5)
    idx = rng.integers(0, 3, size=(3, 60))
    vals = (rng.random(60) * 10).astype(np.float32)
    cidx, cvals = O.coalesce([3, 3, 3], idx, vals)
    acc = {}
    for e in range(60):
        key = tuple(int(idx[k][e]) for k in range(3))
        acc[key] = np.float32(acc.get(key, np.float32(0.0)) + vals[e]) if key in acc else np.float32(vals[e])
    keys = sorted(acc)
    np.testing.assert_array_equal(cidx.T, np.array(keys))
    np.testing.assert_array_equal(cvals, np.array([acc[k] for k in keys], dtype=np.float32))


# ---------------------------------------------------------------- the pins catch plausible mistakes


def test_pins_catch_planted_mistakes(monkeypatch):
    """Plant plausible mistakes in the oracle (CPU only) and check that a pin fails."""
    dims, R, nnz, seed = CASES[0]

    def mttkrp_dropped_value(d, i, v, F, n):
        return O.__dict__["_orig_mttkrp"](d, i, np.ones_like(v), F, n)

    O._orig_mttkrp = O.mttkrp
    with monkeypatch.context() as m:
        m.setattr(O, "mttkrp", mttkrp_dropped_value)
        with pytest.raises(AssertionError):
            test_mttkrp_equals_unfolding_times_khatri_rao(dims, R, nnz, seed)
    with monkeypatch.context() as m:
        m.setattr(O, "gradient", lambda A, H, M: M - A @ H)  # sign flipped
        with pytest.raises(AssertionError):
            test_gradient_is_half_derivative_of_dense_objective(dims, R, nnz, seed)
    with monkeypatch.context() as m:
        m.setattr(O, "importance", lambda g, s, L: -g * s + 0.5 * L * s * s)  # wrong sign of the L term
        with pytest.raises(AssertionError):
            test_importance_is_exact_decrease(dims, R, nnz, seed)
    with monkeypatch.context() as m:
        m.setattr(O, "hadamard_of_grams", lambda F, n: np.prod([O.gram(A) for k, A in enumerate(F) if k != n], axis=0).T @ np.eye(R) * 1.0001)
        with pytest.raises(AssertionError):
            test_hadamard_of_grams_equals_krp_gram(dims, R, nnz, seed)
    with monkeypatch.context() as m:
        m.setattr(O, "select", lambda Z, Zp, ti, tip, first: (Z > 0) if first else ((Z - Zp) if ti > tip else (Zp - Z)) > 0)
        with pytest.raises(AssertionError):
            test_hand_worked_selection_table()
    del O._orig_mttkrp


def test_round_bf16_against_torch_and_hand_values():
    torch = pytest.importorskip("torch")
    # hand values: 1 + 2^-8 is a tie between 1 and 1 + 2^-7 -> even (1); 1 + 3*2^-8 -> 1 + 2^-6
    hand = np.array([1.0, 1.0 + 2**-8, 1.0 + 3 * 2**-8, 1.0 + 2**-8 + 2**-20, 0.0, 3.0e-39], np.float32)
    want = np.array([1.0, 1.0, 1.0 + 2**-6, 1.0 + 2**-7, 0.0, np.float32(3.0e-39)], np.float64)
    got = O.round_bf16(hand)
    np.testing.assert_array_equal(got[:5], want[:5])
    rng = np.random.default_rng(3)
    x = (rng.random(100_000) * 10.0 ** rng.integers(-8, 8, 100_000)).astype(np.float32)
    ref = torch.from_numpy(x).bfloat16().float().numpy().astype(np.float64)
    np.testing.assert_array_equal(O.round_bf16(x), ref)


def test_rmse_against_dense_reconstruction():
    dims, R, nnz, seed = CASES[1]
    idx, vals, F = random_case(dims, R, nnz, seed)
    Xh = reconstruct(F)
    want = np.sqrt(np.mean([(float(vals[e]) - Xh[tuple(idx[:, e])]) ** 2 for e in range(nnz)]))
    assert O.rmse(idx, vals, F) == pytest.approx(want, rel=1e-13)
    assert O.rmse(np.zeros((4, 0), np.int64), np.zeros(0), F) == 0.0


def test_pattern_distinctiveness_special_cases():
    scipy = pytest.importorskip("scipy.spatial.distance")
    I = np.eye(6)[:, :4]  # orthogonal columns
    assert O.pattern_distinctiveness(I) == 0.0
    same = np.ones((5, 3))  # identical columns
    assert O.pattern_distinctiveness(same) == pytest.approx(1.0, abs=1e-15)
    rng = np.random.default_rng(2)
    W = rng.random((40, 5))
    pairs = [1 - scipy.cosine(W[:, i], W[:, r]) for i in range(5) for r in range(i + 1, 5)]
    assert O.pattern_distinctiveness(W) == pytest.approx(np.mean(pairs), rel=1e-13)
    W[:, 2] = 0  # a zero column has no direction
    pairs = [1 - scipy.cosine(W[:, i], W[:, r]) for i in (0, 1, 3, 4) for r in (0, 1, 3, 4) if i < r]
    assert O.pattern_distinctiveness(W) == pytest.approx(np.mean(pairs), rel=1e-13)


def test_negligible_curvature_takes_no_step():
    """Reading of h_rr <= 0 extended to a numerically negligible h_rr (<= max(2^-40 max_j h_jj,
    2^-126)): such a column takes no step and has z = 0. The case: column 2 of the other factors
    shrunk by 1e-25, so h_22 ~ 1e-100; the exact constrained minimiser along that coordinate (from
    the dense objective) is then far outside the FP32 range, while the other columns still take
    their exact 1-D steps."""
    dims, R = (4, 5, 3), 3
    idx, vals, F = random_case(dims, R, 25, 5)
    F[1][:, 2] *= 1e-25
    F[2][:, 2] *= 1e-25
    X = dense_from_coo(dims, idx, vals)
    n = 0
    H = O.hadamard_of_grams(F, n)
    h = O.curvatures(H)
    assert H[2, 2] > 0 and h[2] == 0.0
    np.testing.assert_array_equal(h[:2], np.diag(H)[:2])
    # the exact step that the reading declines: f(A + t e_q2) = c0 + c1 t + c2 t^2 with c2 the
    # squared norm of KRP column 2 and c1 = 2 (a_q K^T K - X_(n) K)_q2 (explicit unfolding and
    # Khatri-Rao product); |t*| is beyond the largest FP32 value in some row
    K = krp_for_mode(F, n)
    Xn = unfold(X, n)
    c2 = float(K[:, 2] @ K[:, 2])
    tstar = []
    for q in range(dims[n]):
        c1 = 2.0 * (float(F[n][q] @ (K.T @ K[:, 2])) - float(Xn[q] @ K[:, 2]))
        tstar.append(max(-F[n][q, 2], -c1 / (2 * c2)))
    assert 0 < c2 < 1e-90 and max(abs(t) for t in tstar) > 3.4e38
    # the oracle's mode step: column 2 unchanged with z = 0; columns 0 and 1 as with the raw h
    o = O.SaCDOracle(dims, idx, vals, [a.astype(np.float32) for a in F])
    o.A = [a.copy() for a in F]
    o.mode_step(n, mask=np.ones((dims[n], R), dtype=bool))
    np.testing.assert_array_equal(o.A[n][:, 2], F[n][:, 2])
    assert (o.last["Z"][:, 2] == 0).all()
    G = O.gradient(F[n], H, O.mttkrp(list(dims), idx, vals, F, n))
    S = O.projected_delta(F[n], G, np.diag(H)[None, :])
    np.testing.assert_allclose(o.A[n][:, 0], F[n][:, 0] + S[:, 0], rtol=1e-12, atol=1e-14)
    # the two thresholds, at and just above them
    assert list(O.curvatures(np.diag([1.0, 2.0**-40, 2.0**-40 * 1.0001]))) == [1.0, 0.0, 2.0**-40 * 1.0001]
    assert list(O.curvatures(np.diag([1e-39, 2.0**-126, 2.0**-125]))) == [0.0, 0.0, 2.0**-125]


@pytest.mark.parametrize("dims,R,nnz,seed", [((30, 20, 10), 5, 400, 2), ((12, 9, 7, 5), 4, 300, 3)])
def test_sttvp_columns_equal_the_mttkrp(dims, R, nnz, seed):
    """FSaCD's column-wise MTTKRP (sttvp) against the MTTKRP, itself pinned against the explicit
    unfolding times the Khatri-Rao product."""
    idx, vals, F = random_case(dims, R, nnz, seed)
    cidx, cvals = O.coalesce(dims, idx, vals)
    for n in range(len(dims)):
        M = O.mttkrp(list(dims), cidx, cvals, F, n)
        for r in range(R):
            np.testing.assert_allclose(O.sttvp(dims, cidx, cvals, F, n, r), M[:, r], rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("dims,R,nnz,seed", [((30, 20, 10), 5, 400, 4), ((12, 9, 7, 5), 4, 300, 5)])
def test_fsacd_equals_sacd_with_lemma2_updates(dims, R, nnz, seed):
    """Algorithm 2 (columns in parallel from the start-of-step factor) takes the same steps as
    Algorithm 1 with the Lemma 2 reading (each selected element moves from the start-of-step
    gradient), over several iterations and every branch of the selection."""
    idx, vals, init = random_case(dims, R, nnz, seed)
    a = O.SaCDOracle(dims, idx, vals, init, fixup="lemma2")
    b = O.FSaCDOracle(dims, idx, vals, init)
    branches = set()
    for it in range(6):
        for n in range(len(dims)):
            na = a.mode_step(n)
            nb = b.mode_step(n)
            branches.add(a.last["branch"])
            assert na == nb
            np.testing.assert_allclose(b.A[n], a.A[n], rtol=1e-12, atol=1e-14)
            np.testing.assert_allclose(b.Zprev[n], a.Zprev[n], rtol=1e-10, atol=1e-14)
    assert branches == {"first", "eq24", "eq27"}
