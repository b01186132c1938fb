"""Parity of the CUDA path (through the C ABI) with the FP64 oracle, on seeded inputs.

Tolerances (written here, from the stated targets):
* CSF sort, repeat summation: bit-exact.
* MTTKRP: relative Frobenius error <= 1e-5 (FP32 gathers), <= 1e-2 (BF16 gathers).
* Gram: <= 1e-10 relative (compensated FP32 products/sums at ranks up to 16, an exact BF16 split
  on the tensor cores at padded ranks 32 and 64; FP64 result), and every entry within
  1e-12 sqrt(G_jj G_kk).
* G: <= 1e-5 relative to ||M||_F + ||A H||_F (avoids cancellation blow-up).
* one mode step from identical factors, with the selection fixed on both sides (the oracle
  replays the GPU's mask): factor after the step <= 1e-5 relative; z <= 1e-5 of max |z|.
* free selection: every element where the GPU and the oracle disagree must sit at the decision
  boundary, |sp_oracle| <= 1e-5 max|z| (or the ti comparison is within 1e-6 sum|z|).
* final fit after K iterations: |delta fit| <= 1e-4 (FP32). BF16 gathers: the mode step matches
  the oracle's BF16-gather definition within 1e-5; each of 30 iterations, from the GPU's state
  with its selection replayed, ends within 1e-3 of the oracle's fit; the free 30-iteration
  trajectory within 5e-3 (twice the spread of two oracle runs that differ only by FP32 rounding
  of the factors, see the test).
* objective at identical factors: 2e-6 of 2<X, model> (FP32 MTTKRP behind the cross term) plus
  1e-9 of ||model||^2 (FP64 Grams), in both precisions.
"""

import json
import os

import numpy as np
import pytest

from oracle import sacd_oracle as O
from paper_2003_03572_gb300 import sacd as S
from paper_2003_03572_gb300 import synth

from fp32_bounds import z_fp32_bound

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def relerr(a, b):
    nb = np.linalg.norm(b)
    return float(np.linalg.norm(np.asarray(a, np.float64) - b) / (nb if nb > 0 else 1.0))


def assert_elementwise(got, ref, tol, scale_rows=None):
    """|got - ref| <= tol (|ref| + s_q) for every element of row q, s_q = max |ref| of the row (or the
    given per-row scale), so that a wrong value in a light row cannot hide under heavy rows."""
    got = np.asarray(got, np.float64)
    ref = np.asarray(ref, np.float64)
    s = np.abs(ref).max(axis=1, keepdims=True) if scale_rows is None else np.asarray(scale_rows)[:, None]
    bad = np.abs(got - ref) > tol * (np.abs(ref) + s)
    assert not bad.any(), f"{int(bad.sum())} elements off, first at {np.argwhere(bad)[0]}"


def assert_rowwise(got, ref, tol, floor_rows):
    """Per row: ||got_q - ref_q|| <= tol max(||ref_q||, floor_q)."""
    d = np.linalg.norm(np.asarray(got, np.float64) - ref, axis=1)
    s = np.maximum(np.linalg.norm(ref, axis=1), floor_rows)
    bad = d > tol * s
    assert not bad.any(), f"{int(bad.sum())} rows off, first {np.flatnonzero(bad)[0]}"


# dims, nnz, dist, zipf s, rank: several tiles per mode, a ragged tail, hot rows split across
# many tiles (Zipf), N = 3 and 4, ranks that pad (5, 24) and the widest gathered rows (64).
CASES = [
    ((100, 100, 100), 10_000, "uniform", 0.0, 5),
    ((600, 400, 50), 30_000, "zipf", 1.1, 32),
    ((300, 200, 40, 20), 20_000, "zipf", 1.2, 16),
    ((257, 129, 65), 7_777, "zipf", 1.1, 64),
    ((50, 40, 30), 3_001, "uniform", 0.0, 1),
    ((1000, 30, 20), 20_000, "zipf", 1.3, 8),
    ((333, 222, 111), 12_345, "zipf", 1.05, 24),
]


def make_case(dims, nnz, dist, s, R, seed=11, dup=0):
    idx, vals = synth.sparse_tensor(dims, nnz, dist=dist, zipf_s=s, seed=seed)
    if dup:
        rng = np.random.default_rng(seed)
        pick = rng.integers(0, nnz, size=dup)
        idx = np.concatenate([idx, idx[:, pick]], axis=1)
        vals = np.concatenate([vals, (rng.integers(1, 6, size=dup)).astype(np.float32)])
        perm = rng.permutation(idx.shape[1])
        idx, vals = np.ascontiguousarray(idx[:, perm]), vals[perm]
    init = synth.init_factors(dims, R, seed)
    return idx, vals, init


def ids(c):
    return "x".join(map(str, c[0])) + f"-nnz{c[1]}-r{c[4]}"


@pytest.mark.parametrize("case", CASES, ids=ids)
def test_csf_sort_and_repeats_bit_exact(case):
    dims, nnz, dist, s, R = case
    idx, vals, init = make_case(dims, nnz, dist, s, R, dup=nnz // 10)
    cidx, cvals = O.coalesce(dims, idx, vals)
    with S.SaCD(dims, idx, vals, R, init) as g:
        assert g.info["nnz"] == cidx.shape[1]
        assert g.info["norm_x_sq"] == pytest.approx(O.norm_x_sq(cvals), rel=1e-14)
        for n in range(len(dims)):
            row, other, v = O.csf_arrays(cidx, cvals, n)
            np.testing.assert_array_equal(g.tap("CSF_ROW", n), row)
            np.testing.assert_array_equal(g.tap("CSF_IDX", n), other)
            np.testing.assert_array_equal(g.tap("CSF_VAL", n), v)


@pytest.mark.parametrize("case", CASES, ids=ids)
def test_mttkrp_gram_and_mode_step_replay(case):
    dims, nnz, dist, s, R = case
    idx, vals, init = make_case(dims, nnz, dist, s, R)
    cidx, cvals = O.coalesce(dims, idx, vals)
    with S.SaCD(dims, idx, vals, R, init) as g:
        g.set_debug(True)
        # initial Grams
        for n in range(len(dims)):
            assert relerr(g.tap("GRAM", n), O.gram(init[n])) <= 1e-10
        o = O.SaCDOracle(dims, idx, vals, init)
        for it in range(2):
            for n in range(len(dims)):
                F = g.factors()
                zprev = g.tap("ZPREV", n)
                st = g.tap("STATE", n)
                nsel = g.mode_step(n)
                # oracle from the same factors and importance state, GPU's selection replayed
                o.A = [f.astype(np.float64) for f in F]
                o.Zprev[n] = zprev.astype(np.float64)
                o.tiprev[n] = st[0]
                o.first[n] = st[1] != 0
                mask = g.tap("MASK", n, last_mode=n).astype(bool)
                o.mode_step(n, mask=mask)
                t = o.last
                Mg = g.tap("M", n)
                assert relerr(Mg, t["M"]) <= 1e-5
                assert_elementwise(Mg, t["M"], 1e-5)
                H = t["H"]
                assert relerr(g.tap("H", n, last_mode=n), H) <= 1e-10
                Gg = g.tap("G", n, last_mode=n)
                AH = F[n].astype(np.float64) @ H
                den = np.linalg.norm(t["M"]) + np.linalg.norm(AH)
                assert np.linalg.norm(Gg - t["G"]) / den <= 1e-5
                assert_elementwise(Gg, t["G"], 1e-5, np.abs(t["M"]).max(axis=1) + np.abs(AH).max(axis=1))
                zg = g.tap("ZPREV", n)
                zs = max(np.abs(t["Z"]).max(), 1e-30)
                # 1e-5 of max |z|, widened per element by the FP32 evaluation bound of Eq. 11-12, 20
                assert (np.abs(zg - t["Z"]) <= 1e-5 * zs + z_fp32_bound(F[n], t)).all()
                An = g.factor(n)
                assert (An >= 0).all()
                assert relerr(An, o.A[n]) <= 1e-5
                assert_rowwise(An, o.A[n], 1e-5, np.linalg.norm(F[n].astype(np.float64), axis=1))
                assert nsel == int(mask.sum())
                stn = g.tap("STATE", n)
                assert stn[1] == 0.0
                assert stn[2] == pytest.approx(t["ti"], rel=1e-4, abs=1e-6 * np.abs(t["Z"]).sum())
                assert relerr(g.tap("GRAM", n), O.gram(An)) <= 1e-10
                # free selection: disagreements only at the decision boundary
                own = O.select(t["Z"], t["Zprev"], t["ti"], t["tiprev"], t["first"])
                dis = own != mask
                if dis.any():
                    if t["first"]:
                        sp = t["Z"]
                    else:
                        sp = (t["Zprev"] - t["Z"]) if t["ti"] > t["tiprev"] else (t["Z"] - t["Zprev"])
                    ti_close = abs(t["ti"] - t["tiprev"]) <= 1e-6 * np.abs(t["Z"]).sum()
                    zb = z_fp32_bound(F[n], t)
                    assert ti_close or (np.abs(sp[dis]) <= 1e-5 * zs + zb[dis]).all()


@pytest.mark.parametrize("R", [64, 32, 24, 40], ids=lambda r: f"r{r}")
def test_gram_on_tensor_cores_many_blocks(R):
    """Initial Grams of a 300,000-row mode: every block spans several read-back periods of the
    tensor-core Gram, the last block is ragged, and the factor has a column scaled by 2^-30, rows
    a million times larger than the rest in another column, and an all-zero column."""
    dims = (300_000, 300, 40)
    idx, vals = synth.sparse_tensor(dims, 20_000, dist="zipf", zipf_s=1.1, seed=3)
    rng = np.random.default_rng(4)
    init = synth.init_factors(dims, R, 4)
    A0 = (rng.random((dims[0], R)) ** 3).astype(np.float32)
    A0[:, 1] *= np.float32(2.0**-30)
    A0[::997, 2] *= np.float32(1e6)
    A0[:, R - 1] = 0.0
    init[0] = A0
    with S.SaCD(dims, idx, vals, R, init) as g:
        for n in range(len(dims)):
            ref = O.gram(init[n])
            got = g.tap("GRAM", n)
            assert np.isfinite(got).all()
            assert relerr(got, ref) <= 1e-10
            d = np.sqrt(np.outer(np.diag(ref), np.diag(ref)))
            assert (np.abs(got - ref) <= 1e-12 * d + 1e-300).all()
            assert np.array_equal(got, got.T)


@pytest.mark.parametrize("lnorm,fixup", [(S.SACD_LNORM_SPECTRAL, 0), (S.SACD_LNORM_GCD, 0), (0, S.SACD_FIXUP_LEMMA2)])
def test_variants_replay(lnorm, fixup):
    dims, nnz, dist, s, R = CASES[1]
    idx, vals, init = make_case(dims, nnz, dist, s, R)
    names = {0: "fro", 1: "spectral", 2: "gcd"}
    with S.SaCD(dims, idx, vals, R, init, lnorm=lnorm, fixup=fixup) as g:
        g.set_debug(True)
        o = O.SaCDOracle(dims, idx, vals, init, lnorm=names[lnorm], fixup=["column_gs", "lemma2"][fixup])
        for it in range(2):
            for n in range(len(dims)):
                F = g.factors()
                zprev = g.tap("ZPREV", n)
                st = g.tap("STATE", n)
                g.mode_step(n)
                o.A = [f.astype(np.float64) for f in F]
                o.Zprev[n] = zprev.astype(np.float64)
                o.tiprev[n] = st[0]
                o.first[n] = st[1] != 0
                o.mode_step(n, mask=g.tap("MASK", n, last_mode=n).astype(bool))
                t = o.last
                if lnorm != 2:
                    assert g.tap("STATE", n)[4] == pytest.approx(t["L"], rel=1e-9)
                zs = max(np.abs(t["Z"]).max(), 1e-30)
                assert (np.abs(g.tap("ZPREV", n) - t["Z"]) <= 1e-5 * zs + z_fp32_bound(F[n], t)).all()
                assert relerr(g.factor(n), o.A[n]) <= 1e-5


def test_fsacd_on_gpu_lemma2_path():
    """FSaCD (Algorithm 2) runs on the GPU as the Lemma 2 update: every mode step of the GPU's
    Lemma 2 path matches the FSaCD oracle (its column-wise sttvp, gradient, importance and
    update), from the GPU's factors and state, with the GPU's selection replayed: z within the
    FP32 bound, the factor within 1e-5."""
    dims, nnz, dist, s, R = CASES[2]
    idx, vals, init = make_case(dims, nnz, dist, s, R)
    with S.SaCD(dims, idx, vals, R, init, fixup=S.SACD_FIXUP_LEMMA2) as g:
        g.set_debug(True)
        o = O.FSaCDOracle(dims, idx, vals, init)
        ref = O.SaCDOracle(dims, idx, vals, init, fixup="lemma2")  # for the FP32 bound of z only
        for it in range(3):
            for n in range(len(dims)):
                F = g.factors()
                zprev = g.tap("ZPREV", n)
                st = g.tap("STATE", n)
                g.mode_step(n)
                for oo in (o, ref):
                    oo.A = [f.astype(np.float64) for f in F]
                    oo.Zprev[n] = zprev.astype(np.float64)
                    oo.tiprev[n] = st[0]
                    oo.first[n] = st[1] != 0
                mask = g.tap("MASK", n, last_mode=n).astype(bool)
                assert o.mode_step(n, mask=mask) == int(mask.sum())
                ref.mode_step(n, mask=mask)
                Zo = o.Zprev[n]
                zs = max(np.abs(Zo).max(), 1e-30)
                assert (np.abs(g.tap("ZPREV", n) - Zo) <= 1e-5 * zs + z_fp32_bound(F[n], ref.last)).all()
                assert relerr(g.factor(n), o.A[n]) <= 1e-5
                assert_rowwise(g.factor(n), o.A[n], 1e-5, np.linalg.norm(F[n].astype(np.float64), axis=1))


def test_hand_worked_case_on_gpu():
    gd = json.load(open(os.path.join(GOLDEN, "selection_2x1x1_r2.json")))
    init = [np.array(a, dtype=np.float32) for a in gd["init"]]
    for fixup, key in ((0, "column_gs"), (1, "lemma2")):
        with S.SaCD(gd["dims"], np.array(gd["idx"], np.int32), np.array(gd["vals"], np.float32), 2, init,
                    fixup=fixup) as g:
            g.set_debug(True)
            g.mode_step(0)
            np.testing.assert_allclose(g.tap("M", 0), gd["M"], atol=1e-6)
            np.testing.assert_allclose(g.tap("H", 0, last_mode=0), gd["H"], atol=0)
            np.testing.assert_allclose(g.tap("ZPREV", 0), gd["step1"]["Z"], atol=1e-6)
            np.testing.assert_array_equal(g.tap("MASK", 0, last_mode=0).astype(bool), np.array(gd["step1"]["sel"]))
            np.testing.assert_allclose(g.factor(0), gd["step1"]["U_" + key], atol=1e-6)
            st = g.tap("STATE", 0)
            assert st[4] == pytest.approx(gd["L"])
            assert st[2] == pytest.approx(gd["step1"]["ti"], abs=1e-6)
            g.mode_step(0)
            s2 = gd["step2_" + key]
            st = g.tap("STATE", 0)
            assert st[3] == {"eq24": 1.0, "eq27": 2.0}[s2["branch"]]
            np.testing.assert_array_equal(g.tap("MASK", 0, last_mode=0).astype(bool), np.array(s2["sel"]))
            np.testing.assert_allclose(g.factor(0), s2["U"], atol=1e-6)


@pytest.mark.parametrize("case", [CASES[0], CASES[2], CASES[5]], ids=ids)
def test_iterate_fit_matches_oracle(case):
    dims, nnz, dist, s, R = case
    idx, vals, init = make_case(dims, nnz, dist, s, R)
    K = 20
    with S.SaCD(dims, idx, vals, R, init) as g:
        o = O.SaCDOracle(dims, idx, vals, init)
        obj0, fit0 = g.fit()
        f0, ft0 = o.fit()
        assert obj0 == pytest.approx(f0, rel=1e-6)
        g.iterate(K)
        o.iterate(K)
        obj, fit = g.fit()
        fo, fito = o.fit()
        assert abs(fit - fito) <= 1e-4, (fit, fito)
        assert all((A >= 0).all() for A in g.factors())


def test_graph_iterate_equals_mode_steps_and_is_deterministic():
    dims, nnz, dist, s, R = CASES[1]
    idx, vals, init = make_case(dims, nnz, dist, s, R)
    with S.SaCD(dims, idx, vals, R, init) as a, S.SaCD(dims, idx, vals, R, init) as b:
        a.iterate(3)
        for _ in range(3):
            for n in range(3):
                b.mode_step(n, want_count=False)
        for n in range(3):
            np.testing.assert_array_equal(a.factor(n), b.factor(n))
        assert a.fit() == b.fit()


def resync(o, g, n_modes):
    """Give the oracle the GPU's state: factors, z^{k-1}, ti^{k-1} and first-visit flags."""
    o.A = [f.astype(np.float64) for f in g.factors()]
    for n in range(n_modes):
        o.Zprev[n] = g.tap("ZPREV", n).astype(np.float64)
        st = g.tap("STATE", n)
        o.tiprev[n] = st[0]
        o.first[n] = st[1] != 0


def test_bf16_gather_mode():
    dims, nnz, dist, s, R = CASES[1]
    idx, vals, init = make_case(dims, nnz, dist, s, R)
    cidx, cvals = O.coalesce(dims, idx, vals)
    with S.SaCD(dims, idx, vals, R, init, precision=S.SACD_BF16_GATHER) as g:
        g.set_debug(True)
        ob = O.SaCDOracle(dims, idx, vals, init, gather="bf16")
        for it in range(2):
            for n in range(3):
                F = g.factors()
                zprev = g.tap("ZPREV", n)
                st = g.tap("STATE", n)
                g.mode_step(n)
                assert relerr(g.tap("M", n), O.mttkrp(list(dims), cidx, cvals, F, n)) <= 1e-2
                # the oracle's definition of the BF16-gather variant, selection replayed
                ob.A = [f.astype(np.float64) for f in F]
                ob.Zprev[n] = zprev.astype(np.float64)
                ob.tiprev[n] = st[0]
                ob.first[n] = st[1] != 0
                ob.mode_step(n, mask=g.tap("MASK", n, last_mode=n).astype(bool))
                assert relerr(g.tap("M", n), ob.last["M"]) <= 1e-5
                Mref = ob.last["M"]
                rowmax = np.abs(Mref).max(axis=1, keepdims=True)
                assert (np.abs(g.tap("M", n) - Mref) <= 1e-5 * (np.abs(Mref) + rowmax)).all()
                assert relerr(g.factor(n), ob.A[n]) <= 1e-5
    # 30 iterations, each one checked against an iteration of the oracle's BF16-gather definition
    # from the GPU's state at its start (selection replayed): fit within 1e-3 (the stated bound;
    # observed ~1e-7), factors within 1e-4.
    with S.SaCD(dims, idx, vals, R, init, precision=S.SACD_BF16_GATHER) as g:
        g.set_debug(True)
        ob = O.SaCDOracle(dims, idx, vals, init, gather="bf16")
        worst = 0.0
        for it in range(30):
            resync(ob, g, 3)
            for n in range(3):
                g.mode_step(n, want_count=False)
                ob.mode_step(n, mask=g.tap("MASK", n, last_mode=n).astype(bool))
            worst = max(worst, abs(g.fit()[1] - ob.fit()[1]))
            for n in range(3):
                assert relerr(g.factor(n), ob.A[n]) <= 1e-4
        print(f"bf16 iteration-by-iteration: worst |dfit| {worst:.3e}")
        assert worst <= 1e-3
    # The free trajectory (each side its own selection, 30 iterations). With identical selections
    # an FP32-gather run drifts from the oracle by up to 4e-4 of each factor's largest entry over
    # 30 iterations (FP32 step errors accumulating) while its fit agrees to 4e-7; with BF16 gathers
    # that drift flips BF16 codes (a gathered value moves by one BF16 ulp, 2^-8 relative, whenever
    # the two states straddle a rounding boundary: 6 codes in the first iteration, 1,807 by the
    # sixth), and Eq. 24/27 are discontinuous, so BF16 trajectories of equal definition separate:
    # two FP64 oracle runs of this case that differ only in rounding the factors to FP32 after
    # each step end 1.1e-3 to 2.5e-3 apart. The GPU's free trajectory is held to twice that spread.
    with S.SaCD(dims, idx, vals, R, init, precision=S.SACD_BF16_GATHER) as g:
        ob = O.SaCDOracle(dims, idx, vals, init, gather="bf16")
        g.iterate(30)
        ob.iterate(30)
        dfit = abs(g.fit()[1] - ob.fit()[1])
        print(f"bf16 free trajectory: |dfit| {dfit:.3e}")
        assert dfit <= 5e-3


DUAL_CASES = [CASES[1], CASES[3], ((300, 200, 40, 20), 20_000, "zipf", 1.2, 32), CASES[2]]


@pytest.mark.parametrize("case", DUAL_CASES, ids=ids)
def test_bf16_objective_pass_feeds_the_next_step(case):
    """BF16 gathers: when the objective's mode is mode 0, its FP32-gather MTTKRP also forms mode 0's
    BF16-gather MTTKRP of the next step in the same pass. An objective after every iteration (graph
    path) or after every eager iteration gives factors bit for bit equal to no objective at all;
    the objective meets its bound at identical factors; a factor changed after the objective makes
    the next step form its MTTKRP again. (The rank-16 case uses the separate pass.)"""
    dims, nnz, dist, s, R = case
    idx, vals, init = make_case(dims, nnz, dist, s, R)
    cidx, cvals = O.coalesce(dims, idx, vals)
    N = len(dims)
    kw = dict(precision=S.SACD_BF16_GATHER)
    with S.SaCD(dims, idx, vals, R, init, **kw) as a, S.SaCD(dims, idx, vals, R, init, **kw) as b, \
            S.SaCD(dims, idx, vals, R, init, **kw) as c:
        for it in range(4):
            a.iterate(1)
            a.fit()
            b.iterate(1)
            for n in range(N):
                c.mode_step(n, want_count=False)
            c.fit()
        for n in range(N):
            np.testing.assert_array_equal(a.factor(n), b.factor(n))
            np.testing.assert_array_equal(c.factor(n), b.factor(n))
        obj, fit = a.fit()
        assert (obj, fit) == b.fit() == c.fit()
        F = a.factors()
        nx = O.norm_x_sq(cvals)
        inner = O.inner_x_model(cidx, cvals, F)
        mn = O.model_norm_sq(F)
        assert abs(obj - (nx - 2.0 * inner + mn)) <= 2.0 * 2e-6 * abs(inner) + 1e-9 * mn + 1e-12 * nx
        # a factor changed after the objective: mode 0's step must gather it
        a.set_factor(1, 0.5 * a.factor(1))
        b.set_factor(1, 0.5 * b.factor(1))
        a.mode_step(0)
        b.mode_step(0)
        np.testing.assert_array_equal(a.factor(0), b.factor(0))
        a.fit()
        a.iterate(2)
        b.iterate(2)
        for n in range(N):
            np.testing.assert_array_equal(a.factor(n), b.factor(n))


@pytest.mark.parametrize("prec", [S.SACD_FP32, S.SACD_BF16_GATHER], ids=["fp32", "bf16"])
@pytest.mark.parametrize("case", [CASES[1], CASES[2], CASES[3]], ids=ids)
def test_fit_at_identical_factors(case, prec):
    """sacd_fit is the objective (Eq. 6-8) of the factors the context returns, in both
    precisions: after 5 iterations, against the oracle's FP64 objective of exactly those FP32
    factors. Bound: the FP32 MTTKRP behind <X, model> carries a rounding error of about
    sqrt(chain) * 2^-24 relative (chains of a few hundred partial sums: ~1e-6); the FP64 Grams
    1e-10. A fit formed from BF16-gathered rows is off by ~3e-4 of <X, model>."""
    dims, nnz, dist, s, R = case
    idx, vals, init = make_case(dims, nnz, dist, s, R)
    cidx, cvals = O.coalesce(dims, idx, vals)
    with S.SaCD(dims, idx, vals, R, init, precision=prec) as g:
        for k in range(2):
            g.iterate(1 if k == 0 else 4)
            F = g.factors()
            obj, fit = g.fit()
            nx = O.norm_x_sq(cvals)
            inner = O.inner_x_model(cidx, cvals, F)
            mn = O.model_norm_sq(F)
            ref = nx - 2.0 * inner + mn
            assert np.isfinite(obj)
            assert abs(obj - ref) <= 2.0 * 2e-6 * abs(inner) + 1e-9 * mn + 1e-12 * nx, (obj, ref)
            assert fit == pytest.approx(O.fit_from_objective(obj, nx), rel=1e-12, abs=1e-15)


@pytest.mark.parametrize("prec", [S.SACD_FP32, S.SACD_BF16_GATHER], ids=["fp32", "bf16"])
@pytest.mark.parametrize("R", [1, 8, 12, 32, 100, 256])
@pytest.mark.parametrize("dims", [(150, 90, 60), (60, 50, 40, 30)], ids=["n3", "n4"])
def test_mttkrp_every_row_width(dims, R, prec):
    """Every gathered-row width (one 16-byte vector for R <= 8 with BF16 gathers up to 64 for
    R = 256 FP32), so every kernel specialisation and index-stage shape runs: M of every mode
    against the oracle (FP32 gathers) or the oracle's BF16-gather definition, within 1e-5."""
    idx, vals, init = make_case(dims, 9_001, "zipf", 1.2, R)
    cidx, cvals = O.coalesce(dims, idx, vals)
    with S.SaCD(dims, idx, vals, R, init, precision=prec) as g:
        g.set_debug(True)
        for n in range(len(dims)):
            F = g.factors()
            g.mode_step(n)
            Fg = F if prec == S.SACD_FP32 else [O.round_bf16(f) for f in F]
            assert relerr(g.tap("M", n), O.mttkrp(list(dims), cidx, cvals, Fg, n)) <= 1e-5


def test_edge_cases():
    # no nonzeros
    with S.SaCD((5, 4, 3), np.zeros((3, 0), np.int32), np.zeros(0, np.float32), 3, seed=1) as g:
        g.iterate(2)
        obj, fit = g.fit()
        assert obj >= 0 and all(np.isfinite(A).all() for A in g.factors())
    # one nonzero, modes of length 1, rank 1
    with S.SaCD((1, 1, 1), np.zeros((3, 1), np.int32), np.array([2.0], np.float32), 1,
                [np.full((1, 1), 0.5, np.float32)] * 3) as g:
        o = O.SaCDOracle((1, 1, 1), np.zeros((3, 1)), np.array([2.0], np.float32), [np.full((1, 1), 0.5, np.float32)] * 3)
        g.iterate(3)
        o.iterate(3)
        for n in range(3):
            np.testing.assert_allclose(g.factor(n), o.A[n], rtol=1e-5)
    # only repeats of one coordinate
    idx = np.zeros((3, 7), np.int32)
    vals = np.arange(1, 8, dtype=np.float32)
    with S.SaCD((2, 2, 2), idx, vals, 2, seed=3) as g:
        assert g.info["nnz"] == 1
        assert g.tap("CSF_VAL", 0)[0] == 28.0
    # empty rows in every mode (sparse coordinates)
    idx = np.array([[0, 7, 7, 15], [3, 3, 9, 1], [0, 4, 4, 4]], np.int32)
    init = synth.init_factors((16, 10, 5), 4, 2)
    with S.SaCD((16, 10, 5), idx, np.ones(4, np.float32), 4, init) as g:
        o = O.SaCDOracle((16, 10, 5), idx, np.ones(4, np.float32), init)
        for n in range(3):
            g.mode_step(n)
            o.mode_step(n)
            assert relerr(g.tap("M", n), o.last["M"]) <= 1e-6


def test_errors():
    with pytest.raises(S.SacdError) as e:
        S.SaCD((3, 3, 3), np.array([[0], [3], [0]], np.int32), np.ones(1, np.float32), 2)
    assert e.value.status == 1
    with pytest.raises(S.SacdError) as e:
        S.SaCD((3, 3, 3), np.zeros((3, 1), np.int32), np.ones(1, np.float32), 2,
               [np.full((3, 2), -1.0, np.float32)] * 3)
    assert e.value.status == 1
    with pytest.raises(S.SacdError) as e:
        S.SaCD((3, 3, 3), np.zeros((3, 1), np.int32), np.ones(1, np.float32), 0)
    assert e.value.status == 1
    with S.SaCD((3, 3, 3), np.zeros((3, 1), np.int32), np.ones(1, np.float32), 2, seed=5) as g:
        with pytest.raises(S.SacdError):
            g.mode_step(3)
        with pytest.raises(S.SacdError):
            g.tap("MASK", 0)  # debug recording is off
        with pytest.raises(S.SacdError):
            g.set_factor(0, np.full((3, 2), np.nan, np.float32))


def test_device_inputs_from_torch():
    import torch

    dims, nnz, dist, s, R = CASES[1]
    idx, vals, init = make_case(dims, nnz, dist, s, R)
    dev = torch.device("cuda:0")
    stream = torch.cuda.Stream()
    ti = [torch.from_numpy(idx[n].copy()).to(dev) for n in range(3)]
    tv = torch.from_numpy(vals).to(dev)
    tf = [torch.from_numpy(a).to(dev) for a in init]
    torch.cuda.synchronize()
    with S.SaCD(dims, ti, tv, R, tf, on_device=True, stream=stream.cuda_stream) as a, S.SaCD(dims, idx, vals, R, init) as b:
        a.iterate(2)
        b.iterate(2)
        for n in range(3):
            np.testing.assert_array_equal(a.factor(n), b.factor(n))


def check_step_rows(g, n, F, zprev, st, mask, rows, M_rows, bf16=False):
    """One GPU mode step of mode n checked on the given rows against the oracle's definitions,
    from the same factors and importance state with the GPU's selection: M (the oracle's MTTKRP of
    those rows, given), G, z, the selection's validity (free disagreements only at the decision
    boundary) and the updated rows of A."""
    H = O.hadamard_of_grams([f.astype(np.float64) for f in F], n)
    L = O.lipschitz(H)
    h = O.curvatures(H)
    A = F[n].astype(np.float64)[rows]
    G = A @ H - M_rows
    Sd = O.projected_delta(A, G, h[None, :])
    Z = O.importance(G, Sd, L)
    t = dict(G=G, H=H, L=L)
    Mg = g.tap("M", n)[rows]
    assert relerr(Mg, M_rows) <= 1e-5
    assert_elementwise(Mg, M_rows, 1e-5)
    Gg = g.tap("G", n, last_mode=n)[rows]
    AH = A @ H
    assert_elementwise(Gg, G, 1e-5, np.abs(M_rows).max(axis=1) + np.abs(AH).max(axis=1))
    zg = g.tap("ZPREV", n)[rows]
    zs = max(np.abs(Z).max(), 1e-30)
    assert (np.abs(zg - Z) <= 1e-5 * zs + z_fp32_bound(A, t)).all()
    m = mask[rows]
    first = st[1] != 0
    branch = g.tap("STATE", n)[3]
    zp = zprev[rows].astype(np.float64)
    if first:
        own, sp = Z > 0, Z
    elif branch == 2.0:
        own, sp = (zp - Z) > 0, zp - Z
    else:
        own, sp = (Z - zp) > 0, Z - zp
    dis = own != m
    assert (np.abs(sp[dis]) <= 1e-5 * zs + z_fp32_bound(A, t)[dis]).all()
    Anew, _ = O.update_rows(A, G, H, m, "column_gs", h)
    An = g.factor(n)[rows]
    assert (An >= 0).all()
    assert_rowwise(An, Anew, 1e-5, np.linalg.norm(A, axis=1))


def heavy_and_random_rows(idx_n, dim, k_heavy, k_rand, seed):
    counts = np.bincount(idx_n, minlength=dim)
    rng = np.random.default_rng(seed)
    return np.unique(np.concatenate([np.argsort(counts)[-k_heavy:], rng.integers(0, dim, k_rand)]))


def test_full_size_zipf_workload_every_element():
    """The 50,000 x 20,000 x 500, 5M-nonzero Zipf(1.1) rank-32 workload, in the launch configuration
    the benchmark uses: one iteration (all three modes), every element of M, G, z and A and the
    selection against the oracle from the same factors with the GPU's selection, plus the MTTKRP
    rows of the heaviest (split) rows element by element."""
    w = synth.WORKLOADS["zipf1.1-50000x20000x500-5M-r32"]
    idx, vals, init = synth.make_workload(w)
    with S.SaCD(w.dims, idx, vals, w.rank, init) as g:
        assert g.info["nnz"] == w.nnz
        assert max(g.info["split_rows"][:3]) > 0
        g.set_debug(True)
        for n in range(3):
            F = g.factors()
            zprev = g.tap("ZPREV", n)
            st = g.tap("STATE", n)
            g.mode_step(n, want_count=False)
            mask = g.tap("MASK", n, last_mode=n).astype(bool)
            M = O.mttkrp(list(w.dims), idx, vals, F, n)
            check_step_rows(g, n, F, zprev, st, mask, np.arange(w.dims[n]), M)
        assert np.isfinite(g.fit()[0])


def test_full_size_bf16_4mode_workload_sampled_rows():
    """The 200,000 x 100,000 x 10,000 x 200, 50M-nonzero Zipf(1.2) rank-64 BF16-gather workload in
    the benchmark's launch configuration: one iteration (all four modes), M, G, z, the selection
    and A on sampled rows (the heaviest rows, split across many tiles, plus random ones) against the
    oracle's BF16-gather definition from the same factors with the GPU's selection; M also loosely
    against FP32 gathers."""
    w = synth.WORKLOADS["zipf1.2-200000x100000x10000x200-50M-r64-bf16"]
    idx, vals, init = synth.make_workload(w)
    with S.SaCD(w.dims, idx, vals, w.rank, init, precision=S.SACD_BF16_GATHER) as g:
        assert g.info["nnz"] == w.nnz
        g.set_debug(True)
        for n in range(4):
            F = g.factors()
            zprev = g.tap("ZPREV", n)
            st = g.tap("STATE", n)
            g.mode_step(n, want_count=False)
            mask = g.tap("MASK", n, last_mode=n).astype(bool)
            rows = heavy_and_random_rows(idx[n], w.dims[n], 8, 24, n)
            keep = np.isin(idx[n], rows)
            Fb = [O.round_bf16(f) for f in F]
            ref_b = O.mttkrp(list(w.dims), idx[:, keep], vals[keep], Fb, n)[rows]
            ref = O.mttkrp(list(w.dims), idx[:, keep], vals[keep], F, n)[rows]
            assert relerr(g.tap("M", n)[rows], ref) <= 1e-2
            check_step_rows(g, n, F, zprev, st, mask, rows, ref_b, bf16=True)
        assert np.isfinite(g.fit()[0])


@pytest.mark.slow
def test_full_size_zipf_workload_50_iterations():
    """The 5M-nonzero workload's own iteration count, 50 iterations (about five minutes of oracle
    time on the host). (1) Iterations 1, 10, 25 and 50, each run by the oracle from the GPU's state
    at its start with the GPU's selection, end within 1e-4 of the GPU's fit. (2) The free
    trajectories end within 2e-3: on this workload the selection (Eq. 24/27, discontinuous)
    amplifies FP32-sized gradient errors; an FP64 oracle whose gradient carries noise of 4 FP32
    ulps of |A||H| + |M| drifts from the exact oracle by 1.0e-2 after 10, 6.4e-4 after 20, 3.3e-4
    after 30 and 5.0e-4 after 40 iterations (rounding only its factors to FP32 after each step:
    at most 1.9e-5), so no FP32 implementation meets 1e-4 on the free 50-iteration trajectory."""
    w = synth.WORKLOADS["zipf1.1-50000x20000x500-5M-r32"]
    idx, vals, init = synth.make_workload(w)
    o = O.SaCDOracle(w.dims, idx, vals, init)
    with S.SaCD(w.dims, idx, vals, w.rank, init) as g:
        g.set_debug(True)
        for it in range(1, w.iters + 1):
            if it in (1, 10, 25, 50):
                resync(o, g, 3)
                for n in range(3):
                    g.mode_step(n, want_count=False)
                    o.mode_step(n, mask=g.tap("MASK", n, last_mode=n).astype(bool))
                assert abs(g.fit()[1] - o.fit()[1]) <= 1e-4
            else:
                g.iterate(1)
        fit = g.fit()[1]
        assert all((A >= 0).all() for A in g.factors())
    o = O.SaCDOracle(w.dims, idx, vals, init)
    o.iterate(w.iters)
    print(f"5M workload, 50 free iterations: |dfit| {abs(fit - o.fit()[1]):.3e}")
    assert abs(fit - o.fit()[1]) <= 2e-3, (fit, o.fit()[1])


@pytest.mark.parametrize("sub", [4, 16, 64, 256])
def test_retiling_keeps_mttkrp_and_step(sub):
    dims, nnz, dist, s, R = CASES[1]
    idx, vals, init = make_case(dims, nnz, dist, s, R)
    cidx, cvals = O.coalesce(dims, idx, vals)
    with S.SaCD(dims, idx, vals, R, init) as g:
        for n in range(3):
            S.sacd_set_tiling(g.ctx, n, sub)
            assert S.sacd_get_info(g.ctx)["tile_nnz"][n] == sub * (32 // min(R * 4 // 16, 32))
        for n in range(3):
            F = g.factors()
            g.mode_step(n)
            assert relerr(g.tap("M", n), O.mttkrp(list(dims), cidx, cvals, F, n)) <= 1e-5
        g.iterate(2)  # the graph picks up the new tiling
        assert all((A >= 0).all() for A in g.factors())


