"""Serving core: continuous batching with HBM-budget admission. Each job's result is the same
alone and in the mix (bit-identical factors), the budget is respected, and failures injected on
the host (bad input, a job larger than the budget) finish only the failing job."""

import numpy as np
import pytest

from oracle import sacd_oracle as O
from paper_2003_03572_gb300 import sacd as S
from paper_2003_03572_gb300 import serve, synth

pytestmark = pytest.mark.gpu


def specs(seed=5):
    shapes = [((300, 200, 50), 16, 0), ((150, 120, 40, 10), 32, 1), ((400, 90, 30), 64, 1), ((200, 220, 60), 8, 0),
              ((90, 80, 70, 6), 16, 0), ((500, 60, 25), 32, 1)]
    out = []
    for j, (dims, R, bf) in enumerate(shapes):
        idx, vals = synth.sparse_tensor(dims, 4000 + 1500 * j, dist="zipf", zipf_s=1.1, seed=seed + j)
        out.append(dict(dims=dims, idx=idx, vals=vals, rank=R, init=synth.init_factors(dims, R, seed + j),
                        precision=S.SACD_BF16_GATHER if bf else S.SACD_FP32))
    return out


def test_served_results_equal_alone():
    sp = specs()
    iters = [5, 8, 3, 6, 4, 7]
    with serve.Server(1 << 34) as srv:
        ids = [srv.submit(s, it) for s, it in zip(sp, iters)]
        done = {}
        while len(done) < len(sp):
            srv.step()
            for r in srv.results():
                assert r["status"] == 0, r
                done[r["job_id"]] = (r, srv.factors(r["job_id"]))
                srv.release(r["job_id"])
    for jid, s, it in zip(ids, sp, iters):
        r, F = done[jid]
        assert r["iters"] == it
        with S.SaCD(s["dims"], s["idx"], s["vals"], s["rank"], s["init"], precision=s["precision"]) as a:
            a.iterate(it)
            for n in range(len(s["dims"])):
                np.testing.assert_array_equal(F[n], a.factor(n))
            assert (r["objective"], r["fit"]) == a.fit()


def test_served_jobs_match_oracle():
    """Each served job against the FP64 oracle. FP32 jobs: final fits within 1e-4 of the oracle's
    own trajectory (as for single contexts). BF16-gather jobs: the served factors are bit-identical
    to the same job run alone, mode step by mode step; every iteration of that run, from the GPU's
    state with its selection replayed, ends within 1e-3 of the fit of an iteration of the oracle's
    BF16-gather definition. (Free BF16 trajectories of equal definition spread apart: BF16
    rounding turns small differences of FP32 master values into BF16-ulp differences of gathered
    values, which flip discontinuous selections.) Every fit is finite."""
    sp = specs(21)
    iters = [6, 4, 5, 6, 3, 5]
    with serve.Server(1 << 34) as srv:
        ids = [srv.submit(s, it) for s, it in zip(sp, iters)]
        done = {}
        while len(done) < len(sp):
            srv.step()
            for r in srv.results():
                assert r["status"] == 0, r
                done[r["job_id"]] = (r, srv.factors(r["job_id"]))
                srv.release(r["job_id"])
    for jid, s, it in zip(ids, sp, iters):
        r, Fs = done[jid]
        assert np.isfinite(r["objective"]) and np.isfinite(r["fit"])
        if s["precision"] == S.SACD_FP32:
            o = O.SaCDOracle(s["dims"], s["idx"], s["vals"], s["init"])
            o.iterate(it)
            assert abs(r["fit"] - o.fit()[1]) <= 1e-4
            continue
        o = O.SaCDOracle(s["dims"], s["idx"], s["vals"], s["init"], gather="bf16")
        N = len(s["dims"])
        with S.SaCD(s["dims"], s["idx"], s["vals"], s["rank"], s["init"], precision=s["precision"]) as a:
            a.set_debug(True)
            for _ in range(it):
                # each iteration from the GPU's state, the selection replayed
                o.A = [f.astype(np.float64) for f in a.factors()]
                for n in range(N):
                    o.Zprev[n] = a.tap("ZPREV", n).astype(np.float64)
                    st = a.tap("STATE", n)
                    o.tiprev[n], o.first[n] = st[0], st[1] != 0
                for n in range(N):
                    a.mode_step(n, want_count=False)
                    o.mode_step(n, mask=a.tap("MASK", n, last_mode=n).astype(bool))
                assert abs(a.fit()[1] - o.fit()[1]) <= 1e-3
            for n in range(N):
                np.testing.assert_array_equal(a.factor(n), Fs[n])
            assert r["fit"] == a.fit()[1]


def test_budget_admission_and_host_failures():
    sp = specs(9)
    bad = dict(sp[0])
    bad["idx"] = sp[0]["idx"].copy()
    bad["idx"][0, 0] = 10_000  # out of range: fails at admission, on the host side of the create
    huge = dict(dims=(100, 100, 100), idx=np.zeros((3, 1), np.int32), vals=np.ones(1, np.float32), rank=8)
    budget = 8 << 20  # two or three of these jobs at a time (each is charged 2 to 4 MB at admission)
    with serve.Server(budget) as srv:
        jobs = [srv.submit(s, 4) for s in sp[:4]] + [srv.submit(bad, 4)] + [srv.submit(s, 4) for s in sp[4:]]
        huge_spec = dict(dims=(2_000_000, 2_000_000, 2_000_000), idx=np.zeros((3, 1), np.int32),
                         vals=np.ones(1, np.float32), rank=256)
        jh = srv.submit(huge_spec, 2)
        status = {}
        max_active = 0
        while len(status) < len(jobs) + 1:
            a, w = srv.step()
            max_active = max(max_active, a)
            st = srv.stats()
            assert st["used_bytes"] <= budget
            for r in srv.results():
                status[r["job_id"]] = (r["status"], r["error"])
                srv.release(r["job_id"])
        assert status[jobs[4]][0] == 1 and "outside" in status[jobs[4]][1]
        assert status[jh][0] == 2
        assert all(status[j][0] == 0 for k, j in enumerate(jobs) if k != 4)
        assert srv.stats()["peak_bytes"] <= budget
        assert max_active <= 4  # running plus being created: the budget held the rest back


def test_admission_overlaps_running_jobs():
    """A job admitted while another runs is created by the preparation thread on its own stream:
    steps keep iterating the running job while the new context is built (stats count it as
    creating), the new job then joins, and both results equal their contexts run alone."""
    small = specs(17)[0]
    dims = (200_000, 100_000, 2_000)
    idx, vals = synth.sparse_tensor(dims, 4_000_000, dist="zipf", zipf_s=1.1, seed=31)
    big = dict(dims=dims, idx=idx, vals=vals, rank=16, init=synth.init_factors(dims, 16, 31))
    with serve.Server(1 << 36) as srv:
        ja = srv.submit(small, 400)
        while srv.stats()["creating"] or srv.stats()["active"] == 0:
            srv.step()
        jb = srv.submit(big, 3)
        steps_while_creating = 0
        res = {}
        while len(res) < 2:
            srv.step()
            st = srv.stats()
            if st["creating"]:
                steps_while_creating += 1
            for r in srv.results():
                res[r["job_id"]] = r
                if r["status"] == 0:
                    r["factors"] = srv.factors(r["job_id"])
                srv.release(r["job_id"])
    assert steps_while_creating >= 2
    assert res[ja]["status"] == 0 and res[jb]["status"] == 0
    for jid, sp, it in ((ja, small, 400), (jb, big, 3)):
        with S.SaCD(sp["dims"], sp["idx"], sp["vals"], sp["rank"], sp["init"],
                    precision=sp.get("precision", S.SACD_FP32)) as g:
            g.iterate(it)
            for n in range(len(sp["dims"])):
                np.testing.assert_array_equal(res[jid]["factors"][n], g.factor(n))


def test_poisson_arrival_driver():
    sp = specs(13) * 3
    arrivals = serve.poisson_arrivals(200.0, len(sp), 3)
    with serve.Server(1 << 34) as srv:
        res, wall = serve.run_arrivals(srv, sp, arrivals, 5)
    assert len(res) == len(sp) and all(r["status"] == 0 for r in res)
    assert all(r["latency"] > 0 for r in res)
    summ = serve.latency_summary(res)
    assert 0 < summ["p50_s"] <= summ["p99_s"]


def device_init(dims, R, seed):
    """The library's counter-based initial factors (init == NULL), restated from the definition in
    the C header: (h >> 40) * 2^-24, h the splitmix64 finaliser of seed + (n+1)*0xD1B54A32D192ED03 +
    (i*R + r + 1)*0x9E3779B97F4A7C15."""
    out = []
    M = np.uint64
    with np.errstate(over="ignore"):
        for n, I in enumerate(dims):
            e = np.arange(int(I) * R, dtype=np.uint64)
            z = M(seed) + M(n + 1) * M(0xD1B54A32D192ED03) + (e + M(1)) * M(0x9E3779B97F4A7C15)
            z = (z ^ (z >> M(30))) * M(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> M(27))) * M(0x94D049BB133111EB)
            z ^= z >> M(31)
            out.append(((z >> M(40)).astype(np.float64) * 2.0**-24).astype(np.float32).reshape(int(I), R))
    return out


def test_collapsed_columns_stay_finite():
    """A job of the served workload (4 modes, 760 x 1310 x 9469 x 20964, 73,939 nonzeros, R = 32,
    U[0,1) initial factors from the seed) whose early steps drive whole columns of the other
    factors to (almost) zero: h_rr falls to ~1e-40, where 1/h_rr and the s^2 term of Eq. 20 leave
    the FP32 range. Such columns take no step (h_rr <= max(2^-40 max h, 2^-126) counts as 0, on both
    sides). Every fit stays finite, alone and served, in both precisions, and the FP32 job matches
    the oracle within 1e-3 (see below)."""
    tensors, jobs = synth.serving_workloads(1000, pool=64)
    ti, R, seed = jobs[937]
    w = tensors[ti]
    idx, vals = synth.sparse_tensor(w.dims, w.nnz, dist=w.dist, zipf_s=w.zipf_s, values=w.values, seed=w.seed)
    init = device_init(w.dims, R, seed)
    spec = dict(dims=w.dims, idx=idx, vals=vals, rank=R, init=None, seed=seed)
    fits = {}
    for prec in (S.SACD_FP32, S.SACD_BF16_GATHER):
        with S.SaCD(w.dims, idx, vals, R, None, seed=seed, precision=prec) as g:
            for n in range(4):
                np.testing.assert_array_equal(g.factor(n), init[n])  # the restated draw
            g.iterate(30)
            obj, fit = g.fit()
            assert np.isfinite(obj) and np.isfinite(fit)
            assert all(np.isfinite(A).all() for A in g.factors())
            fits[prec] = fit
    with serve.Server(1 << 34) as srv:
        ids = [srv.submit(dict(spec, precision=p), 30) for p in (S.SACD_FP32, S.SACD_BF16_GATHER)]
        done = 0
        while done < 2:
            srv.step()
            for r in srv.results():
                assert r["status"] == 0, r
                assert r["fit"] == fits[S.SACD_FP32 if r["job_id"] == ids[0] else S.SACD_BF16_GATHER]
                srv.release(r["job_id"])
                done += 1
    o = O.SaCDOracle(w.dims, idx, vals, init)
    frozen = 0
    for _ in range(30):
        for n in range(4):
            o.mode_step(n)
            frozen += int(((np.diag(o.last["H"]) > 0) & (O.curvatures(o.last["H"]) == 0)).sum())
    assert frozen > 0  # the case really has collapsed columns
    # Its initial model is ~1e9 times the data (objective ~3e5 ||X||^2 after 3 iterations), so the
    # FP32 gradients of the early steps carry errors far above the data's scale that FP64 does not:
    # FP32 arithmetic, not the reading, separates the trajectories (rounding only the oracle's
    # factors to FP32 after each step moves its fit by 3e-9). Bound: 1e-3.
    assert abs(fits[S.SACD_FP32] - o.fit()[1]) <= 1e-3


def test_device_init_scale_is_exact():
    """init == NULL with init_log2_scale = s: every value is the restated draw times 2^s exactly;
    a scale outside [-60, 60] is rejected."""
    dims, R = (70, 40, 9), 12
    idx, vals = synth.sparse_tensor(dims, 900, dist="zipf", zipf_s=1.1, seed=3)
    ref = device_init(dims, R, 77)
    for sc in (0, -4, 3):
        with S.SaCD(dims, idx, vals, R, None, seed=77, init_log2_scale=sc) as g:
            for n in range(3):
                np.testing.assert_array_equal(g.factor(n), ref[n] * np.float32(2.0**sc))
    with pytest.raises(S.SacdError) as e:
        S.SaCD(dims, idx, vals, R, None, seed=77, init_log2_scale=61)
    assert e.value.status == 1
