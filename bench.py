#!/usr/bin/env python3
"""Benchmark of the SaCD hot path on one GB300 (or N independent replicas under torchrun).

A "step" is one SaCD outer iteration (the mode steps 0..N-1: MTTKRP, H/L, gradient and
importance, selection and update, Gram refresh) followed by the objective/fit evaluation, on the
workload's tensor resident in HBM. value = mode steps per second over the timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Prints one JSON line (rank 0). The reference arm (--impl reference) times the FP64 CPU oracle
on the host cores, on the same workload and metric.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

DEFAULT_WORKLOAD = "zipf1.1-50000x20000x500-5M-r32"
L2_BYTES = 129 * 2**20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def mttkrp_bytes(w, nnz, mode):
    """Algorithmic bytes of one MTTKRP launch (COO model): per nonzero its value, its N
    coordinates and the N-1 gathered factor rows (R columns each), plus the I_n x R output."""
    s = 2 if w.precision == "bf16" else 4
    N = w.nmodes
    return nnz * (4 + 4 * N + (N - 1) * w.rank * s) + w.dims[mode] * w.rank * 4


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, mx, reasons, pw = [], None, set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            try:
                pw.append(float(f[3]))
            except ValueError:
                pass
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "sm_min_mhz": min(sm),
                "power_w_max": max(pw) if pw else None, "reasons": sorted(reasons), "samples": len(sm)}


def traffic_from_profile(src_sha, workload):
    """DRAM bytes per MTTKRP launch of `workload` from the committed ncu summary, if it was taken
    on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "mttkrp_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p))
    if d.get("mttkrp_source_sha256") != src_sha:
        return None
    return d.get("workloads", {}).get(workload, {}).get("dram_bytes_per_launch")


def cpu_baseline_child(workload, nsteps):
    """Run in a fresh single-threaded process: time the FP64 oracle on the workload."""
    from oracle import sacd_oracle as O
    from paper_2003_03572_gb300 import synth

    w = synth.WORKLOADS[workload]
    idx, vals, init = synth.make_workload(w)
    o = O.SaCDOracle(w.dims, idx, vals, init)  # one-time coalescing, not timed
    t = time.perf_counter()
    for s in range(nsteps):
        o.mode_step(s % w.nmodes)
    dt = time.perf_counter() - t
    print(json.dumps({"steps": nsteps, "seconds": dt}))


def run_cpu_baseline(workload, nsteps):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-child", "--workload", workload,
                        "--steps", str(nsteps)], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode != 0:
        return None
    d = json.loads(r.stdout.strip().splitlines()[-1])
    return d["steps"] / d["seconds"], d


def aggregate_over_ranks(local_value, ws, device=None, op="max"):
    """The slowest rank's time (or the sum of a count) over all ranks of the job; with one rank,
    the value itself. Used for the timed region (max over ranks) of the replicas."""
    if ws <= 1:
        return float(local_value)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(local_value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replicas_value(units_per_rank, ws, max_seconds):
    """Whole-job throughput of independent replicas: all ranks' units over the slowest rank's time."""
    return ws * units_per_rank / max_seconds


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


REF_FRACTION = 0.125  # share of the nonzeros in one reference-arm step


def reference_arm(args):
    ws, rank, local = dist_env()
    if rank != 0:
        return 0
    from oracle import sacd_oracle as O
    from paper_2003_03572_gb300 import synth

    import numpy as np

    w = synth.WORKLOADS[args.workload]
    idx, vals, init = synth.make_workload(w)
    # Each step is a bounded sample of the workload: the oracle as it stands, on a sub-tensor of
    # a seeded random REF_FRACTION of the nonzeros (same dims, rank, initial factors), so that
    # --steps 200 ends within a few minutes. A mode step of the oracle costs a fixed per-row part
    # (the dense Gram / gradient / update work, independent of the nonzeros) plus a per-nonzero
    # part (its MTTKRP); the full-workload step time per mode is extrapolated through this sample
    # and a second one 8x smaller.
    nnz = vals.shape[0]
    rng = np.random.default_rng(w.seed ^ 0x5A5A)

    def sample_oracle(frac):
        pick = np.sort(rng.choice(nnz, size=max(1, int(nnz * frac)), replace=False))
        return O.SaCDOracle(w.dims, np.ascontiguousarray(idx[:, pick]), vals[pick], init), pick.size

    N = w.nmodes
    o, n1 = sample_oracle(REF_FRACTION)
    step = 0
    for _ in range(args.warmup):
        o.mode_step(step % N)
        step += 1
    t1 = np.zeros(N)
    c1 = np.zeros(N)
    t = time.perf_counter()
    for _ in range(args.steps):
        n = step % N
        ts = time.perf_counter()
        o.mode_step(n)
        t1[n] += time.perf_counter() - ts
        c1[n] += 1
        step += 1
    dt = time.perf_counter() - t
    # the second point of the per-mode cost model: a few mode steps on a sample 8x smaller
    o0, n0 = sample_oracle(REF_FRACTION / 8)
    t0 = np.zeros(N)
    c0 = np.zeros(N)
    for cyc in range(3):
        for n in range(N):
            ts = time.perf_counter()
            o0.mode_step(n)
            if cyc > 0:  # the first cycle is a warm-up
                t0[n] += time.perf_counter() - ts
                c0[n] += 1
    f1, f0 = n1 / nnz, n0 / nnz
    a1 = np.where(c1 > 0, t1 / np.maximum(c1, 1), 0.0)
    a0 = t0 / c0
    # per mode: time = fixed + per_nonzero * nonzeros, through the two measured points
    full = a0 + (a1 - a0) * (1.0 - f0) / (f1 - f0)
    full = np.where(c1 > 0, full, a0 / max(f0, 1e-12))
    v = N / float(np.sum(full))
    sample = (f"{args.steps} FP64 oracle mode steps (cycling modes) on a seeded {n1}-nonzero sample "
              f"({f1:.4g} of the nonzeros, same dims and rank) after {args.warmup} warm-up steps, and "
              f"{2 * N} on a {n0}-nonzero sample; per mode, the full-workload step time is extrapolated "
              f"linearly in the nonzero count through the two (fixed per-row work + per-nonzero work); "
              f"one process")
    line = {
        "impl": "reference",
        "metric": "SaCD mode-steps/s",
        "value": v,
        "unit": "mode-steps/s",
        "n_gpus": args.gpus,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": dt * 1e3 / args.steps,
        "full_step_ms_by_mode": [round(float(x) * 1e3, 4) for x in full],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": w.name, "dims": list(w.dims), "nnz": w.nnz, "rank": w.rank,
                   "step": f"one mode step on a {REF_FRACTION:g} nonzero sample"},
        "cpu_baseline": {"value": v, "unit": "mode-steps/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "mode-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def ours_arm(args):
    import numpy as np
    import torch

    from paper_2003_03572_gb300 import sacd as S
    from paper_2003_03572_gb300 import synth

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    w = synth.WORKLOADS[args.workload]
    if args.scale != 1.0 and not args.kernels_only:
        raise SystemExit("--scale is for --kernels-only profiling runs")
    idx, vals, init = synth.make_workload(w, scale=args.scale)
    N = w.nmodes
    prec = S.SACD_BF16_GATHER if w.precision == "bf16" else S.SACD_FP32
    stream = torch.cuda.Stream(device=dev)

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # ---------------------------------------------------------------- device-resident timing
    g = S.SaCD(w.dims, idx, vals, w.rank, init, precision=prec, stream=stream.cuda_stream)
    info = g.info
    nnz = info["nnz"]
    for _ in range(args.warmup):
        g.iterate(1)
        g.fit()
    torch.cuda.synchronize(dev)
    barrier()
    torch.cuda.synchronize(dev)
    clk = ClockSampler(local)
    clk.start()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        g.iterate(1)
        obj, fit = g.fit()
    e1.record(stream)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = clk.stop()
    ms = aggregate_over_ranks(e0.elapsed_time(e1), ws, dev)
    value = replicas_value(args.steps * N, ws, ms / 1e3)

    # ---------------------------------------------------------------- per-kernel timing
    S.sacd_profile_enable(g.ctx, True)
    for _ in range(args.steps):
        g.iterate(1)
        g.fit()
    stats = S.sacd_profile_read(g.ctx)
    S.sacd_profile_enable(g.ctx, False)
    launches = sum(v[0] for v in stats.values())
    mt_launches, mt_ms = stats["mttkrp"]
    tot_bytes = args.steps * sum(mttkrp_bytes(w, nnz, n) for n in range(N))
    achieved = tot_bytes / (mt_ms / 1e3) / 1e9 if mt_ms > 0 else None
    peak, peak_kind = peaks()
    src_sha = hashlib.sha256(open(os.path.join(ROOT, "paper_2003_03572_gb300", "csrc", "mttkrp.cu"), "rb").read()).hexdigest()
    traffic = traffic_from_profile(src_sha, w.name)
    kernel_ms = {k: v[1] for k, v in stats.items()}
    total_kernel_ms = sum(kernel_ms.values())
    upd = update_roofline(w, prec == S.SACD_BF16_GATHER, kernel_ms, args.steps, peak)
    g.close()

    if args.kernels_only:  # short run for a profiler: device-resident steps only
        if rank == 0:
            print(json.dumps({"kernels_only": True, "scale": args.scale, "value": value, "unit": "mode-steps/s",
                              "kernel_ms_per_step": {k: v / args.steps for k, v in kernel_ms.items()}}))
        return 0

    # ---------------------------------------------------------------- end to end, host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_idx = [pin(idx[n]) for n in range(N)]
    h_vals = pin(vals)
    h_init = [pin(a) for a in init]
    h_out = [torch.empty(a.shape, dtype=torch.float32).pin_memory() for a in init]
    iters = w.iters
    e2e_times = []
    clk2 = ClockSampler(local)
    clk2.start()
    for rep in range(max(args.e2e_reps, 1) + 1):
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        ctx = S.sacd_create(w.dims, [t.numpy() for t in h_idx], h_vals.numpy(), w.rank,
                            [t.numpy() for t in h_init], precision=prec, stream=stream.cuda_stream)
        S.sacd_iterate(ctx, iters)
        S.sacd_fit(ctx)
        for n in range(N):
            S.sacd_get_factor(ctx, n, h_out[n].numpy())
        S.sacd_destroy(ctx)
        t1 = time.perf_counter()
        if rep > 0:  # first solve is a warm-up (allocator, graph instantiation)
            e2e_times.append(t1 - t0)
    e2e_clocks = clk2.stop()
    e2e_s = aggregate_over_ranks(statistics.median(e2e_times), ws, dev)
    e2e_value = replicas_value(N * iters, ws, e2e_s)
    h2d = int(len(vals) * (4 * N + 4) + sum(a.nbytes for a in init))
    d2h = int(sum(a.nbytes for a in init) + 16)

    # ---------------------------------------------------------------- CPU baseline (rank 0, N=1)
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        res = run_cpu_baseline(args.workload, N)
        if res:
            v, d = res
            cpu = {"value": v, "unit": "mode-steps/s", "cores": 1, "kind": "oracle",
                   "sample": f"one SaCD iteration ({N} mode steps) of the FP64 oracle on the full workload, "
                             f"single-threaded, after its one-time coalescing ({d['seconds']:.1f} s)"}

    if rank == 0:
        csf_bytes = nnz * (4 * N + 4) * N
        line = {
            "metric": "SaCD mode-steps/s",
            "value": value,
            "unit": "mode-steps/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": ms / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32" if prec == S.SACD_FP32 else "bf16-gather/f32",
            "data": "synthetic",
            "config": {
                "workload": w.name,
                "dims": list(w.dims),
                "nnz": nnz,
                "rank": w.rank,
                "step": "one SaCD iteration (all modes) + objective/fit",
                "l2": f"inputs larger than L2: {csf_bytes / 1e6:.0f} MB of sorted nonzeros per step vs "
                      f"{L2_BYTES / 1e6:.0f} MB L2",
                "parallelism": "replicas" if ws > 1 else "single GPU",
                "final_fit": fit,
            },
            "roofline": {
                "bound": "hbm",
                "kernel": "mttkrp",
                "achieved": achieved,
                "peak": peak,
                "peak_kind": f"{peak_kind} HBM copy bandwidth",
                "unit": "GB/s",
                "frac": (achieved / peak) if achieved else None,
                "traffic": traffic,
                "bytes_model": "COO model: nnz*(4 + 4N + (N-1)*R*s) + I_n*R*4 per launch",
                "mttkrp_share": mt_ms / total_kernel_ms if total_kernel_ms else None,
            },
            "update_roofline": upd,
            "kernel_ms_per_step": {k: v / args.steps for k, v in kernel_ms.items()},
            "gpu_launches": int(launches),
            "e2e": {
                "value": e2e_value,
                "unit": "mode-steps/s",
                "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h,
                "step": f"one full solve from pinned host COO: create (copy + CSF build) + {iters} iterations "
                        f"+ fit + factors back",
                "seconds_per_solve": e2e_s,
                "solve_seconds": [round(t, 5) for t in e2e_times],
                "clocks": e2e_clocks,
            },
            "clocks": clocks,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# FP32 instruction peak of one GB300: 152 SMs x 128 FP32 lanes x 2.07 GHz (maximum SM clock),
# one FP32 operation (an FMA counts as one) per lane and clock.
FP32_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12


def update_roofline(w, bf16, kernel_ms, steps, hbm_peak, compensated=False):
    """Select/update roofline of pass 1 + pass 2 (one element = one factor entry of a mode step):
    algorithmic bytes 20 per element (read M, A, z^{k-1}; write A, z^{k-1}; 22 with the BF16
    mirror) against the HBM copy peak, and, for pass 1, its R products per element against the FP32
    instruction peak: one fused multiply-add each (Frobenius or spectral L, the bench's setting),
    or 10 FP32 operations each when compensated (exact product 2, TwoSum 6, error terms 2; GCD)."""
    elems = sum(w.dims) * w.rank * steps
    bpe = 20 + (2 if bf16 else 0)
    t = (kernel_ms.get("pass1_grad_importance", 0.0) + kernel_ms.get("pass2_select_update", 0.0)) / 1e3
    t1 = kernel_ms.get("pass1_grad_importance", 0.0) / 1e3
    if t <= 0 or t1 <= 0:
        return None
    gbs = elems * bpe / t / 1e9
    opp = 10 if compensated else 1
    tops = elems * w.rank * opp / t1 / 1e12
    return {"kernels": ["pass1_grad_importance", "pass2_select_update"], "bytes_per_element": bpe,
            "elements_per_step": elems // steps, "achieved_gbs": gbs, "hbm_peak_gbs": hbm_peak,
            "frac_hbm": gbs / hbm_peak,
            "pass1": {"bound": "alu", "ops_per_element": opp * w.rank, "achieved_tops": tops,
                      "peak_tops": FP32_PEAK_TOPS, "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz",
                      "frac": tops / FP32_PEAK_TOPS}}


def _gen_job(w):
    from paper_2003_03572_gb300 import synth

    idx, vals = synth.sparse_tensor(w.dims, w.nnz, dist=w.dist, zipf_s=w.zipf_s, values=w.values, seed=w.seed)
    return idx, vals, synth.init_factors(w.dims, w.rank, w.seed)


def batched_arm(args):
    """Many small independent jobs: one batched launch set per mode step (CUDA graph) against
    the same jobs solved one at a time, each from its own context, on the same GPU."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import numpy as np
    import torch

    from paper_2003_03572_gb300 import sacd as S
    from paper_2003_03572_gb300 import synth

    ws = synth.batched_workloads(args.jobs)
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 4), mp_context=mp.get_context("spawn")) as ex:
        data = list(ex.map(_gen_job, ws, chunksize=8))
    torch.cuda.init()
    stream = torch.cuda.Stream()
    specs = [dict(dims=w.dims, idx=d[0], vals=d[1], rank=w.rank, init=d[2]) for w, d in zip(ws, data)]
    iters = ws[0].iters
    nnz_total = sum(w.nnz for w in ws)
    mode_steps = sum(w.nmodes for w in ws) * iters
    # batched
    b = S.SaCDBatch(specs, stream=stream.cuda_stream)
    b.iterate(1)  # graph capture and warm-up
    torch.cuda.synchronize()
    del b
    times_b = []
    fits_b = None
    for rep in range(args.e2e_reps):
        b = S.SaCDBatch(specs, stream=stream.cuda_stream)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        b.iterate(iters)
        obj, fits_b = b.fit()
        times_b.append(time.perf_counter() - t0)
        b.close()
    # one at a time (same contexts, same arithmetic)
    ctxs = [S.SaCD(sp["dims"], sp["idx"], sp["vals"], sp["rank"], sp["init"], stream=stream.cuda_stream)
            for sp in specs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    fits_1 = []
    for g in ctxs:
        g.iterate(iters)
        fits_1.append(g.fit()[1])
    t1 = time.perf_counter() - t0
    for g in ctxs:
        g.close()
    tb = statistics.median(times_b)
    line = {
        "metric": "batched SaCD jobs/s",
        "value": len(ws) / tb,
        "unit": "jobs/s",
        "one_at_a_time": len(ws) / t1,
        "speedup": t1 / tb,
        "mode_steps_per_s": mode_steps / tb,
        "same_final_fit": bool(np.array_equal(np.asarray(fits_b), np.asarray(fits_1))),
        "config": {"workload": f"batched {len(ws)} jobs: dims U[200,5000]xU[200,5000]xU[20,200], nnz U[10k,500k] "
                               f"Zipf(1.1), R in {{8,16,32}}, FP32, {iters} iterations", "nnz_total": nnz_total},
        "seconds_batched": tb,
        "seconds_one_at_a_time": t1,
    }
    print(json.dumps(line), flush=True)
    return 0


def serve_arm(args):
    """Served workload: Poisson arrivals of 3- and 4-mode BF16-gather jobs, continuous batching
    with HBM-budget admission; solves/s and arrival-to-result latency percentiles."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import numpy as np
    import torch

    from paper_2003_03572_gb300 import sacd as S
    from paper_2003_03572_gb300 import serve, synth

    tensors, jobs = synth.serving_workloads(args.jobs, pool=args.pool)
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 4), mp_context=mp.get_context("spawn")) as ex:
        data = list(ex.map(_gen_job_tensor, tensors, chunksize=1))
    torch.cuda.init()
    stream = torch.cuda.Stream()
    specs = []
    for ti, R, seed in jobs:
        w = tensors[ti]
        specs.append(dict(dims=w.dims, idx=data[ti][0], vals=data[ti][1], rank=R, init=None, seed=seed,
                          precision=S.SACD_BF16_GATHER))
    iters = tensors[0].iters
    arrivals = serve.poisson_arrivals(args.rate, len(specs), 0x5ACD0004)
    sample = set(range(0, len(specs), max(1, len(specs) // 4)))
    with serve.Server(int(args.budget_gb * 2**30), stream=stream.cuda_stream) as srv:
        # warm-up: one small job (module loading, allocator) before the clock starts
        sm = min(range(len(specs)), key=lambda i: tensors[jobs[i][0]].nnz)
        serve.run_arrivals(srv, [specs[sm]], [0.0], 2)
        res, wall = serve.run_arrivals(srv, specs, arrivals, iters, keep_for=sample)
        st = srv.stats()
    ok = [r for r in res if r["status"] == 0]
    # each sampled job again, alone, from its own context: same factors as in the mix
    same = True
    for r in res:
        if r["index"] in sample and "factors" in r:
            sp = specs[r["index"]]
            with S.SaCD(sp["dims"], sp["idx"], sp["vals"], sp["rank"], None, seed=sp["seed"],
                        precision=sp["precision"], stream=stream.cuda_stream) as a:
                a.iterate(iters)
                same &= all(np.array_equal(a.factor(n), r["factors"][n]) for n in range(len(sp["dims"])))
    summ = serve.latency_summary(res)
    base = None
    if args.serve_baseline:
        # the same arrival stream served one job at a time with FP32 gathers
        specs32 = [dict(sp, precision=S.SACD_FP32) for sp in specs]
        with serve.Server(int(args.budget_gb * 2**30), max_active=1, stream=stream.cuda_stream) as srv1:
            res1, wall1 = serve.run_arrivals(srv1, specs32, arrivals, iters)
        ok1 = [r for r in res1 if r["status"] == 0]
        fit_b = {r["index"]: r["fit"] for r in ok}
        dfit = [abs(fit_b[r["index"]] - r["fit"]) for r in ok1 if r["index"] in fit_b]
        base = {"solves_per_s": len(ok1) / wall1, "latency": serve.latency_summary(res1), "wall_s": wall1,
                "fit_abs_diff_mean": float(np.mean(dfit)) if dfit else None,
                "fit_abs_diff_max": float(np.max(dfit)) if dfit else None}
    line = {
        "metric": "served SaCD solves/s",
        "value": len(ok) / wall,
        "unit": "solves/s",
        "latency": summ,
        "jobs": len(specs),
        "completed": len(ok),
        "failed": len(res) - len(ok),
        "wall_s": wall,
        "same_alone_and_in_mix": bool(same),
        "peak_device_bytes": st["peak_bytes"],
        "server_steps": st["steps"],
        "one_at_a_time_fp32": base,
        "config": {"workload": f"Poisson arrivals {args.rate}/s, {len(specs)} jobs, N in {{3,4}}, dims log-uniform "
                               f"[500,100000], nnz log-uniform [50k,5M], Zipf(1.1), R in {{16,32,64}}, BF16 gathers, "
                               f"{iters} iterations, {args.budget_gb} GiB budget, {len(tensors)} distinct tensors",
                   "nnz_per_job_mean": float(np.mean([tensors[t].nnz for t, _, _ in jobs]))},
    }
    print(json.dumps(line), flush=True)
    return 0


def _gen_job_tensor(w):
    from paper_2003_03572_gb300 import synth

    return synth.sparse_tensor(w.dims, w.nnz, dist=w.dist, zipf_s=w.zipf_s, values=w.values, seed=w.seed)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--e2e-reps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--kernels-only", action="store_true", help="skip the end-to-end and CPU legs (profiling)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="with --kernels-only: keep this fraction of the workload's nonzeros (same dims and rank), "
                         "for profiler captures of a smaller case")
    ap.add_argument("--cpu-baseline-child", action="store_true")
    ap.add_argument("--batched", action="store_true", help="the many-small-jobs workload (batched vs one at a time)")
    ap.add_argument("--jobs", type=int, default=512)
    ap.add_argument("--serve", action="store_true", help="the served workload (Poisson arrivals, continuous batching)")
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--pool", type=int, default=64)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-baseline", action="store_true", help="also serve the stream one job at a time, FP32")
    args = ap.parse_args()
    if args.cpu_baseline_child:
        cpu_baseline_child(args.workload, args.steps)
        return 0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return reference_arm(args)
    if args.batched:
        return batched_arm(args)
    if args.serve:
        return serve_arm(args)
    return ours_arm(args)


if __name__ == "__main__":
    sys.exit(main())
