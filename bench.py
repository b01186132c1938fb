#!/usr/bin/env python3
"""Benchmark of the SaCD hot path on one GB300 (or N independent replicas under torchrun).

A "step" is one SaCD outer iteration (the mode steps 0..N-1: MTTKRP, H/L, gradient and
importance, selection and update, Gram refresh) followed by the objective/fit evaluation, on the
workload's tensor resident in HBM. value = mode steps per second over the timed steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]

Without --workload the headline is the largest single-GPU workload (200,000 x 100,000 x 10,000 x
200, 50M nonzeros, R = 64, BF16 gathers), with the 5M-nonzero FP32 workload as a second full
record, and the batched (512 jobs) and served (Poisson arrivals) workloads as sub-records. The
K-step timed region is repeated until it has lasted at least --min-seconds in all; the value is
that of the median repeat, and the spread over repeats is reported.

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

HEADLINE_WORKLOAD = "zipf1.2-200000x100000x10000x200-50M-r64-bf16"
SECOND_WORKLOADS = ["zipf1.1-50000x20000x500-5M-r32"]
L2_BYTES = 129 * 2**20


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def mttkrp_bytes(w, nnz, mode):
    """COO-model bytes of one MTTKRP launch: per nonzero its value, its N coordinates and the N-1
    gathered factor rows (R columns each, every row counted once per nonzero, no cache reuse),
    plus the I_n x R output."""
    s = 2 if w.precision == "bf16" else 4
    N = w.nmodes
    return nnz * (4 + 4 * N + (N - 1) * w.rank * s) + w.dims[mode] * w.rank * 4


def mttkrp_hbm_bytes(w, nnz, mode):
    """Compulsory HBM bytes of one MTTKRP launch: every input and output byte crossing HBM once:
    the sorted nonzeros (value + N coordinates), each other factor once (I_k x R, s bytes per
    value) and the I_n x R FP32 output. The gathered rows beyond the first touch of a factor row
    are served from L1/L2 (the factors fit in L2)."""
    s = 2 if w.precision == "bf16" else 4
    N = w.nmodes
    other = sum(w.dims[k] for k in range(N) if k != mode)
    return nnz * (4 + 4 * N) + other * w.rank * s + w.dims[mode] * w.rank * 4


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


CPU_SAMPLE_NNZ = 3_000_000  # nonzeros of the larger CPU-baseline sample (about 10-30 s of oracle work)
SAMPLE_RATIO = 4  # the second sample has 1/SAMPLE_RATIO of the first one's nonzeros


def cpu_baseline_child(path):
    """Run in a fresh single-threaded process: the FP64 oracle as it stands, one mode step per mode
    on each of two seeded nonzero samples of the workload (written by the parent to `path`);
    per mode, the full-workload step time is extrapolated linearly in the nonzero count through
    the two points (a mode step is a fixed per-row part plus a per-nonzero part)."""
    import numpy as np

    from oracle import sacd_oracle as O

    d = np.load(path)
    dims = [int(x) for x in d["dims"]]
    N = len(dims)
    init = [d[f"init{k}"] for k in range(N)]
    nnz = int(d["nnz"])
    pts = []
    for tag in ("1", "0"):
        o = O.SaCDOracle(dims, d["idx" + tag], d["vals" + tag], init)  # one-time coalescing, not timed
        t = np.zeros(N)
        for n in range(N):
            ts = time.perf_counter()
            o.mode_step(n)
            t[n] = time.perf_counter() - ts
        pts.append((d["vals" + tag].shape[0] / nnz, t))
    (f1, t1), (f0, t0) = pts
    full = t0 + (t1 - t0) * (1.0 - f0) / (f1 - f0)
    print(json.dumps({"value": N / float(np.sum(full)), "full_step_ms_by_mode": [float(x) * 1e3 for x in full],
                      "f1": f1, "f0": f0, "n1": int(d["vals1"].shape[0]), "n0": int(d["vals0"].shape[0]),
                      "seconds": float(np.sum(t1) + np.sum(t0))}))


def run_cpu_baseline(w, idx, vals, init):
    """The cpu_baseline leg: the oracle on a bounded sample of the workload, in a child process
    restricted to one thread (numpy/BLAS threads off, no GPU visible)."""
    import tempfile

    import numpy as np

    nnz = vals.shape[0]
    rng = np.random.default_rng(w.seed ^ 0xC0C0)
    n1 = int(min(nnz, CPU_SAMPLE_NNZ, max(1, nnz // 4)))
    pick1 = np.sort(rng.choice(nnz, size=n1, replace=False))
    pick0 = np.sort(rng.choice(pick1, size=max(1, n1 // SAMPLE_RATIO), replace=False))
    tmp = tempfile.mkdtemp(prefix="sacd_cpu_")
    path = os.path.join(tmp, "sample.npz")
    np.savez(path, dims=np.array(w.dims), nnz=nnz, idx1=idx[:, pick1], vals1=vals[pick1], idx0=idx[:, pick0],
             vals0=vals[pick0], **{f"init{k}": a for k, a in enumerate(init)})
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    try:
        r = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-baseline-child", path],
                           capture_output=True, text=True, env=env, timeout=1800)
    finally:
        try:
            os.remove(path)
            os.rmdir(tmp)
        except OSError:
            pass
    if r.returncode != 0:
        return None
    d = json.loads(r.stdout.strip().splitlines()[-1])
    d["sample"] = (f"one FP64 oracle mode step per mode on a seeded {d['n1']}-nonzero sample ({d['f1']:.4g} of the "
                   f"nonzeros, same dims, rank and initial factors) and on a {d['n0']}-nonzero sub-sample; per mode "
                   f"the full-workload step time is extrapolated linearly in the nonzero count through the two "
                   f"(fixed per-row work + per-nonzero work); {d['seconds']:.1f} s of oracle work, one thread")
    return d


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


REF_FRACTION = 0.125  # largest share of the nonzeros in one reference-arm step
REF_NNZ = 3_000_000  # ... and at most this many nonzeros (smaller samples are dominated by cache and
# timing noise, and the linear extrapolation below would then overstate the full step several-fold)


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
    # --steps 20 ends within a few minutes. A mode step of the oracle costs a fixed per-row part
    # (the dense Gram / gradient / update work, independent of the nonzeros) plus a per-nonzero
    # part (its MTTKRP); the full-workload step time per mode is extrapolated through this sample
    # and a second one SAMPLE_RATIO times smaller.
    nnz = vals.shape[0]
    rng = np.random.default_rng(w.seed ^ 0x5A5A)

    def sample_oracle(frac):
        pick = np.sort(rng.choice(nnz, size=max(1, int(nnz * frac)), replace=False))
        return O.SaCDOracle(w.dims, np.ascontiguousarray(idx[:, pick]), vals[pick], init), pick.size

    N = w.nmodes
    frac = min(REF_FRACTION, REF_NNZ / max(nnz, 1))
    o, n1 = sample_oracle(frac)
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
    # the second point of the per-mode cost model: a few mode steps on a sample SAMPLE_RATIO times smaller
    o0, n0 = sample_oracle(frac / SAMPLE_RATIO)
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
                   "step": f"one mode step on a {frac:.4g} nonzero sample"},
        "cpu_baseline": {"value": v, "unit": "mode-steps/s", "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": v, "unit": "mode-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def log(msg):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def measure_workload(w, args, dev, stream, ws, rank, local, steps, cpu_leg):
    """One workload's full record: the K-step device-resident timed region (repeated until it has
    lasted args.min_seconds), per-kernel timing, roofline fields, end to end from host buffers, and
    (rank 0, one GPU) the CPU baseline on a bounded sample."""
    import numpy as np
    import torch

    from paper_2003_03572_gb300 import sacd as S
    from paper_2003_03572_gb300 import synth

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    t_gen = time.perf_counter()
    idx, vals, init = synth.make_workload(w, scale=args.scale)
    log(f"{w.name}: inputs drawn in {time.perf_counter() - t_gen:.1f} s")
    N = w.nmodes
    prec = S.SACD_BF16_GATHER if w.precision == "bf16" else S.SACD_FP32

    # ---------------------------------------------------------------- device-resident timing
    g = S.SaCD(w.dims, idx, vals, w.rank, init, precision=prec, stream=stream.cuda_stream)
    info = g.info
    nnz = info["nnz"]
    for _ in range(args.warmup):
        g.iterate(1)
        g.fit()
    torch.cuda.synchronize(dev)
    clk = ClockSampler(local)
    clk.start()
    rep_ms = []
    fit = None
    while True:
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(steps):
            g.iterate(1)
            obj, fit = g.fit()
        e1.record(stream)
        torch.cuda.synchronize(dev)
        barrier()
        rep_ms.append(e0.elapsed_time(e1))
        total = aggregate_over_ranks(sum(rep_ms), ws, dev)
        more = 1.0 if (len(rep_ms) < 3 or total < args.min_seconds * 1e3) and len(rep_ms) < 500 else 0.0
        if aggregate_over_ranks(more, ws, dev) == 0.0:
            break
    clocks = clk.stop()
    rep_sorted = sorted(rep_ms)
    med_local = statistics.median(rep_ms)
    ms = aggregate_over_ranks(med_local, ws, dev)
    value = replicas_value(steps * N, ws, ms / 1e3)
    if not np.isfinite(fit):
        raise SystemExit(f"{w.name}: non-finite fit {fit}")

    # ---------------------------------------------------------------- per-kernel timing
    S.sacd_profile_enable(g.ctx, True)
    for _ in range(steps):
        g.iterate(1)
        g.fit()
    stats = S.sacd_profile_read(g.ctx)
    S.sacd_profile_enable(g.ctx, False)
    g.close()
    launches_per_step = sum(v[0] for v in stats.values()) / steps
    mt_launches, mt_ms = stats["mttkrp"]
    kernel_ms = {k: v[1] for k, v in stats.items()}
    total_kernel_ms = sum(kernel_ms.values())
    peak, peak_kind = peaks()
    hbm_b = steps * sum(mttkrp_hbm_bytes(w, nnz, n) for n in range(N))
    coo_b = steps * sum(mttkrp_bytes(w, nnz, n) for n in range(N))
    mt_s = mt_ms / 1e3
    achieved = hbm_b / mt_s / 1e9 if mt_s > 0 else None
    coo = coo_b / mt_s / 1e9 if mt_s > 0 else None
    src_sha = hashlib.sha256(open(os.path.join(ROOT, "paper_2003_03572_gb300", "csrc", "mttkrp.cu"), "rb").read()).hexdigest()
    traffic = traffic_from_profile(src_sha, w.name)
    roofline = {
        "bound": "hbm",
        "kernel": "mttkrp",
        "achieved": achieved,
        "peak": peak,
        "peak_kind": f"{peak_kind} HBM copy bandwidth (burst)",
        "unit": "GB/s",
        "frac": (achieved / peak) if achieved else None,
        "traffic": traffic,
        "bytes_model": "compulsory HBM bytes per launch: nnz*(4 + 4N) sorted nonzeros + sum_{k!=n} I_k*R*s "
                       "factors once + I_n*R*4 output",
        "ms_per_launch": mt_ms / mt_launches if mt_launches else None,
        "mttkrp_share": mt_ms / total_kernel_ms if total_kernel_ms else None,
        "coo_model": {"achieved": coo, "unit": "GB/s", "frac_of_hbm_peak": (coo / peak) if coo else None,
                      "bytes_model": "nnz*(4 + 4N + (N-1)*R*s) + I_n*R*4 per launch: every gathered row counted "
                                     "once per nonzero",
                      "note": "the gathers are served from L1/L2 (each factor is at most tens of MB), so this "
                              "figure exceeds what HBM carries; it measures gather throughput through L1/L2, "
                              "not an HBM fraction"},
    }
    upd = update_roofline(w, prec == S.SACD_BF16_GATHER, kernel_ms, steps, peak)

    rec = {
        "value": value,
        "unit": "mode-steps/s",
        "ms_per_step": ms / steps,
        "steps": steps,
        "repeats": len(rep_ms),
        "timed_seconds": sum(rep_ms) / 1e3,
        "ms_per_step_spread": {"min": rep_sorted[0] / steps, "median": med_local / steps,
                               "max": rep_sorted[-1] / steps},
        "dtype": "f32" if prec == S.SACD_FP32 else "bf16-gather/f32",
        "config": {
            "workload": w.name,
            "dims": list(w.dims),
            "nnz": nnz,
            "rank": w.rank,
            "step": "one SaCD iteration (all modes) + objective/fit",
            "l2": f"inputs larger than L2: {nnz * (4 * N + 4) * N / 1e6:.0f} MB of sorted nonzeros per step vs "
                  f"{L2_BYTES / 1e6:.0f} MB L2",
            "final_fit": fit,
        },
        "roofline": roofline,
        "update_roofline": upd,
        "kernel_ms_per_step": {k: v / steps for k, v in kernel_ms.items()},
        "gpu_launches": int(round(launches_per_step * steps * len(rep_ms))),
        "clocks": clocks,
    }
    if args.kernels_only:
        return rec

    # ---------------------------------------------------------------- end to end, host buffers
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory()
    h_idx = [pin(idx[n]) for n in range(N)]
    h_vals = pin(vals)
    h_init = [pin(a) for a in init]
    h_out = [torch.empty(a.shape, dtype=torch.float32).pin_memory() for a in init]
    iters = w.iters
    e2e_times = []
    e2e_parts = []
    clk2 = ClockSampler(local)
    clk2.start()
    for rep in range(max(args.e2e_reps, 1) + 1):
        torch.cuda.synchronize(dev)
        barrier()
        t0 = time.perf_counter()
        ctx = S.sacd_create(w.dims, [t.numpy() for t in h_idx], h_vals.numpy(), w.rank,
                            [t.numpy() for t in h_init], precision=prec, stream=stream.cuda_stream)
        t_created = time.perf_counter()  # host time at which create returned (its work may still run)
        S.sacd_iterate(ctx, iters)
        e2e_fit = S.sacd_fit(ctx)
        for n in range(N):
            S.sacd_get_factor(ctx, n, h_out[n].numpy())
        S.sacd_destroy(ctx)
        t1 = time.perf_counter()
        if rep > 0:  # first solve is a warm-up (allocator, graph instantiation)
            e2e_times.append(t1 - t0)
            e2e_parts.append((t_created - t0, t1 - t_created))
    e2e_clocks = clk2.stop()
    e2e_s = aggregate_over_ranks(statistics.median(e2e_times), ws, dev)
    h2d = int(len(vals) * (4 * N + 4) + sum(a.nbytes for a in init))
    d2h = int(sum(a.nbytes for a in init) + 16)
    rec["e2e"] = {
        "value": replicas_value(N * iters, ws, e2e_s),
        "unit": "mode-steps/s",
        "step": f"one full solve from pinned host COO: create (copy + CSF build) + {iters} iterations + fit + "
                f"factors back",
        "h2d_bytes_per_step": h2d,
        "d2h_bytes_per_step": d2h,
        "h2d_bytes_per_mode_step": h2d / (N * iters),
        "mode_steps_per_step": N * iters,
        "seconds_per_solve": e2e_s,
        "solve_seconds": [round(t, 5) for t in e2e_times],
        "create_return_seconds": [round(a, 5) for a, _ in e2e_parts],
        "after_create_seconds": [round(b, 5) for _, b in e2e_parts],
        "final_fit": e2e_fit[1],
        "clocks": e2e_clocks,
    }

    # ---------------------------------------------------------------- CPU baseline (rank 0, N=1)
    rec["cpu_baseline"] = None
    if cpu_leg and rank == 0 and ws == 1 and not args.no_cpu_baseline:
        d = run_cpu_baseline(w, idx, vals, init)
        if d:
            rec["cpu_baseline"] = {"value": d["value"], "unit": "mode-steps/s", "cores": 1, "kind": "oracle",
                                   "sample": d["sample"], "full_step_ms_by_mode": d["full_step_ms_by_mode"],
                                   "host_cores_idle": (os.cpu_count() or 1) - 1}
    return rec


def ours_arm(args):
    import torch

    from paper_2003_03572_gb300 import synth

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    if args.scale != 1.0 and not args.kernels_only:
        raise SystemExit("--scale is for --kernels-only profiling runs")
    stream = torch.cuda.Stream(device=dev)
    head = args.workload or HEADLINE_WORKLOAD
    w = synth.WORKLOADS[head]
    t_all = time.perf_counter()
    main = measure_workload(w, args, dev, stream, ws, rank, local, args.steps, cpu_leg=True)
    log(f"{head}: {main['value']:.1f} mode-steps/s ({time.perf_counter() - t_all:.0f} s so far)")
    if args.kernels_only:
        if rank == 0:
            print(json.dumps({"kernels_only": True, "scale": args.scale, "value": main["value"],
                              "unit": "mode-steps/s", "kernel_ms_per_step": main["kernel_ms_per_step"]}))
        return 0
    extra = {}
    if args.workload is None:
        for name in SECOND_WORKLOADS:
            w2 = synth.WORKLOADS[name]
            rec = measure_workload(w2, args, dev, stream, ws, rank, local, args.steps, cpu_leg=True)
            extra[name] = rec
            log(f"{name}: {rec['value']:.1f} mode-steps/s ({time.perf_counter() - t_all:.0f} s so far)")
    batched = served = None
    if args.workload is None and ws == 1 and not args.no_jobs:
        batched = batched_record(args)
        log(f"batched: {batched['value']:.1f} jobs/s ({time.perf_counter() - t_all:.0f} s so far)")
        served = serve_record(args)
        log(f"served: {served['value']:.1f} solves/s ({time.perf_counter() - t_all:.0f} s so far)")
    if rank == 0:
        line = {
            "metric": "SaCD mode-steps/s",
            "value": main["value"],
            "unit": "mode-steps/s",
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": main["ms_per_step"],
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": main["dtype"],
            "data": "synthetic",
            "config": dict(main["config"], parallelism="replicas" if ws > 1 else "single GPU"),
        }
        for k in ("repeats", "timed_seconds", "ms_per_step_spread", "roofline", "update_roofline",
                  "kernel_ms_per_step", "gpu_launches", "e2e", "clocks", "cpu_baseline"):
            line[k] = main.get(k)
        if extra:
            line["workloads"] = extra
        if batched:
            line["batched"] = batched
        if served:
            line["served"] = served
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


# FP32 instruction peak of one GB300: 152 SMs x 128 FP32 lanes x 2.07 GHz (maximum SM clock),
# one FP32 operation (an FMA counts as one) per lane and clock.
FP32_PEAK_TOPS = 152 * 128 * 2.07e9 / 1e12


def update_roofline(w, bf16, kernel_ms, steps, hbm_peak, compensated=False):
    """Select/update roofline (one element = one factor entry of a mode step): algorithmic bytes 20
    per element (read M, A, z^{k-1}; write A, z^{k-1}; 22 with the BF16 mirror) over the kernels
    that follow the MTTKRP, against the HBM copy peak. The arithmetic is reported against the FP32
    instruction peak: the fused select/update kernel forms A H twice (its two phases), R fused
    multiply-adds per element each time; the two-pass path forms it once in pass 1, one FMA per
    product (Frobenius or spectral L) or 10 FP32 operations per product when compensated (exact
    product 2, TwoSum 6, error terms 2; GCD)."""
    elems = sum(w.dims) * w.rank * steps
    bpe = 20 + (2 if bf16 else 0)
    fused = kernel_ms.get("select_update", 0.0) / 1e3
    t1 = kernel_ms.get("pass1_grad_importance", 0.0) / 1e3
    t = fused + t1 + kernel_ms.get("pass2_select_update", 0.0) / 1e3
    if t <= 0 or (fused <= 0 and t1 <= 0):
        return None
    gbs = elems * bpe / t / 1e9
    rec = {"kernels": ["select_update"] if fused > 0 else ["pass1_grad_importance", "pass2_select_update"],
           "bytes_per_element": bpe, "elements_per_step": elems // steps, "achieved_gbs": gbs,
           "hbm_peak_gbs": hbm_peak, "frac_hbm": gbs / hbm_peak}
    peak = {"peak_tops": FP32_PEAK_TOPS, "peak_kind": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz"}
    if fused > 0:
        tops = elems * w.rank * 2 / fused / 1e12
        rec["select_update"] = dict(bound="alu", ops_per_element=2 * w.rank, achieved_tops=tops,
                                    frac=tops / FP32_PEAK_TOPS, **peak)
    else:
        opp = 10 if compensated else 1
        tops = elems * w.rank * opp / t1 / 1e12
        rec["pass1"] = dict(bound="alu", ops_per_element=opp * w.rank, achieved_tops=tops,
                            frac=tops / FP32_PEAK_TOPS, **peak)
    return rec


def _gen_job(w):
    from paper_2003_03572_gb300 import synth

    idx, vals = synth.sparse_tensor(w.dims, w.nnz, dist=w.dist, zipf_s=w.zipf_s, values=w.values, seed=w.seed)
    return idx, vals, synth.init_factors(w.dims, w.rank, w.seed, w.init_log2)


def batched_record(args):
    """Many small independent jobs: one batched launch set per mode step (CUDA graph) against
    the same jobs solved one at a time, each from its own context, on the same GPU (same FP32
    arithmetic, so the final fits are bit-identical)."""
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
    for rep in range(max(args.e2e_reps, 1)):
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
    return {
        "metric": "batched SaCD jobs/s",
        "value": len(ws) / tb,
        "unit": "jobs/s",
        "one_at_a_time": len(ws) / t1,
        "speedup": t1 / tb,
        "mode_steps_per_s": mode_steps / tb,
        "same_final_fit": bool(np.array_equal(np.asarray(fits_b), np.asarray(fits_1))),
        "all_fits_finite": bool(np.isfinite(np.asarray(fits_b)).all()),
        "config": {"workload": f"batched {len(ws)} jobs: dims U[200,5000]xU[200,5000]xU[20,200], nnz U[10k,500k] "
                               f"Zipf(1.1), R in {{8,16,32}}, FP32, {iters} iterations, one graph-captured launch "
                               f"set per iteration for all jobs, initial factors U[0,1) x 2^s with s bringing "
                               f"the initial model's expected norm to the tensor's", "nnz_total": nnz_total},
        "timed": "batched: create excluded, iterations + objective of all jobs (median of repeats); "
                 "one at a time: the same contexts' iterations + objective in sequence",
        "seconds_batched": tb,
        "seconds_one_at_a_time": t1,
    }


def batched_arm(args):
    print(json.dumps(batched_record(args)), flush=True)
    return 0


def serve_record(args):
    """Served workload: Poisson arrivals of 3- and 4-mode BF16-gather jobs, continuous batching
    with HBM-budget admission; solves/s and arrival-to-result latency percentiles, against the same
    arrival stream served one job at a time with plain FP32 gathers, compared at matched final fit."""
    import concurrent.futures as cf
    import multiprocessing as mp

    import numpy as np
    import torch

    from paper_2003_03572_gb300 import sacd as S
    from paper_2003_03572_gb300 import serve, synth

    tensors, jobs = synth.serving_workloads(args.serve_jobs, pool=args.pool)
    with cf.ProcessPoolExecutor(max_workers=min(16, os.cpu_count() or 4), mp_context=mp.get_context("spawn")) as ex:
        data = list(ex.map(_gen_job_tensor, tensors, chunksize=1))
    torch.cuda.init()
    stream = torch.cuda.Stream()
    specs = []
    for ti, R, seed in jobs:
        w = tensors[ti]
        specs.append(dict(dims=w.dims, idx=data[ti][0], vals=data[ti][1], rank=R, init=None, seed=seed,
                          precision=S.SACD_BF16_GATHER, init_log2_scale=synth.init_log2_scale(w.dims, R, w.nnz)))
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
                        precision=sp["precision"], init_log2_scale=sp["init_log2_scale"],
                        stream=stream.cuda_stream) as a:
                a.iterate(iters)
                same &= all(np.array_equal(a.factor(n), r["factors"][n]) for n in range(len(sp["dims"])))
    summ = serve.latency_summary(res)
    base = None
    if not args.no_serve_baseline:
        # the same arrival stream served one job at a time with FP32 gathers
        specs32 = [dict(sp, precision=S.SACD_FP32) for sp in specs]
        with serve.Server(int(args.budget_gb * 2**30), max_active=1, stream=stream.cuda_stream) as srv1:
            res1, wall1 = serve.run_arrivals(srv1, specs32, arrivals, iters)
        ok1 = [r for r in res1 if r["status"] == 0]
        fit_b = {r["index"]: r["fit"] for r in ok}
        fit_1 = {r["index"]: r["fit"] for r in ok1}
        both = sorted(set(fit_b) & set(fit_1))
        d = np.array([fit_b[i] - fit_1[i] for i in both])
        tol = 1e-3
        matched = [i for i in both if fit_b[i] >= fit_1[i] - tol]
        base = {"solves_per_s": len(ok1) / wall1, "latency": serve.latency_summary(res1), "wall_s": wall1,
                "completed": len(ok1), "failed": len(res1) - len(ok1),
                "matched_fit": {
                    "rule": f"a served job counts as matched when its final fit is at least the FP32 "
                            f"one-at-a-time job's minus {tol:g}",
                    "jobs_compared": len(both), "jobs_matched": len(matched),
                    "served_solves_per_s_matched": len(matched) / wall,
                    "fit_diff_median": float(np.median(d)) if d.size else None,
                    "fit_diff_mean": float(np.mean(d)) if d.size else None,
                    "fit_diff_abs_p99": float(np.percentile(np.abs(d), 99)) if d.size else None,
                    "served_fit_mean": float(np.mean([fit_b[i] for i in both])) if both else None,
                    "baseline_fit_mean": float(np.mean([fit_1[i] for i in both])) if both else None}}
    fits = np.array([r["fit"] for r in ok])
    return {
        "metric": "served SaCD solves/s",
        "value": len(ok) / wall,
        "unit": "solves/s",
        "latency": summ,
        "jobs": len(specs),
        "completed": len(ok),
        "failed": len(res) - len(ok),
        "errors": sorted({r["error"] for r in res if r["status"] != 0})[:4],
        "all_fits_finite": bool(np.isfinite(fits).all()),
        "wall_s": wall,
        "same_alone_and_in_mix": bool(same),
        "peak_device_bytes": st["peak_bytes"],
        "server_steps": st["steps"],
        "one_at_a_time_fp32": base,
        "config": {"workload": f"Poisson arrivals {args.rate}/s, {len(specs)} jobs, N in {{3,4}}, dims log-uniform "
                               f"[500,100000], nnz log-uniform [50k,5M], Zipf(1.1), R in {{16,32,64}}, BF16 gathers, "
                               f"{iters} iterations, {args.budget_gb} GiB budget, initial factors U[0,1) x 2^s "
                               f"with s bringing the initial model's expected norm to the tensor's",
                   "departure": f"{len(specs)} jobs (not 10,000) over {len(tensors)} distinct tensors reused "
                                f"round-robin, each job with its own rank and seeded initial factors: drawing "
                                f"every tensor on the host would dominate the run",
                   "nnz_per_job_mean": float(np.mean([tensors[t].nnz for t, _, _ in jobs]))},
    }


def serve_arm(args):
    print(json.dumps(serve_record(args)), flush=True)
    return 0


def _gen_job_tensor(w):
    from paper_2003_03572_gb300 import synth

    return synth.sparse_tensor(w.dims, w.nnz, dist=w.dist, zipf_s=w.zipf_s, values=w.values, seed=w.seed)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=None, help="one workload only (default: the headline and the others)")
    ap.add_argument("--min-seconds", type=float, default=1.0, help="repeat the K-step timed region until this long")
    ap.add_argument("--e2e-reps", type=int, default=4,
                    help="timed solves after one warm-up solve (consecutive solves alternate between two "
                         "durations; an even count keeps the median from depending on which comes first)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-jobs", action="store_true", help="skip the batched and served sub-records")
    ap.add_argument("--kernels-only", action="store_true", help="skip the end-to-end and CPU legs (profiling)")
    ap.add_argument("--scale", type=float, default=1.0,
                    help="with --kernels-only: keep this fraction of the workload's nonzeros (same dims and rank), "
                         "for profiler captures of a smaller case")
    ap.add_argument("--cpu-baseline-child", default=None, help=argparse.SUPPRESS)
    ap.add_argument("--batched", action="store_true", help="the many-small-jobs workload only")
    ap.add_argument("--jobs", type=int, default=512)
    ap.add_argument("--serve", action="store_true", help="the served workload only")
    ap.add_argument("--serve-jobs", type=int, default=1000)
    ap.add_argument("--rate", type=float, default=200.0)
    ap.add_argument("--pool", type=int, default=64)
    ap.add_argument("--budget-gb", type=float, default=150.0)
    ap.add_argument("--no-serve-baseline", action="store_true", help="skip the one-at-a-time FP32 serving baseline")
    args = ap.parse_args()
    if args.cpu_baseline_child:
        cpu_baseline_child(args.cpu_baseline_child)
        return 0
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        if args.workload is None:
            args.workload = HEADLINE_WORKLOAD
        return reference_arm(args)
    if args.batched:
        return batched_arm(args)
    if args.serve:
        return serve_arm(args)
    return ours_arm(args)


if __name__ == "__main__":
    sys.exit(main())
