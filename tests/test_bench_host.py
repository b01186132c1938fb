"""Host-side logic of bench.py: the replicas' timing aggregation across ranks (2 gloo ranks on
CPU) and the reference arm's JSON line (the FP64 oracle on a small workload)."""

import json
import os
import socket
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, q):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local_ms = [120.0, 150.0][rank]
    ms = bench.aggregate_over_ranks(local_ms, ws, "cpu")
    q.put((rank, ms, bench.replicas_value(30, ws, ms / 1e3)))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_sum_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    out = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == 150.0
        assert value == pytest.approx(2 * 30 / 0.150)
    assert bench.aggregate_over_ranks(7.0, 1) == 7.0


def test_reference_arm_json_line():
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                        "uniform-100^3-r5", "--steps", "3", "--warmup", "3"], capture_output=True, text=True,
                       timeout=600, env=dict(os.environ, CUDA_VISIBLE_DEVICES=""))
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "mode-steps/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    # per mode, the full-workload step time extrapolated from the two samples
    ms = line["full_step_ms_by_mode"]
    assert len(ms) == 3 and all(x > 0 for x in ms)
    assert line["value"] == pytest.approx(3 / (sum(ms) / 1e3), rel=1e-2)


def test_update_roofline_arithmetic():
    """Select/update roofline: 20 B per element (22 with the BF16 mirror) over pass 1 + pass 2,
    and R FP32 operations per element over pass 1 (10 R when compensated), against the stated
    peaks."""
    from paper_2003_03572_gb300 import synth

    w = synth.WORKLOADS["zipf1.1-50000x20000x500-5M-r32"]
    E = sum(w.dims) * w.rank
    km = {"pass1_grad_importance": 2.0, "pass2_select_update": 3.0}  # ms over 4 steps
    r = bench.update_roofline(w, False, km, 4, 6765.7)
    assert r["elements_per_step"] == E
    assert r["achieved_gbs"] == pytest.approx(4 * E * 20 / 5e-3 / 1e9)
    assert r["frac_hbm"] == pytest.approx(r["achieved_gbs"] / 6765.7)
    assert r["pass1"]["achieved_tops"] == pytest.approx(4 * E * 32 / 2e-3 / 1e12)  # one FMA per product
    rc = bench.update_roofline(w, False, km, 4, 6765.7, compensated=True)
    assert rc["pass1"]["achieved_tops"] == pytest.approx(4 * E * 32 * 10 / 2e-3 / 1e12)
    assert r["pass1"]["peak_tops"] == pytest.approx(152 * 128 * 2.07e9 / 1e12)
    assert bench.update_roofline(w, True, km, 4, 6765.7)["bytes_per_element"] == 22
    assert bench.update_roofline(w, False, {}, 4, 6765.7) is None
    # the fused kernel: both phases form A H (2R FMAs per element)
    rf = bench.update_roofline(w, False, {"select_update": 1.0}, 4, 6765.7)
    assert rf["achieved_gbs"] == pytest.approx(4 * E * 20 / 1e-3 / 1e9)
    assert rf["select_update"]["achieved_tops"] == pytest.approx(4 * E * 64 / 1e-3 / 1e12)


def test_traffic_is_per_workload_and_per_kernel_source():
    """The roofline's DRAM traffic comes from the committed ncu summary of the same workload, and
    only while the MTTKRP source is the one that was captured."""
    import hashlib

    sha = hashlib.sha256(open(os.path.join(bench.ROOT, "paper_2003_03572_gb300", "csrc", "mttkrp.cu"), "rb").read())
    sha = sha.hexdigest()
    t5 = bench.traffic_from_profile(sha, "zipf1.1-50000x20000x500-5M-r32")
    t50 = bench.traffic_from_profile(sha, "zipf1.2-200000x100000x10000x200-50M-r64-bf16")
    if t5 is not None:  # captured on this source
        assert 50e6 < t5 < 200e6  # ~ the compulsory stream of 5M sorted nonzeros (16 B each)
        assert t50 is None or t50 > 10 * t5
    assert bench.traffic_from_profile(sha, "no-such-workload") is None
    assert bench.traffic_from_profile("0" * 64, "zipf1.1-50000x20000x500-5M-r32") is None
