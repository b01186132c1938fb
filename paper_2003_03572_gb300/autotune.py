"""Autotuner of the MTTKRP tile schedule, run on a GB300.

The MTTKRP cuts the mode-n sorted nonzeros into warp tiles of (32 / LPR) lane groups x ``sub``
nonzeros (``sacd_set_tiling``). Small ``sub`` gives more, shorter tiles (more parallelism, more
rows split across tiles and so more fix-up work); large ``sub`` the reverse. This sweeps ``sub``
over representative synthetic shapes, times the MTTKRP and its fix-up with the library's event
timer, and writes ``tuning.json``: for each (precision, 16-byte vectors per row, number of other
modes, nonzero-count bucket) the fastest ``sub``. The build compiles the table into the library,
and context creation looks it up from the job's own shape only, so a job's tiling (and thus its
results) never depends on what else runs.

    python -m paper_2003_03572_gb300.autotune [--quick]
"""

from __future__ import annotations

import argparse
import json
import os
import time

import numpy as np

from . import sacd as S
from . import synth

SUBS = (8, 16, 32, 64, 128, 256)
BUCKETS = ((0, 150_000), (150_000, 1_500_000), (1_500_000, 15_000_000), (15_000_000, 2**31))
OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tuning.json")


def shapes(quick=False):
    out = []
    nnzs = (50_000, 500_000, 5_000_000, 20_000_000) if not quick else (50_000, 500_000)
    for R in (8, 16, 32, 64):
        for N in (3, 4):
            for prec in (S.SACD_FP32, S.SACD_BF16_GATHER):
                if prec == S.SACD_BF16_GATHER and R < 16:
                    continue
                for nnz in nnzs:
                    if nnz > 5_000_000 and R < 32:  # the largest bucket only for the wide ranks
                        continue
                    if N == 3:
                        dims = (max(1000, nnz // 40), max(500, nnz // 100), 300)
                    else:
                        dims = (max(1000, nnz // 40), max(500, nnz // 100), 200, 40)
                    out.append((dims, nnz, R, prec))
    return out


def rv_of(R, prec):
    Rp = 8
    while Rp < R:
        Rp *= 2
    return Rp // (4 if prec == S.SACD_FP32 else 8)


def time_mode(g, mode, steps):
    S.sacd_profile_enable(g.ctx, True)
    for _ in range(steps):
        g.mode_step(mode, want_count=False)
    st = S.sacd_profile_read(g.ctx)
    S.sacd_profile_enable(g.ctx, False)
    return (st["mttkrp"][1] + st["mttkrp_fixup"][1]) / steps


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--out", default=OUT)
    args = ap.parse_args(argv)
    records = []
    t0 = time.time()
    for dims, nnz, R, prec in shapes(args.quick):
        idx, vals = synth.sparse_tensor(dims, nnz, dist="zipf", zipf_s=1.1, seed=nnz + R)
        init = synth.init_factors(dims, R, 1)
        with S.SaCD(dims, idx, vals, R, init, precision=prec) as g:
            default = [g.info["tile_nnz"][n] for n in range(len(dims))]
            for n in range(len(dims)):  # warm-up
                g.mode_step(n, want_count=False)
            times = {}
            for sub in SUBS:
                tot = 0.0
                for n in range(len(dims)):
                    S.sacd_set_tiling(g.ctx, n, sub)
                    tot += time_mode(g, n, args.steps)
                times[sub] = tot
        records.append(dict(dims=list(dims), nnz=nnz, R=R, prec=prec, rv=rv_of(R, prec), nother=len(dims) - 1,
                            ms=times, default_tile_nnz=default))
        print(f"{dims} nnz={nnz} R={R} prec={prec}: " + " ".join(f"{k}:{v:.3f}" for k, v in times.items()), flush=True)
    # per key: the sub with the least total time over the key's shapes
    entries = []
    keys = sorted({(r["prec"], r["rv"], r["nother"]) for r in records})
    for prec, rv, nother in keys:
        for lo, hi in BUCKETS:
            rs = [r for r in records if (r["prec"], r["rv"], r["nother"]) == (prec, rv, nother) and lo <= r["nnz"] < hi]
            if not rs:
                continue
            tot = {sub: sum(r["ms"][sub] for r in rs) for sub in SUBS}
            best = min(tot, key=tot.get)
            entries.append(dict(prec=prec, rv=rv, nother=nother, nnz_lo=lo, nnz_hi=hi, sub=best,
                                ms_best=tot[best], ms_by_sub=tot))
    out = dict(device="GB300", note="sub = nonzeros per lane group of an MTTKRP warp tile; times are the MTTKRP "
                                    "and its fix-up per mode step summed over the modes of each shape (ms)",
               subs=list(SUBS), entries=entries, records=records, seconds=time.time() - t0)
    with open(args.out, "w") as f:
        json.dump(out, f, indent=1)
    print(f"wrote {args.out}: {len(entries)} entries")


if __name__ == "__main__":
    main()
