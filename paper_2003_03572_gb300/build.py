"""Build libsacd.so in-tree for sm_103a with nvcc (no cmake, no torch extension machinery).

Each .cu translation unit is compiled in parallel, then linked into
``paper_2003_03572_gb300/libsacd.so``. Used by ``__graft_entry__.build()``.
"""

from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libsacd.so")
SOURCES = ["prep.cu", "mttkrp.cu", "update.cu", "selupd.cu", "gram_tc.cu", "sacd.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def flags(extra=()):
    return [
        *ARCH,
        "-O3",
        "-lineinfo",
        "-std=c++17",
        "-Xcompiler",
        "-fPIC,-O2",
        "-I" + os.path.join(ROOT, "include"),
        "-I" + CSRC,
        "-I" + BUILD,
        *extra,
    ]


def _compile(src, verbose, extra):
    obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), "-c", os.path.join(CSRC, src), "-o", obj, *flags(extra)]
    if verbose:
        cmd.append("-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    return obj, (r.stdout + r.stderr)


TUNING = os.path.join(PKG, "tuning.json")
TUNE_HEADER = os.path.join(BUILD, "tune_table.h")


def write_tune_header():
    """Turn the autotuned table (tuning.json, written by autotune.py on a GB300) into the C header
    the library compiles in. Without a table the header holds only a sentinel entry."""
    import json

    rows = []
    if os.path.exists(TUNING):
        for e in json.load(open(TUNING))["entries"]:
            rows.append(f"  {{{int(e['prec'])}, {int(e['rv'])}, {int(e['nother'])}, {int(e['nnz_lo'])}LL, "
                        f"{int(e['nnz_hi'])}LL, {int(e['sub'])}}},")
    rows.append("  {-1, 0, 0, 0LL, 0LL, 0},  // sentinel")
    text = ("// Generated by paper_2003_03572_gb300/build.py from tuning.json (written by autotune.py).\n"
            "#pragma once\n#include <stdint.h>\n"
            "struct TuneEntry {\n  int prec, rv, nother;\n  int64_t nnz_lo, nnz_hi;\n  int sub;\n};\n"
            "static const TuneEntry kTuneTable[] = {\n" + "\n".join(rows) + "\n};\n")
    old = open(TUNE_HEADER).read() if os.path.exists(TUNE_HEADER) else None
    if old != text:
        with open(TUNE_HEADER, "w") as f:
            f.write(text)


def build(verbose=False, extra=()):
    """Compile every CUDA source and link libsacd.so. Returns the library path."""
    os.makedirs(BUILD, exist_ok=True)
    write_tune_header()
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, verbose, extra), SOURCES))
    objs = [o for o, _ in results]
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    if verbose:
        for _, log in results:
            sys.stdout.write(log)
    return LIB


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
