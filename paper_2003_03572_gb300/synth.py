"""Seeded synthetic inputs for SaCD: sparse N-mode tensors and initial factors.

This module only draws inputs. It holds none of the method's arithmetic, so both the
CUDA path (through the C-ABI binding) and the FP64 oracle under ``oracle/`` may be fed
from it. It uses numpy only and never touches the GPU.

The paper's synthetic tensors (Section 6.3) are "randomly generated" with no stated index or
value distribution, and its real data sets (Table 3) are not available. The workloads below
stand in for both: uniform or Zipf-distributed coordinates per mode, de-duplicated to an exact
number of distinct nonzeros, with integer or lognormal values.

Recipe (every draw comes from ``numpy.random.Generator(PCG64(seed))``):

* Zipf(s) on a finite support: P(rank k) proportional to k^-s for k = 1..I_n, sampled by the
  inverse CDF over an FP64 cumulative table; rank k maps to index ``perm_n[k-1]`` through a
  seeded permutation, so the hot rows are scattered over the mode.
* Uniform coordinates: ``integers(0, I_n)`` per mode.
* De-duplication: draw tuples in batches, keep the distinct ones, top up the shortfall until
  at least ``nnz`` are distinct, then keep a seeded random subset of exactly ``nnz``.
* Values: uniform integers 1..5 as FP32, or lognormal(0, 1) rounded to FP32.
* The nonzeros come out in a seeded random order (COO is unsorted on purpose).
* Initial factors: U[0, 1) drawn as ``k * 2^-24`` with k uniform in [0, 2^24), so each value
  is exact in FP32 and FP64 and both sides start from identical numbers. The batched and served
  workloads scale them by a power of two (exact) chosen so that the initial CP model's expected
  norm matches the tensor's (``init_log2_scale``); the other workloads use U[0, 1) as drawn.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Workload",
    "WORKLOADS",
    "sparse_tensor",
    "init_factors",
    "zipf_indices",
    "make_workload",
    "batched_workloads",
    "serving_workloads",
    "init_log2_scale",
]

_I32_MAX = 2**31 - 1


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed) & (2**64 - 1)))


def zipf_indices(rng: np.random.Generator, dim: int, s: float, n: int) -> np.ndarray:
    """Draw ``n`` indices in [0, dim) with P(rank k) ~ k^-s, ranks scattered by a permutation."""
    ranks = np.arange(1, dim + 1, dtype=np.float64)
    cdf = np.cumsum(ranks ** (-float(s)))
    cdf /= cdf[-1]
    u = rng.random(n)
    k = np.searchsorted(cdf, u, side="right")
    np.minimum(k, dim - 1, out=k)
    perm = rng.permutation(dim).astype(np.int64)
    return perm[k]


def _draw_tuples(rng, dims, n, dist, zipf_s):
    cols = []
    for d in dims:
        if dist == "uniform":
            cols.append(rng.integers(0, d, size=n, dtype=np.int64))
        elif dist == "zipf":
            cols.append(zipf_indices(rng, d, zipf_s, n))
        else:
            raise ValueError(f"unknown coordinate distribution {dist!r}")
    return np.stack(cols)  # (N, n) int64


def _linear_keys(tup, dims):
    key = np.zeros(tup.shape[1], dtype=np.int64)
    for k in range(len(dims)):
        key *= np.int64(dims[k])
        key += tup[k]
    return key


def _decode_keys(key, dims):
    out = np.empty((len(dims), key.shape[0]), dtype=np.int64)
    rem = key.copy()
    for k in range(len(dims) - 1, -1, -1):
        out[k] = rem % np.int64(dims[k])
        rem //= np.int64(dims[k])
    return out


def _hash_keys(tup):
    # splitmix64-style mixing of the tuple; only used to detect repeats when the
    # linear key would overflow int64. Equal tuples always hash equal, so the
    # result is always distinct; a (vanishingly rare) false collision only drops a draw.
    h = np.zeros(tup.shape[1], dtype=np.uint64)
    with np.errstate(over="ignore"):
        for k in range(tup.shape[0]):
            h ^= tup[k].astype(np.uint64) + np.uint64(0x9E3779B97F4A7C15) + (h << np.uint64(6)) + (h >> np.uint64(2))
            z = h
            z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
            z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
            h = z ^ (z >> np.uint64(31))
    return h


def sparse_tensor(dims, nnz, *, dist="uniform", zipf_s=1.1, values="int15", seed=0, max_rounds=64):
    """Seeded sparse tensor with exactly ``nnz`` distinct coordinates.

    Returns ``(idx, vals)``: ``idx`` is an (N, nnz) int32 array of 0-based coordinates and
    ``vals`` an (nnz,) float32 array, in a seeded random order.
    """
    dims = [int(d) for d in dims]
    if any(d < 1 or d > _I32_MAX for d in dims):
        raise ValueError("every mode length must be in [1, 2^31-1]")
    cells = math.prod(dims)
    if nnz > cells:
        raise ValueError("more nonzeros requested than cells")
    rng = _rng(seed)
    linear = cells < 2**62
    have_keys = np.zeros(0, dtype=np.int64 if linear else np.uint64)
    have_tup = np.zeros((len(dims), 0), dtype=np.int64)
    rounds = 0
    while have_keys.shape[0] < nnz:
        rounds += 1
        if rounds > max_rounds:
            raise RuntimeError("could not draw enough distinct coordinates")
        need = nnz - have_keys.shape[0]
        m = int(need * 1.25) + 1024
        tup = _draw_tuples(rng, dims, m, dist, zipf_s)
        if linear:
            keys = np.concatenate([have_keys, _linear_keys(tup, dims)])
            keys.sort()
            keep = np.empty(keys.shape[0], dtype=bool)
            keep[:1] = True
            np.not_equal(keys[1:], keys[:-1], out=keep[1:])
            have_keys = keys[keep]
        else:
            keys = np.concatenate([have_keys, _hash_keys(tup)])
            allt = np.concatenate([have_tup, tup], axis=1)
            order = np.argsort(keys, kind="stable")
            keys = keys[order]
            keep = np.empty(keys.shape[0], dtype=bool)
            keep[:1] = True
            np.not_equal(keys[1:], keys[:-1], out=keep[1:])
            have_keys = keys[keep]
            have_tup = allt[:, order[keep]]
    # seeded random subset of exactly nnz, in a seeded random order
    pick = rng.permutation(have_keys.shape[0])[:nnz]
    if linear:
        idx = _decode_keys(have_keys[pick], dims)
    else:
        idx = have_tup[:, pick]
    if values == "int15":
        vals = rng.integers(1, 6, size=nnz).astype(np.float32)
    elif values == "lognormal":
        vals = rng.lognormal(0.0, 1.0, size=nnz).astype(np.float32)
    elif values == "uniform01":
        vals = (rng.integers(0, 2**24, size=nnz) * 2.0**-24).astype(np.float32)
    else:
        raise ValueError(f"unknown value distribution {values!r}")
    return np.ascontiguousarray(idx.astype(np.int32)), vals


def init_factors(dims, rank, seed, log2_scale=0):
    """Nonnegative U[0,1) initial factors, each value k*2^-24 (exact in FP32 and FP64), times
    2^log2_scale (still exact)."""
    rng = _rng(seed ^ 0x1F1F1F1F)
    out = []
    for d in dims:
        k = rng.integers(0, 2**24, size=(int(d), int(rank)))
        out.append(np.ascontiguousarray((k * 2.0 ** (int(log2_scale) - 24)).astype(np.float32)))
    return out


def init_log2_scale(dims, rank, nnz, mean_sq=11.0):
    """Power-of-two scale of U[0,1) initial factors that brings the initial model's expected squared
    norm to the tensor's expected squared norm, nnz * mean_sq (11 for uniform integers 1..5). With
    U[0,1) entries a factor's Gram averages I/3 on its diagonal and I/4 off it, so the model's
    squared norm (the sum over r, s of the product of the Grams) averages about
    R prod_k I_k/3 + R (R-1) prod_k I_k/4; each of the N factors takes an equal share of the scale.
    An input recipe only: nothing here is part of the factorisation."""
    N = len(dims)
    m0 = rank * math.prod(d / 3.0 for d in dims) + rank * (rank - 1) * math.prod(d / 4.0 for d in dims)
    c = math.sqrt(max(nnz, 1) * mean_sq / m0) ** (1.0 / N)
    return int(round(math.log2(c)))


@dataclasses.dataclass(frozen=True)
class Workload:
    """One synthetic SaCD job: tensor shape and distribution, rank, iterations, precision."""

    name: str
    dims: tuple
    nnz: int
    dist: str
    zipf_s: float
    values: str
    rank: int
    iters: int
    precision: str  # "fp32" or "bf16"
    seed: int
    init_log2: int = 0  # initial factors U[0,1) * 2^init_log2

    @property
    def nmodes(self):
        return len(self.dims)


# Seeds are 0x5ACD0000 + workload number.
WORKLOADS = {
    "uniform-100^3-r5": Workload(
        "uniform-100^3-r5", (100, 100, 100), 10_000, "uniform", 0.0, "int15", 5, 20, "fp32", 0x5ACD0000
    ),
    "zipf1.1-50000x20000x500-5M-r32": Workload(
        "zipf1.1-50000x20000x500-5M-r32",
        (50_000, 20_000, 500),
        5_000_000,
        "zipf",
        1.1,
        "int15",
        32,
        50,
        "fp32",
        0x5ACD0001,
    ),
    "zipf1.2-200000x100000x10000x200-50M-r64-bf16": Workload(
        "zipf1.2-200000x100000x10000x200-50M-r64-bf16",
        (200_000, 100_000, 10_000, 200),
        50_000_000,
        "zipf",
        1.2,
        "lognormal",
        64,
        30,
        "bf16",
        0x5ACD0002,
    ),
}


def make_workload(w: Workload, scale: float = 1.0):
    """Draw a workload's tensor and initial factors. ``scale`` shrinks nnz (and nothing else)."""
    nnz = max(1, int(round(w.nnz * scale)))
    idx, vals = sparse_tensor(w.dims, nnz, dist=w.dist, zipf_s=w.zipf_s, values=w.values, seed=w.seed)
    init = init_factors(w.dims, w.rank, w.seed)
    return idx, vals, init


def batched_workloads(njobs=512, seed=0x5ACD0003, nnz_range=(10_000, 500_000), ranks=(8, 16, 32), iters=30):
    """Many independent small 3-mode jobs: dims U[200,5000] x U[200,5000] x U[20,200],
    nnz U[nnz_range], Zipf(1.1) coordinates, rank uniform from ``ranks``, FP32."""
    rng = _rng(seed)
    jobs = []
    for j in range(njobs):
        dims = (int(rng.integers(200, 5001)), int(rng.integers(200, 5001)), int(rng.integers(20, 201)))
        nnz = int(rng.integers(nnz_range[0], nnz_range[1] + 1))
        nnz = min(nnz, math.prod(dims) // 2)
        rank = int(rng.choice(ranks))
        jobs.append(
            Workload(f"job{j}", dims, nnz, "zipf", 1.1, "int15", rank, iters, "fp32", seed * 1000003 + j,
                     init_log2_scale(dims, rank, nnz))
        )
    return jobs


def serving_workloads(njobs, seed=0x5ACD0004, pool=None, iters=30):
    """Jobs of the served workload: N in {3, 4} (p = 1/2 each), every mode length log-uniform in
    [500, 100000], nnz log-uniform in [50k, 5M] (at most half the cells), Zipf(1.1) coordinates,
    R uniform from {16, 32, 64}, BF16 gathers, `iters` iterations. Each job's initial factors are
    drawn on the device from its seed, scaled by 2^init_log2_scale(dims, R, nnz).

    With ``pool`` = P, only P distinct tensors are drawn and job i uses tensor i % P (its own rank
    and initial factors): a stand-in that keeps the shape and size mix while bounding the time
    spent drawing inputs. Returns (tensor workloads, per-job (tensor index, rank, init seed))."""
    rng = _rng(seed)
    P = njobs if pool is None else min(pool, njobs)
    tensors = []
    for t in range(P):
        N = 3 if rng.random() < 0.5 else 4
        dims = tuple(int(round(math.exp(rng.uniform(math.log(500), math.log(100_000))))) for _ in range(N))
        nnz = int(round(math.exp(rng.uniform(math.log(50_000), math.log(5_000_000)))))
        nnz = min(nnz, math.prod(dims) // 2)
        tensors.append(Workload(f"serve{t}", dims, nnz, "zipf", 1.1, "int15", 0, iters, "bf16", seed * 7919 + t))
    jobs = []
    for j in range(njobs):
        jobs.append((j % P, int(rng.choice([16, 32, 64])), int(seed * 104729 + j)))
    return tensors, jobs
