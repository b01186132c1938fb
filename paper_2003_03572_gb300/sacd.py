"""Thin ctypes binding of libsacd.so (C ABI in include/sacd.h), with the same entry-point names.

Argument marshalling only: every step of SaCD runs in the library's CUDA kernels. There is no
CPU fallback; if the library is missing or a GPU is absent the calls raise.

Inputs may be numpy arrays (host) or CUDA tensors from PyTorch (device pointers are passed with
``inputs_on_device=1``; PyTorch is only used here as a source of device memory and streams).
"""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = [
    "SacdError",
    "SACD_FP32",
    "SACD_BF16_GATHER",
    "SACD_LNORM_FRO",
    "SACD_LNORM_SPECTRAL",
    "SACD_LNORM_GCD",
    "SACD_FIXUP_COLUMN_GS",
    "SACD_FIXUP_LEMMA2",
    "TAPS",
    "lib",
    "lib_path",
    "sacd_create",
    "sacd_mode_step",
    "sacd_iterate",
    "sacd_fit",
    "sacd_get_factor",
    "sacd_set_factor",
    "sacd_debug_tap",
    "sacd_set_debug",
    "sacd_replay_mask",
    "sacd_get_info",
    "sacd_set_tiling",
    "sacd_rmse",
    "sacd_pattern_distinctiveness",
    "sacd_save",
    "sacd_load",
    "sacd_sync",
    "sacd_set_wait_budget",
    "sacd_profile_enable",
    "sacd_profile_read",
    "sacd_mttkrp_noalloc",
    "sacd_destroy",
    "sacd_last_error",
    "sacd_batch_create",
    "sacd_batch_iterate",
    "sacd_batch_fit",
    "sacd_batch_job",
    "sacd_batch_destroy",
    "SaCDBatch",
    "sacd_server_create",
    "sacd_server_submit",
    "sacd_server_step",
    "sacd_server_results",
    "sacd_server_get_factor",
    "sacd_server_release",
    "sacd_server_stats",
    "sacd_server_destroy",
    "SaCD",
]

SACD_FP32, SACD_BF16_GATHER = 0, 1
SACD_LNORM_FRO, SACD_LNORM_SPECTRAL, SACD_LNORM_GCD = 0, 1, 2
SACD_FIXUP_COLUMN_GS, SACD_FIXUP_LEMMA2 = 0, 1
TAPS = {"M": 0, "G": 1, "ZPREV": 2, "MASK": 3, "H": 4, "GRAM": 5, "STATE": 6, "CSF_ROW": 7, "CSF_IDX": 8, "CSF_VAL": 9}
_STATUS = {0: "SACD_OK", 1: "SACD_EINVAL", 2: "SACD_ENOMEM", 3: "SACD_ECUDA", 4: "SACD_ETIMEOUT", 5: "SACD_ESTATE"}


class SacdError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{_STATUS.get(status, status)}: {msg}")
        self.status = status


class sacd_config(C.Structure):
    _fields_ = [
        ("nmodes", C.c_int32),
        ("dims", C.POINTER(C.c_int64)),
        ("nnz", C.c_int64),
        ("idx", C.POINTER(C.c_void_p)),
        ("vals", C.c_void_p),
        ("rank", C.c_int32),
        ("init", C.POINTER(C.c_void_p)),
        ("seed", C.c_uint64),
        ("precision", C.c_int32),
        ("lnorm", C.c_int32),
        ("fixup", C.c_int32),
        ("inputs_on_device", C.c_int32),
        ("stream", C.c_void_p),
        ("init_log2_scale", C.c_int32),
    ]


class sacd_info(C.Structure):
    _fields_ = [
        ("nmodes", C.c_int32),
        ("rank", C.c_int32),
        ("rank_padded", C.c_int32),
        ("precision", C.c_int32),
        ("dims", C.c_int64 * 8),
        ("nnz", C.c_int64),
        ("norm_x_sq", C.c_double),
        ("device_bytes", C.c_int64),
        ("tiles", C.c_int64 * 8),
        ("tile_nnz", C.c_int64 * 8),
        ("split_rows", C.c_int64 * 8),
    ]


class sacd_job_result(C.Structure):
    _fields_ = [
        ("job_id", C.c_int64),
        ("status", C.c_int32),
        ("iters", C.c_int32),
        ("objective", C.c_double),
        ("fit", C.c_double),
        ("t_submit", C.c_double),
        ("t_admit", C.c_double),
        ("t_done", C.c_double),
        ("device_bytes", C.c_int64),
        ("error", C.c_char * 128),
    ]


class sacd_server_stats_t(C.Structure):
    _fields_ = [
        ("active", C.c_int32),
        ("waiting", C.c_int32),
        ("finished", C.c_int32),
        ("used_bytes", C.c_int64),
        ("peak_bytes", C.c_int64),
        ("budget_bytes", C.c_int64),
        ("steps", C.c_int64),
        ("creating", C.c_int32),
    ]


class sacd_kernel_stat(C.Structure):
    _fields_ = [("name", C.c_char * 24), ("launches", C.c_int64), ("total_ms", C.c_double)]


_LIB = None


def lib_path():
    return os.path.join(os.path.dirname(os.path.abspath(__file__)), "libsacd.so")


def lib():
    """Load libsacd.so (built in-tree by __graft_entry__.build()). Raises if it is missing."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is not built; run `python -c 'import __graft_entry__ as g; g.build()'`")
    L = C.CDLL(path)
    vp, i32, i64, dbl = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sigs = {
        "sacd_create": (C.c_int, [C.POINTER(sacd_config), C.POINTER(vp)]),
        "sacd_mode_step": (C.c_int, [vp, i32, C.POINTER(i64)]),
        "sacd_iterate": (C.c_int, [vp, i32]),
        "sacd_fit": (C.c_int, [vp, C.POINTER(dbl), C.POINTER(dbl)]),
        "sacd_get_factor": (C.c_int, [vp, i32, vp]),
        "sacd_set_factor": (C.c_int, [vp, i32, vp]),
        "sacd_debug_tap": (C.c_int, [vp, i32, i32, vp]),
        "sacd_set_debug": (C.c_int, [vp, i32]),
        "sacd_replay_mask": (C.c_int, [vp, i32, vp]),
        "sacd_get_info": (C.c_int, [vp, C.POINTER(sacd_info)]),
        "sacd_set_tiling": (C.c_int, [vp, i32, i32]),
        "sacd_rmse": (C.c_int, [vp, i64, C.POINTER(vp), vp, i32, C.POINTER(dbl)]),
        "sacd_pattern_distinctiveness": (C.c_int, [vp, i32, C.POINTER(dbl)]),
        "sacd_save": (C.c_int, [vp, vp, C.c_size_t, C.POINTER(C.c_size_t)]),
        "sacd_load": (C.c_int, [vp, vp, C.c_size_t]),
        "sacd_sync": (C.c_int, [vp]),
        "sacd_set_wait_budget": (C.c_int, [vp, i64]),
        "sacd_profile_enable": (C.c_int, [vp, i32]),
        "sacd_profile_read": (C.c_int, [vp, C.POINTER(sacd_kernel_stat), i32, C.POINTER(i32)]),
        "sacd_mttkrp_noalloc": (C.c_int, [i32, i32, C.POINTER(i64), i64, vp, vp, vp, C.POINTER(vp), i32, i32, vp, vp]),
        "sacd_batch_create": (C.c_int, [C.POINTER(sacd_config), i32, vp, C.POINTER(vp)]),
        "sacd_batch_iterate": (C.c_int, [vp, i32]),
        "sacd_batch_fit": (C.c_int, [vp, C.POINTER(dbl), C.POINTER(dbl)]),
        "sacd_batch_job": (C.c_int, [vp, i32, C.POINTER(vp)]),
        "sacd_batch_destroy": (None, [vp]),
        "sacd_server_create": (C.c_int, [i64, i32, i32, vp, C.POINTER(vp)]),
        "sacd_server_submit": (C.c_int, [vp, C.POINTER(sacd_config), i32, C.POINTER(i64)]),
        "sacd_server_step": (C.c_int, [vp, C.POINTER(i32), C.POINTER(i32)]),
        "sacd_server_results": (C.c_int, [vp, C.POINTER(sacd_job_result), i32, C.POINTER(i32)]),
        "sacd_server_get_factor": (C.c_int, [vp, i64, i32, vp]),
        "sacd_server_release": (C.c_int, [vp, i64]),
        "sacd_server_stats": (C.c_int, [vp, C.POINTER(sacd_server_stats_t)]),
        "sacd_server_destroy": (None, [vp]),
        "sacd_destroy": (None, [vp]),
        "sacd_last_error": (C.c_char_p, []),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _LIB = L
    return L


def sacd_last_error():
    return lib().sacd_last_error().decode()


def _check(status):
    if status != 0:
        raise SacdError(status, sacd_last_error())


def _ptr(a):
    """Device pointer of a CUDA tensor, or host pointer of a contiguous numpy array."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr()
    return a.ctypes.data


def _make_config(dims, idx, vals, rank, init=None, *, seed=0, precision=SACD_FP32, lnorm=SACD_LNORM_FRO,
                 fixup=SACD_FIXUP_COLUMN_GS, stream=None, on_device=False, init_log2_scale=0):
    """A sacd_config plus the Python objects that must stay alive while it is used."""
    N = len(dims)
    keep = []
    if on_device:
        idx_list = [idx[n] for n in range(N)]
        vals_a = vals
        init_list = None if init is None else [init[n] for n in range(N)]
        nnz = int(vals_a.numel())
    else:
        idx_list = [np.ascontiguousarray(idx[n], dtype=np.int32) for n in range(N)]
        vals_a = np.ascontiguousarray(vals, dtype=np.float32)
        init_list = None if init is None else [np.ascontiguousarray(a, dtype=np.float32) for a in init]
        nnz = int(vals_a.shape[0])
    keep += idx_list + [vals_a] + (init_list or [])
    dims_a = (C.c_int64 * N)(*[int(d) for d in dims])
    idx_p = (C.c_void_p * N)(*[_ptr(a) for a in idx_list])
    init_p = None if init_list is None else (C.c_void_p * N)(*[_ptr(a) for a in init_list])
    cfg = sacd_config()
    cfg.nmodes = N
    cfg.dims = dims_a
    cfg.nnz = nnz
    cfg.idx = idx_p
    cfg.vals = _ptr(vals_a) if nnz else None
    cfg.rank = int(rank)
    cfg.init = init_p
    cfg.seed = int(seed) & (2**64 - 1)
    cfg.precision = int(precision)
    cfg.lnorm = int(lnorm)
    cfg.fixup = int(fixup)
    cfg.inputs_on_device = 1 if on_device else 0
    cfg.stream = stream
    cfg.init_log2_scale = int(init_log2_scale)
    keep += [dims_a, idx_p, init_p]
    return cfg, keep


def sacd_create(dims, idx, vals, rank, init=None, **kw):
    """Create a context. ``idx``: sequence of N int32 arrays (or an (N, nnz) array), ``vals``:
    float32 (nnz,), ``init``: N float32 (I_n, R) arrays or None. With ``on_device=True`` the arrays
    are CUDA tensors. Returns the opaque context handle (an int)."""
    cfg, keep = _make_config(dims, idx, vals, rank, init, **kw)
    out = C.c_void_p()
    _check(lib().sacd_create(C.byref(cfg), C.byref(out)))
    del keep
    return out.value


def sacd_batch_create(jobs, stream=None):
    """Create a batch from a list of dicts with the keyword arguments of ``sacd_create``
    (dims, idx, vals, rank, init, precision, ...). Returns the opaque batch handle."""
    cfgs = (sacd_config * len(jobs))()
    keep = []
    for j, spec in enumerate(jobs):
        spec = dict(spec)
        cfg, k = _make_config(spec.pop("dims"), spec.pop("idx"), spec.pop("vals"), spec.pop("rank"),
                              spec.pop("init", None), **spec)
        cfgs[j] = cfg
        keep.append(k)
    out = C.c_void_p()
    _check(lib().sacd_batch_create(cfgs, len(jobs), stream, C.byref(out)))
    del keep
    return out.value


def sacd_batch_iterate(b, iters):
    _check(lib().sacd_batch_iterate(b, int(iters)))


def sacd_batch_fit(b, njobs):
    o = (C.c_double * njobs)()
    f = (C.c_double * njobs)()
    _check(lib().sacd_batch_fit(b, o, f))
    return np.array(o[:]), np.array(f[:])


def sacd_batch_job(b, job):
    out = C.c_void_p()
    _check(lib().sacd_batch_job(b, int(job), C.byref(out)))
    return out.value


def sacd_batch_destroy(b):
    if b:
        lib().sacd_batch_destroy(b)


def sacd_mode_step(ctx, mode, want_count=True):
    n = C.c_int64(0)
    _check(lib().sacd_mode_step(ctx, int(mode), C.byref(n) if want_count else None))
    return int(n.value) if want_count else None


def sacd_iterate(ctx, iters):
    _check(lib().sacd_iterate(ctx, int(iters)))


def sacd_fit(ctx):
    o, f = C.c_double(), C.c_double()
    _check(lib().sacd_fit(ctx, C.byref(o), C.byref(f)))
    return o.value, f.value


def sacd_get_info(ctx):
    info = sacd_info()
    _check(lib().sacd_get_info(ctx, C.byref(info)))
    N = info.nmodes
    return dict(
        nmodes=N,
        rank=info.rank,
        rank_padded=info.rank_padded,
        precision=info.precision,
        dims=list(info.dims)[:N],
        nnz=info.nnz,
        norm_x_sq=info.norm_x_sq,
        device_bytes=info.device_bytes,
        tiles=list(info.tiles)[:N],
        tile_nnz=list(info.tile_nnz)[:N],
        split_rows=list(info.split_rows)[:N],
    )


def sacd_get_factor(ctx, mode, out=None):
    info = sacd_get_info(ctx)
    shape = (info["dims"][mode], info["rank"])
    if out is None:
        out = np.empty(shape, dtype=np.float32)
    _check(lib().sacd_get_factor(ctx, int(mode), out.ctypes.data))
    return out


def sacd_set_factor(ctx, mode, A):
    A = np.ascontiguousarray(A, dtype=np.float32)
    _check(lib().sacd_set_factor(ctx, int(mode), A.ctypes.data))


def sacd_debug_tap(ctx, what, mode=0, last_mode=None):
    """Copy one piece of device state to a new numpy array (see sacd_tap in include/sacd.h)."""
    info = sacd_get_info(ctx)
    w = TAPS[what] if isinstance(what, str) else int(what)
    R = info["rank"]
    N = info["nmodes"]
    lm = mode if last_mode is None else last_mode
    if w in (0, 2):
        out = np.empty((info["dims"][mode], R), np.float32)
    elif w == 1:
        out = np.empty((info["dims"][lm], R), np.float32)
    elif w == 3:
        out = np.empty((info["dims"][lm], R), np.uint8)
    elif w in (4, 5):
        out = np.empty((R, R), np.float64)
    elif w == 6:
        out = np.empty(8, np.float64)
    elif w == 7:
        out = np.empty(info["nnz"], np.int32)
    elif w == 8:
        out = np.empty((N - 1, info["nnz"]), np.int32)
    elif w == 9:
        out = np.empty(info["nnz"], np.float32)
    else:
        raise ValueError(what)
    _check(lib().sacd_debug_tap(ctx, w, int(mode), out.ctypes.data))
    return out


def sacd_set_debug(ctx, on):
    _check(lib().sacd_set_debug(ctx, 1 if on else 0))


def sacd_replay_mask(ctx, mode, mask):
    if mask is None:
        _check(lib().sacd_replay_mask(ctx, int(mode), None))
        return
    m = np.ascontiguousarray(mask, dtype=np.uint8)
    _check(lib().sacd_replay_mask(ctx, int(mode), m.ctypes.data))


def sacd_set_tiling(ctx, mode, sub):
    _check(lib().sacd_set_tiling(ctx, int(mode), int(sub)))


def sacd_rmse(ctx, idx, vals, on_device=False):
    """RMSE (Eq. 30) of the current model over test entries (idx: N arrays, vals)."""
    N = len(idx)
    if on_device:
        arrs, v = list(idx), vals
        n = int(v.numel())
    else:
        arrs = [np.ascontiguousarray(a, dtype=np.int32) for a in idx]
        v = np.ascontiguousarray(vals, dtype=np.float32)
        n = int(v.shape[0])
    ptrs = (C.c_void_p * N)(*[_ptr(a) for a in arrs])
    out = C.c_double()
    _check(lib().sacd_rmse(ctx, n, ptrs, _ptr(v) if n else None, 1 if on_device else 0, C.byref(out)))
    return out.value


def sacd_pattern_distinctiveness(ctx, mode):
    out = C.c_double()
    _check(lib().sacd_pattern_distinctiveness(ctx, int(mode), C.byref(out)))
    return out.value


def sacd_save(ctx):
    """The full SaCD state (factors, z^{k-1}, ti^{k-1}, first-visit flags) as bytes."""
    n = C.c_size_t()
    _check(lib().sacd_save(ctx, None, 0, C.byref(n)))
    buf = (C.c_char * n.value)()
    _check(lib().sacd_save(ctx, buf, n.value, C.byref(n)))
    return bytes(buf)


def sacd_load(ctx, state):
    buf = C.create_string_buffer(state, len(state))
    _check(lib().sacd_load(ctx, buf, len(state)))


def sacd_sync(ctx):
    _check(lib().sacd_sync(ctx))


def sacd_set_wait_budget(ctx, cycles):
    _check(lib().sacd_set_wait_budget(ctx, int(cycles)))


def sacd_profile_enable(ctx, on):
    _check(lib().sacd_profile_enable(ctx, 1 if on else 0))


def sacd_profile_read(ctx):
    buf = (sacd_kernel_stat * 16)()
    n = C.c_int32(0)
    _check(lib().sacd_profile_read(ctx, buf, 16, C.byref(n)))
    return {buf[i].name.decode(): (int(buf[i].launches), float(buf[i].total_ms)) for i in range(min(n.value, 16))}


def sacd_mttkrp_noalloc(dims, mode, nnz, rowid, cidx, vals, factors, rank, ld, M, stream=None):
    """MTTKRP of one mode without any device allocation (see include/sacd.h). Every array
    argument is a device pointer (an int, or a CUDA tensor); ``factors`` holds one per mode."""
    N = len(dims)
    dims_a = (C.c_int64 * N)(*[int(d) for d in dims])
    fp = (C.c_void_p * N)(*[(_ptr(f) if f is not None and not isinstance(f, int) else f) for f in factors])
    p = lambda a: a if (a is None or isinstance(a, int)) else _ptr(a)
    _check(lib().sacd_mttkrp_noalloc(N, int(mode), dims_a, int(nnz), p(rowid), p(cidx), p(vals), fp, int(rank),
                                     int(ld), p(M), stream))


def sacd_destroy(ctx):
    if ctx:
        lib().sacd_destroy(ctx)


class SaCD:
    """Owning wrapper around a context: ``SaCD(dims, idx, vals, rank, init=...)``."""

    def __init__(self, dims, idx, vals, rank, init=None, **kw):
        self.ctx = sacd_create(dims, idx, vals, rank, init, **kw)
        self.info = sacd_get_info(self.ctx)

    def mode_step(self, mode, want_count=True):
        return sacd_mode_step(self.ctx, mode, want_count)

    def iterate(self, iters):
        sacd_iterate(self.ctx, iters)

    def fit(self):
        return sacd_fit(self.ctx)

    def factor(self, mode):
        return sacd_get_factor(self.ctx, mode)

    def factors(self):
        return [self.factor(n) for n in range(self.info["nmodes"])]

    def set_factor(self, mode, A):
        sacd_set_factor(self.ctx, mode, A)

    def tap(self, what, mode=0, last_mode=None):
        return sacd_debug_tap(self.ctx, what, mode, last_mode)

    def rmse(self, idx, vals, on_device=False):
        return sacd_rmse(self.ctx, idx, vals, on_device)

    def pattern_distinctiveness(self, mode):
        return sacd_pattern_distinctiveness(self.ctx, mode)

    def save(self):
        return sacd_save(self.ctx)

    def load(self, state):
        sacd_load(self.ctx, state)

    def set_debug(self, on):
        sacd_set_debug(self.ctx, on)

    def replay_mask(self, mode, mask):
        sacd_replay_mask(self.ctx, mode, mask)

    def sync(self):
        sacd_sync(self.ctx)

    def close(self):
        if self.ctx:
            sacd_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SaCDBatch:
    """Owning wrapper around a batch of independent jobs (see sacd_batch_* in include/sacd.h)."""

    def __init__(self, jobs, stream=None):
        self.njobs = len(jobs)
        self.b = sacd_batch_create(jobs, stream)

    def iterate(self, iters):
        sacd_batch_iterate(self.b, iters)

    def fit(self):
        return sacd_batch_fit(self.b, self.njobs)

    def job(self, j):
        """The j-th job's context handle (borrowed: the batch keeps owning it)."""
        return sacd_batch_job(self.b, j)

    def factor(self, j, mode):
        return sacd_get_factor(self.job(j), mode)

    def close(self):
        if self.b:
            sacd_batch_destroy(self.b)
            self.b = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ------------------------------------------------------------------------------------ serving


def sacd_server_create(hbm_budget_bytes, max_active=1024, max_admit_per_step=16, stream=None):
    out = C.c_void_p()
    _check(lib().sacd_server_create(int(hbm_budget_bytes), int(max_active), int(max_admit_per_step), stream,
                                    C.byref(out)))
    return out.value


def sacd_server_submit(s, spec, iters):
    """Queue a job (dict with the keyword arguments of sacd_create). Returns (job_id, keep): the
    arrays in ``keep`` must stay alive until the job's result has been drained."""
    spec = dict(spec)
    cfg, keep = _make_config(spec.pop("dims"), spec.pop("idx"), spec.pop("vals"), spec.pop("rank"),
                             spec.pop("init", None), **spec)
    jid = C.c_int64()
    _check(lib().sacd_server_submit(s, C.byref(cfg), int(iters), C.byref(jid)))
    return jid.value, keep


def sacd_server_step(s):
    a, w = C.c_int32(), C.c_int32()
    _check(lib().sacd_server_step(s, C.byref(a), C.byref(w)))
    return a.value, w.value


def sacd_server_results(s, cap=256):
    buf = (sacd_job_result * cap)()
    n = C.c_int32()
    _check(lib().sacd_server_results(s, buf, cap, C.byref(n)))
    out = []
    for i in range(n.value):
        r = buf[i]
        out.append(dict(job_id=r.job_id, status=r.status, iters=r.iters, objective=r.objective, fit=r.fit,
                        t_submit=r.t_submit, t_admit=r.t_admit, t_done=r.t_done, device_bytes=r.device_bytes,
                        error=r.error.decode()))
    return out


def sacd_server_get_factor(s, job_id, mode, shape):
    out = np.empty(shape, dtype=np.float32)
    _check(lib().sacd_server_get_factor(s, int(job_id), int(mode), out.ctypes.data))
    return out


def sacd_server_release(s, job_id):
    _check(lib().sacd_server_release(s, int(job_id)))


def sacd_server_stats(s):
    st = sacd_server_stats_t()
    _check(lib().sacd_server_stats(s, C.byref(st)))
    return {k: getattr(st, k) for k, _ in sacd_server_stats_t._fields_}


def sacd_server_destroy(s):
    if s:
        lib().sacd_server_destroy(s)
