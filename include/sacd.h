/*
 * sacd.h -- C ABI of libsacd.so: Saturating Coordinate Descent (SaCD) for nonnegative CP
 * factorisation of sparse N-mode tensors, on one NVIDIA GB300 (sm_103a).
 *
 * Method: Balasubramaniam, Nayak, Yuen, "Efficient Nonnegative Tensor Factorization via
 * Saturating Coordinate Descent" (ACM TKDD 2020). Algorithm 1; Eq. 9-15 (gradient G and second
 * derivative H), Eq. 11-13 (nonnegative coordinate update), Eq. 20 (Lipschitz element
 * importance), Eq. 24-27 (saturation point and total importance), Lemma 2 (gradient fix-up),
 * Eq. 6-8 (objective).
 *
 * Conventions shared by every entry point:
 *  - Every call returns a sacd_status. On any error a thread-local message is available from
 *    sacd_last_error(). No C++ exception crosses this ABI.
 *  - Host pointers passed in are owned by the caller and are only read during the call (the
 *    library copies what it keeps). A sacd_ctx owns all device memory it allocates; it is
 *    released by sacd_destroy().
 *  - All device work of a context runs on one CUDA stream (the caller's, or one the context
 *    creates). Calls on one context must not be made concurrently from several threads.
 *  - A CUDA error (including an asynchronous fault seen at a later synchronisation) returns
 *    SACD_ECUDA and poisons the context: afterwards every call but sacd_destroy returns
 *    SACD_ESTATE.
 *  - Factor matrices cross the ABI as row-major I_n x R FP32 arrays.
 */
#ifndef SACD_H
#define SACD_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  SACD_OK = 0,
  SACD_EINVAL = 1,   /* bad argument: ranges, null pointers, out-of-range indices, bad init */
  SACD_ENOMEM = 2,   /* device (or pinned host) allocation failed */
  SACD_ECUDA = 3,    /* CUDA runtime error; the context is poisoned */
  SACD_ETIMEOUT = 4, /* a bounded device-side wait gave up */
  SACD_ESTATE = 5    /* call not legal in the context's state (poisoned, wrong mode, ...) */
} sacd_status;

/* Storage of the factor rows that the MTTKRP gathers. FP32 master factors are kept in both. */
typedef enum {
  SACD_FP32 = 0,        /* gather FP32 rows */
  SACD_BF16_GATHER = 1  /* gather a BF16 mirror of the factors, accumulate in FP32 */
} sacd_precision;

/* Constant L in the element importance z = -g s - (L/2) s^2 (Eq. 20). */
typedef enum {
  SACD_LNORM_FRO = 0,      /* L = ||H||_F (symbol table: ||.|| is the Frobenius norm) */
  SACD_LNORM_SPECTRAL = 1, /* L = largest eigenvalue of H (H is symmetric positive semidefinite) */
  SACD_LNORM_GCD = 2       /* L replaced by h_rr per column: the GCD importance of Eq. 18 */
} sacd_lnorm;

/* Gradient fix-up after a coordinate update u_qr += s within one mode step. */
typedef enum {
  SACD_FIXUP_COLUMN_GS = 0, /* g_q. += s * H[r,.]: later columns of row q see the exact gradient */
  SACD_FIXUP_LEMMA2 = 1     /* Lemma 2 read literally: only g_qr changes (Jacobi within the row) */
} sacd_fixup;

typedef struct sacd_ctx sacd_ctx; /* opaque */

typedef struct {
  int32_t nmodes;             /* N, 2 <= N <= 8 */
  const int64_t* dims;        /* host, N entries, each in [1, 2^31-1] */
  int64_t nnz;                /* number of COO entries, 0 <= nnz <= 2^31-1 */
  const int32_t* const* idx;  /* host array of N pointers; idx[n][e] is the 0-based mode-n index */
  const float* vals;          /* nnz values (any sign; repeated coordinates are summed) */
  int32_t rank;               /* R, 1 <= R <= 256 */
  const float* const* init;   /* host array of N pointers to I_n x R row-major FP32, or NULL:
                                 U[0,1) values (h >> 40) * 2^-24 * 2^init_log2_scale drawn on the
                                 device, h the splitmix64 finaliser of seed + (n+1)*0xD1B54A32D192ED03
                                 + (i*R + r + 1)*0x9E3779B97F4A7C15. Values must be finite, >= 0 */
  uint64_t seed;              /* used only when init == NULL */
  int32_t precision;          /* sacd_precision */
  int32_t lnorm;              /* sacd_lnorm */
  int32_t fixup;              /* sacd_fixup */
  int32_t inputs_on_device;   /* 0: idx[n], vals, init[n] point to host memory;
                                 1: they point to device memory of the current device */
  void* stream;               /* cudaStream_t to run on, or NULL: the context creates its own */
  int32_t init_log2_scale;    /* init == NULL only: every drawn value is scaled by 2^init_log2_scale
                                 (exact), in [-60, 60]; 0 = U[0,1) */
} sacd_config;

/* Sizes and constants of a context (sacd_get_info). */
typedef struct {
  int32_t nmodes;
  int32_t rank;
  int32_t rank_padded;        /* row stride of the device factor matrices */
  int32_t precision;
  int64_t dims[8];
  int64_t nnz;                /* distinct coordinates after summing repeats */
  double norm_x_sq;           /* ||X||^2 in FP64 */
  int64_t device_bytes;       /* device memory held by the context */
  int64_t tiles[8];           /* MTTKRP warp tiles per mode */
  int64_t tile_nnz[8];        /* nonzeros per warp tile per mode */
  int64_t split_rows[8];      /* rows whose nonzeros straddle a tile boundary, per mode */
} sacd_info;

/*
 * sacd_create -- copy a sparse tensor and initial factors to the device and build the per-mode
 * sorted slice structure (the sets Omega^(n)_q of the symbol table: nonzeros ordered by i_n, then
 * by the other modes in ascending mode order), summing repeated coordinates in FP32 in input
 * order. Computes ||X||^2 and the FP64 Gram matrices A_k^T A_k of the initial factors.
 * Every factor starts "unvisited" (Algorithm 1, k == 1 branch).
 * On success *out receives the context; on error *out is set to NULL.
 * Errors: SACD_EINVAL (cfg ranges, an index outside [0, dims[n]), negative or non-finite init,
 * init_log2_scale out of range), SACD_ENOMEM, SACD_ECUDA.
 */
sacd_status sacd_create(const sacd_config* cfg, sacd_ctx** out);

/*
 * sacd_mode_step -- one SaCD mode step for factor `mode` (Algorithm 1, one of its three
 * factor blocks): MTTKRP M = X_(n)(Khatri-Rao of the other factors) (Eq. 9), H = Hadamard of
 * the other Grams (Eq. 10), L (Algorithm 1), G = A H - M (Eq. 9, 14), z (Eq. 20), ti (Eq. 25),
 * selection (z > 0 on the first visit, else sp > 0 from Eq. 24 / Eq. 27), the projected
 * update of the selected elements (Eq. 11-13) with the configured fix-up, z^{k-1} <- z, and
 * the refreshed FP64 Gram of the updated factor. Enqueued on the context's stream.
 * n_selected (nullable): if given, the call waits for the step and stores |E|, the number of
 * selected elements. Errors: SACD_EINVAL (mode out of range), SACD_ECUDA, SACD_ESTATE.
 */
sacd_status sacd_mode_step(sacd_ctx* ctx, int32_t mode, int64_t* n_selected);

/*
 * sacd_iterate -- `iters` outer SaCD iterations, each the mode steps 0..N-1 in order
 * (Algorithm 1's loop over k). The first call captures one iteration in a CUDA graph and
 * replays it; nothing is synchronised. Errors: SACD_EINVAL (iters < 0), SACD_ECUDA, SACD_ESTATE.
 */
sacd_status sacd_iterate(sacd_ctx* ctx, int32_t iters);

/*
 * sacd_fit -- objective f = ||X - [[A]]||^2 over all cells (Eq. 6-8), as
 * ||X||^2 - 2<X, [[A]]> + sum_{r,s} prod_k (A_k^T A_k)_{rs}, in FP64, and
 * fit = 1 - sqrt(max(f, 0)) / ||X||. Waits for the stream. Either output pointer may be NULL.
 * The first call allocates a 32-byte pinned host buffer for the read-back, owned by the context.
 * In the BF16-gather mode the cross term comes from FP32 gathers of the FP32 master factors (one
 * extra MTTKRP per call), so the objective is that of the factors sacd_get_factor returns.
 * Errors: SACD_ETIMEOUT (see sacd_set_wait_budget), SACD_ECUDA.
 */
sacd_status sacd_fit(sacd_ctx* ctx, double* objective, double* fit);

/* sacd_get_factor -- copy factor `mode` (I_n x R row-major FP32) to host_out. Waits.
 * Errors: SACD_EINVAL, SACD_ETIMEOUT (see sacd_set_wait_budget), SACD_ECUDA. */
sacd_status sacd_get_factor(sacd_ctx* ctx, int32_t mode, float* host_out);

/*
 * sacd_set_factor -- replace factor `mode` with host_in (I_n x R row-major FP32, finite, >= 0)
 * and refresh its Gram (and BF16 mirror). The importance state (z^{k-1}, ti^{k-1}, first
 * visit) is left as it is. Errors: SACD_EINVAL (mode, bad values), SACD_ECUDA.
 */
sacd_status sacd_set_factor(sacd_ctx* ctx, int32_t mode, const float* host_in);

/* Debug taps (sacd_debug_tap `what`). "last step" = the most recent mode step of any mode. */
typedef enum {
  SACD_TAP_M = 0,        /* float  I_mode x R   : MTTKRP of `mode` from its most recent step */
  SACD_TAP_G = 1,        /* float  I_n x R      : gradient at the start of the last step (n = its mode) */
  SACD_TAP_ZPREV = 2,    /* float  I_mode x R   : z^{k-1} of `mode` (z of its most recent step) */
  SACD_TAP_MASK = 3,     /* uint8  I_n x R      : selection of the last step (needs sacd_set_debug) */
  SACD_TAP_H = 4,        /* double R x R        : H of the last step */
  SACD_TAP_GRAM = 5,     /* double R x R        : A_mode^T A_mode */
  SACD_TAP_STATE = 6,    /* double 8            : per `mode`: ti^{k-1}, first-visit flag, ti of the
                                                   last step of `mode`, branch (0 first, 1 Eq. 24,
                                                   2 Eq. 27), L, |E|, 0, 0 */
  SACD_TAP_CSF_ROW = 7,  /* int32  nnz          : mode-`mode` sorted row index per nonzero */
  SACD_TAP_CSF_IDX = 8,  /* int32  (N-1) x nnz  : the other modes' indices, ascending mode order */
  SACD_TAP_CSF_VAL = 9   /* float  nnz          : values in mode-`mode` sorted order */
} sacd_tap;

/*
 * sacd_debug_tap -- copy one piece of device state to host_out (layout per sacd_tap). Waits.
 * For tests and diagnostics only. Errors: SACD_EINVAL (what/mode), SACD_ESTATE (MASK without
 * sacd_set_debug(ctx, 1), or G/H/MASK before any step).
 */
sacd_status sacd_debug_tap(sacd_ctx* ctx, int32_t what, int32_t mode, void* host_out);

/* sacd_set_debug -- when on, mode steps also record the selection mask (one byte per element). */
sacd_status sacd_set_debug(sacd_ctx* ctx, int32_t on);

/*
 * sacd_replay_mask -- make the next mode step of `mode` apply host_mask (uint8 I_mode x R,
 * nonzero = selected) instead of its own selection, everything else unchanged. For parity
 * tests that compare the arithmetic with a selection fixed on both sides. NULL clears it.
 */
sacd_status sacd_replay_mask(sacd_ctx* ctx, int32_t mode, const uint8_t* host_mask);

/*
 * sacd_set_tiling -- re-cut the MTTKRP warp tiles of `mode`: `sub` nonzeros per lane group
 * (a multiple of 4 in [4, 1024]; a tile is 32/LPR groups, LPR = 16-byte vectors per gathered
 * row, at most 32). The default comes from the autotuned table compiled into the library for the
 * job's shape. Changes the summation order of M (results stay within the MTTKRP tolerance).
 * Used by the autotuner; waits. Errors: SACD_EINVAL, SACD_ENOMEM, SACD_ECUDA.
 */
sacd_status sacd_set_tiling(sacd_ctx* ctx, int32_t mode, int32_t sub);

/*
 * sacd_rmse -- RMSE of the current model over n test entries, sqrt(sum (x - x_hat)^2 / n)
 * (Eq. 30), x_hat = sum_r prod_k A_k[i_k, r] (Eq. 8) evaluated in FP64. idx: array of N pointers
 * to n int32 coordinates each, vals: n FP32; host memory, or device memory if on_device != 0.
 * Waits. Errors: SACD_EINVAL (a coordinate out of range), SACD_ENOMEM, SACD_ECUDA.
 */
sacd_status sacd_rmse(sacd_ctx* ctx, int64_t n, const int32_t* const* idx, const float* vals, int32_t on_device,
                      double* rmse);

/*
 * sacd_pattern_distinctiveness -- PD of factor `mode` (Eq. pd): the cosine similarity of its
 * columns i < r, averaged over the pairs (columns of zero norm left out), from the factor's FP64
 * Gram. Lower is more distinct. Waits.
 */
sacd_status sacd_pattern_distinctiveness(sacd_ctx* ctx, int32_t mode, double* pd);

/*
 * Checkpoint and resume of the whole SaCD state: the factors, z^{k-1}, ti^{k-1} and the
 * first-visit flags of every mode (Algorithm 1 needs all of them to continue exactly).
 * sacd_save with host_buf == NULL stores the size needed in *bytes; otherwise it writes the state
 * (cap >= that size) and waits. sacd_load restores a state saved from a context of the same
 * tensor shape, nonzero count and rank (the tensor itself is not saved: create the context from
 * the same tensor first). A resumed context continues bit-identically to one never interrupted.
 * Errors: SACD_EINVAL (size, magic, shape mismatch, bad factor values), SACD_ECUDA. sacd_load
 * checks the whole buffer before it copies anything, so an SACD_EINVAL leaves the context unchanged.
 */
sacd_status sacd_save(sacd_ctx* ctx, void* host_buf, size_t cap, size_t* bytes);
sacd_status sacd_load(sacd_ctx* ctx, const void* host_buf, size_t bytes);

/* sacd_get_info -- sizes and constants of the context. */
sacd_status sacd_get_info(sacd_ctx* ctx, sacd_info* out);

/* sacd_sync -- wait for all work enqueued on the context's stream. Errors: SACD_ETIMEOUT (see
 * sacd_set_wait_budget), SACD_ECUDA. */
sacd_status sacd_sync(sacd_ctx* ctx);

/*
 * sacd_set_wait_budget -- the bound, in SM clock cycles (default 2^31, about a second), of every
 * wait inside the fused select/update kernel: its blocks meet at a grid barrier between the sum
 * of z (ti, Eq. 25) and the selection (Eq. 24/27). A block that waits longer sets an error word
 * and every block skips the update; the next call that waits for the stream (sacd_sync,
 * sacd_fit, sacd_get_factor, sacd_mode_step with a count) returns SACD_ETIMEOUT and the context
 * is poisoned. For tests of that path (a budget of a few cycles makes the wait run out).
 * Errors: SACD_EINVAL (cycles < 1).
 */
sacd_status sacd_set_wait_budget(sacd_ctx* ctx, int64_t cycles);

/*
 * Per-kernel timing. While enabled, mode steps and fits are launched one kernel at a time (no
 * CUDA graph) with a CUDA event pair around each kernel, on the context's stream.
 * sacd_profile_read waits, then fills up to `cap` entries (kernel class, launches, total ms)
 * and returns the number of classes in *n. Timing pairs beyond 65536 per enable are dropped.
 */
typedef struct {
  char name[24];
  int64_t launches;
  double total_ms;
} sacd_kernel_stat;

sacd_status sacd_profile_enable(sacd_ctx* ctx, int32_t on);
sacd_status sacd_profile_read(sacd_ctx* ctx, sacd_kernel_stat* out, int32_t cap, int32_t* n);

/*
 * sacd_mttkrp_noalloc -- the MTTKRP of one mode, M = X_(mode) (Khatri-Rao of the other
 * factors), computed without allocating any device memory. The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, such as code inside a host
 * framework that owns the whole device memory pool and forbids allocations outside its plan,
 * or latency-critical loops that cannot afford the synchronisation cudaMalloc/cudaFree may imply.
 *
 * All array arguments are device pointers owned by the caller:
 *   rowid  nnz int32, the mode-`mode` index of each nonzero, sorted ascending (e.g. the
 *          SACD_TAP_CSF_ROW layout of a context);
 *   cidx   (nmodes-1) x nnz int32, the other modes' indices in ascending mode order;
 *   vals   nnz FP32 values;
 *   factors host array of nmodes device pointers; factors[k] (k != mode) is I_k x ld FP32
 *          row-major, 16-byte aligned, with columns >= rank set to zero (factors[mode] unused);
 *   M      output, I_mode x ld FP32 row-major, 16-byte aligned; every entry is written.
 * ld must be the padded rank, the next power of two >= max(8, rank). dims is a host array.
 * The work runs on `stream` (cudaStream_t, NULL = legacy default stream) and is not waited for.
 * Preconditions on the device arrays, which this call cannot check without waiting for the GPU:
 * every rowid[e] lies in [0, dims[mode]), every index of row j of cidx lies in [0, dims[k]) for
 * the j-th other mode k, and rowid is sorted ascending. An index out of range makes the kernels
 * read or write outside the caller's arrays; an unsorted rowid gives a wrong M.
 *
 * Scratch: a file-scope static device array of SACD_NOALLOC_SCRATCH_MIB MiB, held by every GPU
 * that loads the library until the process exits. A call needs 4 KiB + 2 * ceil(nnz / tile) *
 * ld * 4 bytes of it (tile = 32 / min(ld/4, 32) lane groups x 8..128 nonzeros, chosen from
 * nnz); larger problems are rejected with SACD_EINVAL before any GPU work. The first call on a
 * device looks up the array's device address (cudaGetSymbolAddress) and keeps it for the rest of
 * the process, so make that first call before any stream capture, and do not use this entry
 * point after a cudaDeviceReset of that device. Every call shares the array: calls that overlap
 * on the GPU race. Errors: SACD_EINVAL (ranges, null or misaligned pointers, too large),
 * SACD_ECUDA.
 */
#define SACD_NOALLOC_SCRATCH_MIB 16
sacd_status sacd_mttkrp_noalloc(int32_t nmodes, int32_t mode, const int64_t* dims, int64_t nnz,
                                const int32_t* rowid, const int32_t* cidx, const float* vals,
                                const float* const* factors, int32_t rank, int32_t ld, float* M,
                                void* stream);

/*
 * Batches (not in the paper; the batched workload of many small tensors). A batch owns `njobs`
 * independent contexts, created from cfgs[0..njobs-1] (their `stream` fields are ignored: all
 * jobs run on the batch's stream, the caller's or one the batch creates). sacd_batch_iterate runs
 * `iters` outer iterations of every job (each job's modes 0..N_j-1 in order), launching each
 * kernel of a mode step once for all jobs that have that mode (the MTTKRP and Gram once per
 * row-width class), from a CUDA graph. A job's results are bit-identical to running its context
 * alone. sacd_batch_fit evaluates every job's objective and fit (arrays of njobs; NULL allowed)
 * and waits. sacd_batch_job lends a job's context (for sacd_get_factor, taps, ...); the batch
 * keeps owning it. Errors: SACD_EINVAL, SACD_ENOMEM, SACD_ECUDA, SACD_ESTATE (poisoned batch,
 * a job with a pending replay mask).
 */
typedef struct sacd_batch sacd_batch;
sacd_status sacd_batch_create(const sacd_config* cfgs, int32_t njobs, void* stream, sacd_batch** out);
sacd_status sacd_batch_iterate(sacd_batch* b, int32_t iters);
sacd_status sacd_batch_fit(sacd_batch* b, double* objective, double* fit);
sacd_status sacd_batch_job(sacd_batch* b, int32_t job, sacd_ctx** ctx_out);
void sacd_batch_destroy(sacd_batch* b);

/*
 * Serving (not in the paper; the served workload): continuous batching of factorisation jobs
 * on one GPU, single-threaded API (one host thread calls it; internally a preparation thread
 * creates the contexts of admitted jobs on a stream of its own, so that the H2D copies and
 * sorts of new jobs overlap the iterations of running ones).
 *  - sacd_server_create: `hbm_budget_bytes` caps the device memory of admitted jobs (each job is
 *    charged an upper bound of its create-time peak until it is admitted, then the bytes its
 *    context holds); at most `max_active` jobs run at once and at most `max_admit_per_step` are
 *    admitted per step; `stream` as for contexts (the iterations run on it).
 *  - sacd_server_submit: queue a job (FIFO) that will run `iters` outer iterations. The arrays
 *    that cfg points to are read when the job's context is created, after its admission, and
 *    must stay valid until its result has been drained by sacd_server_results. cfg->stream is
 *    ignored.
 *  - sacd_server_step: add the jobs whose contexts are ready to the running set; admit waiting
 *    jobs in order while they fit the budget, handing them to the preparation thread (a job
 *    larger than the whole budget finishes with SACD_ENOMEM; a job whose create fails finishes
 *    with that status at a later step); if nothing is running yet, wait for the first context;
 *    run one outer iteration of every running job with one batched launch set, and
 *    finish the jobs that reached their iteration count: objective and fit evaluated, factors
 *    copied to host memory, device memory freed (a job whose objective is not finite finishes
 *    with SACD_ESTATE and no factors). Waits for the iteration stream. Reports active (running or
 *    being created) and waiting counts (nullable).
 *  - sacd_server_results: drain up to `cap` finished jobs' results (times are seconds since the
 *    server was created, host clock); their factors stay available through
 *    sacd_server_get_factor (I_n x R FP32) until sacd_server_release.
 * A job's results are the same as those of its own context run alone.
 */
typedef struct sacd_server sacd_server;
typedef struct {
  int64_t job_id;
  int32_t status;      /* sacd_status of the job */
  int32_t iters;       /* iterations run */
  double objective;
  double fit;
  double t_submit, t_admit, t_done;
  int64_t device_bytes;
  char error[128];
} sacd_job_result;
typedef struct {
  int32_t active, waiting, finished;   /* active counts running jobs and jobs being created */
  int64_t used_bytes, peak_bytes, budget_bytes, steps;
  int32_t creating;                    /* admitted jobs whose contexts are not ready yet */
} sacd_server_stats_t;
sacd_status sacd_server_create(int64_t hbm_budget_bytes, int32_t max_active, int32_t max_admit_per_step,
                               void* stream, sacd_server** out);
sacd_status sacd_server_submit(sacd_server* s, const sacd_config* cfg, int32_t iters, int64_t* job_id);
sacd_status sacd_server_step(sacd_server* s, int32_t* n_active, int32_t* n_waiting);
sacd_status sacd_server_results(sacd_server* s, sacd_job_result* out, int32_t cap, int32_t* n);
sacd_status sacd_server_get_factor(sacd_server* s, int64_t job_id, int32_t mode, float* host_out);
sacd_status sacd_server_release(sacd_server* s, int64_t job_id);
sacd_status sacd_server_stats(sacd_server* s, sacd_server_stats_t* out);
void sacd_server_destroy(sacd_server* s);

/* sacd_destroy -- release everything the context owns. NULL-safe; legal on a poisoned context. */
void sacd_destroy(sacd_ctx* ctx);

/* sacd_last_error -- message of the last failed call on this thread ("" if none). */
const char* sacd_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* SACD_H */
