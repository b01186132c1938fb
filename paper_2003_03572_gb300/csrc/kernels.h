// Host-side launchers of the libsacd kernels (all enqueue on the given stream, no sync).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

struct StepDesc;
struct FitDesc;
struct GridBar;

namespace sacd {

// message returned by sacd_last_error() on this thread
void set_last_error(const char* msg);

// ---- MTTKRP (mttkrp.cu)
void launch_mttkrp(const StepDesc* d_descs, const int64_t* d_tile_base, int njobs, int64_t total_tiles, int prec,
                   int rv, int nother, cudaStream_t st);
void launch_rowfix(const int4* light, int64_t nl, const int4* heavy, int64_t nh, int32_t* rowfix, cudaStream_t st);
// One pass for the objective's FP32-gather MTTKRP (dF: FP32 factors, output, partials) and the
// mode's BF16-gather MTTKRP (dB), bit-identical to launch_mttkrp with dB; BF16 rows of 4 or 8
// vectors (padded rank 32, 64), 2 or 3 other modes (mttkrp_dual_supported).
bool mttkrp_dual_supported(int rv, int nother);
void launch_mttkrp_dual(const StepDesc* dB, const StepDesc* dF, int64_t total_tiles, int rv, int nother,
                        cudaStream_t st);
void launch_fixup_light(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total, cudaStream_t st);
void launch_fixup_chunks(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total, cudaStream_t st);
constexpr int kFixChunk = 128;  // partials per level-1 chunk of a heavy split row
void launch_fixup_heavy(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total, cudaStream_t st);

// ---- update path (update.cu)
void configure_kernels();  // one-time kernel attributes (large dynamic shared memory)
int rows_per_block_pass1(int Rp);
int rows_per_block_pass2(int Rp);
__host__ __device__ int gram_chunk_rows(int Rp);
void launch_hl(const StepDesc* d_descs, int njobs, cudaStream_t st);
size_t pass_smem_bytes(int Rp);  // dynamic shared memory of pass1/pass2 for padded rank Rp
void launch_pass1(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total_blocks, size_t smem,
                  cudaStream_t st);
void launch_pass2(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total_blocks, size_t smem,
                  cudaStream_t st);
void launch_gram(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total_blocks, int Rp, bool tc,
                 cudaStream_t st);
// Gram on the tensor cores (gram_tc.cu) for padded ranks 32 and 64 and tall factors (I Rp >= 2^20;
// below that its fixed per-block cost loses to the FP32-pipe Gram): exact BF16 split, FP64 result
bool gram_on_tensor_cores(int Rp, int64_t I);
int gram_tc_blocks(int64_t I);  // blocks (per-block partials) of one Gram on the tensor cores
void launch_gram_tc(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total_blocks, int Rp,
                    cudaStream_t st);
int gram_reduce_blocks(int Rp);
void launch_gram_reduce(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total_blocks,
                        cudaStream_t st);
// ---- fused select/update (selupd.cu): one cooperative launch per mode step (GCD uses pass1/pass2)
__host__ __device__ int selupd_chunk_rows(int Rp, int rt);
size_t selupd_smem_bytes(int Rp, int rt);
int64_t selupd_chunks(int64_t I, int Rp, int rt);
int selupd_choose_rt(int64_t rows, int Rp);  // rows per thread (1 or 4) for a launch over `rows` rows
// smem: the largest selupd_smem_bytes over the launch's padded ranks (not monotonic in the rank);
// the descriptors' sel_chunks must be those of `rt`
cudaError_t launch_selupd(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total_chunks, int rt,
                          size_t smem, GridBar* bar, long long budget, cudaStream_t st);
constexpr long long kWaitBudgetCycles = 1LL << 31;  // ~1 s at the maximum SM clock

int64_t fit_blocks_for(int64_t I, int Rp);
void launch_fit(const FitDesc* d_fit, const int64_t* d_base, int njobs, int64_t total_blocks, cudaStream_t st);
void launch_to_bf16(const float* src, void* dst, int64_t n, cudaStream_t st);
void launch_rmse(const int32_t* idx, const float* vals, int64_t n, const float* const* fac, int N, int R, int Rp,
                 double* part, int64_t blocks, double* out, unsigned int* counter, cudaStream_t st);
void launch_pd(const double* gram, int R, int Rp, double* out, cudaStream_t st);
void launch_init_factor(float* A, int64_t rows, int R, int Rp, unsigned long long seed, int mode, int log2_scale,
                        cudaStream_t st);
void launch_check_factor(const float* A, int64_t rows, int R, int Rp, unsigned int* bad, cudaStream_t st);

// ---- preprocessing (prep.cu)
struct SortWord {
  int nfields;
  int mode[8];
  int shift[8];
};
// Exclusive scan of n uint32 values (out may alias in); total written to *d_total if non-null.
void scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* d_total, void* tmp, cudaStream_t st);
size_t scan_tmp_bytes(int64_t n);
// Stable LSD radix sort of (key, value) pairs on the low `bits` bits; returns 0 if the result is
// in (keys, vals), 1 if in (keys_alt, vals_alt).
int radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n, int bits,
                     void* tmp, cudaStream_t st);
size_t radix_tmp_bytes(int64_t n);
void launch_iota(uint32_t* p, int64_t n, cudaStream_t st);
void launch_build_keys(const int32_t* idx, int64_t stride, const uint32_t* perm, int64_t n, SortWord w,
                       uint64_t* keys, cudaStream_t st);
void launch_gather_i32(const int32_t* src, const uint32_t* perm, int32_t* dst, int64_t n, cudaStream_t st);
void launch_gather_f32(const float* src, const uint32_t* perm, float* dst, int64_t n, cudaStream_t st);
void launch_validate_idx(const int32_t* idx, int64_t stride, int N, const int64_t* d_dims, int64_t n,
                         unsigned int* bad, cudaStream_t st);
void launch_dup_heads(const int32_t* sidx, int64_t stride, int N, int64_t n, uint32_t* heads, cudaStream_t st);
void launch_dup_compact(const int32_t* sidx, int64_t stride, int N, const float* svals, const uint32_t* heads,
                        const uint32_t* pos, int64_t n, int32_t* uidx, int64_t ustride, float* uvals,
                        cudaStream_t st);
void launch_sumsq(const float* v, int64_t n, double* part, int64_t nparts, double* out, unsigned int* counter,
                  cudaStream_t st);
void launch_split_flags(const int32_t* rowid, int64_t nnz, int64_t tile, int64_t ntiles, uint32_t* flags,
                        cudaStream_t st);
void launch_split_emit(const int32_t* rowid, int64_t nnz, int64_t tile, int64_t ntiles, const uint32_t* flags,
                       const uint32_t* pos, int4* out, cudaStream_t st);

}  // namespace sacd
