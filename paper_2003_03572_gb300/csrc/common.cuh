// Shared device-side definitions of libsacd: step descriptors, small helpers.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#define SACD_MAXN 8
#define SACD_MAXR 256

// Per-mode scalar state kept on the device (doubles), indexed by mode:
//   [0] ti^{k-1}  [1] first-visit flag (1 until the factor's first step)  [2] ti of the last step
//   [3] branch of the last step (0 first visit, 1 Eq. 24, 2 Eq. 27)  [4] L of the last step
//   [5] |E| of the last step  [6] replay-mask flag  [7] unused
#define ST_TIPREV 0
#define ST_FIRST 1
#define ST_TI 2
#define ST_BRANCH 3
#define ST_L 4
#define ST_NSEL 5
#define ST_REPLAY 6
#define ST_STRIDE 8

// One job's mode-n step. Everything a kernel of the step needs; built on the host, copied to
// the device once per context (pointers are fixed for the context's lifetime).
struct StepDesc {
  // ---- mode-n sorted nonzeros (slice structure)
  const int32_t* rowid;  // nnz: i_n per nonzero, ascending
  const int32_t* cidx;   // (N-1) rows of cstride: the other modes' indices, ascending mode order
  const float* val;      // nnz
  int64_t nnz;
  int64_t cstride;       // row stride of cidx (nnz rounded up to a multiple of 4 in a context)
  int32_t nother;        // N-1
  int32_t prec;          // 0: gather FP32 rows, 1: gather BF16 rows
  const void* fac[SACD_MAXN - 1];  // the other factors (FP32 master or BF16 mirror), row stride Rp
  int32_t R;             // rank
  int32_t Rp;            // padded rank: row stride of every I x R matrix on the device
  int32_t rv;            // 16-byte vectors per gathered row (Rp*4/16 or Rp*2/16)
  int32_t sub;           // nonzeros per lane group in a warp tile
  int32_t tile;          // nonzeros per warp tile
  int32_t _pad0;
  int64_t ntiles;
  int64_t I;             // rows of mode n
  float* M;              // I x Rp MTTKRP output
  float* carry;          // ntiles x 2 x Rp open-segment partials
  const int4* split_light;  // {row, first tile, last tile, 0}: rows straddling tiles, few partials
  int64_t nsplit_light;
  const int4* split_heavy;  // {row, first chunk, chunk count, 0}: rows with many partials
  int64_t nsplit_heavy;
  const int4* fix_chunks;   // {row, first tile, first partial, count} chunks of heavy rows
  int64_t nfix_chunks;
  float* carry2;            // nfix_chunks x Rp chunk sums
  const int32_t* rowfix;    // I: -1, or i >= 0 (split_light[i]), or -2 - j (split_heavy[j]);
                            // pass 1 finishes these rows of M when the fix-up was folded into it
  // ---- update of factor n
  float* A;              // I x Rp FP32 master
  __nv_bfloat16* A16;    // I x Rp BF16 mirror (or null)
  float* G;              // I x Rp gradient at the start of the step (rounded to FP32)
  float* Glo;            // I x Rp its rounding error: G + Glo carries the compensated sum unrounded
  float* zprev;          // I x Rp z^{k-1}
  uint8_t* mask;         // I x Rp selection record (or null)
  const uint8_t* replay; // I x Rp selection to apply instead (used when state[ST_REPLAY] != 0)
  const double* gram[SACD_MAXN];  // Rp x Rp FP64 Grams of all factors
  double* gram_out;      // Gram of factor n (written after the update)
  double* gpart;         // gram partials (gram_blocks x Rp x Rp)
  int32_t gram_blocks;
  int32_t N;
  int32_t n;
  int32_t lnorm;         // 0 Frobenius, 1 spectral, 2 GCD (h_rr)
  int32_t fixup;         // 0 column Gauss-Seidel, 1 Lemma 2
  int32_t p1_blocks;     // blocks of the row passes
  int32_t sel_chunks;    // row chunks of the fused select/update kernel
  int32_t _pad1;
  double* H;             // R x R FP64 (Rp stride)
  float* Hf;             // Rp x Rp FP32
  float* invh;           // Rp: 1/h_rr (0 where h_rr <= 0)
  float* lh;             // Rp: L/2 per column
  double* tipart;        // p1_blocks partial sums of z
  double* state;         // ST_STRIDE doubles of mode n
  unsigned int* counters;  // [0] pass-1 blocks (or select/update chunks) done, [1] gram blocks done,
                           // [2] fit blocks done
  unsigned long long* nsel;  // selected elements of the step
};

// Grid barrier words of one persistent launch (count, generation, error word: nonzero after a
// bounded wait gave up) and its two work queues (next item of phase 1 and of phase 2; the launch
// empties each when no block can still take from it).
struct GridBar {
  unsigned int count, gen, err, queue1, queue2, pad[3];
};

// Result of the objective evaluation (sacd_fit).
struct FitDesc {
  const float* A;        // the factor of the objective's mode (I x Rp)
  const float* M;        // that mode's MTTKRP with the current other factors (FP32 gathers)
  int64_t I;
  int32_t R, Rp, N;
  const double* gram[SACD_MAXN];
  double norm_x_sq;
  double* part;          // per-block partials: 2 x blocks (<X, model>, ||model||^2)
  double* out;           // [0] objective [1] wait-error word of the mode steps [2] <X, model> [3] ||model||^2
  unsigned int* counter;
  const unsigned int* wait_err;  // GridBar::err of the launches that produced the factors (or null)
};

__device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }

// Projected coordinate step and Lipschitz importance of one element, written with explicit
// round-to-nearest intrinsics so that every call site gives bit-identical results:
//   s = max(0, a - g/h) - a    (Eq. 11-12; 1/h precomputed, 0 where h <= 0 so that s = 0)
//   z = -g s - (L/2) s^2       (Eq. 20)
__device__ __forceinline__ float sacd_step(float a, float g, float invh) {
  float t = __fsub_rn(a, __fmul_rn(g, invh));
  return __fsub_rn(fmaxf(t, 0.0f), a);
}
__device__ __forceinline__ float sacd_importance(float g, float s, float lh) {
  return __fsub_rn(__fmul_rn(-g, s), __fmul_rn(lh, __fmul_rn(s, s)));
}

// Error-free product and sum (Ogita, Rump, Oishi, "Accurate sum and dot product", 2005):
// a*b = p + e exactly; a+b = s + t exactly.
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = __fmul_rn(a, b);
  e = __fmaf_rn(a, b, -p);
}
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& t) {
  s = __fadd_rn(a, b);
  float z = __fsub_rn(s, a);
  t = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// Packed FP32 pairs (sm_100 family): one 64-bit register holds two floats (the first in the low
// half, as in memory). Every lane of these operations is an IEEE round-to-nearest add, subtract,
// multiply or fused multiply-add, identical to the scalar operation, at half the instructions.
typedef unsigned long long f2p;
__device__ __forceinline__ f2p f2_pack(float a, float b) {
  f2p r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ float f2_x(f2p v) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
  return a;
}
__device__ __forceinline__ float f2_y(f2p v) {
  float a, b;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
  return b;
}
__device__ __forceinline__ f2p f2_add(f2p a, f2p b) {
  f2p r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2p f2_sub(f2p a, f2p b) {
  f2p r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2p f2_mul(f2p a, f2p b) {
  f2p r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2p f2_fma(f2p a, f2p b, f2p c) {
  f2p r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// Compensated accumulation of a * b into (hi, lo), two lanes at once: p = a b rounded,
// -e = RN(p - a b) exactly (na = -a), TwoSum of hi and p, lo += t + e (as t - (-e), the same
// rounding). Lane for lane the same result as the scalar two_prod / two_sum sequence.
__device__ __forceinline__ void dot2_acc2(f2p a, f2p na, f2p b, f2p& hi, f2p& lo) {
  const f2p p = f2_mul(a, b);
  const f2p ne = f2_fma(na, b, p);
  const f2p s = f2_add(hi, p);
  const f2p z = f2_sub(s, hi);
  const f2p t = f2_add(f2_sub(hi, f2_sub(s, z)), f2_sub(p, z));
  hi = s;
  lo = f2_add(lo, f2_sub(t, ne));
}

// Map a global work item to (job, local item) with a prefix array base[0..njobs].
__device__ __forceinline__ int find_job(const int64_t* base, int njobs, int64_t item) {
  int lo = 0, hi = njobs - 1;
  while (lo < hi) {
    int mid = (lo + hi + 1) >> 1;
    if (base[mid] <= item) lo = mid; else hi = mid - 1;
  }
  return lo;
}
