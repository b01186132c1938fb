// Gram matrices A^T A (Eq. 10's V^T V, W^T W) on the 5th-generation tensor cores (tcgen05), for
// padded ranks 32 and 64, with an FP64-accurate result from an exact split of the FP32 factor.
//
// Split. Block b takes a contiguous range of rows. Pass 1 streams the range once for the column
// maxima; e_j is the exponent of column j's largest magnitude over the range, so every scaled value
// t = a 2^-e_j lies in (-1, 1). Pass 2 cuts t into kTcSlices signed base-128 digits:
// s_1 = rint(128 t), t <- 128 t - s_1 (now in [-1/2, 1/2]), and so on. |s_1| <= 128 and
// |s_p| <= 64 after it; all are integers exact in BF16, and a_ij = 2^e_j sum_p s_p,ij 2^-7p up to
// 2^(e_j - 50). Then
// (A^T A)_jk = 2^(e_j + e_k) sum_d 2^-7d D_d,jk with D_d = sum over slice pairs p + q = d of
// S_p^T S_q; the pairs with d <= 8 are formed (the next diagonal weighs 2^-56 of the first).
//
// Products. One tcgen05.mma (kind::f16: BF16 operands, FP32 accumulator in tensor memory) forms a
// 128 x 128 x 16 product from shared-memory operands in the canonical K-major layout without
// swizzle (core matrices of 8 rows x 16 bytes; LBO = 128 B between core matrices along K, SBO
// between those along M or N). Both operands stack G = 128 / Rp consecutive slices (slices are
// stored back to back, zero past the seventh): the product of stacks p and q holds in its block
// (r, c) the slice pair (p + r, q + c), diagonal p + q + r + c. The stacks start at
// p, q in {1, 1+G, 1+2G, ..}; the products with p + q <= 8 cover every pair with d <= 8 exactly
// once (10 products at Rp = 64, 3 at Rp = 32), and those with equal p + q = t share accumulator
// T_t. Small products (N = Rp) would be bound by the operand reads from shared memory; at
// 128 x 128 the reads and the arithmetic take about the same time.
//
// Exactness. Slice products are exact in FP32 and their sums are integers. Every accumulator is
// read back (tcgen05.ld) and restarted after each period of kTcPeriod = 1024 rows. Each block of
// an accumulator with d <= 5 holds pairs whose digit products add up to at most 2^14 per row
// (the first digits are at most 128, the others at most 64), so over a period its sums stay
// within 2^24 and are exact. Blocks with d >= 6 may round: at most 64 accumulation steps of at
// most one unit each per period, weighted 2^-7d <= 2^-42, i.e. below 2^-36 2^(e_j + e_k) per
// period. Each worker thread owns one tensor-memory lane (row j of one block row r) and half of
// the columns, that is the Gram entries (j, k) of one or two block columns c, and keeps the
// scaled sums as unevaluated FP32 pairs (hi, lo) built with error-free two_sum (Knuth),
// renormalised after every read-back. At the end the pairs of all blocks are summed the same way
// and each entry becomes one FP64 number, 2^(e_j + e_k) (hi + lo), assembled from the FP32 bit
// fields (one FP64 add per entry: FP64 arithmetic is scarce on this part). The per-block partials
// are summed by gram_reduce_kernel, as for the FP32-pipe Gram.
//
// Pipeline. Eight worker warps and one issuing warp. Pass 1 keeps up to NST1 bulk copies
// (cp.async.bulk, completion counted on an mbarrier) in flight over all of shared memory. In pass
// 2 the issuing warp's elected thread keeps kTcNraw copies of raw FP32 rows in flight and issues
// each fill's MMAs once the workers have sliced it (an mbarrier per slice buffer), committing them
// to another mbarrier per buffer; meanwhile the workers slice the next fill. Every wait is bounded
// by a clock64() budget; on expiry the block stops issuing work, waits (again bounded) for what it
// has in flight, writes NaN as its partial (so the step's result is visibly wrong), and frees its
// tensor memory.
#include <cstdint>

#include "common.cuh"
#include "kernels.h"

namespace sacd {

namespace {

constexpr int kTcSlices = 7;      // base-128 digits below the column scale
constexpr int kTcKB = 64;         // rows per fill (4 MMA k-steps of 16)
constexpr int kTcWorkers = 256;   // 8 worker warps: slicing, read-backs, the final sums
constexpr int kTcThreads = kTcWorkers + 32;  // and the issuing warp
constexpr int kTcMinRows = 512;   // fewest rows a block is given
constexpr int kTcPeriod = 1024;   // rows between read-backs of the accumulators
constexpr int kTcNraw = 4;        // raw fills in flight in pass 2
constexpr int kTcN = 128;         // MMA shape 128 x 128 x 16
constexpr long long kTcWaitCycles = 1LL << 31;

template <int NR>
struct TcShape {
  static constexpr int G = kTcN / NR;                         // slices stacked in one operand
  static constexpr int NSLICE = 8;                            // the last stack reaches slice 8
  static constexpr int SBO = (kTcKB / 8) * 128;               // bytes between core matrices along M / N
  static constexpr int SLICE_BYTES = NR * kTcKB * 2;          // one slice: NR rows x kTcKB BF16
  static constexpr int SLICEBUF = NSLICE * SLICE_BYTES;       // one fill's slices
  static constexpr int STAGE = kTcKB * NR * 4;                // one fill's raw FP32 rows
  static constexpr int REGION = 2 * SLICEBUF + kTcNraw * STAGE;
  static constexpr int NST1 = REGION / STAGE;                 // pass-1 copies in flight
  static constexpr int PERIOD_FILLS = kTcPeriod / kTcKB;
  static constexpr int NACC = (8 - 2) / G + 1;                // accumulators T_2, T_2+G, .. T_8
  static constexpr int TALLOC = NACC * kTcN;                  // tensor-memory columns (512 or 256)
  static constexpr int NQ = 2 * G;                            // (block row, column half) groups
  static constexpr int CSTRIDE = NR + 1;                      // padded row of the group sums (float2)
  static constexpr int NBAR = NST1 + kTcNraw + 4;             // pass 1, raw, done x2, ready x2
  static constexpr size_t SMEM = (size_t)REGION + 2 * NR * sizeof(int) + NBAR * sizeof(uint64_t) + 64;
  static_assert(REGION % STAGE == 0, "stages tile the region");
  static_assert((size_t)NQ * NR * CSTRIDE * 8 <= (size_t)REGION, "group sums fit the region");
  static_assert(TALLOC == 256 || TALLOC == 512, "tensor-memory allocation");
  static_assert((1 + G * ((7 - 1) / G)) + G - 1 <= NSLICE, "stacks stay inside the slice buffer");
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: start address, leading and stride byte offsets (16-byte units),
// descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | (1ull << 46);
}

__device__ __forceinline__ void mbar_init(uint32_t addr, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}

// true once the phase of the given parity has completed; false if the budget ran out first
__device__ __forceinline__ bool mbar_wait(uint32_t addr, uint32_t parity, long long budget) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > budget) return false;
  }
}

// bulk copy of `bytes` (a multiple of 16) from global to shared memory, counted on `bar`
__device__ __forceinline__ void bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
               "l"(src), "r"(bytes), "r"(bar)
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// error-free sum (Knuth): hi + lo + x = hi' + lo' up to the rounding of the lo update
__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float x) {
  const float s = __fadd_rn(hi, x);
  const float bb = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(x, bb));
  hi = s;
  lo = __fadd_rn(lo, err);
}

__device__ __forceinline__ void renorm(float& hi, float& lo) {
  const float s = __fadd_rn(hi, lo);
  lo = __fsub_rn(lo, __fsub_rn(s, hi));
  hi = s;
}

__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }  // e in [-126, 127]

// 2^s x as an FP64 number, assembled from the FP32 bit fields of x (exact; zero and FP32
// subnormals give 0, non-finite x stays non-finite)
__device__ __forceinline__ double f32_scaled_to_f64(float x, int s) {
  const uint32_t b = __float_as_uint(x);
  const uint32_t ef = (b >> 23) & 0xFFu;
  if (ef == 0u) return 0.0;
  if (ef == 0xFFu) return (double)x;
  const uint64_t sign = (uint64_t)(b >> 31) << 63;
  const int64_t e = (int64_t)ef - 127 + 1023 + s;
  if (e <= 0) return 0.0;
  if (e >= 2047) return __longlong_as_double((long long)(sign | 0x7FF0000000000000ull));
  return __longlong_as_double((long long)(sign | ((uint64_t)e << 52) | ((uint64_t)(b & 0x7FFFFFu) << 29)));
}

// a barrier's completed phases as this thread knows them, and the operations issued on it
struct BarTrack {
  uint32_t issued = 0, done = 0;
};

// wait until the operation with index `idx` on the barrier has completed
__device__ __forceinline__ bool bar_wait_upto(uint32_t addr, BarTrack& t, uint32_t idx,
                                              long long budget = kTcWaitCycles) {
  while (t.done <= idx) {
    if (!mbar_wait(addr, t.done & 1u, budget)) return false;
    ++t.done;
  }
  return true;
}

__device__ __forceinline__ void bar_drain(uint32_t addr, BarTrack& t) {
  if (t.issued > t.done) bar_wait_upto(addr, t, t.issued - 1, kTcWaitCycles / 16);
}

}  // namespace

// worker-only barrier (named barrier 1, the 8 worker warps) and its AND-reduction
__device__ __forceinline__ void workers_sync() { asm volatile("bar.sync 1, %0;" ::"n"(kTcWorkers) : "memory"); }
__device__ __forceinline__ bool workers_and(bool v) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbar.red.and.pred q, 1, %2, p;\n\tselp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)v), "n"(kTcWorkers)
      : "memory");
  return r != 0;
}
__device__ __forceinline__ void mbar_arrive(uint32_t addr) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(addr) : "memory");
}

template <int NR>
__global__ void __launch_bounds__(kTcThreads, 1)
    gram_tc_kernel(const StepDesc* __restrict__ descs, const int64_t* __restrict__ base, int njobs) {
  using TS = TcShape<NR>;
  extern __shared__ __align__(1024) unsigned char tsm[];
  const int64_t gb = blockIdx.x;
  const int jb = njobs > 1 ? find_job(base, njobs, gb) : 0;
  const StepDesc* __restrict__ dp = descs + jb;
  const int64_t lb = gb - base[jb];
  const int nb = dp->gram_blocks;
  const int64_t I = dp->I;
  const float* __restrict__ A = dp->A;  // I x NR, padding columns zero
  // this block's rows [r0, r1): contiguous, whole fills except the last
  const int64_t per = ((I + nb - 1) / nb + kTcKB - 1) / kTcKB * kTcKB;
  const int64_t r0 = min(I, lb * per), r1 = min(I, r0 + per);
  const int nf = (int)((r1 - r0 + kTcKB - 1) / kTcKB);

  unsigned char* slices = tsm;                      // 2 fills of slices
  unsigned char* raw = tsm + 2 * TS::SLICEBUF;      // kTcNraw fills of raw rows
  unsigned* cmax = reinterpret_cast<unsigned*>(tsm + TS::REGION);
  int* cexp = reinterpret_cast<int*>(cmax + NR);
  uint64_t* bars = reinterpret_cast<uint64_t*>(cexp + NR);  // 8-byte aligned: REGION and 2 NR ints are
  uint32_t* misc = reinterpret_cast<uint32_t*>(bars + TS::NBAR);  // tslot, abort, issued counts
  volatile uint32_t* abort_flag = misc + 1;
  uint32_t* iss = misc + 2;  // [0, kTcNraw): raw copies per stage; [kTcNraw, +2): commits per buffer
  const uint32_t bar1 = smem_u32(bars), bar2 = bar1 + 8 * TS::NST1, barm = bar2 + 8 * kTcNraw, bary = barm + 16;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const bool worker = warp < kTcWorkers / 32;

  if (tid < NR) cmax[tid] = 0u;
  if (tid == 0) {
    for (int i = 0; i < TS::NST1 + kTcNraw + 2; ++i) mbar_init(bar1 + 8 * i, 1);
    for (int i = 0; i < 2; ++i) mbar_init(bary + 8 * i, kTcWorkers);
    *abort_flag = 0u;
    for (int i = 0; i < kTcNraw + 2; ++i) iss[i] = 0u;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  if (warp == kTcWorkers / 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(misc)),
                 "r"(TS::TALLOC)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = misc[0];
  bool ok = ((reinterpret_cast<uintptr_t>(A) & 15u) == 0) && dp->Rp == NR;  // bulk copies need 16-byte rows
  auto fill_bytes = [&](int f) { return (uint32_t)(min((int64_t)kTcKB, r1 - r0 - (int64_t)f * kTcKB) * NR * 4); };
  auto fill_src = [&](int f) { return A + (r0 + (int64_t)f * kTcKB) * NR; };

  BarTrack t1[TS::NST1], t2[kTcNraw], tm[2];
  // ---- pass 1 (workers): column maxima over the block's rows
  if (worker) {
    if (ok) {
      if (tid == 0)
        for (int f = 0; f < min(nf, TS::NST1); ++f)
          bulk_load(smem_u32(tsm + f * TS::STAGE), fill_src(f), fill_bytes(f), bar1 + 8 * f);
      for (int f = 0; f < min(nf, TS::NST1); ++f) t1[f].issued = 1;
      unsigned mx[4] = {0u, 0u, 0u, 0u};  // bits of |x|: they order as |x|, NaN above +inf
      const int c4 = (tid % (NR / 4)) * 4, rstep = kTcWorkers / (NR / 4);
      for (int f = 0; f < nf; ++f) {
        const int s = f % TS::NST1;
        ok = workers_and(ok && bar_wait_upto(bar1 + 8 * s, t1[s], (uint32_t)(f / TS::NST1)));
        if (!ok) break;
        const int nrb = (int)(fill_bytes(f) / (NR * 4));
        const float* st = reinterpret_cast<const float*>(tsm + s * TS::STAGE);
        for (int r = tid / (NR / 4); r < nrb; r += rstep) {
          const float4 v = *reinterpret_cast<const float4*>(st + r * NR + c4);
          mx[0] = max(mx[0], __float_as_uint(v.x) & 0x7FFFFFFFu);
          mx[1] = max(mx[1], __float_as_uint(v.y) & 0x7FFFFFFFu);
          mx[2] = max(mx[2], __float_as_uint(v.z) & 0x7FFFFFFFu);
          mx[3] = max(mx[3], __float_as_uint(v.w) & 0x7FFFFFFFu);
        }
        workers_sync();  // stage s consumed
        if (f + TS::NST1 < nf) {
          if (tid == 0)
            bulk_load(smem_u32(tsm + s * TS::STAGE), fill_src(f + TS::NST1), fill_bytes(f + TS::NST1), bar1 + 8 * s);
          ++t1[s].issued;
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) atomicMax(&cmax[c4 + u], mx[u]);
    }
    if (!ok) {
      for (int s = 0; s < TS::NST1; ++s) bar_drain(bar1 + 8 * s, t1[s]);
      if (tid == 0) *abort_flag = 1u;
    }
    workers_sync();
    if (tid < NR) {
      const float m = __uint_as_float(cmax[tid]);
      int E = 0;
      if (m > 0.f && m <= 3.0e38f) frexpf(m, &E);  // m < 2^E; non-finite columns keep E = 0 and stay non-finite
      cexp[tid] = E;
    }
    // the stacks read past the seventh slice: that one stays zero
    for (int e = tid; e < 2 * TS::SLICE_BYTES / 16; e += kTcWorkers) {
      const int bsel = e / (TS::SLICE_BYTES / 16), off = e % (TS::SLICE_BYTES / 16);
      reinterpret_cast<uint4*>(slices + bsel * TS::SLICEBUF + kTcSlices * TS::SLICE_BYTES)[off] = make_uint4(0, 0, 0, 0);
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  }
  __syncthreads();
  ok = ok && *abort_flag == 0u;

  // ---- pass 2
  // kind::f16 instruction descriptor: FP32 accumulator, BF16 A and B, both K-major, M = N = 128
  const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTcN >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
  // worker's tensor-memory lane (quadrant warp % 4) and column half (warp / 4)
  const int qd = warp & 3, half = (warp >> 2) & 1;
  const int mrow = 32 * qd + lane, br = mrow / NR;
  const uint32_t tlane = tbase + ((uint32_t)(32 * qd) << 16);
  float hi[NR], lo[NR];
#pragma unroll
  for (int i = 0; i < NR; ++i) hi[i] = lo[i] = 0.f;
  // read back every accumulator into the (hi, lo) sums of entries (j, k)
  auto readback = [&]() {
#pragma unroll
    for (int a = 0; a < TS::NACC; ++a) {
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        float v[16];
        tmem_ld16(tlane + (uint32_t)(a * kTcN + 64 * half + 16 * g), v);
        const int bc = (64 * half + 16 * g) / NR;                 // block column
        const float w = pow2f(-7 * (2 + a * TS::G + br + bc));    // diagonal t + r + c
        const int k0 = (16 * g) % NR;                             // 64 * half is a multiple of NR
#pragma unroll
        for (int i = 0; i < 16; ++i) two_sum_acc(hi[k0 + i], lo[k0 + i], __fmul_rn(v[i], w));
      }
    }
#pragma unroll
    for (int i = 0; i < NR; ++i) renorm(hi[i], lo[i]);
  };

  if (!worker) {
    // ---- the issuing warp: copies and products
    if (lane == 0 && ok && nf > 0) {
      uint32_t niss[kTcNraw + 2] = {};
      for (int f = 0; f < min(nf, kTcNraw); ++f) {
        bulk_load(smem_u32(raw + f * TS::STAGE), fill_src(f), fill_bytes(f), bar2 + 8 * f);
        ++niss[f];
      }
      BarTrack ty[2];
      unsigned live = 0;  // accumulators written since their restart
      for (int f = 0; f < nf; ++f) {
        const int b = f & 1;
        if (!bar_wait_upto(bary + 8 * b, ty[b], (uint32_t)(f >> 1))) {  // workers sliced fill f
          *abort_flag = 1u;
          break;
        }
        if (*abort_flag) break;
        tc_fence_after();
        if (f + kTcNraw < nf) {  // raw stage f % kTcNraw was consumed by the slicing of fill f
          const int st = f % kTcNraw;
          bulk_load(smem_u32(raw + st * TS::STAGE), fill_src(f + kTcNraw), fill_bytes(f + kTcNraw), bar2 + 8 * st);
          ++niss[st];
        }
        if (f % TS::PERIOD_FILLS == 0) live = 0u;
        // descriptors differ only in the start-address field, which stays below 2^14 (16-byte
        // units of shared memory), so each is the buffer's descriptor plus a constant
        const uint64_t d0 = smem_desc(smem_u32(slices + b * TS::SLICEBUF), 128, TS::SBO);
#pragma unroll
        for (int p = 1; p <= 7; p += TS::G)
#pragma unroll
          for (int q = 1; p + q <= 8; q += TS::G) {
            const int a = (p + q - 2) / TS::G;
            const uint32_t dcol = tbase + (uint32_t)(a * kTcN);
            const uint32_t first = (live >> a) & 1u;
#pragma unroll
            for (int ks = 0; ks < kTcKB / 16; ++ks) {
              const uint64_t ad = d0 + (uint64_t)(((p - 1) * TS::SLICE_BYTES + ks * 256) >> 4);
              const uint64_t bd = d0 + (uint64_t)(((q - 1) * TS::SLICE_BYTES + ks * 256) >> 4);
              asm volatile(
                  "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                  "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(dcol),
                  "l"(ad), "l"(bd), "r"(idesc), "r"(ks == 0 ? first : 1u)
                  : "memory");
            }
            live |= 1u << a;
          }
        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(barm + 8 * b)
                     : "memory");
        ++niss[kTcNraw + b];
      }
      for (int i = 0; i < kTcNraw + 2; ++i) iss[i] = niss[i];
    }
  } else if (ok && nf > 0) {
    // ---- the workers: slices and read-backs
    for (int f = 0; f < nf; ++f) {
      const int b = f & 1, st = f % kTcNraw;
      bool w = bar_wait_upto(bar2 + 8 * st, t2[st], (uint32_t)(f / kTcNraw));  // raw rows of fill f
      if (f >= 2) w = w && bar_wait_upto(barm + 8 * b, tm[b], (uint32_t)((f - 2) >> 1));  // slices b free
      ok = workers_and(ok && w && *abort_flag == 0u);
      if (!ok) {
        if (tid == 0) *abort_flag = 1u;
        mbar_arrive(bary + 8 * b);  // the issuing warp waits for this fill: let it see the abort
        break;
      }
      tc_fence_after();
      // slices of fill f: task (column m, 8-row group g); rows past the range are zero
      const int nrb = (int)(fill_bytes(f) / (NR * 4));
      const float* rw = reinterpret_cast<const float*>(raw + st * TS::STAGE);
      unsigned char* sb = slices + b * TS::SLICEBUF;
      for (int e = tid; e < NR * (kTcKB / 8); e += kTcWorkers) {
        const int m = e % NR, g = e / NR;
        const int E = cexp[m], Eh = E / 2;
        const float sc1 = pow2f(-Eh), sc2 = pow2f(Eh - E);
        float t[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int k = 8 * g + i;
          t[i] = k < nrb ? __fmul_rn(__fmul_rn(rw[k * NR + m], sc1), sc2) : 0.f;
        }
        unsigned char* dst = sb + (m / 8) * TS::SBO + g * 128 + (m % 8) * 16;
        // digit: rint(128 t) as (128 t + 1.5 2^23) - 1.5 2^23 (|128 t| <= 128 < 2^22, so exact
        // round-to-nearest), remainder 128 t - s exactly; an integer of at most 8 bits has its
        // BF16 value in the upper half of its FP32 bits
        constexpr float kMagic = 12582912.0f;
#pragma unroll
        for (int p = 0; p < kTcSlices; ++p) {
          uint32_t wv[4];
#pragma unroll
          for (int i = 0; i < 8; i += 2) {
            const float s0 = __fsub_rn(__fmaf_rn(t[i], 128.f, kMagic), kMagic);
            const float s1 = __fsub_rn(__fmaf_rn(t[i + 1], 128.f, kMagic), kMagic);
            t[i] = __fmaf_rn(t[i], 128.f, -s0);
            t[i + 1] = __fmaf_rn(t[i + 1], 128.f, -s1);
            wv[i / 2] = __byte_perm(__float_as_uint(s0), __float_as_uint(s1), 0x7632);
          }
          *reinterpret_cast<uint4*>(dst + p * TS::SLICE_BYTES) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
        }
      }
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      tc_fence_before();
      mbar_arrive(bary + 8 * b);  // fill f sliced
      if ((f + 1) % TS::PERIOD_FILLS == 0 && f + 1 < nf) {  // read back and restart every accumulator
        ok = workers_and(ok && bar_wait_upto(barm + 8 * b, tm[b], (uint32_t)(f >> 1)));
        if (!ok) {
          if (tid == 0) *abort_flag = 1u;
          mbar_arrive(bary + 8 * ((f + 1) & 1));  // the issuing warp waits for fill f + 1
          break;
        }
        tc_fence_after();
        readback();
        tc_fence_before();
      }
    }
    if (ok) {
      const int fl = nf - 1;
      ok = workers_and(bar_wait_upto(barm + 8 * (fl & 1), tm[fl & 1], (uint32_t)(fl >> 1)));
    }
    if (ok) {
      tc_fence_after();
      readback();
    }
  }
  tc_fence_before();
  __syncthreads();
  ok = ok && *abort_flag == 0u;
  if (worker && !ok) {  // let every copy and product in flight land before the memory is released
    for (int s = 0; s < kTcNraw; ++s) {
      t2[s].issued = iss[s];
      bar_drain(bar2 + 8 * s, t2[s]);
    }
    for (int b = 0; b < 2; ++b) {
      tm[b].issued = iss[kTcNraw + b];
      bar_drain(barm + 8 * b, tm[b]);
    }
  }
  double* out = dp->gpart + lb * (int64_t)NR * NR;
  if (!ok) {
    for (int e = tid; e < NR * NR; e += kTcThreads) out[e] = __longlong_as_double(0x7ff8000000000000ll);
  } else {
    // ---- group sums into shared memory, then one FP64 entry each
    float2* comb = reinterpret_cast<float2*>(tsm);  // [group][column k][row j], rows padded to NR + 1
    if (worker) {
      const int j = mrow % NR, grp = br * 2 + half;
#pragma unroll
      for (int k = 0; k < NR; ++k) comb[(grp * NR + k) * TS::CSTRIDE + j] = make_float2(hi[k], lo[k]);
    }
    __syncthreads();
    for (int e = tid; e < NR * NR; e += kTcThreads) {
      const int j = e / NR, k = e % NR;
      const int a = min(j, k), c = max(j, k);  // the upper triangle, mirrored: the result is symmetric
      float H = 0.f, L = 0.f;
#pragma unroll
      for (int r = 0; r < TS::NQ; ++r) {
        const float2 v = comb[(r * NR + c) * TS::CSTRIDE + a];
        two_sum_acc(H, L, v.x);
        two_sum_acc(H, L, v.y);
      }
      renorm(H, L);
      const int sc = cexp[a] + cexp[c];
      out[e] = f32_scaled_to_f64(H, sc) + f32_scaled_to_f64(L, sc);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == kTcWorkers / 32)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "r"(TS::TALLOC) : "memory");
}

bool gram_on_tensor_cores(int Rp, int64_t I) { return (Rp == 32 || Rp == 64) && I * Rp >= (int64_t)1 << 20; }

int gram_tc_blocks(int64_t I) {
  const int64_t want = (I + kTcMinRows - 1) / kTcMinRows;
  return (int)std::max<int64_t>(1, std::min<int64_t>(want, 152));
}

void launch_gram_tc(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total_blocks, int Rp,
                    cudaStream_t st) {
  if (total_blocks <= 0) return;
  static const bool configured = [] {  // once per process, thread-safe
    cudaFuncSetAttribute(gram_tc_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcShape<32>::SMEM);
    cudaFuncSetAttribute(gram_tc_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TcShape<64>::SMEM);
    return true;
  }();
  (void)configured;
  if (Rp == 32)
    gram_tc_kernel<32><<<(unsigned)total_blocks, kTcThreads, TcShape<32>::SMEM, st>>>(d_descs, d_base, njobs);
  else
    gram_tc_kernel<64><<<(unsigned)total_blocks, kTcThreads, TcShape<64>::SMEM, st>>>(d_descs, d_base, njobs);
}

}  // namespace sacd
