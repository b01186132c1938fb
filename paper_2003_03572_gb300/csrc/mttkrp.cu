// Sparse MTTKRP M = X_(n) (Khatri-Rao of A_k, k != n)   (Eq. 9, first term; the slice form
// m_r = sum over Omega^(n)_q of x * prod_k a_k[i_k, r] of Sec. 4.4, all r at once).
//
// Layout: the nonzeros of mode n are sorted by row i_n (slice structure built at create time).
// They are cut into warp tiles of a fixed number of nonzeros (load balance does not depend on
// the row-length skew). Inside a warp, lane groups of LPR lanes each own one gathered factor
// row (LPR 16-byte vectors, 128-bit loads) and walk a contiguous sub-range of the tile,
// accumulating in FP32 registers. A row that lies wholly inside a sub-range is stored at once.
// Segments cut by a sub-range border are merged inside the warp (shared memory, fixed order);
// segments cut by a tile border become per-tile partials ("carries") that a fix-up kernel sums
// in a fixed order over a static list of split rows. No floating-point atomics: the result is
// bitwise reproducible for a given tiling.
#include "common.cuh"
#include "kernels.h"

namespace sacd {

template <int PREC>
struct GatherVec;

template <>
struct GatherVec<0> {  // FP32 rows: 4 columns per 16-byte vector
  static constexpr int W = 4;
  __device__ __forceinline__ static void load(const void* base, int64_t vec, float* out) {
    float4 v = __ldg(reinterpret_cast<const float4*>(base) + vec);
    out[0] = v.x; out[1] = v.y; out[2] = v.z; out[3] = v.w;
  }
};

template <>
struct GatherVec<1> {  // BF16 rows: 8 columns per 16-byte vector
  static constexpr int W = 8;
  __device__ __forceinline__ static void load(const void* base, int64_t vec, float* out) {
    uint4 v = __ldg(reinterpret_cast<const uint4*>(base) + vec);
    const uint32_t w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      out[2 * i] = __uint_as_float(w[i] << 16);
      out[2 * i + 1] = __uint_as_float(w[i] & 0xffff0000u);
    }
  }
};

// Per-warp scratch for the in-warp merge of open segments.
struct WarpPieces {
  float acc[2][256];     // [head/tail][group * Rp + column]; G * Rp <= 256 for every shape used
  int32_t row[2][32];
  int32_t flags[32];     // bit0 head valid (left-open), bit1 head also right-open, bit2 tail valid
};

#ifndef SACD_MTTKRP_WARPS
#define SACD_MTTKRP_WARPS 4
#endif
constexpr int kWarpsPerBlock = SACD_MTTKRP_WARPS;

// Index staging: a warp copies its lane groups' next nonzeros (row, value, other-mode indices)
// into shared memory with 16-byte asynchronous copies while it gathers and
// multiplies the current ones, so the DRAM latency of the sorted-nonzero stream overlaps the L2
// latency of the factor-row gathers. Two stages per warp; completion is the hardware's
// cp.async group wait (no spin loop). Copies of fewer than 16 valid bytes read only the valid
// bytes and zero-fill the rest, so nothing past a lane group's range is read.
#ifndef SACD_MTTKRP_STAGED
#define SACD_MTTKRP_STAGED 1
#endif
#ifndef SACD_MTTKRP_STAGE_NNZ
#define SACD_MTTKRP_STAGE_NNZ 0
#endif

// Packed two-lane FP32 arithmetic (sm_100 family): each lane is an IEEE round-to-nearest
// multiply or add, so the results equal the scalar operations element by element, at half the
// instruction count.
#ifndef SACD_MTTKRP_F32X2
#define SACD_MTTKRP_F32X2 1
#endif
__device__ __forceinline__ void mul2_inplace(float& a0, float& a1, float b0, float b1) {
#if !SACD_MTTKRP_F32X2
  a0 = __fmul_rn(a0, b0);
  a1 = __fmul_rn(a1, b1);
  return;
#endif
  asm("{\n\t.reg .b64 ra, rb;\n\tmov.b64 ra, {%0, %1};\n\tmov.b64 rb, {%2, %3};\n\t"
      "mul.rn.f32x2 ra, ra, rb;\n\tmov.b64 {%0, %1}, ra;\n\t}"
      : "+f"(a0), "+f"(a1)
      : "f"(b0), "f"(b1));
}
__device__ __forceinline__ void add2_inplace(float& a0, float& a1, float b0, float b1) {
#if !SACD_MTTKRP_F32X2
  a0 = __fadd_rn(a0, b0);
  a1 = __fadd_rn(a1, b1);
  return;
#endif
  asm("{\n\t.reg .b64 ra, rb;\n\tmov.b64 ra, {%0, %1};\n\tmov.b64 rb, {%2, %3};\n\t"
      "add.rn.f32x2 ra, ra, rb;\n\tmov.b64 {%0, %1}, ra;\n\t}"
      : "+f"(a0), "+f"(a1)
      : "f"(b0), "f"(b1));
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::: "memory"); }
// Nonzeros whose gathers a lane group issues together, resident warps per SM (which bound the
// registers) and index-stage size, per kernel variant, measured on GB300: rows of up to 4 floats
// per lane (5M-nonzero Zipf R = 32 FP32) 4 nonzeros, 16 warps, 128-nonzero stages; wider rows
// (50M-nonzero 4-mode R = 64 BF16) 2 nonzeros, 24 warps, 64-nonzero stages. The other pairs
// measured 5-30% slower.
#ifndef SACD_MTTKRP_UNROLL
#define SACD_MTTKRP_UNROLL 0
#endif
#ifndef SACD_MTTKRP_MINB
#define SACD_MTTKRP_MINB 0
#endif
// Resident warps per SM for rows of more than 4 floats per lane (BF16 gathers), measured on the
// 50M-nonzero rank-64 tensor: 28 (72 registers, 84 bytes spilled) 4.77 ms per iteration, 24 (80,
// 52 bytes) 4.84 ms, 20 (96, 8 bytes) 5.16 ms: more gathers in flight outweigh the spills.
#ifndef SACD_MTTKRP_WIDE_WARPS
#define SACD_MTTKRP_WIDE_WARPS 28
#endif

// Staged index rows of the lane groups start `cp` words apart; each group reads `rw` consecutive
// words of its row at once. The number of groups whose words fall in the busiest bank (the
// wavefronts of one such read when the groups' addresses differ).
__host__ __device__ constexpr int stage_bank_load(int g, int cp, int rw) {
  int worst = 0;
  for (int b = 0; b < 32; ++b) {
    int hits = 0;
    for (int x = 0; x < g; ++x)
      if (((b - x * cp) % 32 + 32) % 32 < rw) ++hits;
    worst = hits > worst ? hits : worst;
  }
  return worst;
}
// The row pitch of the stage: among sc, sc + 4, ..., sc + 28 (multiples of 4 keep every row
// 16-byte aligned for cp.async) the one with the lightest busiest bank, the smallest on ties.
__host__ __device__ constexpr int stage_pitch(int g, int sc, int rw) {
  int best = sc, cost = stage_bank_load(g, sc, rw);
  for (int k = 1; k < 8; ++k) {
    const int c = stage_bank_load(g, sc + 4 * k, rw);
    if (c < cost) {
      cost = c;
      best = sc + 4 * k;
    }
  }
  return best;
}

template <int PREC, int RV>
struct TileShape {
  static constexpr int W = GatherVec<PREC>::W;
  static constexpr int LPR = RV < 32 ? RV : 32;  // lanes per row
  static constexpr int CPL = RV / LPR;           // vectors per lane
  static constexpr int G = 32 / LPR;             // lane groups per warp
  static constexpr int NV = CPL * W;             // floats per lane
  static constexpr int U = SACD_MTTKRP_UNROLL ? SACD_MTTKRP_UNROLL : (NV <= 4 ? 4 : 2);
  // resident warps per SM: 16 for rows of up to 4 floats per lane, SACD_MTTKRP_WIDE_WARPS for wider ones
  static constexpr int MINB = SACD_MTTKRP_MINB ? SACD_MTTKRP_MINB : (NV <= 4 ? 16 : SACD_MTTKRP_WIDE_WARPS) / kWarpsPerBlock;
  // nonzeros of a warp in one index stage (measured: 128 for the narrow rows, 64 for the wide
  // ones), and per lane group: whole 16-byte pieces and whole unroll steps
  static constexpr int SNNZ = SACD_MTTKRP_STAGE_NNZ ? SACD_MTTKRP_STAGE_NNZ : (NV <= 4 ? 128 : 64);
  static constexpr int SMIN = U > 4 ? U : 4;
  static constexpr int SC = SNNZ / G > SMIN ? SNNZ / G : SMIN;
  // Words between the lane groups' rows of a staged array. The groups read their next RW words
  // (one int4, int2 or int32 per array) at once. At a pitch of SC (a multiple of 16 from 16 up)
  // groups g and g + 2 share banks: in the BF16 kernel at R = 64 (two words per read) every shared
  // load took two wavefronts (ncu), so reads narrower than 16 bytes take the pitch search (the
  // BF16 mode-step and objective passes gained 1.8% and 2.3%). Padding the 16-byte reads of the
  // FP32 kernel at R = 32 made it 4% slower, so those keep SC.
  static constexpr int RW = (U == 4 || U == 2) ? U : 1;
  static constexpr int CP = RW == 4 ? SC : stage_pitch(G, SC, RW);
  __host__ __device__ static constexpr int stage_words(int nother) { return (2 + nother) * G * CP; }
};

template <int NV>
__device__ __forceinline__ void store_row_chunk(float* Mrow, int col0, const float* v) {
  // col0 is a multiple of 4; NV is 4 or 8
#pragma unroll
  for (int i = 0; i < NV; i += 4)
    *reinterpret_cast<float4*>(Mrow + col0 + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
}

template <int PREC, int RV>
__device__ __forceinline__ void lane_cols(int lig, int k, int& col0) {
  // column of the k-th vector owned by lane `lig` of its group
  col0 = (lig + k * TileShape<PREC, RV>::LPR) * GatherVec<PREC>::W;
}

template <int PREC, int RV>
__device__ void zero_rows(float* __restrict__ Mout, int Rp, int64_t r0, int64_t r1, int lig) {
  using S = TileShape<PREC, RV>;
  float z[S::W];
#pragma unroll
  for (int i = 0; i < S::W; ++i) z[i] = 0.f;
  for (int64_t r = r0; r < r1; ++r) {
    float* Mrow = Mout + r * Rp;
#pragma unroll
    for (int k = 0; k < S::CPL; ++k) {
      int c0;
      lane_cols<PREC, RV>(lig, k, c0);
      store_row_chunk<S::W>(Mrow, c0, z);
    }
  }
}

// One warp tile. NO = number of other modes (N-1) when known at compile time, 0 = any.
// Element positions fit in 32 bits (nnz <= 2^31 - 1); addresses are formed in 64 bits.
// DUAL (BF16 layout only): the rows are gathered from the FP32 master factors of `dpf`; each value
// rounded to BF16 (round to nearest even, the BF16 mirror's own rounding) feeds the same product
// chain as a BF16 gather, so dp's M and partials are bit for bit those of the BF16 kernel, and the
// unrounded values feed a second chain whose sums go to dpf's M and partials (the same segments,
// merges and tile slots).
template <int PREC, int RV, int NO, bool DUAL = false>
__device__ void mttkrp_tile(const StepDesc* __restrict__ dp, int64_t tile, WarpPieces& wp, int32_t* sbuf,
                            const StepDesc* __restrict__ dpf = nullptr, WarpPieces* wpf = nullptr) {
  static_assert(!DUAL || PREC == 1, "the dual tile keeps the BF16 layout");
  using S = TileShape<PREC, RV>;
  constexpr int MAXO = NO > 0 ? NO : SACD_MAXN - 1;
  constexpr int kUnroll = S::U;
  const int lane = lane_id();
  const int g = lane / S::LPR;   // group
  const int lig = lane % S::LPR; // lane in group
  // descriptor fields in registers (stores below cannot alias them)
  const int nnz = (int)dp->nnz;
  const int tile_nnz = dp->tile, sub = dp->sub, Rp = dp->Rp;
  const int64_t I = dp->I;
  float* __restrict__ Mout = dp->M;
  float* __restrict__ carry = dp->carry;
  const int32_t* __restrict__ rowid = dp->rowid;
  const float* __restrict__ val = dp->val;
  const int nother = NO > 0 ? NO : dp->nother;
  const int32_t* ci[MAXO];
  const void* fac[MAXO];
  const int64_t cstride = dp->cstride;
#pragma unroll
  for (int m = 0; m < MAXO; ++m) {
    ci[m] = dp->cidx + (int64_t)m * cstride;
    fac[m] = dp->fac[m];
  }
  constexpr int NVF = DUAL ? TileShape<PREC, RV>::NV : 1;  // floats per lane of the second chain
  const float* fac32[DUAL ? MAXO : 1];
  float* __restrict__ Mf = nullptr;
  float* __restrict__ carryf = nullptr;
  if constexpr (DUAL) {
#pragma unroll
    for (int m = 0; m < MAXO; ++m) fac32[m] = static_cast<const float*>(dpf->fac[m]);
    Mf = dpf->M;
    carryf = dpf->carry;
  }
  // 128-bit index loads of 4 consecutive nonzeros when every index row is 16-byte aligned
  // (tiles and sub-ranges start at multiples of 4 nonzeros)
  const bool vec = (((reinterpret_cast<uintptr_t>(rowid) | reinterpret_cast<uintptr_t>(val) |
                      reinterpret_cast<uintptr_t>(dp->cidx)) & 15) == 0) && ((cstride & 3) == 0);
  const int t0 = (int)(tile * tile_nnz);
  const int t1 = min(t0 + tile_nnz, nnz);
  const int a = min(t0 + g * sub, t1);
  const int b = min(a + sub, t1);

  float acc[S::NV];
  float accf[NVF];
#pragma unroll
  for (int i = 0; i < S::NV; ++i) acc[i] = 0.f;
#pragma unroll
  for (int i = 0; i < NVF; ++i) accf[i] = 0.f;
  int32_t cur = -1;
  int seg = a;
  int flags = 0;
  const int32_t before = (a > 0 && a < b) ? __ldg(rowid + a - 1) : -1;
  const int32_t after = (b < nnz && a < b) ? __ldg(rowid + b) : -1;

  // close the segment [s, e_end) of row `row`
  auto close_seg = [&](int32_t row, int s, int e_end) {
    const bool lopen = (s == a) && (before == row);
    const bool ropen = (e_end == b) && (after == row);
    if (!lopen && !ropen) {
      float* Mrow = Mout + (int64_t)row * Rp;
#pragma unroll
      for (int k = 0; k < S::CPL; ++k) {
        int c0;
        lane_cols<PREC, RV>(lig, k, c0);
        store_row_chunk<S::W>(Mrow, c0, acc + k * S::W);
        if constexpr (DUAL) store_row_chunk<S::W>(Mf + (int64_t)row * Rp, c0, accf + k * S::W);
      }
    } else {
      const int slot = lopen ? 0 : 1;
      float* dst = &wp.acc[slot][0] + (g * Rp);
#pragma unroll
      for (int k = 0; k < S::CPL; ++k) {
        int c0;
        lane_cols<PREC, RV>(lig, k, c0);
#pragma unroll
        for (int i = 0; i < S::W; ++i) dst[c0 + i] = acc[k * S::W + i];
        if constexpr (DUAL) {
          float* dstf = &wpf->acc[slot][0] + (g * Rp);
#pragma unroll
          for (int i = 0; i < S::W; ++i) dstf[c0 + i] = accf[k * S::W + i];
        }
      }
      if (lig == 0) wp.row[slot][g] = row;
      flags |= lopen ? (ropen ? 3 : 1) : 4;
    }
  };

  // gathers, products and row accumulation of the nonzeros e0 .. e0+kUnroll-1 below `lim`
  auto consume = [&](int e0, const int32_t* rows, const float* xs, const uint32_t (*ix)[kUnroll], int lim) {
    float prod[kUnroll][S::NV];
    float prodf[kUnroll][NVF];
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      if (e0 + u < lim) {
#pragma unroll
        for (int i = 0; i < S::NV; ++i) prod[u][i] = xs[u];
        if constexpr (DUAL) {
#pragma unroll
          for (int i = 0; i < NVF; ++i) prodf[u][i] = xs[u];
        }
#pragma unroll
        for (int m = 0; m < MAXO; ++m) {
          if (NO > 0 || m < nother) {
#pragma unroll
            for (int k = 0; k < S::CPL; ++k) {
              float v[S::W];
              if constexpr (DUAL) {
                int c0;
                lane_cols<PREC, RV>(lig, k, c0);
                const float4* src = reinterpret_cast<const float4*>(fac32[m] + (int64_t)ix[m][u] * Rp + c0);
                const float4 f0 = __ldg(src), f1 = __ldg(src + 1);
                const float vf[8] = {f0.x, f0.y, f0.z, f0.w, f1.x, f1.y, f1.z, f1.w};
#pragma unroll
                for (int i = 0; i < S::W; ++i) v[i] = __bfloat162float(__float2bfloat16_rn(vf[i]));
#pragma unroll
                for (int i = 0; i < S::W; i += 2)
                  mul2_inplace(prodf[u][k * S::W + i], prodf[u][k * S::W + i + 1], vf[i], vf[i + 1]);
              } else {
                GatherVec<PREC>::load(fac[m], (int64_t)ix[m][u] * RV + lig + k * S::LPR, v);
              }
#pragma unroll
              for (int i = 0; i < S::W; i += 2)
                mul2_inplace(prod[u][k * S::W + i], prod[u][k * S::W + i + 1], v[i], v[i + 1]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) {
      const int e = e0 + u;
      if (e < lim) {
        if (rows[u] != cur) {
          if (cur >= 0) close_seg(cur, seg, e);
          // rows strictly between the previous nonzero's row and this one are empty
          const int32_t prev = (e == a) ? before : cur;
          if (prev != rows[u]) {
            zero_rows<PREC, RV>(Mout, Rp, (int64_t)prev + 1, rows[u], lig);
            if constexpr (DUAL) zero_rows<PREC, RV>(Mf, Rp, (int64_t)prev + 1, rows[u], lig);
          }
          cur = rows[u];
          seg = e;
#pragma unroll
          for (int i = 0; i < S::NV; ++i) acc[i] = 0.f;
#pragma unroll
          for (int i = 0; i < NVF; ++i) accf[i] = 0.f;
        }
#pragma unroll
        for (int i = 0; i < S::NV; i += 2) add2_inplace(acc[i], acc[i + 1], prod[u][i], prod[u][i + 1]);
        if constexpr (DUAL) {
#pragma unroll
          for (int i = 0; i < NVF; i += 2) add2_inplace(accf[i], accf[i + 1], prodf[u][i], prodf[u][i + 1]);
        }
      }
    }
  };

  bool staged = false;
  if constexpr (SACD_MTTKRP_STAGED && (NO == 2 || NO == 3)) staged = vec && (sub & 3) == 0;
  if constexpr (SACD_MTTKRP_STAGED && (NO == 2 || NO == 3)) {
   if (staged) {
    constexpr int NA = 2 + NO;  // staged arrays: rows, values, other-mode indices
    constexpr int C = S::SC;                    // nonzeros per lane group per stage
    constexpr int CP = S::CP;                   // words between lane groups' rows
    constexpr int QPG = C / 4;                  // 16-byte pieces per lane group and array
    constexpr int NQ = NA * S::G * QPG;         // pieces per stage
    constexpr int SLOT = S::stage_words(NA - 2);  // int32 words per stage
    static_assert(C % 4 == 0 && C % kUnroll == 0 && CP % 4 == 0 && CP >= C,
                  "a stage holds whole 16-byte pieces and unroll steps, rows 16-byte aligned");
    const int32_t* cidx0 = dp->cidx;
    const int nch = (sub + C - 1) / C;
    auto issue = [&](int k) {
      int32_t* dst0 = sbuf + (k & 1) * SLOT;
      for (int q = lane; q < NQ; q += 32) {
        const int m = q / (S::G * QPG);
        const int r = q - m * (S::G * QPG);
        const int gg = r / QPG, p = r - gg * QPG;
        const int ag = min(t0 + gg * sub, t1), bg = min(ag + sub, t1);
        const int e = ag + k * C + 4 * p;
        const int valid = max(0, min(4, bg - e));
        const int32_t* arr = m == 0 ? rowid
                           : (m == 1 ? reinterpret_cast<const int32_t*>(val) : cidx0 + (int64_t)(m - 2) * cstride);
        cp_async16(dst0 + (m * S::G + gg) * CP + 4 * p, valid > 0 ? arr + e : arr, valid * 4);
      }
      cp_async_commit();
    };
    issue(0);
    for (int k = 0; k < nch; ++k) {
      if (k + 1 < nch) issue(k + 1); else cp_async_commit();  // one group per chunk, possibly empty
      cp_async_wait1();
      __syncwarp();
      const int32_t* sb = sbuf + (k & 1) * SLOT;
      const int cs = a + k * C, ce = min(cs + C, b);
      for (int e0 = cs; e0 < ce; e0 += kUnroll) {
        const int o = e0 - cs;
        int32_t rows[kUnroll];
        float xs[kUnroll];
        uint32_t ix[MAXO][kUnroll];
        // o is a multiple of kUnroll and every array row starts 16-byte aligned
        if constexpr (kUnroll == 4) {
          const int4 r4 = *reinterpret_cast<const int4*>(sb + (0 * S::G + g) * CP + o);
          const int4 x4 = *reinterpret_cast<const int4*>(sb + (1 * S::G + g) * CP + o);
          rows[0] = r4.x; rows[1] = r4.y; rows[2] = r4.z; rows[3] = r4.w;
          xs[0] = __int_as_float(x4.x); xs[1] = __int_as_float(x4.y);
          xs[2] = __int_as_float(x4.z); xs[3] = __int_as_float(x4.w);
#pragma unroll
          for (int m = 0; m < MAXO; ++m) {
            const int4 c4 = *reinterpret_cast<const int4*>(sb + ((2 + m) * S::G + g) * CP + o);
            ix[m][0] = c4.x; ix[m][1] = c4.y; ix[m][2] = c4.z; ix[m][3] = c4.w;
          }
        } else if constexpr (kUnroll == 2) {
          const int2 r2 = *reinterpret_cast<const int2*>(sb + (0 * S::G + g) * CP + o);
          const int2 x2 = *reinterpret_cast<const int2*>(sb + (1 * S::G + g) * CP + o);
          rows[0] = r2.x; rows[1] = r2.y;
          xs[0] = __int_as_float(x2.x); xs[1] = __int_as_float(x2.y);
#pragma unroll
          for (int m = 0; m < MAXO; ++m) {
            const int2 c2 = *reinterpret_cast<const int2*>(sb + ((2 + m) * S::G + g) * CP + o);
            ix[m][0] = c2.x; ix[m][1] = c2.y;
          }
        } else {
#pragma unroll
          for (int u = 0; u < kUnroll; ++u) {
            rows[u] = sb[(0 * S::G + g) * CP + o + u];
            xs[u] = __int_as_float(sb[(1 * S::G + g) * CP + o + u]);
#pragma unroll
            for (int m = 0; m < MAXO; ++m) ix[m][u] = (uint32_t)sb[((2 + m) * S::G + g) * CP + o + u];
          }
        }
        consume(e0, rows, xs, ix, ce);
      }
      __syncwarp();  // the slot is refilled by the next issue
    }
   }
  }
  if (!staged) {
    for (int e0 = a; e0 < b; e0 += kUnroll) {
      int32_t rows[kUnroll];
      float xs[kUnroll];
      uint32_t ix[MAXO][kUnroll];
      bool loaded = false;
      if constexpr (kUnroll == 2) {
        if (vec && e0 + 2 <= b) {
          const int2 r2 = __ldg(reinterpret_cast<const int2*>(rowid + e0));
          const float2 x2 = __ldg(reinterpret_cast<const float2*>(val + e0));
          rows[0] = r2.x; rows[1] = r2.y;
          xs[0] = x2.x; xs[1] = x2.y;
#pragma unroll
          for (int m = 0; m < MAXO; ++m) {
            if (NO > 0 || m < nother) {
              const int2 c2 = __ldg(reinterpret_cast<const int2*>(ci[m] + e0));
              ix[m][0] = c2.x; ix[m][1] = c2.y;
            }
          }
          loaded = true;
        }
      } else if constexpr (kUnroll == 4) {
        if (vec && e0 + 4 <= b) {
          const int4 r4 = __ldg(reinterpret_cast<const int4*>(rowid + e0));
          const float4 x4 = __ldg(reinterpret_cast<const float4*>(val + e0));
          rows[0] = r4.x; rows[1] = r4.y; rows[2] = r4.z; rows[3] = r4.w;
          xs[0] = x4.x; xs[1] = x4.y; xs[2] = x4.z; xs[3] = x4.w;
#pragma unroll
          for (int m = 0; m < MAXO; ++m) {
            if (NO > 0 || m < nother) {
              const int4 c4 = __ldg(reinterpret_cast<const int4*>(ci[m] + e0));
              ix[m][0] = c4.x; ix[m][1] = c4.y; ix[m][2] = c4.z; ix[m][3] = c4.w;
            }
          }
          loaded = true;
        }
      }
      if (!loaded) {
#pragma unroll
        for (int u = 0; u < kUnroll; ++u) {
          const int e = e0 + u;
          rows[u] = e < b ? __ldg(rowid + e) : -1;
          xs[u] = e < b ? __ldg(val + e) : 0.f;
#pragma unroll
          for (int m = 0; m < MAXO; ++m)
            if (NO > 0 || m < nother) ix[m][u] = e < b ? (uint32_t)__ldg(ci[m] + e) : 0u;
        }
      }
      consume(e0, rows, xs, ix, b);
    }
  }
  if (cur >= 0) {
    close_seg(cur, seg, b);
    if (b == nnz) {
      zero_rows<PREC, RV>(Mout, Rp, (int64_t)cur + 1, I, lig);
      if constexpr (DUAL) zero_rows<PREC, RV>(Mf, Rp, (int64_t)cur + 1, I, lig);
    }
  }
  if (lig == 0) wp.flags[g] = flags;
  __syncwarp();

  // In-warp merge of the open pieces, groups in order, by the lanes of group 0.
  if (g == 0) {
    bool run_valid = false, run_tile_left = false;
    int32_t run_row = -1;
    float run[S::NV];
    float runf[NVF];
    auto finish = [&](bool right_open_at_tile) {
      int64_t off;
      float* dst;
      float* dstf = nullptr;
      if (run_tile_left || right_open_at_tile) {
        const int slot = run_tile_left ? 0 : 1;
        off = (tile * 2 + slot) * (int64_t)Rp;
        dst = carry + off;
        if constexpr (DUAL) dstf = carryf + off;
      } else {
        off = (int64_t)run_row * Rp;
        dst = Mout + off;
        if constexpr (DUAL) dstf = Mf + off;
      }
#pragma unroll
      for (int k = 0; k < S::CPL; ++k) {
        int c0;
        lane_cols<PREC, RV>(lig, k, c0);
        store_row_chunk<S::W>(dst, c0, run + k * S::W);
        if constexpr (DUAL) store_row_chunk<S::W>(dstf, c0, runf + k * S::W);
      }
    };
    for (int gg = 0; gg < S::G; ++gg) {
      const int f = wp.flags[gg];
      if (f & 1) {
        const float* src = &wp.acc[0][0] + gg * Rp;
        const float* srcf = DUAL ? &wpf->acc[0][0] + gg * Rp : nullptr;
        if (!run_valid) {
          run_valid = true;
          run_tile_left = true;  // only possible for the tile's first group
          run_row = wp.row[0][gg];
#pragma unroll
          for (int k = 0; k < S::CPL; ++k) {
            int c0;
            lane_cols<PREC, RV>(lig, k, c0);
#pragma unroll
            for (int i = 0; i < S::W; ++i) run[k * S::W + i] = src[c0 + i];
            if constexpr (DUAL) {
#pragma unroll
              for (int i = 0; i < S::W; ++i) runf[k * S::W + i] = srcf[c0 + i];
            }
          }
        } else {
#pragma unroll
          for (int k = 0; k < S::CPL; ++k) {
            int c0;
            lane_cols<PREC, RV>(lig, k, c0);
#pragma unroll
            for (int i = 0; i < S::W; ++i) run[k * S::W + i] += src[c0 + i];
            if constexpr (DUAL) {
#pragma unroll
              for (int i = 0; i < S::W; ++i) runf[k * S::W + i] += srcf[c0 + i];
            }
          }
        }
        if (!(f & 2)) {
          finish(false);
          run_valid = false;
        }
      }
      if (f & 4) {
        const float* src = &wp.acc[1][0] + gg * Rp;
        run_valid = true;
        run_tile_left = false;
        run_row = wp.row[1][gg];
#pragma unroll
        for (int k = 0; k < S::CPL; ++k) {
          int c0;
          lane_cols<PREC, RV>(lig, k, c0);
#pragma unroll
          for (int i = 0; i < S::W; ++i) run[k * S::W + i] = src[c0 + i];
          if constexpr (DUAL) {
            const float* srcf = &wpf->acc[1][0] + gg * Rp;
#pragma unroll
            for (int i = 0; i < S::W; ++i) runf[k * S::W + i] = srcf[c0 + i];
          }
        }
      }
    }
    if (run_valid) finish(true);
  }
}

// 8 warps per block; TileShape::MINB resident blocks per SM bound the registers, so that
// enough gathers are in flight to cover the L2 latency.
template <int PREC, int RV, int NO>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, (TileShape<PREC, RV>::MINB))
    mttkrp_kernel(const StepDesc* __restrict__ descs, const int64_t* __restrict__ tile_base, int njobs,
                  int64_t total_tiles) {
  __shared__ WarpPieces pieces[kWarpsPerBlock];
  constexpr int kSlot = TileShape<PREC, RV>::stage_words(NO > 0 ? NO : 1);
  __shared__ __align__(16) int32_t stage[kWarpsPerBlock][(SACD_MTTKRP_STAGED && (NO == 2 || NO == 3)) ? 2 * kSlot : 4];
  const int warp = threadIdx.x >> 5;
  const int64_t gt = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
  if (gt >= total_tiles) return;
  const int j = njobs > 1 ? find_job(tile_base, njobs, gt) : 0;
  mttkrp_tile<PREC, RV, NO>(descs + j, gt - tile_base[j], pieces[warp], stage[warp]);
}

// The objective's FP32-gather MTTKRP of a mode and the BF16-gather MTTKRP of that mode's next step
// in one pass over its nonzeros (mttkrp_tile with DUAL): dB is the mode's descriptor (BF16 tiling,
// output M, partial buffer), dF the objective's (FP32 master factors, its own output and partial
// buffer). One job per launch. Resident warps per SM, measured on the 50M-nonzero rank-64 tensor:
// 20 (96 registers, 4 bytes spilled) beats 16 (127 registers, no spill) by 9% and 24 (80
// registers, 100 bytes spilled) by 7%.
#ifndef SACD_MTTKRP_DUAL_WARPS
#define SACD_MTTKRP_DUAL_WARPS 20
#endif
template <int RV, int NO>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, SACD_MTTKRP_DUAL_WARPS / kWarpsPerBlock)
    mttkrp_dual_kernel(const StepDesc* __restrict__ dB, const StepDesc* __restrict__ dF, int64_t total_tiles) {
  __shared__ WarpPieces pieces[kWarpsPerBlock];
  __shared__ WarpPieces piecesf[kWarpsPerBlock];
  constexpr int kSlot = TileShape<1, RV>::stage_words(NO);
  __shared__ __align__(16) int32_t stage[kWarpsPerBlock][SACD_MTTKRP_STAGED ? 2 * kSlot : 4];
  const int warp = threadIdx.x >> 5;
  const int64_t gt = (int64_t)blockIdx.x * kWarpsPerBlock + warp;
  if (gt >= total_tiles) return;
  mttkrp_tile<1, RV, NO, true>(dB, gt, pieces[warp], stage[warp], dF, &piecesf[warp]);
}

// Rows split across tiles, with few partials: one warp per row, partials summed in tile order.
__global__ void __launch_bounds__(256)
    fixup_light_kernel(const StepDesc* __restrict__ descs, const int64_t* __restrict__ item_base, int njobs,
                       int64_t total) {
  const int64_t gi = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (gi >= total) return;
  const int j = njobs > 1 ? find_job(item_base, njobs, gi) : 0;
  const StepDesc& d = descs[j];
  const int4 s = d.split_light[gi - item_base[j]];
  const int nvec = d.Rp >> 2;
  const float4* carry = reinterpret_cast<const float4*>(d.carry);
  float4* Mrow = reinterpret_cast<float4*>(d.M + (int64_t)s.x * d.Rp);
  for (int c = lane_id(); c < nvec; c += 32) {
    float4 acc = carry[((int64_t)s.y * 2 + 1) * nvec + c];
    for (int64_t t = s.y + 1; t <= s.z; ++t) {
      const float4 v = carry[(t * 2) * nvec + c];
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    Mrow[c] = acc;
  }
}

// Rows split across many tiles, two levels. Level 1: one block per chunk of at most
// kFixChunk partials of one row ({row, first tile, first partial, count}); threads take partials
// strided, then a fixed-shape tree in shared memory; the chunk sum goes to carry2. Level 2: one
// block per row sums its chunks' sums the same way into M. Partial k of a row whose first tile
// is tf is slot 1 of tile tf for k = 0 and slot 0 of tile tf + k otherwise.
__device__ __forceinline__ void block_tree_sum(const float4* __restrict__ src, int64_t stride_vec, int64_t P,
                                               int nvec, float4* __restrict__ dst, float4* red,
                                               const int64_t* __restrict__ idx_of /* nullable */,
                                               int64_t tf, int64_t k0) {
  for (int c0 = 0; c0 < nvec; c0 += 256) {
    const int cw = min(256, nvec - c0);  // vectors handled in this pass (cw divides 256)
    const int lanes = 256 / cw;
    const int c = c0 + (threadIdx.x % cw);
    const int pl = threadIdx.x / cw;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t p = pl; p < P; p += lanes) {
      int64_t off;
      if (idx_of == nullptr) {
        const int64_t k = k0 + p;
        off = ((tf + k) * 2 + (k == 0 ? 1 : 0)) * stride_vec;
      } else {
        off = (idx_of[0] + p) * stride_vec;
      }
      const float4 v = src[off + c];
      acc.x += v.x; acc.y += v.y; acc.z += v.z; acc.w += v.w;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int w = lanes >> 1; w >= 1; w >>= 1) {
      if (pl < w) {
        const float4 o = red[threadIdx.x + w * cw];
        float4 m = red[threadIdx.x];
        m.x += o.x; m.y += o.y; m.z += o.z; m.w += o.w;
        red[threadIdx.x] = m;
      }
      __syncthreads();
    }
    if (pl == 0) dst[c] = red[threadIdx.x];
    __syncthreads();
  }
}

__global__ void __launch_bounds__(256)
    fixup_chunk_kernel(const StepDesc* __restrict__ descs, const int64_t* __restrict__ item_base, int njobs,
                       int64_t total) {
  __shared__ float4 red[256];
  const int64_t gi = blockIdx.x;
  if (gi >= total) return;
  const int j = njobs > 1 ? find_job(item_base, njobs, gi) : 0;
  const StepDesc* __restrict__ dp = descs + j;
  const int64_t li = gi - item_base[j];
  const int4 it = dp->fix_chunks[li];  // {row (unused here), first tile, first partial, count}
  const int nvec = dp->Rp >> 2;
  block_tree_sum(reinterpret_cast<const float4*>(dp->carry), nvec, it.w, nvec,
                 reinterpret_cast<float4*>(dp->carry2) + li * nvec, red, nullptr, it.y, it.z);
}

__global__ void __launch_bounds__(256)
    fixup_heavy_kernel(const StepDesc* __restrict__ descs, const int64_t* __restrict__ item_base, int njobs,
                       int64_t total) {
  __shared__ float4 red[256];
  const int64_t gi = blockIdx.x;
  if (gi >= total) return;
  const int j = njobs > 1 ? find_job(item_base, njobs, gi) : 0;
  const StepDesc* __restrict__ dp = descs + j;
  const int4 s = dp->split_heavy[gi - item_base[j]];  // {row, first chunk, chunk count, 0}
  const int nvec = dp->Rp >> 2;
  const int64_t first = s.y;
  block_tree_sum(reinterpret_cast<const float4*>(dp->carry2), nvec, s.z, nvec,
                 reinterpret_cast<float4*>(dp->M + (int64_t)s.x * dp->Rp), red, &first, 0, 0);
}

template <int PREC, int NO>
static void launch_mttkrp_no(const StepDesc* d_descs, const int64_t* d_tile_base, int njobs, int64_t total_tiles,
                             int rv, cudaStream_t st) {
  const unsigned blocks = (unsigned)((total_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock);
  const int T = kWarpsPerBlock * 32;
  switch (rv) {
    case 1: if (PREC == 1) mttkrp_kernel<PREC, 1, NO><<<blocks, T, 0, st>>>(d_descs, d_tile_base, njobs, total_tiles); break;
    case 2: mttkrp_kernel<PREC, 2, NO><<<blocks, T, 0, st>>>(d_descs, d_tile_base, njobs, total_tiles); break;
    case 4: mttkrp_kernel<PREC, 4, NO><<<blocks, T, 0, st>>>(d_descs, d_tile_base, njobs, total_tiles); break;
    case 8: mttkrp_kernel<PREC, 8, NO><<<blocks, T, 0, st>>>(d_descs, d_tile_base, njobs, total_tiles); break;
    case 16: mttkrp_kernel<PREC, 16, NO><<<blocks, T, 0, st>>>(d_descs, d_tile_base, njobs, total_tiles); break;
    case 32: mttkrp_kernel<PREC, 32, NO><<<blocks, T, 0, st>>>(d_descs, d_tile_base, njobs, total_tiles); break;
    case 64: if (PREC == 0) mttkrp_kernel<PREC, 64, NO><<<blocks, T, 0, st>>>(d_descs, d_tile_base, njobs, total_tiles); break;
    default: break;
  }
}

template <int PREC>
static void launch_mttkrp_prec(const StepDesc* d_descs, const int64_t* d_tile_base, int njobs, int64_t total_tiles,
                               int rv, int nother, cudaStream_t st) {
  if (nother == 2)
    launch_mttkrp_no<PREC, 2>(d_descs, d_tile_base, njobs, total_tiles, rv, st);
  else if (nother == 3)
    launch_mttkrp_no<PREC, 3>(d_descs, d_tile_base, njobs, total_tiles, rv, st);
  else
    launch_mttkrp_no<PREC, 0>(d_descs, d_tile_base, njobs, total_tiles, rv, st);
}

// All jobs of one launch share the gathered-row width `rv` (16-byte vectors per row) and the
// number of other modes `nother`.
void launch_mttkrp(const StepDesc* d_descs, const int64_t* d_tile_base, int njobs, int64_t total_tiles, int prec,
                   int rv, int nother, cudaStream_t st) {
  if (total_tiles <= 0) return;
  if (prec == 0)
    launch_mttkrp_prec<0>(d_descs, d_tile_base, njobs, total_tiles, rv, nother, st);
  else
    launch_mttkrp_prec<1>(d_descs, d_tile_base, njobs, total_tiles, rv, nother, st);
}

bool mttkrp_dual_supported(int rv, int nother) { return (rv == 4 || rv == 8) && (nother == 2 || nother == 3); }

void launch_mttkrp_dual(const StepDesc* dB, const StepDesc* dF, int64_t total_tiles, int rv, int nother,
                        cudaStream_t st) {
  if (total_tiles <= 0) return;
  const unsigned blocks = (unsigned)((total_tiles + kWarpsPerBlock - 1) / kWarpsPerBlock);
  const int T = kWarpsPerBlock * 32;
  if (rv == 4 && nother == 2) mttkrp_dual_kernel<4, 2><<<blocks, T, 0, st>>>(dB, dF, total_tiles);
  else if (rv == 4 && nother == 3) mttkrp_dual_kernel<4, 3><<<blocks, T, 0, st>>>(dB, dF, total_tiles);
  else if (rv == 8 && nother == 2) mttkrp_dual_kernel<8, 2><<<blocks, T, 0, st>>>(dB, dF, total_tiles);
  else if (rv == 8 && nother == 3) mttkrp_dual_kernel<8, 3><<<blocks, T, 0, st>>>(dB, dF, total_tiles);
}

// row -> split entry map (-1 elsewhere; the caller fills it with -1 first)
__global__ void rowfix_kernel(const int4* __restrict__ light, int64_t nl, const int4* __restrict__ heavy, int64_t nh,
                              int32_t* __restrict__ rowfix) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nl) rowfix[light[i].x] = (int32_t)i;
  else if (i < nl + nh) rowfix[heavy[i - nl].x] = (int32_t)(-2 - (i - nl));
}

void launch_rowfix(const int4* light, int64_t nl, const int4* heavy, int64_t nh, int32_t* rowfix, cudaStream_t st) {
  if (nl + nh <= 0) return;
  rowfix_kernel<<<(unsigned)((nl + nh + 255) / 256), 256, 0, st>>>(light, nl, heavy, nh, rowfix);
}

void launch_fixup_light(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total, cudaStream_t st) {
  if (total <= 0) return;
  const int64_t blocks = (total * 32 + 255) / 256;
  fixup_light_kernel<<<(unsigned)blocks, 256, 0, st>>>(d_descs, d_base, njobs, total);
}

void launch_fixup_chunks(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total, cudaStream_t st) {
  if (total <= 0) return;
  fixup_chunk_kernel<<<(unsigned)total, 256, 0, st>>>(d_descs, d_base, njobs, total);
}

void launch_fixup_heavy(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total, cudaStream_t st) {
  if (total <= 0) return;
  fixup_heavy_kernel<<<(unsigned)total, 256, 0, st>>>(d_descs, d_base, njobs, total);
}

}  // namespace sacd
