// The part of a SaCD mode step that follows the MTTKRP (Algorithm 1, one factor block):
//   hl     H = Hadamard of the other Grams (Eq. 10), L = ||H|| (Algorithm 1), 1/h_rr, L/2
//   pass1  G = A H - M (Eq. 9, 14), z (Eq. 20) for every element, ti = sum z (Eq. 25); the last
//          block picks the selection branch (first visit / Eq. 24 / Eq. 27)
//   pass2  selection and the projected update of the selected elements (Eq. 11-13), columns in
//          order within a row, with the gradient fix-up; z^{k-1} <- z; BF16 mirror refresh
//   gram   A^T A of the updated factor, FP64 result from compensated FP32 products and sums;
//          gram_reduce sums the per-block partials
//   fit    f = ||X||^2 - 2 <X, model> + ||model||^2 (Eq. 6-8) in FP64
// GB300 runs FP64 at a small fraction of its FP32 rate, so the sums that decide accuracy (the
// Gauss-Seidel gradient corrections, the Grams, A H - M for the GCD variant) use error-free FP32
// transformations (exact products and sums carried as (hi, lo) pairs) instead of FP64 FMAs;
// A H - M with the Frobenius or spectral L is a plain FP32 FMA sum, accurate enough for the step.
#include <algorithm>

#include "common.cuh"
#include "kernels.h"
#include "rowpass.cuh"

namespace sacd {

// ------------------------------------------------------------------------------------------
// H, L, 1/h, L/2
__global__ void __launch_bounds__(256) hl_kernel(const StepDesc* __restrict__ descs) {
  const StepDesc* __restrict__ dp = descs + blockIdx.x;
  __shared__ double red[256];
  __shared__ double v[SACD_MAXR];
  __shared__ const double* grams[SACD_MAXN];
  const int R = dp->R, Rp = dp->Rp, N = dp->N, n = dp->n, lnorm = dp->lnorm;
  double* __restrict__ H = dp->H;
  float* __restrict__ Hf = dp->Hf;
  if (threadIdx.x < SACD_MAXN) grams[threadIdx.x] = threadIdx.x < N ? dp->gram[threadIdx.x] : nullptr;
  __syncthreads();
  double ss = 0.0;
  for (int e = threadIdx.x; e < Rp * Rp; e += blockDim.x) {
    const int i = e / Rp, j = e - (e / Rp) * Rp;
    double h = 0.0;
    if (i < R && j < R) {
      h = 1.0;
      for (int k = 0; k < N; ++k)
        if (k != n) h *= __ldg(grams[k] + e);
    }
    H[e] = h;
    Hf[e] = (float)h;
    ss += h * h;
  }
  const double Lfro = sqrt(block_sum(ss, red));
  double L = Lfro;
  if (lnorm == 1 && R > 0) {
    // largest eigenvalue of the symmetric PSD matrix H by power iteration
    for (int i = threadIdx.x; i < R; i += blockDim.x) v[i] = 1.0 / sqrt((double)R);
    __syncthreads();
    double lam = 0.0;
    for (int it = 0; it < 500; ++it) {
      double w = 0.0;
      const int i = threadIdx.x;
      if (i < R) {
        for (int j = 0; j < R; ++j) w += H[i * Rp + j] * v[j];
      }
      const double nn = sqrt(block_sum(i < R ? w * w : 0.0, red));
      if (i < R) v[i] = nn > 0 ? w / nn : 0.0;
      __syncthreads();
      const bool done = fabs(nn - lam) <= 1e-15 * nn;
      lam = nn;
      if (done) break;
    }
    L = lam;
  }
  // h_rr of the coordinate steps; an h_rr at or below max(2^-40 max_j h_jj, 2^-126) counts as 0
  // (a column whose other-mode factors have collapsed takes no step: its exact step g/h_rr
  // would leave the FP32 range, and 1/h_rr must stay a finite FP32 value)
  double hmax = 0.0;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double h = 1.0;
    for (int k = 0; k < N; ++k)
      if (k != n) h *= __ldg(grams[k] + r * Rp + r);
    v[r] = h;
    hmax = fmax(hmax, h);
  }
  red[threadIdx.x] = hmax;
  __syncthreads();
  for (int w = blockDim.x >> 1; w >= 1; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
    __syncthreads();
  }
  const double hthr = fmax(0x1p-40 * red[0], 0x1p-126);
  __syncthreads();
  for (int r = threadIdx.x; r < Rp; r += blockDim.x) {
    float ih = 0.f, lhv = 0.f;
    if (r < R) {
      const double h = v[r];
      if (h > hthr) ih = (float)(1.0 / h);
      lhv = (float)(0.5 * (lnorm == 2 ? h : L));
    }
    dp->invh[r] = ih;
    dp->lh[r] = lhv;
  }
  if (threadIdx.x == 0) {
    dp->state[ST_L] = (lnorm == 2) ? 0.0 : L;
    *dp->nsel = 0ull;
  }
}

void launch_hl(const StepDesc* d_descs, int njobs, cudaStream_t st) {
  hl_kernel<<<njobs, 256, 0, st>>>(d_descs);
}

// Row passes: 256 threads per block, TPR = Rp/8 threads per row, each thread owns 8 adjacent
// columns of one row; RB = 256/TPR rows per block.
int rows_per_block(int Rp) { return 256 / (Rp / 8); }
int rows_per_block_pass1(int Rp) { return rows_per_block(Rp); }
int rows_per_block_pass2(int Rp) { return rows_per_block(Rp); }
size_t pass_smem_bytes(int Rp) {
  const int RB = rows_per_block(Rp);
  size_t b = (size_t)RB * (Rp + 1) * sizeof(float);  // staged A rows
  if (Rp <= 64) b += (size_t)Rp * Rp * sizeof(float);  // H
  b += (size_t)RB * 32;                                // selection bytes (pass 2)
  b += (size_t)2 * Rp * sizeof(float);                 // 1/h_rr and L/2 (pass 2)
  return (b + 15) / 16 * 16;
}

// ------------------------------------------------------------------------------------------
// pass 1: G = A H - M (FP32 fused multiply-adds; compensated products for the GCD variant), z, ti
__global__ void __launch_bounds__(256, 4) pass1_kernel(const StepDesc* __restrict__ descs,
                                                   const int64_t* __restrict__ base, int njobs) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  __shared__ double red[256];
  __shared__ int amlast;
  const int64_t gb = blockIdx.x;
  const int jb = njobs > 1 ? find_job(base, njobs, gb) : 0;
  const StepDesc* __restrict__ dp = descs + jb;
  const int64_t lb = gb - base[jb];
  const int R = dp->R, Rp = dp->Rp, ST = Rp + 1;
  const int64_t I = dp->I;
  const float* __restrict__ A = dp->A;
  float* __restrict__ M = dp->M;
  const int32_t* __restrict__ rowfix = dp->rowfix;
  float* __restrict__ G = dp->G;
  const float* __restrict__ invh = dp->invh;
  const float* __restrict__ lh = dp->lh;
  const int TPR = Rp >> 3, RB = 256 / TPR;
  const int64_t row0 = lb * RB;
  const int nrows = (int)min((int64_t)RB, I - row0);
  float* As = sm;
  float* Hs = sm + RB * ST;
  const float* __restrict__ Hsrc = dp->Hf;
  stage_rows(A + row0 * Rp, As, nrows, Rp);
  if (Rp <= 64) {
    for (int e = threadIdx.x; e < Rp * Rp / 4; e += blockDim.x)
      reinterpret_cast<float4*>(Hs)[e] = __ldg(reinterpret_cast<const float4*>(Hsrc) + e);
  }
  const float* Hr = Rp <= 64 ? Hs : Hsrc;
  __syncthreads();
  const int rl = threadIdx.x / TPR, c0 = (threadIdx.x % TPR) * 8;
  float zsum = 0.f;
  float4 m0 = make_float4(0.f, 0.f, 0.f, 0.f), m1 = m0;
  if (rl < nrows) {
    // M of the row; rows split across MTTKRP tiles are finished here and written back
    const int64_t row = row0 + rl;
    float4* m4 = reinterpret_cast<float4*>(M + row * Rp + c0);
    const int32_t fx = rowfix ? __ldg(rowfix + row) : -1;
    if (fx != -1) {
      split_row_sum(dp, fx, c0, m0, m1);
      m4[0] = m0;
      m4[1] = m1;
    } else if (c0 < R) {
      m0 = m4[0];
      m1 = m4[1];
    }
  }
  if (rl < nrows && c0 < R) {
    const int64_t row = row0 + rl;
    // column pairs (c0 + 2k, c0 + 2k + 1) in packed registers
    f2p hi2[4], lo2[4] = {0ull, 0ull, 0ull, 0ull};
    const float* arow = As + rl * ST;
    if (dp->lnorm == 2) {
      // GCD's h_rr in place of L selects far more elements with larger steps, which amplify the
      // gradient error: compensated products (exact product + TwoSum), G + Glo unrounded
      hi2[0] = f2_pack(-m0.x, -m0.y); hi2[1] = f2_pack(-m0.z, -m0.w);
      hi2[2] = f2_pack(-m1.x, -m1.y); hi2[3] = f2_pack(-m1.z, -m1.w);
      for (int j = 0; j < R; ++j) {
        const float aj = arow[j];
        const f2p a2 = f2_pack(aj, aj), na2 = f2_pack(-aj, -aj);
        const ulonglong2 h0 = *reinterpret_cast<const ulonglong2*>(Hr + j * Rp + c0);
        const ulonglong2 h1 = *reinterpret_cast<const ulonglong2*>(Hr + j * Rp + c0 + 4);
        dot2_acc2(a2, na2, h0.x, hi2[0], lo2[0]);
        dot2_acc2(a2, na2, h0.y, hi2[1], lo2[1]);
        dot2_acc2(a2, na2, h1.x, hi2[2], lo2[2]);
        dot2_acc2(a2, na2, h1.y, hi2[3], lo2[3]);
      }
    } else {
      // Frobenius or spectral L: A H by FP32 fused multiply-adds (one rounding per product),
      // then one rounded subtraction of M; the step error stays two orders below the mode-step
      // tolerance (an emulation of this order on the parity shapes: <= 6e-7 of ||A||)
      hi2[0] = hi2[1] = hi2[2] = hi2[3] = 0ull;
      for (int j = 0; j < R; ++j) {
        const float aj = arow[j];
        const f2p a2 = f2_pack(aj, aj);
        const ulonglong2 h0 = *reinterpret_cast<const ulonglong2*>(Hr + j * Rp + c0);
        const ulonglong2 h1 = *reinterpret_cast<const ulonglong2*>(Hr + j * Rp + c0 + 4);
        hi2[0] = f2_fma(a2, h0.x, hi2[0]);
        hi2[1] = f2_fma(a2, h0.y, hi2[1]);
        hi2[2] = f2_fma(a2, h1.x, hi2[2]);
        hi2[3] = f2_fma(a2, h1.y, hi2[3]);
      }
      hi2[0] = f2_sub(hi2[0], f2_pack(m0.x, m0.y));
      hi2[1] = f2_sub(hi2[1], f2_pack(m0.z, m0.w));
      hi2[2] = f2_sub(hi2[2], f2_pack(m1.x, m1.y));
      hi2[3] = f2_sub(hi2[3], f2_pack(m1.z, m1.w));
    }
    float hi[8], lo[8];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      hi[2 * k] = f2_x(hi2[k]);
      hi[2 * k + 1] = f2_y(hi2[k]);
      lo[2 * k] = f2_x(lo2[k]);
      lo[2 * k + 1] = f2_y(lo2[k]);
    }
    float g[8], gl[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      two_sum(hi[u], lo[u], g[u], gl[u]);  // g + gl = hi + lo exactly; g is the rounded value
      const int c = c0 + u;
      if (c < R) {
        const float s = sacd_step(arow[c], g[u], __ldg(invh + c));
        zsum += sacd_importance(g[u], s, __ldg(lh + c));
      } else {
        g[u] = gl[u] = 0.f;
      }
    }
    float4* g4 = reinterpret_cast<float4*>(G + row * Rp + c0);
    g4[0] = make_float4(g[0], g[1], g[2], g[3]);
    g4[1] = make_float4(g[4], g[5], g[6], g[7]);
    float4* gl4 = reinterpret_cast<float4*>(dp->Glo + row * Rp + c0);
    gl4[0] = make_float4(gl[0], gl[1], gl[2], gl[3]);
    gl4[1] = make_float4(gl[4], gl[5], gl[6], gl[7]);
  }
  const double bz = block_sum((double)zsum, red);
  if (threadIdx.x == 0) {
    dp->tipart[lb] = bz;
    __threadfence();
    const unsigned prev = atomicAdd(&dp->counters[0], 1u);
    amlast = (prev == (unsigned)dp->p1_blocks - 1u);
  }
  __syncthreads();
  if (amlast) {
    __threadfence();
    double s = 0.0;
    for (int i = threadIdx.x; i < dp->p1_blocks; i += blockDim.x) s += __ldcg(dp->tipart + i);
    const double ti = block_sum(s, red);
    if (threadIdx.x == 0) {
      double* stt = dp->state;
      const bool first = stt[ST_FIRST] != 0.0;
      const double branch = first ? 0.0 : (ti > stt[ST_TIPREV] ? 2.0 : 1.0);
      stt[ST_TI] = ti;
      stt[ST_BRANCH] = branch;
      stt[ST_TIPREV] = ti;
      stt[ST_FIRST] = 0.0;
      dp->counters[0] = 0u;
    }
  }
}

void launch_pass1(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total_blocks, size_t smem,
                  cudaStream_t st) {
  if (total_blocks <= 0) return;
  pass1_kernel<<<(unsigned)total_blocks, 256, smem, st>>>(d_descs, d_base, njobs);
}

// ------------------------------------------------------------------------------------------
// pass 2: phase A (element-parallel): z from the stored gradient, selection, z^{k-1} <- z.
// phase B (the lanes of a row that has a selected element): the selected columns in order,
// s = max(0, u - g/h) - u (Eq. 12-13), with the gradient fix-up described below.
__global__ void __launch_bounds__(256, 4) pass2_kernel(const StepDesc* __restrict__ descs,
                                                   const int64_t* __restrict__ base, int njobs) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  __shared__ long long cred[256];
  const int64_t gb = blockIdx.x;
  const int jb = njobs > 1 ? find_job(base, njobs, gb) : 0;
  const StepDesc* __restrict__ dp = descs + jb;
  const int64_t lb = gb - base[jb];
  const int R = dp->R, Rp = dp->Rp, ST = Rp + 1;
  const int64_t I = dp->I;
  float* __restrict__ A = dp->A;
  const float* __restrict__ G = dp->G;
  float* __restrict__ zprev = dp->zprev;
  const float* __restrict__ invh = dp->invh;
  const float* __restrict__ lh = dp->lh;
  uint8_t* __restrict__ mask = dp->mask;
  const int TPR = Rp >> 3, RB = 256 / TPR;
  const int64_t row0 = lb * RB;
  const int nrows = (int)min((int64_t)RB, I - row0);
  float* As = sm;
  float* Hs = sm + RB * ST;
  uint8_t* selb = reinterpret_cast<uint8_t*>(sm + RB * ST + (Rp <= 64 ? Rp * Rp : 0));
  float* ihs = reinterpret_cast<float*>(selb + RB * 32);    // Rp: 1/h_rr
  float* lhs = ihs + Rp;                                     // Rp: L/2
  const float* __restrict__ Hsrc = dp->Hf;
  stage_rows(A + row0 * Rp, As, nrows, Rp);
  if (Rp <= 64) {
    for (int e = threadIdx.x; e < Rp * Rp / 4; e += blockDim.x)
      reinterpret_cast<float4*>(Hs)[e] = __ldg(reinterpret_cast<const float4*>(Hsrc) + e);
  }
  for (int c = threadIdx.x; c < Rp; c += blockDim.x) {
    ihs[c] = __ldg(invh + c);
    lhs[c] = __ldg(lh + c);
  }
  const float* Hr = Rp <= 64 ? Hs : Hsrc;
  __syncthreads();
  const int branch = (int)dp->state[ST_BRANCH];
  const bool replay = dp->state[ST_REPLAY] != 0.0;
  const int rl = threadIdx.x / TPR, ch = threadIdx.x % TPR, c0 = ch * 8;
  long long count = 0;
  float gv[8];  // this lane's 8 gradient entries of its row, kept for phase B
#pragma unroll
  for (int u = 0; u < 8; ++u) gv[u] = 0.f;
  // ---- phase A
  if (rl < nrows) {
    const int64_t row = row0 + rl;
    unsigned bits = 0;
    if (c0 < R) {
      const float4* g4 = reinterpret_cast<const float4*>(G + row * Rp + c0);
      float4* z4 = reinterpret_cast<float4*>(zprev + row * Rp + c0);
      const float4 ga = g4[0], gb4 = g4[1], za = z4[0], zb = z4[1];
      gv[0] = ga.x; gv[1] = ga.y; gv[2] = ga.z; gv[3] = ga.w;
      gv[4] = gb4.x; gv[5] = gb4.y; gv[6] = gb4.z; gv[7] = gb4.w;
      const float zp[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
      float zn[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = c0 + u;
        zn[u] = zp[u];
        if (c < R) {
          const float a = As[rl * ST + c];
          const float s0 = sacd_step(a, gv[u], ihs[c]);
          const float z = sacd_importance(gv[u], s0, lhs[c]);
          bool sel;
          if (replay) sel = dp->replay[row * Rp + c] != 0;
          else if (branch == 0) sel = z > 0.f;                    // first visit: z > 0
          else if (branch == 2) sel = __fsub_rn(zp[u], z) > 0.f;  // Eq. 27: sp = z^{k-1} - z^k
          else sel = __fsub_rn(z, zp[u]) > 0.f;                   // Eq. 24: sp = z^k - z^{k-1}
          zn[u] = z;
          if (sel) bits |= 1u << u;
        }
      }
      z4[0] = make_float4(zn[0], zn[1], zn[2], zn[3]);
      z4[1] = make_float4(zn[4], zn[5], zn[6], zn[7]);
      if (mask) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (c0 + u < R) mask[row * Rp + c0 + u] = (bits >> u) & 1u;
      }
    }
    selb[rl * TPR + ch] = (uint8_t)bits;
    count = __popc(bits);
  }
  const long long tot = block_sum(count, cred);  // also orders phase A before phase B
  if (threadIdx.x == 0 && tot) atomicAdd(dp->nsel, (unsigned long long)tot);
  if (tot == 0) return;
  // ---- phase B. Each lane keeps its 8 columns of the row (the phase-A layout).
  __nv_bfloat16* __restrict__ A16 = dp->A16;
  const int64_t row = row0 + rl;
  float* arow = As + rl * ST;
  bool dirty = false;  // this lane changed one of its own columns
  if (dp->fixup != 0) {
    // Lemma 2: every selected element steps from the start-of-step gradient, independently.
    if (rl < nrows && c0 < R) {
      const unsigned bits = selb[rl * TPR + ch];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if ((bits >> u) & 1u) {
          const int c = c0 + u;
          const float a = arow[c];
          arow[c] = __fadd_rn(a, sacd_step(a, gv[u], ihs[c]));
          dirty = true;
        }
    }
  } else {
    // Column Gauss-Seidel: the selected columns of the row in order; the current gradient of
    // column r is
    //   g_r = (G + Glo)_r + sum over updated columns q < r of s_q H[q][r].
    // When column q moves by s_q, every lane adds s_q H[q][c] to a compensated (hi, lo)
    // accumulator of each of its own columns c (error-free products and sums), so g_r is the
    // exact start-of-step gradient plus an exactly accumulated correction, rounded once. The
    // warp walks the union of its rows' selected columns with uniform control flow (each row
    // applies only its own selections), so its rows never serialise on divergent paths.
    float glv[8];
    f2p ahi2[4], alo2[4];  // the pushed corrections of this lane's columns, as column pairs
    const float* __restrict__ Glo = dp->Glo;
    const uint8_t* rsel = selb + rl * TPR;
    const bool live = rl < nrows;
    if (live) {
      const float4* gl4 = reinterpret_cast<const float4*>(Glo + row * Rp + c0);
      const float4 la = __ldg(gl4), lb2 = __ldg(gl4 + 1);
      glv[0] = la.x; glv[1] = la.y; glv[2] = la.z; glv[3] = la.w;
      glv[4] = lb2.x; glv[5] = lb2.y; glv[6] = lb2.z; glv[7] = lb2.w;
    } else {
#pragma unroll
      for (int u = 0; u < 8; ++u) glv[u] = 0.f;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) ahi2[k] = alo2[k] = 0ull;
    // 8-column blocks in order; lane o of a row owns block o, and within a block the column's
    // register index u is static, so each lane forms its candidate gradient directly and the
    // owner's value reaches the row by one shuffle
    for (int o = 0; o < TPR; ++o) {
      const uint32_t rowbyte = live ? (uint32_t)rsel[o] : 0u;
      const uint32_t wb = __reduce_or_sync(0xffffffffu, rowbyte);
      if (wb == 0u) continue;
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        if (!((wb >> u) & 1u)) continue;
        const int r = 8 * o + u;
        const float ah = (u & 1) ? f2_y(ahi2[u >> 1]) : f2_x(ahi2[u >> 1]);
        const float al = (u & 1) ? f2_y(alo2[u >> 1]) : f2_x(alo2[u >> 1]);
        float s2, t2;
        two_sum(gv[u], ah, s2, t2);
        const float gown = __fadd_rn(s2, __fadd_rn(__fadd_rn(t2, al), glv[u]));
        const float g = __shfl_sync(0xffffffffu, gown, o, TPR);
        const float ar = arow[r];
        const float s = ((rowbyte >> u) & 1u) ? sacd_step(ar, g, ihs[r]) : 0.f;
        if (s != 0.f) {
          if (o == ch) {
            arow[r] = __fadd_rn(ar, s);
            dirty = true;
          }
          const f2p s2p = f2_pack(s, s), ns2p = f2_pack(-s, -s);
          const ulonglong2 hq0 = *reinterpret_cast<const ulonglong2*>(Hr + r * Rp + c0);
          const ulonglong2 hq1 = *reinterpret_cast<const ulonglong2*>(Hr + r * Rp + c0 + 4);
          dot2_acc2(s2p, ns2p, hq0.x, ahi2[0], alo2[0]);
          dot2_acc2(s2p, ns2p, hq0.y, ahi2[1], alo2[1]);
          dot2_acc2(s2p, ns2p, hq1.x, ahi2[2], alo2[2]);
          dot2_acc2(s2p, ns2p, hq1.y, ahi2[3], alo2[3]);
        }
      }
    }
  }
  if (dirty) {
    // this lane's 8 columns of the row
    float4* a4 = reinterpret_cast<float4*>(A + row * Rp + c0);
    a4[0] = make_float4(arow[c0], arow[c0 + 1], arow[c0 + 2], arow[c0 + 3]);
    a4[1] = make_float4(arow[c0 + 4], arow[c0 + 5], arow[c0 + 6], arow[c0 + 7]);
    if (A16) {
#pragma unroll
      for (int u = 0; u < 8; ++u) A16[row * Rp + c0 + u] = __float2bfloat16_rn(arow[c0 + u]);
    }
  }
}

void launch_pass2(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total_blocks, size_t smem,
                  cudaStream_t st) {
  if (total_blocks <= 0) return;
  pass2_kernel<<<(unsigned)total_blocks, 256, smem, st>>>(d_descs, d_base, njobs);
}

// ------------------------------------------------------------------------------------------
// Gram A^T A. Each product is split exactly (two_prod) and summed with two_sum into an FP32
// (hi, lo) pair per output entry ("Dot2", Ogita-Rump-Oishi 2005); every staged chunk of rows is
// flushed into an FP64 accumulator; each block writes its FP64 partial, and gram_reduce sums
// the partials in block order with a fixed-shape tree.
__host__ __device__ int gram_chunk_rows(int Rp) { return 4096 / Rp; }

template <int TS>
__device__ void gram_tile_pass(const StepDesc* __restrict__ dp, int64_t lb, int oi, int oj, int TD, float* As,
                               double* out) {
  const int Rp = dp->Rp;
  const int64_t I = dp->I;
  const int nb = dp->gram_blocks;
  const float* __restrict__ A = dp->A;
  const int CH = gram_chunk_rows(Rp);
  const int ti = threadIdx.x / TD, tj = threadIdx.x - (threadIdx.x / TD) * TD;
  const bool active = threadIdx.x < TD * TD;
  const int i0 = oi * TD * TS + ti * TS, j0 = oj * TD * TS + tj * TS;
  double accd[TS][TS];
#pragma unroll
  for (int x = 0; x < TS; ++x)
#pragma unroll
    for (int y = 0; y < TS; ++y) accd[x][y] = 0.0;
  for (int64_t chunk = lb; chunk * CH < I; chunk += nb) {
    const int64_t r0 = chunk * CH;
    const int nr = (int)min((int64_t)CH, I - r0);
    const float4* src = reinterpret_cast<const float4*>(A + r0 * Rp);
    float4* dst = reinterpret_cast<float4*>(As);
    for (int e = threadIdx.x; e < nr * Rp / 4; e += blockDim.x) dst[e] = src[e];
    __syncthreads();
    if (active) {
      if constexpr (TS >= 2) {
        // entries (x, y) and (x, y + 1) as packed pairs (j0 is even, so the pair loads align)
        f2p hi2[TS][TS / 2], lo2[TS][TS / 2];
#pragma unroll
        for (int x = 0; x < TS; ++x)
#pragma unroll
          for (int y = 0; y < TS / 2; ++y) hi2[x][y] = lo2[x][y] = 0ull;
        for (int r = 0; r < nr; ++r) {
          f2p aj2[TS / 2];
#pragma unroll
          for (int y = 0; y < TS / 2; ++y) aj2[y] = *reinterpret_cast<const f2p*>(As + r * Rp + j0 + 2 * y);
#pragma unroll
          for (int x = 0; x < TS; ++x) {
            const float ai = As[r * Rp + i0 + x];
            const f2p a2 = f2_pack(ai, ai), na2 = f2_pack(-ai, -ai);
#pragma unroll
            for (int y = 0; y < TS / 2; ++y) dot2_acc2(a2, na2, aj2[y], hi2[x][y], lo2[x][y]);
          }
        }
#pragma unroll
        for (int x = 0; x < TS; ++x)
#pragma unroll
          for (int y = 0; y < TS / 2; ++y) {
            accd[x][2 * y] += (double)f2_x(hi2[x][y]) + (double)f2_x(lo2[x][y]);
            accd[x][2 * y + 1] += (double)f2_y(hi2[x][y]) + (double)f2_y(lo2[x][y]);
          }
      } else {
        float hi[TS][TS], lo[TS][TS];
#pragma unroll
        for (int x = 0; x < TS; ++x)
#pragma unroll
          for (int y = 0; y < TS; ++y) hi[x][y] = lo[x][y] = 0.f;
        for (int r = 0; r < nr; ++r) {
          float ai[TS], aj[TS];
#pragma unroll
          for (int x = 0; x < TS; ++x) ai[x] = As[r * Rp + i0 + x];
#pragma unroll
          for (int y = 0; y < TS; ++y) aj[y] = As[r * Rp + j0 + y];
#pragma unroll
          for (int x = 0; x < TS; ++x)
#pragma unroll
            for (int y = 0; y < TS; ++y) dot2_acc(ai[x], aj[y], hi[x][y], lo[x][y]);
        }
#pragma unroll
        for (int x = 0; x < TS; ++x)
#pragma unroll
          for (int y = 0; y < TS; ++y) accd[x][y] += (double)hi[x][y] + (double)lo[x][y];
      }
    }
    __syncthreads();
  }
  if (active) {
#pragma unroll
    for (int x = 0; x < TS; ++x)
#pragma unroll
      for (int y = 0; y < TS; ++y) out[(int64_t)(i0 + x) * Rp + (j0 + y)] = accd[x][y];
  }
}

template <int TS>
__global__ void __launch_bounds__(256) gram_kernel(const StepDesc* __restrict__ descs,
                                                  const int64_t* __restrict__ base, int njobs) {
  __shared__ float4 As4[1024];  // 16 KB: gram_chunk_rows(Rp) rows of Rp floats
  float* As = reinterpret_cast<float*>(As4);
  const int64_t gb = blockIdx.x;
  const int jb = njobs > 1 ? find_job(base, njobs, gb) : 0;
  const StepDesc* __restrict__ dp = descs + jb;
  const int64_t lb = gb - base[jb];
  const int Rp = dp->Rp;
  const int TD = Rp >= 16 ? 16 : Rp;
  const int OB = Rp / (TD * TS);
  double* out = dp->gpart + lb * (int64_t)Rp * Rp;
  for (int oi = 0; oi < OB; ++oi)
    for (int oj = 0; oj < OB; ++oj) gram_tile_pass<TS>(dp, lb, oi, oj, TD, As, out);
}

// sum of the per-block partials: 32 entries per block, 8 partial lanes each, fixed tree
__global__ void __launch_bounds__(256) gram_reduce_kernel(const StepDesc* __restrict__ descs,
                                                         const int64_t* __restrict__ base, int njobs) {
  __shared__ double red[8][32];
  const int64_t gb = blockIdx.x;
  const int jb = njobs > 1 ? find_job(base, njobs, gb) : 0;
  const StepDesc* __restrict__ dp = descs + jb;
  const int Rp = dp->Rp;
  const int nb = dp->gram_blocks;
  const int64_t e = (gb - base[jb]) * 32 + (threadIdx.x & 31);
  const int p = threadIdx.x >> 5;
  double s = 0.0;
  if (e < (int64_t)Rp * Rp)
    for (int b = p; b < nb; b += 8) s += dp->gpart[(int64_t)b * Rp * Rp + e];
  red[p][threadIdx.x & 31] = s;
  __syncthreads();
  for (int w = 4; w >= 1; w >>= 1) {
    if (p < w) red[p][threadIdx.x & 31] += red[p + w][threadIdx.x & 31];
    __syncthreads();
  }
  if (p == 0 && e < (int64_t)Rp * Rp) dp->gram_out[e] = red[0][threadIdx.x & 31];
}

void launch_gram(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total_blocks, int Rp, bool tc,
                 cudaStream_t st) {
  if (total_blocks <= 0) return;
  if (tc) {
    launch_gram_tc(d_descs, d_base, njobs, total_blocks, Rp, st);
    return;
  }
  if (Rp <= 16)
    gram_kernel<1><<<(unsigned)total_blocks, 256, 0, st>>>(d_descs, d_base, njobs);
  else if (Rp == 32)
    gram_kernel<2><<<(unsigned)total_blocks, 256, 0, st>>>(d_descs, d_base, njobs);
  else
    gram_kernel<4><<<(unsigned)total_blocks, 256, 0, st>>>(d_descs, d_base, njobs);
}

int gram_reduce_blocks(int Rp) { return (Rp * Rp + 31) / 32; }

void launch_gram_reduce(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total_blocks,
                        cudaStream_t st) {
  if (total_blocks <= 0) return;
  gram_reduce_kernel<<<(unsigned)total_blocks, 256, 0, st>>>(d_descs, d_base, njobs);
}

// ------------------------------------------------------------------------------------------
// objective and fit
__global__ void __launch_bounds__(256) fit_kernel(const FitDesc* __restrict__ fds, const int64_t* __restrict__ base,
                                                 int njobs) {
  const int jb = njobs > 1 ? find_job(base, njobs, (int64_t)blockIdx.x) : 0;
  const FitDesc& f = fds[jb];
  const int64_t lb = (int64_t)blockIdx.x - base[jb];
  const int64_t nblk = base[jb + 1] - base[jb];
  __shared__ double red[256];
  __shared__ int amlast;
  // <X, model> = sum of A .* M over the last mode (Eq. 8 contracted with the MTTKRP), as 16-byte
  // vectors over all I x Rp entries (the padding columns of A are zero): exact products and
  // TwoSum on packed FP32 pairs, one conversion to FP64 per thread (this part runs FP64 at a
  // small fraction of its FP32 rate).
  const int64_t nv = f.I * f.Rp / 4;
  const float4* __restrict__ a4 = reinterpret_cast<const float4*>(f.A);
  const float4* __restrict__ m4 = reinterpret_cast<const float4*>(f.M);
  f2p hi0 = 0ull, lo0 = 0ull, hi1 = 0ull, lo1 = 0ull;
  for (int64_t v = lb * blockDim.x + threadIdx.x; v < nv; v += nblk * blockDim.x) {
    const float4 a = a4[v], m = m4[v];
    dot2_acc2(f2_pack(a.x, a.y), f2_pack(-a.x, -a.y), f2_pack(m.x, m.y), hi0, lo0);
    dot2_acc2(f2_pack(a.z, a.w), f2_pack(-a.z, -a.w), f2_pack(m.z, m.w), hi1, lo1);
  }
  const double part = ((double)f2_x(hi0) + (double)f2_y(hi0)) + ((double)f2_x(hi1) + (double)f2_y(hi1)) +
                      (((double)f2_x(lo0) + (double)f2_y(lo0)) + ((double)f2_x(lo1) + (double)f2_y(lo1)));
  // ||model||^2 = sum over (r, c) of prod_k (A_k^T A_k)_{rc}: this block's share of the entries
  double mn = 0.0;
  for (int64_t e = lb * blockDim.x + threadIdx.x; e < (int64_t)f.R * f.R; e += nblk * blockDim.x) {
    const int r = (int)(e / f.R), c = (int)(e - (e / f.R) * f.R);
    double p = 1.0;
    for (int k = 0; k < f.N; ++k) p *= f.gram[k][r * f.Rp + c];
    mn += p;
  }
  const double bs = block_sum(part, red);
  const double bm = block_sum(mn, red);
  if (threadIdx.x == 0) {
    f.part[2 * lb] = bs;
    f.part[2 * lb + 1] = bm;
    __threadfence();
    const unsigned prev = atomicAdd(f.counter, 1u);
    amlast = (prev == (unsigned)nblk - 1u);
  }
  __syncthreads();
  if (amlast) {
    __threadfence();
    double s = 0.0, sm = 0.0;
    for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) {
      s += __ldcg(f.part + 2 * b);
      sm += __ldcg(f.part + 2 * b + 1);
    }
    const double inner = block_sum(s, red);
    const double mnorm = block_sum(sm, red);
    if (threadIdx.x == 0) {
      f.out[0] = f.norm_x_sq - 2.0 * inner + mnorm;  // the fit is formed on the host
      f.out[1] = f.wait_err ? (double)*(volatile const unsigned int*)f.wait_err : 0.0;
      f.out[2] = inner;
      f.out[3] = mnorm;
      *f.counter = 0u;
    }
  }
}

// base[0..njobs]: prefix of the jobs' block counts (fit_blocks_for of their last mode)
void launch_fit(const FitDesc* d_fit, const int64_t* d_base, int njobs, int64_t total_blocks, cudaStream_t st) {
  fit_kernel<<<(unsigned)(total_blocks > 0 ? total_blocks : 1), 256, 0, st>>>(d_fit, d_base, njobs);
}

int64_t fit_blocks_for(int64_t I, int Rp) {
  const int64_t vecs = I * Rp / 4;
  return std::max<int64_t>(1, std::min<int64_t>((vecs + 1023) / 1024, 152 * 4));  // ~4 vectors per thread
}


// ------------------------------------------------------------------------------------------
__global__ void to_bf16_kernel(const float* __restrict__ src, __nv_bfloat16* __restrict__ dst, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    dst[i] = __float2bfloat16_rn(src[i]);
}
void launch_to_bf16(const float* src, void* dst, int64_t n, cudaStream_t st) {
  if (n <= 0) return;
  const int64_t blocks = min((n + 255) / 256, (int64_t)152 * 16);
  to_bf16_kernel<<<(unsigned)blocks, 256, 0, st>>>(src, reinterpret_cast<__nv_bfloat16*>(dst), n);
}

// ------------------------------------------------------------------------------------------
// evaluation: RMSE over test entries (Eq. 30) and pattern distinctiveness (Eq. pd)
struct EvalDesc {
  const int32_t* idx;  // N x n (row stride n)
  const float* vals;   // n
  int64_t n;
  const float* fac[SACD_MAXN];
  int32_t N, R, Rp;
  double* part;        // per-block partial sums of squared errors
  double* out;         // [0] RMSE
  unsigned int* counter;
};

// x_hat = sum_r prod_k a_k[i_k, r] with the products and the sum in FP64 (evaluation is not on
// the iteration path; FP64 keeps x - x_hat exact enough when the model fits the entry closely)
__global__ void __launch_bounds__(256) rmse_kernel(EvalDesc d) {
  __shared__ double red[256];
  __shared__ int amlast;
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double sq = 0.0;
  if (e < d.n) {
    int64_t rowoff[SACD_MAXN];
    for (int k = 0; k < d.N; ++k) rowoff[k] = (int64_t)d.idx[(int64_t)k * d.n + e] * d.Rp;
    double xh = 0.0;
    for (int r = 0; r < d.R; ++r) {
      double p = 1.0;
      for (int k = 0; k < d.N; ++k) p *= (double)d.fac[k][rowoff[k] + r];
      xh += p;
    }
    const double diff = (double)d.vals[e] - xh;
    sq = diff * diff;
  }
  const double bs = block_sum(sq, red);
  if (threadIdx.x == 0) {
    d.part[blockIdx.x] = bs;
    __threadfence();
    amlast = atomicAdd(d.counter, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (amlast) {
    __threadfence();
    double s = 0.0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) s += __ldcg(d.part + b);
    const double tot = block_sum(s, red);
    if (threadIdx.x == 0) {
      d.out[0] = d.n > 0 ? sqrt(tot / (double)d.n) : 0.0;
      *d.counter = 0u;
    }
  }
}

// mean over column pairs i < r of gram_ir / sqrt(gram_ii gram_rr), columns of zero norm left out
__global__ void __launch_bounds__(256) pd_kernel(const double* __restrict__ gram, int R, int Rp, double* out) {
  __shared__ double red[256];
  __shared__ double cnt[256];
  double s = 0.0, c = 0.0;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    const int i = e / R, r = e - (e / R) * R;
    if (i < r) {
      const double gi = gram[i * Rp + i], gr = gram[r * Rp + r];
      if (gi > 0.0 && gr > 0.0) {
        s += gram[i * Rp + r] / sqrt(gi * gr);
        c += 1.0;
      }
    }
  }
  const double ts = block_sum(s, red);
  const double tc = block_sum(c, cnt);
  if (threadIdx.x == 0) out[0] = tc > 0 ? ts / tc : 0.0;
}

void launch_rmse(const int32_t* idx, const float* vals, int64_t n, const float* const* fac, int N, int R, int Rp,
                 double* part, int64_t blocks, double* out, unsigned int* counter, cudaStream_t st) {
  EvalDesc d;
  d.idx = idx;
  d.vals = vals;
  d.n = n;
  for (int k = 0; k < SACD_MAXN; ++k) d.fac[k] = k < N ? fac[k] : nullptr;
  d.N = N;
  d.R = R;
  d.Rp = Rp;
  d.part = part;
  d.out = out;
  d.counter = counter;
  rmse_kernel<<<(unsigned)(blocks > 0 ? blocks : 1), 256, 0, st>>>(d);
}

void launch_pd(const double* gram, int R, int Rp, double* out, cudaStream_t st) {
  pd_kernel<<<1, 256, 0, st>>>(gram, R, Rp, out);
}

// U[0,1) initial factor values (h >> 40) * 2^-24, times 2^log2_scale (exact), where h is the
// splitmix64 finaliser of seed + (mode + 1) * 0xD1B54A32D192ED03 + (element + 1) * 0x9E3779B97F4A7C15
// (a counter-based generator: every element is drawn independently, so the draw is the same on any
// grid).
__global__ void init_factor_kernel(float* __restrict__ A, int64_t rows, int R, int Rp, unsigned long long seed,
                                   int mode, int log2_scale) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * R;
       e += (int64_t)gridDim.x * blockDim.x) {
    unsigned long long z = seed + (unsigned long long)(mode + 1) * 0xD1B54A32D192ED03ull +
                           (unsigned long long)(e + 1) * 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    const int64_t i = e / R;
    const int r = (int)(e - i * R);
    A[i * Rp + r] = ldexpf((float)(z >> 40), log2_scale - 24);
  }
}
void launch_init_factor(float* A, int64_t rows, int R, int Rp, unsigned long long seed, int mode, int log2_scale,
                        cudaStream_t st) {
  if (rows * R <= 0) return;
  const int64_t blocks = min((rows * R + 255) / 256, (int64_t)152 * 16);
  init_factor_kernel<<<(unsigned)blocks, 256, 0, st>>>(A, rows, R, Rp, seed, mode, log2_scale);
}

__global__ void check_factor_kernel(const float* __restrict__ A, int64_t rows, int R, int Rp,
                                    unsigned int* bad) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * R;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / R;
    const int r = (int)(e - i * R);
    const float v = A[i * Rp + r];
    if (!(v >= 0.f) || !isfinite(v)) atomicOr(bad, 1u);
  }
}
void launch_check_factor(const float* A, int64_t rows, int R, int Rp, unsigned int* bad, cudaStream_t st) {
  if (rows * R <= 0) return;
  const int64_t blocks = min((rows * R + 255) / 256, (int64_t)152 * 8);
  check_factor_kernel<<<(unsigned)blocks, 256, 0, st>>>(A, rows, R, Rp, bad);
}

void configure_kernels() {
  // once per process, also when contexts are created from several host threads
  static const bool done = [] {
    cudaFuncSetAttribute(pass1_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    cudaFuncSetAttribute(pass2_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 64 * 1024);
    return true;
  }();
  (void)done;
}

}  // namespace sacd
