// Fused select/update of a mode step (Algorithm 1, one factor block), after the MTTKRP:
//   phase 1  G = A H - M (Eq. 9, 14) and z (Eq. 20) of every element, ti = sum z (Eq. 25); the
//            last chunk of a job to finish reduces its ti and picks the selection branch (first
//            visit / Eq. 24 / Eq. 27);
//   barrier  every chunk of every job must have contributed to its ti before any selection;
//   phase 2  z again from the stored G (the same operations, so the same values), the selection,
//            the projected update of the selected elements in column order (Eq. 11-13) with the
//            gradient fix-up, z^{k-1} <- z, and the BF16 mirror.
// One persistent cooperative launch per mode step, for one job or a whole batch: blocks walk the
// (job, row chunk) work list twice (the same chunks in the same blocks both times). G is stored
// once (its rounding error, which the compensated GCD variant also keeps, is not needed here),
// and the split rows of M are written back in phase 1. The barrier's wait is bounded
// by a clock64() budget; a block that gives up sets the error word and every block then skips
// phase 2, and the host reports SACD_ETIMEOUT.
//
// A H is a small dense product per chunk: a thread owns 8 columns of RT rows and keeps their sums
// in registers (each H row read from shared memory serves RT rows). Every element's sum
// is the FP32 fused multiply-add chain over j = 0..R-1 followed by one rounded subtraction of M,
// the same operations as the two-pass kernels. The GCD variant (h_rr in place of L), which needs
// compensated gradients, keeps the two-pass kernels.
#include "common.cuh"
#include "kernels.h"
#include "rowpass.cuh"

namespace sacd {

// Rows per thread in the blocked A H product: 4 for large modes (each H row read from shared memory
// serves 4 rows), 1 for small ones (4 times the chunks, so more blocks share the work).
__host__ __device__ int selupd_chunk_rows(int Rp, int rt) { return (256 / (Rp / 8)) * rt; }

size_t selupd_smem_bytes(int Rp, int rt) {
  const int CR = selupd_chunk_rows(Rp, rt);
  size_t b = (size_t)CR * (Rp + 1) * sizeof(float);    // staged A rows
  if (Rp <= 64) b += (size_t)Rp * Rp * sizeof(float);  // H
  b += (size_t)256;                                    // selection bytes of one sub-pass
  b += (size_t)2 * Rp * sizeof(float);                 // 1/h_rr and L/2
  return (b + 15) / 16 * 16;
}

namespace {

struct ChunkSmem {
  float* As;
  float* Hs;
  uint8_t* selb;
  float* ihs;
  float* lhs;
};

template <int RT>
__device__ __forceinline__ ChunkSmem carve(float* sm, int Rp) {
  const int CR = selupd_chunk_rows(Rp, RT), ST = Rp + 1;
  ChunkSmem c;
  c.As = sm;
  c.Hs = sm + CR * ST;
  c.selb = reinterpret_cast<uint8_t*>(c.Hs + (Rp <= 64 ? Rp * Rp : 0));
  c.ihs = reinterpret_cast<float*>(c.selb + 256);
  c.lhs = c.ihs + Rp;
  return c;
}

// stage the chunk's A rows, H (Rp <= 64), 1/h_rr and L/2
__device__ __forceinline__ void stage_chunk(const StepDesc* __restrict__ dp, const ChunkSmem& s, int64_t row0,
                                            int nrows) {
  const int Rp = dp->Rp;
  stage_rows(dp->A + row0 * Rp, s.As, nrows, Rp);
  if (Rp <= 64) {
    for (int e = threadIdx.x; e < Rp * Rp / 4; e += blockDim.x)
      reinterpret_cast<float4*>(s.Hs)[e] = __ldg(reinterpret_cast<const float4*>(dp->Hf) + e);
  }
  for (int c = threadIdx.x; c < Rp; c += blockDim.x) {
    s.ihs[c] = __ldg(dp->invh + c);
    s.lhs[c] = __ldg(dp->lh + c);
  }
  __syncthreads();
}

// M of the thread's kSelRT rows (columns c0..c0+7); in phase 1 the rows split across MTTKRP tiles
// are finished from the partials and written back, in phase 2 they are read finished
template <int RT, bool FINISH>
__device__ __forceinline__ void load_m(const StepDesc* __restrict__ dp, int64_t row0, int nrows, int rg, int RG,
                                       int c0, float4 (&m)[RT][2]) {
  const int Rp = dp->Rp, R = dp->R;
  const int32_t* __restrict__ rowfix = dp->rowfix;
#pragma unroll
  for (int q = 0; q < RT; ++q) {
    m[q][0] = m[q][1] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int rl = rg + q * RG;
    if (rl >= nrows) continue;
    const int64_t row = row0 + rl;
    float4* m4 = reinterpret_cast<float4*>(dp->M + row * Rp + c0);
    const int32_t fx = (FINISH && rowfix) ? __ldg(rowfix + row) : -1;
    if (fx != -1) {
      split_row_sum(dp, fx, c0, m[q][0], m[q][1]);
      m4[0] = m[q][0];
      m4[1] = m[q][1];
    } else if (c0 < R) {
      m[q][0] = m4[0];
      m[q][1] = m4[1];
    }
  }
}

// G = A H - M for the thread's RT rows and 8 columns: for each element the FMA chain over
// j = 0..R-1 from zero, then one rounded subtraction of M (column pairs in packed registers). M is
// read after the products, so that it holds no registers during them.
template <int RT, bool FINISH>
__device__ __forceinline__ void grad_rows(const StepDesc* __restrict__ dp, const ChunkSmem& s, int64_t row0,
                                          int nrows, int rg, int RG, int c0, float (&g)[RT][8]) {
  const int R = dp->R, Rp = dp->Rp, ST = Rp + 1;
  const float* Hr = Rp <= 64 ? s.Hs : dp->Hf;
  f2p acc[RT][4];
#pragma unroll
  for (int q = 0; q < RT; ++q)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[q][k] = 0ull;
  const float* a0 = s.As + rg * ST;
  for (int j = 0; j < R; ++j) {
    const ulonglong2 h0 = *reinterpret_cast<const ulonglong2*>(Hr + j * Rp + c0);
    const ulonglong2 h1 = *reinterpret_cast<const ulonglong2*>(Hr + j * Rp + c0 + 4);
#pragma unroll
    for (int q = 0; q < RT; ++q) {
      const float aj = a0[q * RG * ST + j];
      const f2p a2 = f2_pack(aj, aj);
      acc[q][0] = f2_fma(a2, h0.x, acc[q][0]);
      acc[q][1] = f2_fma(a2, h0.y, acc[q][1]);
      acc[q][2] = f2_fma(a2, h1.x, acc[q][2]);
      acc[q][3] = f2_fma(a2, h1.y, acc[q][3]);
    }
  }
  float4 m[RT][2];
  load_m<RT, FINISH>(dp, row0, nrows, rg, RG, c0, m);
#pragma unroll
  for (int q = 0; q < RT; ++q) {
    const f2p d0 = f2_sub(acc[q][0], f2_pack(m[q][0].x, m[q][0].y));
    const f2p d1 = f2_sub(acc[q][1], f2_pack(m[q][0].z, m[q][0].w));
    const f2p d2 = f2_sub(acc[q][2], f2_pack(m[q][1].x, m[q][1].y));
    const f2p d3 = f2_sub(acc[q][3], f2_pack(m[q][1].z, m[q][1].w));
    g[q][0] = f2_x(d0); g[q][1] = f2_y(d0);
    g[q][2] = f2_x(d1); g[q][3] = f2_y(d1);
    g[q][4] = f2_x(d2); g[q][5] = f2_y(d2);
    g[q][6] = f2_x(d3); g[q][7] = f2_y(d3);
  }
}

// phase 1 of one chunk: the chunk's sum of z (FP64, fixed order: the block's threads in order)
template <int RT>
__device__ double chunk_phase1(const StepDesc* __restrict__ dp, int64_t lc, const ChunkSmem& s, double* red) {
  const int R = dp->R, Rp = dp->Rp, ST = Rp + 1;
  const int TPR = Rp >> 3, RG = 256 / TPR, CR = RG * RT;
  const int64_t row0 = lc * CR;
  const int nrows = (int)min((int64_t)CR, dp->I - row0);
  stage_chunk(dp, s, row0, nrows);
  const int rg = threadIdx.x / TPR, c0 = (threadIdx.x % TPR) * 8;
  float g[RT][8];
  grad_rows<RT, true>(dp, s, row0, nrows, rg, RG, c0, g);
  double zsum = 0.0;
#pragma unroll
  for (int q = 0; q < RT; ++q) {
    const int rl = rg + q * RG;
    if (rl >= nrows || c0 >= R) continue;
    float4* g4 = reinterpret_cast<float4*>(dp->G + (row0 + rl) * Rp + c0);  // for phase 2
    g4[0] = make_float4(g[q][0], g[q][1], g[q][2], g[q][3]);
    g4[1] = make_float4(g[q][4], g[q][5], g[q][6], g[q][7]);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int c = c0 + u;
      if (c < R) {
        const float st = sacd_step(s.As[rl * ST + c], g[q][u], s.ihs[c]);
        zsum += (double)sacd_importance(g[q][u], st, s.lhs[c]);
      }
    }
  }
  const double bz = block_sum(zsum, red);  // ends with a barrier: the shared tiles may be reused
  return bz;
}

// phase 2 of one chunk
template <int RT>
__device__ void chunk_phase2(const StepDesc* __restrict__ dp, int64_t lc, const ChunkSmem& s, int branch,
                             bool replay, long long* red) {
  const int R = dp->R, Rp = dp->Rp, ST = Rp + 1;
  const int TPR = Rp >> 3, RG = 256 / TPR, CR = RG * RT;
  const int64_t row0 = lc * CR;
  const int nrows = (int)min((int64_t)CR, dp->I - row0);
  stage_chunk(dp, s, row0, nrows);
  const int rg = threadIdx.x / TPR, ch = threadIdx.x % TPR, c0 = ch * 8;
  // the gradient that phase 1 stored (the warp walk below needs every lane's 8 values)
  float g[RT][8];
#pragma unroll
  for (int q = 0; q < RT; ++q) {
    const int rl = rg + q * RG;
#pragma unroll
    for (int u = 0; u < 8; ++u) g[q][u] = 0.f;
    if (rl < nrows && c0 < R) {
      const float4* g4 = reinterpret_cast<const float4*>(dp->G + (row0 + rl) * Rp + c0);
      const float4 ga = __ldcg(g4), gb = __ldcg(g4 + 1);
      g[q][0] = ga.x; g[q][1] = ga.y; g[q][2] = ga.z; g[q][3] = ga.w;
      g[q][4] = gb.x; g[q][5] = gb.y; g[q][6] = gb.z; g[q][7] = gb.w;
    }
  }
  float* __restrict__ A = dp->A;
  float* __restrict__ zprev = dp->zprev;
  uint8_t* __restrict__ mask = dp->mask;
  __nv_bfloat16* __restrict__ A16 = dp->A16;
  const float* Hr = Rp <= 64 ? s.Hs : dp->Hf;
  long long count = 0;
#pragma unroll
  for (int q = 0; q < RT; ++q) {
    const int rl = rg + q * RG;
    const bool live = rl < nrows;
    const int64_t row = row0 + rl;
    float* arow = s.As + rl * ST;
    const float* gv = g[q];
    // ---- selection of the row's 8 columns, z^{k-1} <- z
    unsigned bits = 0;
    if (live && c0 < R) {
      float4* z4 = reinterpret_cast<float4*>(zprev + row * Rp + c0);
      const float4 za = z4[0], zb = z4[1];
      const float zp[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
      float zn[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = c0 + u;
        zn[u] = zp[u];
        if (c < R) {
          const float st = sacd_step(arow[c], gv[u], s.ihs[c]);
          const float z = sacd_importance(gv[u], st, s.lhs[c]);
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
      if (mask) {  // debug recording of the selection
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (c0 + u < R) mask[row * Rp + c0 + u] = (bits >> u) & 1u;
      }
    }
    count += __popc(bits);
    s.selb[rg * TPR + ch] = (uint8_t)bits;
    __syncwarp();
    // ---- the update of the selected elements
    bool dirty = false;
    if (dp->fixup != 0) {
      // Lemma 2: every selected element steps from the start-of-step gradient, independently
      if (live && c0 < R) {
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if ((bits >> u) & 1u) {
            const int c = c0 + u;
            const float a = arow[c];
            arow[c] = __fadd_rn(a, sacd_step(a, gv[u], s.ihs[c]));
            dirty = true;
          }
      }
    } else {
      // Column Gauss-Seidel: the selected columns of the row in order; the current gradient of
      // column r is g_r plus the compensated sum of s_q H[q][r] over the updated columns q < r
      // (pushed into every lane's (hi, lo) accumulators when column q moves). The warp walks the
      // union of its rows' selected columns with uniform control flow.
      f2p ahi2[4], alo2[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) ahi2[k] = alo2[k] = 0ull;
      const uint8_t* rsel = s.selb + rg * TPR;
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
          const float gown = __fadd_rn(s2, __fadd_rn(t2, al));
          const float gr = __shfl_sync(0xffffffffu, gown, o, TPR);
          const float ar = arow[r];
          const float st = ((rowbyte >> u) & 1u) ? sacd_step(ar, gr, s.ihs[r]) : 0.f;
          if (st != 0.f) {
            if (o == ch) {
              arow[r] = __fadd_rn(ar, st);
              dirty = true;
            }
            const f2p s2p = f2_pack(st, st), ns2p = f2_pack(-st, -st);
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
      float4* a4 = reinterpret_cast<float4*>(A + row * Rp + c0);
      a4[0] = make_float4(arow[c0], arow[c0 + 1], arow[c0 + 2], arow[c0 + 3]);
      a4[1] = make_float4(arow[c0 + 4], arow[c0 + 5], arow[c0 + 6], arow[c0 + 7]);
      if (A16) {
#pragma unroll
        for (int u = 0; u < 8; ++u) A16[row * Rp + c0 + u] = __float2bfloat16_rn(arow[c0 + u]);
      }
    }
    __syncwarp();  // the row's selection bytes are rewritten by the next sub-pass
  }
  const long long tot = block_sum(count, red);  // ends with a barrier: the shared tiles may be reused
  if (threadIdx.x == 0 && tot) atomicAdd(dp->nsel, (unsigned long long)tot);
}

// Bounded grid barrier: returns false (in every thread of the block) if this block gave up
// waiting or another block has set the error word.
__device__ bool grid_barrier(GridBar* bar, unsigned nblocks, long long budget) {
  __shared__ int ok_s;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &bar->gen;
    volatile unsigned int* verr = &bar->err;
    const unsigned g0 = *vgen;
    __threadfence();
    const unsigned arrived = atomicAdd(&bar->count, 1u) + 1u;
    bool ok = true;
    if (arrived == nblocks) {
      atomicExch(&bar->count, 0u);
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g0) {
        if (*verr != 0u || clock64() - t0 > budget) {
          atomicOr(&bar->err, 1u);
          ok = false;
          break;
        }
        __nanosleep(128);
      }
    }
    __threadfence();
    ok_s = ok && (*verr == 0u);
  }
  __syncthreads();
  return ok_s != 0;
}

}  // namespace

template <int RT>
__global__ void __launch_bounds__(256, RT == 1 ? 4 : 2)
    selupd_kernel(const StepDesc* __restrict__ descs, const int64_t* __restrict__ base, int njobs, int64_t total,
                  GridBar* bar, long long budget) {
  extern __shared__ float4 smem4[];
  float* sm = reinterpret_cast<float*>(smem4);
  __shared__ double red[33];
  __shared__ long long cred[33];
  __shared__ int amlast;
  // ---- phase 1: z of every element, ti per job
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int j = njobs > 1 ? find_job(base, njobs, item) : 0;
    const StepDesc* __restrict__ dp = descs + j;
    const int64_t lc = item - base[j];
    const ChunkSmem s = carve<RT>(sm, dp->Rp);
    const double bz = chunk_phase1<RT>(dp, lc, s, red);
    if (threadIdx.x == 0) {
      dp->tipart[lc] = bz;
      __threadfence();
      const unsigned prev = atomicAdd(&dp->counters[0], 1u);
      amlast = (prev == (unsigned)dp->sel_chunks - 1u);
    }
    __syncthreads();
    if (amlast) {
      __threadfence();
      double sum = 0.0;
      for (int i = threadIdx.x; i < dp->sel_chunks; i += blockDim.x) sum += __ldcg(dp->tipart + i);
      const double ti = block_sum(sum, red);
      if (threadIdx.x == 0) {
        double* stt = dp->state;
        const bool first = stt[ST_FIRST] != 0.0;
        const double br = first ? 0.0 : (ti > stt[ST_TIPREV] ? 2.0 : 1.0);
        stt[ST_TI] = ti;
        stt[ST_BRANCH] = br;
        stt[ST_TIPREV] = ti;
        stt[ST_FIRST] = 0.0;
        dp->counters[0] = 0u;
        __threadfence();
      }
    }
    __syncthreads();
  }
  // ---- every job's ti and branch are final past this point
  if (!grid_barrier(bar, gridDim.x, budget)) return;
  // ---- phase 2: selection and update
  for (int64_t item = blockIdx.x; item < total; item += gridDim.x) {
    const int j = njobs > 1 ? find_job(base, njobs, item) : 0;
    const StepDesc* __restrict__ dp = descs + j;
    const int64_t lc = item - base[j];
    const ChunkSmem s = carve<RT>(sm, dp->Rp);
    const int branch = (int)__ldcg(dp->state + ST_BRANCH);
    const bool replay = __ldcg(dp->state + ST_REPLAY) != 0.0;
    chunk_phase2<RT>(dp, lc, s, branch, replay, cred);
  }
}

namespace {
int g_sm_count = 0;
// resident blocks per SM for each (rows per thread, dynamic shared memory) used so far
struct OccEntry {
  int rt;
  size_t smem;
  int blocks;
};
OccEntry g_occ[32] = {};
int g_nocc = 0;

template <int RT>
int blocks_per_sm(size_t smem) {
  for (int i = 0; i < g_nocc; ++i)
    if (g_occ[i].rt == RT && g_occ[i].smem == smem) return g_occ[i].blocks;
  int nb = 0;
  cudaFuncSetAttribute(selupd_kernel<RT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 96 * 1024);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, selupd_kernel<RT>, 256, smem);
  if (nb < 1) nb = 1;
  if (g_nocc < 32) g_occ[g_nocc++] = OccEntry{RT, smem, nb};
  return nb;
}

template <int RT>
cudaError_t launch_rt(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total_chunks, size_t smem,
                      GridBar* bar, long long budget, cudaStream_t st) {
  const int64_t cap = (int64_t)g_sm_count * blocks_per_sm<RT>(smem);
  const unsigned grid = (unsigned)std::min<int64_t>(total_chunks, cap);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, selupd_kernel<RT>, d_descs, d_base, njobs, total_chunks, bar, budget);
}
}  // namespace

int64_t selupd_chunks(int64_t I, int Rp, int rt) {
  return (I + selupd_chunk_rows(Rp, rt) - 1) / selupd_chunk_rows(Rp, rt);
}

// Rows per thread for a launch over `rows` factor rows of padded rank Rp: 4 when the 4-row chunks
// still fill the GPU twice over, else 1.
int selupd_choose_rt(int64_t rows, int Rp) {
  const int64_t chunks4 = (rows + selupd_chunk_rows(Rp, 4) - 1) / selupd_chunk_rows(Rp, 4);
  return chunks4 >= 2 * 152 * 2 ? 4 : 1;
}

// Cooperative launch (every block resident at once, which the grid barrier needs) of a grid no
// larger than what the GPU holds, capped by the work. `smem` must cover every job of the launch
// (the largest selupd_smem_bytes over their padded ranks; it is not monotonic in the rank) and
// the descriptors' chunk counts must be those of `rt` rows per thread.
cudaError_t launch_selupd(const StepDesc* d_descs, const int64_t* d_base, int njobs, int64_t total_chunks, int rt,
                          size_t smem, GridBar* bar, long long budget, cudaStream_t st) {
  if (total_chunks <= 0) return cudaSuccess;
  if (g_sm_count == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
  }
  return rt == 4 ? launch_rt<4>(d_descs, d_base, njobs, total_chunks, smem, bar, budget, st)
                 : launch_rt<1>(d_descs, d_base, njobs, total_chunks, smem, bar, budget, st);
}

}  // namespace sacd
