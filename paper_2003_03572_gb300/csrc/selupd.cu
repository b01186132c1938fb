// Fused select/update of a mode step (Algorithm 1, one factor block), after the MTTKRP:
//   phase 1  G = A H - M (Eq. 9, 14) and z (Eq. 20) of every element, ti = sum z (Eq. 25); the
//            last chunk of a job to finish reduces its ti and picks the selection branch (first
//            visit / Eq. 24 / Eq. 27);
//   barrier  every chunk of every job must have contributed to its ti before any selection;
//   phase 2  z again from the stored G (the same operations, so the same values), the selection,
//            the projected update of the selected elements in column order (Eq. 11-13) with the
//            gradient fix-up, z^{k-1} <- z, and the BF16 mirror.
// One persistent cooperative launch per mode step, for one job or a whole batch. Phase 1 takes
// (job, row chunk) items from a queue (an atomic counter), so that no block idles at the barrier
// while another still has two chunks to go; it stages each chunk's A and M rows in one pass,
// stores G (its rounding error, which the compensated GCD variant also keeps, is not needed
// here), and writes back the split rows of M. Phase 2 takes warp units (a chunk's rows of one warp
// slot) from a second queue and needs no shared memory or block barrier. Every result is
// independent of which block or warp did the work. The barrier's wait is bounded by a clock64()
// budget; a block that gives up sets the error word and every block then skips phase 2, and the
// host reports SACD_ETIMEOUT.
//
// A H is a small dense product per chunk: a thread owns 8 columns of RT rows and keeps their sums
// in registers (each H row read from shared memory serves RT rows). Every element's sum
// is the FP32 fused multiply-add chain over j = 0..R-1 followed by one rounded subtraction of M,
// the same operations as the two-pass kernels. H, 1/h_rr and L/2 are staged once per job in a
// block (they are constant over the mode step). The Gauss-Seidel corrections s_q H[q][r] are
// pushed into FP32 fused multiply-add sums, rounded like the gradient itself; the GCD variant
// (h_rr in place of L), whose larger steps need compensated gradients and corrections, keeps the
// two-pass kernels. Each thread sums its z in an FP32 TwoSum pair and hands one FP64 value to the
// block's fixed-order FP64 reduction (no FP64 arithmetic per element: FP64 is scarce here).
#include <mutex>

#include "common.cuh"
#include "kernels.h"
#include "rowpass.cuh"

namespace sacd {

// Rows per thread in the blocked A H product of phase 1: 4 for large modes (each H row read from
// shared memory serves 4 rows), 1 for small ones (4 times the chunks, so more blocks share the
// work).
__host__ __device__ int selupd_chunk_rows(int Rp, int rt) { return (256 / (Rp / 8)) * rt; }

namespace {

__host__ __device__ inline int a_tile_floats(int Rp, int rt) {  // padded A rows, rounded to 16 bytes
  return (selupd_chunk_rows(Rp, rt) * (Rp + 1) + 3) / 4 * 4;
}

}  // namespace

size_t selupd_smem_bytes(int Rp, int rt) {
  const int CR = selupd_chunk_rows(Rp, rt);
  size_t b = (size_t)a_tile_floats(Rp, rt) * sizeof(float);  // staged A rows (stride Rp + 1)
  b += (size_t)CR * Rp * sizeof(float);                      // staged M rows
  if (Rp <= 64) b += (size_t)Rp * Rp * sizeof(float);        // H
  b += (size_t)2 * Rp * sizeof(float);                       // 1/h_rr and L/2
  return (b + 15) / 16 * 16;
}

namespace {

struct ChunkSmem {
  float* As;
  float* Ms;
  float* Hs;
  float* ihs;
  float* lhs;
};

template <int RT>
__device__ __forceinline__ ChunkSmem carve(float* sm, int Rp) {
  const int CR = selupd_chunk_rows(Rp, RT);
  ChunkSmem c;
  c.As = sm;
  c.Ms = sm + a_tile_floats(Rp, RT);
  c.Hs = c.Ms + CR * Rp;
  c.ihs = c.Hs + (Rp <= 64 ? Rp * Rp : 0);
  c.lhs = c.ihs + Rp;
  return c;
}

// stage H (Rp <= 64), 1/h_rr and L/2 of the job, once per job in a block (the caller syncs)
__device__ __forceinline__ void stage_job(const StepDesc* __restrict__ dp, const ChunkSmem& s) {
  const int Rp = dp->Rp;
  if (Rp <= 64) {
    for (int e = threadIdx.x; e < Rp * Rp / 4; e += blockDim.x)
      reinterpret_cast<float4*>(s.Hs)[e] = __ldg(reinterpret_cast<const float4*>(dp->Hf) + e);
  }
  for (int c = threadIdx.x; c < Rp; c += blockDim.x) {
    s.ihs[c] = __ldg(dp->invh + c);
    s.lhs[c] = __ldg(dp->lh + c);
  }
}

// stage the chunk's A rows (stride Rp + 1) and M rows (and the job's constants when the block moves
// to another job). A full chunk is 2 RT float4 of each per thread; their loads are issued four
// iterations at a time before any is stored, so that the staging waits for two memory round trips
// rather than 2 RT.
template <int RT>
__device__ __forceinline__ void stage_chunk(const StepDesc* __restrict__ dp, const ChunkSmem& s, int64_t row0,
                                            int nrows, bool new_job) {
  const int Rp = dp->Rp, ST = Rp + 1;
  const float4* __restrict__ a4 = reinterpret_cast<const float4*>(dp->A + row0 * Rp);
  const float4* __restrict__ m4 = reinterpret_cast<const float4*>(dp->M + row0 * Rp);
  const int n4 = nrows * Rp / 4;
  constexpr int NI = 2 * RT, NB = NI < 4 ? NI : 4;
#pragma unroll
  for (int k0 = 0; k0 < NI; k0 += NB) {
    float4 va[NB], vm[NB];
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      const int e = threadIdx.x + (k0 + k) * 256;
      if (e < n4) {
        va[k] = a4[e];
        vm[k] = m4[e];
      }
    }
#pragma unroll
    for (int k = 0; k < NB; ++k) {
      const int e = threadIdx.x + (k0 + k) * 256;
      if (e < n4) {
        const int f = e * 4;
        const int r = f / Rp, c = f - r * Rp;
        float* p = s.As + r * ST + c;
        p[0] = va[k].x; p[1] = va[k].y; p[2] = va[k].z; p[3] = va[k].w;
        reinterpret_cast<float4*>(s.Ms)[e] = vm[k];
      }
    }
  }
  if (new_job) stage_job(dp, s);
  __syncthreads();
}

// G = A H - M for the thread's RT rows and 8 columns: for each element the FMA chain over
// j = 0..R-1 from zero, then one rounded subtraction of M (column pairs in packed registers). M
// comes from the staged rows, or, for a row split across MTTKRP tiles, from its partials (the row
// is then written back finished).
template <int RT>
__device__ __forceinline__ void grad_rows(const StepDesc* __restrict__ dp, const ChunkSmem& s, int64_t row0,
                                          int nrows, int rg, int RG, int c0, const int32_t (&fx)[RT],
                                          float (&g)[RT][8]) {
  const int R = dp->R, Rp = dp->Rp, ST = Rp + 1;
  f2p acc[RT][4];
#pragma unroll
  for (int q = 0; q < RT; ++q)
#pragma unroll
    for (int k = 0; k < 4; ++k) acc[q][k] = 0ull;
  const float* a0 = s.As + rg * ST;
  const float* Hr = Rp <= 64 ? s.Hs : dp->Hf;
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
#pragma unroll
  for (int q = 0; q < RT; ++q) {
    const int rl = rg + q * RG;
    float4 m0 = make_float4(0.f, 0.f, 0.f, 0.f), m1 = m0;
    if (rl < nrows) {
      if (fx[q] != -1) {
        split_row_sum(dp, fx[q], c0, m0, m1);
        float4* mg = reinterpret_cast<float4*>(dp->M + (row0 + rl) * Rp + c0);
        mg[0] = m0;
        mg[1] = m1;
      } else if (c0 < R) {
        const float4* ms = reinterpret_cast<const float4*>(s.Ms + rl * Rp + c0);
        m0 = ms[0];
        m1 = ms[1];
      }
    }
    const f2p d0 = f2_sub(acc[q][0], f2_pack(m0.x, m0.y));
    const f2p d1 = f2_sub(acc[q][1], f2_pack(m0.z, m0.w));
    const f2p d2 = f2_sub(acc[q][2], f2_pack(m1.x, m1.y));
    const f2p d3 = f2_sub(acc[q][3], f2_pack(m1.z, m1.w));
    g[q][0] = f2_x(d0); g[q][1] = f2_y(d0);
    g[q][2] = f2_x(d1); g[q][3] = f2_y(d1);
    g[q][4] = f2_x(d2); g[q][5] = f2_y(d2);
    g[q][6] = f2_x(d3); g[q][7] = f2_y(d3);
  }
}

// phase 1 of one chunk: the chunk's sum of z (FP64 of each thread's FP32 TwoSum pair, fixed-order
// block reduction). Thread 0 also takes the block's next work item and leaves it in *next, which
// the block reads after the closing barrier (and not before the staging barrier: until then the
// block may still be reading the current item from *next).
template <int RT>
__device__ double chunk_phase1(const StepDesc* __restrict__ dp, int64_t lc, const ChunkSmem& s, bool new_job,
                               double* red, unsigned* queue, long long* next) {
  const int R = dp->R, Rp = dp->Rp, ST = Rp + 1;
  const int TPR = Rp >> 3, RG = 256 / TPR, CR = RG * RT;
  const int64_t row0 = lc * CR;
  const int nrows = (int)min((int64_t)CR, dp->I - row0);
  const int rg = threadIdx.x / TPR, c0 = (threadIdx.x % TPR) * 8;
  int32_t fx[RT];  // split-row entries, loaded before the staging wait
#pragma unroll
  for (int q = 0; q < RT; ++q) {
    const int rl = rg + q * RG;
    fx[q] = (dp->rowfix && rl < nrows) ? __ldg(dp->rowfix + row0 + rl) : -1;
  }
  stage_chunk<RT>(dp, s, row0, nrows, new_job);
  // past the staging barrier every thread holds its item, so *next may be overwritten
  if (threadIdx.x == 0) *next = (long long)atomicAdd(queue, 1u);
  float g[RT][8];
  grad_rows<RT>(dp, s, row0, nrows, rg, RG, c0, fx, g);
  float zh = 0.f, zl = 0.f;  // the thread's z sum as an unevaluated FP32 pair
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
        float hs, ht;
        two_sum(zh, sacd_importance(g[q][u], st, s.lhs[c]), hs, ht);
        zh = hs;
        zl = __fadd_rn(zl, ht);
      }
    }
  }
  return block_sum((double)zh + (double)zl, red);  // ends with a barrier: the tiles may be reused
}

struct RowData {
  float a[8], g[8], z[8];
};

__device__ __forceinline__ void load_row(const StepDesc* __restrict__ dp, int64_t row, bool on, int c0,
                                         RowData& d) {
  if (on) {
    const int Rp = dp->Rp;
    const float4* a4 = reinterpret_cast<const float4*>(dp->A + row * Rp + c0);
    const float4* g4 = reinterpret_cast<const float4*>(dp->G + row * Rp + c0);
    const float4* z4 = reinterpret_cast<const float4*>(dp->zprev + row * Rp + c0);
    const float4 a0 = a4[0], a1 = a4[1], g0 = __ldcg(g4), g1 = __ldcg(g4 + 1), z0 = z4[0], z1 = z4[1];
    d.a[0] = a0.x; d.a[1] = a0.y; d.a[2] = a0.z; d.a[3] = a0.w; d.a[4] = a1.x; d.a[5] = a1.y; d.a[6] = a1.z; d.a[7] = a1.w;
    d.g[0] = g0.x; d.g[1] = g0.y; d.g[2] = g0.z; d.g[3] = g0.w; d.g[4] = g1.x; d.g[5] = g1.y; d.g[6] = g1.z; d.g[7] = g1.w;
    d.z[0] = z0.x; d.z[1] = z0.y; d.z[2] = z0.z; d.z[3] = z0.w; d.z[4] = z1.x; d.z[5] = z1.y; d.z[6] = z1.z; d.z[7] = z1.w;
  } else {
#pragma unroll
    for (int u = 0; u < 8; ++u) d.a[u] = d.g[u] = d.z[u] = 0.f;
  }
}

// phase 2 of one warp unit: the rows of chunk lc that warp slot `wslot` of a block would own (lane
// group of TPR lanes per row, RT rows per group). No shared memory and no block barrier: A, G and
// z^{k-1} come from global memory (the next row's are loaded while the current one is worked on),
// H, 1/h_rr and L/2 from the read-only cache, and the lanes of a row exchange what the walk needs
// with shuffles. Returns the number of selected elements of the unit (in every lane).
template <int RT>
__device__ long long unit_phase2(const StepDesc* __restrict__ dp, int64_t lc, int wslot, int branch, bool replay) {
  const int R = dp->R, Rp = dp->Rp;
  const bool lemma2 = dp->fixup != 0;
  const uint8_t* __restrict__ rep_mask = dp->replay;
  const int TPR = Rp >> 3, RG = 256 / TPR, CR = RG * RT;
  const int64_t row0 = lc * CR;
  const int nrows = (int)min((int64_t)CR, dp->I - row0);
  const int lane = threadIdx.x & 31;
  const int rg = (wslot * 32 + lane) / TPR, ch = lane % TPR, c0 = ch * 8;
  const bool colok = c0 < R;
  const float* __restrict__ H = dp->Hf;
  float ih[8], lh[8];
#pragma unroll
  for (int u = 0; u < 8; ++u) {
    ih[u] = __ldg(dp->invh + c0 + u);  // invh and lh hold Rp entries (zero past R)
    lh[u] = __ldg(dp->lh + c0 + u);
  }
  float* __restrict__ A = dp->A;
  float* __restrict__ zprev = dp->zprev;
  uint8_t* __restrict__ mask = dp->mask;
  __nv_bfloat16* __restrict__ A16 = dp->A16;
  long long count = 0;
  RowData cur, nxt;
  load_row(dp, row0 + rg, rg < nrows && colok, c0, cur);
#pragma unroll
  for (int q = 0; q < RT; ++q) {
    const int rl = rg + q * RG;
    const bool live = rl < nrows;
    const int64_t row = row0 + rl;
    if (q + 1 < RT) load_row(dp, row + RG, rl + RG < nrows && colok, c0, nxt);
    // ---- selection of the row's 8 columns, z^{k-1} <- z
    unsigned bits = 0;
    if (live && colok) {
      float zn[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) {
        const int c = c0 + u;
        zn[u] = cur.z[u];
        if (c < R) {
          const float st = sacd_step(cur.a[u], cur.g[u], ih[u]);
          const float z = sacd_importance(cur.g[u], st, lh[u]);
          bool sel;
          if (replay) sel = rep_mask[row * Rp + c] != 0;
          else if (branch == 0) sel = z > 0.f;                        // first visit: z > 0
          else if (branch == 2) sel = __fsub_rn(cur.z[u], z) > 0.f;   // Eq. 27: sp = z^{k-1} - z^k
          else sel = __fsub_rn(z, cur.z[u]) > 0.f;                    // Eq. 24: sp = z^k - z^{k-1}
          zn[u] = z;
          if (sel) bits |= 1u << u;
        }
      }
      float4* z4 = reinterpret_cast<float4*>(zprev + row * Rp + c0);
      z4[0] = make_float4(zn[0], zn[1], zn[2], zn[3]);
      z4[1] = make_float4(zn[4], zn[5], zn[6], zn[7]);
      if (mask) {  // debug recording of the selection
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (c0 + u < R) mask[row * Rp + c0 + u] = (bits >> u) & 1u;
      }
    }
    count += __popc(bits);
    // ---- the update of the selected elements
    bool dirty = false;
    if (lemma2) {
      // Lemma 2: every selected element steps from the start-of-step gradient, independently
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if ((bits >> u) & 1u) {
          cur.a[u] = __fadd_rn(cur.a[u], sacd_step(cur.a[u], cur.g[u], ih[u]));
          dirty = true;
        }
    } else {
      // Column Gauss-Seidel: the selected columns of the row in order; the current gradient of
      // column r is g_r plus the sum of s_q H[q][r] over the updated columns q < r (pushed into
      // every lane's FP32 sums when column q moves), rounded once more. The warp walks the union
      // of its rows' selected columns with uniform control flow; the lane group that owns column
      // r takes the step and hands it to the rest of the row by shuffle.
      f2p acc2[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) acc2[k] = 0ull;
      for (int o = 0; o < TPR; ++o) {
        const uint32_t rowbyte = __shfl_sync(0xffffffffu, bits, o, TPR);
        const uint32_t wb = __reduce_or_sync(0xffffffffu, rowbyte);
        if (wb == 0u) continue;
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          if (!((wb >> u) & 1u)) continue;
          const int r = 8 * o + u;
          const ulonglong2 hq0 = __ldg(reinterpret_cast<const ulonglong2*>(H + r * Rp + c0));
          const ulonglong2 hq1 = __ldg(reinterpret_cast<const ulonglong2*>(H + r * Rp + c0 + 4));
          const float ah = (u & 1) ? f2_y(acc2[u >> 1]) : f2_x(acc2[u >> 1]);
          // meaningful in the owning lane group (o == ch), whose value is broadcast
          const float own = ((rowbyte >> u) & 1u) ? sacd_step(cur.a[u], __fadd_rn(cur.g[u], ah), ih[u]) : 0.f;
          const float st = __shfl_sync(0xffffffffu, own, o, TPR);
          if (st != 0.f) {
            if (o == ch) {
              cur.a[u] = __fadd_rn(cur.a[u], st);
              dirty = true;
            }
            const f2p s2p = f2_pack(st, st);
            acc2[0] = f2_fma(s2p, hq0.x, acc2[0]);
            acc2[1] = f2_fma(s2p, hq0.y, acc2[1]);
            acc2[2] = f2_fma(s2p, hq1.x, acc2[2]);
            acc2[3] = f2_fma(s2p, hq1.y, acc2[3]);
          }
        }
      }
    }
    if (dirty) {
      float4* a4 = reinterpret_cast<float4*>(A + row * Rp + c0);
      a4[0] = make_float4(cur.a[0], cur.a[1], cur.a[2], cur.a[3]);
      a4[1] = make_float4(cur.a[4], cur.a[5], cur.a[6], cur.a[7]);
      if (A16) {
        uint32_t w[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const __nv_bfloat162 pr = __floats2bfloat162_rn(cur.a[2 * u], cur.a[2 * u + 1]);
          w[u] = *reinterpret_cast<const uint32_t*>(&pr);
        }
        *reinterpret_cast<uint4*>(A16 + row * Rp + c0) = make_uint4(w[0], w[1], w[2], w[3]);
      }
    }
    if (q + 1 < RT) cur = nxt;
  }
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) count += __shfl_xor_sync(0xffffffffu, count, o);
  return count;
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
  __shared__ int amlast;
  __shared__ long long next_item;
  // the phase-2 queue is untouched until the grid barrier; block 0 empties it now
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&bar->queue2, 0u);
  int staged = -1;  // job whose constants are in shared memory
  // ---- phase 1: z of every element, ti per job; chunks taken from a queue
  if (threadIdx.x == 0) next_item = (long long)atomicAdd(&bar->queue1, 1u);
  __syncthreads();
  for (int64_t item = next_item; item < total; item = next_item) {
    const int j = njobs > 1 ? find_job(base, njobs, item) : 0;
    const StepDesc* __restrict__ dp = descs + j;
    const int64_t lc = item - base[j];
    const ChunkSmem s = carve<RT>(sm, dp->Rp);
    const double bz = chunk_phase1<RT>(dp, lc, s, j != staged, red, &bar->queue1, &next_item);
    staged = j;
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
  const bool ok = grid_barrier(bar, gridDim.x, budget);
  if (blockIdx.x == 0 && threadIdx.x == 0) atomicExch(&bar->queue1, 0u);  // every block is past phase 1
  if (!ok) return;
  // ---- phase 2: selection and update; warp units (8 per chunk) taken from a second queue
  const unsigned units = (unsigned)(total * 8);
  const int lane = threadIdx.x & 31;
  while (true) {
    unsigned u = 0;
    if (lane == 0) u = atomicAdd(&bar->queue2, 1u);
    u = __shfl_sync(0xffffffffu, u, 0);
    if (u >= units) break;
    const int64_t chunk = u >> 3;
    const int j = njobs > 1 ? find_job(base, njobs, chunk) : 0;
    const StepDesc* __restrict__ dp = descs + j;
    const int branch = (int)__ldcg(dp->state + ST_BRANCH);
    const bool replay = __ldcg(dp->state + ST_REPLAY) != 0.0;
    const long long cnt = unit_phase2<RT>(dp, chunk - base[j], (int)(u & 7u), branch, replay);
    if (lane == 0 && cnt) atomicAdd(dp->nsel, (unsigned long long)cnt);
  }
}

namespace {
// Both caches below are filled on first use and guarded by g_occ_mu: contexts may be stepped from
// several host threads at once.
std::mutex g_occ_mu;
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
  std::lock_guard<std::mutex> lk(g_occ_mu);
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
                      GridBar* bar, long long budget, int sms, cudaStream_t st) {
  const int64_t cap = (int64_t)sms * blocks_per_sm<RT>(smem);
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
  int sms = 0;
  {
    std::lock_guard<std::mutex> lk(g_occ_mu);
    if (g_sm_count == 0) {
      int dev = 0;
      cudaGetDevice(&dev);
      cudaDeviceGetAttribute(&g_sm_count, cudaDevAttrMultiProcessorCount, dev);
    }
    sms = g_sm_count;
  }
  return rt == 4 ? launch_rt<4>(d_descs, d_base, njobs, total_chunks, smem, bar, budget, sms, st)
                 : launch_rt<1>(d_descs, d_base, njobs, total_chunks, smem, bar, budget, sms, st);
}

}  // namespace sacd
