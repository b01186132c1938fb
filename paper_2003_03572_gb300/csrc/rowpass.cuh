// Device helpers shared by the row passes of a mode step (update.cu, selupd.cu): fixed-shape
// block reductions, row staging into shared memory, compensated accumulation, and the finish of
// MTTKRP rows that were split across warp tiles.
#pragma once

#include "common.cuh"

namespace sacd {

// ------------------------------------------------------------------------------------------
// block reductions with a fixed shape (deterministic)
// (warp butterflies, then the warps' sums in warp order; `red` holds at least 33 entries)
template <typename T>
__device__ T block_sum(T v, T* red) {
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  if (w == 0) {
    T r = l < (int)(blockDim.x >> 5) ? red[l] : T(0);
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) r += __shfl_xor_sync(0xffffffffu, r, o);
    if (l == 0) red[32] = r;
  }
  __syncthreads();
  const T r = red[32];
  __syncthreads();
  return r;
}

// stage `nrows` rows of an I x Rp matrix into shared memory with row stride Rp+1
__device__ __forceinline__ void stage_rows(const float* __restrict__ src, float* dst, int nrows, int Rp) {
  const int ST = Rp + 1;
  const float4* s4 = reinterpret_cast<const float4*>(src);
  const int n4 = nrows * Rp / 4;
  for (int e = threadIdx.x; e < n4; e += blockDim.x) {
    const float4 v = s4[e];
    const int f = e * 4;
    const int r = f / Rp, c = f - r * Rp;
    float* p = dst + r * ST + c;
    p[0] = v.x; p[1] = v.y; p[2] = v.z; p[3] = v.w;
  }
}

// compensated (hi, lo) accumulation of a*b
__device__ __forceinline__ void dot2_acc(float a, float b, float& hi, float& lo) {
  float p, e, s, t;
  two_prod(a, b, p, e);
  two_sum(hi, p, s, t);
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(t, e));
}

// ------------------------------------------------------------------------------------------
// A row of M split across MTTKRP tiles, finished from the partials (columns c0 .. c0+7): a light
// row sums slot 1 of its first tile and slot 0 of the following tiles in tile order (the order of
// the separate light fix-up), a heavy row its chunk sums in chunk order.
__device__ __forceinline__ void split_row_sum(const StepDesc* __restrict__ dp, int32_t fx, int c0, float4& m0,
                                              float4& m1) {
  const int nvec = dp->Rp >> 2, v0 = c0 >> 2;
  const float4* __restrict__ src;
  int64_t first, count, stride;
  if (fx >= 0) {
    const int4 s = dp->split_light[fx];  // {row, first tile, last tile, 0}
    src = reinterpret_cast<const float4*>(dp->carry);
    m0 = src[((int64_t)s.y * 2 + 1) * nvec + v0];
    m1 = src[((int64_t)s.y * 2 + 1) * nvec + v0 + 1];
    first = (int64_t)s.y * 2 + 2;  // slot 0 of tile s.y + 1
    count = (int64_t)s.z - s.y;
    stride = 2 * (int64_t)nvec;
  } else {
    const int4 s = dp->split_heavy[-2 - fx];  // {row, first chunk, chunk count, 0}
    src = reinterpret_cast<const float4*>(dp->carry2);
    m0 = src[(int64_t)s.y * nvec + v0];
    m1 = src[(int64_t)s.y * nvec + v0 + 1];
    first = (int64_t)s.y + 1;
    count = (int64_t)s.z - 1;
    stride = nvec;
  }
  // four partials' loads in flight at a time, added in order
  int64_t k = 0;
  for (; k + 4 <= count; k += 4) {
    float4 a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int64_t o = first * nvec + (k + i) * stride;
      a[i] = src[o + v0];
      b[i] = src[o + v0 + 1];
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      m0.x += a[i].x; m0.y += a[i].y; m0.z += a[i].z; m0.w += a[i].w;
      m1.x += b[i].x; m1.y += b[i].y; m1.z += b[i].z; m1.w += b[i].w;
    }
  }
  for (; k < count; ++k) {
    const int64_t o = first * nvec + k * stride;
    const float4 a = src[o + v0], b = src[o + v0 + 1];
    m0.x += a.x; m0.y += a.y; m0.z += a.z; m0.w += a.w;
    m1.x += b.x; m1.y += b.y; m1.z += b.z; m1.w += b.w;
  }
}

}  // namespace sacd
