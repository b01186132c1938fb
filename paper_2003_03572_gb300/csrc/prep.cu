// Preprocessing of a sparse tensor on the device (once per context):
//  * index validation;
//  * stable LSD radix sort of (64-bit key, 32-bit position) pairs, 8 bits per pass, built from
//    per-block digit histograms, a global exclusive scan in digit-major order, and a stable
//    scatter whose in-block ranks come from warp match masks processed in element order;
//  * lexicographic order of the coordinates for each mode (keys packed from the least
//    significant mode upward into as many 64-bit words as needed, one stable sort per word);
//  * summation of repeated coordinates (FP32, in input order) and ||X||^2 (FP64);
//  * the list of rows that straddle MTTKRP tile borders.
#include "common.cuh"
#include "kernels.h"

namespace sacd {

// ------------------------------------------------------------------------------------------
// exclusive scan of uint32
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t warp_incl_scan(uint32_t v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t n = __shfl_up_sync(0xffffffffu, v, o);
    if (lane_id() >= o) v += n;
  }
  return v;
}

// exclusive scan of one value per thread over the block; returns the block total in *total
__device__ uint32_t block_excl_scan(uint32_t v, uint32_t* wsum, uint32_t* total) {
  const int lane = lane_id(), w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  const uint32_t inc = warp_incl_scan(v);
  if (lane == 31) wsum[w] = inc;
  __syncthreads();
  if (w == 0) {
    uint32_t s = lane < nw ? wsum[lane] : 0u;
    const uint32_t si = warp_incl_scan(s);
    if (lane < nw) wsum[lane] = si - s;
    if (lane == 31) *total = si;
  }
  __syncthreads();
  const uint32_t r = inc - v + wsum[w];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kScanThreads) scan_partials_kernel(const uint32_t* __restrict__ in, int64_t n,
                                                                    uint32_t* __restrict__ part) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t tot;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i)
    if (base + i < n) s += in[base + i];
  block_excl_scan(s, wsum, &tot);
  if (threadIdx.x == 0) part[blockIdx.x] = tot;
}

__global__ void __launch_bounds__(kScanThreads) scan_top_kernel(uint32_t* part, int64_t nb, uint32_t* d_total) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t tot;
  uint32_t carry = 0;
  for (int64_t c = 0; c < nb; c += kScanThreads) {
    const int64_t i = c + threadIdx.x;
    const uint32_t v = i < nb ? part[i] : 0u;
    const uint32_t ex = block_excl_scan(v, wsum, &tot);
    if (i < nb) part[i] = ex + carry;
    carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0 && d_total) *d_total = carry;
}

__global__ void __launch_bounds__(kScanThreads) scan_final_kernel(const uint32_t* in, int64_t n,
                                                                 const uint32_t* __restrict__ part,
                                                                 uint32_t* out) {
  __shared__ uint32_t wsum[32];
  __shared__ uint32_t tot;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0u;
    s += v[i];
  }
  uint32_t ex = block_excl_scan(s, wsum, &tot) + part[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = ex;
    ex += v[i];
  }
}

size_t scan_tmp_bytes(int64_t n) { return (size_t)((n + kScanTile - 1) / kScanTile + 1) * sizeof(uint32_t); }

void scan_u32(const uint32_t* in, uint32_t* out, int64_t n, uint32_t* d_total, void* tmp, cudaStream_t st) {
  const int64_t nb = (n + kScanTile - 1) / kScanTile;
  uint32_t* part = reinterpret_cast<uint32_t*>(tmp);
  if (n <= 0) {
    if (d_total) cudaMemsetAsync(d_total, 0, sizeof(uint32_t), st);
    return;
  }
  scan_partials_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, part);
  scan_top_kernel<<<1, kScanThreads, 0, st>>>(part, nb, d_total);
  scan_final_kernel<<<(unsigned)nb, kScanThreads, 0, st>>>(in, n, part, out);
}

// ------------------------------------------------------------------------------------------
// radix sort
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortRounds = 8;
constexpr int kSortTile = kSortThreads * kSortRounds;  // 2048 keys per block

__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint64_t* __restrict__ keys, int64_t n,
                                                                 int shift, int64_t nb, uint32_t* counts) {
  __shared__ uint32_t h[256];
  h[threadIdx.x] = 0;
  __syncthreads();
  const int64_t base = (int64_t)blockIdx.x * kSortTile;
  for (int i = threadIdx.x; i < kSortTile; i += kSortThreads) {
    const int64_t e = base + i;
    if (e < n) atomicAdd(&h[(unsigned)((keys[e] >> shift) & 255u)], 1u);
  }
  __syncthreads();
  counts[(int64_t)threadIdx.x * nb + blockIdx.x] = h[threadIdx.x];
}

// Stable scatter of one 8-bit digit. Each warp ranks its 256 keys per digit (match_any); the
// block then places its keys in shared memory in digit order (block-local start of each digit
// from a 256-entry scan, then the warps' shares, then the in-warp rank), and consecutive threads
// write consecutive keys of each digit run to their global positions, so the writes coalesce.
__global__ void __launch_bounds__(kSortThreads)
    radix_scatter_kernel(const uint64_t* __restrict__ keys, const uint32_t* __restrict__ vals, uint64_t* kout,
                         uint32_t* vout, int64_t n, int shift, int64_t nb, const uint32_t* __restrict__ offs) {
  __shared__ uint32_t wcnt[kSortWarps][256];
  __shared__ uint32_t wbase[kSortWarps][256];
  __shared__ uint32_t dstart[256];
  __shared__ uint64_t skey[kSortTile];
  __shared__ uint32_t sval[kSortTile];
  const int lane = lane_id(), w = threadIdx.x >> 5;
  for (int i = threadIdx.x; i < kSortWarps * 256; i += kSortThreads) (&wcnt[0][0])[i] = 0;
  __syncthreads();
  const int64_t blk0 = (int64_t)blockIdx.x * kSortTile;
  const int64_t base = blk0 + (int64_t)w * (32 * kSortRounds);
  const uint32_t lt_mask = (1u << lane) - 1u;
  uint64_t k[kSortRounds];
  uint32_t v[kSortRounds];
  uint32_t dg[kSortRounds];
  uint32_t rk[kSortRounds];
#pragma unroll
  for (int rd = 0; rd < kSortRounds; ++rd) {
    const int64_t e = base + rd * 32 + lane;
    const bool valid = e < n;
    k[rd] = valid ? keys[e] : 0ull;
    v[rd] = valid ? vals[e] : 0u;
    const uint32_t d = valid ? (uint32_t)((k[rd] >> shift) & 255u) : (256u + lane);
    dg[rd] = d;
    const uint32_t peers = __match_any_sync(0xffffffffu, d);
    const uint32_t before = valid ? wcnt[w][d] : 0u;
    rk[rd] = before + __popc(peers & lt_mask);
    __syncwarp();
    if (valid && lane == __ffs(peers) - 1) wcnt[w][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  {
    const int d = threadIdx.x;  // 256 threads, one digit each
    uint32_t run = 0;
#pragma unroll
    for (int ww = 0; ww < kSortWarps; ++ww) {
      wbase[ww][d] = run;
      run += wcnt[ww][d];
    }
    dstart[d] = run;  // the block's count of digit d, scanned below
  }
  __syncthreads();
  if (w == 0) {  // exclusive scan of the 256 counts: 8 consecutive digits per lane
    uint32_t c[8], sum = 0;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      c[i] = dstart[lane * 8 + i];
      sum += c[i];
    }
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    uint32_t ex = incl - sum;
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      dstart[lane * 8 + i] = ex;
      ex += c[i];
    }
  }
  __syncthreads();
#pragma unroll
  for (int rd = 0; rd < kSortRounds; ++rd) {
    const int64_t e = base + rd * 32 + lane;
    if (e < n) {
      const uint32_t d = dg[rd];
      const uint32_t lp = dstart[d] + wbase[w][d] + rk[rd];
      skey[lp] = k[rd];
      sval[lp] = v[rd];
    }
  }
  __syncthreads();
  const int cnt = (int)min((int64_t)kSortTile, n - blk0);
  for (int t = threadIdx.x; t < cnt; t += kSortThreads) {
    const uint64_t key = skey[t];
    const uint32_t d = (uint32_t)((key >> shift) & 255u);
    const uint32_t pos = offs[(int64_t)d * nb + blockIdx.x] + (uint32_t)t - dstart[d];
    kout[pos] = key;
    vout[pos] = sval[t];
  }
}

size_t radix_tmp_bytes(int64_t n) {
  const int64_t nb = (n + kSortTile - 1) / kSortTile;
  const int64_t nc = nb * 256;
  return (size_t)nc * sizeof(uint32_t) * 2 + scan_tmp_bytes(nc) + 256;
}

int radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n, int bits,
                     void* tmp, cudaStream_t st) {
  if (n <= 1 || bits <= 0) return 0;
  const int64_t nb = (n + kSortTile - 1) / kSortTile;
  const int64_t nc = nb * 256;
  uint32_t* counts = reinterpret_cast<uint32_t*>(tmp);
  uint32_t* offs = counts + nc;
  void* stmp = offs + nc;
  int cur = 0;
  uint64_t* kb[2] = {keys, keys_alt};
  uint32_t* vb[2] = {vals, vals_alt};
  for (int shift = 0; shift < bits; shift += 8) {
    radix_hist_kernel<<<(unsigned)nb, kSortThreads, 0, st>>>(kb[cur], n, shift, nb, counts);
    scan_u32(counts, offs, nc, nullptr, stmp, st);
    radix_scatter_kernel<<<(unsigned)nb, kSortThreads, 0, st>>>(kb[cur], vb[cur], kb[cur ^ 1], vb[cur ^ 1], n,
                                                                  shift, nb, offs);
    cur ^= 1;
  }
  return cur;
}

// ------------------------------------------------------------------------------------------
__global__ void iota_kernel(uint32_t* p, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    p[i] = (uint32_t)i;
}
static unsigned grid_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  if (b > 152 * 32) b = 152 * 32;
  return (unsigned)(b > 0 ? b : 1);
}
void launch_iota(uint32_t* p, int64_t n, cudaStream_t st) {
  if (n > 0) iota_kernel<<<grid_for(n), 256, 0, st>>>(p, n);
}

__global__ void build_keys_kernel(const int32_t* __restrict__ idx, int64_t stride,
                                  const uint32_t* __restrict__ perm, int64_t n, SortWord w, uint64_t* keys) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t p = perm[e];
    uint64_t k = 0;
    for (int f = 0; f < w.nfields; ++f)
      k |= (uint64_t)(uint32_t)idx[(int64_t)w.mode[f] * stride + p] << w.shift[f];
    keys[e] = k;
  }
}
void launch_build_keys(const int32_t* idx, int64_t stride, const uint32_t* perm, int64_t n, SortWord w,
                       uint64_t* keys, cudaStream_t st) {
  if (n > 0) build_keys_kernel<<<grid_for(n), 256, 0, st>>>(idx, stride, perm, n, w, keys);
}

__global__ void gather_i32_kernel(const int32_t* __restrict__ src, const uint32_t* __restrict__ perm,
                                  int32_t* __restrict__ dst, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[perm[e]];
}
__global__ void gather_f32_kernel(const float* __restrict__ src, const uint32_t* __restrict__ perm,
                                  float* __restrict__ dst, int64_t n) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[perm[e]];
}
void launch_gather_i32(const int32_t* src, const uint32_t* perm, int32_t* dst, int64_t n, cudaStream_t st) {
  if (n > 0) gather_i32_kernel<<<grid_for(n), 256, 0, st>>>(src, perm, dst, n);
}
void launch_gather_f32(const float* src, const uint32_t* perm, float* dst, int64_t n, cudaStream_t st) {
  if (n > 0) gather_f32_kernel<<<grid_for(n), 256, 0, st>>>(src, perm, dst, n);
}

__global__ void validate_idx_kernel(const int32_t* __restrict__ idx, int64_t stride, int N,
                                    const int64_t* __restrict__ dims, int64_t n, unsigned int* bad) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    for (int k = 0; k < N; ++k) {
      const int32_t v = idx[(int64_t)k * stride + e];
      if (v < 0 || (int64_t)v >= dims[k]) atomicOr(bad, 1u);
    }
  }
}
void launch_validate_idx(const int32_t* idx, int64_t stride, int N, const int64_t* d_dims, int64_t n,
                         unsigned int* bad, cudaStream_t st) {
  if (n > 0) validate_idx_kernel<<<grid_for(n), 256, 0, st>>>(idx, stride, N, d_dims, n, bad);
}

__global__ void dup_heads_kernel(const int32_t* __restrict__ sidx, int64_t stride, int N, int64_t n,
                                 uint32_t* heads) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (e == 0) ? 1u : 0u;
    if (e > 0)
      for (int k = 0; k < N; ++k)
        if (sidx[(int64_t)k * stride + e] != sidx[(int64_t)k * stride + e - 1]) h = 1u;
    heads[e] = h;
  }
}
void launch_dup_heads(const int32_t* sidx, int64_t stride, int N, int64_t n, uint32_t* heads, cudaStream_t st) {
  if (n > 0) dup_heads_kernel<<<grid_for(n), 256, 0, st>>>(sidx, stride, N, n, heads);
}

// every run head sums its run's values in order (FP32) and writes the distinct coordinate
__global__ void dup_compact_kernel(const int32_t* __restrict__ sidx, int64_t stride, int N,
                                   const float* __restrict__ svals, const uint32_t* __restrict__ heads,
                                   const uint32_t* __restrict__ pos, int64_t n, int32_t* uidx, int64_t ustride,
                                   float* uvals) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    if (!heads[e]) continue;
    const int64_t p = pos[e];
    float s = svals[e];
    for (int64_t f = e + 1; f < n && !heads[f]; ++f) s = __fadd_rn(s, svals[f]);
    uvals[p] = s;
    for (int k = 0; k < N; ++k) uidx[(int64_t)k * ustride + p] = sidx[(int64_t)k * stride + e];
  }
}
void launch_dup_compact(const int32_t* sidx, int64_t stride, int N, const float* svals, const uint32_t* heads,
                        const uint32_t* pos, int64_t n, int32_t* uidx, int64_t ustride, float* uvals,
                        cudaStream_t st) {
  if (n > 0)
    dup_compact_kernel<<<grid_for(n), 256, 0, st>>>(sidx, stride, N, svals, heads, pos, n, uidx, ustride, uvals);
}

// sum of squares in FP64 (squares of FP32 values are exact in FP64)
__global__ void __launch_bounds__(256) sumsq_kernel(const float* __restrict__ v, int64_t n, double* part,
                                                   double* out, unsigned int* counter) {
  __shared__ double red[256];
  __shared__ int amlast;
  double s = 0.0;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const double x = v[e];
    s += x * x;
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = 128; w >= 1; w >>= 1) {
    if ((int)threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[blockIdx.x] = red[0];
    __threadfence();
    amlast = atomicAdd(counter, 1u) == gridDim.x - 1u;
  }
  __syncthreads();
  if (amlast && threadIdx.x == 0) {
    __threadfence();
    double t = 0.0;
    for (unsigned b = 0; b < gridDim.x; ++b) t += __ldcg(part + b);
    *out = t;
    *counter = 0u;
  }
}
void launch_sumsq(const float* v, int64_t n, double* part, int64_t nparts, double* out, unsigned int* counter,
                  cudaStream_t st) {
  sumsq_kernel<<<(unsigned)nparts, 256, 0, st>>>(v, n, part, out, counter);
}

// A row crosses tile border t (between tiles t-1 and t) if rowid[t*T-1] == rowid[t*T]; the row is
// listed once, at the first border it crosses.
__global__ void split_flags_kernel(const int32_t* __restrict__ rowid, int64_t nnz, int64_t T, int64_t ntiles,
                                   uint32_t* flags) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
    uint32_t f = 0;
    if (t >= 1) {
      const int64_t p = t * T;
      const int32_t row = rowid[p];
      if (rowid[p - 1] == row) f = (t == 1 || rowid[(t - 1) * T - 1] != row) ? 1u : 0u;
    }
    flags[t] = f;
  }
}
void launch_split_flags(const int32_t* rowid, int64_t nnz, int64_t tile, int64_t ntiles, uint32_t* flags,
                        cudaStream_t st) {
  if (ntiles > 0) split_flags_kernel<<<grid_for(ntiles), 256, 0, st>>>(rowid, nnz, tile, ntiles, flags);
}

__global__ void split_emit_kernel(const int32_t* __restrict__ rowid, int64_t nnz, int64_t T, int64_t ntiles,
                                  const uint32_t* __restrict__ flags, const uint32_t* __restrict__ pos, int4* out) {
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ntiles; t += (int64_t)gridDim.x * blockDim.x) {
    if (!flags[t]) continue;
    const int64_t p = t * T;
    const int32_t row = rowid[p];
    // last nonzero of the row: upper bound of `row` in [p, nnz)
    int64_t lo = p, hi = nnz;
    while (lo < hi) {
      const int64_t mid = (lo + hi) >> 1;
      if (rowid[mid] <= row) lo = mid + 1; else hi = mid;
    }
    const int64_t last = lo - 1;
    out[pos[t]] = make_int4(row, (int)(t - 1), (int)(last / T), 0);
  }
}
void launch_split_emit(const int32_t* rowid, int64_t nnz, int64_t tile, int64_t ntiles, const uint32_t* flags,
                       const uint32_t* pos, int4* out, cudaStream_t st) {
  if (ntiles > 0) split_emit_kernel<<<grid_for(ntiles), 256, 0, st>>>(rowid, nnz, tile, ntiles, flags, pos, out);
}

}  // namespace sacd
