// sacd_mttkrp_noalloc: the MTTKRP of one mode with no device allocation at all.
//
// Some callers cannot call cudaMalloc: code embedded in a host framework that owns the whole
// device memory pool and forbids allocations outside its plan (fixed-memory inference or
// serving processes), and latency-critical loops that cannot afford the device-wide
// synchronisation that cudaMalloc/cudaFree may imply. This entry point takes the caller's
// inputs and output as device pointers and keeps its only scratch (the per-tile partial rows of
// the MTTKRP and the kernel descriptor) in a file-scope static device array, which every GPU
// that loads the library holds until the process exits.
//
// The array is shared by every call on a device and keeps the previous call's contents; the
// kernels write every scratch word they read, so nothing has to be cleared between calls.
// Calls that overlap on the GPU (from several streams or threads) race on the array.
#include <cstddef>
#include <cstring>
#include <mutex>

#include "sacd.h"
#include "common.cuh"
#include "kernels.h"

namespace {

constexpr size_t kScratchBytes = (size_t)SACD_NOALLOC_SCRATCH_MIB << 20;
constexpr size_t kDescBytes = 1024;       // StepDesc + tile base, at the start of the array
constexpr size_t kCarryOffset = 4096;     // per-tile partial rows after it

static_assert(sizeof(StepDesc) + sizeof(int64_t) <= kDescBytes, "descriptor area too small");

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct Head {
  StepDesc desc;
  int64_t tile_base;
};

// Writes the call's descriptor into the static array. The descriptor travels as a kernel
// argument (copied when the launch is enqueued), so no host memory is read after this call
// returns, and no host-to-device copy of a pageable stack object is needed.
__global__ void put_head_kernel(Head h, Head* dst) { *dst = h; }

// Rows split across tiles, found from the tile borders themselves (no precomputed list):
// one block per border; the block of the first border a row crosses sums the row's partials
// (slot 1 of its first tile, slot 0 of the following ones) with a fixed-shape tree.
__global__ void __launch_bounds__(256) fixup_borders_kernel(const StepDesc* __restrict__ dp) {
  __shared__ float4 red[256];
  const int64_t t = (int64_t)blockIdx.x + 1;  // border between tiles t-1 and t
  const int64_t T = dp->tile;
  const int64_t nnz = dp->nnz;
  const int32_t* __restrict__ rowid = dp->rowid;
  const int64_t p = t * T;
  const int32_t row = rowid[p];
  if (rowid[p - 1] != row) return;
  if (t > 1 && rowid[(t - 1) * T - 1] == row) return;  // not the first border of this row
  int64_t lo = p, hi = nnz;                            // upper bound of `row`
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (rowid[mid] <= row) lo = mid + 1; else hi = mid;
  }
  const int64_t tf = t - 1, tl = (lo - 1) / T;
  const int nvec = dp->Rp >> 2;
  const float4* carry = reinterpret_cast<const float4*>(dp->carry);
  float4* Mrow = reinterpret_cast<float4*>(dp->M + (int64_t)row * dp->Rp);
  const int64_t P = tl - tf + 1;
  for (int c0 = 0; c0 < nvec; c0 += 256) {
    const int cw = min(256, nvec - c0);
    const int lanes = 256 / cw;
    const int c = c0 + (threadIdx.x % cw);
    const int pl = threadIdx.x / cw;
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t q = pl; q < P; q += lanes) {
      const float4 v = carry[((tf + q) * 2 + (q == 0 ? 1 : 0)) * nvec + c];
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
    if (pl == 0) Mrow[c] = red[threadIdx.x];
    __syncthreads();
  }
}

sacd_status bad(sacd_status s, const char* msg) {
  sacd::set_last_error(msg);
  return s;
}

std::mutex g_mu;
void* g_addr[256] = {};

}  // namespace

extern "C" {

sacd_status sacd_mttkrp_noalloc(int32_t nmodes, int32_t mode, const int64_t* dims, int64_t nnz,
                                const int32_t* rowid, const int32_t* cidx, const float* vals,
                                const float* const* factors, int32_t rank, int32_t ld, float* M, void* stream) {
  // ---- arguments (host-side checks only; nothing touches the GPU before they pass)
  if (nmodes < 2 || nmodes > SACD_MAXN) return bad(SACD_EINVAL, "nmodes must be in [2, 8]");
  if (mode < 0 || mode >= nmodes) return bad(SACD_EINVAL, "mode out of range");
  if (!dims || !factors || !M) return bad(SACD_EINVAL, "null dims, factors or M");
  for (int k = 0; k < nmodes; ++k)
    if (dims[k] < 1 || dims[k] > 2147483647LL) return bad(SACD_EINVAL, "dims[k] must be in [1, 2^31-1]");
  if (nnz < 0 || nnz > 2147483647LL) return bad(SACD_EINVAL, "nnz must be in [0, 2^31-1]");
  if (rank < 1 || rank > SACD_MAXR) return bad(SACD_EINVAL, "rank must be in [1, 256]");
  int rp = 8;
  while (rp < rank) rp <<= 1;
  if (ld != rp) return bad(SACD_EINVAL, "ld must be the padded rank: the next power of two >= max(8, rank)");
  if (nnz > 0 && (!rowid || !cidx || !vals)) return bad(SACD_EINVAL, "null rowid, cidx or vals");
  for (int k = 0; k < nmodes; ++k) {
    if (k == mode) continue;
    if (!factors[k] || (reinterpret_cast<uintptr_t>(factors[k]) & 15))
      return bad(SACD_EINVAL, "every other factor must be a non-null, 16-byte aligned device pointer");
  }
  if (reinterpret_cast<uintptr_t>(M) & 15) return bad(SACD_EINVAL, "M must be 16-byte aligned");
  const int rv = rp / 4;  // FP32 gathers
  const int groups = 32 / (rv < 32 ? rv : 32);
  int64_t sub = nnz / ((int64_t)groups * 152 * 64);
  sub = sub < 8 ? 8 : (sub > 128 ? 128 : sub);
  sub = (sub + 3) / 4 * 4;
  const int64_t tile = groups * sub;
  const int64_t ntiles = (nnz + tile - 1) / tile;
  if (kCarryOffset + (size_t)ntiles * 2 * rp * sizeof(float) > kScratchBytes)
    return bad(SACD_EINVAL, "problem too large for the static scratch: 2 * ceil(nnz / tile) * ld * 4 bytes "
                            "must fit in SACD_NOALLOC_SCRATCH_MIB MiB minus 4 KiB");

  // ---- per-device set-up: the device address of the static array
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= 256) return bad(SACD_ECUDA, "cudaGetDevice failed");
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess || !p) {
        cudaGetLastError();
        return bad(SACD_ECUDA, "cudaGetSymbolAddress of the static scratch failed");
      }
      g_addr[dev] = p;
    }
    base = reinterpret_cast<unsigned char*>(g_addr[dev]);
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int64_t I = dims[mode];
  if (nnz == 0) {
    e = cudaMemsetAsync(M, 0, (size_t)I * rp * sizeof(float), st);
    return e == cudaSuccess ? SACD_OK : bad(SACD_ECUDA, cudaGetErrorString(e));
  }

  // ---- descriptor into the static array, then the MTTKRP and the border fix-up
  Head h;
  memset(&h, 0, sizeof(h));
  StepDesc& d = h.desc;
  d.rowid = rowid;
  d.cidx = cidx;
  d.val = vals;
  d.nnz = nnz;
  d.cstride = nnz;
  d.nother = nmodes - 1;
  d.prec = 0;
  int o = 0;
  for (int k = 0; k < nmodes; ++k)
    if (k != mode) d.fac[o++] = factors[k];
  d.R = rank;
  d.Rp = rp;
  d.rv = rv;
  d.sub = (int)sub;
  d.tile = (int)tile;
  d.ntiles = ntiles;
  d.I = I;
  d.M = M;
  d.carry = reinterpret_cast<float*>(base + kCarryOffset);
  d.N = nmodes;
  d.n = mode;
  h.tile_base = 0;
  put_head_kernel<<<1, 1, 0, st>>>(h, reinterpret_cast<Head*>(base));
  const StepDesc* dd = reinterpret_cast<const StepDesc*>(base);
  const int64_t* tb = reinterpret_cast<const int64_t*>(base + offsetof(Head, tile_base));
  sacd::launch_mttkrp(dd, tb, 1, ntiles, 0, rv, nmodes - 1, st);
  if (ntiles > 1) fixup_borders_kernel<<<(unsigned)(ntiles - 1), 256, 0, st>>>(dd);
  e = cudaGetLastError();
  if (e != cudaSuccess) return bad(SACD_ECUDA, cudaGetErrorString(e));
  return SACD_OK;
}

}  // extern "C"
