// Host side of libsacd: the C ABI declared in include/sacd.h.
//
// A context owns one sparse tensor (per-mode sorted slice structures), the FP32 master factors
// (plus BF16 mirrors in the BF16-gather mode), z^{k-1}, the FP64 Grams and the per-mode scalar
// state of Algorithm 1 (ti^{k-1}, first visit). Every mode step is a fixed sequence of kernels
// on the context's stream; sacd_iterate captures one outer iteration (modes 0..N-1) in a CUDA
// graph and replays it, so that no host round trip happens between mode steps.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <condition_variable>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "sacd.h"
#include "common.cuh"
#include "kernels.h"
#include "tune_table.h"

using namespace sacd;

namespace {

thread_local std::string g_err;

sacd_status fail(sacd_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

enum KClass { K_HL = 0, K_MTTKRP, K_FIXUP, K_PASS1, K_PASS2, K_GRAM, K_FIT, K_FIT_MTTKRP, K_SELUPD, K_NCLASS };
const char* kClassName[K_NCLASS] = {"hl", "mttkrp", "mttkrp_fixup", "pass1_grad_importance",
                                    "pass2_select_update", "gram", "fit", "fit_mttkrp",
                                    "select_update"};

struct ModeData {
  int64_t I = 0;
  // slice structure
  int32_t* rowid = nullptr;
  int32_t* cidx = nullptr;
  float* val = nullptr;
  int64_t ntiles = 0;
  int sub = 0, tile = 0;
  int4* split_light = nullptr;
  int64_t nlight = 0;
  int4* split_heavy = nullptr;
  int64_t nheavy = 0;
  int4* chunks = nullptr;
  int64_t nchunks = 0;
  int32_t* rowfix = nullptr;     // I: row -> split entry (see StepDesc::rowfix)
  int4* split_tmp = nullptr;     // create-time list of split rows (ntiles entries)
  uint32_t* split_pos = nullptr;
  uint32_t* split_tot = nullptr;
  // state
  float* A = nullptr;
  __nv_bfloat16* A16 = nullptr;
  float* zprev = nullptr;
  float* M = nullptr;
  double* gram = nullptr;
  int64_t p1_blocks = 0, p2_blocks = 0, gram_blocks = 0, sel_chunks = 0;
  int sel_rt = 1;        // rows per thread of the fused select/update kernel for this mode
  bool gram_tc = false;  // this mode's Gram runs on the tensor cores
};

struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> ev;  // pairs
  std::vector<int> cls;         // class of each used pair
  int used = 0;
  int64_t launches[K_NCLASS] = {0};
  double ms[K_NCLASS] = {0};
  int64_t dropped = 0;
};

}  // namespace

void sacd::set_last_error(const char* msg) { g_err = msg; }

struct sacd_ctx {
  int N = 0;
  int64_t dims[SACD_MAXN] = {0};
  int64_t nnz = 0;
  int64_t cstride = 0;  // row stride of the index arrays: nnz rounded up to a multiple of 4
  int R = 0, Rp = 0, rv = 0;
  int prec = 0, lnorm = 0, fixup = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  bool poisoned = false;
  bool debug = false;
  int last_mode = -1;
  bool mlast_valid = false;
  int replay_mode = -1;
  double norm_x_sq = 0.0;
  int64_t device_bytes = 0;
  std::vector<void*> allocs;
  ModeData m[SACD_MAXN];
  // shared scratch
  float* G = nullptr;
  float* Glo = nullptr;
  uint8_t* mask = nullptr;
  uint8_t* replay = nullptr;
  float* carry = nullptr;
  float* carry2 = nullptr;
  int64_t carry_cap = 0, carry2_cap = 0;  // tiles / chunks the two buffers can hold
  double* gpart = nullptr;
  double* H = nullptr;
  float* Hf = nullptr;
  float* invh = nullptr;
  float* lh = nullptr;
  double* tipart = nullptr;
  double* state = nullptr;
  unsigned int* counters = nullptr;
  GridBar* bar = nullptr;             // grid barrier of the fused select/update launches
  long long wait_budget = kWaitBudgetCycles;
  unsigned int* wait_host = nullptr;  // pinned read-back of the barrier's error word
  unsigned long long* nsel = nullptr;
  int64_t* zero64 = nullptr;
  StepDesc hdesc[SACD_MAXN + 1];  // [n] mode-n steps; [N] the objective's FP32-gather MTTKRP (BF16 mode)
  StepDesc* ddesc = nullptr;
  float* Mfit = nullptr;  // BF16 mode: MTTKRP of mode fit_mode from the FP32 master factors (objective)
  int fit_mode = 0;       // the mode whose M the objective contracts with its factor
  // BF16 mode with fit_mode 0 and a supported width: the objective's MTTKRP also forms mode 0's
  // BF16-gather MTTKRP of the next step in the same pass (launch_mttkrp_dual). The objective's
  // partials then go to buffers of their own, and mpre says that m[0].M and its tile partials in
  // `carry` are current (no factor has changed and no other MTTKRP has run since): the next step
  // of mode 0 skips its MTTKRP kernel.
  bool dual_fit = false;
  bool mpre = false;
  float* carryF = nullptr;
  float* carry2F = nullptr;
  FitDesc hfit;
  FitDesc* dfit = nullptr;
  double* fitpart = nullptr;
  double* fitout = nullptr;
  double* fit_host = nullptr;  // pinned, 4 doubles: the objective read back by sacd_fit
  int64_t* fitbase = nullptr;  // {0, fit_blocks}
  int64_t fit_blocks = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaGraph_t graph_pre = nullptr;  // the iteration with mode 0's MTTKRP kernel left out (mpre)
  cudaGraphExec_t gexec_pre = nullptr;
  // second stream and events for the graph's parallel branch (Gram and H of the next mode
  // run beside the next mode's MTTKRP)
  cudaStream_t side = nullptr;
  cudaEvent_t ev[3 * SACD_MAXN + 2] = {};
  Prof prof;
};

namespace {

sacd_status cuda_fail(sacd_ctx* c, cudaError_t e, const char* where) {
  if (c) c->poisoned = true;
  return fail(SACD_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(expr)                                              \
  do {                                                        \
    cudaError_t _e = (expr);                                  \
    if (_e != cudaSuccess) return cuda_fail(c, _e, #expr);    \
  } while (0)

// Device allocations come from the device's stream-ordered memory pool (cudaMallocAsync on the
// context's stream), so that contexts created and destroyed at a high rate (serving) reuse
// cached memory instead of paying for cudaMalloc/cudaFree each time.
template <typename T>
sacd_status dalloc(sacd_ctx* c, T** p, size_t count) {
  *p = nullptr;
  if (count == 0) count = 1;
  void* q = nullptr;
  const cudaError_t e = cudaMallocAsync(&q, count * sizeof(T), c->st);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(SACD_ENOMEM, "cudaMalloc of " + std::to_string(count * sizeof(T)) + " bytes failed");
  }
  c->allocs.push_back(q);
  c->device_bytes += (int64_t)(count * sizeof(T));
  *p = reinterpret_cast<T*>(q);
  return SACD_OK;
}

#define TRY(expr)                        \
  do {                                   \
    sacd_status _s = (expr);             \
    if (_s != SACD_OK) return _s;        \
  } while (0)

// temporaries that are freed (stream-ordered) at the end of sacd_create
struct TmpAllocs {
  cudaStream_t st;
  std::vector<void*> p;
  explicit TmpAllocs(cudaStream_t s) : st(s) {}
  ~TmpAllocs() {
    for (auto it = p.rbegin(); it != p.rend(); ++it) cudaFreeAsync(*it, st);  // last in, first out
  }
  template <typename T>
  sacd_status get(T** out, size_t count) {
    *out = nullptr;
    if (count == 0) count = 1;
    void* q = nullptr;
    if (cudaMallocAsync(&q, count * sizeof(T), st) != cudaSuccess) {
      cudaGetLastError();
      return fail(SACD_ENOMEM, "cudaMalloc of temporary " + std::to_string(count * sizeof(T)) + " bytes failed");
    }
    p.push_back(q);
    *out = reinterpret_cast<T*>(q);
    return SACD_OK;
  }
};

int bits_for(int64_t dim) {
  int b = 0;
  while (b < 63 && ((int64_t)1 << b) < dim) ++b;
  return b;  // dim <= 2^b, indices < 2^b
}

int next_pow2(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}


void prof_record(sacd_ctx* c, int cls, bool start) {
  Prof& p = c->prof;
  if (!p.on) return;
  if (start) {
    if (p.used * 2 + 2 > (int)p.ev.size()) {  // pool full: harvest
      cudaStreamSynchronize(c->st);
      for (int i = 0; i < p.used; ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]) == cudaSuccess) {
          p.ms[p.cls[i]] += ms;
          p.launches[p.cls[i]] += 1;
        } else {
          cudaGetLastError();
          p.dropped++;
        }
      }
      p.used = 0;
    }
    p.cls[p.used] = cls;
    cudaEventRecord(p.ev[2 * p.used], c->st);
  } else {
    cudaEventRecord(p.ev[2 * p.used + 1], c->st);
    p.used++;
  }
}

struct KScope {
  sacd_ctx* c;
  int cls;
  KScope(sacd_ctx* c_, int cls_) : c(c_), cls(cls_) { prof_record(c, cls, true); }
  ~KScope() { prof_record(c, cls, false); }
};

// MTTKRP of mode n from descriptor `dd` (gathers of precision `prec`, `rv` 16-byte vectors per
// row) into `Mout`, with the mode's tiling and split-row lists. With `fold`, pass 1 of the same
// mode step finishes the rows split across tiles (light rows and the chunk sums of heavy rows,
// StepDesc::rowfix) and writes them into M, so only the chunk level runs here; without it (M
// needed on its own, e.g. for the objective) every level runs.
void enqueue_mttkrp_desc(sacd_ctx* c, int n, const StepDesc* dd, int prec, int rv, float* Mout, bool fold,
                         int cls_main, int cls_fix, bool skip_main = false) {
  ModeData& md = c->m[n];
  if (c->nnz == 0) {
    cudaMemsetAsync(Mout, 0, (size_t)md.I * c->Rp * sizeof(float), c->st);
    return;
  }
  if (!skip_main) {  // skipped when the dual pass of the objective has already formed M and its partials
    KScope k(c, cls_main);
    launch_mttkrp(dd, c->zero64, 1, md.ntiles, prec, rv, c->N - 1, c->st);
  }
  if (md.nlight && !fold) {
    KScope k(c, cls_fix);
    launch_fixup_light(dd, c->zero64, 1, md.nlight, c->st);
  }
  if (md.nheavy) {
    KScope k(c, cls_fix);
    launch_fixup_chunks(dd, c->zero64, 1, md.nchunks, c->st);
    if (!fold) launch_fixup_heavy(dd, c->zero64, 1, md.nheavy, c->st);
  }
}

void enqueue_mttkrp(sacd_ctx* c, int n, bool fold, bool skip_main = false) {
  enqueue_mttkrp_desc(c, n, c->ddesc + n, c->prec, c->rv, c->m[n].M, fold, K_MTTKRP, K_FIXUP, skip_main);
}

// The M that the objective contracts with factor fit_mode (<X, model> = sum of A_n .* M_n for any
// mode n). FP32 mode: the last mode's MTTKRP itself (recomputed only if a factor changed since the
// last mode step). BF16-gather mode: an MTTKRP from FP32 gathers of the FP32 master factors (the
// factors the caller gets back), into Mfit, every time: the BF16-gathered M of the mode steps is
// not the model of those factors. It runs on the longest mode, whose other factors are the
// smallest (the most gathered rows served from L1/L2). With dual_fit the same pass also forms mode
// 0's BF16-gather MTTKRP of the next step (mpre), for a context's own objective and in a batch alike,
// so that the objective's value does not depend on the path.
void enqueue_fit_mttkrp(sacd_ctx* c) {
  if (c->prec == SACD_BF16_GATHER) {
    const int L = c->fit_mode;
    if (c->dual_fit && c->nnz > 0) {
      {
        KScope k(c, K_FIT_MTTKRP);
        launch_mttkrp_dual(c->ddesc + L, c->ddesc + c->N, c->m[L].ntiles, c->rv, c->N - 1, c->st);
      }
      // the objective's split rows from its own partials; mode 0's stay in `carry` for its step
      enqueue_mttkrp_desc(c, L, c->ddesc + c->N, SACD_FP32, c->Rp / 4, c->Mfit, false, K_FIT_MTTKRP, K_FIT_MTTKRP,
                          true);
      c->mpre = true;
      return;
    }
    enqueue_mttkrp_desc(c, L, c->ddesc + c->N, SACD_FP32, c->Rp / 4, c->Mfit, false, K_FIT_MTTKRP,
                        K_FIT_MTTKRP);
  } else if (!c->mlast_valid) {
    enqueue_mttkrp(c, c->N - 1, false);
    c->mlast_valid = true;
  }
}

void enqueue_gram(sacd_ctx* c, int n) {
  KScope k(c, K_GRAM);
  launch_gram(c->ddesc + n, c->zero64, 1, c->m[n].gram_blocks, c->Rp, c->m[n].gram_tc, c->st);
  launch_gram_reduce(c->ddesc + n, c->zero64, 1, gram_reduce_blocks(c->Rp), c->st);
}

// Gradient, importance, ti, selection and update of mode n: the fused cooperative kernel, or the
// two row passes for the GCD variant (its compensated gradient is stored between them).
void enqueue_select_update(sacd_ctx* c, int n, cudaStream_t st) {
  ModeData& md = c->m[n];
  StepDesc* dd = c->ddesc + n;
  if (c->lnorm != SACD_LNORM_GCD) {
    KScope k(c, K_SELUPD);
    launch_selupd(dd, c->zero64, 1, md.sel_chunks, md.sel_rt, selupd_smem_bytes(c->Rp, md.sel_rt), c->bar,
                  c->wait_budget, st);
    return;
  }
  {
    KScope k(c, K_PASS1);
    launch_pass1(dd, c->zero64, 1, md.p1_blocks, pass_smem_bytes(c->Rp), st);
  }
  {
    KScope k(c, K_PASS2);
    launch_pass2(dd, c->zero64, 1, md.p2_blocks, pass_smem_bytes(c->Rp), st);
  }
}

void enqueue_step(sacd_ctx* c, int n) {
  StepDesc* dd = c->ddesc + n;
  const bool pre = c->mpre && n == c->fit_mode;  // M and its partials formed by the objective's pass
  c->mpre = false;                               // any step changes a factor
  {
    KScope k(c, K_HL);
    launch_hl(dd, 1, c->st);
  }
  enqueue_mttkrp(c, n, true, pre);
  enqueue_select_update(c, n, c->st);
  enqueue_gram(c, n);
}

// One outer iteration as a DAG, captured into the CUDA graph. Main stream: MTTKRP(n) ->
// pass1(n) -> pass2(n) -> MTTKRP(n+1) ...; side stream: Gram(n) -> H/L(n+1), which only needs
// the updated factor n and the Grams, so it overlaps MTTKRP(n+1). Same kernels and inputs as the
// sequential order, so the results are identical. With `pre0`, mode 0's MTTKRP kernel is left out
// (the objective's dual pass has formed it: mpre).
void enqueue_iteration_dag(sacd_ctx* c, bool pre0 = false) {
  cudaEvent_t* ev = c->ev;  // [0] fork, [1..N] H ready, [N+1..2N] pass2 done, [2N+1] join
  const int N = c->N;
  cudaEventRecord(ev[0], c->st);
  cudaStreamWaitEvent(c->side, ev[0], 0);
  launch_hl(c->ddesc + 0, 1, c->side);
  cudaEventRecord(ev[1], c->side);
  for (int n = 0; n < N; ++n) {
    ModeData& md = c->m[n];
    StepDesc* dd = c->ddesc + n;
    enqueue_mttkrp(c, n, true, pre0 && n == 0);
    cudaStreamWaitEvent(c->st, ev[1 + n], 0);
    enqueue_select_update(c, n, c->st);
    cudaEventRecord(ev[N + 1 + n], c->st);
    cudaStreamWaitEvent(c->side, ev[N + 1 + n], 0);
    launch_gram(dd, c->zero64, 1, md.gram_blocks, c->Rp, md.gram_tc, c->side);
    launch_gram_reduce(dd, c->zero64, 1, gram_reduce_blocks(c->Rp), c->side);
    if (n + 1 < N) {
      launch_hl(c->ddesc + n + 1, 1, c->side);
      cudaEventRecord(ev[2 + n], c->side);
    }
  }
  cudaEventRecord(ev[2 * N + 1], c->side);
  cudaStreamWaitEvent(c->st, ev[2 * N + 1], 0);
}

void invalidate_graph(sacd_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->gexec_pre) cudaGraphExecDestroy(c->gexec_pre);
  if (c->graph_pre) cudaGraphDestroy(c->graph_pre);
  c->gexec = nullptr;
  c->graph = nullptr;
  c->gexec_pre = nullptr;
  c->graph_pre = nullptr;
  c->mpre = false;  // descriptors or tiles may have changed
}

// BF16 mode: the objective's MTTKRP of mode fit_mode gathers FP32 rows of the master factors. It
// keeps the mode's tiles (same nonzeros per warp tile, so the same split-row lists and partial
// buffers): the lane groups are half as many (FP32 rows are twice as wide), each with twice the
// nonzeros.
void fill_fit_desc(sacd_ctx* c) {
  if (c->prec != SACD_BF16_GATHER) return;
  const int L = c->fit_mode;
  StepDesc d = c->hdesc[L];
  d.prec = SACD_FP32;
  d.rv = c->Rp / 4;
  int o = 0;
  for (int k = 0; k < c->N; ++k)
    if (k != L) d.fac[o++] = c->m[k].A;
  const int groups32 = 32 / std::min(d.rv, 32);
  d.sub = d.tile / groups32;
  d.M = c->Mfit;
  d.mask = nullptr;
  if (c->dual_fit) {  // the objective's partials apart from the mode's (which the dual pass keeps)
    d.carry = c->carryF;
    d.carry2 = c->carry2F;
  }
  c->hdesc[c->N] = d;
}

sacd_status upload_descs(sacd_ctx* c) {
  for (int n = 0; n < c->N; ++n) c->hdesc[n].mask = c->debug ? c->mask : nullptr;
  fill_fit_desc(c);
  const int nd = c->N + (c->prec == SACD_BF16_GATHER ? 1 : 0);
  CK(cudaMemcpyAsync(c->ddesc, c->hdesc, sizeof(StepDesc) * nd, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  invalidate_graph(c);
  return SACD_OK;
}

// fit = 1 - sqrt(max(f, 0)) / ||X|| (0 for an all-zero tensor)
double fit_from_objective(double objective, double norm_x_sq) {
  return norm_x_sq > 0 ? 1.0 - std::sqrt(std::max(objective, 0.0)) / std::sqrt(norm_x_sq) : 0.0;
}

// The error word of the fused select/update launches (a bounded grid-barrier wait gave up): read
// at the calls that wait for the stream anyway. A step that gave up left its factor half updated,
// so the context is poisoned.
sacd_status check_wait(sacd_ctx* c) {
  CK(cudaMemcpyAsync(c->wait_host, &c->bar->err, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (*c->wait_host) {
    c->poisoned = true;
    return fail(SACD_ETIMEOUT, "a bounded wait of the select/update kernel gave up (grid barrier)");
  }
  return SACD_OK;
}

sacd_status check_ctx(sacd_ctx* c) {
  if (!c) return fail(SACD_EINVAL, "null context");
  if (c->poisoned) return fail(SACD_ESTATE, "context is poisoned by an earlier CUDA error");
  return SACD_OK;
}

struct SortBufs {
  uint64_t *k0 = nullptr, *k1 = nullptr;
  uint32_t *p0 = nullptr, *p1 = nullptr;
  char* tmp = nullptr;
  sacd_status alloc(TmpAllocs& T, int64_t n) {
    TRY(T.get(&k0, n));
    TRY(T.get(&k1, n));
    TRY(T.get(&p0, n));
    TRY(T.get(&p1, n));
    TRY(T.get(&tmp, radix_tmp_bytes(n)));
    return SACD_OK;
  }
};

// Sort permutation of n coordinates (SoA idx with row stride `stride`) in the lexicographic
// order of the modes listed in `order` (most significant first).
sacd_status sort_order(sacd_ctx* c, SortBufs& B, const int32_t* idx, int64_t stride, int64_t n,
                       const std::vector<int>& order, uint32_t** perm_out) {
  uint64_t* k0 = B.k0;
  uint64_t* k1 = B.k1;
  uint32_t* p0 = B.p0;
  uint32_t* p1 = B.p1;
  void* tmp = B.tmp;
  launch_iota(p0, n, c->st);
  // pack words from the least significant mode upward
  std::vector<SortWord> words;
  SortWord cur{};
  int cur_bits = 0;
  for (int i = (int)order.size() - 1; i >= 0; --i) {
    const int md = order[i];
    const int b = bits_for(c->dims[md]);
    if (b == 0) continue;
    if (cur_bits + b > 64) {
      words.push_back(cur);
      cur = SortWord{};
      cur_bits = 0;
    }
    cur.mode[cur.nfields] = md;
    cur.shift[cur.nfields] = cur_bits;
    cur.nfields++;
    cur_bits += b;
  }
  if (cur.nfields) words.push_back(cur);
  uint32_t* perm = p0;
  uint32_t* alt = p1;
  for (const SortWord& w : words) {
    int wbits = 0;
    for (int f = 0; f < w.nfields; ++f) wbits = std::max(wbits, w.shift[f] + bits_for(c->dims[w.mode[f]]));
    launch_build_keys(idx, stride, perm, n, w, k0, c->st);
    const int which = radix_sort_pairs(k0, perm, k1, alt, n, wbits, tmp, c->st);
    if (which == 1) std::swap(perm, alt);
  }
  CK(cudaGetLastError());
  *perm_out = perm;
  return SACD_OK;
}

// Nonzeros per lane group of a warp tile ("sub"; a tile is 32/LPR groups of sub nonzeros).
// Taken from the autotuned table (tune_table.h, generated from tuning.json by the build) for the
// job's own shape: precision, row width, number of other modes, nonzero count; otherwise a rule
// that aims at several waves of warps over the GPU.
int choose_sub(const sacd_ctx* c, int n) {
  (void)n;
  const int64_t nnz = c->nnz;
  for (const TuneEntry& t : kTuneTable)
    if (t.prec == c->prec && t.rv == c->rv && t.nother == c->N - 1 && nnz >= t.nnz_lo && nnz < t.nnz_hi)
      return t.sub;
  const int groups = 32 / std::min(c->rv, 32);
  int64_t sub = nnz / ((int64_t)groups * 152 * 64);
  sub = std::max<int64_t>(8, std::min<int64_t>(128, sub));
  return (int)((sub + 3) / 4 * 4);
}

void drop_alloc(sacd_ctx* c, void* p, size_t bytes) {
  if (!p) return;
  for (size_t i = 0; i < c->allocs.size(); ++i)
    if (c->allocs[i] == p) {
      cudaFreeAsync(p, c->st);
      c->allocs.erase(c->allocs.begin() + i);
      c->device_bytes -= (int64_t)bytes;
      return;
    }
}

// Warp tiles of mode n and the list of rows split across their borders (flags, positions and the
// list are computed here; finish_split_lists reads the lists of all modes back at once).
sacd_status build_tiling(sacd_ctx* c, TmpAllocs& T, int n, int sub) {
  ModeData& md = c->m[n];
  const int64_t nnz = c->nnz;
  const int groups = 32 / std::min(c->rv, 32);
  md.sub = sub;
  md.tile = groups * sub;
  md.ntiles = (nnz + md.tile - 1) / md.tile;
  md.nlight = md.nheavy = md.nchunks = 0;
  md.split_tmp = nullptr;
  md.split_tot = nullptr;
  if (md.ntiles > 1) {
    uint32_t* flags;
    void* stmp;
    TRY(T.get(&flags, md.ntiles));
    TRY(T.get(&md.split_pos, md.ntiles));
    TRY(T.get(&md.split_tot, 1));
    TRY(T.get(reinterpret_cast<char**>(&stmp), scan_tmp_bytes(md.ntiles)));  // NOLINT
    TRY(T.get(&md.split_tmp, md.ntiles));
    launch_split_flags(md.rowid, nnz, md.tile, md.ntiles, flags, c->st);
    scan_u32(flags, md.split_pos, md.ntiles, md.split_tot, stmp, c->st);
    launch_split_emit(md.rowid, nnz, md.tile, md.ntiles, flags, md.split_pos, md.split_tmp, c->st);
    CK(cudaGetLastError());
  }
  return SACD_OK;
}

sacd_status build_mode(sacd_ctx* c, TmpAllocs& T, SortBufs& B, int n, const int32_t* uidx, const float* uvals) {
  ModeData& md = c->m[n];
  const int64_t nnz = c->nnz;
  const int N = c->N;
  if (n == 0 && nnz > 0) {
    // the distinct coordinates are already in mode-0 order (i_0, i_1, ..., i_{N-1}): alias them
    md.rowid = const_cast<int32_t*>(uidx);
    md.cidx = const_cast<int32_t*>(uidx) + c->cstride;
    md.val = const_cast<float*>(uvals);
  } else {
    TRY(dalloc(c, &md.rowid, nnz));
    TRY(dalloc(c, &md.cidx, (size_t)(N - 1) * c->cstride));
    TRY(dalloc(c, &md.val, nnz));
  }
  // The distinct coordinates are in lexicographic (i_0, ..., i_{N-1}) order, so a stable sort by
  // i_n alone yields (i_n, then the other modes in ascending mode order): the radix sort runs
  // over the bits of I_n only, not over the whole coordinate tuple.
  const std::vector<int> order{n};
  if (nnz > 0 && n > 0) {
    uint32_t* perm = nullptr;
    const int64_t cs = c->cstride;
    TRY(sort_order(c, B, uidx, cs, nnz, order, &perm));
    launch_gather_i32(uidx + (int64_t)n * cs, perm, md.rowid, nnz, c->st);
    int o = 0;
    for (int k = 0; k < N; ++k)
      if (k != n) launch_gather_i32(uidx + (int64_t)k * cs, perm, md.cidx + (int64_t)(o++) * cs, nnz, c->st);
    launch_gather_f32(uvals, perm, md.val, nnz, c->st);
    CK(cudaGetLastError());
  }
  return build_tiling(c, T, n, choose_sub(c, n));
}

// Light rows (<= 16 partials) are summed by one warp each; heavy rows are cut into chunks of
// kFixChunk partials (level 1) whose sums are added per row (level 2).
sacd_status finish_split_lists(sacd_ctx* c) {
  std::vector<std::vector<int4>> lists(c->N);
  std::vector<uint32_t> tots(c->N, 0);
  bool any = false;
  for (int n = 0; n < c->N; ++n) {
    ModeData& md = c->m[n];
    if (!md.split_tmp) continue;
    any = true;
    lists[n].resize(md.ntiles);
    CK(cudaMemcpyAsync(&tots[n], md.split_tot, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(lists[n].data(), md.split_tmp, sizeof(int4) * md.ntiles, cudaMemcpyDeviceToHost, c->st));
  }
  if (any) CK(cudaStreamSynchronize(c->st));
  for (int n = 0; n < c->N; ++n) {
    ModeData& md = c->m[n];
    if (!md.split_tmp && md.ntiles > 1) continue;  // not re-tiled in this call
    md.split_tmp = nullptr;
    md.split_tot = nullptr;
    md.split_pos = nullptr;
    std::vector<int4> light, heavy, chunks;
    for (uint32_t i = 0; i < tots[n]; ++i) {
      const int4 s = lists[n][i];
      const int64_t P = (int64_t)s.z - s.y + 1;  // partials of the row
      if (P <= 16) {
        light.push_back(s);
      } else {
        const int first = (int)chunks.size();
        for (int64_t k0 = 0; k0 < P; k0 += kFixChunk)
          chunks.push_back(make_int4(s.x, s.y, (int)k0, (int)std::min<int64_t>(kFixChunk, P - k0)));
        heavy.push_back(make_int4(s.x, first, (int)chunks.size() - first, 0));
      }
    }
    drop_alloc(c, md.split_light, sizeof(int4) * std::max<int64_t>(md.nlight, 1));
    drop_alloc(c, md.split_heavy, sizeof(int4) * std::max<int64_t>(md.nheavy, 1));
    drop_alloc(c, md.chunks, sizeof(int4) * std::max<int64_t>(md.nchunks, 1));
    md.nlight = (int64_t)light.size();
    md.nheavy = (int64_t)heavy.size();
    md.nchunks = (int64_t)chunks.size();
    TRY(dalloc(c, &md.split_light, light.size()));
    TRY(dalloc(c, &md.split_heavy, heavy.size()));
    TRY(dalloc(c, &md.chunks, chunks.size()));
    // pageable host sources: each copy has read its source when it returns
    if (!chunks.empty())
      CK(cudaMemcpyAsync(md.chunks, chunks.data(), sizeof(int4) * chunks.size(), cudaMemcpyHostToDevice, c->st));
    if (!light.empty())
      CK(cudaMemcpyAsync(md.split_light, light.data(), sizeof(int4) * light.size(), cudaMemcpyHostToDevice, c->st));
    if (!heavy.empty())
      CK(cudaMemcpyAsync(md.split_heavy, heavy.data(), sizeof(int4) * heavy.size(), cudaMemcpyHostToDevice, c->st));
    if (!md.rowfix) TRY(dalloc(c, &md.rowfix, std::max<int64_t>(md.I, 1)));
    CK(cudaMemsetAsync(md.rowfix, 0xff, sizeof(int32_t) * std::max<int64_t>(md.I, 1), c->st));
    launch_rowfix(md.split_light, md.nlight, md.split_heavy, md.nheavy, md.rowfix, c->st);
    CK(cudaGetLastError());
  }
  return SACD_OK;
}

sacd_status create_impl(const sacd_config* cfg, sacd_ctx** out) {
  *out = nullptr;
  if (!cfg) return fail(SACD_EINVAL, "null config");
  const int N = cfg->nmodes;
  if (N < 2 || N > SACD_MAXN) return fail(SACD_EINVAL, "nmodes must be in [2, 8]");
  if (!cfg->dims) return fail(SACD_EINVAL, "null dims");
  for (int n = 0; n < N; ++n)
    if (cfg->dims[n] < 1 || cfg->dims[n] > 2147483647LL) return fail(SACD_EINVAL, "dims[n] must be in [1, 2^31-1]");
  if (cfg->nnz < 0 || cfg->nnz > 2147483647LL) return fail(SACD_EINVAL, "nnz must be in [0, 2^31-1]");
  if (cfg->rank < 1 || cfg->rank > SACD_MAXR) return fail(SACD_EINVAL, "rank must be in [1, 256]");
  if (cfg->precision != SACD_FP32 && cfg->precision != SACD_BF16_GATHER) return fail(SACD_EINVAL, "bad precision");
  if (cfg->lnorm < 0 || cfg->lnorm > 2) return fail(SACD_EINVAL, "bad lnorm");
  if (cfg->fixup < 0 || cfg->fixup > 1) return fail(SACD_EINVAL, "bad fixup");
  if (cfg->nnz > 0 && (!cfg->idx || !cfg->vals)) return fail(SACD_EINVAL, "null idx or vals");
  if (cfg->nnz > 0)
    for (int n = 0; n < N; ++n)
      if (!cfg->idx[n]) return fail(SACD_EINVAL, "null idx[n]");
  if (cfg->init)
    for (int n = 0; n < N; ++n)
      if (!cfg->init[n]) return fail(SACD_EINVAL, "null init[n]");
  if (cfg->init_log2_scale < -60 || cfg->init_log2_scale > 60) return fail(SACD_EINVAL, "init_log2_scale must be in [-60, 60]");

  sacd_ctx* c = new (std::nothrow) sacd_ctx();
  if (!c) return fail(SACD_ENOMEM, "host allocation failed");
  struct Guard {
    sacd_ctx*& c;
    bool ok = false;
    ~Guard() {
      if (!ok && c) sacd_destroy(c);
    }
  } guard{c};

  c->N = N;
  for (int n = 0; n < N; ++n) c->dims[n] = cfg->dims[n];
  c->R = cfg->rank;
  c->Rp = std::max(8, next_pow2(c->R));
  c->prec = cfg->precision;
  c->rv = c->prec == SACD_FP32 ? c->Rp / 4 : c->Rp / 8;
  c->lnorm = cfg->lnorm;
  c->fixup = cfg->fixup;
  configure_kernels();
  {
    // keep freed blocks of the stream-ordered pool cached in this process (a process-local pool
    // attribute, not a device setting): contexts created and destroyed back to back reuse them
    static bool pool_done[64] = {};
    static std::mutex pool_mu;  // contexts may be created from several host threads
    std::lock_guard<std::mutex> lk(pool_mu);
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess && dev >= 0 && dev < 64 && !pool_done[dev]) {
      cudaMemPool_t pool;
      if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
      }
      cudaGetLastError();
      pool_done[dev] = true;
    }
  }
  if (cfg->stream) {
    c->st = reinterpret_cast<cudaStream_t>(cfg->stream);
  } else {
    CK(cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking));
    c->own_stream = true;
  }
  CK(cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking));
  for (auto& e : c->ev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  const int R = c->R, Rp = c->Rp;
  const cudaMemcpyKind in_kind = cfg->inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;

  // ---- small shared state
  TRY(dalloc(c, &c->zero64, 1));
  CK(cudaMemsetAsync(c->zero64, 0, sizeof(int64_t), c->st));
  TRY(dalloc(c, &c->state, (size_t)N * ST_STRIDE));
  {
    std::vector<double> st0((size_t)N * ST_STRIDE, 0.0);
    for (int n = 0; n < N; ++n) st0[(size_t)n * ST_STRIDE + ST_FIRST] = 1.0;
    CK(cudaMemcpyAsync(c->state, st0.data(), sizeof(double) * st0.size(), cudaMemcpyHostToDevice, c->st));
  }
  TRY(dalloc(c, &c->counters, 8));
  CK(cudaMemsetAsync(c->counters, 0, 8 * sizeof(unsigned int), c->st));
  TRY(dalloc(c, &c->bar, 1));
  CK(cudaMemsetAsync(c->bar, 0, sizeof(GridBar), c->st));
  {
    void* h = nullptr;
    CK(cudaMallocHost(&h, sizeof(unsigned int)));
    c->wait_host = static_cast<unsigned int*>(h);
    *c->wait_host = 0u;
  }
  TRY(dalloc(c, &c->nsel, N));
  CK(cudaMemsetAsync(c->nsel, 0, N * sizeof(unsigned long long), c->st));
  int64_t* d_dims;
  TRY(dalloc(c, &d_dims, N));
  CK(cudaMemcpyAsync(d_dims, c->dims, sizeof(int64_t) * N, cudaMemcpyHostToDevice, c->st));

  TmpAllocs T(c->st);
  SortBufs B;
  const int64_t nnz_in = cfg->nnz;
  TRY(B.alloc(T, std::max<int64_t>(nnz_in, 1)));
  int32_t* uidx = nullptr;
  float* uvals = nullptr;
  {
    // ---- COO in, validated, sorted (mode 0 order), repeats summed
    int32_t* idx_in;
    float* vals_in;
    unsigned int* bad;
    TRY(T.get(&idx_in, (size_t)N * std::max<int64_t>(nnz_in, 1)));
    TRY(T.get(&vals_in, std::max<int64_t>(nnz_in, 1)));
    TRY(T.get(&bad, 1));
    CK(cudaMemsetAsync(bad, 0, sizeof(unsigned int), c->st));
    if (nnz_in > 0) {
      for (int n = 0; n < N; ++n)
        CK(cudaMemcpyAsync(idx_in + (int64_t)n * nnz_in, cfg->idx[n], sizeof(int32_t) * nnz_in, in_kind, c->st));
      CK(cudaMemcpyAsync(vals_in, cfg->vals, sizeof(float) * nnz_in, in_kind, c->st));
      launch_validate_idx(idx_in, nnz_in, N, d_dims, nnz_in, bad, c->st);
    }
    // (an out-of-range coordinate only makes the sort below order garbage keys; it is reported
    // with the count of distinct coordinates, in one synchronisation)
    unsigned int h_bad = 0;
    CK(cudaMemcpyAsync(&h_bad, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->st));
    if (nnz_in == 0) {
      CK(cudaStreamSynchronize(c->st));
      if (h_bad) return fail(SACD_EINVAL, "a coordinate is outside [0, dims[n])");
    }

    int64_t nnz = 0;
    if (nnz_in > 0) {
      std::vector<int> order(N);
      for (int n = 0; n < N; ++n) order[n] = n;
      uint32_t* perm = nullptr;
      TRY(sort_order(c, B, idx_in, nnz_in, nnz_in, order, &perm));
      int32_t* sidx;
      float* svals;
      uint32_t *heads, *pos, *tot;
      void* stmp;
      TRY(T.get(&sidx, (size_t)N * nnz_in));
      TRY(T.get(&svals, nnz_in));
      TRY(T.get(&heads, nnz_in));
      TRY(T.get(&pos, nnz_in));
      TRY(T.get(&tot, 1));
      TRY(T.get(reinterpret_cast<char**>(&stmp), scan_tmp_bytes(nnz_in)));
      for (int n = 0; n < N; ++n)
        launch_gather_i32(idx_in + (int64_t)n * nnz_in, perm, sidx + (int64_t)n * nnz_in, nnz_in, c->st);
      launch_gather_f32(vals_in, perm, svals, nnz_in, c->st);
      launch_dup_heads(sidx, nnz_in, N, nnz_in, heads, c->st);
      scan_u32(heads, pos, nnz_in, tot, stmp, c->st);
      uint32_t h_tot = 0;
      CK(cudaMemcpyAsync(&h_tot, tot, sizeof(uint32_t), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      if (h_bad) return fail(SACD_EINVAL, "a coordinate is outside [0, dims[n])");
      nnz = h_tot;
      c->cstride = (nnz + 3) / 4 * 4;
      TRY(dalloc(c, &uidx, (size_t)N * c->cstride));  // kept: mode 0's slice structure
      TRY(dalloc(c, &uvals, nnz));
      launch_dup_compact(sidx, nnz_in, N, svals, heads, pos, nnz_in, uidx, c->cstride, uvals, c->st);
      CK(cudaGetLastError());
    }
    c->nnz = nnz;
  }
  // ||X||^2
  {
    double *part, *outp;
    TRY(T.get(&part, 1024));
    TRY(T.get(&outp, 1));
    if (c->nnz > 0) {
      launch_sumsq(uvals, c->nnz, part, 1024, outp, c->counters + 4, c->st);
      CK(cudaMemcpyAsync(&c->norm_x_sq, outp, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    }
  }
  // ---- per-mode slice structures
  for (int n = 0; n < N; ++n) {
    c->m[n].I = c->dims[n];
    TRY(build_mode(c, T, B, n, uidx, uvals));
  }
  TRY(finish_split_lists(c));  // one synchronisation (also completes the ||X||^2 read-back)
  // ---- factors and state
  int64_t Imax = 0, tiles_max = 0, p1_max = 0, gb_max = 0, chunks_max = 0;
  const int RB1 = rows_per_block_pass1(Rp), RB2 = rows_per_block_pass2(Rp);
  const int CH = gram_chunk_rows(Rp);
  for (int n = 0; n < N; ++n) {
    ModeData& md = c->m[n];
    const int64_t I = md.I;
    Imax = std::max(Imax, I);
    tiles_max = std::max(tiles_max, md.ntiles);
    chunks_max = std::max(chunks_max, md.nchunks);
    md.p1_blocks = (I + RB1 - 1) / RB1;
    md.p2_blocks = (I + RB2 - 1) / RB2;
    md.sel_rt = selupd_choose_rt(I, Rp);
    md.sel_chunks = selupd_chunks(I, Rp, md.sel_rt);
    md.gram_tc = gram_on_tensor_cores(Rp, I);
    md.gram_blocks = md.gram_tc ? gram_tc_blocks(I) : std::min<int64_t>((I + CH - 1) / CH, 4 * 152);
    p1_max = std::max(p1_max, md.p1_blocks);
    gb_max = std::max(gb_max, md.gram_blocks);
    TRY(dalloc(c, &md.A, (size_t)I * Rp));
    TRY(dalloc(c, &md.zprev, (size_t)I * Rp));
    TRY(dalloc(c, &md.M, (size_t)I * Rp));
    TRY(dalloc(c, &md.gram, (size_t)Rp * Rp));
    if (c->prec == SACD_BF16_GATHER) TRY(dalloc(c, &md.A16, (size_t)I * Rp));
    CK(cudaMemsetAsync(md.A, 0, sizeof(float) * I * Rp, c->st));
    CK(cudaMemsetAsync(md.zprev, 0, sizeof(float) * I * Rp, c->st));
    CK(cudaMemsetAsync(md.M, 0, sizeof(float) * I * Rp, c->st));
    if (cfg->init) {
      const cudaMemcpyKind k = cfg->inputs_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
      CK(cudaMemcpy2DAsync(md.A, sizeof(float) * Rp, cfg->init[n], sizeof(float) * R, sizeof(float) * R, I, k,
                           c->st));
    } else {
      launch_init_factor(md.A, I, R, Rp, cfg->seed, n, cfg->init_log2_scale, c->st);
    }
    if (md.A16) launch_to_bf16(md.A, md.A16, I * Rp, c->st);
  }
  // initial factors from the caller are checked on the device (finite, >= 0); the flag is read
  // at the synchronisation that ends context creation
  unsigned int* init_bad = nullptr;
  if (cfg->init) {
    TRY(T.get(&init_bad, 1));
    CK(cudaMemsetAsync(init_bad, 0, sizeof(unsigned int), c->st));
    for (int n = 0; n < N; ++n) launch_check_factor(c->m[n].A, c->m[n].I, R, Rp, init_bad, c->st);
  }
  TRY(dalloc(c, &c->G, (size_t)Imax * Rp));
  TRY(dalloc(c, &c->Glo, (size_t)Imax * Rp));
  TRY(dalloc(c, &c->mask, (size_t)Imax * Rp));
  TRY(dalloc(c, &c->replay, (size_t)Imax * Rp));
  c->carry_cap = std::max<int64_t>(tiles_max, 1);
  c->carry2_cap = std::max<int64_t>(chunks_max, 1);
  TRY(dalloc(c, &c->carry, (size_t)c->carry_cap * 2 * Rp));
  TRY(dalloc(c, &c->gpart, (size_t)gb_max * Rp * Rp));
  TRY(dalloc(c, &c->carry2, (size_t)c->carry2_cap * Rp));
  TRY(dalloc(c, &c->H, (size_t)Rp * Rp));
  TRY(dalloc(c, &c->Hf, (size_t)Rp * Rp));
  TRY(dalloc(c, &c->invh, Rp));
  TRY(dalloc(c, &c->lh, Rp));
  TRY(dalloc(c, &c->tipart, p1_max));
  CK(cudaMemsetAsync(c->G, 0, sizeof(float) * Imax * Rp, c->st));
  CK(cudaMemsetAsync(c->mask, 0, Imax * Rp, c->st));
  CK(cudaMemsetAsync(c->replay, 0, Imax * Rp, c->st));
  CK(cudaMemsetAsync(c->H, 0, sizeof(double) * Rp * Rp, c->st));

  // ---- step descriptors
  TRY(dalloc(c, &c->ddesc, N + 1));
  c->fit_mode = N - 1;
  if (c->prec == SACD_BF16_GATHER) {
    for (int n = 0; n < N; ++n)
      if (c->m[n].I > c->m[c->fit_mode].I || (c->m[n].I == c->m[c->fit_mode].I && n < c->fit_mode)) c->fit_mode = n;
    const int64_t If = c->m[c->fit_mode].I;
    TRY(dalloc(c, &c->Mfit, (size_t)If * Rp));
    CK(cudaMemsetAsync(c->Mfit, 0, sizeof(float) * If * Rp, c->st));
    c->dual_fit = c->fit_mode == 0 && mttkrp_dual_supported(c->rv, N - 1);
    if (c->dual_fit) {
      TRY(dalloc(c, &c->carryF, (size_t)c->carry_cap * 2 * Rp));
      TRY(dalloc(c, &c->carry2F, (size_t)c->carry2_cap * Rp));
    }
  }
  for (int n = 0; n < N; ++n) {
    ModeData& md = c->m[n];
    StepDesc& d = c->hdesc[n];
    memset(&d, 0, sizeof(d));
    d.rowid = md.rowid;
    d.cidx = md.cidx;
    d.val = md.val;
    d.nnz = c->nnz;
    d.cstride = c->cstride;
    d.nother = N - 1;
    d.prec = c->prec;
    int o = 0;
    for (int k = 0; k < N; ++k)
      if (k != n) d.fac[o++] = c->prec == SACD_FP32 ? (const void*)c->m[k].A : (const void*)c->m[k].A16;
    d.R = R;
    d.Rp = Rp;
    d.rv = c->rv;
    d.sub = md.sub;
    d.tile = md.tile;
    d.ntiles = md.ntiles;
    d.I = md.I;
    d.M = md.M;
    d.carry = c->carry;
    d.split_light = md.split_light;
    d.nsplit_light = md.nlight;
    d.split_heavy = md.split_heavy;
    d.nsplit_heavy = md.nheavy;
    d.fix_chunks = md.chunks;
    d.nfix_chunks = md.nchunks;
    d.carry2 = c->carry2;
    d.rowfix = md.rowfix;
    d.A = md.A;
    d.A16 = md.A16;
    d.G = c->G;
    d.Glo = c->Glo;
    d.zprev = md.zprev;
    d.mask = nullptr;
    d.replay = c->replay;
    for (int k = 0; k < N; ++k) d.gram[k] = c->m[k].gram;
    d.gram_out = md.gram;
    d.gpart = c->gpart;
    d.gram_blocks = (int)md.gram_blocks;
    d.N = N;
    d.n = n;
    d.lnorm = c->lnorm;
    d.fixup = c->fixup;
    d.p1_blocks = (int)md.p1_blocks;
    d.sel_chunks = (int)md.sel_chunks;
    d.H = c->H;
    d.Hf = c->Hf;
    d.invh = c->invh;
    d.lh = c->lh;
    d.tipart = c->tipart;
    d.state = c->state + (size_t)n * ST_STRIDE;
    d.counters = c->counters;
    d.nsel = c->nsel + n;
  }
  TRY(upload_descs(c));
  // ---- fit descriptor
  {
    const int L = c->fit_mode;
    c->fit_blocks = fit_blocks_for(c->m[L].I, c->Rp);
    TRY(dalloc(c, &c->fitpart, 2 * c->fit_blocks));
    TRY(dalloc(c, &c->fitout, 4));
    TRY(dalloc(c, &c->dfit, 1));
    TRY(dalloc(c, &c->fitbase, 2));
    {
      const int64_t fb[2] = {0, c->fit_blocks};
      CK(cudaMemcpyAsync(c->fitbase, fb, sizeof(fb), cudaMemcpyHostToDevice, c->st));
    }
    FitDesc& f = c->hfit;
    memset(&f, 0, sizeof(f));
    f.A = c->m[L].A;
    f.M = c->prec == SACD_BF16_GATHER ? c->Mfit : c->m[L].M;
    f.I = c->m[L].I;
    f.R = R;
    f.Rp = Rp;
    f.N = N;
    for (int k = 0; k < N; ++k) f.gram[k] = c->m[k].gram;
    f.norm_x_sq = c->norm_x_sq;
    f.part = c->fitpart;
    f.out = c->fitout;
    f.counter = c->counters + 2;
    f.wait_err = &c->bar->err;
    CK(cudaMemcpyAsync(c->dfit, &f, sizeof(f), cudaMemcpyHostToDevice, c->st));
  }
  // ---- initial Grams
  for (int n = 0; n < N; ++n) enqueue_gram(c, n);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  if (init_bad) {
    unsigned int h_bad = 0;
    CK(cudaMemcpy(&h_bad, init_bad, sizeof(unsigned int), cudaMemcpyDeviceToHost));
    if (h_bad) return fail(SACD_EINVAL, "init values must be finite and >= 0");
  }
  guard.ok = true;
  *out = c;
  return SACD_OK;
}

}  // namespace

// ==========================================================================================
// C ABI
extern "C" {

sacd_status sacd_create(const sacd_config* cfg, sacd_ctx** out) {
  if (!out) return fail(SACD_EINVAL, "null out");
  *out = nullptr;
  try {
    return create_impl(cfg, out);
  } catch (const std::bad_alloc&) {
    return fail(SACD_ENOMEM, "host allocation failed");
  } catch (...) {
    return fail(SACD_EINVAL, "unexpected exception");
  }
}

sacd_status sacd_mode_step(sacd_ctx* c, int32_t mode, int64_t* n_selected) {
  TRY(check_ctx(c));
  if (mode < 0 || mode >= c->N) return fail(SACD_EINVAL, "mode out of range");
  enqueue_step(c, mode);
  if (c->replay_mode == mode) {
    const double zero = 0.0;
    CK(cudaMemcpyAsync(c->state + (size_t)mode * ST_STRIDE + ST_REPLAY, &zero, sizeof(double),
                       cudaMemcpyHostToDevice, c->st));
    CK(cudaStreamSynchronize(c->st));
    c->replay_mode = -1;
  }
  CK(cudaGetLastError());
  c->last_mode = mode;
  c->mlast_valid = (mode == c->N - 1);  // M of the last mode depends on every other factor
  if (n_selected) {
    unsigned long long v = 0;
    CK(cudaMemcpyAsync(&v, c->nsel + mode, sizeof(v), cudaMemcpyDeviceToHost, c->st));
    TRY(check_wait(c));
    *n_selected = (int64_t)v;
  }
  return SACD_OK;
}

sacd_status sacd_iterate(sacd_ctx* c, int32_t iters) {
  TRY(check_ctx(c));
  if (iters < 0) return fail(SACD_EINVAL, "iters < 0");
  if (c->replay_mode >= 0) return fail(SACD_ESTATE, "a replay mask is pending; run sacd_mode_step first");
  if (iters == 0) return SACD_OK;
  if (c->prof.on) {
    for (int it = 0; it < iters; ++it)
      for (int n = 0; n < c->N; ++n) enqueue_step(c, n);
    CK(cudaGetLastError());
  } else {
    auto capture = [c](bool pre0, cudaGraph_t* graph, cudaGraphExec_t* exec) -> sacd_status {
      CK(cudaStreamBeginCapture(c->st, cudaStreamCaptureModeThreadLocal));
      enqueue_iteration_dag(c, pre0);
      cudaGraph_t g = nullptr;
      const cudaError_t e = cudaStreamEndCapture(c->st, &g);
      if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamEndCapture");
      *graph = g;
      CK(cudaGraphInstantiate(exec, g, 0));
      return SACD_OK;
    };
    int it = 0;
    if (c->mpre && c->fit_mode == 0) {  // the first iteration's mode-0 MTTKRP is already formed
      if (!c->gexec_pre) TRY(capture(true, &c->graph_pre, &c->gexec_pre));
      CK(cudaGraphLaunch(c->gexec_pre, c->st));
      it = 1;
    }
    c->mpre = false;
    if (it < iters && !c->gexec) TRY(capture(false, &c->graph, &c->gexec));
    for (; it < iters; ++it) CK(cudaGraphLaunch(c->gexec, c->st));
  }
  c->last_mode = c->N - 1;
  c->mlast_valid = true;
  return SACD_OK;
}

sacd_status sacd_fit(sacd_ctx* c, double* objective, double* fit) {
  TRY(check_ctx(c));
  enqueue_fit_mttkrp(c);
  {
    KScope k(c, K_FIT);
    launch_fit(c->dfit, c->fitbase, 1, c->fit_blocks, c->st);
  }
  if (!c->fit_host) {
    void* h = nullptr;
    CK(cudaMallocHost(&h, 4 * sizeof(double)));
    c->fit_host = static_cast<double*>(h);
  }
  CK(cudaMemcpyAsync(c->fit_host, c->fitout, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  if (c->fit_host[1] != 0.0) {
    c->poisoned = true;
    return fail(SACD_ETIMEOUT, "a bounded wait of the select/update kernel gave up (grid barrier)");
  }
  if (objective) *objective = c->fit_host[0];
  if (fit) *fit = fit_from_objective(c->fit_host[0], c->norm_x_sq);
  return SACD_OK;
}

sacd_status sacd_get_factor(sacd_ctx* c, int32_t mode, float* host_out) {
  TRY(check_ctx(c));
  if (mode < 0 || mode >= c->N || !host_out) return fail(SACD_EINVAL, "bad mode or null output");
  CK(cudaMemcpy2DAsync(host_out, sizeof(float) * c->R, c->m[mode].A, sizeof(float) * c->Rp, sizeof(float) * c->R,
                       c->m[mode].I, cudaMemcpyDeviceToHost, c->st));
  return check_wait(c);
}

sacd_status sacd_set_factor(sacd_ctx* c, int32_t mode, const float* host_in) {
  TRY(check_ctx(c));
  if (mode < 0 || mode >= c->N || !host_in) return fail(SACD_EINVAL, "bad mode or null input");
  const int64_t I = c->m[mode].I;
  for (int64_t e = 0; e < I * c->R; ++e)
    if (!(host_in[e] >= 0.f) || !std::isfinite(host_in[e]))
      return fail(SACD_EINVAL, "factor values must be finite and >= 0");
  c->mpre = false;  // before the factor changes, so that an error below cannot leave it set
  CK(cudaMemcpy2DAsync(c->m[mode].A, sizeof(float) * c->Rp, host_in, sizeof(float) * c->R, sizeof(float) * c->R, I,
                       cudaMemcpyHostToDevice, c->st));
  if (c->m[mode].A16) launch_to_bf16(c->m[mode].A, c->m[mode].A16, I * c->Rp, c->st);
  enqueue_gram(c, mode);
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  if (mode != c->N - 1) c->mlast_valid = false;
  c->mpre = false;
  return SACD_OK;
}

sacd_status sacd_debug_tap(sacd_ctx* c, int32_t what, int32_t mode, void* host_out) {
  TRY(check_ctx(c));
  if (!host_out) return fail(SACD_EINVAL, "null output");
  if (mode < 0 || mode >= c->N) return fail(SACD_EINVAL, "mode out of range");
  const int R = c->R, Rp = c->Rp;
  const ModeData& md = c->m[mode];
  const int64_t lastI = c->last_mode >= 0 ? c->m[c->last_mode].I : 0;
  switch (what) {
    case SACD_TAP_M:
      CK(cudaMemcpy2DAsync(host_out, sizeof(float) * R, md.M, sizeof(float) * Rp, sizeof(float) * R, md.I,
                           cudaMemcpyDeviceToHost, c->st));
      break;
    case SACD_TAP_G:
      if (c->last_mode < 0) return fail(SACD_ESTATE, "no mode step yet");
      CK(cudaMemcpy2DAsync(host_out, sizeof(float) * R, c->G, sizeof(float) * Rp, sizeof(float) * R, lastI,
                           cudaMemcpyDeviceToHost, c->st));
      break;
    case SACD_TAP_ZPREV:
      CK(cudaMemcpy2DAsync(host_out, sizeof(float) * R, md.zprev, sizeof(float) * Rp, sizeof(float) * R, md.I,
                           cudaMemcpyDeviceToHost, c->st));
      break;
    case SACD_TAP_MASK:
      if (!c->debug) return fail(SACD_ESTATE, "mask recording is off (sacd_set_debug)");
      if (c->last_mode < 0) return fail(SACD_ESTATE, "no mode step yet");
      CK(cudaMemcpy2DAsync(host_out, R, c->mask, Rp, R, lastI, cudaMemcpyDeviceToHost, c->st));
      break;
    case SACD_TAP_H:
      if (c->last_mode < 0) return fail(SACD_ESTATE, "no mode step yet");
      CK(cudaMemcpy2DAsync(host_out, sizeof(double) * R, c->H, sizeof(double) * Rp, sizeof(double) * R, R,
                           cudaMemcpyDeviceToHost, c->st));
      break;
    case SACD_TAP_GRAM:
      CK(cudaMemcpy2DAsync(host_out, sizeof(double) * R, md.gram, sizeof(double) * Rp, sizeof(double) * R, R,
                           cudaMemcpyDeviceToHost, c->st));
      break;
    case SACD_TAP_STATE: {
      double* o = reinterpret_cast<double*>(host_out);
      unsigned long long ns = 0;
      CK(cudaMemcpyAsync(o, c->state + (size_t)mode * ST_STRIDE, sizeof(double) * ST_STRIDE,
                         cudaMemcpyDeviceToHost, c->st));
      CK(cudaMemcpyAsync(&ns, c->nsel + mode, sizeof(ns), cudaMemcpyDeviceToHost, c->st));
      CK(cudaStreamSynchronize(c->st));
      o[ST_NSEL] = (double)ns;
      o[6] = 0.0;
      o[7] = 0.0;
      break;
    }
    case SACD_TAP_CSF_ROW:
      if (c->nnz) CK(cudaMemcpyAsync(host_out, md.rowid, sizeof(int32_t) * c->nnz, cudaMemcpyDeviceToHost, c->st));
      break;
    case SACD_TAP_CSF_IDX:
      if (c->nnz)
        CK(cudaMemcpy2DAsync(host_out, sizeof(int32_t) * c->nnz, md.cidx, sizeof(int32_t) * c->cstride,
                             sizeof(int32_t) * c->nnz, c->N - 1, cudaMemcpyDeviceToHost, c->st));
      break;
    case SACD_TAP_CSF_VAL:
      if (c->nnz) CK(cudaMemcpyAsync(host_out, md.val, sizeof(float) * c->nnz, cudaMemcpyDeviceToHost, c->st));
      break;
    default:
      return fail(SACD_EINVAL, "unknown tap");
  }
  CK(cudaStreamSynchronize(c->st));
  return SACD_OK;
}

sacd_status sacd_set_debug(sacd_ctx* c, int32_t on) {
  TRY(check_ctx(c));
  c->debug = on != 0;
  return upload_descs(c);
}

sacd_status sacd_replay_mask(sacd_ctx* c, int32_t mode, const uint8_t* host_mask) {
  TRY(check_ctx(c));
  if (mode < 0 || mode >= c->N) return fail(SACD_EINVAL, "mode out of range");
  double flag = 0.0;
  if (host_mask) {
    const int64_t I = c->m[mode].I;
    CK(cudaMemsetAsync(c->replay, 0, (size_t)I * c->Rp, c->st));
    CK(cudaMemcpy2DAsync(c->replay, c->Rp, host_mask, c->R, c->R, I, cudaMemcpyHostToDevice, c->st));
    flag = 1.0;
    if (c->replay_mode >= 0 && c->replay_mode != mode) {
      const double zero = 0.0;
      CK(cudaMemcpyAsync(c->state + (size_t)c->replay_mode * ST_STRIDE + ST_REPLAY, &zero, sizeof(double),
                         cudaMemcpyHostToDevice, c->st));
    }
    c->replay_mode = mode;
  } else if (c->replay_mode == mode) {
    c->replay_mode = -1;
  }
  CK(cudaMemcpyAsync(c->state + (size_t)mode * ST_STRIDE + ST_REPLAY, &flag, sizeof(double), cudaMemcpyHostToDevice,
                     c->st));
  CK(cudaStreamSynchronize(c->st));
  return SACD_OK;
}

sacd_status sacd_rmse(sacd_ctx* c, int64_t n, const int32_t* const* idx, const float* vals, int32_t on_device,
                      double* rmse) {
  TRY(check_ctx(c));
  if (n < 0 || n > 2147483647LL || !rmse || (n > 0 && (!idx || !vals))) return fail(SACD_EINVAL, "bad arguments");
  for (int k = 0; n > 0 && k < c->N; ++k)
    if (!idx[k]) return fail(SACD_EINVAL, "null idx[k]");
  try {
    TmpAllocs T(c->st);
    int32_t* didx;
    float* dvals;
    double *part, *outp;
    unsigned int *bad, *cnt;
    const int64_t blocks = std::max<int64_t>(1, (n + 255) / 256);
    TRY(T.get(&didx, (size_t)c->N * std::max<int64_t>(n, 1)));
    TRY(T.get(&dvals, std::max<int64_t>(n, 1)));
    TRY(T.get(&part, blocks));
    TRY(T.get(&outp, 1));
    TRY(T.get(&bad, 2));
    cnt = bad + 1;
    CK(cudaMemsetAsync(bad, 0, 2 * sizeof(unsigned int), c->st));
    const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (n > 0) {
      for (int k = 0; k < c->N; ++k)
        CK(cudaMemcpyAsync(didx + (int64_t)k * n, idx[k], sizeof(int32_t) * n, kind, c->st));
      CK(cudaMemcpyAsync(dvals, vals, sizeof(float) * n, kind, c->st));
      int64_t* ddims;
      TRY(T.get(&ddims, c->N));
      CK(cudaMemcpyAsync(ddims, c->dims, sizeof(int64_t) * c->N, cudaMemcpyHostToDevice, c->st));
      launch_validate_idx(didx, n, c->N, ddims, n, bad, c->st);
    }
    const float* fac[SACD_MAXN];
    for (int k = 0; k < c->N; ++k) fac[k] = c->m[k].A;
    launch_rmse(didx, dvals, n, fac, c->N, c->R, c->Rp, part, blocks, outp, cnt, c->st);
    unsigned int h_bad = 0;
    CK(cudaMemcpyAsync(&h_bad, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpyAsync(rmse, outp, sizeof(double), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (h_bad) return fail(SACD_EINVAL, "a test coordinate is outside [0, dims[n])");
  } catch (const std::bad_alloc&) {
    return fail(SACD_ENOMEM, "host allocation failed");
  }
  return SACD_OK;
}

sacd_status sacd_pattern_distinctiveness(sacd_ctx* c, int32_t mode, double* pd) {
  TRY(check_ctx(c));
  if (mode < 0 || mode >= c->N || !pd) return fail(SACD_EINVAL, "bad mode or null output");
  TmpAllocs T(c->st);
  double* outp;
  TRY(T.get(&outp, 1));
  launch_pd(c->m[mode].gram, c->R, c->Rp, outp, c->st);
  CK(cudaMemcpyAsync(pd, outp, sizeof(double), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  return SACD_OK;
}

// Checkpoint layout (host byte order): "SACDSTv1", int32 N, int32 R, int64 nnz, int64 dims[N];
// then per mode: double ti^{k-1}, double first-visit flag, float A[I x R], float z^{k-1}[I x R].
static size_t state_bytes(const sacd_ctx* c) {
  size_t b = 8 + 4 + 4 + 8 + 8 * (size_t)c->N;
  for (int n = 0; n < c->N; ++n) b += 16 + 2 * sizeof(float) * (size_t)c->m[n].I * c->R;
  return b;
}

sacd_status sacd_save(sacd_ctx* c, void* host_buf, size_t cap, size_t* bytes) {
  TRY(check_ctx(c));
  const size_t need = state_bytes(c);
  if (bytes) *bytes = need;
  if (!host_buf) return SACD_OK;
  if (cap < need) return fail(SACD_EINVAL, "buffer smaller than the state (query the size with a NULL buffer)");
  char* p = reinterpret_cast<char*>(host_buf);
  memcpy(p, "SACDSTv1", 8);
  p += 8;
  const int32_t N = c->N, R = c->R;
  memcpy(p, &N, 4);
  memcpy(p + 4, &R, 4);
  memcpy(p + 8, &c->nnz, 8);
  memcpy(p + 16, c->dims, 8 * (size_t)N);
  p += 16 + 8 * (size_t)N;
  std::vector<double> st((size_t)N * ST_STRIDE);
  CK(cudaMemcpyAsync(st.data(), c->state, sizeof(double) * st.size(), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (int n = 0; n < N; ++n) {
    const double s2[2] = {st[(size_t)n * ST_STRIDE + ST_TIPREV], st[(size_t)n * ST_STRIDE + ST_FIRST]};
    memcpy(p, s2, 16);
    p += 16;
    const size_t mb = sizeof(float) * (size_t)c->m[n].I * R;
    CK(cudaMemcpy2DAsync(p, sizeof(float) * R, c->m[n].A, sizeof(float) * c->Rp, sizeof(float) * R, c->m[n].I,
                         cudaMemcpyDeviceToHost, c->st));
    CK(cudaMemcpy2DAsync(p + mb, sizeof(float) * R, c->m[n].zprev, sizeof(float) * c->Rp, sizeof(float) * R,
                         c->m[n].I, cudaMemcpyDeviceToHost, c->st));
    p += 2 * mb;
  }
  CK(cudaStreamSynchronize(c->st));
  return SACD_OK;
}

sacd_status sacd_load(sacd_ctx* c, const void* host_buf, size_t bytes) {
  TRY(check_ctx(c));
  if (!host_buf || bytes < state_bytes(c)) return fail(SACD_EINVAL, "buffer too small for this context's state");
  const char* p = reinterpret_cast<const char*>(host_buf);
  if (memcmp(p, "SACDSTv1", 8) != 0) return fail(SACD_EINVAL, "not a SaCD state buffer");
  int32_t N, R;
  int64_t nnz;
  memcpy(&N, p + 8, 4);
  memcpy(&R, p + 12, 4);
  memcpy(&nnz, p + 16, 8);
  if (N != c->N || R != c->R || nnz != c->nnz) return fail(SACD_EINVAL, "state of another tensor or rank");
  for (int n = 0; n < N; ++n) {
    int64_t d;
    memcpy(&d, p + 24 + 8 * n, 8);
    if (d != c->dims[n]) return fail(SACD_EINVAL, "state of another tensor shape");
  }
  p += 24 + 8 * (size_t)N;
  std::vector<double> st((size_t)N * ST_STRIDE);
  CK(cudaMemcpyAsync(st.data(), c->state, sizeof(double) * st.size(), cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  {  // every factor is checked before anything is copied: a rejected buffer leaves the context as it was
    const char* q = p;
    for (int n = 0; n < N; ++n) {
      const float* a = reinterpret_cast<const float*>(q + 16);
      for (int64_t e = 0; e < c->m[n].I * R; ++e)
        if (!(a[e] >= 0.f) || !std::isfinite(a[e])) return fail(SACD_EINVAL, "factor values must be finite and >= 0");
      q += 16 + 2 * sizeof(float) * (size_t)c->m[n].I * R;
    }
  }
  c->mlast_valid = false;  // before the factors change, so that an error below cannot leave them set
  c->mpre = false;
  for (int n = 0; n < N; ++n) {
    double s2[2];
    memcpy(s2, p, 16);
    st[(size_t)n * ST_STRIDE + ST_TIPREV] = s2[0];
    st[(size_t)n * ST_STRIDE + ST_FIRST] = s2[1];
    p += 16;
    const size_t mb = sizeof(float) * (size_t)c->m[n].I * R;
    CK(cudaMemcpy2DAsync(c->m[n].A, sizeof(float) * c->Rp, p, sizeof(float) * R, sizeof(float) * R, c->m[n].I,
                         cudaMemcpyHostToDevice, c->st));
    CK(cudaMemcpy2DAsync(c->m[n].zprev, sizeof(float) * c->Rp, p + mb, sizeof(float) * R, sizeof(float) * R,
                         c->m[n].I, cudaMemcpyHostToDevice, c->st));
    if (c->m[n].A16) launch_to_bf16(c->m[n].A, c->m[n].A16, c->m[n].I * c->Rp, c->st);
    enqueue_gram(c, n);
    p += 2 * mb;
  }
  CK(cudaMemcpyAsync(c->state, st.data(), sizeof(double) * st.size(), cudaMemcpyHostToDevice, c->st));
  CK(cudaGetLastError());
  CK(cudaStreamSynchronize(c->st));
  c->mlast_valid = false;
  c->mpre = false;
  return SACD_OK;
}

sacd_status sacd_set_tiling(sacd_ctx* c, int32_t mode, int32_t sub) {
  TRY(check_ctx(c));
  if (mode < 0 || mode >= c->N) return fail(SACD_EINVAL, "mode out of range");
  if (sub < 4 || sub > 1024 || (sub & 3)) return fail(SACD_EINVAL, "sub must be a multiple of 4 in [4, 1024]");
  // the tile partials of the objective's pass may move or be dropped below, also on an error path
  c->mpre = false;
  try {
    {
      TmpAllocs T(c->st);
      TRY(build_tiling(c, T, mode, sub));
      TRY(finish_split_lists(c));
      CK(cudaStreamSynchronize(c->st));
    }
    ModeData& md = c->m[mode];
    if (md.ntiles > c->carry_cap) {
      drop_alloc(c, c->carry, sizeof(float) * c->carry_cap * 2 * c->Rp);
      if (c->carryF) drop_alloc(c, c->carryF, sizeof(float) * c->carry_cap * 2 * c->Rp);
      c->carry_cap = md.ntiles;
      TRY(dalloc(c, &c->carry, (size_t)c->carry_cap * 2 * c->Rp));
      if (c->dual_fit) TRY(dalloc(c, &c->carryF, (size_t)c->carry_cap * 2 * c->Rp));
    }
    if (md.nchunks > c->carry2_cap) {
      drop_alloc(c, c->carry2, sizeof(float) * c->carry2_cap * c->Rp);
      if (c->carry2F) drop_alloc(c, c->carry2F, sizeof(float) * c->carry2_cap * c->Rp);
      c->carry2_cap = md.nchunks;
      TRY(dalloc(c, &c->carry2, (size_t)c->carry2_cap * c->Rp));
      if (c->dual_fit) TRY(dalloc(c, &c->carry2F, (size_t)c->carry2_cap * c->Rp));
    }
    for (int n = 0; n < c->N; ++n) {
      StepDesc& d = c->hdesc[n];
      d.carry = c->carry;
      d.carry2 = c->carry2;
    }
    StepDesc& d = c->hdesc[mode];
    d.sub = md.sub;
    d.tile = md.tile;
    d.ntiles = md.ntiles;
    d.split_light = md.split_light;
    d.nsplit_light = md.nlight;
    d.split_heavy = md.split_heavy;
    d.nsplit_heavy = md.nheavy;
    d.fix_chunks = md.chunks;
    d.nfix_chunks = md.nchunks;
    d.rowfix = md.rowfix;
    return upload_descs(c);
  } catch (const std::bad_alloc&) {
    return fail(SACD_ENOMEM, "host allocation failed");
  }
}

sacd_status sacd_get_info(sacd_ctx* c, sacd_info* out) {
  if (!c || !out) return fail(SACD_EINVAL, "null argument");
  memset(out, 0, sizeof(*out));
  out->nmodes = c->N;
  out->rank = c->R;
  out->rank_padded = c->Rp;
  out->precision = c->prec;
  for (int n = 0; n < c->N; ++n) {
    out->dims[n] = c->dims[n];
    out->tiles[n] = c->m[n].ntiles;
    out->tile_nnz[n] = c->m[n].tile;
    out->split_rows[n] = c->m[n].nlight + c->m[n].nheavy;
  }
  out->nnz = c->nnz;
  out->norm_x_sq = c->norm_x_sq;
  out->device_bytes = c->device_bytes;
  return SACD_OK;
}

sacd_status sacd_sync(sacd_ctx* c) {
  TRY(check_ctx(c));
  return check_wait(c);
}

sacd_status sacd_set_wait_budget(sacd_ctx* c, int64_t cycles) {
  TRY(check_ctx(c));
  if (cycles < 1) return fail(SACD_EINVAL, "the wait budget must be at least one cycle");
  c->wait_budget = cycles;
  invalidate_graph(c);  // the budget is a kernel argument of the captured iteration
  return SACD_OK;
}

sacd_status sacd_profile_enable(sacd_ctx* c, int32_t on) {
  TRY(check_ctx(c));
  Prof& p = c->prof;
  if (on && p.ev.empty()) {
    p.ev.resize(4096);
    p.cls.resize(2048);
    for (auto& e : p.ev) CK(cudaEventCreate(&e));
  }
  if (on) {
    for (int i = 0; i < K_NCLASS; ++i) {
      p.launches[i] = 0;
      p.ms[i] = 0.0;
    }
    p.used = 0;
    p.dropped = 0;
  }
  p.on = on != 0;
  return SACD_OK;
}

sacd_status sacd_profile_read(sacd_ctx* c, sacd_kernel_stat* out, int32_t cap, int32_t* n) {
  TRY(check_ctx(c));
  Prof& p = c->prof;
  CK(cudaStreamSynchronize(c->st));
  for (int i = 0; i < p.used; ++i) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p.ev[2 * i], p.ev[2 * i + 1]) == cudaSuccess) {
      p.ms[p.cls[i]] += ms;
      p.launches[p.cls[i]] += 1;
    } else {
      cudaGetLastError();
      p.dropped++;
    }
  }
  p.used = 0;
  int k = 0;
  for (int i = 0; i < K_NCLASS; ++i) {
    if (k < cap && out) {
      memset(out[k].name, 0, sizeof(out[k].name));
      strncpy(out[k].name, kClassName[i], sizeof(out[k].name) - 1);
      out[k].launches = p.launches[i];
      out[k].total_ms = p.ms[i];
    }
    ++k;
  }
  if (n) *n = k;
  return SACD_OK;
}

void sacd_destroy(sacd_ctx* c) {
  if (!c) return;
  if (c->st) cudaStreamSynchronize(c->st);
  invalidate_graph(c);
  for (auto& e : c->prof.ev) cudaEventDestroy(e);
  for (auto it = c->allocs.rbegin(); it != c->allocs.rend(); ++it) cudaFreeAsync(*it, c->st);  // last in, first out
  if (c->st) cudaStreamSynchronize(c->st);
  for (auto& e : c->ev)
    if (e) cudaEventDestroy(e);
  if (c->side) cudaStreamDestroy(c->side);
  if (c->own_stream && c->st) cudaStreamDestroy(c->st);
  if (c->fit_host) cudaFreeHost(c->fit_host);
  if (c->wait_host) cudaFreeHost(c->wait_host);
  cudaGetLastError();
  delete c;
}

const char* sacd_last_error(void) { return g_err.c_str(); }

}  // extern "C"

// ==========================================================================================
// Batches: many independent contexts stepped together. Every kernel of a mode step is launched
// once for all the jobs that have that mode (descriptor arrays + per-job prefix sums of the
// work items); the MTTKRP and the Gram, which are specialised on the row width, are launched
// once per width class. Each job's arithmetic is exactly what its own context would do, so a
// job's results are bit-identical alone and in any mix.
namespace {

struct PlanClass {
  int rv = 0, nother = 0, Rp = 0, prec = 0;
  bool gram_tc = false;
  int njobs = 0;
  StepDesc* d_descs = nullptr;
  int64_t* d_tile_base = nullptr;
  int64_t tiles = 0;
  int64_t* d_gram_base = nullptr;
  int64_t gram_blocks = 0;
};

struct PlanMode {
  int njobs = 0;
  std::vector<sacd_ctx*> jobs;
  StepDesc* d_descs = nullptr;
  int64_t *d_chunk = nullptr, *d_p1 = nullptr, *d_p2 = nullptr, *d_gr = nullptr, *d_sel = nullptr;
  int64_t chunk = 0, p1 = 0, p2 = 0, gr = 0, sel = 0;  // (light rows and heavy rows' chunk sums: in pass 1)
  bool fused = true;  // no job uses the GCD variant: one fused select/update launch for all jobs
  size_t sel_smem = 0;  // the largest shared memory need of the fused kernel over the jobs
  int sel_rt = 1;       // its rows per thread
  size_t smem = 0;
  std::vector<PlanClass> classes;
  std::vector<sacd_ctx*> empty_jobs;  // no nonzeros: M is zeroed instead of an MTTKRP
};

struct BatchPlan {
  int maxN = 0;
  int njobs = 0;
  PlanMode modes[SACD_MAXN];
  FitDesc* d_fit = nullptr;
  int64_t* d_fit_base = nullptr;
  int64_t fit_blocks = 0;
  double* d_fit_out = nullptr;  // njobs x 4
  GridBar* d_bar = nullptr;      // grid barrier of the fused select/update launches
  long long wait_budget = kWaitBudgetCycles;
  std::vector<void*> allocs;
  cudaStream_t alloc_st = nullptr;

  template <typename T>
  sacd_status alloc_copy(T** dst, const std::vector<T>& src, cudaStream_t st) {
    void* q = nullptr;
    const size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
    alloc_st = st;
    if (cudaMallocAsync(&q, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      return fail(SACD_ENOMEM, "cudaMalloc of a batch plan array failed");
    }
    allocs.push_back(q);
    *dst = reinterpret_cast<T*>(q);
    if (!src.empty() && cudaMemcpyAsync(q, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, st) != cudaSuccess)
      return fail(SACD_ECUDA, "copy of a batch plan array failed");
    return SACD_OK;
  }

  void release() {
    for (void* p : allocs) cudaFreeAsync(p, alloc_st);  // after the work already enqueued
    allocs.clear();
  }

  static std::vector<int64_t> prefix(const std::vector<int64_t>& counts) {
    std::vector<int64_t> b(counts.size() + 1, 0);
    for (size_t i = 0; i < counts.size(); ++i) b[i + 1] = b[i] + counts[i];
    return b;
  }

  sacd_status build(const std::vector<sacd_ctx*>& jobs, cudaStream_t st) {
    njobs = (int)jobs.size();
    maxN = 0;
    for (sacd_ctx* c : jobs) maxN = std::max(maxN, c->N);
    for (int n = 0; n < maxN; ++n) {
      PlanMode& pm = modes[n];
      pm = PlanMode();
      std::vector<StepDesc> descs;
      std::vector<int64_t> chunk, p1, p2, gr, sel;
      // rows per thread of the mode's fused select/update launch: 4 when the jobs' 4-row chunks
      // fill the GPU twice over
      int64_t chunks4 = 0;
      for (sacd_ctx* c : jobs)
        if (n < c->N) chunks4 += selupd_chunks(c->m[n].I, c->Rp, 4);
      pm.sel_rt = chunks4 >= 2 * 152 * 2 ? 4 : 1;
      for (sacd_ctx* c : jobs) {
        if (n >= c->N) continue;
        pm.jobs.push_back(c);
        descs.push_back(c->hdesc[n]);
        const ModeData& md = c->m[n];
        chunk.push_back(md.nchunks);
        p1.push_back(md.p1_blocks);
        p2.push_back(md.p2_blocks);
        gr.push_back(gram_reduce_blocks(c->Rp));
        sel.push_back(selupd_chunks(md.I, c->Rp, pm.sel_rt));
        descs.back().sel_chunks = (int)sel.back();
        if (c->lnorm == SACD_LNORM_GCD) pm.fused = false;
        pm.sel_smem = std::max(pm.sel_smem, selupd_smem_bytes(c->Rp, pm.sel_rt));
        pm.smem = std::max(pm.smem, pass_smem_bytes(c->Rp));
        if (c->nnz == 0) pm.empty_jobs.push_back(c);
      }
      pm.njobs = (int)pm.jobs.size();
      if (!pm.njobs) continue;
      auto tot = [](const std::vector<int64_t>& v) { int64_t s = 0; for (auto x : v) s += x; return s; };
      pm.chunk = tot(chunk);
      pm.p1 = tot(p1); pm.p2 = tot(p2); pm.gr = tot(gr); pm.sel = tot(sel);
      TRY(alloc_copy(&pm.d_descs, descs, st));
      TRY(alloc_copy(&pm.d_sel, prefix(sel), st));
      TRY(alloc_copy(&pm.d_chunk, prefix(chunk), st));
      TRY(alloc_copy(&pm.d_p1, prefix(p1), st));
      TRY(alloc_copy(&pm.d_p2, prefix(p2), st));
      TRY(alloc_copy(&pm.d_gr, prefix(gr), st));
      // width classes for the MTTKRP (rv, number of other modes, precision) and the Gram (Rp, and
      // whether it runs on the tensor cores)
      std::vector<std::vector<sacd_ctx*>> groups;
      for (sacd_ctx* c : pm.jobs) {
        bool placed = false;
        for (auto& gcls : groups)
          if (gcls[0]->rv == c->rv && gcls[0]->N == c->N && gcls[0]->prec == c->prec && gcls[0]->Rp == c->Rp &&
              gcls[0]->m[n].gram_tc == c->m[n].gram_tc) {
            gcls.push_back(c);
            placed = true;
            break;
          }
        if (!placed) groups.push_back({c});
      }
      for (auto& gcls : groups) {
        PlanClass pc;
        pc.rv = gcls[0]->rv;
        pc.nother = gcls[0]->N - 1;
        pc.Rp = gcls[0]->Rp;
        pc.prec = gcls[0]->prec;
        pc.gram_tc = gcls[0]->m[n].gram_tc;
        pc.njobs = (int)gcls.size();
        std::vector<StepDesc> cd;
        std::vector<int64_t> tl, gb;
        for (sacd_ctx* c : gcls) {
          cd.push_back(c->hdesc[n]);
          tl.push_back(c->m[n].ntiles);
          gb.push_back(c->m[n].gram_blocks);
        }
        pc.tiles = tot(tl);
        pc.gram_blocks = tot(gb);
        TRY(alloc_copy(&pc.d_descs, cd, st));
        TRY(alloc_copy(&pc.d_tile_base, prefix(tl), st));
        TRY(alloc_copy(&pc.d_gram_base, prefix(gb), st));
        pm.classes.push_back(pc);
      }
    }
    // batched objective
    std::vector<FitDesc> fds;
    std::vector<int64_t> fb;
    for (int j = 0; j < njobs; ++j) fds.push_back(jobs[j]->hfit), fb.push_back(jobs[j]->fit_blocks);
    fit_blocks = 0;
    for (auto x : fb) fit_blocks += x;
    std::vector<double> zeros((size_t)njobs * 4, 0.0);
    TRY(alloc_copy(&d_fit_out, zeros, st));
    TRY(alloc_copy(&d_bar, std::vector<GridBar>(1, GridBar{}), st));
    for (int j = 0; j < njobs; ++j) {
      fds[j].out = d_fit_out + 4 * j;
      fds[j].wait_err = &d_bar->err;
    }
    TRY(alloc_copy(&d_fit, fds, st));
    TRY(alloc_copy(&d_fit_base, prefix(fb), st));
    if (cudaStreamSynchronize(st) != cudaSuccess) return fail(SACD_ECUDA, "batch plan upload failed");
    return SACD_OK;
  }

  // One outer iteration of every job (mode steps 0..maxN-1; a job takes part in the modes it has).
  void enqueue_iteration(cudaStream_t st) const {
    for (int n = 0; n < maxN; ++n) {
      const PlanMode& pm = modes[n];
      if (!pm.njobs) continue;
      launch_hl(pm.d_descs, pm.njobs, st);
      for (sacd_ctx* c : pm.empty_jobs)
        cudaMemsetAsync(c->m[n].M, 0, (size_t)c->m[n].I * c->Rp * sizeof(float), st);
      for (const PlanClass& pc : pm.classes)
        launch_mttkrp(pc.d_descs, pc.d_tile_base, pc.njobs, pc.tiles, pc.prec, pc.rv, pc.nother, st);
      launch_fixup_chunks(pm.d_descs, pm.d_chunk, pm.njobs, pm.chunk, st);  // the rest is folded into pass 1
      if (pm.fused) {
        launch_selupd(pm.d_descs, pm.d_sel, pm.njobs, pm.sel, pm.sel_rt, pm.sel_smem, d_bar, wait_budget, st);
      } else {
        launch_pass1(pm.d_descs, pm.d_p1, pm.njobs, pm.p1, pm.smem, st);
        launch_pass2(pm.d_descs, pm.d_p2, pm.njobs, pm.p2, pm.smem, st);
      }
      for (const PlanClass& pc : pm.classes)
        launch_gram(pc.d_descs, pc.d_gram_base, pc.njobs, pc.gram_blocks, pc.Rp, pc.gram_tc, st);
      launch_gram_reduce(pm.d_descs, pm.d_gr, pm.njobs, pm.gr, st);
    }
  }

  void enqueue_fit(cudaStream_t st) const { launch_fit(d_fit, d_fit_base, njobs, fit_blocks, st); }
};

}  // namespace

struct sacd_batch {
  std::vector<sacd_ctx*> jobs;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  bool poisoned = false;
  BatchPlan plan;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
};

extern "C" {

sacd_status sacd_batch_create(const sacd_config* cfgs, int32_t njobs, void* stream, sacd_batch** out) {
  if (!out) return fail(SACD_EINVAL, "null out");
  *out = nullptr;
  if (!cfgs || njobs < 1) return fail(SACD_EINVAL, "need at least one job configuration");
  sacd_batch* b = new (std::nothrow) sacd_batch();
  if (!b) return fail(SACD_ENOMEM, "host allocation failed");
  try {
    if (stream) {
      b->st = reinterpret_cast<cudaStream_t>(stream);
    } else {
      if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess) {
        delete b;
        return fail(SACD_ECUDA, "cudaStreamCreate failed");
      }
      b->own_stream = true;
    }
    for (int j = 0; j < njobs; ++j) {
      sacd_config c = cfgs[j];
      c.stream = b->st;
      sacd_ctx* ctx = nullptr;
      const sacd_status s = sacd_create(&c, &ctx);
      if (s != SACD_OK) {
        const std::string msg = "job " + std::to_string(j) + ": " + g_err;
        sacd_batch_destroy(b);
        return fail(s, msg);
      }
      b->jobs.push_back(ctx);
    }
    const sacd_status s = b->plan.build(b->jobs, b->st);
    if (s != SACD_OK) {
      sacd_batch_destroy(b);
      return s;
    }
  } catch (const std::bad_alloc&) {
    sacd_batch_destroy(b);
    return fail(SACD_ENOMEM, "host allocation failed");
  }
  *out = b;
  return SACD_OK;
}

sacd_status sacd_batch_iterate(sacd_batch* b, int32_t iters) {
  if (!b) return fail(SACD_EINVAL, "null batch");
  if (b->poisoned) return fail(SACD_ESTATE, "batch is poisoned by an earlier CUDA error");
  if (iters < 0) return fail(SACD_EINVAL, "iters < 0");
  if (iters == 0) return SACD_OK;
  for (sacd_ctx* c : b->jobs)
    if (c->replay_mode >= 0) return fail(SACD_ESTATE, "a job has a pending replay mask");
  cudaError_t e;
  if (!b->gexec) {
    e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      b->plan.enqueue_iteration(b->st);
      cudaGraph_t g = nullptr;
      e = cudaStreamEndCapture(b->st, &g);
      b->graph = g;
      if (e == cudaSuccess) e = cudaGraphInstantiate(&b->gexec, b->graph, 0);
    }
    if (e != cudaSuccess) {
      b->poisoned = true;
      return fail(SACD_ECUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
    }
  }
  for (int it = 0; it < iters; ++it) {
    e = cudaGraphLaunch(b->gexec, b->st);
    if (e != cudaSuccess) {
      b->poisoned = true;
      return fail(SACD_ECUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
    }
  }
  for (sacd_ctx* c : b->jobs) {
    c->last_mode = c->N - 1;
    c->mlast_valid = true;
    c->mpre = false;
  }
  return SACD_OK;
}

sacd_status sacd_batch_fit(sacd_batch* b, double* objective, double* fit) {
  if (!b) return fail(SACD_EINVAL, "null batch");
  if (b->poisoned) return fail(SACD_ESTATE, "batch is poisoned by an earlier CUDA error");
  for (sacd_ctx* c : b->jobs) enqueue_fit_mttkrp(c);
  b->plan.enqueue_fit(b->st);
  std::vector<double> out((size_t)b->jobs.size() * 4);
  cudaError_t e = cudaMemcpyAsync(out.data(), b->plan.d_fit_out, sizeof(double) * out.size(), cudaMemcpyDeviceToHost,
                                  b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) {
    b->poisoned = true;
    return fail(SACD_ECUDA, std::string("batch fit: ") + cudaGetErrorString(e));
  }
  for (size_t j = 0; j < b->jobs.size(); ++j)
    if (out[4 * j + 1] != 0.0) {
      b->poisoned = true;
      return fail(SACD_ETIMEOUT, "a bounded wait of the select/update kernel gave up (grid barrier)");
    }
  for (size_t j = 0; j < b->jobs.size(); ++j) {
    if (objective) objective[j] = out[4 * j];
    if (fit) fit[j] = fit_from_objective(out[4 * j], b->jobs[j]->norm_x_sq);
  }
  return SACD_OK;
}

sacd_status sacd_batch_job(sacd_batch* b, int32_t job, sacd_ctx** ctx_out) {
  if (!b || !ctx_out || job < 0 || job >= (int)b->jobs.size()) return fail(SACD_EINVAL, "bad batch or job");
  *ctx_out = b->jobs[job];
  return SACD_OK;
}

void sacd_batch_destroy(sacd_batch* b) {
  if (!b) return;
  if (b->st) cudaStreamSynchronize(b->st);
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->plan.release();
  for (sacd_ctx* c : b->jobs) sacd_destroy(c);
  if (b->own_stream && b->st) cudaStreamDestroy(b->st);
  cudaGetLastError();
  delete b;
}

}  // extern "C"

// ==========================================================================================
// Serving: continuous batching of factorisation jobs. Jobs wait in FIFO order until the device
// memory they need fits the budget; every step runs one outer iteration of every admitted job
// with one batched launch set; a job that reached its iteration count is finished (objective,
// fit and factors copied to the host) and its device memory is freed at once, so waiting jobs
// join at the next step. Per-job arithmetic is the context's own: results do not depend on the
// mix.
#include <chrono>
#include <deque>
#include <map>

namespace {

struct ServerJob {
  int64_t id = 0;
  sacd_config cfg{};
  std::vector<int64_t> dims;
  std::vector<const int32_t*> idx;
  std::vector<const float*> init;
  int32_t iters = 0, done_iters = 0;
  int64_t est_bytes = 0, bytes = 0;
  double t_submit = 0, t_admit = -1, t_done = -1;
  sacd_ctx* ctx = nullptr;
  int32_t status = 0;
  sacd_status create_status = SACD_OK;  // set by the preparation thread
  std::string error;
  double objective = 0, fit = 0;
  std::vector<std::vector<float>> factors;
};

// Upper bound of the device bytes a context of this configuration holds at its peak (during
// sacd_create, when the sort buffers and the unsorted copy coexist with the slice structures).
int64_t estimate_bytes(const sacd_config* c) {
  const int64_t N = c->nmodes, nnz = c->nnz;
  int Rp = 8;
  while (Rp < c->rank) Rp <<= 1;
  int64_t rows = 0, Imax = 0;
  for (int n = 0; n < N; ++n) {
    rows += c->dims[n];
    Imax = std::max<int64_t>(Imax, c->dims[n]);
  }
  const int64_t csf = N * nnz * 4 * (N + 1);
  const int64_t facs = rows * Rp * (12 + (c->precision == SACD_BF16_GATHER ? 2 : 0)) + N * (int64_t)Rp * Rp * 8 +
                       rows * 4;  // + the row -> split entry maps
  const int64_t tiles = nnz / 32 + 1;
  const int64_t gram_blocks = std::min<int64_t>((Imax + 4096 / Rp - 1) / (4096 / Rp), 4 * 152);
  // tile partials (a second set for the objective's own in BF16 mode), chunk sums, Gram partials
  const int64_t partial_sets = c->precision == SACD_BF16_GATHER ? 2 : 1;
  const int64_t scratch =
      Imax * Rp * 6 + partial_sets * tiles * (2 * Rp * 4 + 16) + gram_blocks * Rp * Rp * 8 + (1 << 20);
  const int64_t temps = nnz * (12 * N + 64) + (nnz / 2048 + 1) * 256 * 12;
  return (csf + facs + scratch + temps) * 11 / 10;
}

double now_s(const std::chrono::steady_clock::time_point& t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace

struct sacd_server {
  int64_t budget = 0;
  int32_t max_active = 0;
  int32_t max_admit = 0;
  cudaStream_t st = nullptr;
  bool own_stream = false;
  bool poisoned = false;
  int64_t used = 0, peak_used = 0;
  int64_t next_id = 1;
  std::chrono::steady_clock::time_point t0;
  std::deque<ServerJob*> waiting;
  std::vector<ServerJob*> active;
  // admitted jobs whose contexts a preparation thread creates on its own stream (H2D copies,
  // sorts) while the iteration stream runs; they join the plan at the next step
  int dev = 0;
  cudaStream_t prep_st = nullptr;
  std::thread prep;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<ServerJob*> to_create;  // guarded by mu
  std::deque<ServerJob*> created;    // guarded by mu
  bool stop = false;                 // guarded by mu
  int32_t inflight = 0;              // admitted, not yet iterating (main thread)
  int64_t reserved = 0;              // their create-time bound (main thread)
  std::deque<ServerJob*> finished;    // results not drained yet
  std::map<int64_t, ServerJob*> kept; // drained, factors kept until released
  BatchPlan plan;
  bool plan_dirty = true;
  int64_t steps = 0;
};

namespace {

// The preparation thread: creates the contexts of admitted jobs, in admission order.
void prep_loop(sacd_server* s) {
  cudaSetDevice(s->dev);
  std::unique_lock<std::mutex> lk(s->mu);
  while (true) {
    s->cv.wait(lk, [s] { return s->stop || !s->to_create.empty(); });
    if (s->stop) return;
    ServerJob* j = s->to_create.front();
    s->to_create.pop_front();
    lk.unlock();
    j->cfg.stream = s->prep_st;
    sacd_ctx* c = nullptr;
    j->create_status = sacd_create(&j->cfg, &c);  // synchronises prep_st before returning
    if (j->create_status != SACD_OK) j->error = g_err;
    j->ctx = c;
    lk.lock();
    s->created.push_back(j);
    s->cv.notify_all();
  }
}

void finish_job(sacd_server* s, ServerJob* j) {
  j->t_done = now_s(s->t0);
  if (j->ctx) {
    s->used -= j->bytes;
    sacd_destroy(j->ctx);
    j->ctx = nullptr;
  }
  s->finished.push_back(j);
}

}  // namespace

extern "C" {

sacd_status sacd_server_create(int64_t hbm_budget_bytes, int32_t max_active, int32_t max_admit_per_step,
                               void* stream, sacd_server** out) {
  if (!out) return fail(SACD_EINVAL, "null out");
  *out = nullptr;
  if (hbm_budget_bytes <= 0 || max_active < 1 || max_admit_per_step < 1)
    return fail(SACD_EINVAL, "budget, max_active and max_admit_per_step must be positive");
  sacd_server* s = new (std::nothrow) sacd_server();
  if (!s) return fail(SACD_ENOMEM, "host allocation failed");
  s->budget = hbm_budget_bytes;
  s->max_active = max_active;
  s->max_admit = max_admit_per_step;
  s->t0 = std::chrono::steady_clock::now();
  if (stream) {
    s->st = reinterpret_cast<cudaStream_t>(stream);
  } else {
    if (cudaStreamCreateWithFlags(&s->st, cudaStreamNonBlocking) != cudaSuccess) {
      delete s;
      return fail(SACD_ECUDA, "cudaStreamCreate failed");
    }
    s->own_stream = true;
  }
  if (cudaGetDevice(&s->dev) != cudaSuccess || cudaStreamCreateWithFlags(&s->prep_st, cudaStreamNonBlocking) != cudaSuccess) {
    if (s->own_stream) cudaStreamDestroy(s->st);
    delete s;
    return fail(SACD_ECUDA, "cudaStreamCreate failed");
  }
  try {
    s->prep = std::thread(prep_loop, s);
  } catch (...) {
    cudaStreamDestroy(s->prep_st);
    if (s->own_stream) cudaStreamDestroy(s->st);
    delete s;
    return fail(SACD_ENOMEM, "could not start the preparation thread");
  }
  *out = s;
  return SACD_OK;
}

sacd_status sacd_server_submit(sacd_server* s, const sacd_config* cfg, int32_t iters, int64_t* job_id) {
  if (!s || !cfg || !job_id) return fail(SACD_EINVAL, "null argument");
  if (s->poisoned) return fail(SACD_ESTATE, "server is poisoned by an earlier CUDA error");
  if (iters < 1) return fail(SACD_EINVAL, "iters must be >= 1");
  if (cfg->nmodes < 2 || cfg->nmodes > SACD_MAXN || !cfg->dims) return fail(SACD_EINVAL, "bad nmodes or dims");
  try {
    ServerJob* j = new ServerJob();
    j->id = s->next_id++;
    j->cfg = *cfg;
    j->dims.assign(cfg->dims, cfg->dims + cfg->nmodes);
    j->cfg.dims = j->dims.data();
    if (cfg->idx) {
      j->idx.assign(cfg->idx, cfg->idx + cfg->nmodes);
      j->cfg.idx = j->idx.data();
    }
    if (cfg->init) {
      j->init.assign(cfg->init, cfg->init + cfg->nmodes);
      j->cfg.init = j->init.data();
    }
    j->cfg.stream = s->st;
    j->iters = iters;
    j->est_bytes = estimate_bytes(&j->cfg);
    j->t_submit = now_s(s->t0);
    s->waiting.push_back(j);
    *job_id = j->id;
  } catch (const std::bad_alloc&) {
    return fail(SACD_ENOMEM, "host allocation failed");
  }
  return SACD_OK;
}

sacd_status sacd_server_step(sacd_server* s, int32_t* n_active, int32_t* n_waiting) {
  if (!s) return fail(SACD_EINVAL, "null server");
  if (s->poisoned) return fail(SACD_ESTATE, "server is poisoned by an earlier CUDA error");
  // ---- jobs whose contexts are ready join the plan; with nothing to iterate yet, wait for one
  auto activate = [&](bool wait) -> sacd_status {
    std::deque<ServerJob*> ready;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (wait) s->cv.wait(lk, [s] { return !s->created.empty(); });
      ready.swap(s->created);
    }
    for (ServerJob* j : ready) {
      --s->inflight;
      s->reserved -= j->est_bytes;
      if (j->create_status != SACD_OK) {
        j->status = j->create_status;
        finish_job(s, j);
        if (j->status == SACD_ECUDA) {
          s->poisoned = true;
          return fail(SACD_ECUDA, "job " + std::to_string(j->id) + ": " + j->error);
        }
        continue;
      }
      j->ctx->st = s->st;  // from now on the job's work (and its frees) follow the iterations
      j->bytes = j->ctx->device_bytes;
      s->used += j->bytes;
      s->active.push_back(j);
      s->plan_dirty = true;
    }
    return SACD_OK;
  };
  TRY(activate(false));
  // ---- admission, FIFO, within the budget, at most max_admit per step (creating a context takes
  // GPU time too; capping it keeps the admitted jobs iterating while a burst arrives): the
  // preparation thread creates the contexts while the iterations below run
  int admitted = 0;
  while (!s->waiting.empty() && (int)s->active.size() + s->inflight < s->max_active && admitted < s->max_admit) {
    ServerJob* j = s->waiting.front();
    const bool idle = s->active.empty() && s->inflight == 0;
    if (!idle && s->used + s->reserved + j->est_bytes > s->budget) break;
    if (j->est_bytes > s->budget) {  // can never fit
      s->waiting.pop_front();
      j->status = SACD_ENOMEM;
      j->error = "job needs more device memory than the whole budget";
      finish_job(s, j);
      continue;
    }
    s->waiting.pop_front();
    j->t_admit = now_s(s->t0);
    ++admitted;
    ++s->inflight;
    s->reserved += j->est_bytes;
    s->peak_used = std::max(s->peak_used, s->used + s->reserved);
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->to_create.push_back(j);
    }
    s->cv.notify_all();
  }
  if (s->active.empty() && s->inflight > 0) TRY(activate(true));
  // ---- one outer iteration of every admitted job
  if (!s->active.empty()) {
    if (s->plan_dirty) {
      s->plan.release();
      std::vector<sacd_ctx*> ctxs;
      for (ServerJob* j : s->active) ctxs.push_back(j->ctx);
      const sacd_status st = s->plan.build(ctxs, s->st);
      if (st != SACD_OK) {
        s->poisoned = true;
        return st;
      }
      s->plan_dirty = false;
    }
    s->plan.enqueue_iteration(s->st);
    s->steps++;
    {
      unsigned int h_err = 0;
      cudaError_t e = cudaMemcpyAsync(&h_err, &s->plan.d_bar->err, sizeof(h_err), cudaMemcpyDeviceToHost, s->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->st);
      if (e != cudaSuccess) {
        s->poisoned = true;
        return fail(SACD_ECUDA, std::string("server step: ") + cudaGetErrorString(e));
      }
      if (h_err) {
        s->poisoned = true;
        return fail(SACD_ETIMEOUT, "a bounded wait of the select/update kernel gave up (grid barrier)");
      }
    }
    std::vector<ServerJob*> still;
    for (ServerJob* j : s->active) {
      j->done_iters++;
      j->ctx->last_mode = j->ctx->N - 1;
      j->ctx->mlast_valid = true;
      j->ctx->mpre = false;
      if (j->done_iters < j->iters) {
        still.push_back(j);
        continue;
      }
      sacd_status st = sacd_fit(j->ctx, &j->objective, &j->fit);
      if (st == SACD_OK && !(std::isfinite(j->objective) && std::isfinite(j->fit))) {
        // the job's arithmetic left the finite range: report it as a failed job, keep serving
        j->status = SACD_ESTATE;
        j->error = "objective is not finite: the factors left the FP32 range";
        finish_job(s, j);
        s->plan_dirty = true;
        continue;
      }
      if (st == SACD_OK) {
        j->factors.resize(j->ctx->N);
        for (int n = 0; n < j->ctx->N && st == SACD_OK; ++n) {
          j->factors[n].resize((size_t)j->ctx->m[n].I * j->ctx->R);
          st = sacd_get_factor(j->ctx, n, j->factors[n].data());
        }
      }
      if (st != SACD_OK) {
        s->poisoned = true;
        j->status = st;
        j->error = g_err;
        finish_job(s, j);
        return fail(st, "job " + std::to_string(j->id) + ": " + j->error);
      }
      finish_job(s, j);
      s->plan_dirty = true;
    }
    s->active.swap(still);
    const cudaError_t e = cudaStreamSynchronize(s->st);
    if (e != cudaSuccess) {
      s->poisoned = true;
      return fail(SACD_ECUDA, std::string("server step: ") + cudaGetErrorString(e));
    }
  }
  if (n_active) *n_active = (int32_t)s->active.size() + s->inflight;
  if (n_waiting) *n_waiting = (int32_t)s->waiting.size();
  return SACD_OK;
}

sacd_status sacd_server_results(sacd_server* s, sacd_job_result* out, int32_t cap, int32_t* n) {
  if (!s || !n) return fail(SACD_EINVAL, "null argument");
  int32_t k = 0;
  while (!s->finished.empty() && k < cap) {
    ServerJob* j = s->finished.front();
    s->finished.pop_front();
    sacd_job_result& r = out[k++];
    memset(&r, 0, sizeof(r));
    r.job_id = j->id;
    r.status = j->status;
    r.iters = j->done_iters;
    r.objective = j->objective;
    r.fit = j->fit;
    r.t_submit = j->t_submit;
    r.t_admit = j->t_admit;
    r.t_done = j->t_done;
    r.device_bytes = j->bytes;
    strncpy(r.error, j->error.c_str(), sizeof(r.error) - 1);
    s->kept[j->id] = j;
  }
  *n = k;
  return SACD_OK;
}

sacd_status sacd_server_get_factor(sacd_server* s, int64_t job_id, int32_t mode, float* host_out) {
  if (!s || !host_out) return fail(SACD_EINVAL, "null argument");
  auto it = s->kept.find(job_id);
  if (it == s->kept.end()) return fail(SACD_EINVAL, "unknown job (not finished, not drained, or released)");
  ServerJob* j = it->second;
  if (j->status != SACD_OK) return fail(SACD_ESTATE, "job failed: " + j->error);
  if (mode < 0 || mode >= (int)j->factors.size()) return fail(SACD_EINVAL, "mode out of range");
  memcpy(host_out, j->factors[mode].data(), j->factors[mode].size() * sizeof(float));
  return SACD_OK;
}

sacd_status sacd_server_release(sacd_server* s, int64_t job_id) {
  if (!s) return fail(SACD_EINVAL, "null server");
  auto it = s->kept.find(job_id);
  if (it == s->kept.end()) return fail(SACD_EINVAL, "unknown job");
  delete it->second;
  s->kept.erase(it);
  return SACD_OK;
}

sacd_status sacd_server_stats(sacd_server* s, sacd_server_stats_t* out) {
  if (!s || !out) return fail(SACD_EINVAL, "null argument");
  out->active = (int32_t)s->active.size() + s->inflight;
  out->waiting = (int32_t)s->waiting.size();
  out->finished = (int32_t)s->finished.size();
  out->used_bytes = s->used;
  out->peak_bytes = s->peak_used;
  out->budget_bytes = s->budget;
  out->steps = s->steps;
  out->creating = s->inflight;
  return SACD_OK;
}

void sacd_server_destroy(sacd_server* s) {
  if (!s) return;
  if (s->prep.joinable()) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->stop = true;
    }
    s->cv.notify_all();
    s->prep.join();  // returns after the context it may be creating is done
  }
  for (ServerJob* j : s->to_create) delete j;
  for (ServerJob* j : s->created) {
    if (j->ctx) sacd_destroy(j->ctx);
    delete j;
  }
  if (s->prep_st) cudaStreamDestroy(s->prep_st);
  if (s->st) cudaStreamSynchronize(s->st);
  s->plan.release();
  for (ServerJob* j : s->active) {
    if (j->ctx) sacd_destroy(j->ctx);
    delete j;
  }
  for (ServerJob* j : s->waiting) delete j;
  for (ServerJob* j : s->finished) delete j;
  for (auto& kv : s->kept) delete kv.second;
  if (s->own_stream && s->st) cudaStreamDestroy(s->st);
  cudaGetLastError();
  delete s;
}

}  // extern "C"
