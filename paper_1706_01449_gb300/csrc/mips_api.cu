// The C ABI of libmips (declared in include/mips.h): argument checks, the
// index object, its workspace arena, and the dispatch of each call to its
// kernels.  No C++ exception crosses the boundary.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "internal.h"
#include "tc_topk.h"

using namespace mips;

namespace {

thread_local std::string g_err;

mips_status fail(mips_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

mips_status cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation)
    return fail(MIPS_ERR_NOMEM, "%s: %s", what, cudaGetErrorString(e));
  return fail(MIPS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define MIPS_CUDA(call)                                  \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

// Bump allocator over one device buffer; grown (stream-ordered) when a call
// needs more than it holds.
struct Arena {
  char* base = nullptr;
  size_t cap = 0;
  size_t used = 0;
  uint64_t gen = 0;  // bumped on every reallocation (captured graphs hold the old base)

  void reset() { used = 0; }
  size_t take(size_t bytes) {
    size_t off = (used + 255) & ~size_t(255);
    used = off + bytes;
    return off;
  }
  cudaError_t ensure(size_t bytes, cudaStream_t s) {
    if (bytes <= cap) return cudaSuccess;
    if (base) {
      cudaError_t e = cudaFreeAsync(base, s);
      if (e != cudaSuccess) return e;
      base = nullptr;
      cap = 0;
    }
    size_t want = bytes + bytes / 8;
    cudaError_t e = cudaMallocAsync((void**)&base, want, s);
    if (e != cudaSuccess) return e;
    cap = want;
    ++gen;
    return cudaSuccess;
  }
  template <typename T>
  T* at(size_t off) const {
    return reinterpret_cast<T*>(base + off);
  }
};

enum Stage { ST_PREP = 0, ST_SCORE, ST_RESCORE, ST_KMEANS, ST_BOUNDS, ST_SORT, ST_WALK, kStages };

}  // namespace

void mips::set_last_error_message(const char* msg) { g_err = msg; }

struct mips_index_s {
  int device = 0;
  int f = 0;
  int64_t n_items = 0;
  int clusters = 0;
  mips_options opt{};
  // centroids fitted by mips_fit_clusters ([fit_C][f], owned; 0 = none)
  float* fit_cent = nullptr;
  int fit_C = 0;
  int64_t fit_cap = 0;   // floats allocated at fit_cent
  uint64_t fit_gen = 0;  // bumped by every fit or clear (captured graphs hold the old state)
  // item data, in the index's item order ("sorted position")
  float* items = nullptr;      // FP32 master rows [n_items][f]
  int32_t* perm = nullptr;     // sorted position -> item id
  float* item_nrm = nullptr;   // upper bounds of ||i|| [n_items]
  // BF16 operand rows with bound columns
  int fp = 0;
  void* items_bf16 = nullptr;  // [n_items_pad][fp] tensor-core operand rows (BF16 or E4M3)
  float2* item_aux = nullptr;  // {nhat_i, alpha_i}
  int esize = 2;               // bytes per operand element: 2 BF16, 1 FP8 E4M3
  float* item_scale = nullptr;  // FP8: the items' scale s_I (one device float)
  int64_t n_items_pad = 0;
  int num_sms = 0;
  int max_smem = 0;
  // per-call state
  Arena ws;
  Arena ws_sel;  // the selector's own buffers (sample, rest, their outputs)
  int* err_dev = nullptr;
  DevStats* stats_dev = nullptr;
  cudaEvent_t done = nullptr;   // end of the last call (orders calls on different streams)
  bool has_done = false;
  cudaStream_t last_stream = nullptr;
  cudaStream_t copy_stream = nullptr;  // host-buffer calls: copies beside the compute (created on first use)
  int64_t last_users = 0;
  int last_dtype = 0;
  int last_clusters = 0;
  // views into the workspace of the last Maximus call (mips_get_buffer)
  struct {
    const void* assign = nullptr;
    const void* cent = nullptr;
    const void* cosb = nullptr;
    const void* bounds = nullptr;
    const void* lists = nullptr;
    const void* visited = nullptr;
    const void* user_perm = nullptr;
    int64_t n_users = 0;
    int C = 0;
  } mx;
  // per-stage timing: ev[0] = call start, ev[1 + stage] = end of stage
  cudaEvent_t ev[kStages + 1] = {};
  // around the launches of the call's dominant kernel (the fused score +
  // select, or the two passes of the Maximus walk): start/end pairs
  cudaEvent_t kev[4] = {};
  int n_kev = 0;
  bool stage_ran[kStages] = {};
  int last_stage = -1;
  int order[kStages] = {};  // stages in the order they ran in the last call
  int n_order = 0;
  int launches = 0;
  // captured calls (mips_topk_graph): replayed while the arguments and the
  // workspace are the same
  bool capturing = false;
  bool shares_items = false;  // a worker of another index: item arrays not owned
  struct Graph {
    int method = 0;
    const float* users = nullptr;
    int64_t n_users = 0;
    int K = 0;
    int32_t* out_idx = nullptr;
    double* out_score = nullptr;
    uint64_t ws_gen = 0;
    // index settings the capture baked in
    int cfg_clusters = 0, cfg_block = 0;
    uint64_t cfg_fit = 0;
    cudaGraphExec_t exec = nullptr;
    // host bookkeeping of the captured call, restored on replay
    bool stage_ran[kStages] = {};
    int order[kStages] = {};
    int n_order = 0, last_stage = -1, launches = 0, clusters = 0, dtype = 0, n_kev = 0;
  };
  std::vector<Graph> graphs;
};

namespace {

mips_status check_device(mips_index_t idx) {
  int dev = -1;
  MIPS_CUDA(cudaGetDevice(&dev));
  if (dev != idx->device) return fail(MIPS_ERR_ARG, "index lives on device %d, current device is %d", idx->device, dev);
  return MIPS_OK;
}

// Stage events; inside a stream capture they become event-record nodes of
// the graph, so a replay times its stages too.
cudaError_t record(mips_index_t idx, cudaEvent_t ev, cudaStream_t s) {
  return idx->capturing ? cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal) : cudaEventRecord(ev, s);
}

mips_status begin_call(mips_index_t idx, cudaStream_t s) {
  // (a captured call is ordered after the previous one at launch time)
  if (idx->has_done && !idx->capturing) MIPS_CUDA(cudaStreamWaitEvent(s, idx->done, 0));
  MIPS_CUDA(cudaMemsetAsync(idx->stats_dev, 0, sizeof(DevStats), s));
  for (int i = 0; i < kStages; ++i) idx->stage_ran[i] = false;
  idx->last_stage = -1;
  idx->n_order = 0;
  idx->launches = 0;
  idx->n_kev = 0;
  MIPS_CUDA(record(idx, idx->ev[0], s));
  return MIPS_OK;
}

// Set by mips_test_expire_next_wait, taken by the next tensor-core launch.
std::atomic<long long> g_test_expire_ns{0};

// Start or end mark of one launch of the dominant kernel (the first four
// marks of a call are kept).
mips_status mark_kernel(mips_index_t idx, cudaStream_t s) {
  if (idx->n_kev < 4) MIPS_CUDA(record(idx, idx->kev[idx->n_kev], s));
  if (idx->n_kev < 4) ++idx->n_kev;
  return MIPS_OK;
}

// Mark the end of a stage (stages run in enum order within one call).
mips_status end_stage(mips_index_t idx, Stage st, cudaStream_t s) {
  MIPS_CUDA(record(idx, idx->ev[1 + st], s));
  if (!idx->stage_ran[st] && idx->n_order < kStages) idx->order[idx->n_order++] = st;
  idx->stage_ran[st] = true;
  idx->last_stage = st;
  return MIPS_OK;
}

mips_status end_call(mips_index_t idx, cudaStream_t s) {
  MIPS_CUDA(cudaEventRecord(idx->done, s));
  idx->has_done = true;
  idx->last_stream = s;
  return MIPS_OK;
}

// Candidate capacity of the FP32 kernels' single list per user over n
// items (no seeding): the record count K (1 + ln(n / K)) with room to spare.
int cap_for(int K, int64_t n) {
  const double r = n > K ? std::log((double)n / K) : 0.0;
  return std::max(4 * K + 96, (int)std::min<int64_t>((int64_t)std::ceil(K * (2.0 + r)) + 96, n + 96));
}

// Candidate capacity of a tensor-core sub-list scanning n items.  With the
// register top-K (K <= 16) the first tile seeds the threshold and the two
// halves of a user merge their seeds: 2K + 64 is ample.  A heap-held top-K
// (K > 16) or an item chunk seeds from few items, and its threshold rises
// like the K-th largest of a stream: about K (1 + ln(n / K)) values pass,
// the count of K-th-largest records (plus the band between lower and upper
// bounds); the capacity is that with K + 64 to spare.
int tc_cap(int K, int64_t n, bool chunked) {
  const int base = K <= kRegTopK ? 2 * K + 64 : 4 * K + 64;
  if (K <= kRegTopK && !chunked) return base;
  const double r = n > K ? std::log((double)n / K) : 0.0;
  const int grow = (int)std::ceil(K * (2.0 + r)) + 64;
  return std::max(base, (int)std::min<int64_t>(grow, n + 64));
}

// Candidate passes on the tensor cores: BF16 (kind::f16) or FP8 E4M3
// (kind::f8f6f4) operand rows.
bool tc_dtype(int d) { return d == MIPS_BF16 || d == MIPS_FP8_E4M3; }

// The users' operand rows for the index's tensor-core dtype; FP8 also
// writes each user's scale (user_scale) and points the plan at the scales.
void quant_users(mips_index_t idx, const float* users, int64_t n_users, void* rows, float2* uaux, float* user_scale,
                 TcParams& p, cudaStream_t s) {
  if (idx->esize == 1) {
    launch_quant_fp8(users, n_users, idx->f, idx->fp, 0, nullptr, rows, n_users, uaux, user_scale, idx->err_dev, s);
    p.user_scale = user_scale;
    p.item_scale = idx->item_scale;
  } else {
    launch_quant_bf16(users, n_users, idx->f, idx->fp, 0, rows, n_users, uaux, idx->err_dev, s);
  }
}

// Blocked multiply (Sec. II-C) over the index's items with fused select,
// then the exact rescore.
// size_only: lay out the workspace, store the bytes it needs there and
// return before any device work (no pointer argument is used).
mips_status run_bmm(mips_index_t idx, const float* users, int64_t n_users, int K, int32_t* out_idx,
                    double* out_score, cudaStream_t s, size_t* size_only = nullptr) {
  const int f = idx->f;
  if (!size_only) idx->mx.C = 0;  // the workspace is reused: earlier Maximus views are gone
  // candidate pass: tcgen05 BF16 when the index has BF16 operands and the
  // tiling fits shared memory for this K, else the FP32 CUDA-core kernel
  TcParams p{};
  p.n_users = n_users;
  p.n_items = idx->n_items;
  p.f = f;
  p.fp = idx->fp;
  p.esize = idx->esize;
  p.K = K;
  const bool use_tc = tc_dtype(idx->opt.dtype) && tc_plan(p, idx->max_smem);
  // Few user tiles would leave SMs idle: the item tiles are then split into
  // nch chunks, (user tile, chunk) pairs become the persistent grid's work
  // items, each with its own two sub-lists per user; the rescore takes the
  // union.  At least 8 item tiles per chunk, at most 16 chunks.
  const int64_t n_ut = (n_users + tc_users_per_tile() - 1) / tc_users_per_tile();
  const int n_it = (int)((idx->n_items + tc_items_per_tile() - 1) / tc_items_per_tile());
  int nch = 1;
  if (use_tc && n_ut * 2 <= idx->num_sms) {
    nch = (int)((idx->num_sms + n_ut - 1) / n_ut);
    nch = std::min(nch, std::min(16, n_it / 8));
    if (nch < 1) nch = 1;
  }
  const int tpc = (n_it + nch - 1) / nch;
  nch = (n_it + tpc - 1) / tpc;
  // BF16: two select threads per user (and chunk), each with its own sub-list
  const int lists = use_tc ? 2 * nch : 1;
  // (FP8's bound band is about 16 times BF16's: 2^-4 against 2^-8 per entry; its lists are 4 times longer)
  const int cap = lists == 1 ? cap_for(K, idx->n_items)
                             : (idx->esize == 1 ? 4 : 1) * tc_cap(K, (int64_t)tpc * tc_items_per_tile() / 2, nch > 1);
  const int64_t nl = n_users * lists;
  idx->ws.reset();
  size_t o_tau = idx->ws.take(sizeof(float) * nl);
  size_t o_n = idx->ws.take(sizeof(int) * nl);
  size_t o_pos = idx->ws.take(sizeof(int32_t) * nl * cap);
  size_t o_ub = idx->ws.take(sizeof(float) * nl * cap);
  size_t o_topl = idx->ws.take(sizeof(float) * nl * K);
  size_t o_ovf = idx->ws.take(sizeof(int32_t) * n_users);
  size_t o_ovfc = idx->ws.take(sizeof(int));
  size_t o_work = idx->ws.take(sizeof(uint32_t) * nl * cap);
  size_t o_workc = idx->ws.take(sizeof(int));
  size_t o_sc = idx->ws.take(sizeof(double) * nl * cap);
  size_t o_wid = idx->ws.take(sizeof(int32_t) * nl * cap), o_wnrm = idx->ws.take(sizeof(float) * nl * cap);
  size_t o_uwork = idx->ws.take(sizeof(int) * 2 * n_users);
  size_t o_tauf = idx->ws.take(sizeof(float) * 2 * n_users);
  size_t o_ub16 = 0, o_uaux = 0, o_us = 0, o_cw = 0, o_cnw = 0, o_crow = 0, o_cpos = 0, o_ctau = 0, o_heap = 0;
  if (use_tc && p.heap_global) o_heap = idx->ws.take(sizeof(float) * idx->num_sms * K * 256);
  if (use_tc) {
    o_ub16 = idx->ws.take((size_t)idx->esize * n_users * idx->fp);
    o_uaux = idx->ws.take(sizeof(float2) * n_users);
    if (idx->esize == 1) o_us = idx->ws.take(sizeof(float) * n_users);
  }
  if (nch > 1) {
    o_cw = idx->ws.take(sizeof(int) * 5 * n_ut * nch);
    o_cnw = idx->ws.take(16);
    o_crow = idx->ws.take(sizeof(int32_t) * n_ut * tc_users_per_tile());
    o_cpos = idx->ws.take(sizeof(int32_t) * idx->n_items_pad);
    o_ctau = idx->ws.take(sizeof(unsigned) * n_users);
  }
  if (size_only) {
    *size_only = idx->ws.used;
    idx->ws.reset();
    return MIPS_OK;
  }
  MIPS_CUDA(idx->ws.ensure(idx->ws.used, s));
  SelectOut so{idx->ws.at<float>(o_tau), idx->ws.at<int>(o_n), idx->ws.at<int32_t>(o_pos),
               idx->ws.at<float>(o_ub), cap, lists,
               lists >= 2 ? idx->ws.at<float>(o_topl) : nullptr, 1,
               idx->ws.at<int32_t>(o_ovf), idx->ws.at<int>(o_ovfc), idx->ws.at<uint32_t>(o_work),
               idx->ws.at<int>(o_workc), idx->ws.at<double>(o_sc), idx->ws.at<float>(o_tauf)};
  so.w_id = idx->ws.at<int32_t>(o_wid);
  so.w_nrm = idx->ws.at<float>(o_wnrm);
  so.u_work = idx->ws.at<int>(o_uwork);
  mips_status st;
  if (!use_tc) {
    if ((st = mark_kernel(idx, s)) != MIPS_OK) return st;
    MIPS_CUDA(launch_fp32_score_select(users, n_users, f, idx->items, idx->item_nrm, idx->n_items, K, so,
                                       idx->stats_dev, idx->err_dev, s));
    if ((st = mark_kernel(idx, s)) != MIPS_OK) return st;
    idx->launches += 1;
    if ((st = end_stage(idx, ST_SCORE, s)) != MIPS_OK) return st;
  } else {
    void* ub16 = idx->ws.at<void>(o_ub16);
    float2* uaux = idx->ws.at<float2>(o_uaux);
    quant_users(idx, users, n_users, ub16, uaux, idx->esize == 1 ? idx->ws.at<float>(o_us) : nullptr, p, s);
    MIPS_CUDA(cudaGetLastError());
    idx->launches += 1;
    if ((st = end_stage(idx, ST_PREP, s)) != MIPS_OK) return st;
    // (the item maps depend on the call's plan: whole or half tiles per load)
    CUtensorMap map_users, map_users_tail, map_items, map_items_tail;
    if (!tc_make_maps(&map_users, &map_users_tail, ub16, n_users, p, tc_users_per_tile()) ||
        !tc_make_maps(&map_items, &map_items_tail, idx->items_bf16, idx->n_items_pad, p, tc_items_box(p)))
      return fail(MIPS_ERR_CUDA, "cuTensorMapEncodeTiled failed for the operands");
    int64_t n_work = n_ut;
    if (nch > 1) {
      int* cw = idx->ws.at<int>(o_cw);
      const int64_t nw = n_ut * nch;
      launch_bmm_chunks((int)n_ut, nch, tpc, n_it, n_users, idx->n_items_pad, cw, idx->ws.at<int>(o_cnw),
                        idx->ws.at<int32_t>(o_crow), idx->ws.at<int32_t>(o_cpos), s);
      idx->launches += 1;
      p.mode = 1;
      p.work = TcWork{cw, cw + nw, cw + 2 * nw, cw + 3 * nw, idx->ws.at<int>(o_cnw), idx->ws.at<int32_t>(o_crow),
                      idx->ws.at<int32_t>(o_cpos), cw + 4 * nw, 0, nullptr, idx->n_items};
      // the chunks of a user share their thresholds (zero bits = none yet)
      so.tau_glob = idx->ws.at<unsigned>(o_ctau);
      MIPS_CUDA(cudaMemsetAsync(so.tau_glob, 0, sizeof(unsigned) * n_users, s));
      n_work = nw;
    }
    const int grid = (int)(n_work < idx->num_sms ? n_work : idx->num_sms);
    if (p.heap_global) p.heap_mem = idx->ws.at<float>(o_heap);
    // counts start at 0: a launch that gives up on a bounded wait leaves
    // unfinished lists, which the rescore then reads as empty
    MIPS_CUDA(cudaMemsetAsync(so.n_cand, 0, sizeof(int) * nl, s));
    if (const long long t = g_test_expire_ns.exchange(0)) {
      p.wait_ns = (unsigned long long)t;
      p.test_withhold = 1;
    }
    if ((st = mark_kernel(idx, s)) != MIPS_OK) return st;
    MIPS_CUDA(launch_tc_score_select(&map_users, &map_users_tail, &map_items, &map_items_tail, p, so, uaux,
                                     idx->item_aux, idx->stats_dev,
                                     idx->err_dev, grid, s));
    if ((st = mark_kernel(idx, s)) != MIPS_OK) return st;
    idx->launches += 1;
    if ((st = end_stage(idx, ST_SCORE, s)) != MIPS_OK) return st;
  }
  MIPS_CUDA(launch_rescore(users, n_users, f, idx->items, idx->perm, idx->item_nrm, idx->n_items, K, so,
                           out_idx, out_score, idx->stats_dev, idx->err_dev, s));
  idx->launches += 4;  // collect, dot, select, overflow
  if ((st = end_stage(idx, ST_RESCORE, s)) != MIPS_OK) return st;
  idx->last_users = n_users;
  idx->last_dtype = use_tc ? idx->opt.dtype : MIPS_FP32;
  return MIPS_OK;
}

// C distinct user ids from a counter-based stream (SplitMix64 of seed and
// counter), Floyd's method: the k-means initial centroids.
// Parameters of a seeded affine permutation of [0, n): u -> (a u + b) mod n
// with a coprime to n (SplitMix64 draws).  The users whose image is below
// ns form a sample of exactly ns distinct users.
void affine_sample(int64_t n, uint64_t seed, uint64_t* a_out, uint64_t* b_out) {
  auto mix = [](uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  };
  uint64_t a = n > 1 ? 1 + mix(seed) % (uint64_t)(n - 1) : 1;
  while (std::gcd(a, (uint64_t)n) != 1) a = a % (uint64_t)(n - 1) + 1;
  *a_out = a;
  *b_out = n > 0 ? mix(seed ^ 1ull) % (uint64_t)n : 0;
}

// Maximus (Sec. III, Algorithm 1): k-means, theta_b + CBound, per-cluster
// sort and user grouping, grouped walk, exact rescore.
mips_status run_maximus(mips_index_t idx, const float* users, int64_t n_users, int K, int32_t* out_idx,
                        double* out_score, cudaStream_t s, size_t* size_only = nullptr) {
  const int f = idx->f;
  const int64_t nI = idx->n_items;
  // with fitted centroids only the clusters that receive users are kept
  const bool fitted = idx->fit_C > 0;
  const int C = (int)std::min<int64_t>(fitted ? idx->fit_C : idx->clusters, n_users);
  const int cap = cap_for(K, nI);
  const int64_t CI = (int64_t)C * nI;
  // walk on tcgen05 when the index has BF16 operands and the tiling fits
  TcParams p{};
  p.n_users = n_users;
  p.n_items = nI;
  p.f = f;
  p.fp = idx->fp;
  p.esize = idx->esize;
  p.K = K;
  // (TMA row coordinates of the per-cluster item copies are 32-bit)
  const bool use_tc = tc_dtype(idx->opt.dtype) && (int64_t)C * round_up(nI, 256) < (int64_t)INT32_MAX &&
                      round_up(n_users, 128) + 128ll * C < (int64_t)INT32_MAX && mx_tc_regroup_fits(C, nI) &&
                      tc_plan(p, idx->max_smem);
  Arena& ws = idx->ws;
  ws.reset();
  size_t o_ids = ws.take(sizeof(int64_t) * C), o_cent = ws.take(sizeof(float) * C * f), o_hn2 = ws.take(sizeof(float) * C);
  size_t o_bits = ws.take(sizeof(uint32_t) * ((n_users + 31) / 32));
  size_t o_assign = ws.take(sizeof(int32_t) * n_users), o_sums = ws.take(sizeof(unsigned long long) * C * f);
  size_t o_cnt = ws.take(sizeof(unsigned) * C), o_amax = ws.take(16), o_scale = ws.take(16);
  size_t o_cosb = ws.take(sizeof(uint32_t) * C), o_cosbf = ws.take(sizeof(float) * C);
  size_t o_keys = ws.take(sizeof(uint32_t) * CI), o_vals = ws.take(sizeof(int32_t) * CI);
  size_t o_keys2 = ws.take(sizeof(uint32_t) * CI), o_vals2 = ws.take(sizeof(int32_t) * CI);
  const int C_fit = fitted ? idx->fit_C : 0;
  size_t o_fhn2 = ws.take(sizeof(float) * C_fit), o_used = ws.take(sizeof(int) * C_fit),
         o_remap = ws.take(sizeof(int) * C_fit);
  // k-means assignment on tcgen05 (BF16 operands) when every centroid stays
  // resident in shared memory
  const int C_km = fitted ? C_fit : C;
  const bool km_tc = idx->opt.dtype != MIPS_FP32 && km_tc_fits(f, C_km, idx->max_smem);
  const int fk = km_tc_row_len(f);
  const size_t o_ukm = km_tc ? ws.take(sizeof(uint16_t) * n_users * fk) : 0;
  const size_t o_ckm = km_tc ? ws.take(sizeof(uint16_t) * (size_t)C_km * fk) : 0;
  const int64_t n_rows_max = round_up(n_users, 128) + 128ll * C;  // A rows of the tensor-core walk
  const int64_t max_work = n_rows_max / 128;
  size_t tmp_bytes = radix_sort_temp_bytes(nI, C);
  if (radix_sort_temp_bytes(n_users, 1) > tmp_bytes) tmp_bytes = radix_sort_temp_bytes(n_users, 1);
  if (radix_sort_temp_bytes(max_work, 1) > tmp_bytes) tmp_bytes = radix_sort_temp_bytes(max_work, 1);
  size_t o_tmp = ws.take(tmp_bytes);
  size_t o_bounds = ws.take(sizeof(float) * CI);
  size_t o_uk = ws.take(sizeof(uint32_t) * n_users), o_ui = ws.take(sizeof(int32_t) * n_users);
  size_t o_uk2 = ws.take(sizeof(uint32_t) * n_users), o_ui2 = ws.take(sizeof(int32_t) * n_users);
  size_t o_ccnt = ws.take(sizeof(int) * C), o_off = ws.take(sizeof(int) * (C + 1)), o_toff = ws.take(sizeof(int) * (C + 1));
  size_t o_wc = ws.take(16), o_vis = ws.take(sizeof(int32_t) * n_users);
  size_t o_tau = ws.take(sizeof(float) * n_users), o_n = ws.take(sizeof(int) * n_users);
  const int64_t cap1 = use_tc ? 0 : cap;  // the FP32 walk's single-list candidate buffers
  size_t o_pos = ws.take(sizeof(int32_t) * n_users * cap1), o_ub = ws.take(sizeof(float) * n_users * cap1);
  size_t o_ovf = ws.take(sizeof(int32_t) * n_users), o_ovfc = ws.take(sizeof(int));
  size_t o_work = ws.take(sizeof(uint32_t) * n_users * cap1), o_workc = ws.take(sizeof(int));
  size_t o_sc = ws.take(sizeof(double) * n_users * cap1), o_tauf = ws.take(sizeof(float) * 2 * n_users);
  size_t o_wid = ws.take(sizeof(int32_t) * n_users * cap1), o_wnrm = ws.take(sizeof(float) * n_users * cap1);
  size_t o_uwork = ws.take(sizeof(int) * 2 * n_users);
  // tensor-core walk buffers: BF16 user rows grouped by cluster (each
  // cluster padded to whole 128-row tiles), per-cluster BF16 item copies in
  // bound order, two work lists, two-list select state
  const int fp = idx->fp;
  const int n_it = (int)((nI + 255) / 256);
  const int blk = idx->opt.block_items > 0 ? idx->opt.block_items : 4096;
  const int t1 = (int)((blk + 255) / 256) < n_it ? (int)((blk + 255) / 256) : n_it;
  const int64_t n_pad = round_up(nI, 256);
  const int cap2 = (idx->esize == 1 ? 4 : 1) * tc_cap(K, (nI + 1) / 2, false);
  const int64_t nl = n_users * 2;
  size_t o_u16 = 0, o_uaux = 0, o_rowu = 0, o_urow = 0, o_padoff = 0, o_arows = 0, o_brows = 0, o_auxc = 0,
         o_posc = 0, o_w1 = 0, o_w2 = 0, o_nw = 0, o_wend = 0, o_tau2 = 0, o_n2 = 0, o_pos2 = 0, o_ub2 = 0,
         o_topl = 0, o_work2 = 0, o_sc2 = 0, o_ustop = 0, o_wk0 = 0, o_wk1 = 0, o_wv0 = 0, o_wv1 = 0, o_clend = 0,
         o_heapm = 0, o_wid2 = 0, o_wnrm2 = 0;
  size_t o_us = 0;
  if (use_tc) {
    const size_t es = (size_t)idx->esize;
    o_u16 = ws.take(es * n_users * fp);
    o_uaux = ws.take(sizeof(float2) * n_users);
    if (es == 1) o_us = ws.take(sizeof(float) * n_users);
    o_rowu = ws.take(sizeof(int32_t) * n_rows_max);
    o_urow = ws.take(sizeof(int32_t) * n_users);
    o_padoff = ws.take(sizeof(int) * (C + 1));
    o_arows = ws.take(es * n_rows_max * fp);
    o_brows = ws.take(es * C * n_pad * fp);
    o_auxc = ws.take(sizeof(float2) * C * n_pad);
    o_posc = ws.take(sizeof(int32_t) * C * n_pad);
    o_w1 = ws.take(sizeof(int) * 4 * max_work);
    o_w2 = ws.take(sizeof(int) * 4 * max_work);
    o_nw = ws.take(16);
    o_wend = ws.take(sizeof(int) * max_work);
    o_tau2 = ws.take(sizeof(float) * nl);
    o_n2 = ws.take(sizeof(int) * nl);
    o_pos2 = ws.take(sizeof(int32_t) * nl * cap2);
    o_ub2 = ws.take(sizeof(float) * nl * cap2);
    o_topl = ws.take(sizeof(float) * nl * K);
    o_work2 = ws.take(sizeof(uint32_t) * nl * cap2);
    o_sc2 = ws.take(sizeof(double) * nl * cap2);
    o_wid2 = ws.take(sizeof(int32_t) * nl * cap2);
    o_wnrm2 = ws.take(sizeof(float) * nl * cap2);
    o_ustop = ws.take(sizeof(int32_t) * n_users);
    o_clend = ws.take(sizeof(int) * C);
    if (p.heap_global) o_heapm = ws.take(sizeof(float) * idx->num_sms * K * 256);
    o_wk0 = ws.take(sizeof(uint32_t) * max_work);
    o_wk1 = ws.take(sizeof(uint32_t) * max_work);
    o_wv0 = ws.take(sizeof(int32_t) * max_work);
    o_wv1 = ws.take(sizeof(int32_t) * max_work);
  }
  if (size_only) {  // (run_bmm's sizing mode)
    *size_only = ws.used;
    ws.reset();
    return MIPS_OK;
  }
  MIPS_CUDA(ws.ensure(ws.used, s));
  KmTc kt;
  if (km_tc) {
    kt.users_km = ws.at<uint16_t>(o_ukm);
    kt.cent_km = ws.at<uint16_t>(o_ckm);
    kt.err = idx->err_dev;
    kt.max_smem = idx->max_smem;
  }

  if (fitted) {
    // dynamic users (Sec. III-E): one assignment step to the fitted centroids
    MIPS_CUDA(maximus_assign_fitted(users, n_users, f, idx->fit_cent, C_fit, ws.at<float>(o_fhn2),
                                    ws.at<int32_t>(o_assign), ws.at<int>(o_used), ws.at<int>(o_remap),
                                    ws.at<float>(o_cent), C, kt, s, &idx->launches));
  } else {
    // k-means initial centroids: a seeded draw of C distinct users (on the
    // device, so that a captured call holds no host data)
    MIPS_CUDA(draw_init_ids(n_users, C, idx->opt.seed, ws.at<uint32_t>(o_bits), ws.at<int64_t>(o_ids), s));
    idx->launches += 1;
    MIPS_CUDA(maximus_kmeans(users, n_users, f, C, idx->opt.kmeans_iters, ws.at<int64_t>(o_ids),
                             ws.at<float>(o_cent), ws.at<float>(o_hn2), ws.at<int32_t>(o_assign),
                             ws.at<unsigned long long>(o_sums), ws.at<unsigned>(o_cnt), ws.at<uint32_t>(o_amax),
                             ws.at<float>(o_scale), idx->opt.kmeans_spherical != 0, kt, s, &idx->launches));
  }
  mips_status st;
  if ((st = end_stage(idx, ST_KMEANS, s)) != MIPS_OK) return st;
  MIPS_CUDA(maximus_bounds(users, n_users, f, ws.at<int32_t>(o_assign), ws.at<float>(o_cent), C, idx->items,
                           idx->item_nrm, nI, ws.at<uint32_t>(o_cosb), ws.at<uint32_t>(o_keys), ws.at<int32_t>(o_vals),
                           ws.at<float>(o_cosbf), s, &idx->launches));
  if ((st = end_stage(idx, ST_BOUNDS, s)) != MIPS_OK) return st;
  // per-cluster lists: items by CBound (its key's leading kListKeyBits bits), descending, stable
  uint32_t* keys = ws.at<uint32_t>(o_keys);
  int32_t* vals = ws.at<int32_t>(o_vals);
  uint32_t* keys2 = ws.at<uint32_t>(o_keys2);
  int32_t* vals2 = ws.at<int32_t>(o_vals2);
  MIPS_CUDA(radix_sort_pairs(keys, vals, keys2, vals2, nI, C, 32 - kListKeyBits, 32, ws.at<uint32_t>(o_tmp), s,
                             &idx->launches));
  MIPS_CUDA(maximus_keys_to_bounds(keys, CI, ws.at<float>(o_bounds), s));
  idx->launches += 1;
  int32_t* user_perm = nullptr;
  MIPS_CUDA(maximus_group(ws.at<int32_t>(o_assign), n_users, C, ws.at<uint32_t>(o_uk), ws.at<int32_t>(o_ui),
                          ws.at<uint32_t>(o_uk2), ws.at<int32_t>(o_ui2), ws.at<uint32_t>(o_tmp), ws.at<int>(o_ccnt),
                          ws.at<int>(o_off), ws.at<int>(o_toff), &user_perm, s, &idx->launches));
  if ((st = end_stage(idx, ST_SORT, s)) != MIPS_OK) return st;
  if (!use_tc) {
    // FP32 walk on CUDA cores, one candidate list per user
    SelectOut so{ws.at<float>(o_tau), ws.at<int>(o_n), ws.at<int32_t>(o_pos), ws.at<float>(o_ub), cap, 1, nullptr, 0,
                 ws.at<int32_t>(o_ovf), ws.at<int>(o_ovfc), ws.at<uint32_t>(o_work), ws.at<int>(o_workc),
                 ws.at<double>(o_sc), ws.at<float>(o_tauf)};
    so.w_id = ws.at<int32_t>(o_wid);
    so.w_nrm = ws.at<float>(o_wnrm);
    so.u_work = ws.at<int>(o_uwork);
    if ((st = mark_kernel(idx, s)) != MIPS_OK) return st;
    MIPS_CUDA(maximus_walk(users, f, idx->items, idx->item_nrm, nI, vals, ws.at<float>(o_bounds), user_perm,
                           ws.at<int>(o_off), ws.at<int>(o_toff), C, K, so, ws.at<int32_t>(o_vis), ws.at<int>(o_wc),
                           idx->stats_dev, idx->err_dev, idx->num_sms, s));
    if ((st = mark_kernel(idx, s)) != MIPS_OK) return st;
    idx->launches += 1;
    if ((st = end_stage(idx, ST_WALK, s)) != MIPS_OK) return st;
    MIPS_CUDA(launch_rescore(users, n_users, f, idx->items, idx->perm, idx->item_nrm, nI, K, so, out_idx, out_score,
                             idx->stats_dev, idx->err_dev, s));
    idx->launches += 4;
  } else {
    // tensor-core walk: cluster-ordered BF16 user rows, per-cluster BF16
    // item copies in bound order; pass 1 = the first block of every list
    // (the paper's item blocking), pass 2 = the rest each user tile needs
    MxTc m;
    m.C = C;
    m.fp = fp;
    m.esize = idx->esize;
    m.t1 = t1;
    m.n_it = n_it;
    m.n_users = n_users;
    m.n_items = nI;
    m.n_pad = n_pad;
    m.n_rows_max = n_rows_max;
    m.max_work = max_work;
    m.counts = ws.at<int>(o_ccnt);
    m.offsets = ws.at<int>(o_off);
    m.pad_off = ws.at<int>(o_padoff);
    m.row_user = ws.at<int32_t>(o_rowu);
    m.user_row = ws.at<int32_t>(o_urow);
    m.users_bf16 = ws.at<void>(o_u16);
    m.a_rows = ws.at<void>(o_arows);
    m.b_rows = ws.at<void>(o_brows);
    m.aux_c = ws.at<float2>(o_auxc);
    m.pos_c = ws.at<int32_t>(o_posc);
    m.w1 = ws.at<int>(o_w1);
    m.w2 = ws.at<int>(o_w2);
    m.n_work = ws.at<int>(o_nw);
    m.work_end = ws.at<int>(o_wend);
    m.ustop = ws.at<int32_t>(o_ustop);
    m.cl_end = ws.at<int>(o_clend);
    m.ukeys[0] = ws.at<uint32_t>(o_uk);  // the user-group sort is done with these
    m.ukeys[1] = ws.at<uint32_t>(o_uk2);
    m.uvals[0] = ws.at<int32_t>(o_ui);
    m.uvals[1] = ws.at<int32_t>(o_ui2);
    m.wkeys[0] = ws.at<uint32_t>(o_wk0);
    m.wkeys[1] = ws.at<uint32_t>(o_wk1);
    m.wvals[0] = ws.at<int32_t>(o_wv0);
    m.wvals[1] = ws.at<int32_t>(o_wv1);
    m.temp = ws.at<uint32_t>(o_tmp);
    quant_users(idx, users, n_users, ws.at<void>(o_u16), ws.at<float2>(o_uaux),
                idx->esize == 1 ? ws.at<float>(o_us) : nullptr, p, s);
    idx->launches += 1;
    MIPS_CUDA(mx_tc_prepare(m, user_perm, idx->items_bf16, idx->item_aux, vals, s, &idx->launches));
    if ((st = end_stage(idx, ST_PREP, s)) != MIPS_OK) return st;
    CUtensorMap map_a, map_at, map_b, map_bt;
    if (!tc_make_maps(&map_a, &map_at, m.a_rows, n_rows_max, p, tc_users_per_tile()) ||
        !tc_make_maps(&map_b, &map_bt, m.b_rows, C * n_pad, p, tc_items_box(p)))
      return fail(MIPS_ERR_CUDA, "cuTensorMapEncodeTiled failed for the Maximus operands");
    SelectOut so{ws.at<float>(o_tau2), ws.at<int>(o_n2), ws.at<int32_t>(o_pos2), ws.at<float>(o_ub2), cap2, 2,
                 ws.at<float>(o_topl), 1, ws.at<int32_t>(o_ovf), ws.at<int>(o_ovfc),
                 ws.at<uint32_t>(o_work2), ws.at<int>(o_workc), ws.at<double>(o_sc2), ws.at<float>(o_tauf)};
    so.w_id = ws.at<int32_t>(o_wid2);
    so.w_nrm = ws.at<float>(o_wnrm2);
    so.u_work = ws.at<int>(o_uwork);
    p.n_users = n_users;
    p.mode = 1;
    if (p.heap_global) p.heap_mem = ws.at<float>(o_heapm);
    const int64_t mw = max_work;
    p.work = TcWork{m.w1, m.w1 + mw, m.w1 + 2 * mw, m.w1 + 3 * mw, m.n_work, m.row_user, m.pos_c, nullptr, 1, nullptr,
                    nI};
    const int grid = (int)(max_work < idx->num_sms ? max_work : idx->num_sms);
    MIPS_CUDA(cudaMemsetAsync(so.n_cand, 0, sizeof(int) * nl, s));  // (as in run_bmm)
    if ((st = mark_kernel(idx, s)) != MIPS_OK) return st;
    MIPS_CUDA(launch_tc_score_select(&map_a, &map_at, &map_b, &map_bt, p, so, ws.at<float2>(o_uaux), m.aux_c,
                                     idx->stats_dev,
                                     idx->err_dev, grid, s));
    if ((st = mark_kernel(idx, s)) != MIPS_OK) return st;
    MIPS_CUDA(mx_tc_pass2(m, ws.at<int32_t>(o_assign), ws.at<float2>(o_uaux), ws.at<float>(o_bounds), so, K,
                          &user_perm, ws.at<int32_t>(o_vis), idx->stats_dev, s, &idx->launches));
    // second pass: uneven work items, claimed dynamically (counter in n_work[2])
    MIPS_CUDA(cudaMemsetAsync(m.n_work + 2, 0, sizeof(int), s));
    p.work = TcWork{m.w2, m.w2 + mw, m.w2 + 2 * mw, m.w2 + 3 * mw, m.n_work + 1, m.row_user, m.pos_c, nullptr, 1,
                    m.n_work + 2, nI};
    if ((st = mark_kernel(idx, s)) != MIPS_OK) return st;
    MIPS_CUDA(launch_tc_score_select(&map_a, &map_at, &map_b, &map_bt, p, so, ws.at<float2>(o_uaux), m.aux_c,
                                     idx->stats_dev,
                                     idx->err_dev, grid, s));
    if ((st = mark_kernel(idx, s)) != MIPS_OK) return st;
    idx->launches += 2;
    if ((st = end_stage(idx, ST_WALK, s)) != MIPS_OK) return st;
    MIPS_CUDA(launch_rescore(users, n_users, f, idx->items, idx->perm, idx->item_nrm, nI, K, so, out_idx, out_score,
                             idx->stats_dev, idx->err_dev, s));
    idx->launches += 4;
  }
  if ((st = end_stage(idx, ST_RESCORE, s)) != MIPS_OK) return st;
  idx->mx.assign = ws.at<int32_t>(o_assign);
  idx->mx.cent = ws.at<float>(o_cent);
  idx->mx.cosb = ws.at<float>(o_cosbf);
  idx->mx.bounds = ws.at<float>(o_bounds);
  idx->mx.lists = vals;
  idx->mx.visited = ws.at<int32_t>(o_vis);
  idx->mx.user_perm = user_perm;
  idx->mx.n_users = n_users;
  idx->mx.C = C;
  idx->last_users = n_users;
  idx->last_clusters = C;
  idx->last_dtype = use_tc ? idx->opt.dtype : MIPS_FP32;
  return MIPS_OK;
}

double elapsed_ms(cudaEvent_t a, cudaEvent_t b) {
  float t = 0.f;
  cudaEventElapsedTime(&t, a, b);
  return t;
}

// Optimus (Sec. IV): time a user sample on both paths, extrapolate, finish
// the other users with the faster one, reuse the sample's results.
mips_status run_select(mips_index_t idx, const float* users, int64_t n_users, int K, int32_t* out_idx,
                       double* out_score, cudaStream_t s, mips_select_report* rep) {
  // sample size: the requested fraction, but at least two waves of user
  // tiles on every SM (the hardware-effects floor, here the GPU's analogue
  // of the L2-sized sample)
  const int64_t floor_users = 2ll * idx->num_sms * 128;
  int64_t ns = (int64_t)ceil(idx->opt.sample_frac * (double)n_users);
  if (ns < floor_users) ns = floor_users;
  if (ns > n_users) ns = n_users;
  // seeded sample: the users u whose image under a seeded affine
  // permutation of [0, n), (a u + b) mod n with a coprime to n, falls below
  // ns -- exactly ns distinct users; sample and rest each ascending, split
  // on the device by a stable one-digit radix pass
  uint64_t a = 1, b = 0;
  affine_sample(n_users, idx->opt.seed ^ 0x5EEDull, &a, &b);
  const int64_t nr = n_users - ns;
  const int f = idx->f;
  Arena& w = idx->ws_sel;
  w.reset();
  size_t o_keys = w.take(4 * n_users), o_ids = w.take(4 * n_users), o_keys2 = w.take(4 * n_users),
         o_ids2 = w.take(4 * n_users), o_tmp = w.take(radix_sort_temp_bytes(n_users, 1));
  size_t o_su = w.take(sizeof(float) * ns * f), o_ru = w.take(sizeof(float) * (nr > 0 ? nr : 1) * f);
  size_t o_bi = w.take(4 * ns * K), o_bs = w.take(8 * ns * K), o_mi = w.take(4 * ns * K), o_ms = w.take(8 * ns * K);
  size_t o_ri = w.take(4 * (nr > 0 ? nr : 1) * K), o_rs = w.take(8 * (nr > 0 ? nr : 1) * K);
  MIPS_CUDA(w.ensure(w.used, s));
  uint32_t* keys = w.at<uint32_t>(o_keys);
  int32_t* ids = w.at<int32_t>(o_ids);
  uint32_t* keys2 = w.at<uint32_t>(o_keys2);
  int32_t* ids2 = w.at<int32_t>(o_ids2);
  launch_sample_keys(n_users, a, b, ns, keys, ids, s);
  MIPS_CUDA(radix_sort_pairs(keys, ids, keys2, ids2, n_users, 1, 0, 8, w.at<uint32_t>(o_tmp), s, nullptr));
  const int32_t* sample_ids = ids;       // the first ns of the split
  const int32_t* rest_ids = ids + ns;    // then the rest
  launch_gather_rows(users, sample_ids, ns, f, w.at<float>(o_su), s);
  if (nr > 0) launch_gather_rows(users, rest_ids, nr, f, w.at<float>(o_ru), s);
  MIPS_CUDA(cudaGetLastError());

  cudaEvent_t e[3];
  for (auto& x : e) MIPS_CUDA(cudaEventCreate(&x));
  struct Guard {
    cudaEvent_t* e;
    ~Guard() {
      for (int i = 0; i < 3; ++i) cudaEventDestroy(e[i]);
    }
  } guard{e};
  mips_status st;
  // blocked multiply on the sample (M_I)
  MIPS_CUDA(cudaEventRecord(e[0], s));
  if ((st = run_bmm(idx, w.at<float>(o_su), ns, K, w.at<int32_t>(o_bi), w.at<double>(o_bs), s)) != MIPS_OK) return st;
  MIPS_CUDA(cudaEventRecord(e[1], s));
  // Maximus on the sample (C_I and Q_I); its stage times restart here
  for (int i = 0; i < kStages; ++i) idx->stage_ran[i] = false;
  idx->n_order = 0;
  idx->last_stage = -1;
  MIPS_CUDA(cudaEventRecord(idx->ev[0], s));
  if ((st = run_maximus(idx, w.at<float>(o_su), ns, K, w.at<int32_t>(o_mi), w.at<double>(o_ms), s)) != MIPS_OK)
    return st;
  MIPS_CUDA(cudaEventRecord(e[2], s));
  MIPS_CUDA(cudaEventSynchronize(e[2]));
  mips_stats mx;
  if ((st = mips_get_stats(idx, &mx)) != MIPS_OK) return st;
  const double t_bmm = elapsed_ms(e[0], e[1]) * 1e-3;
  const double t_mx = elapsed_ms(e[1], e[2]) * 1e-3;
  // construction: k-means work grows with the users, bounds and sort do not
  const double c_i = (mx.ms_kmeans * (double)n_users / (double)ns + mx.ms_bounds + mx.ms_sort) * 1e-3;
  const double q_i = (t_mx - (mx.ms_kmeans + mx.ms_bounds + mx.ms_sort) * 1e-3) / (double)ns;
  const double m_i = t_bmm / (double)ns;
  mips_select_report r{};
  r.t_build = c_i;
  r.q_user = q_i;
  r.m_user = m_i;
  r.sample_users = ns;
  r.est_index = c_i + (double)n_users * q_i;
  r.est_bmm = (double)n_users * m_i;
  r.choice = r.est_index < r.est_bmm ? 1 : 0;
  if (rep) *rep = r;
  // the sample's results (both paths are exact and agree), then the rest
  launch_scatter_topk(w.at<int32_t>(r.choice ? o_mi : o_bi), w.at<double>(r.choice ? o_ms : o_bs), sample_ids, ns, K,
                      out_idx, out_score, s);
  if (nr > 0) {
    // the call's stage times are those of this last run
    for (int i = 0; i < kStages; ++i) idx->stage_ran[i] = false;
    idx->n_order = 0;
    idx->last_stage = -1;
    MIPS_CUDA(cudaEventRecord(idx->ev[0], s));
    if (r.choice == 1)
      st = run_maximus(idx, w.at<float>(o_ru), nr, K, w.at<int32_t>(o_ri), w.at<double>(o_rs), s);
    else
      st = run_bmm(idx, w.at<float>(o_ru), nr, K, w.at<int32_t>(o_ri), w.at<double>(o_rs), s);
    if (st != MIPS_OK) return st;
    launch_scatter_topk(w.at<int32_t>(o_ri), w.at<double>(o_rs), rest_ids, nr, K, out_idx, out_score, s);
  }
  MIPS_CUDA(cudaGetLastError());
  idx->last_users = n_users;
  return MIPS_OK;
}

// Two-sided 95% quantile of Student's t with d = 1 .. 15 degrees of freedom
// (the textbook table).
double t975(int d) {
  static const double q[16] = {0.0,   12.706, 4.303, 3.182, 2.776, 2.571, 2.447, 2.365,
                               2.306, 2.262,  2.228, 2.201, 2.179, 2.160, 2.145, 2.131};
  return d < 1 ? 0.0 : q[d < 15 ? d : 15];
}

// One timed run of arm (index, method) on n users: returns the device
// seconds, and for Maximus the stage times of the run.
mips_status time_arm(mips_index_t idx, int method, const float* users, int64_t n, int K, int32_t* oi, double* os,
                     cudaStream_t s, cudaEvent_t e0, cudaEvent_t e1, double* secs, mips_stats* st_out) {
  for (int i = 0; i < kStages; ++i) idx->stage_ran[i] = false;
  idx->n_order = 0;
  idx->last_stage = -1;
  MIPS_CUDA(cudaEventRecord(e0, s));
  MIPS_CUDA(cudaEventRecord(idx->ev[0], s));
  mips_status st = method == 1 ? run_maximus(idx, users, n, K, oi, os, s) : run_bmm(idx, users, n, K, oi, os, s);
  if (st != MIPS_OK) return st;
  MIPS_CUDA(cudaEventRecord(e1, s));
  MIPS_CUDA(cudaEventSynchronize(e1));
  *secs = elapsed_ms(e0, e1) * 1e-3;
  if (st_out) return mips_get_stats(idx, st_out);
  return MIPS_OK;
}

mips_status run_select_arms(const mips_index_t* ix, int n_ix, const float* users, int64_t n_users, int K,
                            int max_rounds, int32_t* out_idx, double* out_score, cudaStream_t s,
                            mips_arms_report* rep) {
  mips_index_t idx0 = ix[0];
  const int f = idx0->f;
  const int rounds_max = max_rounds <= 0 ? 6 : max_rounds;
  // the sample: as mips_select's (the requested fraction, at least two waves
  // of user tiles per SM, seeded affine split)
  const int64_t floor_users = 2ll * idx0->num_sms * 128;
  int64_t ns = (int64_t)ceil(idx0->opt.sample_frac * (double)n_users);
  if (ns < floor_users) ns = floor_users;
  if (ns > n_users) ns = n_users;
  uint64_t a = 1, b = 0;
  affine_sample(n_users, idx0->opt.seed ^ 0x5EEDull, &a, &b);
  const int64_t nr = n_users - ns;
  const int n_arms = 2 * n_ix;
  Arena& w = idx0->ws_sel;
  w.reset();
  size_t o_keys = w.take(4 * n_users), o_ids = w.take(4 * n_users), o_keys2 = w.take(4 * n_users),
         o_ids2 = w.take(4 * n_users), o_tmp = w.take(radix_sort_temp_bytes(n_users, 1));
  size_t o_su = w.take(sizeof(float) * ns * f), o_ru = w.take(sizeof(float) * (nr > 0 ? nr : 1) * f);
  size_t o_ri = w.take(4 * (nr > 0 ? nr : 1) * K), o_rs = w.take(8 * (nr > 0 ? nr : 1) * K);
  size_t o_ai[MIPS_MAX_ARMS], o_as[MIPS_MAX_ARMS];
  for (int k = 0; k < n_arms; ++k) {
    o_ai[k] = w.take(4 * ns * K);
    o_as[k] = w.take(8 * ns * K);
  }
  MIPS_CUDA(w.ensure(w.used, s));
  uint32_t* keys = w.at<uint32_t>(o_keys);
  int32_t* ids = w.at<int32_t>(o_ids);
  uint32_t* keys2 = w.at<uint32_t>(o_keys2);
  int32_t* ids2 = w.at<int32_t>(o_ids2);
  launch_sample_keys(n_users, a, b, ns, keys, ids, s);
  MIPS_CUDA(radix_sort_pairs(keys, ids, keys2, ids2, n_users, 1, 0, 8, w.at<uint32_t>(o_tmp), s, nullptr));
  const int32_t* sample_ids = ids;
  const int32_t* rest_ids = ids + ns;
  launch_gather_rows(users, sample_ids, ns, f, w.at<float>(o_su), s);
  if (nr > 0) launch_gather_rows(users, rest_ids, nr, f, w.at<float>(o_ru), s);
  MIPS_CUDA(cudaGetLastError());

  cudaEvent_t ev[4];
  for (auto& x : ev) MIPS_CUDA(cudaEventCreate(&x));
  struct EvGuard {
    cudaEvent_t* e;
    ~EvGuard() {
      for (int i = 0; i < 4; ++i) cudaEventDestroy(e[i]);
    }
  } eg{ev};
  MIPS_CUDA(cudaEventRecord(ev[2], s));
  mips_arms_report r{};
  r.n_arms = n_arms;
  r.sample_users = ns;
  std::vector<std::vector<double>> est(n_arms);
  mips_status st;
  // one untimed run per arm first: workspace growth and first-launch costs
  // are not the arm's
  for (int k = 0; k < n_arms; ++k) {
    double t;
    if ((st = time_arm(ix[k / 2], k & 1, w.at<float>(o_su), ns, K, w.at<int32_t>(o_ai[k]), w.at<double>(o_as[k]), s,
                       ev[0], ev[1], &t, nullptr)) != MIPS_OK)
      return st;
  }
  auto mean_of = [&](int k) {
    double m = 0.0;
    for (double x : est[k]) m += x;
    return m / (double)est[k].size();
  };
  auto ci_of = [&](int k) {
    const int n = (int)est[k].size();
    if (n < 2) return 0.0;
    const double m = mean_of(k);
    double v = 0.0;
    for (double x : est[k]) v += (x - m) * (x - m);
    return t975(n - 1) * sqrt(v / (double)(n - 1)) / sqrt((double)n);
  };
  for (int rd = 0; rd < rounds_max; ++rd) {
    for (int k = 0; k < n_arms; ++k) {
      if (r.arm[k].dropped) continue;
      mips_index_t ik = ix[k / 2];
      const int method = k & 1;
      double t = 0.0;
      mips_stats ms{};
      if ((st = time_arm(ik, method, w.at<float>(o_su), ns, K, w.at<int32_t>(o_ai[k]), w.at<double>(o_as[k]), s,
                         ev[0], ev[1], &t, method == 1 ? &ms : nullptr)) != MIPS_OK)
        return st;
      r.t_sample += t;
      double e;
      if (method == 1) {  // construction: k-means grows with the users, bounds and sort do not
        const double c_i = (ms.ms_kmeans * (double)n_users / (double)ns + ms.ms_bounds + ms.ms_sort) * 1e-3;
        const double q_i = (t - (ms.ms_kmeans + ms.ms_bounds + ms.ms_sort) * 1e-3) / (double)ns;
        e = c_i + (double)n_users * q_i;
      } else {
        e = t * (double)n_users / (double)ns;
      }
      est[k].push_back(e);
      r.arm[k].rounds = (int)est[k].size();
    }
    r.rounds = rd + 1;
    if (rd + 1 < 3) continue;
    int best = -1;
    for (int k = 0; k < n_arms; ++k)
      if (!r.arm[k].dropped && (best < 0 || mean_of(k) < mean_of(best))) best = k;
    const double hi_best = mean_of(best) + ci_of(best);
    bool all_sep = true;
    for (int k = 0; k < n_arms; ++k) {
      if (k == best || r.arm[k].dropped) continue;
      if (mean_of(k) - ci_of(k) > hi_best) r.arm[k].dropped = 1;
      else all_sep = false;
    }
    if (all_sep) {
      r.separated = 1;
      break;
    }
  }
  int choice = 0;
  for (int k = 0; k < n_arms; ++k) {
    mips_arm_report& ar = r.arm[k];
    ar.index = k / 2;
    ar.dtype = ix[k / 2]->opt.dtype;
    ar.method = k & 1;
    ar.est_mean = mean_of(k);
    ar.est_ci = ci_of(k);
  }
  for (int k = 1; k < n_arms; ++k)
    if (r.arm[k].est_mean < r.arm[choice].est_mean) choice = k;
  r.choice = choice;
  // the chosen arm's sample results (every arm is exact), then the rest with it
  launch_scatter_topk(w.at<int32_t>(o_ai[choice]), w.at<double>(o_as[choice]), sample_ids, ns, K, out_idx,
                      out_score, s);
  mips_index_t ic = ix[choice / 2];
  if (nr > 0) {
    double t;
    if ((st = time_arm(ic, choice & 1, w.at<float>(o_ru), nr, K, w.at<int32_t>(o_ri), w.at<double>(o_rs), s, ev[0],
                       ev[1], &t, nullptr)) != MIPS_OK)
      return st;
    launch_scatter_topk(w.at<int32_t>(o_ri), w.at<double>(o_rs), rest_ids, nr, K, out_idx, out_score, s);
  }
  MIPS_CUDA(cudaGetLastError());
  MIPS_CUDA(cudaEventRecord(ev[3], s));
  MIPS_CUDA(cudaEventSynchronize(ev[3]));
  r.t_total = elapsed_ms(ev[2], ev[3]) * 1e-3;
  for (int i = 0; i < n_ix; ++i) ix[i]->last_users = n_users;
  if (rep) *rep = r;
  return MIPS_OK;
}

mips_status check_call(mips_index_t idx, const void* users, int64_t n_users, int K, const void* oi,
                       const void* os) {
  if (!idx) return fail(MIPS_ERR_ARG, "null index");
  if (!users || !oi || !os) return fail(MIPS_ERR_ARG, "null buffer");
  if (n_users <= 0 || n_users >= (1ll << 31)) return fail(MIPS_ERR_ARG, "n_users out of range: %lld", (long long)n_users);
  if (K < 1 || K > idx->n_items || K > 128) return fail(MIPS_ERR_ARG, "K out of range: %d", K);
  return check_device(idx);
}

}  // namespace

// A worker handle of an index for concurrent calls on other streams: the
// same (read-only) item arrays and tensor maps, its own workspace, error
// flag, counters and events.  Freed with mips_free_index, which leaves the
// shared item arrays to their owner.
mips_index_t mips::index_worker_clone(mips_index_t src) {
  mips_index_s* w = new (std::nothrow) mips_index_s();
  if (!w) return nullptr;
  w->device = src->device;
  w->f = src->f;
  w->n_items = src->n_items;
  w->clusters = src->clusters;
  w->opt = src->opt;
  w->items = src->items;
  w->perm = src->perm;
  w->item_nrm = src->item_nrm;
  w->fp = src->fp;
  w->items_bf16 = src->items_bf16;
  w->item_aux = src->item_aux;
  w->esize = src->esize;
  w->item_scale = src->item_scale;
  w->n_items_pad = src->n_items_pad;
  w->num_sms = src->num_sms;
  w->max_smem = src->max_smem;
  w->shares_items = true;
  bool ok = cudaEventCreateWithFlags(&w->done, cudaEventDisableTiming) == cudaSuccess;
  if (ok && src->fit_C > 0) {  // its own copy of the fitted centroids
    const size_t bytes = sizeof(float) * (size_t)src->fit_C * src->f;
    if (src->has_done) ok = cudaEventSynchronize(src->done) == cudaSuccess;
    ok = ok && cudaMalloc(&w->fit_cent, bytes) == cudaSuccess &&
         cudaMemcpy(w->fit_cent, src->fit_cent, bytes, cudaMemcpyDeviceToDevice) == cudaSuccess;
    if (ok) {
      w->fit_C = src->fit_C;
      w->fit_cap = (int64_t)src->fit_C * src->f;
      w->fit_gen = src->fit_gen;
    }
  }
  for (int i = 0; i <= kStages && ok; ++i) ok = cudaEventCreate(&w->ev[i]) == cudaSuccess;
  for (int i = 0; i < 4 && ok; ++i) ok = cudaEventCreate(&w->kev[i]) == cudaSuccess;
  ok = ok && cudaMalloc(&w->err_dev, sizeof(int)) == cudaSuccess && cudaMemset(w->err_dev, 0, sizeof(int)) == cudaSuccess;
  ok = ok && cudaMalloc(&w->stats_dev, sizeof(DevStats)) == cudaSuccess;
  if (!ok) {
    mips_free_index(w);
    return nullptr;
  }
  return w;
}

int mips::index_f(mips_index_t idx) { return idx->f; }
int64_t mips::index_n_items(mips_index_t idx) { return idx->n_items; }

size_t mips::call_workspace_bytes(mips_index_t idx, int64_t n_users, int K, int method) {
  size_t bytes = 0;
  if (method == 0)
    run_bmm(idx, nullptr, n_users, K, nullptr, nullptr, nullptr, &bytes);
  else
    run_maximus(idx, nullptr, n_users, K, nullptr, nullptr, nullptr, &bytes);
  return bytes;
}

size_t mips::index_workspace_used(mips_index_t idx) { return idx->ws.used; }
size_t mips::index_workspace_held(mips_index_t idx) { return idx->ws.cap; }

cudaError_t mips::index_release_workspace(mips_index_t idx, cudaStream_t s) {
  if (!idx->ws.base) return cudaSuccess;
  cudaError_t e = cudaFreeAsync(idx->ws.base, s);
  idx->ws.base = nullptr;
  idx->ws.cap = 0;
  idx->ws.used = 0;
  ++idx->ws.gen;  // graphs captured over it are stale
  idx->mx.C = 0;
  return e;
}

extern "C" {

int mips_version(void) { return 100; }

mips_status mips_test_expire_next_wait(int64_t wait_ns) {
  if (wait_ns < 100000 || wait_ns > 1000000000) return fail(MIPS_ERR_ARG, "wait_ns out of [1e5, 1e9]: %lld",
                                                            (long long)wait_ns);
  g_test_expire_ns.store(wait_ns);
  return MIPS_OK;
}

const char* mips_last_error(void) { return g_err.c_str(); }

void mips_default_options(mips_options* opt) {
  if (!opt) return;
  opt->dtype = MIPS_BF16;
  opt->kmeans_iters = 3;
  opt->block_items = 0;
  opt->sample_frac = 0.005;
  opt->autotune = 0;
  opt->seed = 0;
  opt->kmeans_spherical = 0;
}

mips_status mips_build_index(const float* items_dev, int64_t n_items, int f, int clusters,
                             const mips_options* opt, void* stream, mips_index_t* out) {
  g_err.clear();
  if (!out) return fail(MIPS_ERR_ARG, "null output handle");
  *out = nullptr;
  if (!items_dev) return fail(MIPS_ERR_ARG, "null items");
  if (f < 1 || f > 128) return fail(MIPS_ERR_ARG, "f out of range [1,128]: %d", f);
  if (n_items < 1 || n_items >= (1ll << 31)) return fail(MIPS_ERR_ARG, "n_items out of range: %lld", (long long)n_items);
  if (clusters < 1 || clusters > 4096) return fail(MIPS_ERR_ARG, "clusters out of range [1,4096]: %d", clusters);
  mips_options o;
  mips_default_options(&o);
  if (opt) o = *opt;
  if (o.dtype != MIPS_FP32 && !tc_dtype(o.dtype)) return fail(MIPS_ERR_ARG, "dtype %d is not a mips_dtype", o.dtype);
  if (o.kmeans_iters < 0 || o.kmeans_iters > 100) return fail(MIPS_ERR_ARG, "kmeans_iters out of range");
  if (o.block_items < 0) return fail(MIPS_ERR_ARG, "block_items must be >= 0 (0 = default)");
  if (!(o.sample_frac > 0.0 && o.sample_frac <= 1.0)) return fail(MIPS_ERR_ARG, "sample_frac out of range (0,1]");
  if (o.kmeans_spherical != 0 && o.kmeans_spherical != 1) return fail(MIPS_ERR_ARG, "kmeans_spherical must be 0 or 1");
  cudaStream_t s = (cudaStream_t)stream;

  mips_index_s* idx = new (std::nothrow) mips_index_s();
  if (!idx) return fail(MIPS_ERR_NOMEM, "host allocation failed");
  auto bail = [&](mips_status st) {
    mips_free_index(idx);
    return st;
  };
  cudaError_t e;
#define BUILD_CUDA(call)                                   \
  do {                                                     \
    e = (call);                                            \
    if (e != cudaSuccess) return bail(cuda_fail(e, #call)); \
  } while (0)
  BUILD_CUDA(cudaGetDevice(&idx->device));
  BUILD_CUDA(cudaDeviceGetAttribute(&idx->num_sms, cudaDevAttrMultiProcessorCount, idx->device));
  BUILD_CUDA(cudaDeviceGetAttribute(&idx->max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, idx->device));
  idx->f = f;
  idx->n_items = n_items;
  idx->clusters = clusters;
  idx->opt = o;
  BUILD_CUDA(cudaEventCreateWithFlags(&idx->done, cudaEventDisableTiming));
  for (int i = 0; i <= kStages; ++i) BUILD_CUDA(cudaEventCreate(&idx->ev[i]));
  for (int i = 0; i < 4; ++i) BUILD_CUDA(cudaEventCreate(&idx->kev[i]));
  BUILD_CUDA(cudaMalloc(&idx->err_dev, sizeof(int)));
  BUILD_CUDA(cudaMemsetAsync(idx->err_dev, 0, sizeof(int), s));
  BUILD_CUDA(cudaMalloc(&idx->stats_dev, sizeof(DevStats)));
  BUILD_CUDA(cudaMalloc(&idx->items, sizeof(float) * n_items * f));
  BUILD_CUDA(cudaMalloc(&idx->perm, sizeof(int32_t) * n_items));
  BUILD_CUDA(cudaMalloc(&idx->item_nrm, sizeof(float) * n_items));
  // item order: by norm bound, descending (ties by item id), so a user's
  // threshold rises within the first item tiles of every scan
  {
    launch_row_norm_ub(items_dev, n_items, f, idx->item_nrm, idx->err_dev, s);
    char* tmp = nullptr;
    const size_t tb = radix_sort_temp_bytes(n_items, 1);
    const size_t nb4 = round_up(sizeof(uint32_t) * n_items, 256);
    BUILD_CUDA(cudaMallocAsync((void**)&tmp, 3 * nb4 + tb, s));
    uint32_t* keys = (uint32_t*)tmp;
    uint32_t* keys_alt = (uint32_t*)(tmp + nb4);
    int32_t* vals_alt = (int32_t*)(tmp + 2 * nb4);
    uint32_t* temp = (uint32_t*)(tmp + 3 * nb4);
    int32_t* vals = idx->perm;
    e = make_float_desc_keys(idx->item_nrm, n_items, keys, vals, n_items, s);
    if (e == cudaSuccess) e = radix_sort_pairs(keys, vals, keys_alt, vals_alt, n_items, 1, 0, 32, temp, s, nullptr);
    // four passes: the result is back in the first buffers
    if (e == cudaSuccess && vals != idx->perm) e = cudaErrorUnknown;
    cudaFreeAsync(tmp, s);
    if (e != cudaSuccess) return bail(cuda_fail(e, "item norm sort"));
  }
  launch_gather_rows(items_dev, idx->perm, n_items, f, idx->items, s);
  launch_row_norm_ub(idx->items, n_items, f, idx->item_nrm, idx->err_dev, s);
  BUILD_CUDA(cudaGetLastError());
  if (tc_dtype(o.dtype)) {
    const bool f8 = o.dtype == MIPS_FP8_E4M3;
    idx->esize = f8 ? 1 : 2;
    idx->fp = f8 ? tc_row_len8(f) : tc_row_len(f);
    idx->n_items_pad = round_up(n_items, tc_items_per_tile());
    BUILD_CUDA(cudaMalloc(&idx->items_bf16, (size_t)idx->esize * idx->n_items_pad * idx->fp));
    BUILD_CUDA(cudaMalloc(&idx->item_aux, sizeof(float2) * idx->n_items_pad));
    if (f8) {  // one item scale from the largest norm bound (item_nrm is sorted, descending)
      BUILD_CUDA(cudaMalloc(&idx->item_scale, sizeof(float)));
      launch_fp8_item_scale(idx->item_nrm, n_items, idx->item_scale, s);
      launch_quant_fp8(idx->items, n_items, f, idx->fp, 1, idx->item_scale, idx->items_bf16, idx->n_items_pad,
                       idx->item_aux, nullptr, idx->err_dev, s);
    } else {
      launch_quant_bf16(idx->items, n_items, f, idx->fp, 1, idx->items_bf16, idx->n_items_pad, idx->item_aux,
                        idx->err_dev, s);
    }
    BUILD_CUDA(cudaGetLastError());
    // (tensor maps are made per call: the plan depends on K)
  }
  BUILD_CUDA(cudaStreamSynchronize(s));
  int herr = 0;
  BUILD_CUDA(cudaMemcpy(&herr, idx->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
  if (herr & DEV_ERR_NONFINITE) return bail(fail(MIPS_ERR_NONFINITE, "items hold NaN or Inf (or a norm overflows FP32)"));
#undef BUILD_CUDA
  *out = idx;
  return MIPS_OK;
}

mips_status mips_topk(mips_index_t idx, const float* users_dev, int64_t n_users, int K,
                      int32_t* out_idx_dev, double* out_score_dev, void* stream) {
  g_err.clear();
  mips_status st = check_call(idx, users_dev, n_users, K, out_idx_dev, out_score_dev);
  if (st != MIPS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = begin_call(idx, s)) != MIPS_OK) return st;
  if ((st = run_bmm(idx, users_dev, n_users, K, out_idx_dev, out_score_dev, s)) != MIPS_OK) return st;
  return end_call(idx, s);
}

mips_status mips_topk_maximus(mips_index_t idx, const float* users_dev, int64_t n_users, int K,
                              int32_t* out_idx_dev, double* out_score_dev, void* stream) {
  g_err.clear();
  mips_status st = check_call(idx, users_dev, n_users, K, out_idx_dev, out_score_dev);
  if (st != MIPS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = begin_call(idx, s)) != MIPS_OK) return st;
  if ((st = run_maximus(idx, users_dev, n_users, K, out_idx_dev, out_score_dev, s)) != MIPS_OK) return st;
  return end_call(idx, s);
}

mips_status mips_fit_clusters(mips_index_t idx, const float* users_dev, int64_t n_users, void* stream) {
  g_err.clear();
  if (!idx) return fail(MIPS_ERR_ARG, "null index");
  if (!users_dev && n_users == 0) {  // back to clustering each call's users
    if (idx->has_done) MIPS_CUDA(cudaEventSynchronize(idx->done));
    if (idx->fit_cent) MIPS_CUDA(cudaFree(idx->fit_cent));
    idx->fit_cent = nullptr;
    idx->fit_C = 0;
    idx->fit_cap = 0;
    ++idx->fit_gen;
    return MIPS_OK;
  }
  if (!users_dev) return fail(MIPS_ERR_ARG, "null users");
  if (n_users < 1 || n_users >= INT32_MAX) return fail(MIPS_ERR_ARG, "n_users out of range");
  mips_status st = check_device(idx);
  if (st != MIPS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = begin_call(idx, s)) != MIPS_OK) return st;
  const int f = idx->f;
  const int C = (int)std::min<int64_t>(idx->clusters, n_users);
  Arena& ws = idx->ws;
  ws.reset();
  size_t o_ids = ws.take(sizeof(int64_t) * C), o_cent = ws.take(sizeof(float) * C * f), o_hn2 = ws.take(sizeof(float) * C);
  size_t o_bits = ws.take(sizeof(uint32_t) * ((n_users + 31) / 32));
  size_t o_assign = ws.take(sizeof(int32_t) * n_users), o_sums = ws.take(sizeof(unsigned long long) * C * f);
  size_t o_cnt = ws.take(sizeof(unsigned) * C), o_amax = ws.take(16), o_scale = ws.take(16);
  const bool km_tc = idx->opt.dtype != MIPS_FP32 && km_tc_fits(f, C, idx->max_smem);
  const int fk = km_tc_row_len(f);
  const size_t o_ukm = km_tc ? ws.take(sizeof(uint16_t) * n_users * fk) : 0;
  const size_t o_ckm = km_tc ? ws.take(sizeof(uint16_t) * (size_t)C * fk) : 0;
  MIPS_CUDA(ws.ensure(ws.used, s));
  KmTc kt;
  if (km_tc) {
    kt.users_km = ws.at<uint16_t>(o_ukm);
    kt.cent_km = ws.at<uint16_t>(o_ckm);
    kt.err = idx->err_dev;
    kt.max_smem = idx->max_smem;
  }
  idx->mx.C = 0;  // the workspace is reused: earlier Maximus views are gone
  MIPS_CUDA(draw_init_ids(n_users, C, idx->opt.seed, ws.at<uint32_t>(o_bits), ws.at<int64_t>(o_ids), s));
  idx->launches += 1;
  MIPS_CUDA(maximus_kmeans(users_dev, n_users, f, C, idx->opt.kmeans_iters, ws.at<int64_t>(o_ids),
                           ws.at<float>(o_cent), ws.at<float>(o_hn2), ws.at<int32_t>(o_assign),
                           ws.at<unsigned long long>(o_sums), ws.at<unsigned>(o_cnt), ws.at<uint32_t>(o_amax),
                           ws.at<float>(o_scale), idx->opt.kmeans_spherical != 0, kt, s, &idx->launches));
  if (idx->fit_cap < (int64_t)C * f) {  // (every call on this index is ordered after idx->done)
    if (idx->has_done) MIPS_CUDA(cudaEventSynchronize(idx->done));
    if (idx->fit_cent) MIPS_CUDA(cudaFree(idx->fit_cent));
    idx->fit_cent = nullptr;
    idx->fit_C = 0;
    idx->fit_cap = 0;
    MIPS_CUDA(cudaMalloc(&idx->fit_cent, sizeof(float) * C * f));
    idx->fit_cap = (int64_t)C * f;
  }
  MIPS_CUDA(cudaMemcpyAsync(idx->fit_cent, ws.at<float>(o_cent), sizeof(float) * C * f, cudaMemcpyDeviceToDevice, s));
  idx->fit_C = C;
  ++idx->fit_gen;
  if ((st = end_stage(idx, ST_KMEANS, s)) != MIPS_OK) return st;
  return end_call(idx, s);
}

mips_status mips_select(mips_index_t idx, const float* users_dev, int64_t n_users, int K,
                        int32_t* out_idx_dev, double* out_score_dev, void* stream,
                        mips_select_report* rep) {
  g_err.clear();
  mips_status st = check_call(idx, users_dev, n_users, K, out_idx_dev, out_score_dev);
  if (st != MIPS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  if ((st = begin_call(idx, s)) != MIPS_OK) return st;
  if ((st = run_select(idx, users_dev, n_users, K, out_idx_dev, out_score_dev, s, rep)) != MIPS_OK) return st;
  return end_call(idx, s);
}

mips_status mips_select_arms(const mips_index_t* indexes, int n_indexes, const float* users_dev, int64_t n_users,
                             int K, int max_rounds, int32_t* out_idx_dev, double* out_score_dev, void* stream,
                             mips_arms_report* rep) {
  g_err.clear();
  if (!indexes || n_indexes < 1 || n_indexes > MIPS_MAX_ARMS / 2)
    return fail(MIPS_ERR_ARG, "n_indexes out of range [1,%d]", MIPS_MAX_ARMS / 2);
  if (max_rounds != 0 && (max_rounds < 3 || max_rounds > 16)) return fail(MIPS_ERR_ARG, "max_rounds out of range");
  mips_status st = check_call(indexes[0], users_dev, n_users, K, out_idx_dev, out_score_dev);
  if (st != MIPS_OK) return st;
  for (int i = 1; i < n_indexes; ++i) {
    if (!indexes[i]) return fail(MIPS_ERR_ARG, "null index %d", i);
    if (indexes[i]->f != indexes[0]->f || indexes[i]->n_items != indexes[0]->n_items ||
        indexes[i]->device != indexes[0]->device)
      return fail(MIPS_ERR_ARG, "index %d differs from index 0 in f, n_items or device", i);
    if ((st = check_device(indexes[i])) != MIPS_OK) return st;
  }
  cudaStream_t s = (cudaStream_t)stream;
  for (int i = 0; i < n_indexes; ++i)
    if ((st = begin_call(indexes[i], s)) != MIPS_OK) return st;
  if ((st = run_select_arms(indexes, n_indexes, users_dev, n_users, K, max_rounds, out_idx_dev, out_score_dev, s,
                            rep)) != MIPS_OK)
    return st;
  for (int i = 0; i < n_indexes; ++i)
    if ((st = end_call(indexes[i], s)) != MIPS_OK) return st;
  return MIPS_OK;
}

mips_status mips_autotune(mips_index_t idx, const float* users_dev, int64_t n_users, int K, void* stream,
                          mips_tune_report* rep) {
  g_err.clear();
  // (the outputs are the tuner's own buffers)
  mips_status st = check_call(idx, users_dev, n_users, K, users_dev, users_dev);
  if (st != MIPS_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  const auto t0 = std::chrono::steady_clock::now();
  // sample: n / 8 users, at least two waves of 128-user tiles on every SM
  int64_t ns = n_users / 8;
  if (ns < 2ll * idx->num_sms * 128) ns = 2ll * idx->num_sms * 128;
  if (ns > n_users) ns = n_users;
  const int f = idx->f;
  Arena& w = idx->ws_sel;
  w.reset();
  size_t o_keys = w.take(4 * n_users), o_ids = w.take(4 * n_users), o_keys2 = w.take(4 * n_users),
         o_ids2 = w.take(4 * n_users), o_tmp = w.take(radix_sort_temp_bytes(n_users, 1));
  size_t o_su = w.take(sizeof(float) * ns * f);
  size_t o_oi = w.take(4 * ns * K), o_os = w.take(8 * ns * K);
  MIPS_CUDA(w.ensure(w.used, s));
  {  // seeded sample of ns distinct users (affine permutation, as the selector's)
    uint64_t a = 1, b = 0;
    affine_sample(n_users, idx->opt.seed ^ 0x7E57ull, &a, &b);
    uint32_t* keys = w.at<uint32_t>(o_keys);
    int32_t* ids = w.at<int32_t>(o_ids);
    uint32_t* keys2 = w.at<uint32_t>(o_keys2);
    int32_t* ids2 = w.at<int32_t>(o_ids2);
    launch_sample_keys(n_users, a, b, ns, keys, ids, s);
    MIPS_CUDA(radix_sort_pairs(keys, ids, keys2, ids2, n_users, 1, 0, 8, w.at<uint32_t>(o_tmp), s, nullptr));
    launch_gather_rows(users_dev, ids, ns, f, w.at<float>(o_su), s);
  }
  MIPS_CUDA(cudaGetLastError());
  const int saved_c = idx->clusters, saved_b = idx->opt.block_items;
  const double scale = (double)ns / (double)n_users;
  struct Cand { int C, B; double est; };
  std::vector<Cand> tried;
  // |C| candidates with the users each sample cluster stands for; fitted
  // centroids fix |C| and leave only B to tune
  std::vector<std::pair<int, int>> cands;
  if (idx->fit_C > 0) {
    cands.push_back({idx->fit_C, idx->fit_C});
  } else {
    for (int C = 16; C <= 1024 && C <= n_users / 32; C *= 2)
      cands.push_back({C, std::max(1, (int)llround(C * scale))});
  }
  for (const auto& cc : cands) {
    const int C = cc.first, Cs = cc.second;
    for (int B : {1024, 4096, 16384}) {
      idx->clusters = Cs;
      idx->opt.block_items = B;
      double ms[kStages] = {};
      for (int rep_i = 0; rep_i < 2 && st == MIPS_OK; ++rep_i) {  // the first run sizes the workspace
        st = begin_call(idx, s);
        if (st == MIPS_OK) st = run_maximus(idx, w.at<float>(o_su), ns, K, w.at<int32_t>(o_oi), w.at<double>(o_os), s);
        if (st == MIPS_OK) st = end_call(idx, s);
      }
      if (st == MIPS_OK) st = mips_sync(idx, stream);
      if (st != MIPS_OK) {
        idx->clusters = saved_c;
        idx->opt.block_items = saved_b;
        return st;
      }
      cudaEvent_t prev = idx->ev[0];
      float t = 0.f;
      for (int q = 0; q < idx->n_order; ++q) {
        const int i = idx->order[q];
        MIPS_CUDA(cudaEventElapsedTime(&t, prev, idx->ev[1 + i]));
        ms[i] = t;
        prev = idx->ev[1 + i];
      }
      const double cr = (double)C / (double)Cs;
      const double est_ms = (ms[ST_BOUNDS] + ms[ST_SORT]) * cr + ms[ST_KMEANS] * cr / scale +
                            (ms[ST_PREP] + ms[ST_WALK] + ms[ST_RESCORE]) / scale;
      tried.push_back({C, B, est_ms / 1e3});
    }
  }
  Cand best{saved_c, saved_b, 0.0};
  if (!tried.empty()) {
    best = tried[0];
    for (const Cand& c : tried)
      if (c.est < best.est) best = c;
  }
  idx->clusters = idx->fit_C > 0 ? saved_c : best.C;
  idx->opt.block_items = best.B;
  if (rep) {
    memset(rep, 0, sizeof(*rep));
    rep->clusters = best.C;
    rep->block_items = best.B;
    rep->sample_users = ns;
    rep->n_tried = (int)(tried.size() < 32 ? tried.size() : 32);
    for (int i = 0; i < rep->n_tried; ++i) {
      rep->tried_clusters[i] = tried[i].C;
      rep->tried_block[i] = tried[i].B;
      rep->tried_est[i] = tried[i].est;
    }
    rep->t_tune = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
  return MIPS_OK;
}

mips_status mips_topk_graph(mips_index_t idx, const float* users_dev, int64_t n_users, int K, int method,
                            int32_t* out_idx_dev, double* out_score_dev, void* stream) {
  g_err.clear();
  mips_status st = check_call(idx, users_dev, n_users, K, out_idx_dev, out_score_dev);
  if (st != MIPS_OK) return st;
  if (method != 0 && method != 1) return fail(MIPS_ERR_ARG, "method must be 0 (blocked multiply) or 1 (Maximus)");
  cudaStream_t s = (cudaStream_t)stream;
  auto plain = [&]() {
    return method == 0 ? mips_topk(idx, users_dev, n_users, K, out_idx_dev, out_score_dev, stream)
                       : mips_topk_maximus(idx, users_dev, n_users, K, out_idx_dev, out_score_dev, stream);
  };
  if (s == nullptr) return plain();  // the legacy default stream cannot be captured
  for (auto& g : idx->graphs) {
    if (g.method != method || g.users != users_dev || g.n_users != n_users || g.K != K || g.out_idx != out_idx_dev ||
        g.out_score != out_score_dev || g.ws_gen != idx->ws.gen || g.cfg_clusters != idx->clusters ||
        g.cfg_block != idx->opt.block_items || g.cfg_fit != idx->fit_gen)
      continue;
    if (idx->has_done) MIPS_CUDA(cudaStreamWaitEvent(s, idx->done, 0));
    MIPS_CUDA(cudaGraphLaunch(g.exec, s));
    for (int i = 0; i < kStages; ++i) {
      idx->stage_ran[i] = g.stage_ran[i];
      idx->order[i] = g.order[i];
    }
    idx->n_order = g.n_order;
    idx->last_stage = g.last_stage;
    idx->launches = g.launches;
    idx->n_kev = g.n_kev;
    idx->last_users = n_users;
    idx->last_clusters = g.clusters;
    idx->last_dtype = g.dtype;
    return end_call(idx, s);
  }
  // first time for these arguments: a plain call (it also sizes the
  // workspace), then the same call captured (not run) for later replays
  if ((st = plain()) != MIPS_OK) return st;
  const uint64_t gen = idx->ws.gen;
  MIPS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
  idx->capturing = true;
  st = begin_call(idx, s);
  if (st == MIPS_OK)
    st = method == 0 ? run_bmm(idx, users_dev, n_users, K, out_idx_dev, out_score_dev, s)
                     : run_maximus(idx, users_dev, n_users, K, out_idx_dev, out_score_dev, s);
  idx->capturing = false;
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(s, &graph);
  if (st != MIPS_OK || ec != cudaSuccess || idx->ws.gen != gen) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    if (st != MIPS_OK) return st;
    if (ec != cudaSuccess) return cuda_fail(ec, "stream capture of the call");
    return MIPS_OK;  // the workspace moved during capture: stay uncaptured
  }
  mips_index_s::Graph g;
  const cudaError_t ei = cudaGraphInstantiate(&g.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ei != cudaSuccess) return cuda_fail(ei, "graph instantiation");
  g.method = method;
  g.users = users_dev;
  g.n_users = n_users;
  g.K = K;
  g.out_idx = out_idx_dev;
  g.out_score = out_score_dev;
  g.ws_gen = gen;
  g.cfg_clusters = idx->clusters;
  g.cfg_block = idx->opt.block_items;
  g.cfg_fit = idx->fit_gen;
  for (int i = 0; i < kStages; ++i) {
    g.stage_ran[i] = idx->stage_ran[i];
    g.order[i] = idx->order[i];
  }
  g.n_order = idx->n_order;
  g.last_stage = idx->last_stage;
  g.launches = idx->launches;
  g.n_kev = idx->n_kev;
  g.clusters = idx->last_clusters;
  g.dtype = idx->last_dtype;
  // keep a few; drop those the workspace has outgrown first
  for (size_t i = 0; i < idx->graphs.size();) {
    if (idx->graphs[i].ws_gen != idx->ws.gen) {
      cudaGraphExecDestroy(idx->graphs[i].exec);
      idx->graphs.erase(idx->graphs.begin() + i);
    } else {
      ++i;
    }
  }
  if (idx->graphs.size() >= 8) {
    cudaGraphExecDestroy(idx->graphs.front().exec);
    idx->graphs.erase(idx->graphs.begin());
  }
  idx->graphs.push_back(g);
  return MIPS_OK;
}

mips_status mips_topk_host(mips_index_t idx, const float* users_host, int64_t n_users, int K, int method,
                           int32_t* out_idx_host, double* out_score_host, void* stream) {
  g_err.clear();
  mips_status st = check_call(idx, users_host, n_users, K, out_idx_host, out_score_host);
  if (st != MIPS_OK) return st;
  if (method < 0 || method > 2) return fail(MIPS_ERR_ARG, "method must be 0, 1 or 2");
  cudaStream_t s = (cudaStream_t)stream;
  const int f = idx->f;
  // device staging for this call (stream-ordered allocation)
  const size_t b_users = sizeof(float) * n_users * f;
  const size_t b_idx = sizeof(int32_t) * n_users * K;
  const size_t b_sc = sizeof(double) * n_users * K;
  char* stage = nullptr;
  MIPS_CUDA(cudaMallocAsync((void**)&stage, b_users + b_idx + b_sc + 512, s));
  float* d_users = (float*)stage;
  int32_t* d_idx = (int32_t*)(stage + ((b_users + 255) & ~size_t(255)));
  double* d_sc = (double*)(stage + ((b_users + 255) & ~size_t(255)) + ((b_idx + 255) & ~size_t(255)));
  // The blocked multiply runs in up to eight chunks of users, so that the
  // copies of one chunk overlap the compute of another:
  // all host-to-device copies go first on the copy stream, each chunk's call
  // waits for its own, and each chunk's results go back on the copy stream
  // once its call is done.  Maximus and the selector take the batch whole.
  constexpr int kMaxChunks = 8;
  int64_t bnd[kMaxChunks + 1] = {0, n_users};  // chunk c is users [bnd[c], bnd[c + 1])
  int nch = 1;
  if (method == 0 && n_users >= 2 * 65536) {
    // whole waves of 128-user tiles over the SMs (the score kernel deals its
    // tiles round-robin), a short first chunk so the compute starts early,
    // the partial wave at the end
    const int64_t wave = 128ll * idx->num_sms;
    const int64_t first = std::min<int64_t>(3 * wave, n_users / 2);
    int64_t rest = 6 * wave;
    if (n_users - first > rest * (kMaxChunks - 1))
      rest = round_up((n_users - first + kMaxChunks - 2) / (kMaxChunks - 1), wave);
    bnd[1] = first;
    for (nch = 1; bnd[nch] < n_users; ++nch) bnd[nch + 1] = std::min<int64_t>(bnd[nch] + rest, n_users);
    if (!idx->copy_stream) MIPS_CUDA(cudaStreamCreateWithFlags(&idx->copy_stream, cudaStreamNonBlocking));
  }
  cudaStream_t cs = nch > 1 ? idx->copy_stream : s;
  // [0, nch): users copied, [kMaxChunks, kMaxChunks + nch): chunk done, last: copies back done
  cudaEvent_t ev[2 * kMaxChunks + 1] = {};
  const int ev_back = 2 * kMaxChunks;
  auto cleanup = [&](mips_status r) {
    cudaFreeAsync(stage, s);
    for (cudaEvent_t& e : ev)
      if (e) cudaEventDestroy(e);
    return r;
  };
  cudaError_t e = cudaSuccess;
  if (nch > 1) {
    for (int i = 0; i <= ev_back && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&ev[i], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(ev[ev_back], s);  // the staging allocation is ordered on s
    if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[ev_back], 0);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "copy stream setup"));
  }
  for (int c = 0; c < nch && e == cudaSuccess; ++c) {
    const int64_t u0 = bnd[c], n = bnd[c + 1] - bnd[c];
    e = cudaMemcpyAsync(d_users + u0 * f, users_host + u0 * f, sizeof(float) * n * f, cudaMemcpyHostToDevice, cs);
    if (e == cudaSuccess && nch > 1) e = cudaEventRecord(ev[c], cs);
  }
  if (e != cudaSuccess) return cleanup(cuda_fail(e, "host-to-device copy of users"));
  for (int c = 0; c < nch && st == MIPS_OK; ++c) {
    const int64_t u0 = bnd[c], n = bnd[c + 1] - bnd[c];
    if (nch > 1 && (e = cudaStreamWaitEvent(s, ev[c], 0)) != cudaSuccess) return cleanup(cuda_fail(e, "stream wait"));
    if (method == 0)
      st = mips_topk(idx, d_users + u0 * f, n, K, d_idx + u0 * K, d_sc + u0 * K, stream);
    else if (method == 1)
      st = mips_topk_maximus(idx, d_users, n_users, K, d_idx, d_sc, stream);
    else
      st = mips_select(idx, d_users, n_users, K, d_idx, d_sc, stream, nullptr);
    if (st == MIPS_OK && nch > 1 && (e = cudaEventRecord(ev[kMaxChunks + c], s)) != cudaSuccess)
      return cleanup(cuda_fail(e, "event record"));
  }
  if (st != MIPS_OK) {
    if (nch > 1) cudaStreamSynchronize(cs);  // (the staging is freed on s)
    return cleanup(st);
  }
  for (int c = 0; c < nch && e == cudaSuccess; ++c) {
    const int64_t u0 = bnd[c], n = bnd[c + 1] - bnd[c];
    if (nch > 1) e = cudaStreamWaitEvent(cs, ev[kMaxChunks + c], 0);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out_idx_host + u0 * K, d_idx + u0 * K, sizeof(int32_t) * n * K, cudaMemcpyDeviceToHost, cs);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(out_score_host + u0 * K, d_sc + u0 * K, sizeof(double) * n * K, cudaMemcpyDeviceToHost, cs);
  }
  if (e == cudaSuccess && nch > 1) {  // s resumes (and frees the staging) after the copies back
    e = cudaEventRecord(ev[ev_back], cs);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(s, ev[ev_back], 0);
  }
  if (e != cudaSuccess) {
    if (nch > 1) cudaStreamSynchronize(cs);
    return cleanup(cuda_fail(e, "device-to-host copy of results"));
  }
  st = mips_sync(idx, stream);
  return cleanup(st);
}

mips_status mips_sync(mips_index_t idx, void* stream) {
  if (!idx) return fail(MIPS_ERR_ARG, "null index");
  MIPS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  int h = 0;
  MIPS_CUDA(cudaMemcpy(&h, idx->err_dev, sizeof(int), cudaMemcpyDeviceToHost));
  if (h) MIPS_CUDA(cudaMemset(idx->err_dev, 0, sizeof(int)));
  if (h & DEV_ERR_NONFINITE) return fail(MIPS_ERR_NONFINITE, "an input row holds NaN or Inf");
  if (h & DEV_ERR_TIMEOUT) return fail(MIPS_ERR_TIMEOUT, "a bounded wait inside a kernel gave up");
  if (h & DEV_ERR_INTERNAL) return fail(MIPS_ERR_CUDA, "an internal consistency check failed in a kernel");
  return MIPS_OK;
}

mips_status mips_get_stats(mips_index_t idx, mips_stats* out) {
  if (!idx || !out) return fail(MIPS_ERR_ARG, "null argument");
  if (idx->has_done) MIPS_CUDA(cudaEventSynchronize(idx->done));
  DevStats d;
  MIPS_CUDA(cudaMemcpy(&d, idx->stats_dev, sizeof d, cudaMemcpyDeviceToHost));
  out->cand_emitted = d.cand_emitted;
  out->cand_rescored = d.cand_rescored;
  out->users_overflow = d.users_overflow;
  out->users_fp64 = d.users_fp64;
  out->pairs_scored = d.pairs_scored;
  out->blocks_walked = d.blocks_walked;
  out->select_slow = d.select_slow;
  out->n_users = idx->last_users;
  out->clusters = idx->last_clusters;
  out->dtype = idx->last_dtype;
  out->launches = idx->launches;
  out->pad_ = 0;
  double ms[kStages] = {};
  cudaEvent_t prev = idx->ev[0];
  float t = 0.f;
  for (int q = 0; q < idx->n_order; ++q) {  // in the order the stages ran
    const int i = idx->order[q];
    MIPS_CUDA(cudaEventElapsedTime(&t, prev, idx->ev[1 + i]));
    ms[i] = t;
    prev = idx->ev[1 + i];
  }
  out->ms_prep = ms[ST_PREP];
  out->ms_score = ms[ST_SCORE];
  out->ms_rescore = ms[ST_RESCORE];
  out->ms_kmeans = ms[ST_KMEANS];
  out->ms_bounds = ms[ST_BOUNDS];
  out->ms_sort = ms[ST_SORT];
  out->ms_walk = ms[ST_WALK];
  out->ms_total = 0.0;
  if (idx->last_stage >= 0) {
    MIPS_CUDA(cudaEventElapsedTime(&t, idx->ev[0], idx->ev[1 + idx->last_stage]));
    out->ms_total = t;
  }
  out->ms_kernel = 0.0;
  for (int i = 0; i + 1 < idx->n_kev; i += 2) {
    MIPS_CUDA(cudaEventElapsedTime(&t, idx->kev[i], idx->kev[i + 1]));
    out->ms_kernel += t;
  }
  return MIPS_OK;
}

mips_status mips_get_buffer(mips_index_t idx, const char* name, const void** dev_ptr, int64_t* bytes) {
  if (!idx || !name || !dev_ptr || !bytes) return fail(MIPS_ERR_ARG, "null argument");
  if (!strcmp(name, "perm")) {
    *dev_ptr = idx->perm;
    *bytes = sizeof(int32_t) * idx->n_items;
  } else if (!strcmp(name, "item_nrm")) {
    *dev_ptr = idx->item_nrm;
    *bytes = sizeof(float) * idx->n_items;
  } else if (idx->fit_C > 0 && !strcmp(name, "fit_centroids")) {
    *dev_ptr = idx->fit_cent;
    *bytes = sizeof(float) * (int64_t)idx->fit_C * idx->f;
  } else if (idx->mx.C > 0 && !strcmp(name, "assign")) {
    *dev_ptr = idx->mx.assign;
    *bytes = sizeof(int32_t) * idx->mx.n_users;
  } else if (idx->mx.C > 0 && !strcmp(name, "centroids")) {
    *dev_ptr = idx->mx.cent;
    *bytes = sizeof(float) * (int64_t)idx->mx.C * idx->f;
  } else if (idx->mx.C > 0 && !strcmp(name, "cos_b")) {
    *dev_ptr = idx->mx.cosb;
    *bytes = sizeof(float) * idx->mx.C;
  } else if (idx->mx.C > 0 && !strcmp(name, "bound_sorted")) {
    *dev_ptr = idx->mx.bounds;
    *bytes = sizeof(float) * (int64_t)idx->mx.C * idx->n_items;
  } else if (idx->mx.C > 0 && !strcmp(name, "list")) {
    *dev_ptr = idx->mx.lists;
    *bytes = sizeof(int32_t) * (int64_t)idx->mx.C * idx->n_items;
  } else if (idx->mx.C > 0 && !strcmp(name, "visited")) {
    *dev_ptr = idx->mx.visited;
    *bytes = sizeof(int32_t) * idx->mx.n_users;
  } else if (idx->mx.C > 0 && !strcmp(name, "user_perm")) {
    *dev_ptr = idx->mx.user_perm;
    *bytes = sizeof(int32_t) * idx->mx.n_users;
  } else {
    return fail(MIPS_ERR_ARG, "unknown buffer name (or no Maximus call yet): %s", name);
  }
  return MIPS_OK;
}

void mips_free_index(mips_index_t idx) {
  if (!idx) return;
  if (idx->has_done) cudaEventSynchronize(idx->done);
  for (auto& g : idx->graphs) cudaGraphExecDestroy(g.exec);
  if (idx->ws.base) cudaFree(idx->ws.base);
  if (idx->ws_sel.base) cudaFree(idx->ws_sel.base);
  if (!idx->shares_items) {
    cudaFree(idx->items);
    cudaFree(idx->perm);
    cudaFree(idx->item_nrm);
    cudaFree(idx->items_bf16);
    cudaFree(idx->item_aux);
    cudaFree(idx->item_scale);
  }
  if (idx->copy_stream) cudaStreamDestroy(idx->copy_stream);
  cudaFree(idx->fit_cent);
  cudaFree(idx->err_dev);
  cudaFree(idx->stats_dev);
  if (idx->done) cudaEventDestroy(idx->done);
  for (int i = 0; i <= kStages; ++i)
    if (idx->ev[i]) cudaEventDestroy(idx->ev[i]);
  for (int i = 0; i < 4; ++i)
    if (idx->kev[i]) cudaEventDestroy(idx->kev[i]);
  delete idx;
}

}  // extern "C"
