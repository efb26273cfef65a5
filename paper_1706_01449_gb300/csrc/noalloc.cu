// mips_topk_noalloc: exact top-K through the FP32 fused score + select and
// the exact rescore, with every byte of scratch taken from one static device
// array instead of device allocations.
//
// Who needs this: code that must not call cudaMalloc / cudaFree -- for
// example a caller running inside a custom device-memory allocator or an
// out-of-memory handler (re-entering the allocator is not allowed there), a
// latency-critical serving path (cudaFree can synchronise the whole device),
// or a process whose memory budget is fixed up front and owned by someone
// else.  Such a caller passes its own device inputs and outputs; the scratch
// lives in g_scratch below, reserved once when the library is loaded.
//
// Limits and sharing (also stated in include/mips.h):
//   * the scratch is kNoAllocScratchBytes (32 MiB) on every GPU that loads
//     the library, held until the process exits;
//   * a call needs 8 n_items + n_users (28 + 28 cap) bytes plus at most 5 KiB
//     of counters and alignment padding, cap = max(4K + 96, K (2 + ln(n_items
//     / K)) + 96) candidate slots per user (the FP32 blocked multiply's list
//     capacity: the expected number of K-th-largest records of a stream of
//     n_items scores, with room to spare), and is rejected with MIPS_ERR_ARG
//     beyond that; a user whose candidates still overflow its list is scored
//     exhaustively by the rescore (exact, slower);
//   * every call uses the same array: calls that overlap on the GPU (two
//     streams, two host threads) race and corrupt each other's results, so
//     callers must serialise them;
//   * the array keeps the last call's contents; the parts that must start
//     at zero (counters, error word) are cleared by each call.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "internal.h"

namespace mips {

namespace {

constexpr size_t kNoAllocScratchBytes = 32ull << 20;

// Host code must not use this name as a device address: its address on each
// device comes from cudaGetSymbolAddress (see scratch_on_current_device).
static __device__ __align__(256) unsigned char g_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_dev[kMaxDevices] = {};

// Once per device, with that device current: look up the device address of
// g_scratch.
cudaError_t scratch_on_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_dev[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_dev[dev] = p;
  }
  *out = g_scratch_dev[dev];
  return cudaSuccess;
}

__global__ void iota_kernel(int32_t* p, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = (int32_t)i;
}

size_t up256(size_t b) { return (b + 255) & ~size_t(255); }

// Candidate slots per user (see the size rule above).
int list_cap(int K, int64_t n) {
  const double r = n > K ? std::log((double)n / K) : 0.0;
  return std::max(4 * K + 96, (int)std::min<int64_t>((int64_t)std::ceil(K * (2.0 + r)) + 96, n + 96));
}

// message for mips_last_error(), formatted locally then handed over
mips_status report(mips_status st, const char* fmt, ...) {
  char buf[256];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_last_error_message(buf);
  return st;
}

}  // namespace

}  // namespace mips

using namespace mips;

extern "C" {

mips_status mips_topk_noalloc(const float* items_dev, int64_t n_items, const float* users_dev, int64_t n_users, int f,
                              int K, int32_t* out_idx_dev, double* out_score_dev, void* stream) {
  set_last_error_message("");
  if (!items_dev || !users_dev || !out_idx_dev || !out_score_dev) return report(MIPS_ERR_ARG, "null buffer");
  if (f < 1 || f > 128 || n_items < 1 || n_items >= (1ll << 31) || n_users < 1 || n_users >= (1ll << 31) || K < 1 ||
      K > 128 || K > n_items)
    return report(MIPS_ERR_ARG, "size out of range (1<=f<=128, 1<=K<=min(n_items,128), n>=1)");
  const int cap = list_cap(K, n_items);
  const size_t slots = (size_t)n_users * cap;
  const size_t need = up256(sizeof(DevStats)) + up256(sizeof(int)) * 3 + up256(4 * (size_t)n_items) * 2 +
                      up256(4 * (size_t)n_users) * 3 + up256(8 * (size_t)n_users) * 2 + up256(4 * slots) * 5 +
                      up256(8 * slots);
  if (need > kNoAllocScratchBytes)
    return report(MIPS_ERR_ARG, "problem needs %zu scratch bytes, the static scratch holds %zu (use fewer users per call)",
                  need, kNoAllocScratchBytes);
  void* base = nullptr;
  cudaError_t e = scratch_on_current_device(&base);
  if (e != cudaSuccess) return report(MIPS_ERR_CUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)stream;
  char* p = (char*)base;
  DevStats* stats = (DevStats*)p;
  p += up256(sizeof(DevStats));
  int* err = (int*)p;
  p += up256(sizeof(int));
  int32_t* perm = (int32_t*)p;
  p += up256(4 * (size_t)n_items);
  float* nrm = (float*)p;
  p += up256(4 * (size_t)n_items);
  SelectOut so;
  so.tau = (float*)p;
  p += up256(4 * (size_t)n_users);
  so.n_cand = (int*)p;
  p += up256(4 * (size_t)n_users);
  so.cand_pos = (int32_t*)p;
  p += up256(4 * (size_t)n_users * cap);
  so.cand_ub = (float*)p;
  p += up256(4 * (size_t)n_users * cap);
  so.cap = cap;
  so.lists = 1;
  so.topl = nullptr;
  so.topl_sorted = 0;
  so.ovf_list = (int32_t*)p;
  p += up256(4 * (size_t)n_users);
  so.ovf_count = (int*)p;
  p += up256(sizeof(int));
  so.work = (uint32_t*)p;
  p += up256(4 * slots);
  so.work_count = (int*)p;
  p += up256(sizeof(int));
  so.cand_sc = (double*)p;
  p += up256(8 * slots);
  so.w_id = (int32_t*)p;
  p += up256(4 * slots);
  so.w_nrm = (float*)p;
  p += up256(4 * slots);
  so.u_work = (int*)p;
  p += up256(8 * (size_t)n_users);
  so.tau_final = (float*)p;

  // counters and the error word must start at zero; the rest is overwritten
  e = cudaMemsetAsync(base, 0, up256(sizeof(DevStats)) + up256(sizeof(int)), s);
  if (e == cudaSuccess) {
    iota_kernel<<<(unsigned)((n_items + 255) / 256), 256, 0, s>>>(perm, n_items);
    launch_row_norm_ub(items_dev, n_items, f, nrm, err, s);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = launch_fp32_score_select(users_dev, n_users, f, items_dev, nrm, n_items, K, so, stats, err, s);
  if (e == cudaSuccess)
    e = launch_rescore(users_dev, n_users, f, items_dev, perm, nrm, n_items, K, so, out_idx_dev, out_score_dev, stats,
                       err, s);
  int h_err = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h_err, err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return report(MIPS_ERR_CUDA, "CUDA error: %s", cudaGetErrorString(e));
  if (h_err & DEV_ERR_NONFINITE) return report(MIPS_ERR_NONFINITE, "an input row holds NaN or Inf");
  if (h_err) return report(MIPS_ERR_CUDA, "internal consistency check failed in a kernel");
  return MIPS_OK;
}

}  // extern "C"
