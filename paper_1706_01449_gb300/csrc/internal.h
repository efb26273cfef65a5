// Host-side declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/mips.h"

namespace mips {

// Bits of the device error word (pinned, host-mapped; sticky until read).
enum DevErr : int {
  DEV_ERR_NONFINITE = 1,   // an input row held NaN or Inf
  DEV_ERR_TIMEOUT = 2,     // a bounded wait in a kernel ran out
  DEV_ERR_INTERNAL = 4,    // an index or size check inside a kernel failed
};

// Counters one call accumulates on the device (read by mips_get_stats).
struct DevStats {
  unsigned long long cand_emitted;    // candidates written by the score kernels
  unsigned long long cand_rescored;   // candidates that passed H >= tau
  unsigned long long users_overflow;  // users whose candidate list overflowed
  unsigned long long users_fp64;      // users resolved by the FP64 tie check
  unsigned long long pairs_scored;    // (user, item) pairs scored (Maximus walk)
  unsigned long long blocks_walked;   // item blocks processed (Maximus walk)
  unsigned long long pad[2];
};

// Round n up to a multiple of m.
inline int64_t round_up(int64_t n, int64_t m) { return (n + m - 1) / m * m; }

// ---- prep kernels (prep.cu) ----------------------------------------------
// Upper bounds on the row norms of an FP32 matrix [n][f].
void launch_row_norm_ub(const float* x, int64_t n, int f, float* nrm_ub, int* err, cudaStream_t s);
// BF16 operand rows with the two bound columns (see prep.cu for the layout).
// role 0 = users (A operand), role 1 = items (B operand).
void launch_quant_bf16(const float* x, int64_t n, int f, int fp, int role, void* out_bf16,
                       int64_t n_rows_out, float2* aux, int* err, cudaStream_t s);
// Gather rows of x by perm into out (out[r] = x[perm[r]]).
void launch_gather_rows(const float* x, const int32_t* perm, int64_t n, int f, float* out, cudaStream_t s);

// ---- FP32 fused score + select (fp32_topk.cu) ------------------------------
struct SelectOut {
  float* tau;          // [n_users]
  int* n_cand;         // [n_users]
  int32_t* cand_pos;   // [n_users][cap]
  float* cand_ub;      // [n_users][cap]
  int cap;
};
bool fp32_supported(int f, int K);
cudaError_t launch_fp32_score_select(const float* users, int64_t n_users, int f, const float* items,
                                     const float* item_nrm_ub, int64_t n_items, int K, SelectOut o,
                                     DevStats* stats, int* err, cudaStream_t s);

// ---- rescore (rescore.cu) -------------------------------------------------
cudaError_t launch_rescore(const float* users, int64_t n_users, int f, const float* items_sorted,
                           const int32_t* perm, const float* item_nrm_ub, int64_t n_items, int K,
                           SelectOut o, int32_t* out_idx, double* out_score, DevStats* stats,
                           int* err, cudaStream_t s);

// Set the calling thread's message returned by mips_last_error().
void set_last_error_message(const char* msg);

}  // namespace mips
