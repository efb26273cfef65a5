// Host-side declarations shared by the library's translation units.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "mips.h"  // include/ is on the include path

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
  unsigned long long select_slow;     // warp-level slow-path entries of the select
  unsigned long long pad;
};

// Maximus lists are sorted by this many leading bits of the bound key.
constexpr int kListKeyBits = 16;

// Unsigned key whose ascending order is the float's DESCENDING order.
__host__ __device__ inline uint32_t float_desc_key(float x) {
#ifdef __CUDA_ARCH__
  const uint32_t b = __float_as_uint(x);
#else
  uint32_t b;
  __builtin_memcpy(&b, &x, 4);
#endif
  const uint32_t asc = (b & 0x80000000u) ? ~b : (b | 0x80000000u);
  return ~asc;
}

// Multiprocessor count of the current device (queried once per device);
// launch sizes of the grid-stride helper kernels scale with it.
int sm_count();

// Round n up to a multiple of m.
inline int64_t round_up(int64_t n, int64_t m) { return (n + m - 1) / m * m; }

// ---- prep kernels (prep.cu) ----------------------------------------------
// Upper bounds on the row norms of an FP32 matrix [n][f].
void launch_row_norm_ub(const float* x, int64_t n, int f, float* nrm_ub, int* err, cudaStream_t s);
// BF16 operand rows with the two bound columns (see prep.cu for the layout).
// role 0 = users (A operand), role 1 = items (B operand).
void launch_quant_bf16(const float* x, int64_t n, int f, int fp, int role, void* out_bf16,
                       int64_t n_rows_out, float2* aux, int* err, cudaStream_t s);
// E4M3 operand rows (prep.cu): role 0 users (row_scale[row] = their scale),
// role 1 items (scale *item_scale, from launch_fp8_item_scale).
void launch_quant_fp8(const float* x, int64_t n, int f, int fp, int role, const float* item_scale, void* out,
                      int64_t n_rows_out, float2* aux, float* row_scale, int* err, cudaStream_t s);
void launch_fp8_item_scale(const float* item_nrm, int64_t n, float* item_scale, cudaStream_t s);
// dst rows[r] <- src row r, for [n][K] top-K outputs.
void launch_scatter_topk(const int32_t* src_idx, const double* src_sc, const int32_t* rows, int64_t n, int K,
                         int32_t* dst_idx, double* dst_sc, cudaStream_t s);
// Gather rows of x by perm into out (out[r] = x[perm[r]]).
void launch_gather_rows(const float* x, const int32_t* perm, int64_t n, int f, float* out, cudaStream_t s);
// Sample split of the selector: keys 0 for the ns users whose image under
// the affine permutation (a u + b) mod n is below ns, else 1; ids = u.
void launch_sample_keys(int64_t n, uint64_t a, uint64_t b, int64_t ns, uint32_t* keys, int32_t* ids, cudaStream_t s);
// Work list of the item-chunked blocked multiply (work5: 5 arrays of
// n_ut * nch ints: a_row, b_row, t_begin, t_end, l_base) and identity maps.
void launch_bmm_chunks(int n_ut, int nch, int tpc, int n_it, int64_t n_users, int64_t n_items_pad, int* work5,
                       int* n_work, int32_t* row_user, int32_t* item_pos, cudaStream_t s);

// ---- FP32 fused score + select (fp32_topk.cu) ------------------------------
// Candidate output of a score kernel: `lists` sub-lists per user (one per
// select thread serving the user), sub-list l of user u at index u*lists+l.
struct SelectOut {
  float* tau;          // [n_users * lists] final threshold of each sub-list
  int* n_cand;         // [n_users * lists] candidates emitted (may exceed cap)
  int32_t* cand_pos;   // [n_users * lists][cap] item positions
  float* cand_ub;      // [n_users * lists][cap] upper bounds H
  int cap;             // capacity of one sub-list
  int lists;
  // optional: the K largest lower bounds each sub-list's select kept
  // ([n_users * lists][K]); with two sub-lists the rescore's threshold is the
  // K-th largest of their union (entries are distinct items)
  float* topl;
  int topl_sorted;     // 1: each topl row is sorted descending (the tensor-core select writes them so)
  // users whose candidate list overflowed, for the exhaustive rescore
  int32_t* ovf_list;   // [n_users]
  int* ovf_count;      // one counter, zero before the rescore
  // rescore scratch: the work list (the slots of the candidates that reach
  // their user's threshold, each user's run contiguous), then per work entry
  // w its exact score, the item's id and norm bound (written in work order,
  // so the final select reads its user's run in one piece)
  uint32_t* work;      // [n_users * lists * cap] candidate slot of entry w
  int* work_count;     // one counter
  double* cand_sc;     // [n_users * lists * cap] exact score of entry w
  float* tau_final;    // [n_users][2]: entry 2u + 1 = ||u||^2 as the collect kernel summed it (2u unused)
  // optional ([n_users], zeroed): the largest threshold any select thread of
  // the user published, as order-preserving bits; threads scanning other
  // item chunks of the same user raise their filter to it
  unsigned* tau_glob = nullptr;
  int32_t* w_id = nullptr;   // [n_users * lists * cap] item id (perm) of entry w; -1: a bad position
  float* w_nrm = nullptr;    // [n_users * lists * cap] the item's norm bound
  int* u_work = nullptr;     // [n_users][2] the user's run in the work list: first entry, count
};

// Bytes of rescore scratch (ovf list, work list, scores, thresholds, counters)
// for n_users users with `lists` sub-lists of `cap` candidates each.
inline size_t rescore_scratch_bytes(int64_t n_users, int lists, int cap) {
  const size_t slots = (size_t)n_users * lists * cap;
  return 4 * (size_t)n_users + 4 * slots + 8 * slots + 8 * (size_t)n_users + 8 * slots + 8 * (size_t)n_users + 2048;
}
bool fp32_supported(int f, int K);
cudaError_t launch_fp32_score_select(const float* users, int64_t n_users, int f, const float* items,
                                     const float* item_nrm_ub, int64_t n_items, int K, SelectOut o,
                                     DevStats* stats, int* err, cudaStream_t s);

// ---- rescore (rescore.cu) -------------------------------------------------
cudaError_t launch_rescore(const float* users, int64_t n_users, int f, const float* items_sorted,
                           const int32_t* perm, const float* item_nrm_ub, int64_t n_items, int K,
                           SelectOut o, int32_t* out_idx, double* out_score, DevStats* stats,
                           int* err, cudaStream_t s);

// ---- radix sort (sort.cu) --------------------------------------------------
// Temp bytes for radix_sort_pairs over n_seg segments of n elements.
size_t radix_sort_temp_bytes(int64_t n, int n_seg);
// Stable ascending sort of keys[begin_bit, end_bit) with values, per segment;
// the sorted arrays end up in (keys, vals) (pointers are swapped per pass).
cudaError_t radix_sort_pairs(uint32_t*& keys, int32_t*& vals, uint32_t*& keys_alt, int32_t*& vals_alt, int64_t n,
                             int n_seg, int begin_bit, int end_bit, uint32_t* temp, cudaStream_t s, int* launches);
// keys[i] = float_desc_key(x[i]); iota[i] = i % seg_len (if iota != null).
cudaError_t make_float_desc_keys(const float* x, int64_t n, uint32_t* keys, int32_t* iota, int64_t seg_len,
                                 cudaStream_t s);

// ---- tensor-core k-means assignment (kmeans_tc.cu) ------------------------
// BF16 operand row length: f + 1 (the bias column) in whole 64-element chunks.
int km_tc_row_len(int f);
size_t km_tc_smem_bytes(int f, int C);
// Whether C centroids of dimension f stay resident in max_smem bytes.
bool km_tc_fits(int f, int C, int max_smem);
// users_km [n_users][km_tc_row_len(f)] = [u, 1, 0 ..] in BF16.
cudaError_t km_tc_users(const float* users, int64_t n_users, int f, uint16_t* users_km, cudaStream_t s);
// One assignment step: cent_km [C][row len] is written from cent and hn2
// (= ||c_j||^2 / 2), then assign[u] = argmax_j of the BF16 u . c_j - hn2_j.
cudaError_t km_tc_assign(const uint16_t* users_km, int64_t n_users, int f, const float* cent, const float* hn2, int C,
                         uint16_t* cent_km, int32_t* assign, int* err, int max_smem, cudaStream_t s);

// Buffers of the tensor-core assignment; users_km null: the CUDA-core kernel.
struct KmTc {
  uint16_t* users_km = nullptr;  // [n_users][km_tc_row_len(f)]
  uint16_t* cent_km = nullptr;   // [C][km_tc_row_len(f)]
  int* err = nullptr;
  int max_smem = 0;
};

// ---- Maximus (maximus.cu) -------------------------------------------------
cudaError_t maximus_kmeans(const float* users, int64_t n_users, int f, int C, int iters, const int64_t* init_ids_dev,
                           float* cent, float* hn2, int32_t* assign, unsigned long long* sums, unsigned int* counts,
                           uint32_t* absmax, float* scale, bool spherical, const KmTc& tc, cudaStream_t s,
                           int* launches);
// Assignment of the call's users to fitted centroids (cent_fit [C_fit][f]),
// then the used clusters packed into slots 0.. of cent [C_eff][f] and the
// assignment renumbered to those slots (C_eff >= the number of used clusters).
cudaError_t maximus_assign_fitted(const float* users, int64_t n_users, int f, const float* cent_fit, int C_fit,
                                  float* hn2_fit, int32_t* assign, int* used, int* remap, float* cent, int C_eff,
                                  const KmTc& tc, cudaStream_t s, int* launches);
cudaError_t maximus_bounds(const float* users, int64_t n_users, int f, const int32_t* assign, const float* cent, int C,
                           const float* items, const float* item_nrm, int64_t n_items, uint32_t* cosb_ord,
                           uint32_t* keys, int32_t* vals, float* cosb_f, cudaStream_t s, int* launches);
cudaError_t maximus_group(const int32_t* assign, int64_t n_users, int C, uint32_t* keys, int32_t* ids, uint32_t* keys_alt,
                          int32_t* ids_alt, uint32_t* temp, int* counts, int* offsets, int* tile_off,
                          int32_t** user_perm, cudaStream_t s, int* launches);
cudaError_t maximus_walk(const float* users, int f, const float* items, const float* item_nrm, int64_t n_items,
                         const int32_t* lists, const float* bounds, const int32_t* user_perm, const int* offsets,
                         const int* tile_off, int C, int K, SelectOut o, int32_t* visited, int* work_counter,
                         DevStats* stats, int* err, int num_sms, cudaStream_t s);
cudaError_t maximus_keys_to_bounds(const uint32_t* keys, int64_t n, float* out, cudaStream_t s);
// tensor-core walk: operand layouts and pass-1 work list / pass-2 work list
// Tensor-core Maximus walk: layout and buffers (device pointers into the
// library's workspace).  A rows: users grouped by cluster, each cluster
// starting at a 128-aligned row; B rows: each cluster's item list copied in
// bound order, n_pad rows per cluster.
struct MxTc {
  int C = 0, fp = 0, t1 = 0, n_it = 0;
  int esize = 2;  // bytes per operand element (2: BF16, 1: FP8)
  int64_t n_users = 0, n_items = 0, n_pad = 0, n_rows_max = 0, max_work = 0;
  const int* counts = nullptr;       // [C] users per cluster
  const int* offsets = nullptr;      // [C + 1] first sorted rank of each cluster
  int* pad_off = nullptr;            // [C + 1] first A row of each cluster
  int32_t* row_user = nullptr;       // [n_rows_max] user of each A row, -1 = padding
  int32_t* user_row = nullptr;       // [n_users]
  const void* users_bf16 = nullptr;  // [n_users][fp] in user order
  void* a_rows = nullptr;            // [n_rows_max][fp]
  void* b_rows = nullptr;            // [C * n_pad][fp]
  float2* aux_c = nullptr;           // [C * n_pad] bound columns of the B rows
  int32_t* pos_c = nullptr;          // [C * n_pad] item positions of the B rows
  int* w1 = nullptr;                 // [4][max_work] a_row, b_row, t_begin, t_end (pass 1)
  int* w2 = nullptr;                 // [4][max_work] (pass 2, longest first)
  int* n_work = nullptr;             // [3] work items of pass 1, pass 2; pass-2 claim counter
  int* work_end = nullptr;           // [max_work] item tiles each A tile walks
  int32_t* ustop = nullptr;          // [n_users] item tiles each user needs
  int* cl_end = nullptr;             // [C] item tiles any member of the cluster needs
  const void* items_bf16 = nullptr;  // set by mx_tc_prepare: the sources of the list copies
  const float2* item_aux = nullptr;
  const int32_t* lists = nullptr;
  uint32_t* ukeys[2] = {};           // [n_users] user regroup sort
  int32_t* uvals[2] = {};
  uint32_t* wkeys[2] = {};           // [max_work] pass-2 work sort
  int32_t* wvals[2] = {};
  uint32_t* temp = nullptr;          // radix sort scratch for max(n_users, max_work) keys
};
// k-means initial centroid ids: C distinct users of n (seeded Floyd draw on
// the device; chosen_bits: scratch of (n + 31) / 32 words).
cudaError_t draw_init_ids(int64_t n, int C, uint64_t seed, uint32_t* chosen_bits, int64_t* ids, cudaStream_t s);
// Whether the regroup sort key (cluster, item tiles) fits 32 bits.
bool mx_tc_regroup_fits(int C, int64_t n_items);
// A rows, the B rows pass 1 reads, pass-1 work list.
cudaError_t mx_tc_prepare(MxTc& m, const int32_t* user_perm, const void* items_bf16, const float2* item_aux,
                          const int32_t* lists, cudaStream_t s, int* launches);
// After pass 1: each user's stop tile, the B rows pass 2 reads, users
// regrouped by stop tile within their cluster (new A rows, *user_perm), the
// pass-2 work list, visited counts.
cudaError_t mx_tc_pass2(MxTc& m, const int32_t* assign, const float2* user_aux, const float* bounds, SelectOut o, int K,
                        int32_t** user_perm, int32_t* visited, DevStats* stats, cudaStream_t s, int* launches);

// Worker handle sharing an index's item arrays (own workspace and events).
mips_index_t index_worker_clone(mips_index_t src);
int index_f(mips_index_t idx);
int64_t index_n_items(mips_index_t idx);
// Workspace bytes a mips_topk (method 0) or mips_topk_maximus (method 1)
// call on n_users users with this K takes: the calls' own layout, run
// without device work (the index must be idle on the host side).
size_t call_workspace_bytes(mips_index_t idx, int64_t n_users, int K, int method);
// Bytes of workspace the last call took, and the capacity the index holds.
size_t index_workspace_used(mips_index_t idx);
size_t index_workspace_held(mips_index_t idx);
// Free the index's workspace (stream-ordered on s; the next call allocates
// again).
cudaError_t index_release_workspace(mips_index_t idx, cudaStream_t s);

// Set the calling thread's message returned by mips_last_error().
void set_last_error_message(const char* msg);

}  // namespace mips
