// Host interface of the tcgen05 fused score + select kernel (tc_topk.cu).
#pragma once
#include <cuda.h>

#include "internal.h"

namespace mips {

constexpr int kMaxStages = 8;
constexpr int kRegTopK = 16;  // K up to this keeps its top-K in registers

// Work list for the kernel's second mode: work item w scores the 128 users
// at A rows [a_row[w], a_row[w] + 128) against the item tiles t in
// [t_begin[w], t_end[w]) of the list whose rank 0 is B row b_row[w], into the
// user's candidate sub-lists l_base[w] and l_base[w] + 1 (of SelectOut.lists).
// Maximus walk (restore = 1): a work item with t_begin > 0 continues the
// select state a first pass left in those sub-lists.  Item-chunked blocked
// multiply (restore = 0): every work item starts afresh (seeded by its first
// tile).  Without a work list (mode 0, the blocked multiply) work item w is
// user tile w against every item tile, and A and B rows are user ids and
// item positions themselves.
struct TcWork {
  const int* a_row;
  const int* b_row;
  const int* t_begin;
  const int* t_end;
  const int* n_work;        // device count of work items
  const int32_t* row_user;  // A row -> user id, -1 for padding rows
  const int32_t* item_pos;  // B row -> item position
  const int* l_base;        // first sub-list of each work item (null: 0)
  int restore;
  int* next;                // zeroed work counter: CTAs claim items dynamically (null: round-robin)
  int64_t n_items_pos;      // item positions in item_pos lie in [0, n_items_pos)
};

struct TcParams {
  int64_t n_users, n_items;
  int f, fp, K;   // fp: operand row length in elements
  int esize;      // bytes per operand element: 2 (BF16, kind::f16) or 1 (FP8 E4M3, kind::f8f6f4)
  // FP8 only: every accumulator entry times user_scale[u] * item_scale[0]
  // (per-row user scale, one item scale) is the score in input units
  const float* user_scale;
  const float* item_scale;
  int kc;         // full K chunks per operand row
  int row_bytes;  // bytes of one full chunk row: 32, 64 or 128 (= swizzle span)
  int row_elems;  // BF16 elements of one full chunk row
  int swizzle;    // tcgen05 descriptor layout code: 6 = 32B, 4 = 64B, 2 = 128B
  int tail_bytes;    // a last, narrower chunk after kc 128-byte ones: 0, 32 or 64 bytes
  int tail_swizzle;  // its layout code (6 or 4)
  int b_split;       // 1, or 2: an item tile is loaded and multiplied as two 128-row halves
                     // (ring stages of half a tile, N = 128 MMAs), when whole tiles do not fit
  int heap_global;   // K > 16 and the heap does not fit shared memory: it lives in heap_mem,
  float* heap_mem;   // [grid][K][256] floats of global memory (L2-resident), set by the caller
  int stages;     // item-tile ring depth
  float g;
  int mode;       // 0: blocked multiply, 1: work list
  TcWork work;
  unsigned long long wait_ns;  // limit of every bounded wait (0: 1 s)
  int test_withhold;           // tests of the bounded waits: the producer publishes no work item
};

// Operand row length (BF16 elements) for dimension f: f + 2 bound columns,
// padded to 16, 32 or 64, or above 64 to whole 64-element chunks plus a
// 16- or 32-element tail chunk when that covers the rest (f = 128: 128 + 16).
inline int tc_row_len(int f) {
  const int n = f + 2;
  if (n <= 16) return 16;
  if (n <= 32) return 32;
  if (n <= 64) return 64;
  const int full = n / 64 * 64, rem = n - full;
  if (rem == 0) return full;
  if (rem <= 16) return full + 16;
  if (rem <= 32) return full + 32;
  return full + 64;
}

// FP8 operand row length (E4M3 elements = bytes) for dimension f: f + 2
// bound columns padded to 32, 64 or 128, or above 128 to whole 128-element
// chunks plus a 32- or 64-element tail chunk when that covers the rest.
inline int tc_row_len8(int f) {
  const int n = f + 2;
  if (n <= 32) return 32;
  if (n <= 64) return 64;
  if (n <= 128) return 128;
  const int full = n / 128 * 128, rem = n - full;
  if (rem == 0) return full;
  if (rem <= 32) return full + 32;
  if (rem <= 64) return full + 64;
  return full + 128;
}

// Fill chunking, swizzle and stages for this problem (p.fp, p.esize) so the
// shared memory fits; returns false if no configuration fits.
bool tc_plan(TcParams& p, int max_smem);
size_t tc_smem_bytes(const TcParams& p);

// K-major operand map [rows][fp] of esize-byte elements (2: BF16, 1: bytes),
// boxes of row_bytes / esize elements x box_rows rows, swizzled by row_bytes
// (32, 64 or 128).
bool tc_make_map(CUtensorMap* map, const void* base, int64_t rows, int fp, int row_bytes, int box_rows,
                 int esize = 2);
// The full-chunk map and, when p.tail_bytes > 0, the tail-chunk map (else a
// copy of the first) of one operand.
bool tc_make_maps(CUtensorMap* map, CUtensorMap* tail, const void* base, int64_t rows, const TcParams& p,
                  int box_rows);
int tc_users_per_tile();  // rows of a user tile (MMA M)
int tc_items_per_tile();  // rows of an item tile (the select's unit)
int tc_items_box(const TcParams& p);  // rows of one item load (tile / b_split): the item maps' box

cudaError_t launch_tc_score_select(const CUtensorMap* map_users, const CUtensorMap* map_users_tail,
                                   const CUtensorMap* map_items, const CUtensorMap* map_items_tail, const TcParams& p,
                                   SelectOut o, const float2* user_aux, const float2* item_aux, DevStats* stats,
                                   int* err, int grid, cudaStream_t s);

}  // namespace mips
