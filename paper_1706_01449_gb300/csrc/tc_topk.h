// Host interface of the tcgen05 fused score + select kernel (tc_topk.cu).
#pragma once
#include <cuda.h>

#include "internal.h"

namespace mips {

constexpr int kMaxStages = 8;
constexpr int kRegTopK = 16;  // K up to this keeps its top-K in registers

struct TcParams {
  int64_t n_users, n_items;
  int f, fp, K;
  int kc;         // K chunks per operand row (fp / row_elems)
  int row_bytes;  // bytes of one chunk row: 32, 64 or 128 (= swizzle span)
  int row_elems;  // BF16 elements of one chunk row
  int swizzle;    // tcgen05 descriptor layout code: 6 = 32B, 4 = 64B, 2 = 128B
  int stages;     // item-tile ring depth
  float g;        // accumulation-error factor used by prep.cu for this fp
};

// Operand row length (BF16 elements) for dimension f: f + 2 bound columns,
// padded to 16, 32 or a multiple of 64 (one swizzle span per chunk).
inline int tc_row_len(int f) {
  int n = f + 2;
  if (n <= 16) return 16;
  if (n <= 32) return 32;
  return (int)round_up(n, 64);
}

// Fill chunking, swizzle and stages for this problem so the shared memory
// fits; returns false if no configuration fits.
bool tc_plan(TcParams& p, int max_smem);
size_t tc_smem_bytes(const TcParams& p);

// K-major BF16 operand map [rows][fp], boxes of row_elems x box_rows rows.
bool tc_make_map(CUtensorMap* map, const void* base, int64_t rows, int fp, int row_bytes, int box_rows);
int tc_users_per_tile();  // rows of a user tile (MMA M)
int tc_items_per_tile();  // rows of an item tile (MMA N)

cudaError_t launch_tc_score_select(const CUtensorMap* map_users, const CUtensorMap* map_items, const TcParams& p,
                                   SelectOut o, const float2* user_aux, const float2* item_aux, DevStats* stats,
                                   int* err, int grid, cudaStream_t s);

}  // namespace mips
