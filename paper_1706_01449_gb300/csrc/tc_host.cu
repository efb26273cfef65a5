// Host helpers of the tcgen05 kernel: tiling plan and TMA tensor maps.
#include <cstring>

#include "tc_topk.h"

namespace mips {

bool tc_plan(TcParams& p, int max_smem) {
  if (p.esize != 1) p.esize = 2;
  const int rb = p.fp * p.esize;  // bytes of one operand row
  p.row_bytes = rb <= 32 ? 32 : (rb <= 64 ? 64 : 128);
  p.row_elems = p.row_bytes / p.esize;
  p.kc = p.fp / p.row_elems;
  p.swizzle = p.row_bytes == 32 ? 6 : (p.row_bytes == 64 ? 4 : 2);
  p.tail_bytes = (p.fp - p.kc * p.row_elems) * p.esize;  // 0, 32 or 64 (tc_row_len, tc_row_len8)
  p.tail_swizzle = p.tail_bytes == 32 ? 6 : 4;
  p.g = (float)(p.fp + 4) * 9.5367432e-07f + (float)p.f * 8.8817842e-16f;
  // whole item tiles per ring stage if two stages fit, else half tiles;
  // for K > 16, the top-K heap in shared memory if it fits, else in global
  // memory
  for (int hg = 0; hg <= (p.K > kRegTopK ? 1 : 0); ++hg) {
    p.heap_global = hg;
    for (int split = 1; split <= 2; ++split) {
      p.b_split = split;
      for (int st = kMaxStages; st >= 2; --st) {
        p.stages = st;
        if (tc_smem_bytes(p) <= (size_t)max_smem) return true;
      }
    }
  }
  p.heap_global = 0;
  p.b_split = 1;
  p.stages = 2;
  return false;
}

namespace {
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* ptr = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)ptr;
  }
  return fn;
}
}  // namespace

bool tc_make_maps(CUtensorMap* map, CUtensorMap* tail, const void* base, int64_t rows, const TcParams& p,
                  int box_rows) {
  if (!tc_make_map(map, base, rows, p.fp, p.row_bytes, box_rows, p.esize)) return false;
  if (p.tail_bytes == 0) {
    *tail = *map;
    return true;
  }
  return tc_make_map(tail, base, rows, p.fp, p.tail_bytes, box_rows, p.esize);
}

bool tc_make_map(CUtensorMap* map, const void* base, int64_t rows, int fp, int row_bytes, int box_rows, int esize) {
  EncodeTiledFn enc = encode_fn();
  if (!enc) return false;
  memset(map, 0, sizeof(*map));
  if (esize != 1) esize = 2;
  cuuint64_t dims[2] = {(cuuint64_t)fp, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)fp * esize};
  cuuint32_t box[2] = {(cuuint32_t)(row_bytes / esize), (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1u, 1u};
  CUtensorMapSwizzle sw = row_bytes == 32 ? CU_TENSOR_MAP_SWIZZLE_32B
                                          : (row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B);
  const CUtensorMapDataType dt = esize == 1 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
  CUresult r = enc(map, dt, 2, const_cast<void*>(base), dims, strides, box, estr,
                   CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                   CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

}  // namespace mips
