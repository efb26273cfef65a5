// Fused FP32 blocked multiply + top-K candidate select on CUDA cores
// (Sec. II-C "Blocked Matrix Multiply", the paper's BMM: every user against
// every item, here with the per-user selection fused so the |U| x |I| score
// matrix never leaves the chip).
//
// One thread owns one user: the user's vector lives in registers, item tiles
// of 32 rows are staged in shared memory with cp.async (double-buffered) and
// read back as warp-wide broadcasts, four items at a time.  Each FP32 dot
// product s~ carries a rigorous error bound:
//   |s~ - u^T i| <= gamma ||u|| ||i||,  gamma = (f + 4) 2^-23,
// so H = s~ + gamma nhat_u nhat_i is an upper bound and L = s~ - gamma ... a
// lower bound on the exact score (and on the FP64 definition's value).  The
// per-user select keeps tau = K-th largest L and emits every item with
// H >= tau; the rescore kernel ranks the survivors exactly.
#include "common.cuh"

namespace mips {

namespace {

constexpr int kThreads = 128;  // users per block
constexpr int kTileItems = 32; // items per shared-memory tile

__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gmem_src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

template <int FP>
__device__ __forceinline__ void load_tile(float* tile, float* nrm, const float* __restrict__ items,
                                          const float* __restrict__ item_nrm, int64_t n_items, int f,
                                          int64_t first) {
  const int tid = threadIdx.x;
  const int64_t rows = min((int64_t)kTileItems, n_items - first);
  const int total = (int)rows * f;
  const float* src = items + first * f;
  for (int e = tid; e < total; e += kThreads) {
    int r = e / f, k = e - r * f;
    cp_async4(tile + r * FP + k, src + e);
  }
  if (tid < rows) cp_async4(nrm + tid, item_nrm + first + tid);
  cp_async_commit();
}

template <int FP>
__global__ void __launch_bounds__(kThreads, 2)
    fp32_score_select_kernel(const float* __restrict__ users, int64_t n_users, int f,
                             const float* __restrict__ items, const float* __restrict__ item_nrm,
                             int64_t n_items, int K, SelectOut o, DevStats* stats, int* err) {
  extern __shared__ float4 smem4[];
  float* tiles = reinterpret_cast<float*>(smem4);     // [2][kTileItems][FP]
  float* nrms = tiles + 2 * kTileItems * FP;           // [2][kTileItems]
  float* heap_base = nrms + 2 * kTileItems;            // [K][kThreads]

  const int tid = threadIdx.x;
  const int64_t u = (int64_t)blockIdx.x * kThreads + tid;
  const bool active = u < n_users;

  // zero both tiles once: padding columns f..FP-1 stay zero forever
  for (int e = tid; e < 2 * kTileItems * FP; e += kThreads) tiles[e] = 0.f;
  __syncthreads();

  float ur[FP];
  float ss = 0.f;
#pragma unroll
  for (int k = 0; k < FP; ++k) {
    ur[k] = (active && k < f) ? users[u * f + k] : 0.f;
    ss = __fmaf_rn(ur[k], ur[k], ss);
  }
  if (active && !isfinite(ss)) atomicOr(err, DEV_ERR_NONFINITE);
  const float nu = __fsqrt_rn(ss) * (1.0f + (float)(f + 2) * 1.1920929e-07f);
  const float gu = fp32_score_gamma(f) * nu;

  UserSelect st;
  st.tau = active ? kNegInf : __int_as_float(0x7f800000);  // inactive: never emit
  st.n_cand = 0;
  st.heap = heap_base + tid;
  st.stride = kThreads;
  st.K = K;
  st.cap = o.cap;
  st.cand_pos = o.cand_pos + (active ? u : 0) * (int64_t)o.cap;
  st.cand_ub = o.cand_ub + (active ? u : 0) * (int64_t)o.cap;
  heap_init(st.heap, st.stride, K);

  const int64_t n_tiles = (n_items + kTileItems - 1) / kTileItems;
  load_tile<FP>(tiles, nrms, items, item_nrm, n_items, f, 0);

  for (int64_t t = 0; t < n_tiles; ++t) {
    const int buf = (int)(t & 1);
    cp_async_wait_all();
    __syncthreads();  // tile t visible; everyone done with tile t-1
    if (t + 1 < n_tiles)
      load_tile<FP>(tiles + (buf ^ 1) * kTileItems * FP, nrms + (buf ^ 1) * kTileItems, items,
                    item_nrm, n_items, f, (t + 1) * kTileItems);
    const float* tile = tiles + buf * kTileItems * FP;
    const float* nrm = nrms + buf * kTileItems;
    const int64_t first = t * kTileItems;
    const int rows = (int)min((int64_t)kTileItems, n_items - first);

    for (int j0 = 0; j0 < rows; j0 += 4) {
      float acc0 = 0.f, acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
      const float4* r0 = reinterpret_cast<const float4*>(tile + (j0 + 0) * FP);
      const float4* r1 = reinterpret_cast<const float4*>(tile + (j0 + 1) * FP);
      const float4* r2 = reinterpret_cast<const float4*>(tile + (j0 + 2) * FP);
      const float4* r3 = reinterpret_cast<const float4*>(tile + (j0 + 3) * FP);
#pragma unroll
      for (int q = 0; q < FP / 4; ++q) {
        float4 a = r0[q], b = r1[q], c = r2[q], d = r3[q];
        acc0 = __fmaf_rn(ur[4 * q + 0], a.x, acc0);
        acc1 = __fmaf_rn(ur[4 * q + 0], b.x, acc1);
        acc2 = __fmaf_rn(ur[4 * q + 0], c.x, acc2);
        acc3 = __fmaf_rn(ur[4 * q + 0], d.x, acc3);
        acc0 = __fmaf_rn(ur[4 * q + 1], a.y, acc0);
        acc1 = __fmaf_rn(ur[4 * q + 1], b.y, acc1);
        acc2 = __fmaf_rn(ur[4 * q + 1], c.y, acc2);
        acc3 = __fmaf_rn(ur[4 * q + 1], d.y, acc3);
        acc0 = __fmaf_rn(ur[4 * q + 2], a.z, acc0);
        acc1 = __fmaf_rn(ur[4 * q + 2], b.z, acc1);
        acc2 = __fmaf_rn(ur[4 * q + 2], c.z, acc2);
        acc3 = __fmaf_rn(ur[4 * q + 2], d.z, acc3);
        acc0 = __fmaf_rn(ur[4 * q + 3], a.w, acc0);
        acc1 = __fmaf_rn(ur[4 * q + 3], b.w, acc1);
        acc2 = __fmaf_rn(ur[4 * q + 3], c.w, acc2);
        acc3 = __fmaf_rn(ur[4 * q + 3], d.w, acc3);
      }
      // rows beyond the tile's end hold stale data: mask their bounds
      const float h0 = __fmaf_rn(gu, nrm[j0 + 0], acc0);
      const float h1 = (j0 + 1 < rows) ? __fmaf_rn(gu, nrm[j0 + 1], acc1) : kNegInf;
      const float h2 = (j0 + 2 < rows) ? __fmaf_rn(gu, nrm[j0 + 2], acc2) : kNegInf;
      const float h3 = (j0 + 3 < rows) ? __fmaf_rn(gu, nrm[j0 + 3], acc3) : kNegInf;
      const float m = fmaxf(fmaxf(h0, h1), fmaxf(h2, h3));
      if (m >= st.tau) {
        const float accs[4] = {acc0, acc1, acc2, acc3};
        const float hs[4] = {h0, h1, h2, h3};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          if (hs[q] >= st.tau && j0 + q < rows) {
            const float lo = __fmaf_rn(-gu, nrm[j0 + q], accs[q]);
            st.offer(hs[q], lo, (int32_t)(first + j0 + q));
          }
        }
      }
    }
  }

  if (active) {
    o.tau[u] = st.tau;
    o.n_cand[u] = st.n_cand;
  }
  unsigned long long c = active ? (unsigned long long)st.n_cand : 0ull;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((tid & 31) == 0 && c) atomicAdd(&stats->cand_emitted, c);
}

template <int FP>
cudaError_t launch_fp(const float* users, int64_t n_users, int f, const float* items, const float* nrm,
                      int64_t n_items, int K, SelectOut o, DevStats* stats, int* err, cudaStream_t s) {
  size_t smem = (size_t)(2 * kTileItems * FP + 2 * kTileItems + K * kThreads) * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(fp32_score_select_kernel<FP>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  unsigned blocks = (unsigned)((n_users + kThreads - 1) / kThreads);
  fp32_score_select_kernel<FP><<<blocks, kThreads, smem, s>>>(users, n_users, f, items, nrm, n_items, K, o, stats, err);
  return cudaGetLastError();
}

}  // namespace

bool fp32_supported(int f, int K) { return f >= 1 && f <= 128 && K >= 1 && K <= 128; }

cudaError_t launch_fp32_score_select(const float* users, int64_t n_users, int f, const float* items,
                                     const float* item_nrm_ub, int64_t n_items, int K, SelectOut o,
                                     DevStats* stats, int* err, cudaStream_t s) {
  const int fp = (int)round_up(f, 8);
  switch (fp) {
#define MIPS_FP_CASE(N) \
  case N:               \
    return launch_fp<N>(users, n_users, f, items, item_nrm_ub, n_items, K, o, stats, err, s);
    MIPS_FP_CASE(8) MIPS_FP_CASE(16) MIPS_FP_CASE(24) MIPS_FP_CASE(32) MIPS_FP_CASE(40)
    MIPS_FP_CASE(48) MIPS_FP_CASE(56) MIPS_FP_CASE(64) MIPS_FP_CASE(72) MIPS_FP_CASE(80)
    MIPS_FP_CASE(88) MIPS_FP_CASE(96) MIPS_FP_CASE(104) MIPS_FP_CASE(112) MIPS_FP_CASE(120)
    MIPS_FP_CASE(128)
#undef MIPS_FP_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

}  // namespace mips
