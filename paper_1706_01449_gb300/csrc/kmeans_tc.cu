// Tensor-core k-means assignment step (Sec. III-A: every user to its nearest
// centroid, argmin_j ||u - c_j||^2 = argmax_j (u . c_j - ||c_j||^2 / 2), ties
// to the smaller j) on tcgen05.  The operands are BF16 rows of fk elements,
// fk = f + 1 rounded up to whole 64-element (128-byte) chunks:
//   user row      [u_1 .. u_f, 1, 0 ..]
//   centroid row  [c_1 .. c_f, -||c_j||^2 / 2, 0 ..]
// so one MMA chain leaves u . c_j - ||c_j||^2 / 2 (of the BF16-rounded
// operands, summed in FP32) in TMEM.  The assignment is thereby approximate
// in the BF16 rounding, as the CUDA-core kernel's is in FP32; no exactness
// rests on it: every pruning bound is computed from the assignment that was
// produced.
//
// Persistent kernel, one CTA per SM, 6 warps:
//   warps 0-3  epilogue: warp w reads TMEM lanes 32 w .. 32 w + 31 (its 32
//              users) of each 256-column accumulator, 64 columns per
//              max-reducing load, and keeps the first column that holds the
//              running maximum;
//   warp 4     allocates / frees TMEM; its lane 0 loads every centroid chunk
//              once (they stay resident in shared memory) and the user tiles
//              into two slots;
//   warp 5     lane 0 issues, per (user tile, centroid chunk), one chain of
//              fk / 16 MMAs (M = 128, N = 256) into one of two accumulators,
//              so the epilogue of one chunk overlaps the MMAs of the next.
// Every wait is bounded as in the score kernel (DEV_ERR_TIMEOUT, drains,
// TMEM freed before exit).
#include <cuda_bf16.h>

#include <algorithm>

#include "common.cuh"
#include "tc_ptx.cuh"
#include "tc_topk.h"

namespace mips {

namespace {

constexpr int kKmWarps = 6;
constexpr int kKmProdWarp = 4;
constexpr int kKmMmaWarp = 5;
constexpr int kKmTileM = 128;   // users per tile (MMA M)
constexpr int kKmChunk = 256;   // centroids per accumulator (MMA N)
constexpr uint32_t kKmAChunkBytes = kKmTileM * 128;   // one 64-element chunk of a user tile
constexpr uint32_t kKmBChunkBytes = kKmChunk * 128;   // one 64-element chunk of a centroid chunk

struct KmSmem {
  uint64_t b_full;
  uint64_t a_full[2], a_empty[2];
  uint64_t acc_full[2], acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort_flag;
};

__global__ void __launch_bounds__(kKmWarps * 32, 1)
    kmeans_assign_tc_kernel(const __grid_constant__ CUtensorMap map_users, const __grid_constant__ CUtensorMap map_cent,
                            int64_t n_users, int C, int nk, int32_t* __restrict__ assign, int* err,
                            unsigned long long wait_ns) {
  extern __shared__ __align__(1024) unsigned char km_smem_raw[];
  unsigned char* base = (unsigned char*)(((uintptr_t)km_smem_raw + 1023) & ~(uintptr_t)1023);
  const int n_chunks = (C + kKmChunk - 1) / kKmChunk;
  unsigned char* b_tiles = base;                                                 // [n_chunks][nk][256 x 128 B]
  unsigned char* a_tiles = b_tiles + (size_t)n_chunks * nk * kKmBChunkBytes;    // [2][nk][128 x 128 B]
  KmSmem* ctl = (KmSmem*)(a_tiles + (size_t)2 * nk * kKmAChunkBytes);
  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const Guard gd{&ctl->abort_flag, err, wait_ns > 0 ? wait_ns : kWaitNs};
  const int64_t n_tiles = (n_users + kKmTileM - 1) / kKmTileM;
  constexpr uint32_t kCols = 2 * kKmChunk;

  if (threadIdx.x == 0) {
    mbar_init(&ctl->b_full, 1);
    for (int s = 0; s < 2; ++s) {
      mbar_init(&ctl->a_full[s], 1);
      mbar_init(&ctl->a_empty[s], 1);
      mbar_init(&ctl->acc_full[s], 1);
      mbar_init(&ctl->acc_empty[s], 4);
    }
    mbar_init(&ctl->drain, 1);
    ctl->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == kKmProdWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;

  if (warp == kKmProdWarp) {
    if (lane == 0) {
      // every centroid chunk, once (rows past C read as zeros and are skipped by the epilogue)
      mbar_expect_tx(&ctl->b_full, (uint32_t)(n_chunks * nk) * kKmBChunkBytes);
      for (int c = 0; c < n_chunks; ++c)
        for (int kk = 0; kk < nk; ++kk)
          tma_load_2d(b_tiles + (size_t)(c * nk + kk) * kKmBChunkBytes, &map_cent, kk * 64, c * kKmChunk,
                      &ctl->b_full);
      bool ok = true;
      long long na = 0;  // user tiles loaded
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++na) {
        const int slot = (int)(na & 1);
        if (na >= 2) ok = mbar_wait(&ctl->a_empty[slot], (uint32_t)(((na >> 1) - 1) & 1), gd);
        if (!ok) break;
        mbar_expect_tx(&ctl->a_full[slot], (uint32_t)nk * kKmAChunkBytes);
        for (int kk = 0; kk < nk; ++kk)
          tma_load_2d(a_tiles + (size_t)(slot * nk + kk) * kKmAChunkBytes, &map_users, kk * 64,
                      (int)(t * kKmTileM), &ctl->a_full[slot]);
      }
      // copies still in flight land before the CTA exits (the last load of
      // each slot; an earlier one was consumed before its slot was reused)
      for (long long aa = (na > 2 ? na - 2 : 0); aa < na; ++aa)
        mbar_drain(&ctl->a_full[aa & 1], (uint32_t)((aa >> 1) & 1));
      mbar_drain(&ctl->b_full, 0);
    }
  } else if (warp == kKmMmaWarp) {
    if (lane == 0) {
      // D = F32, A = B = BF16, both K-major, N = 256, M = 128
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kKmChunk >> 3) << 17) |
                             ((uint32_t)(kKmTileM >> 4) << 24);
      const uint64_t a_desc0 = smem_desc(smem_u32(a_tiles), 1024, 2);  // 128-byte swizzle, 8-row groups of 1 KB
      const uint64_t b_desc0 = smem_desc(smem_u32(b_tiles), 1024, 2);
      bool ok = mbar_wait(&ctl->b_full, 0, gd);
      long long g = 0;   // (tile, chunk) pairs so far
      long long lt = 0;  // tiles so far
      for (int64_t t = blockIdx.x; t < n_tiles && ok; t += gridDim.x, ++lt) {
        const int slot = (int)(lt & 1);
        ok = mbar_wait(&ctl->a_full[slot], (uint32_t)((lt >> 1) & 1), gd);
        if (!ok) break;
        tc_fence_after();
        for (int c = 0; c < n_chunks; ++c, ++g) {
          const int acc = (int)(g & 1);
          if (g >= 2) ok = mbar_wait(&ctl->acc_empty[acc], (uint32_t)(((g >> 1) - 1) & 1), gd);
          if (!ok) break;
          tc_fence_after();
          const uint32_t d = tmem + (uint32_t)(acc * kKmChunk);
          for (int kk = 0; kk < nk; ++kk) {
            const uint64_t ad = a_desc0 + (uint64_t)(((slot * nk + kk) * kKmAChunkBytes) >> 4);
            const uint64_t bd = b_desc0 + (uint64_t)(((c * nk + kk) * kKmBChunkBytes) >> 4);
#pragma unroll
            for (int k = 0; k < 4; ++k)  // K = 16 BF16 = 32 bytes per MMA
              mma_bf16_rt(d, ad + 2 * k, bd + 2 * k, idesc, (uint32_t)(kk | k));
          }
          mma_commit(&ctl->acc_full[acc]);
        }
        if (!ok) break;
        mma_commit(&ctl->a_empty[slot]);
      }
      // every MMA issued by this thread completes before TMEM is released
      mma_commit(&ctl->drain);
      mbar_drain(&ctl->drain, 0);
    }
  } else {
    // ------------------------------------------------------------ epilogue
    const int q = warp;  // lane quarter
    long long g = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
      float best = -__int_as_float(0x7f800000);
      int bj = 0;
      for (int c = 0; c < n_chunks; ++c, ++g) {
        const int acc = (int)(g & 1);
        ok = __all_sync(kFull, mbar_wait(&ctl->acc_full[acc], (uint32_t)((g >> 1) & 1), gd));
        if (!ok) break;
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(acc * kKmChunk);
#pragma unroll 1
        for (int h = 0; h < kKmChunk / 64; ++h) {
          const int j0 = c * kKmChunk + h * 64;
          if (j0 >= C) break;  // warp-uniform
          const int nv = min(64, C - j0);
          uint32_t v[64];
          float m = tmem_ldmax64v(taddr + 64 * h, v);
          if (nv < 64) {  // columns past C hold zeros: leave them out
            m = -__int_as_float(0x7f800000);
#pragma unroll
            for (int j = 0; j < 64; ++j)
              if (j < nv) m = fmaxf(m, __uint_as_float(v[j]));
          }
          if (m > best) {  // a later group wins only by a strictly larger value
            int qi = 0;
#pragma unroll
            for (int j = 63; j >= 0; --j)
              if (j < nv && __uint_as_float(v[j]) == m) qi = j;  // the first column holding it
            best = m;
            bj = j0 + qi;
          }
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->acc_empty[acc]);
      }
      if (!ok) break;
      const int64_t row = t * kKmTileM + 32 * q + lane;
      if (row < n_users) assign[row] = bj;
    }
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kKmProdWarp)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols) : "memory");
}

// Users as BF16 rows [u, 1, 0 ..] of fk elements: a thread per 8-element
// chunk (one 16-byte store), a block per 256 / (fk / 8) whole rows, so the
// row and chunk come from 32-bit arithmetic on the thread index.
__global__ void km_users_bf16_kernel(const float* __restrict__ users, int64_t n, int f, int fk,
                                     __nv_bfloat16* __restrict__ out) {
  const int cpr = fk / 8;                        // chunks per row (fk is a multiple of 64)
  const int rows_per_block = blockDim.x / cpr;
  const int r = threadIdx.x / cpr, c = threadIdx.x - r * cpr;
  if (r >= rows_per_block) return;
  const int64_t u = (int64_t)blockIdx.x * rows_per_block + r;
  if (u >= n) return;
  const float* ur = users + u * f;
  __align__(16) __nv_bfloat16 q[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    const int k = 8 * c + i;
    q[i] = __float2bfloat16_rn(k < f ? ur[k] : (k == f ? 1.f : 0.f));
  }
  reinterpret_cast<uint4*>(out + u * fk)[c] = *reinterpret_cast<const uint4*>(q);
}

// Centroids as BF16 rows [c_j, -||c_j||^2 / 2, 0 ..] (hn2 = ||c_j||^2 / 2).
__global__ void km_cent_bf16_kernel(const float* __restrict__ cent, const float* __restrict__ hn2, int C, int f,
                                    int fk, __nv_bfloat16* __restrict__ out) {
  const int total = C * fk;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < total; e += gridDim.x * blockDim.x) {
    const int j = e / fk, k = e - j * fk;
    const float x = k < f ? cent[(int64_t)j * f + k] : (k == f ? -hn2[j] : 0.f);
    out[e] = __float2bfloat16_rn(x);
  }
}

}  // namespace

int km_tc_row_len(int f) { return (int)round_up(f + 1, 64); }

size_t km_tc_smem_bytes(int f, int C) {
  const size_t nk = (size_t)km_tc_row_len(f) / 64;
  const size_t n_chunks = ((size_t)C + kKmChunk - 1) / kKmChunk;
  return 1024 + n_chunks * nk * kKmBChunkBytes + 2 * nk * kKmAChunkBytes + sizeof(KmSmem);
}

bool km_tc_fits(int f, int C, int max_smem) {
  return C >= 1 && f >= 1 && km_tc_smem_bytes(f, C) <= (size_t)max_smem;
}

cudaError_t km_tc_users(const float* users, int64_t n_users, int f, uint16_t* users_km, cudaStream_t s) {
  if (n_users <= 0) return cudaSuccess;
  const int fk = km_tc_row_len(f);
  const int rows_per_block = 256 / (fk / 8);  // fk <= 192 (f <= 128): at least 10 rows
  const unsigned blocks = (unsigned)((n_users + rows_per_block - 1) / rows_per_block);
  km_users_bf16_kernel<<<blocks, 256, 0, s>>>(users, n_users, f, fk, (__nv_bfloat16*)users_km);
  return cudaGetLastError();
}

cudaError_t km_tc_assign(const uint16_t* users_km, int64_t n_users, int f, const float* cent, const float* hn2, int C,
                         uint16_t* cent_km, int32_t* assign, int* err, int max_smem, cudaStream_t s) {
  if (n_users <= 0) return cudaSuccess;
  const int fk = km_tc_row_len(f);
  km_cent_bf16_kernel<<<(unsigned)std::max(1, std::min((C * fk + 255) / 256, 1024)), 256, 0, s>>>(
      cent, hn2, C, f, fk, (__nv_bfloat16*)cent_km);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap mu, mc;
  if (!tc_make_map(&mu, users_km, n_users, fk, 128, kKmTileM) || !tc_make_map(&mc, cent_km, C, fk, 128, kKmChunk))
    return cudaErrorInvalidValue;
  size_t smem = km_tc_smem_bytes(f, C);
  if (smem > (size_t)max_smem) return cudaErrorInvalidValue;
  // at least half the SM's shared memory: one CTA per SM, so no two CTAs
  // compete for the 512 TMEM columns
  if (smem < (size_t)max_smem / 2 + 1024) smem = (size_t)max_smem / 2 + 1024;
  e = cudaFuncSetAttribute(kmeans_assign_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t n_tiles = (n_users + kKmTileM - 1) / kKmTileM;
  const int grid = (int)std::min<int64_t>(n_tiles, sm_count());
  kmeans_assign_tc_kernel<<<grid, kKmWarps * 32, smem, s>>>(mu, mc, n_users, C, fk / 64, assign, err, 0ull);
  return cudaGetLastError();
}

}  // namespace mips
