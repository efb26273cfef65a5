// Fused BF16 blocked multiply + top-K candidate select on tcgen05 tensor
// cores (the paper's BMM, Sec. III-B, with the per-user selection fused so
// the |U| x |I| score matrix never leaves the SM).
//
// Persistent kernel, one CTA per SM, 12 warps:
//   warp 0      TMA producer: the CTA's user tile (UT = 128 * NH rows, NH in
//               {1, 2}) once per tile, then item tiles of 128 rows through an
//               S-stage shared-memory ring;
//   warp 1      MMA issuer (one thread): for each item tile and user half h,
//               D[h] = A[h] . B^T with tcgen05.mma kind::f16 (BF16 x BF16 ->
//               FP32) into a TMEM accumulator of 128 lanes x 128 columns;
//               two accumulator buffers, so the MMAs of item tile j+1 overlap
//               the select of tile j;
//   warp 2      allocates / frees TMEM;
//   warps 4..   select: thread t of epilogue warp e owns user row
//               h * 128 + 32 * (e % 4) + t (TMEM lane restriction: a warp
//               reads lanes 32 * (warp % 4) .. + 31), loads its 128 scores
//               per item tile with tcgen05.ld, and keeps the per-user select
//               state of common.cuh.
// Operands are K-major rows (see prep.cu): the two bound columns make every
// accumulator entry an upper bound H >= u^T i, so the common case costs one
// three-input max per two scores plus one compare per 64 scores.
//
// Every mbarrier wait is bounded (1 s of %globaltimer); on expiry the kernel
// raises DEV_ERR_TIMEOUT, every role leaves its loop, the MMA thread drains
// its in-flight MMAs and the producer its in-flight copies (each with a
// bounded wait), and TMEM is freed before exit.
#include <cuda.h>
#include <cuda_bf16.h>

#include "common.cuh"
#include "tc_topk.h"

namespace mips {

namespace {

constexpr int kWarps = 12;
constexpr int kEpiWarp0 = 4;
constexpr int kTileN = 128;    // items per tile (MMA N)
constexpr int kTileM = 128;    // users per half (MMA M)
constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the phase with the given parity.  Returns false when the
// CTA is aborting (this or another role timed out).
__device__ __noinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*abort_flag) return false;
    if (globaltimer() - t0 > kWaitNs) {
      *abort_flag = 1;
      atomicOr(err, DEV_ERR_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor (tcgen05): start address, leading byte
// offset (unused for swizzled K-major), stride byte offset = one 8-row group,
// fixed version bits 46..48 = 0b001, swizzle mode in bits 61..63.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t sbo, uint32_t layout) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)layout << 61);
}

__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 lanes x 32 bits, 64 consecutive columns: r[j] = column (col + j) of this
// thread's lane.
__device__ __forceinline__ void tmem_ld64(uint32_t taddr, uint32_t (&r)[64]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x64.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
      "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,"
      "%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]),
        "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]),
        "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]),
        "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]),
        "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ float max3(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

struct TcUser {
  UserSelect st;
  float beta_u, nhat_u;  // bound columns of this user (prep.cu)
  float g;               // accumulation-error factor of prep.cu
};

// Slow path for one score: lower bound L from the bound columns, then offer.
//   A = beta_u nhat_i + nhat_u alpha_i,  L = H - 2A - g (nhat_u nhat_i + A),
// evaluated with outward margins for the FP32 rounding of this arithmetic.
__device__ __noinline__ void tc_offer(TcUser& s, float H, int32_t pos, const float2* __restrict__ item_aux) {
  const float2 ia = item_aux[pos];  // {nhat_i, alpha_i}
  const float A = __fmaf_rn(s.beta_u, ia.x, s.nhat_u * ia.y);
  const float nn = s.nhat_u * ia.x;
  const float slack = __fmaf_rn(2.0f, A, s.g * (nn + A)) * (1.0f + 3.814697265625e-06f);  // 2^-18
  const float L = (H - slack) - fabsf(H) * 2.384185791015625e-07f;                     // 2^-22
  s.st.offer(H, L, pos);
}

__device__ __forceinline__ void select64(TcUser& s, uint32_t (&r)[64], int32_t pos0, int valid,
                                         const float2* __restrict__ item_aux) {
  if (valid < 64) {
#pragma unroll
    for (int q = 0; q < 64; ++q)
      if (q >= valid) r[q] = 0xff800000u;  // -inf
  }
  float m[21];
#pragma unroll
  for (int q = 0; q < 21; ++q)
    m[q] = max3(__uint_as_float(r[3 * q]), __uint_as_float(r[3 * q + 1]), __uint_as_float(r[3 * q + 2]));
  float a = max3(m[0], m[1], m[2]), b = max3(m[3], m[4], m[5]), c = max3(m[6], m[7], m[8]);
  float d = max3(m[9], m[10], m[11]), e = max3(m[12], m[13], m[14]), f = max3(m[15], m[16], m[17]);
  float g = max3(m[18], m[19], m[20]);
  float mm = max3(max3(a, b, c), max3(d, e, f), fmaxf(g, __uint_as_float(r[63])));
  if (mm >= s.st.tau) {
#pragma unroll
    for (int q = 0; q < 64; ++q) {
      const float v = __uint_as_float(r[q]);
      if (v >= s.st.tau && q < valid) tc_offer(s, v, pos0 + q, item_aux);
    }
  }
}

struct Smem {
  uint64_t b_full[kMaxStages];
  uint64_t b_empty[kMaxStages];
  uint64_t a_full, a_empty;
  uint64_t acc_full[2], acc_empty[2];
  uint64_t drain;
  uint32_t tmem_base;
  int abort_flag;
};

__global__ void __launch_bounds__(kWarps * 32, 1)
    tc_score_select_kernel(const __grid_constant__ CUtensorMap map_users, const __grid_constant__ CUtensorMap map_items,
                           TcParams p, SelectOut o, const float2* __restrict__ user_aux,
                           const float2* __restrict__ item_aux, DevStats* stats, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned carve-up: A tiles, B ring, heap, control block
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t chunk_bytes = kTileM * p.row_bytes;  // one K chunk of a 128-row tile
  unsigned char* a_tiles = base;                                            // [NH][KC][chunk]
  unsigned char* b_tiles = a_tiles + (size_t)p.nh * p.kc * chunk_bytes;    // [S][KC][chunk]
  float* heap_base = (float*)(b_tiles + (size_t)p.stages * p.kc * chunk_bytes);  // [K][NH*128]
  Smem* ctl = (Smem*)(heap_base + (size_t)p.K * p.nh * kTileM);

  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  volatile int* abort_flag = &ctl->abort_flag;
  const int n_ut = (int)((p.n_users + p.nh * kTileM - 1) / (p.nh * kTileM));
  const int n_it = (int)((p.n_items + kTileN - 1) / kTileN);
  const uint32_t tmem_cols = p.nh == 2 ? 512u : 256u;

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&ctl->b_full[s], 1);
      mbar_init(&ctl->b_empty[s], 1);
    }
    mbar_init(&ctl->a_full, 1);
    mbar_init(&ctl->a_empty, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl->acc_full[b], 1);
      mbar_init(&ctl->acc_empty[b], 4 * p.nh);
    }
    mbar_init(&ctl->drain, 1);
    ctl->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                 "r"(tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;

  if (warp == 0) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_users)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_items)) : "memory");
      long long g = 0;
      int lt = 0;
      bool ok = true;
      for (int ut = blockIdx.x; ut < n_ut && ok; ut += gridDim.x, ++lt) {
        if (lt > 0) ok = mbar_wait(&ctl->a_empty, (lt - 1) & 1, abort_flag, err);
        if (!ok) break;
        mbar_expect_tx(&ctl->a_full, p.nh * p.kc * chunk_bytes);
        for (int h = 0; h < p.nh; ++h)
          for (int c = 0; c < p.kc; ++c)
            tma_load_2d(a_tiles + (size_t)(h * p.kc + c) * chunk_bytes, &map_users, c * p.row_elems,
                        ut * p.nh * kTileM + h * kTileM, &ctl->a_full);
        for (int j = 0; j < n_it; ++j, ++g) {
          const int s = (int)(g % p.stages);
          if (g >= p.stages) ok = mbar_wait(&ctl->b_empty[s], (uint32_t)(((g / p.stages) - 1) & 1), abort_flag, err);
          if (!ok) break;
          mbar_expect_tx(&ctl->b_full[s], p.kc * chunk_bytes);
          for (int c = 0; c < p.kc; ++c)
            tma_load_2d(b_tiles + (size_t)(s * p.kc + c) * chunk_bytes, &map_items, c * p.row_elems, j * kTileN,
                        &ctl->b_full[s]);
        }
      }
      if (!ok) {  // drain the copies still in flight before the CTA exits
        for (long long gg = (g > p.stages ? g - p.stages : 0); gg < g; ++gg) {
          uint64_t* bar = &ctl->b_full[gg % p.stages];
          const unsigned long long t0 = globaltimer();
          while (!mbar_try_wait(bar, (uint32_t)((gg / p.stages) & 1)) && globaltimer() - t0 < kWaitNs) {
          }
        }
      }
    }
  } else if (warp == 1) {
    // ------------------------------------------------------------ MMA issuer
    if (lane == 0) {
      // instruction descriptor: D = F32, A = B = BF16, both K-major, N, M
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kTileN >> 3) << 17) |
                             ((uint32_t)(kTileM >> 4) << 24);
      const uint32_t sbo = 8 * p.row_bytes;
      const int ksteps = p.row_bytes / 32;  // K = 16 BF16 = 32 bytes per MMA
      long long g = 0;
      int lt = 0;
      bool ok = true;
      for (int ut = blockIdx.x; ut < n_ut && ok; ut += gridDim.x, ++lt) {
        ok = mbar_wait(&ctl->a_full, lt & 1, abort_flag, err);
        if (!ok) break;
        tc_fence_after();
        for (int j = 0; j < n_it; ++j, ++g) {
          const int s = (int)(g % p.stages);
          const int b = (int)(g & 1);
          ok = mbar_wait(&ctl->b_full[s], (uint32_t)((g / p.stages) & 1), abort_flag, err);
          if (ok && g >= 2) ok = mbar_wait(&ctl->acc_empty[b], (uint32_t)(((g >> 1) - 1) & 1), abort_flag, err);
          if (!ok) break;
          tc_fence_after();
          for (int h = 0; h < p.nh; ++h) {
            const uint32_t d = tmem + (uint32_t)(b * p.nh * kTileN + h * kTileN);
            for (int c = 0; c < p.kc; ++c) {
              const uint32_t a_addr = smem_u32(a_tiles + (size_t)(h * p.kc + c) * chunk_bytes);
              const uint32_t b_addr = smem_u32(b_tiles + (size_t)(s * p.kc + c) * chunk_bytes);
              for (int k = 0; k < ksteps; ++k) {
                mma_bf16(d, smem_desc(a_addr + 32 * k, sbo, p.swizzle), smem_desc(b_addr + 32 * k, sbo, p.swizzle),
                         idesc, (c | k) != 0);
              }
            }
          }
          mma_commit(&ctl->b_empty[s]);
          mma_commit(&ctl->acc_full[b]);
        }
        if (ok) mma_commit(&ctl->a_empty);
      }
      // all MMAs issued by this thread complete before TMEM is released
      mma_commit(&ctl->drain);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(&ctl->drain, 0) && globaltimer() - t0 < kWaitNs) {
      }
    }
  } else if (warp >= kEpiWarp0 && warp < kEpiWarp0 + 4 * p.nh) {
    // ------------------------------------------------------------ select
    const int e = warp - kEpiWarp0;
    const int h = e / 4, q = e % 4;
    const int row = h * kTileM + 32 * q + lane;  // row within the user tile
    TcUser s;
    s.st.heap = heap_base + row;
    s.st.stride = p.nh * kTileM;
    s.st.K = p.K;
    s.st.cap = o.cap;
    s.g = p.g;
    long long g = 0;
    bool ok = true;
    unsigned long long emitted = 0;
    for (int ut = blockIdx.x; ut < n_ut && ok; ut += gridDim.x) {
      const int64_t u = (int64_t)ut * p.nh * kTileM + row;
      const bool active = u < p.n_users;
      s.st.tau = active ? kNegInf : __int_as_float(0x7f800000);
      s.st.n_cand = 0;
      s.st.cand_pos = o.cand_pos + (active ? u : 0) * (int64_t)o.cap;
      s.st.cand_ub = o.cand_ub + (active ? u : 0) * (int64_t)o.cap;
      heap_init(s.st.heap, s.st.stride, p.K);
      if (active) {
        const float2 ua = user_aux[u];
        s.beta_u = ua.x;
        s.nhat_u = ua.y;
      }
      for (int j = 0; j < n_it; ++j, ++g) {
        const int b = (int)(g & 1);
        ok = mbar_wait(&ctl->acc_full[b], (uint32_t)((g >> 1) & 1), abort_flag, err);
        if (!ok) break;
        tc_fence_after();
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * p.nh * kTileN + h * kTileN);
        const int valid = (int)min((int64_t)kTileN, p.n_items - (int64_t)j * kTileN);
        uint32_t r[64];
        tmem_ld64(taddr, r);
        select64(s, r, j * kTileN, valid, item_aux);
        tmem_ld64(taddr + 64, r);
        select64(s, r, j * kTileN + 64, valid - 64, item_aux);
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->acc_empty[b]);
      }
      if (!ok) break;
      if (active) {
        o.tau[u] = s.st.tau;
        o.n_cand[u] = s.st.n_cand;
        emitted += (unsigned long long)s.st.n_cand;
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) emitted += __shfl_xor_sync(0xffffffffu, emitted, off);
    if (lane == 0 && emitted) atomicAdd(&stats->cand_emitted, emitted);
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 2) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(tmem_cols) : "memory");
  }
}

}  // namespace

size_t tc_smem_bytes(const TcParams& p) {
  const size_t chunk = (size_t)kTileM * p.row_bytes;
  return 1024 + (size_t)p.nh * p.kc * chunk + (size_t)p.stages * p.kc * chunk +
         sizeof(float) * (size_t)p.K * p.nh * kTileM + sizeof(Smem);
}

cudaError_t launch_tc_score_select(const CUtensorMap* map_users, const CUtensorMap* map_items, const TcParams& p,
                                   SelectOut o, const float2* user_aux, const float2* item_aux, DevStats* stats,
                                   int* err, int grid, cudaStream_t s) {
  // at least half the SM's shared memory: one CTA per SM, so no two CTAs
  // ever compete for the TMEM columns this kernel allocates
  size_t smem = tc_smem_bytes(p);
  int max_smem = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem < (size_t)max_smem / 2 + 1024) smem = (size_t)max_smem / 2 + 1024;
  cudaError_t e = cudaFuncSetAttribute(tc_score_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  tc_score_select_kernel<<<grid, kWarps * 32, smem, s>>>(*map_users, *map_items, p, o, user_aux, item_aux, stats, err);
  return cudaGetLastError();
}

}  // namespace mips
