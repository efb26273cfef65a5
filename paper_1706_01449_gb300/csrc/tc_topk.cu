// Fused BF16 blocked multiply + top-K candidate select on tcgen05 tensor
// cores (the paper's BMM, Sec. III-B, with the per-user selection fused so
// the |U| x |I| score matrix never leaves the SM), and the same machinery
// walking Maximus's per-cluster item lists (Sec. IV, Algorithm 1).
//
// Persistent kernel, one CTA per SM, 12 warps, user tiles of 128 rows and
// item tiles of 256 rows (an M = 128, N = 256 MMA runs at the tensor pipe's
// full rate; N = 128 costs nearly the same time per instruction):
//   warp 0      TMA producer: takes the CTA's next work item (user tile x
//               range of item tiles), publishes it in a shared-memory ring
//               for the other roles, loads the user tile, then the item
//               tiles through an S-stage ring (whole tiles, or two 128-row
//               halves when whole tiles do not fit shared memory; operand
//               rows of 128-byte chunks plus a 32/64-byte tail chunk, each
//               with its own tensor map and swizzle);
//   warp 1      MMA issuer (one thread): D = A . B^T with tcgen05.mma
//               kind::f16 (BF16 x BF16 -> FP32) into one of two TMEM
//               accumulators of 128 lanes x 256 columns, so the MMAs of item
//               tile j+1 overlap the select of tile j;
//   warp 2      allocates / frees TMEM;
//   warps 4-11  select: epilogue warp e reads TMEM lanes 32 * (e % 4) .. +31
//               (a warp may only touch the lane quarter of its warp % 4) and
//               columns 128 * (e / 4) .. +127 of each item tile, so every
//               user is served by two threads, each with its own threshold,
//               top-K of lower bounds and candidate sub-list; the two share
//               their thresholds through shared memory (either one is a valid
//               lower bound on the user's K-th score, so the larger filters
//               both halves).
// Work items: without a work list (blocked multiply) user tile w against
// every item tile; with one (item-chunked blocked multiply, Maximus walk)
// as the list gives them, claimed round-robin or from a global counter.
// Operands are K-major rows (prep.cu): the two bound columns make every
// accumulator entry an upper bound H >= u^T i, so the common case costs one
// maximum over 16 scores and a compare.
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
constexpr int kEpiWarps = 8;
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kTileN = 256;    // items per tile (MMA N)
constexpr int kTileM = 128;    // users per tile (MMA M)
constexpr int kHalfN = 128;    // columns per epilogue thread and tile
constexpr int kQueue = 16;     // hit-queue slots per thread
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
__device__ __noinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err) {
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

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, volatile int* abort_flag, int* err) {
  if (mbar_try_wait(bar, parity)) return true;
  return mbar_wait_slow(bar, parity, abort_flag, err);
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

// maximum of 16 scores (a tree of three-input maxima)
__device__ __forceinline__ float max16(const uint32_t* r) {
  const float m0 = max3(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]));
  const float m1 = max3(__uint_as_float(r[3]), __uint_as_float(r[4]), __uint_as_float(r[5]));
  const float m2 = max3(__uint_as_float(r[6]), __uint_as_float(r[7]), __uint_as_float(r[8]));
  const float m3 = max3(__uint_as_float(r[9]), __uint_as_float(r[10]), __uint_as_float(r[11]));
  const float m4 = max3(__uint_as_float(r[12]), __uint_as_float(r[13]), __uint_as_float(r[14]));
  return max3(max3(m0, m1, m2), m3, fmaxf(m4, __uint_as_float(r[15])));
}

// A threshold published for the partner thread, tagged with its user tile
// so that a value from another user is never taken.
__device__ __forceinline__ unsigned long long pack_tau(float t, int ut) {
  return ((unsigned long long)(uint32_t)ut << 32) | (unsigned long long)__float_as_uint(t);
}

// Per-thread select state (registers).  KR > 0: the K largest lower bounds
// live in a register array d[0..KR-1] sorted descending (K <= KR); KR = 0:
// in the shared-memory min-heap of common.cuh.
template <int KR>
struct TcUser {
  float tau;      // this thread's K-th largest lower bound so far
  float tau_eff;  // max(tau, partner thread's tau): the filter threshold
  int n_cand;
  int ut;         // current user tile (tag of the published threshold)
  float beta_u, nhat_u;  // bound columns of this user (prep.cu)
  float d[KR > 0 ? KR : 1];
};

// Warp-uniform parameters of the select.
struct TcSel {
  float* heap;        // &heap_base[slot] (stride kEpiThreads), KR = 0 only
  int K;
  int cap;
  int32_t* cand_pos;  // this thread's candidate sub-list
  float* cand_ub;
  float* qh;          // hit queue: qh[t * kEpiThreads]
  int32_t* qp;
  volatile unsigned long long* tau_mine;  // published thresholds: mine, partner's
  const volatile unsigned long long* tau_partner;
  unsigned* tau_glob;                     // this user's shared threshold (item-chunked scan) or null
  volatile int* seed_mine;                // [2][256] user tile whose seed list is published
  const volatile int* seed_partner;
  float* seed_list;                       // [2][K][256] first-tile top-K lists
  const float* seed_list_partner;
  float g;            // accumulation-error factor of prep.cu
};

template <int KR>
__device__ __forceinline__ void topk_init(TcUser<KR>& s, const TcSel& c) {
  if constexpr (KR > 0) {
#pragma unroll
    for (int i = 0; i < KR; ++i) s.d[i] = kNegInf;
  } else {
    heap_init(c.heap, kEpiThreads, c.K);
  }
}

// Insert lower bound L (> the current K-th largest) and return the new K-th
// largest.
template <int KR>
__device__ __forceinline__ float topk_insert(TcUser<KR>& s, const TcSel& c, float L) {
  if constexpr (KR > 0) {
    float nd[KR];
    nd[0] = fmaxf(s.d[0], L);
#pragma unroll
    for (int i = 1; i < KR; ++i) nd[i] = (L > s.d[i - 1]) ? s.d[i - 1] : fmaxf(s.d[i], L);
#pragma unroll
    for (int i = 0; i < KR; ++i) s.d[i] = nd[i];
    if (c.K == KR) return nd[KR - 1];  // K fills the array (warp-uniform)
    float t = nd[0];  // ends as nd[K - 1] (static indices keep d in registers)
#pragma unroll
    for (int i = 0; i < KR; ++i) t = (i < c.K) ? nd[i] : t;
    return t;
  } else {
    return heap_replace_min(c.heap, kEpiThreads, c.K, L);
  }
}

// Lower bound of the exact score from the upper bound H and the bound
// columns:  A = beta_u nhat_i + nhat_u alpha_i,  L = H - 2A - g (nhat_u nhat_i + A),
// evaluated with outward margins for the FP32 rounding of this arithmetic.
template <int KR>
__device__ __forceinline__ float tc_lower(const TcUser<KR>& s, const TcSel& c, float H, float2 ia) {
  const float A = __fmaf_rn(s.beta_u, ia.x, s.nhat_u * ia.y);
  const float nn = s.nhat_u * ia.x;
  const float slack = __fmaf_rn(2.0f, A, c.g * (nn + A)) * (1.0f + 3.814697265625e-06f);  // 2^-18
  return (H - slack) - fabsf(H) * 2.384185791015625e-07f;                             // 2^-22
}

// After the first-tile pass: this thread's K best lower bounds go to its
// queue slots (shared memory), published with a tagged flag; it then waits a
// bounded time for the partner's (the other half of the same user) and
// takes the K-th largest of the union as its threshold.  The two halves
// hold distinct items, so the union's K-th largest is a valid lower bound.
// If the partner's list is not there within the bound, the thread goes on
// with its own threshold, which is valid too.
// The lists are double-buffered by user-tile parity: a partner that is one
// user tile ahead cannot overwrite the list being read (the accumulator
// handshake keeps the halves within one user tile of each other).
template <int KR>
__device__ __forceinline__ void seed_merge(TcUser<KR>& s, const TcSel& c, int ut, int par) {
  if constexpr (KR > 0) {
    float* mine = c.seed_list + par * c.K * kEpiThreads;
#pragma unroll
    for (int i = 0; i < KR; ++i)
      if (i < c.K) mine[i * kEpiThreads] = s.d[i];
    __threadfence_block();
    c.seed_mine[par * kEpiThreads] = ut;
    const float* pq = c.seed_list_partner + par * c.K * kEpiThreads;
    const volatile int* pflag = c.seed_partner + par * kEpiThreads;
    int spins = 0;
    while (*pflag != ut && ++spins < 20000) {
    }
    if (*pflag == ut) {
      __threadfence_block();
      // K-th largest of two descending lists of K
      int ia = 0, ib = 0;
      float v = s.d[0];
      for (int r = 0; r < c.K; ++r) {
        float a = kNegInf;
#pragma unroll
        for (int i = 0; i < KR; ++i)
          if (i == ia) a = s.d[i];
        const float b = ((volatile const float*)pq)[ib * kEpiThreads];
        if (a >= b) {
          v = a;
          ++ia;
        } else {
          v = b;
          ++ib;
        }
      }
      if (v > s.tau_eff) s.tau_eff = v;
    }
  }
}

// Publish this thread's threshold (tagged with its user tile) for the partner.
// float <-> unsigned with the same order (for atomicMax on thresholds)
__device__ __forceinline__ unsigned tau_ord(float x) {
  const unsigned b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float tau_from_ord(unsigned o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

template <int KR>
__device__ __forceinline__ void tc_publish(const TcUser<KR>& s, const TcSel& c) {
  *c.tau_mine = pack_tau(s.tau, s.ut);
  if (c.tau_glob) atomicMax(c.tau_glob, tau_ord(s.tau));  // every threshold is valid for the user
}

// One hit (H >= tau_eff when queued): threshold update from its lower bound,
// then the candidate emission.  Lower bounds at or below the current filter
// threshold cannot raise it and are not kept.  With emit_only (second pass
// over a user tile's first item tile, whose lower bounds are already in the
// top-K) only the emission is done, so no item is counted twice.  The
// item's position is pos0 + col, or pos_tile[col] for a walk of a
// cluster's sorted list (MX).
template <int KR, bool MX>
__device__ __forceinline__ void tc_offer(TcUser<KR>& s, const TcSel& c, float H, int col, const float2* aux_tile,
                                         int32_t pos0, const int32_t* pos_tile, bool emit_only) {
  if (H < s.tau_eff) return;  // the threshold rose since the hit was queued
  const float L = emit_only ? kNegInf : tc_lower(s, c, H, aux_tile[col]);
  if (L > s.tau_eff) {
    s.tau = topk_insert(s, c, L);
    if (s.tau > s.tau_eff) {
      s.tau_eff = s.tau;
      tc_publish(s, c);
    }
  }
  if (H >= s.tau_eff) {
    if (s.n_cand < c.cap) {
      c.cand_pos[s.n_cand] = MX ? pos_tile[col] : pos0 + col;
      c.cand_ub[s.n_cand] = H;
    }
    ++s.n_cand;
  }
}

// 16 scores r[0..15] of items pos0.. (valid: how many are real items).
// Fast path: one maximum over the 16 and a compare.  Slow path (any lane of
// the warp has a hit): this thread's hits are queued in shared memory, then
// drained in order through one offer site.
template <int KR, bool MX>
__device__ __forceinline__ void select16(TcUser<KR>& s, const TcSel& c, const uint32_t* r, int col0, int valid,
                                         const float2* aux_tile, int32_t pos0, const int32_t* pos_tile,
                                         unsigned long long& slow, bool emit_only) {
  const float m0 = max3(__uint_as_float(r[0]), __uint_as_float(r[1]), __uint_as_float(r[2]));
  const float m1 = max3(__uint_as_float(r[3]), __uint_as_float(r[4]), __uint_as_float(r[5]));
  const float m2 = max3(__uint_as_float(r[6]), __uint_as_float(r[7]), __uint_as_float(r[8]));
  const float m3 = max3(__uint_as_float(r[9]), __uint_as_float(r[10]), __uint_as_float(r[11]));
  const float m4 = max3(__uint_as_float(r[12]), __uint_as_float(r[13]), __uint_as_float(r[14]));
  const float mm = max3(max3(m0, m1, m2), m3, fmaxf(m4, __uint_as_float(r[15])));
  const bool hit = mm >= s.tau_eff;
  if (__any_sync(0xffffffffu, hit)) {  // warp-uniform: counts warp-level entries
    ++slow;
    int n = 0;
    if (hit) {
      // only the groups of three whose maximum reached the threshold
      const float t = s.tau_eff;
      const float gm[6] = {m0, m1, m2, m3, m4, __uint_as_float(r[15])};
#pragma unroll
      for (int gq = 0; gq < 6; ++gq) {
        if (gm[gq] >= t) {
#pragma unroll
          for (int q = 3 * gq; q < (gq < 5 ? 3 * gq + 3 : 16); ++q) {
            const float v = __uint_as_float(r[q]);
            if (v >= t && q < valid) {
              c.qh[n * kEpiThreads] = v;
              c.qp[n * kEpiThreads] = col0 + q;
              ++n;
            }
          }
        }
      }
    }
    // one offer site for the queued hits (keeps the code small)
    for (int t = 0; t < n; ++t)
      tc_offer<KR, MX>(s, c, c.qh[t * kEpiThreads], c.qp[t * kEpiThreads], aux_tile, pos0, pos_tile, emit_only);
  }
}

template <int KR, bool MX>
__device__ __forceinline__ void select64(TcUser<KR>& s, const TcSel& c, uint32_t (&r)[64], int col0, int valid,
                                         const float2* aux_tile, int32_t pos0, const int32_t* pos_tile,
                                         unsigned long long& slow, bool emit_only) {
  if (valid < 64) {
#pragma unroll
    for (int q = 0; q < 64; ++q)
      if (q >= valid) r[q] = 0xff800000u;  // -inf
  }
  // fast path: one maximum over the 64 scores and one warp vote (the four
  // groups of 16 are looked at only when some lane has a hit)
  const float g0 = max16(r), g1 = max16(r + 16), g2 = max16(r + 32), g3 = max16(r + 48);
  const float mm = max3(g0, g1, fmaxf(g2, g3));
  if (!__any_sync(0xffffffffu, mm >= s.tau_eff)) return;
#pragma unroll
  for (int g = 0; g < 4; ++g)
    select16<KR, MX>(s, c, r + 16 * g, col0 + 16 * g, valid - 16 * g, aux_tile, pos0, pos_tile, slow, emit_only);
}

// First pass over a user tile's first item tile (the items of largest norm:
// the index stores items by norm, descending), so that the threshold starts
// the scan near its final value instead of at -inf; nothing is emitted.
// K = 1: the 64 scores form 8 groups of 8 and each group's largest lower
// bound goes to the top-1 -- branch-free, and the result is the exact
// maximum.  K > 1: every lower bound above the threshold is queued, then
// inserted (group maxima would be cheaper but give a lower threshold,
// which measured slower overall on large catalogues).
template <int KR>
__device__ __forceinline__ void seed64(TcUser<KR>& s, const TcSel& c, const uint32_t (&r)[64], int col0, int valid,
                                       const float2* aux_tile) {
  if constexpr (KR == 1) {
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      float m = kNegInf;
#pragma unroll
      for (int q = 8 * g; q < 8 * g + 8; ++q) {
        const float L = tc_lower(s, c, __uint_as_float(r[q]), aux_tile[col0 + q]);
        m = fmaxf(m, q < valid ? L : kNegInf);
      }
      c.qh[g * kEpiThreads] = m;
    }
    // inserted from shared memory in a rolled loop (keeps the registers down)
#pragma unroll 1
    for (int g = 0; g < 8; ++g) {
      const float m = c.qh[g * kEpiThreads];
      if (m > s.tau) s.tau = topk_insert(s, c, m);
    }
  } else {
#pragma unroll
    for (int g = 0; g < 4; ++g) {
      int n = 0;
#pragma unroll
      for (int q = 16 * g; q < 16 * g + 16; ++q) {
        const float H = __uint_as_float(r[q]);
        if (H > s.tau && q < valid) {  // L <= H: nothing at or below tau can enter
          const float L = tc_lower(s, c, H, aux_tile[col0 + q]);
          if (L > s.tau) {
            c.qh[n * kEpiThreads] = L;
            ++n;
          }
        }
      }
      for (int t = 0; t < n; ++t) {
        const float L = c.qh[t * kEpiThreads];
        if (L > s.tau) s.tau = topk_insert(s, c, L);
      }
    }
  }
}

struct WorkItem {
  int a_row;   // first A row of the user tile
  int b_row;   // B row of list rank 0
  int tb, te;  // item tiles [tb, te)
  int q;       // index into the work arrays
};

template <bool MX>
__device__ __forceinline__ WorkItem get_work(const TcParams& p, int wi, int n_it) {
  WorkItem w;
  if constexpr (!MX) {
    w.a_row = wi * kTileM;
    w.b_row = 0;
    w.tb = 0;
    w.te = n_it;
    w.q = wi;
  } else {
    // without a work counter, CTAs take work items round-robin (item wi in
    // round wi / gridDim.x); odd rounds run backwards, so a list sorted by
    // length does not hand the longest item of every round to the same CTA
    int q = wi;
    if (!p.work.next) {
      const int G = (int)gridDim.x, r = wi / G, k = wi - r * G;
      const int in_round = min(G, *p.work.n_work - r * G);
      q = (r & 1) ? r * G + (in_round - 1 - k) : wi;
    }
    w.a_row = p.work.a_row[q];
    w.b_row = p.work.b_row[q];
    w.tb = p.work.t_begin[q];
    w.te = p.work.t_end[q];
    w.q = q;
  }
  return w;
}

// The CTA's work sequence: the producer takes its lt-th work item (static:
// round-robin over the CTAs; with a work counter: the next unclaimed item)
// and publishes the index in ring slot lt % kWQ, where the MMA thread and the
// select warps read it; an index >= n_work ends the sequence.
constexpr int kWQ = 4;

struct Smem {
  uint64_t b_full[kMaxStages];
  uint64_t b_empty[kMaxStages];
  uint64_t a_full, a_empty;
  uint64_t acc_full[2], acc_empty[2];
  uint64_t drain;
  uint64_t wq_full[kWQ], wq_empty[kWQ];
  int wq[kWQ];
  uint32_t tmem_base;
  int abort_flag;
};

// MX: work items from p.work (Maximus walk of per-cluster sorted lists);
// otherwise every user tile against every item tile (blocked multiply).
template <int KR, bool MX>
__global__ void __launch_bounds__(kWarps * 32, 1)
    tc_score_select_kernel(const __grid_constant__ CUtensorMap map_users, const __grid_constant__ CUtensorMap map_users_t,
                           const __grid_constant__ CUtensorMap map_items, const __grid_constant__ CUtensorMap map_items_t,
                           TcParams p, SelectOut o, const float2* __restrict__ user_aux,
                           const float2* __restrict__ item_aux, DevStats* stats, int* err) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  // 1024-byte aligned carve-up (sizes in tc_smem_bytes)
  unsigned char* base = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const uint32_t a_chunk = kTileM * p.row_bytes;  // one K chunk of the user tile
  const int bs = p.b_split;                        // loads (ring stages) per item tile
  const uint32_t sub_rows = kTileN / bs;          // item rows per load
  const uint32_t b_chunk = sub_rows * p.row_bytes;  // one K chunk of a load
  const uint32_t a_bytes = p.kc * a_chunk + kTileM * p.tail_bytes;  // user tile (full chunks, then the tail)
  const uint32_t b_bytes = p.kc * b_chunk + sub_rows * p.tail_bytes;  // one ring stage
  unsigned char* a_tiles = base;                                              // [KC][a_chunk] + tail
  unsigned char* b_tiles = a_tiles + a_bytes;                                 // [S]([KC][b_chunk] + tail)
  float* heap_smem = (float*)(b_tiles + (size_t)p.stages * b_bytes);          // [K][256] (KR = 0)
  const bool heap_in_smem = KR == 0 && !p.heap_global;
  float* heap_base = heap_in_smem ? heap_smem : p.heap_mem + (size_t)blockIdx.x * p.K * kEpiThreads;
  float2* aux_base = (float2*)(heap_smem + (heap_in_smem ? (size_t)p.K * kEpiThreads : 0));  // [8 warps][128]
  int32_t* posb_base = (int32_t*)(aux_base + (size_t)kEpiWarps * kHalfN);      // [8 warps][128]
  float* qh_base = (float*)(posb_base + (size_t)kEpiWarps * kHalfN);          // [16][256]
  int32_t* qp_base = (int32_t*)(qh_base + (size_t)kQueue * kEpiThreads);     // [16][256]
  unsigned long long* tau_sh = (unsigned long long*)(qp_base + (size_t)kQueue * kEpiThreads);  // [256]
  int* seed_sh = (int*)(tau_sh + kEpiThreads);                                                // [2][256]
  float* seed_lists = (float*)(seed_sh + 2 * kEpiThreads);  // [2][K][256] (KR > 0)
  Smem* ctl = (Smem*)(seed_lists + (KR > 0 ? (size_t)2 * p.K * kEpiThreads : 0));

  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  volatile int* abort_flag = &ctl->abort_flag;
  const int n_it = (int)((p.n_items + kTileN - 1) / kTileN);
  const int n_work = MX ? *p.work.n_work : (int)((p.n_users + kTileM - 1) / kTileM);
  constexpr uint32_t kTmemCols = 2 * kTileN;  // two accumulators

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&ctl->b_full[s], 1);
      mbar_init(&ctl->b_empty[s], 1);
    }
    mbar_init(&ctl->a_full, 1);
    mbar_init(&ctl->a_empty, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl->acc_full[b], 1);
      mbar_init(&ctl->acc_empty[b], kEpiWarps);
    }
    mbar_init(&ctl->drain, 1);
    for (int w = 0; w < kWQ; ++w) {
      mbar_init(&ctl->wq_full[w], 1);
      mbar_init(&ctl->wq_empty[w], 1 + kEpiWarps);  // the MMA thread and every select warp
    }
    ctl->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < kEpiThreads; i += blockDim.x) {
    tau_sh[i] = pack_tau(kNegInf, -1);
    seed_sh[i] = -1;
    seed_sh[kEpiThreads + i] = -1;
  }
  if (warp == 2) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                 "r"(kTmemCols)
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
      const int tail_x = p.kc * p.row_elems;  // element column of the tail chunk
      long long g = 0;  // item tiles issued so far
      int st = 0;        // ring stage of tile g
      uint32_t ph = 0;   // ring pass parity of tile g
      bool ok = true;
      const bool dyn = MX && p.work.next;
      for (int lt = 0; ok; ++lt) {
        // take and publish the next work item
        const int slot = lt % kWQ;
        if (lt >= kWQ) ok = mbar_wait(&ctl->wq_empty[slot], (uint32_t)((lt / kWQ - 1) & 1), abort_flag, err);
        if (!ok) break;
        int wi = dyn ? atomicAdd(p.work.next, 1) : (int)blockIdx.x + lt * (int)gridDim.x;
        if (wi > n_work) wi = n_work;
        ctl->wq[slot] = wi;
        mbar_arrive(&ctl->wq_full[slot]);
        if (wi >= n_work) break;
        const WorkItem wk = get_work<MX>(p, wi, n_it);
        if (lt > 0) ok = mbar_wait(&ctl->a_empty, (lt - 1) & 1, abort_flag, err);
        if (!ok) break;
        mbar_expect_tx(&ctl->a_full, a_bytes);
        for (int c = 0; c < p.kc; ++c)
          tma_load_2d(a_tiles + (size_t)c * a_chunk, &map_users, c * p.row_elems, wk.a_row, &ctl->a_full);
        if (p.tail_bytes)
          tma_load_2d(a_tiles + (size_t)p.kc * a_chunk, &map_users_t, tail_x, wk.a_row, &ctl->a_full);
        for (int j = wk.tb; j < wk.te && ok; ++j) {
          for (int h = 0; h < bs; ++h, ++g) {  // g: loads issued so far
            if (g >= p.stages) ok = mbar_wait(&ctl->b_empty[st], ph ^ 1u, abort_flag, err);
            if (!ok) break;
            mbar_expect_tx(&ctl->b_full[st], b_bytes);
            unsigned char* dst = b_tiles + (size_t)st * b_bytes;
            const int y = wk.b_row + j * kTileN + h * (int)sub_rows;
            for (int c = 0; c < p.kc; ++c)
              tma_load_2d(dst + (size_t)c * b_chunk, &map_items, c * p.row_elems, y, &ctl->b_full[st]);
            if (p.tail_bytes) tma_load_2d(dst + (size_t)p.kc * b_chunk, &map_items_t, tail_x, y, &ctl->b_full[st]);
            if (++st == p.stages) {
              st = 0;
              ph ^= 1u;
            }
          }
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
      const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(sub_rows >> 3) << 17) |
                             ((uint32_t)(kTileM >> 4) << 24);
      const uint32_t sbo = 8 * p.row_bytes;
      const int ksteps = p.row_bytes / 32;  // K = 16 BF16 = 32 bytes per MMA
      // descriptors of the first A chunk and of ring stage 0; every other
      // operand is a fixed address offset, added to the 14-bit address field
      // (addresses >> 4), as is the 32-byte step of each K = 16 slice
      const uint64_t a_desc0 = smem_desc(smem_u32(a_tiles), sbo, p.swizzle);
      const uint64_t b_desc0 = smem_desc(smem_u32(b_tiles), sbo, p.swizzle);
      const uint32_t a16 = a_chunk >> 4, b16 = b_chunk >> 4;
      const uint32_t stage16 = b_bytes >> 4;
      // the tail chunk: its own swizzle and row stride
      const uint32_t tsbo = 8 * p.tail_bytes;
      const int tsteps = p.tail_bytes / 32;
      const uint64_t a_tdesc = smem_desc(smem_u32(a_tiles + (size_t)p.kc * a_chunk), tsbo, p.tail_swizzle);
      const uint64_t b_tdesc0 = smem_desc(smem_u32(b_tiles + (size_t)p.kc * b_chunk), tsbo, p.tail_swizzle);
      long long g = 0;
      int st = 0;
      uint32_t ph = 0;   // ring pass parity
      int b = 0;         // accumulator of tile g
      uint32_t aph = 0;  // accumulator pass parity
      bool ok = true;
      for (int lt = 0; ok; ++lt) {
        const int slot = lt % kWQ;
        ok = mbar_wait(&ctl->wq_full[slot], (uint32_t)((lt / kWQ) & 1), abort_flag, err);
        if (!ok) break;
        const int wi = *(volatile int*)&ctl->wq[slot];
        mbar_arrive(&ctl->wq_empty[slot]);
        if (wi >= n_work) break;
        const WorkItem wk = get_work<MX>(p, wi, n_it);
        ok = mbar_wait(&ctl->a_full, lt & 1, abort_flag, err);
        if (!ok) break;
        tc_fence_after();
        for (int j = wk.tb; j < wk.te; ++j, ++g) {  // g: item tiles so far
          for (int h = 0; h < bs && ok; ++h) {
            ok = mbar_wait(&ctl->b_full[st], ph, abort_flag, err);
            if (ok && h == 0 && g >= 2) ok = mbar_wait(&ctl->acc_empty[b], aph ^ 1u, abort_flag, err);
            if (!ok) break;
            tc_fence_after();
            // this load's rows go to accumulator columns [h sub_rows, (h + 1) sub_rows)
            const uint32_t d = tmem + (uint32_t)(b * kTileN) + (uint32_t)h * sub_rows;
            const uint64_t bst = b_desc0 + (uint64_t)(st * stage16);
            for (int c = 0; c < p.kc; ++c) {
              const uint64_t ad = a_desc0 + (uint64_t)(c * a16);
              const uint64_t bd = bst + (uint64_t)(c * b16);
              for (int k = 0; k < ksteps; ++k)
                mma_bf16(d, ad + (uint64_t)(2 * k), bd + (uint64_t)(2 * k), idesc, (c | k) != 0);
            }
            const uint64_t btd = b_tdesc0 + (uint64_t)(st * stage16);
            for (int k = 0; k < tsteps; ++k)
              mma_bf16(d, a_tdesc + (uint64_t)(2 * k), btd + (uint64_t)(2 * k), idesc, 1u);
            mma_commit(&ctl->b_empty[st]);
            if (++st == p.stages) {
              st = 0;
              ph ^= 1u;
            }
          }
          if (!ok) break;
          mma_commit(&ctl->acc_full[b]);
          b ^= 1;
          if (b == 0) aph ^= 1u;
        }
        if (ok) mma_commit(&ctl->a_empty);
      }
      // all MMAs issued by this thread complete before TMEM is released
      mma_commit(&ctl->drain);
      const unsigned long long t0 = globaltimer();
      while (!mbar_try_wait(&ctl->drain, 0) && globaltimer() - t0 < kWaitNs) {
      }
    }
  } else if (warp >= kEpiWarp0) {
    // ------------------------------------------------------------ select
    const int e = warp - kEpiWarp0;
    const int q = e % 4, c2 = e / 4;       // lane quarter, column half
    const int row = 32 * q + lane;         // user row within the tile
    const int slot = c2 * kTileM + row;    // this thread's index among the 256
    TcUser<KR> s;
    TcSel c;
    c.heap = heap_base + slot;
    c.K = p.K;
    c.cap = o.cap;
    c.qh = qh_base + slot;
    c.qp = qp_base + slot;
    c.tau_mine = tau_sh + slot;
    c.tau_partner = tau_sh + (c2 ^ 1) * kTileM + row;
    c.seed_mine = seed_sh + slot;
    c.seed_partner = seed_sh + (c2 ^ 1) * kTileM + row;
    c.seed_list = seed_lists + slot;
    c.seed_list_partner = seed_lists + (c2 ^ 1) * kTileM + row;
    c.g = p.g;
    long long g = 0;
    bool ok = true;
    unsigned long long emitted = 0, slow = 0;
    // this warp's copy of the bound columns and item positions of its 128
    // items of the current tile, prefetched one tile ahead into registers
    // (4 entries per lane); the tile after the last of a work item is the
    // first of the CTA's next work item
    float2* aux_tile = aux_base + (size_t)e * kHalfN;
    int32_t* pos_tile = posb_base + (size_t)e * kHalfN;
    float2 pre[4];
    int32_t prep[4];
    auto prefetch = [&](int64_t brow0) {  // B row of this warp's first column
#pragma unroll
      for (int t = 0; t < 4; ++t) {
        const int64_t br = brow0 + lane * 4 + t;
        pre[t] = item_aux[br];
        if constexpr (MX) prep[t] = p.work.item_pos[br];
      }
    };
    // the index of the CTA's lt-th work item (waits for the producer to
    // publish it; warp-uniform)
    auto peek_work = [&](int lt_, int* wi_out) {
      bool okp = mbar_wait(&ctl->wq_full[lt_ % kWQ], (uint32_t)((lt_ / kWQ) & 1), abort_flag, err);
      okp = __all_sync(0xffffffffu, okp);
      *wi_out = okp ? *(volatile int*)&ctl->wq[lt_ % kWQ] : n_work;
      return okp;
    };
    {
      int w0i = n_work;
      ok = peek_work(0, &w0i);
      if (ok && w0i < n_work) {
        const WorkItem w0 = get_work<MX>(p, w0i, n_it);
        prefetch((int64_t)w0.b_row + (int64_t)w0.tb * kTileN + c2 * kHalfN);
      }
    }
    for (int lt = 0; ok; ++lt) {  // work items of this CTA
      int wi = n_work;
      ok = peek_work(lt, &wi);
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->wq_empty[lt % kWQ]);
      if (!ok || wi >= n_work) break;
      const WorkItem wk = get_work<MX>(p, wi, n_it);
      const int64_t u = MX ? (int64_t)p.work.row_user[wk.a_row + row] : (int64_t)wk.a_row + row;
      const bool active = u >= 0 && u < p.n_users;
      s.tau = active ? kNegInf : __int_as_float(0x7f800000);  // inactive: never a hit
      s.tau_eff = s.tau;
      s.n_cand = 0;
      s.ut = wi;
      s.beta_u = 0.f;
      s.nhat_u = 0.f;
      const int lbase = (MX && p.work.l_base) ? p.work.l_base[wk.q] : 0;
      const int64_t list = (active ? u : 0) * (int64_t)o.lists + lbase + c2;
      const bool restoring = MX && p.work.restore && wk.tb > 0;
      c.cand_pos = o.cand_pos + list * (int64_t)o.cap;
      c.cand_ub = o.cand_ub + list * (int64_t)o.cap;
      c.tau_glob = (active && o.tau_glob) ? o.tau_glob + u : nullptr;
      topk_init(s, c);
      if (active) {
        const float2 ua = user_aux[u];
        s.beta_u = ua.x;
        s.nhat_u = ua.y;
        if (restoring) {  // continue a walk: restore the select state
          s.n_cand = o.n_cand[list];
          const float* src = o.topl + list * (int64_t)p.K;
          if constexpr (KR > 0) {
#pragma unroll
            for (int i = 0; i < KR; ++i) s.d[i] = i < p.K ? src[i] : kNegInf;
            s.tau = s.d[0];
#pragma unroll
            for (int i = 0; i < KR; ++i) s.tau = (i < p.K) ? s.d[i] : s.tau;
          } else {  // the row is descending: reversed, it is a min-heap
            for (int i = 0; i < p.K; ++i) c.heap[i * kEpiThreads] = src[p.K - 1 - i];
            s.tau = c.heap[0];
          }
          s.tau_eff = fmaxf(s.tau, o.tau[list]);
          tc_publish(s, c);
        }
      }
      for (int j = wk.tb; j < wk.te; ++j, ++g) {
        const int b = (int)(g & 1);
        ok = mbar_wait(&ctl->acc_full[b], (uint32_t)((g >> 1) & 1), abort_flag, err);
        // lanes leave together: the tcgen05.ld below needs the whole warp
        ok = __all_sync(0xffffffffu, ok);
        if (!ok) break;
        tc_fence_after();
        __syncwarp();  // the previous tile's offers are done with aux_tile / pos_tile
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          aux_tile[lane * 4 + t] = pre[t];
          if constexpr (MX) pos_tile[lane * 4 + t] = prep[t];
        }
        __syncwarp();
        if constexpr (MX) {
          if (j + 1 < wk.te) {
            prefetch((int64_t)wk.b_row + (int64_t)(j + 1) * kTileN + c2 * kHalfN);
          } else {  // the first tile of the next work item, once published
            int wni = n_work;
            if (peek_work(lt + 1, &wni) && wni < n_work) {
              const WorkItem wn = get_work<MX>(p, wni, n_it);
              prefetch((int64_t)wn.b_row + (int64_t)wn.tb * kTileN + c2 * kHalfN);
            }
          }
        } else {  // next tile (wraps to the first of the next user tile)
          prefetch((int64_t)((j + 1 < n_it) ? j + 1 : 0) * kTileN + c2 * kHalfN);
        }
        {  // the partner's threshold, if it is for this work item
          const unsigned long long pt = *c.tau_partner;
          if ((int)(pt >> 32) == wi) s.tau_eff = fmaxf(s.tau_eff, __uint_as_float((uint32_t)pt));
          // and the one shared by the user's other item chunks (zero bits: none yet, NaN, ignored)
          if constexpr (MX)
            if (c.tau_glob) s.tau_eff = fmaxf(s.tau_eff, tau_from_ord(*(volatile unsigned*)c.tau_glob));
        }
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kTileN + c2 * kHalfN);
        const int32_t rank0 = j * kTileN + c2 * kHalfN;  // (list) rank of this thread's first column
        const int valid = (int)min((int64_t)kHalfN, p.n_items - rank0);
        uint32_t r[64];
        const bool first = j == wk.tb && !restoring;  // a fresh work item's first tile
        if (first) {  // warp-uniform: tcgen05.ld is a warp-collective instruction
          // (inactive lanes hold tau = +inf and insert nothing)
#pragma unroll 1
          for (int h = 0; h < 2; ++h) {
            tmem_ld64(taddr + 64 * h, r);
            seed64(s, c, r, 64 * h, valid - 64 * h, aux_tile);
          }
          if (active) {
            s.tau_eff = s.tau;
            tc_publish(s, c);
            if constexpr (KR > 0) seed_merge(s, c, wi, lt & 1);
          }
        }
        // the two 64-column halves run through one copy of the select code
        // (a second inlined copy costs more in instruction-cache misses)
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          tmem_ld64(taddr + 64 * h, r);
          select64<KR, MX>(s, c, r, 64 * h, valid - 64 * h, aux_tile, rank0, pos_tile, slow, first);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) mbar_arrive(&ctl->acc_empty[b]);
      }
      if (!ok) break;
      if (active) {
        o.tau[list] = s.tau_eff;
        o.n_cand[list] = s.n_cand;
        emitted += (unsigned long long)s.n_cand;
        if (o.topl) {  // the K largest lower bounds this thread kept
          float* dst = o.topl + list * (int64_t)p.K;
          if constexpr (KR > 0) {
#pragma unroll
            for (int i = 0; i < KR; ++i)
              if (i < p.K) dst[i] = s.d[i];
          } else {  // heap sort: the minima, popped in turn, fill the row from the back
            for (int n = p.K; n > 0; --n) {
              dst[n - 1] = c.heap[0];
              if (n > 1) heap_replace_min(c.heap, kEpiThreads, n - 1, c.heap[(n - 1) * kEpiThreads]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) emitted += __shfl_xor_sync(0xffffffffu, emitted, off);
    if (lane == 0 && emitted) atomicAdd(&stats->cand_emitted, emitted);
    if (lane == 0 && slow) atomicAdd(&stats->select_slow, slow);  // warp-level slow-path entries
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 2) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
  }
}

}  // namespace

size_t tc_smem_bytes(const TcParams& p) {
  const size_t sub_rows = kTileN / (p.b_split > 0 ? p.b_split : 1);
  const size_t a_chunk = (size_t)kTileM * p.row_bytes, b_chunk = sub_rows * p.row_bytes;
  const size_t heap = p.K > kRegTopK && !p.heap_global ? sizeof(float) * (size_t)p.K * kEpiThreads : 0;
  const size_t a_bytes = (size_t)p.kc * a_chunk + (size_t)kTileM * p.tail_bytes;
  const size_t b_bytes = (size_t)p.kc * b_chunk + sub_rows * p.tail_bytes;
  return 1024 + a_bytes + (size_t)p.stages * b_bytes + heap +
         (sizeof(float2) + sizeof(int32_t)) * kEpiWarps * kHalfN + 2 * sizeof(float) * kQueue * kEpiThreads +
         sizeof(unsigned long long) * kEpiThreads + 2 * sizeof(int) * kEpiThreads +
         (p.K <= kRegTopK ? 2 * sizeof(float) * (size_t)p.K * kEpiThreads : 0) + sizeof(Smem);
}

int tc_users_per_tile() { return kTileM; }
int tc_items_per_tile() { return kTileN; }
int tc_items_box(const TcParams& p) { return kTileN / (p.b_split > 0 ? p.b_split : 1); }

namespace {

template <int KR, bool MX>
cudaError_t launch_variant(const CUtensorMap* mu, const CUtensorMap* mut, const CUtensorMap* mi, const CUtensorMap* mit,
                           const TcParams& p, SelectOut o, const float2* user_aux, const float2* item_aux,
                           DevStats* stats, int* err, int grid, size_t smem, cudaStream_t s) {
  cudaError_t e =
      cudaFuncSetAttribute(tc_score_select_kernel<KR, MX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  tc_score_select_kernel<KR, MX><<<grid, kWarps * 32, smem, s>>>(*mu, *mut, *mi, *mit, p, o, user_aux, item_aux,
                                                                 stats, err);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_tc_score_select(const CUtensorMap* map_users, const CUtensorMap* map_users_tail,
                                   const CUtensorMap* map_items, const CUtensorMap* map_items_tail, const TcParams& p,
                                   SelectOut o, const float2* user_aux, const float2* item_aux, DevStats* stats,
                                   int* err, int grid, cudaStream_t s) {
  // at least half the SM's shared memory: one CTA per SM, so no two CTAs
  // ever compete for the TMEM columns this kernel allocates
  size_t smem = tc_smem_bytes(p);
  int max_smem = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (smem < (size_t)max_smem / 2 + 1024) smem = (size_t)max_smem / 2 + 1024;
  const bool mx = p.mode != 0;
  // register top-K sized to K: the insertion cost grows with the array
#define MIPS_TC_LAUNCH(KR)                                                                                       \
  return mx ? launch_variant<KR, true>(map_users, map_users_tail, map_items, map_items_tail, p, o, user_aux,   \
                                       item_aux, stats, err, grid, smem, s)                                    \
            : launch_variant<KR, false>(map_users, map_users_tail, map_items, map_items_tail, p, o, user_aux,  \
                                        item_aux, stats, err, grid, smem, s)
  if (p.K == 1) MIPS_TC_LAUNCH(1);
  if (p.K <= 10) MIPS_TC_LAUNCH(10);
  if (p.K <= kRegTopK) MIPS_TC_LAUNCH(kRegTopK);
  MIPS_TC_LAUNCH(0);
#undef MIPS_TC_LAUNCH
}

}  // namespace mips
