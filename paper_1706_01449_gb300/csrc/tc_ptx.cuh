// Inline-PTX building blocks shared by the tcgen05 kernels (tc_topk.cu,
// kmeans_tc.cu): mbarriers with bounded waits, TMA and bulk copies, the
// shared-memory matrix descriptor, MMA issue and commit, TMEM loads.
#pragma once
#include <cuda.h>
#include <cstdint>

#include "common.cuh"

namespace mips {

namespace {

constexpr unsigned long long kWaitNs = 1000000000ull;  // 1 s
constexpr unsigned kFull = 0xffffffffu;

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

// What a bounded wait needs: the CTA's abort flag, the error word, and the
// wait limit (1 s; shorter only when a test asks for it).
struct Guard {
  volatile int* abort_flag;
  int* err;
  unsigned long long wait_ns;
};

// Bounded wait for the phase with the given parity.  Returns false when the
// CTA is aborting (this or another role timed out).
__device__ __noinline__ bool mbar_wait_slow(uint64_t* bar, uint32_t parity, Guard gd) {
  const unsigned long long t0 = globaltimer();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (*gd.abort_flag) return false;
    if (globaltimer() - t0 > gd.wait_ns) {
      *gd.abort_flag = 1;
      atomicOr(gd.err, DEV_ERR_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity, const Guard& gd) {
  if (mbar_try_wait(bar, parity)) return true;
  return mbar_wait_slow(bar, parity, gd);
}

// Non-blocking test of the phase with the given parity.
__device__ __forceinline__ bool mbar_test_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred P1;\n\t"
      "mbarrier.test_wait.parity.shared::cta.b64 P1, [%1], %2;\n\t"
      "selp.b32 %0, 1, 0, P1;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// The same bounded wait as mbar_wait, spinning on the non-blocking test (no
// suspend, so no wake-up delay) and looking at the abort flag and the
// timer once every 64 tests.  For a thread whose wait is on the critical
// path and that shares its sub-partition with little else.
__device__ __noinline__ bool mbar_spin_slow(uint64_t* bar, uint32_t parity, Guard gd) {
  const unsigned long long t0 = globaltimer();
  while (true) {
    for (int i = 0; i < 64; ++i)
      if (mbar_test_wait(bar, parity)) return true;
    if (*gd.abort_flag) return false;
    if (globaltimer() - t0 > gd.wait_ns) {
      *gd.abort_flag = 1;
      atomicOr(gd.err, DEV_ERR_TIMEOUT);
      return false;
    }
  }
}

__device__ __forceinline__ bool mbar_spin(uint64_t* bar, uint32_t parity, const Guard& gd) {
  if (mbar_test_wait(bar, parity)) return true;
  return mbar_spin_slow(bar, parity, gd);
}

// Wait (bounded) for a phase whose completion nothing else depends on any
// more: used only to drain copies and MMAs before the CTA exits.
__device__ __forceinline__ void mbar_drain(uint64_t* bar, uint32_t parity) {
  const unsigned long long t0 = globaltimer();
  while (!mbar_try_wait(bar, parity) && globaltimer() - t0 < kWaitNs) {
  }
}

__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::
          "r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Untiled bulk copy global -> shared (both addresses 16-byte aligned, bytes a
// multiple of 16), completing on the mbarrier's transaction count.
__device__ __forceinline__ void bulk_load(void* smem_dst, const void* gmem_src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(gmem_src)), "r"(bytes), "r"(smem_u32(bar))
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

// One MMA; ACC (compile time): 0 overwrites the accumulator, 1 adds to it.
template <int ACC>
__device__ __forceinline__ void mma_bf16(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "n"(ACC)
      : "memory");
}

// One FP8 MMA (E4M3 x E4M3 -> FP32, kind::f8f6f4, K = 32); ACC as for
// mma_bf16.
template <int ACC>
__device__ __forceinline__ void mma_f8(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "n"(ACC)
      : "memory");
}

// K steps (K = 16 each) of one operand row, at most: two full 64-element
// chunks and a 32-element tail (f = 128 needs 8 + 1).
constexpr int kMaxSteps = 10;

// The N MMAs of one item load, fully unrolled: a single thread issues them
// back to back, so a loop, a branch or a computed predicate per MMA would
// add issue time the tensor pipe waits for.  aoff, boff: the user-tile slot
// and the item load's ring stage (descriptor address units).
template <int N, bool F8 = false>
__device__ __forceinline__ void mma_steps(uint32_t d, const uint64_t (&a_d)[kMaxSteps],
                                          const uint64_t (&b_d)[kMaxSteps], uint64_t aoff, uint64_t boff,
                                          uint32_t idesc) {
  if constexpr (F8) {
    mma_f8<0>(d, a_d[0] + aoff, b_d[0] + boff, idesc);
#pragma unroll
    for (int s = 1; s < N; ++s) mma_f8<1>(d, a_d[s] + aoff, b_d[s] + boff, idesc);
  } else {
    mma_bf16<0>(d, a_d[0] + aoff, b_d[0] + boff, idesc);
#pragma unroll
    for (int s = 1; s < N; ++s) mma_bf16<1>(d, a_d[s] + aoff, b_d[s] + boff, idesc);
  }
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

#define MIPS_R8(r, o)                                                                                       \
  "=r"(r[o + 0]), "=r"(r[o + 1]), "=r"(r[o + 2]), "=r"(r[o + 3]), "=r"(r[o + 4]), "=r"(r[o + 5]), "=r"(r[o + 6]), \
      "=r"(r[o + 7])
#define MIPS_R16(r, o) MIPS_R8(r, o), MIPS_R8(r, o + 8)
#define MIPS_R64(r) MIPS_R16(r, 0), MIPS_R16(r, 16), MIPS_R16(r, 32), MIPS_R16(r, 48)

// The TMEM loads are warp-collective (.sync.aligned): every lane must issue
// the same load together, so each wrapper first reconverges the warp (the
// select's offer loops before a load diverge lane by lane).

// 32 lanes x 32 bits, 64 consecutive columns, reduced: this thread's maximum
// of its lane's 64 columns (the values themselves are not used).
__device__ __forceinline__ float tmem_ldmax64(uint32_t taddr) {
  uint32_t r[64];  // destinations the instruction needs; only the maximum is read
  float m;
  __syncwarp();
  asm volatile(
      "tcgen05.ld.red.sync.aligned.32x32b.x64.max.f32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,"
      "%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,"
      "%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, %64, [%65];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : MIPS_R64(r), "=f"(m)
      : "r"(taddr)
      : "memory");
  (void)r;
  return m;
}

// 64 consecutive columns with their values: r[j] = column (col + j) of this
// thread's lane, and their maximum.
__device__ __forceinline__ float tmem_ldmax64v(uint32_t taddr, uint32_t (&r)[64]) {
  float m;
  __syncwarp();
  asm volatile(
      "tcgen05.ld.red.sync.aligned.32x32b.x64.max.f32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,"
      "%28,%29,%30,%31,%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,"
      "%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, %64, [%65];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : MIPS_R64(r), "=f"(m)
      : "r"(taddr)
      : "memory");
  return m;
}

// One MMA with the accumulate flag in a register (0 overwrites).
__device__ __forceinline__ void mma_bf16_rt(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                            uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

// 16 consecutive columns: r[j] = column (col + j) of this thread's lane, and
// their maximum.
__device__ __forceinline__ float tmem_ldmax16(uint32_t taddr, uint32_t (&r)[16]) {
  float m;
  __syncwarp();
  asm volatile(
      "tcgen05.ld.red.sync.aligned.32x32b.x16.max.f32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, %16, "
      "[%17];\n\t"
      "tcgen05.wait::ld.sync.aligned;"
      : MIPS_R16(r, 0), "=f"(m)
      : "r"(taddr)
      : "memory");
  return m;
}

// 8 consecutive columns, no wait: the caller reads r only after
// tmem_wait_ld8(r), whose operands tie the wait to these registers.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&r)[8]) {
  __syncwarp();
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];" : MIPS_R8(r, 0) : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld8(uint32_t (&r)[8]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7])
               :
               : "memory");
}

#undef MIPS_R64
#undef MIPS_R16
#undef MIPS_R8

}  // namespace

}  // namespace mips
