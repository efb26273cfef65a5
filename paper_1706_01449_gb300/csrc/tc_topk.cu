// Fused BF16 / FP8 blocked multiply + top-K candidate select on tcgen05 tensor
// cores (the paper's BMM, Sec. II-C, with the per-user selection fused so
// the |U| x |I| score matrix never leaves the SM), and the same machinery
// walking Maximus's per-cluster item lists (Sec. III, Algorithm 1).
//
// Persistent kernel, one CTA per SM, 12 warps, user tiles of 128 rows and
// item tiles of 256 rows (an M = 128, N = 256 MMA runs at the tensor pipe's
// full rate):
//   warps 0-7   select: epilogue warp e reads TMEM lanes 32 * (e % 4) .. +31
//               (a warp may only touch the lane quarter of its warp % 4) and
//               columns 128 * (e / 4) .. +127 of each item tile, so every
//               user is served by two threads, each with its own threshold,
//               top-K of lower bounds and candidate sub-list; the two share
//               their thresholds through shared memory (either one is a valid
//               lower bound on the user's K-th score, so the larger filters
//               both halves);
//   warp 8      allocates / frees TMEM; its lane 0 is the TMA producer: it
//               takes the CTA's next work item (user tile x
//               range of item tiles), publishes it in a shared-memory ring
//               for the other roles, loads the user tile, then the item
//               tiles through an S-stage ring (whole tiles, or two 128-row
//               halves when whole tiles do not fit shared memory; operand
//               rows of 128-byte chunks plus a 32/64-byte tail chunk, each
//               with its own tensor map and swizzle);
//   warps 9-10  MMA issuers (lane 0 of each): D = A . B^T with tcgen05.mma
//               kind::f16 (BF16 x BF16 -> FP32) or kind::f8f6f4 (E4M3 x
//               E4M3 -> FP32, entries scaled by s_u s_I) into two TMEM
//               accumulators of 128 lanes x 256 columns, so the MMAs of item
//               tile j+1 overlap the select of tile j.  Warp 9 issues the
//               even item tiles (accumulator 0), warp 10 the odd ones
//               (accumulator 1): a thread's tcgen05 instructions and barrier
//               waits queue behind its own MMAs, so one thread leaves the
//               tensor pipe idle while it waits for and sets up the next
//               tile; with two, each waits while the other's MMAs run.
//               (Only where even and odd tiles use disjoint ring stages;
//               otherwise warp 9 issues every tile.)
//   warp 11     lane 0 copies each item tile's bound columns (and, for list
//               walks, its item positions) into a small ring the select
//               warps read.  Like the MMA issue, the producer's copies are
//               split over threads so that neither thread's queue of barrier
//               and copy instructions sets the pace, and so that an item
//               tile's operand load waits only for its ring stage's MMAs,
//               not for the select of the tile whose bound-column slot it
//               reuses.
// The select's common case is one max-reducing TMEM load per 64 scores
// (tcgen05.ld.red: the values and each thread's maximum of them) and one
// warp vote: the operands carry two bound columns, so every accumulator
// entry is an upper bound H >= u^T i and a maximum below the threshold
// clears 64 items at once.  Only 16-column groups holding a hit are looked
// at item by item, from a second, narrow TMEM load.
// Work items: without a work list (blocked multiply) user tile w against
// every item tile; with one (item-chunked blocked multiply, Maximus walk)
// as the list gives them, claimed round-robin or from a global counter.
//
// Every mbarrier wait is bounded (1 s of %globaltimer); on expiry the kernel
// raises DEV_ERR_TIMEOUT, every role leaves its loop, the MMA issuers drain
// their in-flight MMAs and the producer its in-flight copies (each with a
// bounded wait), and TMEM is freed before exit.
#include <cuda.h>
#include <cuda_bf16.h>

#include <type_traits>

#include "common.cuh"
#include "tc_ptx.cuh"
#include "tc_topk.h"

namespace mips {

namespace {

constexpr int kWarps = 12;
constexpr int kEpiWarps = 8;   // warps 0-7 select
constexpr int kProdWarp = 8;   // producer (lane 0) and TMEM allocation (whole warp)
constexpr int kMmaWarp = 9;    // MMA issuer of accumulator 0 (lane 0)
constexpr int kMmaWarp2 = 10;  // MMA issuer of accumulator 1 (lane 0)
constexpr int kAuxWarp = 11;   // bound-column (and list-position) copies (lane 0)
constexpr int kEpiThreads = kEpiWarps * 32;
constexpr int kTileN = 256;    // items per tile (MMA N)
constexpr int kTileM = 128;    // users per tile (MMA M)
constexpr int kHalfN = 128;    // columns per epilogue thread and tile
constexpr int kQueue = 16;     // staging slots per thread: one 16-column group of scores
constexpr int kAuxSlots = 4;   // item tiles whose bound columns / positions are staged at a time

// A threshold published for the partner thread, tagged with its work item
// so that a value from another work item is never taken.
__device__ __forceinline__ unsigned long long pack_tau(float t, int ut) {
  return ((unsigned long long)(uint32_t)ut << 32) | (unsigned long long)__float_as_uint(t);
}

// float <-> unsigned with the same order (for atomicMax on thresholds)
__device__ __forceinline__ unsigned tau_ord(float x) {
  const unsigned b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float tau_from_ord(unsigned o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Per-thread select state (registers).  KR > 0: the K largest lower bounds
// live in a register array d[0..KR-1] sorted descending (K <= KR); KR = 0:
// in the shared-memory min-heap of common.cuh.
template <int KR>
struct TcUser {
  float tau;      // this thread's K-th largest lower bound so far
  float tau_eff;  // max(tau, partner thread's tau, merged seed lists): the filter threshold
  int n_cand;
  int ut;         // current work item (tag of the published threshold)
  float beta_u, nhat_u;  // bound columns of this user (prep.cu)
  float au, am;          // FP8: user_scale[u] * item_scale (the accumulator's unit) and 2^-21; BF16: 1 and 0
  float d[KR > 0 ? KR : 1];
};

// Per-thread arrays in shared memory, one column per select thread (slot
// 0..255), laid out back to back from `qbase`:
//   staged scores of a hit group [16][256] floats,
//   published thresholds [256] (64-bit: tag << 32 | float bits),
//   seed-list tags [2][256] ints (work item whose first-tile list is
//   published, -1: none), first-tile top-K lists [2][K][256] floats.
constexpr int kTauOfs = kQueue * kEpiThreads;  // in 4-byte words from qbase (8-byte aligned)
constexpr int kSeedTagOfs = kTauOfs + 2 * kEpiThreads;
constexpr int kSeedListOfs = kSeedTagOfs + 2 * kEpiThreads;

// Parameters of one select thread (warp-uniform but for the slots).
struct TcSel {
  float* heap;        // &heap_base[slot] (stride kEpiThreads), KR = 0 only
  int K;
  int cap;
  int32_t* cand_pos;  // this thread's candidate sub-list
  float* cand_ub;
  int64_t n_items;    // positions emitted must lie in [0, n_items)
  int* err;
  float* qbase;       // the per-thread arrays above
  int slot, pslot;    // this thread's column and its partner's (the other half of the same user)
  unsigned* tau_glob;  // this user's shared threshold (item-chunked scan) or null
  float g;            // accumulation-error factor of prep.cu
  bool f8;            // FP8 operands: accumulator entries are scaled (hv)
  __device__ __forceinline__ float* qh() const { return qbase + slot; }  // qh()[t * kEpiThreads]
  __device__ __forceinline__ volatile unsigned long long* tau(int sl) const {
    return (volatile unsigned long long*)(qbase + kTauOfs) + sl;
  }
  __device__ __forceinline__ volatile int* seed_tag(int sl) const { return (volatile int*)qbase + kSeedTagOfs + sl; }
  __device__ __forceinline__ volatile float* seed_list(int sl) const { return qbase + kSeedListOfs + sl; }
};

// An accumulator entry in input units: BF16 entries are scores already;
// FP8 entries count in units of au = s_u s_I.  The scaled value gets an
// upward margin am = 2^-21 of its size for the roundings of au and of the
// product (2^-24 each), so it stays an upper bound; the map is increasing,
// so the maximum of scaled entries is the scaled maximum.  No branch: BF16
// threads hold au = 1 and am = 0, which return the entry itself.
template <int KR>
__device__ __forceinline__ float hv(const TcUser<KR>& s, const TcSel&, float raw) {
  const float t = s.au * raw;
  return __fmaf_rn(fabsf(t), s.am, t);
}

template <int KR>
__device__ __forceinline__ void topk_init(TcUser<KR>& s, const TcSel& c) {
  if constexpr (KR > 0) {
#pragma unroll
    for (int i = 0; i < KR; ++i) s.d[i] = kNegInf;
  } else {
    heap_init(c.heap, kEpiThreads, c.K);
  }
}

// The K-th largest kept value (static indices keep d in registers).
template <int KR>
__device__ __forceinline__ float topk_kth(const TcUser<KR>& s, int K) {
  float t = s.d[0];
#pragma unroll
  for (int i = 0; i < KR; ++i) t = (i < K) ? s.d[i] : t;
  return t;
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
    return topk_kth(s, c.K);
  } else {
    return heap_replace_min(c.heap, kEpiThreads, c.K, L);
  }
}

// Branch-free insertion of any L into the descending array d (the smallest
// entry drops out; an L below all of them changes nothing): entry i becomes
// max(d[i], min(d[i-1], L)), two instructions per entry and no divergence
// between lanes.
template <int KR>
__device__ __forceinline__ void topk_push(TcUser<KR>& s, float L) {
  float prev = s.d[0];
  s.d[0] = fmaxf(prev, L);
#pragma unroll
  for (int i = 1; i < KR; ++i) {
    const float cur = s.d[i];
    s.d[i] = fmaxf(cur, fminf(prev, L));
    prev = cur;
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

// Publish this thread's threshold (tagged with its work item) for the partner.
template <int KR>
__device__ __forceinline__ void tc_publish(const TcUser<KR>& s, const TcSel& c) {
  *c.tau(c.slot) = pack_tau(s.tau, s.ut);
  if (c.tau_glob) atomicMax(c.tau_glob, tau_ord(s.tau));  // every threshold is valid for the user
}

// One hit: column col of the tile, whose staged upper bound H reached the
// threshold when it was staged.  Threshold update from its lower bound,
// then the candidate emission; lower bounds at or below the current filter
// threshold cannot raise it and are not kept.  The item's position is
// pos0 + col, or pos[col] for a walk of a cluster's sorted list (MX).  The
// three loads (H, the item's bound columns, its position) are issued first,
// and only the rare threshold publication and the stores are conditional:
// the register top-K takes the lower bound through its branch-free network
// (-inf when it does not qualify, which changes nothing).
template <int KR, bool MX>
__device__ __forceinline__ void tc_offer(TcUser<KR>& s, const TcSel& c, const float* Hp, int col, const float2* aux,
                                         int32_t pos0, const int32_t* pos) {
  const float H = *Hp;
  const float2 ia = aux[col];
  const int32_t ip = MX ? pos[col] : pos0 + col;
  const bool live = H >= s.tau_eff;  // (the threshold may have risen since the hit was staged)
  const float L = tc_lower(s, c, H, ia);
  const bool ins = live && L > s.tau_eff;
  if constexpr (KR > 0) {
    topk_push(s, ins ? L : kNegInf);
    s.tau = c.K == KR ? s.d[KR - 1] : topk_kth(s, c.K);
  } else {
    if (ins) s.tau = topk_insert(s, c, L);
  }
  if (s.tau > s.tau_eff) {
    s.tau_eff = s.tau;
    tc_publish(s, c);
  }
  const bool em = live && H >= s.tau_eff;
  const bool in = ip >= 0 && ip < c.n_items;
  if (em && !in) atomicOr(c.err, DEV_ERR_INTERNAL);  // never for consistent lists: flagged, not emitted
  if (em && in && s.n_cand < c.cap) {
    c.cand_pos[s.n_cand] = ip;
    c.cand_ub[s.n_cand] = H;
  }
  s.n_cand += (em && in) ? 1 : 0;
}

// Seed step of the heap-held top-K for 8 columns col0.. of the first item
// tile: every lower bound that passes the heap's minimum goes in.
template <int KR>
__device__ __forceinline__ void seed8_heap(TcUser<KR>& s, const TcSel& c, const uint32_t (&r)[8], int col0,
                                           int valid, const float2* aux) {
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    const float L = col0 + q < valid ? tc_lower(s, c, hv(s, c, __uint_as_float(r[q])), aux[col0 + q]) : kNegInf;
    if (L > s.tau) s.tau = heap_replace_min(c.heap, kEpiThreads, c.K, L);
  }
}

// The two largest of 8 values (hi >= lo): pairwise maxima and minima, then
// three merges of (max, second) pairs.
__device__ __forceinline__ void top2_of8(const float (&x)[8], float& hi, float& lo) {
  float a[4], b[4];
#pragma unroll
  for (int p = 0; p < 4; ++p) {
    a[p] = fmaxf(x[2 * p], x[2 * p + 1]);
    b[p] = fminf(x[2 * p], x[2 * p + 1]);
  }
  const float h01 = fmaxf(a[0], a[1]), l01 = fmaxf(fminf(a[0], a[1]), fmaxf(b[0], b[1]));
  const float h23 = fmaxf(a[2], a[3]), l23 = fmaxf(fminf(a[2], a[3]), fmaxf(b[2], b[3]));
  hi = fmaxf(h01, h23);
  lo = fmaxf(fminf(h01, h23), fmaxf(l01, l23));
}

// Register top-K seed step for 8 columns: each column's lower bound, then
// the group's two largest go into the top-K (K = 1: its largest).
template <int KR>
__device__ __forceinline__ void seed8_reg(TcUser<KR>& s, const TcSel& c, const uint32_t (&r)[8], int col0,
                                          int valid, const float2* aux) {
  float L[8];
#pragma unroll
  for (int q = 0; q < 8; ++q)
    L[q] = col0 + q < valid ? tc_lower(s, c, hv(s, c, __uint_as_float(r[q])), aux[col0 + q]) : kNegInf;
  float hi, lo;
  top2_of8(L, hi, lo);
  if constexpr (KR == 1) {
    s.d[0] = fmaxf(s.d[0], hi);
  } else {
    topk_push(s, hi);
    topk_push(s, lo);
  }
}

// First pass over a fresh work item's first item tile (the items of largest
// norm: the index stores items by norm, descending), so that the threshold
// starts the scan near its final value instead of at -inf; nothing is
// emitted.  TMEM is read 8 columns at a time with the next 8 in flight.
// Register top-K: only the two largest lower bounds of each 8-column group
// are kept.  They belong to distinct items and the K-th largest of a subset
// is at most the K-th largest of the whole, so the K-th kept value is a
// valid threshold; it equals the tile's K-th largest lower bound unless some
// group holds three of the K largest.  Heap: every lower bound.
// Inactive lanes (padding rows) keep tau = +inf.
template <int KR>
__device__ __forceinline__ void seed_tile(TcUser<KR>& s, const TcSel& c, uint32_t taddr, int valid,
                                          const float2* aux, bool active) {
  uint32_t ra[8], rb[8];
  tmem_ld8(taddr, ra);
  tmem_wait_ld8(ra);
#pragma unroll 1
  for (int c8 = 0; c8 < kHalfN; c8 += 16) {
    tmem_ld8(taddr + c8 + 8, rb);
    if constexpr (KR > 0) seed8_reg(s, c, ra, c8, valid, aux);
    else seed8_heap(s, c, ra, c8, valid, aux);
    tmem_wait_ld8(rb);
    if (c8 + 16 < kHalfN) tmem_ld8(taddr + c8 + 16, ra);
    if constexpr (KR > 0) seed8_reg(s, c, rb, c8 + 8, valid, aux);
    else seed8_heap(s, c, rb, c8 + 8, valid, aux);
    if (c8 + 16 < kHalfN) tmem_wait_ld8(ra);
  }
  if constexpr (KR > 0) s.tau = active ? topk_kth(s, c.K) : __int_as_float(0x7f800000);
}

// After the seed: this thread's K best lower bounds go to its list slot for
// the work item's parity, under a tag that is cleared while the list is
// rewritten (so a reader that sees the same tag before and after reading
// the list has read it whole).
template <int KR>
__device__ __forceinline__ void seed_publish(const TcUser<KR>& s, const TcSel& c, int wi, int par) {
  if constexpr (KR > 0) {
    volatile int* flag = c.seed_tag(c.slot) + par * kEpiThreads;
    *flag = -1;
    __threadfence_block();
    volatile float* mine = c.seed_list(c.slot) + par * c.K * kEpiThreads;
#pragma unroll
    for (int i = 0; i < KR; ++i)
      if (i < c.K) mine[i * kEpiThreads] = s.d[i];
    __threadfence_block();
    *flag = wi;
  }
}

// Once the partner thread (the other half of the same user) has published
// its first-tile list for this work item: the K-th largest of the union of
// the two lists raises this thread's filter threshold (the halves hold
// distinct items, so the union's K-th largest lower bound is a lower bound
// on the user's K-th score).  Warp-uniform; returns true when there is
// nothing more to wait for (merged, or the list was overwritten meanwhile).
template <int KR>
__device__ __forceinline__ bool seed_try_merge(TcUser<KR>& s, const TcSel& c, int wi, int par, bool active) {
  if constexpr (KR > 0) {
    const volatile int* pflag = c.seed_tag(c.pslot) + par * kEpiThreads;
    if (!__all_sync(kFull, *pflag == wi)) return false;
    __threadfence_block();
    const volatile float* pq = c.seed_list(c.pslot) + par * c.K * kEpiThreads;
    int ia = 0, ib = 0;
    float v = kNegInf;
    for (int r = 0; r < c.K; ++r) {
      float a = kNegInf;
#pragma unroll
      for (int i = 0; i < KR; ++i)
        if (i == ia) a = s.d[i];
      const float b = pq[ib * kEpiThreads];
      if (a >= b) {
        v = a;
        ++ia;
      } else {
        v = b;
        ++ib;
      }
    }
    __threadfence_block();
    if (*pflag == wi && active && v > s.tau_eff) s.tau_eff = v;
  }
  return true;
}

// The 16-column groups of this thread's 128 columns whose 64-column half had
// a hit somewhere in the warp (bit h of `halves`): each group is read again
// with its maximum; a lane whose maximum reaches its threshold stages the
// group's 16 scores in shared memory (independent stores) and marks its hits
// in a bit mask, then offers them in column order (the index of a hit is its
// bit; no queue counter to wait on).
template <int KR, bool MX>
__device__ __forceinline__ void select_hits(TcUser<KR>& s, const TcSel& c, uint32_t taddr, int valid,
                                            const float2* aux, int32_t pos0, const int32_t* pos, unsigned halves) {
  float* const stage = c.qh();
#pragma unroll 1
  for (int gi = 0; gi < kHalfN / 16; ++gi) {
    if (!((halves >> (gi >> 2)) & 1u)) continue;  // warp-uniform
    uint32_t v[16];
    const float mg = hv(s, c, tmem_ldmax16(taddr + 16 * gi, v));
    const bool hit = mg >= s.tau_eff;
    if (!__any_sync(kFull, hit)) continue;
    const int col0 = 16 * gi;
    unsigned mask = 0;
    if (hit) {
      const float t = s.tau_eff;
      const int nv = valid - col0;  // columns of the group below `valid`
#pragma unroll
      for (int q = 0; q < 16; ++q) {
        const float x = hv(s, c, __uint_as_float(v[q]));
        stage[q * kEpiThreads] = x;
        mask |= (x >= t && q < nv) ? (1u << q) : 0u;
      }
    }
    while (mask) {
      const int q = __ffs(mask) - 1;
      mask &= mask - 1;
      tc_offer<KR, MX>(s, c, stage + q * kEpiThreads, col0 + q, aux, pos0, pos);
    }
  }
}

// A fresh work item's first item tile, after its seed: every column whose
// upper bound reaches the filter threshold becomes a candidate.  The seed
// already took the tile's lower bounds into the top-K, so nothing is
// inserted and the threshold does not move during the pass: a hit is only
// stored (position, H), without the offer's lower bound and insertion.
// Only the 16-column groups of the 64-column halves with a hit in the warp
// (`halves`) are read again.
template <int KR, bool MX>
__device__ __forceinline__ void emit_tile(TcUser<KR>& s, const TcSel& c, uint32_t taddr, int valid, int32_t pos0,
                                          const int32_t* pos, unsigned halves) {
  const float t = s.tau_eff;
  int n = s.n_cand;
  bool bad = false;
#pragma unroll 1
  for (int gi = 0; gi < kHalfN / 16; ++gi) {
    if (!((halves >> (gi >> 2)) & 1u)) continue;  // warp-uniform
    uint32_t v[16];
    const float mg = hv(s, c, tmem_ldmax16(taddr + 16 * gi, v));
    if (!__any_sync(kFull, mg >= t)) continue;
    const int col0 = 16 * gi;
    const int nv = valid - col0;
    // list walks: the group's 16 positions in four 16-byte loads (the ring
    // slot and the group start are 16-byte aligned; every lane reads the same)
    int4 p4[4] = {};
    if constexpr (MX) {
#pragma unroll
      for (int k = 0; k < 4; ++k) p4[k] = reinterpret_cast<const int4*>(pos + col0)[k];
    }
    // every column in turn, each store under its own predicate: the lanes
    // stay together however their hits are spread
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      const float x = hv(s, c, __uint_as_float(v[q]));
      const bool hit = x >= t && q < nv;
      const int4 pq = p4[q >> 2];
      const int32_t ip = MX ? ((q & 3) == 0 ? pq.x : (q & 3) == 1 ? pq.y : (q & 3) == 2 ? pq.z : pq.w)
                            : pos0 + col0 + q;
      const bool in = ip >= 0 && ip < c.n_items;
      bad |= hit && !in;
      if (hit && in && n < c.cap) {
        c.cand_pos[n] = ip;
        c.cand_ub[n] = x;
      }
      n += (hit && in) ? 1 : 0;
    }
  }
  // a position outside the item range is never written by consistent
  // lists; were one met, it is flagged rather than emitted
  if (bad) atomicOr(c.err, DEV_ERR_INTERNAL);
  s.n_cand = n;
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
// and publishes the index in ring slot lt % kWQ, where the MMA issuers and the
// select warps read it; an index >= n_work ends the sequence.
constexpr int kWQ = 4;

struct Smem {
  uint64_t b_full[kMaxStages];
  uint64_t b_empty[kMaxStages];
  uint64_t a_full[2], a_empty[2];  // user tiles: two slots, so the next one loads during the current one
  uint64_t acc_full[2], acc_empty[2];
  uint64_t aux_full[kAuxSlots], aux_empty[kAuxSlots];
  uint64_t drain;
  uint64_t wq_full[kWQ], wq_empty[kWQ];
  int wq[kWQ];
  uint32_t tmem_base;
  int abort_flag;
};

// Bytes of one aux ring slot: an item tile's bound columns, then (list walks)
// its item positions.
constexpr uint32_t kAuxBytes = kTileN * sizeof(float2);
constexpr uint32_t kPosBytes = kTileN * sizeof(int32_t);

// MX: work items from p.work (Maximus walk of per-cluster sorted lists,
// item-chunked blocked multiply); otherwise every user tile against every
// item tile (blocked multiply).
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
  unsigned char* a_tiles = base;                                              // [2]([KC][a_chunk] + tail)
  unsigned char* b_tiles = a_tiles + 2 * (size_t)a_bytes;                     // [S]([KC][b_chunk] + tail)
  float2* aux_ring = (float2*)(b_tiles + (size_t)p.stages * b_bytes);        // [kAuxSlots][256]
  int32_t* pos_ring = (int32_t*)(aux_ring + (size_t)kAuxSlots * kTileN);     // [kAuxSlots][256]
  float* heap_smem = (float*)(pos_ring + (size_t)kAuxSlots * kTileN);        // [K][256] (KR = 0)
  const bool heap_in_smem = KR == 0 && !p.heap_global;
  float* heap_base = heap_in_smem ? heap_smem : p.heap_mem + (size_t)blockIdx.x * p.K * kEpiThreads;
  float* qh_base = heap_smem + (heap_in_smem ? (size_t)p.K * kEpiThreads : 0);  // [16][256]
  unsigned long long* tau_sh = (unsigned long long*)(qh_base + (size_t)kQueue * kEpiThreads);  // [256]
  int* seed_sh = (int*)(tau_sh + kEpiThreads);                                                // [2][256]
  float* seed_lists = (float*)(seed_sh + 2 * kEpiThreads);  // [2][K][256] (KR > 0)
  Smem* ctl = (Smem*)(seed_lists + (KR > 0 ? (size_t)2 * p.K * kEpiThreads : 0));
  static_assert(kSeedListOfs == kQueue * kEpiThreads + 2 * kEpiThreads + 2 * kEpiThreads, "layout");

  const int warp = threadIdx.x / 32, lane = threadIdx.x & 31;
  const Guard gd{&ctl->abort_flag, err, p.wait_ns > 0 ? p.wait_ns : kWaitNs};
  const int n_it = (int)((p.n_items + kTileN - 1) / kTileN);
  const int n_work = MX ? *p.work.n_work : (int)((p.n_users + kTileM - 1) / kTileM);
  constexpr uint32_t kTmemCols = 2 * kTileN;  // two accumulators

  if (threadIdx.x == 0) {
    for (int s = 0; s < p.stages; ++s) {
      mbar_init(&ctl->b_full[s], 1);
      mbar_init(&ctl->b_empty[s], 1);
    }
    for (int a = 0; a < 2; ++a) {
      mbar_init(&ctl->a_full[a], 1);
      mbar_init(&ctl->a_empty[a], 2);  // a commit by each MMA issuer
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&ctl->acc_full[b], 1);
      mbar_init(&ctl->acc_empty[b], kEpiWarps);
    }
    for (int a = 0; a < kAuxSlots; ++a) {
      mbar_init(&ctl->aux_full[a], 1);
      mbar_init(&ctl->aux_empty[a], kEpiWarps);
    }
    mbar_init(&ctl->drain, 2);
    for (int w = 0; w < kWQ; ++w) {
      mbar_init(&ctl->wq_full[w], 1);
      mbar_init(&ctl->wq_empty[w], 3 + kEpiWarps);  // the MMA issuers, the bound-column copier, the select warps
    }
    ctl->abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  for (int i = threadIdx.x; i < kEpiThreads; i += blockDim.x) {
    tau_sh[i] = pack_tau(kNegInf, -1);
    seed_sh[i] = -1;
    seed_sh[kEpiThreads + i] = -1;
  }
  if (warp == kProdWarp) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&ctl->tmem_base)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = ctl->tmem_base;

  if (warp == kProdWarp) {
    // ------------------------------------------------------------ producer
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_users)) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&map_items)) : "memory");
      const int tail_x = p.kc * p.row_elems;  // element column of the tail chunk
      long long g = 0;   // item loads issued so far
      long long na = 0;  // user tiles loaded so far
      int st = 0;        // ring stage of load g
      uint32_t ph = 0;   // ring pass parity of load g
      bool ok = true;
      const bool dyn = MX && p.work.next;
      // a test of the bounded waits: publish no work item at all, so that
      // the MMA issuers, the bound-column copier and the select warps wait
      // for one until the limit
      if (p.test_withhold) ok = false;
      for (int lt = 0; ok; ++lt) {
        // take and publish the next work item
        const int slot = lt % kWQ;
        if (lt >= kWQ) ok = mbar_wait(&ctl->wq_empty[slot], (uint32_t)((lt / kWQ - 1) & 1), gd);
        if (!ok) break;
        int wi = dyn ? atomicAdd(p.work.next, 1) : (int)blockIdx.x + lt * (int)gridDim.x;
        if (wi > n_work) wi = n_work;
        ctl->wq[slot] = wi;
        mbar_arrive(&ctl->wq_full[slot]);
        if (wi >= n_work) break;
        const WorkItem wk = get_work<MX>(p, wi, n_it);
        const int asl = (int)(na & 1);  // user-tile slot of this work item
        if (na >= 2) ok = mbar_wait(&ctl->a_empty[asl], (uint32_t)(((na >> 1) - 1) & 1), gd);
        if (!ok) break;
        unsigned char* a_dst = a_tiles + (size_t)asl * a_bytes;
        mbar_expect_tx(&ctl->a_full[asl], a_bytes);
        for (int c = 0; c < p.kc; ++c)
          tma_load_2d(a_dst + (size_t)c * a_chunk, &map_users, c * p.row_elems, wk.a_row, &ctl->a_full[asl]);
        if (p.tail_bytes)
          tma_load_2d(a_dst + (size_t)p.kc * a_chunk, &map_users_t, tail_x, wk.a_row, &ctl->a_full[asl]);
        ++na;
        for (int j = wk.tb; j < wk.te && ok; ++j) {
          for (int h = 0; h < bs; ++h, ++g) {  // g: loads issued so far
            if (g >= p.stages) ok = mbar_wait(&ctl->b_empty[st], ph ^ 1u, gd);
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
      if (!ok) {  // drain the operand copies still in flight before the CTA exits
        for (long long gg = (g > p.stages ? g - p.stages : 0); gg < g; ++gg)
          mbar_drain(&ctl->b_full[gg % p.stages], (uint32_t)((gg / p.stages) & 1));
        for (long long aa = (na > 2 ? na - 2 : 0); aa < na; ++aa)
          mbar_drain(&ctl->a_full[aa & 1], (uint32_t)((aa >> 1) & 1));
      }
    }
  } else if (warp == kAuxWarp) {
    // ------------------------------------------------------------ bound-column copies
    if (lane == 0) {
      long long at = 0;  // item tiles whose bound columns (and positions) were copied so far
      bool ok = true;
      const uint32_t aux_tx = kAuxBytes + (MX ? kPosBytes : 0u);
      for (int lt = 0; ok; ++lt) {
        const int slot = lt % kWQ;
        ok = mbar_wait(&ctl->wq_full[slot], (uint32_t)((lt / kWQ) & 1), gd);
        if (!ok) break;
        const int wi = *(volatile int*)&ctl->wq[slot];
        mbar_arrive(&ctl->wq_empty[slot]);
        if (wi >= n_work) break;
        const WorkItem wk = get_work<MX>(p, wi, n_it);
        for (int j = wk.tb; j < wk.te && ok; ++j) {
          // the tile's bound columns (and list positions) into aux slot at % kAuxSlots,
          // once the select warps are done with the slot's last tile AND that
          // tile's copy has landed: the select warps wait for a copy only when
          // they read it, so nothing else orders it before this one (re-arming
          // the barrier while its previous phase still waits for bytes would
          // be an arrival too many, and the two copies would overlap)
          const int as = (int)(at % kAuxSlots);
          if (at >= kAuxSlots) {
            const uint32_t prev = (uint32_t)((at / kAuxSlots - 1) & 1);
            ok = mbar_wait(&ctl->aux_empty[as], prev, gd) && mbar_wait(&ctl->aux_full[as], prev, gd);
          }
          if (!ok) break;
          const int64_t row0 = (int64_t)wk.b_row + (int64_t)j * kTileN;
          mbar_expect_tx(&ctl->aux_full[as], aux_tx);
          bulk_load(aux_ring + (size_t)as * kTileN, item_aux + row0, kAuxBytes, &ctl->aux_full[as]);
          if constexpr (MX) bulk_load(pos_ring + (size_t)as * kTileN, p.work.item_pos + row0, kPosBytes, &ctl->aux_full[as]);
          ++at;
        }
      }
      // the select warps wait for a tile's bound columns only when they need
      // them: the last copies may still be landing, on either path
      for (long long aa = (at > kAuxSlots ? at - kAuxSlots : 0); aa < at; ++aa)
        mbar_drain(&ctl->aux_full[aa % kAuxSlots], (uint32_t)((aa / kAuxSlots) & 1));
    }
  } else if (warp == kMmaWarp || warp == kMmaWarp2) {
    // ------------------------------------------------------------ MMA issuers
    if (lane == 0) {
      const int mine = warp - kMmaWarp;  // the accumulator (item-tile parity) this thread serves
      // The two issuers split the item tiles by parity only where that also
      // splits the ring stages: with S a multiple of 2 bs, tile g's loads
      // take stages bs g .. bs g + bs - 1 (mod S), even tiles and odd tiles
      // never share a stage, and the one issuer of a stage waits for every
      // phase of its barriers in turn (a parity wait cannot tell phase k
      // from phase k + 2, so a thread that skipped phases could take a
      // stale one for the one it waits for).  Otherwise warp 9 issues every
      // tile and warp 10 only keeps its part of the work-item and user-tile
      // protocol.
      const bool split = p.stages % (2 * bs) == 0;
      bool ok_init = true;
      // instruction descriptor: D = F32, A = B = BF16 (kind::f16 format 1) or
      // E4M3 (kind::f8f6f4 format 0), both K-major, N, M
      const bool f8 = p.esize == 1;
      const uint32_t ab_fmt = f8 ? 0u : ((1u << 7) | (1u << 10));
      const uint32_t idesc = (1u << 4) | ab_fmt | ((uint32_t)(sub_rows >> 3) << 17) | ((uint32_t)(kTileM >> 4) << 24);
      const uint32_t sbo = 8 * p.row_bytes;
      const int ksteps = p.row_bytes / 32;  // 32 bytes per MMA: K = 16 BF16 or K = 32 E4M3
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
      // the descriptors of every K step, once (B relative to ring stage 0)
      const int nfull = p.kc * ksteps, nst = nfull + tsteps;
      uint64_t a_d[kMaxSteps], b_d[kMaxSteps];
#pragma unroll
      for (int i = 0; i < kMaxSteps; ++i) {
        const int c = i / ksteps, k = i - c * ksteps, tk = i - nfull;
        a_d[i] = i < nfull ? a_desc0 + (uint64_t)(c * a16 + 2 * k) : a_tdesc + (uint64_t)(2 * tk);
        b_d[i] = i < nfull ? b_desc0 + (uint64_t)(c * b16 + 2 * k) : b_tdesc0 + (uint64_t)(2 * tk);
      }
      if (nst < 1 || nst > kMaxSteps) {  // (tc_plan never makes such rows)
        atomicOr(err, DEV_ERR_INTERNAL);
        ok_init = false;
      }
      // the issue loop, once per operand type (no type branch per load)
      auto issue_loop = [&](auto f8_tag) {
        constexpr bool F8 = decltype(f8_tag)::value;
        long long g = 0;
        int st = 0;
        uint32_t ph = 0;   // ring pass parity
        int b = 0;         // accumulator of tile g
        uint32_t aph = 0;  // accumulator pass parity
        bool ok = ok_init;
        for (int lt = 0; ok; ++lt) {
          const int slot = lt % kWQ;
          ok = mbar_wait(&ctl->wq_full[slot], (uint32_t)((lt / kWQ) & 1), gd);
          if (!ok) break;
          const int wi = *(volatile int*)&ctl->wq[slot];
          mbar_arrive(&ctl->wq_empty[slot]);
          if (wi >= n_work) break;
          const WorkItem wk = get_work<MX>(p, wi, n_it);
          const int asl = lt & 1;  // user-tile slot of this work item
          ok = mbar_wait(&ctl->a_full[asl], (uint32_t)((lt >> 1) & 1), gd);
          const uint64_t aoff = (uint64_t)(asl * (a_bytes >> 4));
          if (!ok) break;
          tc_fence_after();
          for (int j = wk.tb; j < wk.te; ++j, ++g) {  // g: item tiles so far
            if (split ? b != mine : mine != 0) {  // another issuer's tile: step over its ring stages
              for (int h = 0; h < bs; ++h)
                if (++st == p.stages) {
                  st = 0;
                  ph ^= 1u;
                }
              b ^= 1;
              if (b == 0) aph ^= 1u;
              continue;
            }
            for (int h = 0; h < bs && ok; ++h) {
              // (spinning waits: an issuer's wait is on the tensor pipe's
              // critical path, and the thread has nothing else to do)
              ok = mbar_spin(&ctl->b_full[st], ph, gd);
              if (ok && h == 0 && g >= 2) ok = mbar_spin(&ctl->acc_empty[b], aph ^ 1u, gd);
              if (!ok) break;
              tc_fence_after();
              // this load's rows go to accumulator columns [h sub_rows, (h + 1) sub_rows)
              const uint32_t d = tmem + (uint32_t)(b * kTileN) + (uint32_t)h * sub_rows;
              const uint64_t boff = (uint64_t)(st * stage16);
              switch (nst) {
                case 1: mma_steps<1, F8>(d, a_d, b_d, aoff, boff, idesc); break;
                case 2: mma_steps<2, F8>(d, a_d, b_d, aoff, boff, idesc); break;
                case 3: mma_steps<3, F8>(d, a_d, b_d, aoff, boff, idesc); break;
                case 4: mma_steps<4, F8>(d, a_d, b_d, aoff, boff, idesc); break;
                case 5: mma_steps<5, F8>(d, a_d, b_d, aoff, boff, idesc); break;
                case 6: mma_steps<6, F8>(d, a_d, b_d, aoff, boff, idesc); break;
                case 7: mma_steps<7, F8>(d, a_d, b_d, aoff, boff, idesc); break;
                case 8: mma_steps<8, F8>(d, a_d, b_d, aoff, boff, idesc); break;
                case 9: mma_steps<9, F8>(d, a_d, b_d, aoff, boff, idesc); break;
                default: mma_steps<10, F8>(d, a_d, b_d, aoff, boff, idesc); break;
              }
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
          if (ok) mma_commit(&ctl->a_empty[asl]);
        }
      };
      if (f8) issue_loop(std::true_type{});
      else issue_loop(std::false_type{});
      // all MMAs issued by this thread complete before TMEM is released
      mma_commit(&ctl->drain);
      mbar_drain(&ctl->drain, 0);
    }
  } else {
    // ------------------------------------------------------------ select
    const int e = warp;
    const int q = e % 4, c2 = e / 4;       // lane quarter, column half
    const int row = 32 * q + lane;         // user row within the tile
    const int slot = c2 * kTileM + row;    // this thread's index among the 256
    TcUser<KR> s;
    TcSel c;
    c.heap = heap_base + slot;
    c.K = p.K;
    c.cap = o.cap;
    c.n_items = MX ? p.work.n_items_pos : p.n_items;
    c.err = err;
    c.qbase = qh_base;
    c.slot = slot;
    c.pslot = (c2 ^ 1) * kTileM + row;
    c.g = p.g;
    c.f8 = p.esize == 1;
    const float item_scale = c.f8 ? *p.item_scale : 0.f;
    long long g = 0;  // item tiles processed: the accumulator and aux-ring sequence
    bool ok = true;
    unsigned long long emitted = 0, slow = 0;
    for (int lt = 0; ok; ++lt) {  // work items of this CTA
      const int wslot = lt % kWQ;
      ok = __all_sync(kFull, mbar_wait(&ctl->wq_full[wslot], (uint32_t)((lt / kWQ) & 1), gd));
      const int wi = ok ? *(volatile int*)&ctl->wq[wslot] : n_work;
      __syncwarp();
      if (lane == 0) mbar_arrive(&ctl->wq_empty[wslot]);
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
      s.au = 1.f;
      s.am = c.f8 ? 4.76837158203125e-07f : 0.f;  // 2^-21
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
        if (c.f8) s.au = __fmul_rn(p.user_scale[u], item_scale);
        if (restoring) {  // continue a walk: restore the select state
          s.n_cand = o.n_cand[list];
          const float* src = o.topl + list * (int64_t)p.K;
          if constexpr (KR > 0) {
#pragma unroll
            for (int i = 0; i < KR; ++i) s.d[i] = i < p.K ? src[i] : kNegInf;
            s.tau = topk_kth(s, p.K);
          } else {  // the row is descending: reversed, it is a min-heap
            for (int i = 0; i < p.K; ++i) c.heap[i * kEpiThreads] = src[p.K - 1 - i];
            s.tau = c.heap[0];
          }
          s.tau_eff = fmaxf(s.tau, o.tau[list]);
          tc_publish(s, c);
        }
      }
      // a fresh work item merges the two halves' first-tile lists once both exist
      bool merged = restoring || KR == 0;
      const int par = lt & 1;
      for (int j = wk.tb; j < wk.te; ++j, ++g) {
        const int b = (int)(g & 1);
        const int as = (int)(g % kAuxSlots);
        const uint32_t aph = (uint32_t)((g / kAuxSlots) & 1);
        const float2* aux = aux_ring + (size_t)as * kTileN + c2 * kHalfN;
        const int32_t* pos = pos_ring + (size_t)as * kTileN + c2 * kHalfN;
        // the tile's bound columns first (their copy runs up to kAuxSlots
        // tiles ahead, so this wait is over long before the accumulator's),
        // read or not: the slot is released only once its copy has landed,
        // or the copier's parity waits could run a phase ahead
        ok = __all_sync(kFull, mbar_wait(&ctl->aux_full[as], aph, gd));
        if (!ok) break;
        // lanes leave together: TMEM loads are warp-collective
        ok = __all_sync(kFull, mbar_wait(&ctl->acc_full[b], (uint32_t)((g >> 1) & 1), gd));
        if (!ok) break;
        tc_fence_after();
        {  // the partner's threshold, if it is for this work item
          const unsigned long long pt = *c.tau(c.pslot);
          if ((int)(pt >> 32) == wi) s.tau_eff = fmaxf(s.tau_eff, __uint_as_float((uint32_t)pt));
          // and the one shared by the user's other item chunks (zero bits: none yet, NaN, ignored)
          if constexpr (MX)
            if (c.tau_glob) s.tau_eff = fmaxf(s.tau_eff, tau_from_ord(*(volatile unsigned*)c.tau_glob));
        }
        const uint32_t taddr = tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(b * kTileN + c2 * kHalfN);
        const int32_t rank0 = j * kTileN + c2 * kHalfN;  // (list) rank of this thread's first column
        const int valid = (int)min((int64_t)kHalfN, p.n_items - rank0);
        const bool first = j == wk.tb && !restoring;  // a fresh work item's first tile
        if (__builtin_expect(first, 0)) {  // (rare paths marked so the common case stays compact)
          seed_tile(s, c, taddr, valid, aux, active);
          if (active) {
            s.tau_eff = fmaxf(s.tau_eff, s.tau);
            tc_publish(s, c);
          }
          seed_publish(s, c, wi, par);
        }
        if (!merged) merged = seed_try_merge(s, c, wi, par, active);
        // common case: the maxima of the two 64-column halves and two votes
        // (one load site in a rolled loop: two unrolled 64-register loads
        // make the compiler keep both destination sets apart)
        unsigned halves = 0;
#pragma unroll 1
        for (int h = 0; h < 2; ++h) {
          const float m = hv(s, c, tmem_ldmax64(taddr + 64 * h));
          halves |= __any_sync(kFull, m >= s.tau_eff) ? (1u << h) : 0u;
        }
        if (__builtin_expect(halves != 0u, 0)) {
          slow += __popc(halves);
          if (first) emit_tile<KR, MX>(s, c, taddr, valid, rank0, pos, halves);
          else select_hits<KR, MX>(s, c, taddr, valid, aux, rank0, pos, halves);
        }
        tc_fence_before();
        __syncwarp();
        if (lane == 0) {
          mbar_arrive(&ctl->acc_empty[b]);
          mbar_arrive(&ctl->aux_empty[as]);
        }
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
    for (int off = 16; off > 0; off >>= 1) emitted += __shfl_xor_sync(kFull, emitted, off);
    if (lane == 0 && emitted) atomicAdd(&stats->cand_emitted, emitted);
    if (lane == 0 && slow) atomicAdd(&stats->select_slow, slow);  // warp x 64-column halves with a hit
  }

  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == kProdWarp) {
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
  return 1024 + 2 * a_bytes + (size_t)p.stages * b_bytes + heap +
         (sizeof(float2) + sizeof(int32_t)) * kAuxSlots * kTileN + sizeof(float) * kQueue * kEpiThreads +
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
