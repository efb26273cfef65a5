// Device helpers shared by the fused score+select kernels and the rescore.
//
// Per-user select state (the on-chip replacement for the per-user min-heap
// of the paper's BMM, Sec. II-C): each user is owned by one thread, which
// keeps
//   * tau   -- the K-th largest LOWER bound on u^T i seen so far (register);
//   * a min-heap of those K lower bounds in shared memory (column layout:
//     heap[k * stride + lane] so threads never collide on a bank when they
//     touch the same heap level);
//   * a count of candidates emitted to its global candidate list.
// A scored item whose UPPER bound H satisfies H >= tau is emitted as a
// candidate (item position + H).  Items with H < tau can never be in the
// top-K: tau is a lower bound on the K-th best score, and H an upper bound on
// this item's score.  The exact ranking of the surviving candidates is done
// by the rescore kernel.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

#include "internal.h"

namespace mips {

#define kNegInf (-__int_as_float(0x7f800000))

// ---------------------------------------------------------------------------
// Min-heap of K floats held in shared memory, column `lane` of a
// [K][stride] array.  Slot 0 is the minimum.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void heap_init(float* heap, int stride, int K) {
  for (int k = 0; k < K; ++k) heap[k * stride] = kNegInf;
}

// Replace the minimum by v (caller guarantees v > heap[0]) and restore the
// heap order.  Returns the new minimum.
__device__ __forceinline__ float heap_replace_min(float* heap, int stride, int K, float v) {
  int pos = 0;
  while (true) {
    int l = 2 * pos + 1;
    if (l >= K) break;
    int r = l + 1;
    float lv = heap[l * stride];
    int c = l;
    float cv = lv;
    if (r < K) {
      float rv = heap[r * stride];
      if (rv < lv) {
        c = r;
        cv = rv;
      }
    }
    if (cv >= v) break;
    heap[pos * stride] = cv;
    pos = c;
  }
  heap[pos * stride] = v;
  return heap[0];
}

// One scored item for a user on the slow path: update tau with its lower
// bound, then emit it if its upper bound still reaches tau.
struct UserSelect {
  float tau;
  int n_cand;
  float* heap;  // &heap_base[lane]
  int stride;
  int K;
  int cap;
  int32_t* cand_pos;  // this user's candidate list
  float* cand_ub;

  __device__ __forceinline__ void offer(float H, float L, int32_t item_pos) {
    if (L > tau) tau = heap_replace_min(heap, stride, K, L);
    if (H >= tau) {
      if (n_cand < cap) {
        cand_pos[n_cand] = item_pos;
        cand_ub[n_cand] = H;
      }
      ++n_cand;
    }
  }
};

// ---------------------------------------------------------------------------
// Compensated dot product in FP32 (Ogita, Rump, Oishi, "Accurate sum and
// dot product", SIAM J. Sci. Comput. 26(6), 2005, Algorithm Dot2), keeping
// the unevaluated pair (hi, lo).  The products are split exactly with FMA
// (TwoProduct) and the running sum with Knuth's TwoSum; the returned double
// hi + lo differs from the exact u^T i by at most gamma_f^2 * sum|u_k i_k|
// (gamma_f = f u / (1 - f u), u = 2^-24) plus one double rounding.
// ---------------------------------------------------------------------------
struct Dot2 {
  float hi, lo;
};

__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

__device__ __forceinline__ void dot2_step(Dot2& acc, float a, float b) {
  float p = __fmul_rn(a, b);
  float pe = __fmaf_rn(a, b, -p);  // exact: a*b = p + pe
  float s, se;
  two_sum(acc.hi, p, s, se);
  acc.hi = s;
  acc.lo = __fadd_rn(acc.lo, __fadd_rn(pe, se));
}

__device__ __forceinline__ double dot2_value(const Dot2& a) { return (double)a.hi + (double)a.lo; }

// Sequential FP64 sum over k = 0..f-1 of the exact products: the same
// arithmetic, in the same order, as the definition of a score.
__device__ __forceinline__ double dot_f64_seq(const float* u, const float* v, int f) {
  double s = 0.0;
  for (int k = 0; k < f; ++k) s = __dadd_rn(s, __dmul_rn((double)u[k], (double)v[k]));
  return s;
}

// ---------------------------------------------------------------------------
// Norm bounds that hold at any magnitude.  A plain FP32 sum of squares loses
// every term below 2^-149 and most bits of those below 2^-126, so the norm of
// a row of tiny entries can come out 0.  The row is therefore scaled by an
// exact power of two 2^k that puts its largest |entry| in [1/2, 1) (then the
// largest square is at least 1/4 and the sum's relative error bound holds),
// and the bound is scaled back by 2^-k rounding upward.
// ---------------------------------------------------------------------------
// 2^e for e in [-126, 127] (exact).
__device__ __forceinline__ float exp2i(int e) { return __int_as_float((127 + e) << 23); }

// k with amax 2^k in [1/2, 1), for finite amax > 0 (k in [-128, 149]).
__device__ __forceinline__ int norm_scale_exp(float amax) {
  int ex;
  frexpf(amax, &ex);
  return -ex;
}

// x 2^k for k in [-128, 149]: exact unless the result falls below 2^-126
// (then the absolute error is below 2^-149).
__device__ __forceinline__ float scale_pow2(float x, int k) {
  const int k1 = k / 2;
  return (x * exp2i(k1)) * exp2i(k - k1);
}

// y 2^-k rounded upward (an upper bound stays an upper bound).
__device__ __forceinline__ float unscale_pow2_ru(float y, int k) {
  const int k1 = -k / 2;
  return __fmul_ru(__fmul_ru(y, exp2i(k1)), exp2i(-k - k1));
}

// Squared norms below this are treated as unreliable (subnormal terms) by
// the bound kernels, which then fall back to no pruning.
#define kTinySq 7.8886090522101181e-31f  // 2^-100

// Upper bound on |computed - exact| for the FP32 fused score with f terms,
// relative to ||u|| ||i||: recursive FMA summation error gamma_f (Higham,
// "Accuracy and Stability of Numerical Algorithms", 2nd ed., Sec. 3.1) with
// margin, plus the rounding of the bound arithmetic itself and the FP64
// definition's own rounding (f 2^-53).
__host__ __device__ inline float fp32_score_gamma(int f) { return (float)(f + 4) * 5.9604645e-08f * 2.0f; }

}  // namespace mips
