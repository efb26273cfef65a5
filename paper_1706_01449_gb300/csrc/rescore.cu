// Exact rescore of the surviving candidates and final top-K (the last step
// of the paper's BMM and of QueryIndex in Algorithm 1: the K best items by
// u^T i, ties to the smaller item index).
//
// One warp per user.  Candidates whose upper bound H reaches the user's
// final threshold tau are scored with a compensated FP32 dot product (Dot2,
// see common.cuh) and inserted into a warp-shared list sorted by
// (score desc, item id asc); the best rejected key is tracked too.  Then
// every adjacent pair of the list (and the K-th entry against the best
// rejected one) is checked against the score error bound
//   e = (2 gamma_2f gamma_f + (f + 2) 2^-53) nhat_u nhat_i_max   (x 2 margin)
// which covers both this computation and the FP64 definition's own
// rounding.  Any gap <= 2e (equal values included) makes the user
// ambiguous, and the user is redone with the FP64 definition's arithmetic
// itself (sequential sum of exact products), whose ranking is the
// definition's.  Otherwise the compensated order equals the exact order,
// which equals the FP64 definition's order.
//
// A user whose candidate list overflowed is rescored against every item.
// A zero user has every score exactly 0: its answer is items 0..K-1.
#include "common.cuh"

namespace mips {

namespace {

constexpr int kWarps = 4;
constexpr int kMaxK = 128;
constexpr int kMaxF = 128;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool ranks_before(double sa, int ia, double sb, int ib) {
  return sa > sb || (sa == sb && ia < ib);
}

struct WarpList {
  double* s;  // [kMaxK]
  int* id;    // [kMaxK]
  int cnt;
  bool has_out;
  double out_s;
  int out_id;

  __device__ __forceinline__ void reject(double v, int i) {
    if (!has_out || ranks_before(v, i, out_s, out_id)) {
      has_out = true;
      out_s = v;
      out_id = i;
    }
  }

  // Warp-uniform insert of key (v, i) into the list of at most K entries.
  __device__ void insert(double v, int i, int K, int lane) {
    int pos = 0;
    for (int k0 = 0; k0 < cnt; k0 += 32) {
      int k = k0 + lane;
      bool b = k < cnt && ranks_before(s[k], id[k], v, i);
      pos += __popc(__ballot_sync(kFull, b));
    }
    if (pos >= K) {
      reject(v, i);
      return;
    }
    if (cnt == K) reject(s[K - 1], id[K - 1]);
    const int last = min(cnt, K - 1);  // entries pos..last-1 move up by one
    for (int c0 = ((last - 1 - pos) / 32) * 32 + pos; c0 >= pos && last > pos; c0 -= 32) {
      int k = c0 + lane;
      double sv = 0.0;
      int iv = 0;
      bool mv = k < last;
      if (mv) {
        sv = s[k];
        iv = id[k];
      }
      __syncwarp();
      if (mv) {
        s[k + 1] = sv;
        id[k + 1] = iv;
      }
      __syncwarp();
    }
    if (lane == 0) {
      s[pos] = v;
      id[pos] = i;
    }
    __syncwarp();
    cnt = min(cnt + 1, K);
  }
};

__global__ void __launch_bounds__(kWarps * 32)
    rescore_kernel(const float* __restrict__ users, int64_t n_users, int f,
                   const float* __restrict__ items, const int32_t* __restrict__ perm,
                   const float* __restrict__ item_nrm, int64_t n_items, int K, SelectOut o,
                   int32_t* __restrict__ out_idx, double* __restrict__ out_score, DevStats* stats,
                   int* err) {
  __shared__ double s_s[kWarps][kMaxK];
  __shared__ int s_id[kWarps][kMaxK];
  __shared__ float s_u[kWarps][kMaxF];
  const int w = threadIdx.x / 32, lane = threadIdx.x & 31;
  const float gf = (float)f * 5.9604645e-08f;
  const double gamma_f = (double)gf / (1.0 - (double)gf);
  const double gamma_2f = 2.0 * gamma_f / (1.0 - gamma_f);
  const double rel_e = 2.0 * (2.0 * gamma_2f * gamma_f + (double)(f + 2) * 1.1102230246251565e-16);
  unsigned long long n_rescored = 0, n_over = 0, n_fp64 = 0;

  for (int64_t u = (int64_t)blockIdx.x * kWarps + w; u < n_users; u += (int64_t)gridDim.x * kWarps) {
    float ss = 0.f;
    for (int k = lane; k < f; k += 32) {
      float v = users[u * f + k];
      s_u[w][k] = v;
      ss = __fmaf_rn(v, v, ss);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(kFull, ss, off);
    __syncwarp();
    if (ss == 0.f) {  // zero user: every score is exactly 0
      for (int k = lane; k < K; k += 32) {
        out_idx[u * K + k] = k;
        out_score[u * K + k] = 0.0;
      }
      continue;
    }
    const double nu = (double)__fsqrt_rn(ss) * (1.0 + (double)(f + 2) * 1.1920929e-07);
    const int n = o.n_cand[u];
    const float tau = o.tau[u];
    const bool overflow = n > o.cap;
    const int64_t nn = overflow ? n_items : (int64_t)n;
    n_over += overflow;
    const int32_t* cpos = o.cand_pos + u * (int64_t)o.cap;
    const float* cub = o.cand_ub + u * (int64_t)o.cap;

    for (int mode = 0; mode < 2; ++mode) {
      WarpList L{s_s[w], s_id[w], 0, false, 0.0, 0};
      float nmax = 0.f;
      for (int64_t base = 0; base < nn; base += 32) {
        const int64_t t = base + lane;
        bool valid = t < nn;
        int32_t pos = 0;
        if (valid) {
          if (overflow) {
            pos = (int32_t)t;
          } else {
            pos = cpos[t];
            valid = cub[t] >= tau;
          }
        }
        double v = 0.0;
        int id = 0;
        if (valid) {
          id = perm[pos];
          const float* row = items + (int64_t)pos * f;
          nmax = fmaxf(nmax, item_nrm[pos]);
          if (mode == 0) {
            Dot2 acc{0.f, 0.f};
            for (int k = 0; k < f; ++k) dot2_step(acc, s_u[w][k], row[k]);
            v = dot2_value(acc);
          } else {
            v = dot_f64_seq(s_u[w], row, f);
          }
        }
        if (mode == 0 && !overflow) n_rescored += valid;
        unsigned mask = __ballot_sync(kFull, valid);
        while (mask) {
          const int src = __ffs(mask) - 1;
          mask &= mask - 1;
          const double vs = __shfl_sync(kFull, v, src);
          const int is = __shfl_sync(kFull, id, src);
          if (L.has_out && !ranks_before(vs, is, L.out_s, L.out_id)) continue;
          L.insert(vs, is, K, lane);
        }
      }
      if (mode == 1) break;
      // tie check on the compensated scores
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) nmax = fmaxf(nmax, __shfl_xor_sync(kFull, nmax, off));
      const double e2 = 2.0 * rel_e * nu * (double)nmax;
      bool amb = false;
      for (int p0 = 0; p0 < L.cnt; p0 += 32) {
        const int p = p0 + lane;
        bool a = false;
        if (p + 1 < L.cnt) a = (L.s[p] - L.s[p + 1]) <= e2;
        if (p == L.cnt - 1 && L.has_out && L.cnt == K) a = (L.s[p] - L.out_s) <= e2;
        amb |= __any_sync(kFull, a) != 0;
      }
      if (L.cnt < K) {  // cannot happen: K lower bounds back tau
        if (lane == 0) atomicOr(err, DEV_ERR_INTERNAL);
        break;
      }
      if (!amb) break;
      ++n_fp64;
      __syncwarp();
    }
    for (int k = lane; k < K; k += 32) {
      out_idx[u * K + k] = s_id[w][k];
      out_score[u * K + k] = s_s[w][k];
    }
    __syncwarp();
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) n_rescored += __shfl_xor_sync(kFull, n_rescored, off);
  if (lane == 0) {
    if (n_rescored) atomicAdd(&stats->cand_rescored, n_rescored);
    if (n_over) atomicAdd(&stats->users_overflow, n_over);
    if (n_fp64) atomicAdd(&stats->users_fp64, n_fp64);
  }
}

}  // namespace

cudaError_t launch_rescore(const float* users, int64_t n_users, int f, const float* items_sorted,
                           const int32_t* perm, const float* item_nrm_ub, int64_t n_items, int K,
                           SelectOut o, int32_t* out_idx, double* out_score, DevStats* stats,
                           int* err, cudaStream_t s) {
  if (K > kMaxK || f > kMaxF) return cudaErrorInvalidValue;
  int64_t blocks = (n_users + kWarps - 1) / kWarps;
  if (blocks > 152 * 32) blocks = 152 * 32;
  rescore_kernel<<<(unsigned)blocks, kWarps * 32, 0, s>>>(users, n_users, f, items_sorted, perm, item_nrm_ub,
                                                          n_items, K, o, out_idx, out_score, stats, err);
  return cudaGetLastError();
}

}  // namespace mips
