// Exact rescore of the surviving candidates and final top-K (the last step
// of the paper's BMM and of QueryIndex in Algorithm 1: the K best items by
// u^T i, ties to the smaller item index).
//
// Three kernels, then one for overflowed users:
//   (A) collect, thread per user: the threshold tau -- the final threshold
//       of its candidate sub-list, or, with two sub-lists whose K best lower
//       bounds are given, the K-th largest of their union (the entries
//       belong to distinct items, so this is a valid lower bound on the
//       user's K-th score) -- and the slots of the candidates whose upper
//       bound H reaches tau, appended to a work list (each user's run in
//       one piece, its first entry and length noted per user);
//   (B) dot, thread per work entry: its compensated FP32 dot product
//       (Dot2, common.cuh), so every lane of a warp has work, stored in
//       work order with the item's id and norm bound (the two gathers by
//       item position happen here, where they overlap across lanes);
//   (C) select, thread per user: the K + 1 best keys (score desc, item id
//       asc) of its work run in a shared-memory heap, sorted;
//   * tie check: every adjacent pair of that list is compared against the
//     score error bound
//       e = (2 gamma_2f gamma_f + (f + 2) 2^-53) nhat_u nhat_i_max  (x 2 margin),
//     which covers this computation and the FP64 definition's own rounding.
//     A gap <= 2e (equal values included) redoes the user with the FP64
//     definition's arithmetic (sequential sum of exact products), whose
//     ranking is the definition's; otherwise the compensated order equals
//     the exact order, which equals the FP64 definition's order;
//   * a zero user has every score exactly 0: its answer is items 0..K-1;
//   * a user whose candidate list overflowed is queued for the warp kernel,
//     one warp per queued user, scoring every item;
//   * so is a non-zero user with ||u||^2 < 2^-100 in FP32 (its squares or
//     products may be subnormal, where the relative bounds above fail): the
//     warp kernel scores it with the FP64 definition's arithmetic only;
//   * the tie-check margin also carries an absolute f 2^-148 for subnormal
//     products of normal-range users (each loses at most 2^-150 in TwoProduct).
#include "common.cuh"

namespace mips {

namespace {

constexpr int kWarpsPerBlock = 4;
constexpr int kMaxK = 128;
constexpr int kMaxF = 128;
constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ bool ranks_before(double sa, int ia, double sb, int ib) {
  return sa > sb || (sa == sb && ia < ib);
}

// Order-preserving 64-bit integer key of a finite double (a larger value has
// a larger key, and both zeros the key of +0, so equal values keep equal
// keys): the select's heap ranks with integer compares, as GB300's FP64
// rate is a small fraction of its integer rate.
__device__ __forceinline__ unsigned long long dkey(double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  if ((b << 1) == 0ull) b = 0ull;  // -0 -> +0
  return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double dkey_value(unsigned long long k) {
  const unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
  return __longlong_as_double((long long)b);
}
__device__ __forceinline__ bool key_before(unsigned long long ka, int ia, unsigned long long kb, int ib) {
  return ka > kb || (ka == kb && ia < ib);
}

// Relative score error bound used by the tie check (see the file comment).
// K-th largest value of the union of m rows of K values, each row sorted
// descending (m <= kMaxLists): K rounds of taking the largest row head.
constexpr int kMaxLists = 64;
__device__ __forceinline__ float union_kth(const float* __restrict__ rows, int m, int K) {
  int head[kMaxLists];
  for (int l = 0; l < m; ++l) head[l] = 0;
  float v = __int_as_float(0xff800000);
  for (int r = 0; r < K; ++r) {
    int best = -1;
    float bv = __int_as_float(0xff800000);
    for (int l = 0; l < m; ++l)
      if (head[l] < K && (best < 0 || rows[l * K + head[l]] > bv)) {
        best = l;
        bv = rows[l * K + head[l]];
      }
    v = bv;
    ++head[best];
  }
  return v;
}

// The same for two rows (a user's two sub-lists), in registers.
__device__ __forceinline__ float union2_kth(const float* __restrict__ rows, int K) {
  const float* a = rows;
  const float* b = rows + K;
  int ia = 0, ib = 0;
  float v = __int_as_float(0xff800000);
  for (int r = 0; r < K; ++r) {
    const float x = ia < K ? a[ia] : __int_as_float(0xff800000);
    const float y = ib < K ? b[ib] : __int_as_float(0xff800000);
    if (x >= y) {
      v = x;
      ++ia;
    } else {
      v = y;
      ++ib;
    }
  }
  return v;
}

// Users with ||u||^2 below this (FP32) are scored in FP64 only.
constexpr float kTinyNorm2 = 7.8886090522101181e-31f;  // 2^-100

// Absolute part of the tie-check margin: subnormal products.
__device__ __forceinline__ double rescore_abs_err(int f) { return (double)f * 2.8025969286496341e-45; }  // f 2^-148

__device__ __forceinline__ bool row_all_zero(const float* __restrict__ r, int f) {
  for (int k = 0; k < f; ++k)
    if (r[k] != 0.f) return false;
  return true;
}

__device__ __forceinline__ double rescore_rel_err(int f) {
  const double gf = (double)f * 5.9604644775390625e-08;  // f 2^-24
  const double gamma_f = gf / (1.0 - gf);
  const double gamma_2f = 2.0 * gamma_f / (1.0 - gamma_f);
  return 2.0 * (2.0 * gamma_2f * gamma_f + (double)(f + 2) * 1.1102230246251565e-16);
}

// Row loads: two elements at a time when both rows start on 8 bytes and f is
// even (half the load instructions), else one.  The arithmetic runs over
// k = 0, 1, ... either way.
__device__ __forceinline__ bool pairs_ok(const float* a, const float* b, int f) {
  return ((reinterpret_cast<uintptr_t>(a) | reinterpret_cast<uintptr_t>(b)) & 7) == 0 && (f & 1) == 0;
}

__device__ __forceinline__ float norm2_seq(const float* __restrict__ r, int f) {
  float ss = 0.f;
  if (pairs_ok(r, r, f)) {
    const float2* r2 = reinterpret_cast<const float2*>(r);
    for (int k = 0; k < f / 2; ++k) {
      const float2 x = r2[k];
      ss = __fmaf_rn(x.x, x.x, ss);
      ss = __fmaf_rn(x.y, x.y, ss);
    }
    return ss;
  }
  for (int k = 0; k < f; ++k) ss = __fmaf_rn(r[k], r[k], ss);
  return ss;
}

__device__ __forceinline__ double score_dot2(const float* __restrict__ u, const float* __restrict__ v, int f) {
  Dot2 acc{0.f, 0.f};
  int k = 0;
  if (pairs_ok(u, v, f)) {
    const float2* u2 = reinterpret_cast<const float2*>(u);
    const float2* v2 = reinterpret_cast<const float2*>(v);
    for (; k + 8 <= f; k += 8) {  // the loads of 8 terms before their arithmetic
      float2 a[4], b[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        a[j] = u2[k / 2 + j];
        b[j] = v2[k / 2 + j];
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        dot2_step(acc, a[j].x, b[j].x);
        dot2_step(acc, a[j].y, b[j].y);
      }
    }
    for (; k < f; k += 2) {
      const float2 a = u2[k / 2], b = v2[k / 2];
      dot2_step(acc, a.x, b.x);
      dot2_step(acc, a.y, b.y);
    }
    return dot2_value(acc);
  }
  for (; k + 8 <= f; k += 8) {  // issue the loads of 8 terms before their arithmetic
    float a[8], b[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      a[j] = u[k + j];
      b[j] = v[k + j];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) dot2_step(acc, a[j], b[j]);
  }
  for (; k < f; ++k) dot2_step(acc, u[k], v[k]);
  return dot2_value(acc);
}

// The same compensated dot with the item row v read 16 bytes at a time: the
// elements before v's first 16-byte boundary one by one, then eight at a
// time from two float4 loads, then the rest; the user row element by element
// (a thread's neighbours score other items of the same users, so its lines
// are shared).  Same terms in the same order k = 0, 1, ... as score_dot2.
__device__ __forceinline__ double score_dot2_v4(const float* __restrict__ u, const float* __restrict__ v, int f) {
  Dot2 acc{0.f, 0.f};
  int k = 0;
  const int peel = (int)(((16u - ((unsigned)reinterpret_cast<uintptr_t>(v) & 15u)) & 15u) >> 2);
  for (; k < peel && k < f; ++k) dot2_step(acc, u[k], v[k]);
  for (; k + 8 <= f; k += 8) {
    const float4 b0 = *reinterpret_cast<const float4*>(v + k);
    const float4 b1 = *reinterpret_cast<const float4*>(v + k + 4);
    float a[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = u[k + j];
    dot2_step(acc, a[0], b0.x);
    dot2_step(acc, a[1], b0.y);
    dot2_step(acc, a[2], b0.z);
    dot2_step(acc, a[3], b0.w);
    dot2_step(acc, a[4], b1.x);
    dot2_step(acc, a[5], b1.y);
    dot2_step(acc, a[6], b1.z);
    dot2_step(acc, a[7], b1.w);
  }
  for (; k < f; ++k) dot2_step(acc, u[k], v[k]);
  return dot2_value(acc);
}

// Sequential FP64 sum of the exact products (the definition's arithmetic),
// with the loads of 8 terms issued before their arithmetic.
__device__ __forceinline__ double score_f64(const float* __restrict__ u, const float* __restrict__ v, int f) {
  double s = 0.0;
  int k = 0;
  for (; k + 8 <= f; k += 8) {
    float a[8], b[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      a[j] = u[k + j];
      b[j] = v[k + j];
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) s = __dadd_rn(s, __dmul_rn((double)a[j], (double)b[j]));
  }
  for (; k < f; ++k) s = __dadd_rn(s, __dmul_rn((double)u[k], (double)v[k]));
  return s;
}

// Binary heap of at most L keys (score, id) in a thread's shared-memory
// column (entry p at [p * T + t]); the root is the key that ranks last, so a
// new key that ranks before the root replaces it.
struct KeyHeap {
  unsigned long long* s;  // dkey of the score
  int* id;
  int T;
  __device__ __forceinline__ unsigned long long sv(int p) const { return s[p * T]; }
  __device__ __forceinline__ int iv(int p) const { return id[p * T]; }
  __device__ __forceinline__ void put(int p, unsigned long long v, int i) {
    s[p * T] = v;
    id[p * T] = i;
  }
  // key_before(a, b): a ranks before b
  __device__ __forceinline__ void sift_down(int p, int n, unsigned long long v, int i) {
    while (true) {
      int c = 2 * p + 1;
      if (c >= n) break;
      if (c + 1 < n && key_before(sv(c), iv(c), sv(c + 1), iv(c + 1))) ++c;  // the worse child
      if (!key_before(v, i, sv(c), iv(c))) break;  // v is already worse than both children
      put(p, sv(c), iv(c));
      p = c;
    }
    put(p, v, i);
  }
  __device__ __forceinline__ void push(int& n, int L, double score, int i) {
    const unsigned long long v = dkey(score);
    if (n < L) {
      int p = n++;
      while (p > 0) {
        const int q = (p - 1) / 2;
        if (!key_before(sv(q), iv(q), v, i)) break;  // parent already worse
        put(p, sv(q), iv(q));
        p = q;
      }
      put(p, v, i);
    } else if (key_before(v, i, sv(0), iv(0))) {
      sift_down(0, n, v, i);
    }
  }
  // In place: entries 0..n-1 best first.
  __device__ __forceinline__ void sort(int n) {
    for (int m = n - 1; m > 0; --m) {
      const unsigned long long v = sv(m);
      const int i = iv(m);
      put(m, sv(0), iv(0));  // the worst of 0..m goes to m
      sift_down(0, m, v, i);
    }
  }
};

// ---------------------------------------------------------------------------
// (A) thread per user: threshold, overflow / zero-user handling, and the
//     valid candidate slots appended to the work list
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256)
    rescore_collect_kernel(const float* __restrict__ users, int64_t n_users, int f, int K, SelectOut o,
                           int32_t* __restrict__ out_idx, double* __restrict__ out_score, DevStats* stats) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31;
  int nvalid = 0;
  float tau = 0.f;
  bool live = false;  // this user goes through the work list
  unsigned long long n_over = 0;
  if (u < n_users) {
    const float* ur = users + u * f;
    const float ss = norm2_seq(ur, f);
    o.tau_final[2 * u + 1] = ss;  // (for the select kernel)
    const int64_t l0 = u * o.lists;
    bool over = false;
    for (int l = 0; l < o.lists; ++l) over |= o.n_cand[l0 + l] > o.cap;
    if (ss == 0.f && row_all_zero(ur, f)) {  // zero user: every score is exactly 0
      for (int k = 0; k < K; ++k) {
        out_idx[u * K + k] = k;
        out_score[u * K + k] = 0.0;
      }
    } else if (over || ss < kTinyNorm2) {
      const int slot = atomicAdd(o.ovf_count, 1);
      o.ovf_list[slot] = (int32_t)u;
      n_over = 1;
    } else {
      // every sub-list's threshold is a valid one; with the sub-lists' K
      // largest lower bounds (distinct items, each row descending) the K-th
      // largest of their union is too, and the tightest
      for (int l = 0; l < o.lists; ++l) tau = l == 0 ? o.tau[l0] : fmaxf(tau, o.tau[l0 + l]);
      if (o.lists > 1 && o.topl && o.topl_sorted)
        tau = fmaxf(tau, o.lists == 2 ? union2_kth(o.topl + l0 * K, K) : union_kth(o.topl + l0 * K, o.lists, K));
      live = true;
      for (int l = 0; l < o.lists; ++l) {
        const float* cu = o.cand_ub + (l0 + l) * (int64_t)o.cap;
        const int nl = o.n_cand[l0 + l];
        for (int c = 0; c < nl; ++c) nvalid += cu[c] >= tau;
      }
    }
  }
  // warp-aggregated append: one atomic per warp
  int incl = nvalid;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int y = __shfl_up_sync(kFull, incl, off);
    if (lane >= off) incl += y;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  int base = 0;
  if (lane == 31 && total) base = atomicAdd(o.work_count, total);
  base = __shfl_sync(kFull, base, 31) + incl - nvalid;
  if (u < n_users) {  // the user's run in the work list (read by the select for live users)
    o.u_work[2 * u] = base;
    o.u_work[2 * u + 1] = live ? nvalid : 0;
  }
  if (live && nvalid) {
    const int64_t l0 = u * o.lists;
    for (int l = 0; l < o.lists; ++l) {
      const int64_t row = (l0 + l) * (int64_t)o.cap;
      const float* cu = o.cand_ub + row;
      const int nl = o.n_cand[l0 + l];
      for (int c = 0; c < nl; ++c)
        if (cu[c] >= tau) o.work[base++] = (uint32_t)(row + c);
    }
  }
  unsigned long long r = nvalid;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    r += __shfl_xor_sync(kFull, r, off);
    n_over += __shfl_xor_sync(kFull, n_over, off);
  }
  if (lane == 0) {
    if (r) atomicAdd(&stats->cand_rescored, r);
    if (n_over) atomicAdd(&stats->users_overflow, n_over);
  }
}

// ---------------------------------------------------------------------------
// (B) thread per valid candidate: its compensated dot product
// ---------------------------------------------------------------------------
// (a position outside [0, n_items) is never written by the score kernels;
// if one is read -- a score kernel that gave up on a bounded wait leaves its
// lists unfinished -- it is flagged, and its entry gets id -1, which the
// select skips, rather than being dereferenced)
__global__ void __launch_bounds__(256)
    rescore_dot_kernel(const float* __restrict__ users, int f, const float* __restrict__ items,
                       const int32_t* __restrict__ perm, const float* __restrict__ item_nrm, int64_t n_items,
                       SelectOut o, int* err) {
  const int count = *o.work_count;
  for (int w = blockIdx.x * blockDim.x + threadIdx.x; w < count; w += gridDim.x * blockDim.x) {
    const uint32_t slot = o.work[w];
    const int64_t u = (int64_t)(slot / (uint32_t)o.cap) / o.lists;
    const int32_t pos = o.cand_pos[slot];
    if (pos < 0 || pos >= n_items) {
      atomicOr(err, DEV_ERR_INTERNAL);
      o.cand_sc[w] = 0.0;
      o.w_id[w] = -1;
      o.w_nrm[w] = 0.f;
      continue;
    }
    const int32_t id = perm[pos];
    const float nrm = item_nrm[pos];
    const float* ur = users + u * f;
    const float* ir = items + (int64_t)pos * f;
    o.cand_sc[w] = pairs_ok(ur, ir, f) ? score_dot2(ur, ir, f) : score_dot2_v4(ur, ir, f);
    o.w_id[w] = id;
    o.w_nrm[w] = nrm;
  }
}

// ---------------------------------------------------------------------------
// (C) thread per user: the K + 1 best keys, the tie check, the output
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128)
    rescore_select_kernel(const float* __restrict__ users, int64_t n_users, int f,
                          const float* __restrict__ items, int K, SelectOut o,
                          int32_t* __restrict__ out_idx,
                          double* __restrict__ out_score, DevStats* stats, int* err) {
  extern __shared__ unsigned char smem_raw[];
  const int T = blockDim.x, t = threadIdx.x;
  const int L = K + 1;  // the K best and the best of the rest
  unsigned long long* ls = reinterpret_cast<unsigned long long*>(smem_raw);  // [L][T] score keys
  int* li = reinterpret_cast<int*>(ls + (size_t)L * T);
  const int64_t u = (int64_t)blockIdx.x * T + t;
  unsigned long long n_fp64 = 0;
  if (u < n_users) {
    const float* ur = users + u * f;
    const int64_t l0 = u * o.lists;
    bool over = false;
    for (int l = 0; l < o.lists; ++l) over |= o.n_cand[l0 + l] > o.cap;
    const float ss = o.tau_final[2 * u + 1];  // ||u||^2 as the collect kernel computed it
    // zero users are done; overflowed and tiny users belong to the warp kernel
    if (ss >= kTinyNorm2 && !over) {
      const double nu = (double)__fsqrt_rn(ss) * (1.0 + (double)(f + 2) * 1.1920929e-07);
      const double rel_e = rescore_rel_err(f);
      // the candidates that reach the threshold: the user's run of the work list
      const int w0 = o.u_work[2 * u], nw = o.u_work[2 * u + 1];
      KeyHeap heap{ls + t, li + t, T};
      for (int mode = 0; mode < 2; ++mode) {
        int cnt = 0;
        float nmax = 0.f;
        for (int w = w0; w < w0 + nw; ++w) {
          const int32_t id = o.w_id[w];
          if (id < 0) continue;  // a bad position, flagged by the dot kernel
          const double v =
              mode == 0 ? o.cand_sc[w] : score_f64(ur, items + (int64_t)o.cand_pos[o.work[w]] * f, f);
          nmax = fmaxf(nmax, o.w_nrm[w]);
          heap.push(cnt, L, v, id);
        }
        heap.sort(cnt);
        if (cnt < K) {  // cannot happen: K lower bounds back tau
          atomicOr(err, DEV_ERR_INTERNAL);
          break;
        }
        if (mode == 1) break;
        const double e2 = 2.0 * rel_e * nu * (double)nmax + rescore_abs_err(f);
        bool amb = false;
        for (int p = 0; p + 1 < cnt; ++p) amb |= (dkey_value(ls[p * T + t]) - dkey_value(ls[(p + 1) * T + t])) <= e2;
        if (!amb) break;
        ++n_fp64;
      }
      for (int k = 0; k < K; ++k) {
        out_idx[u * K + k] = li[k * T + t];
        out_score[u * K + k] = dkey_value(ls[k * T + t]);
      }
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) n_fp64 += __shfl_xor_sync(kFull, n_fp64, off);
  if ((t & 31) == 0 && n_fp64) atomicAdd(&stats->users_fp64, n_fp64);
}

// ---------------------------------------------------------------------------
// warp per user, every item (users whose candidate list overflowed)
// ---------------------------------------------------------------------------
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

__global__ void __launch_bounds__(kWarpsPerBlock * 32)
    rescore_warp_kernel(const float* __restrict__ users, int f, const float* __restrict__ items,
                        const int32_t* __restrict__ perm, const float* __restrict__ item_nrm, int64_t n_items, int K,
                        const int32_t* __restrict__ list, const int* __restrict__ list_count,
                        int32_t* __restrict__ out_idx, double* __restrict__ out_score, DevStats* stats, int* err) {
  __shared__ double s_s[kWarpsPerBlock][kMaxK];
  __shared__ int s_id[kWarpsPerBlock][kMaxK];
  __shared__ float s_u[kWarpsPerBlock][kMaxF];
  const int w = threadIdx.x / 32, lane = threadIdx.x & 31;
  const double rel_e = rescore_rel_err(f);
  unsigned long long n_fp64 = 0;
  const int count = *list_count;

  for (int q = blockIdx.x * kWarpsPerBlock + w; q < count; q += gridDim.x * kWarpsPerBlock) {
    const int64_t u = list[q];
    float ss = 0.f;
    for (int k = lane; k < f; k += 32) {
      float v = users[u * f + k];
      s_u[w][k] = v;
      ss = __fmaf_rn(v, v, ss);
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) ss += __shfl_xor_sync(kFull, ss, off);
    __syncwarp();
    const double nu = (double)__fsqrt_rn(ss) * (1.0 + (double)(f + 2) * 1.1920929e-07);
    for (int mode = ss < kTinyNorm2 ? 1 : 0; mode < 2; ++mode) {
      WarpList Lw{s_s[w], s_id[w], 0, false, 0.0, 0};
      float nmax = 0.f;
      for (int64_t base = 0; base < n_items; base += 32) {
        const int64_t t = base + lane;
        const bool valid = t < n_items;
        double v = 0.0;
        int id = 0;
        if (valid) {
          id = perm[t];
          const float* row = items + t * f;
          nmax = fmaxf(nmax, item_nrm[t]);
          v = mode == 0 ? score_dot2(s_u[w], row, f) : dot_f64_seq(s_u[w], row, f);
        }
        unsigned mask = __ballot_sync(kFull, valid);
        while (mask) {
          const int src = __ffs(mask) - 1;
          mask &= mask - 1;
          const double vs = __shfl_sync(kFull, v, src);
          const int is = __shfl_sync(kFull, id, src);
          if (Lw.has_out && !ranks_before(vs, is, Lw.out_s, Lw.out_id)) continue;
          Lw.insert(vs, is, K, lane);
        }
      }
      if (Lw.cnt < K) {
        if (lane == 0) atomicOr(err, DEV_ERR_INTERNAL);
        break;
      }
      if (mode == 1) break;
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) nmax = fmaxf(nmax, __shfl_xor_sync(kFull, nmax, off));
      const double e2 = 2.0 * rel_e * nu * (double)nmax + rescore_abs_err(f);
      bool amb = false;
      for (int p0 = 0; p0 < Lw.cnt; p0 += 32) {
        const int p = p0 + lane;
        bool a = false;
        if (p + 1 < Lw.cnt) a = (Lw.s[p] - Lw.s[p + 1]) <= e2;
        if (p == Lw.cnt - 1 && Lw.has_out && Lw.cnt == K) a = (Lw.s[p] - Lw.out_s) <= e2;
        amb |= __any_sync(kFull, a) != 0;
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
  if (lane == 0 && n_fp64) atomicAdd(&stats->users_fp64, n_fp64);
}

}  // namespace

cudaError_t launch_rescore(const float* users, int64_t n_users, int f, const float* items_sorted,
                           const int32_t* perm, const float* item_nrm_ub, int64_t n_items, int K,
                           SelectOut o, int32_t* out_idx, double* out_score, DevStats* stats,
                           int* err, cudaStream_t s) {
  if (K > kMaxK || f > kMaxF) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(o.ovf_count, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(o.work_count, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  rescore_collect_kernel<<<(unsigned)((n_users + 255) / 256), 256, 0, s>>>(users, n_users, f, K, o, out_idx,
                                                                            out_score, stats);
  rescore_dot_kernel<<<sm_count() * 8, 256, 0, s>>>(users, f, items_sorted, perm, item_nrm_ub, n_items, o, err);
  // threads per block so that the per-thread lists of K + 1 keys fit in 96 KiB
  int T = 128;
  while (T > 32 && (size_t)T * (K + 1) * 12 > 96 * 1024) T -= 32;
  const size_t smem = (size_t)T * (K + 1) * 12;
  e = cudaFuncSetAttribute(rescore_select_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  rescore_select_kernel<<<(unsigned)((n_users + T - 1) / T), T, smem, s>>>(users, n_users, f, items_sorted, K, o,
                                                                           out_idx, out_score, stats, err);
  rescore_warp_kernel<<<sm_count() * 2, kWarpsPerBlock * 32, 0, s>>>(users, f, items_sorted, perm, item_nrm_ub, n_items, K,
                                                             o.ovf_list, o.ovf_count, out_idx, out_score, stats,
                                                             err);
  return cudaGetLastError();
}

}  // namespace mips
