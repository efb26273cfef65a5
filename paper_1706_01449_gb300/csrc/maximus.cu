// Maximus (Sec. III, Algorithm 1) on the GPU: k-means user clusters,
// theta_b per cluster, CBound (Eq. appx_bound) for every (cluster, item),
// per-cluster item lists sorted by CBound, users grouped by cluster, and a
// grouped walk of each cluster's list that stops once no remaining item can
// enter any of the walking users' top-K.  The walk emits candidates into the
// same per-user lists as the blocked multiply, so the exact rescore is
// shared.
//
// Rounding: every quantity that decides pruning is rounded outward so that
// the exactness argument (Lemma "upper bound in index lists" and Theorem
// "exact") holds for the computed values:
//   * cos_b[j] = a LOWER bound of min over members of cos(u, c_j);
//   * x = an UPPER bound of cos(c_j, i);
//   * CBound = nhat_i g(x, cos_b) with g(x, y) = 1 if x >= y, else
//     x y + sqrt((1 - x)(1 + x)) sqrt((1 - y)(1 + y))   (= cos(theta_ic - theta_b)),
//     g rounded up; g increases with x and decreases with y on x < y, so
//     the outward inputs give an upper bound.
#include <algorithm>
#include <cmath>
#include <cstring>

#include "common.cuh"

namespace mips {

namespace {

constexpr int kThreads = 128;   // users per walk / assign block
constexpr int kBlockItems = 32; // items per walk shared-memory tile (a "block" of Algorithm 1's walk)

__device__ __forceinline__ void cp_async4(float* smem_dst, const float* gmem_src) {
  unsigned d = (unsigned)__cvta_generic_to_shared(smem_dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(gmem_src));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::); }

// float <-> order-preserving unsigned (ascending)
__device__ __forceinline__ uint32_t f2ord(float x) {
  const uint32_t b = __float_as_uint(x);
  return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float ord2f(uint32_t o) {
  return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// ---------------------------------------------------------------- k-means
__global__ void gather_rows_i64(const float* __restrict__ x, const int64_t* __restrict__ ids, int n, int f,
                                float* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * f) return;
  const int r = (int)(t / f), k = (int)(t % f);
  out[t] = x[ids[r] * f + k];
}

// max |x| over all entries, as an order-preserving unsigned
__global__ void absmax_kernel(const float* __restrict__ x, int64_t n, uint32_t* out) {
  float m = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(x[i]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, __float_as_uint(m));  // non-negative: bits are ordered
}

// ||c_j||^2 / 2 per centroid
__global__ void half_norm2_kernel(const float* __restrict__ cent, int C, int f, float* __restrict__ hn2) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= C) return;
  float s = 0.f;
  for (int k = 0; k < f; ++k) s = __fmaf_rn(cent[j * f + k], cent[j * f + k], s);
  hn2[j] = 0.5f * s;
}

// Assignment step: argmin_j ||u - c_j||^2 = argmax_j (u . c_j - ||c_j||^2 / 2);
// ties to the smaller j.  Centroids are staged through shared memory in
// tiles of 64.
template <int FP>
__global__ void __launch_bounds__(kThreads) kmeans_assign_kernel(const float* __restrict__ users, int64_t n_users,
                                                                 int f, const float* __restrict__ cent,
                                                                 const float* __restrict__ hn2, int C,
                                                                 int32_t* __restrict__ assign) {
  __shared__ float cs[64 * FP];
  __shared__ float hs[64];
  const int64_t u = (int64_t)blockIdx.x * kThreads + threadIdx.x;
  const bool active = u < n_users;
  float ur[FP];
#pragma unroll
  for (int k = 0; k < FP; ++k) ur[k] = (active && k < f) ? users[u * f + k] : 0.f;
  float best = -__int_as_float(0x7f800000);
  int bj = 0;
  for (int j0 = 0; j0 < C; j0 += 64) {
    const int nj = min(64, C - j0);
    __syncthreads();
    for (int e = threadIdx.x; e < 64 * FP; e += kThreads) {
      const int r = e / FP, k = e % FP;
      cs[e] = (r < nj && k < f) ? cent[(int64_t)(j0 + r) * f + k] : 0.f;
    }
    for (int e = threadIdx.x; e < 64; e += kThreads) hs[e] = e < nj ? hn2[j0 + e] : 0.f;
    __syncthreads();
    for (int r = 0; r < nj; ++r) {
      float d = 0.f;
#pragma unroll
      for (int k = 0; k < FP; ++k) d = __fmaf_rn(ur[k], cs[r * FP + k], d);
      const float v = d - hs[r];
      if (v > best) {
        best = v;
        bj = j0 + r;
      }
    }
  }
  if (active) assign[u] = bj;
}

// Fixed-point scale 2^e for the centroid sums: n_users entries of
// magnitude <= max|x| sum to less than 2^62.  scale[0] = 2^e, scale[1] = 2^-e.
__global__ void kmeans_scale_kernel(const uint32_t* __restrict__ absmax_bits, int64_t n_users, float* scale) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  float amax = __uint_as_float(*absmax_bits);
  if (!(amax > 0.f)) amax = 1.f;
  const double mag = (double)amax * (double)n_users;
  int ex = 61 - (int)ceil(log2(mag));
  if (ex > 100) ex = 100;
  scale[0] = ldexpf(1.f, ex);
  scale[1] = ldexpf(1.f, -ex);
}

// Update step, part 1: per-cluster sums in fixed point (int64, scale 2^e),
// so that the result does not depend on the order of the atomic adds.
__global__ void kmeans_accum_kernel(const float* __restrict__ users, int64_t n_users, int f,
                                    const int32_t* __restrict__ assign, int C, const float* __restrict__ scale,
                                    unsigned long long* __restrict__ sums, unsigned int* __restrict__ counts) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_users * f) return;
  const int64_t u = t / f;
  const int k = (int)(t - u * f);
  const int j = assign[u];
  const long long q = __float2ll_rn(users[t] * scale[0]);
  atomicAdd(&sums[(int64_t)j * f + k], (unsigned long long)q);
  if (k == 0) atomicAdd(&counts[j], 1u);
}

// The same sums for the clusters [j0, j0 + cc) of this block's chunk
// (blockIdx.y), partial sums of a grid-stride share of the users kept in
// shared memory, then one global add per (cluster, dimension) and block.
// Integer sums: the same result as kmeans_accum_kernel in any order.
__global__ void kmeans_accum_smem_kernel(const float* __restrict__ users, int64_t n_users, int f,
                                         const int32_t* __restrict__ assign, int C, int cc,
                                         const float* __restrict__ scale, unsigned long long* __restrict__ sums,
                                         unsigned int* __restrict__ counts) {
  extern __shared__ unsigned long long km_acc[];        // [cc][f]
  unsigned int* km_cnt = (unsigned int*)(km_acc + (size_t)cc * f);  // [cc]
  const int j0 = blockIdx.y * cc;
  const int nc = min(cc, C - j0);
  for (int e = threadIdx.x; e < nc * f; e += blockDim.x) km_acc[e] = 0ull;
  for (int e = threadIdx.x; e < nc; e += blockDim.x) km_cnt[e] = 0u;
  __syncthreads();
  const float sc = scale[0];
  const int64_t total = n_users * f;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t u = t / f;
    const int k = (int)(t - u * f);
    const int j = assign[u] - j0;
    if (j >= 0 && j < nc) {
      atomicAdd(&km_acc[j * f + k], (unsigned long long)__float2ll_rn(users[t] * sc));
      if (k == 0) atomicAdd(&km_cnt[j], 1u);
    }
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nc * f; e += blockDim.x)
    if (km_acc[e]) atomicAdd(&sums[(int64_t)j0 * f + e], km_acc[e]);
  for (int e = threadIdx.x; e < nc; e += blockDim.x)
    if (km_cnt[e]) atomicAdd(&counts[j0 + e], km_cnt[e]);
}

// The same sums with partial sums private to a group of G = ceil(f / 32)
// warps: group c of the block owns rows [C][f] (and counts [C]) of shared
// memory, and its warp g adds dimensions 32 g + lane of each of the group's
// users to its cluster's row with plain adds (one lane per address, users in
// order; the G warps of a group touch disjoint dimensions, so they need no
// atomics); then the block sums its groups' copies and adds each (cluster,
// dimension) to the global sums once.  One copy per G warps instead of one
// per warp: the copies are what limits the warps an SM holds.
// Integer sums: the same result as kmeans_accum_kernel in any order.
__global__ void kmeans_accum_warp_kernel(const float* __restrict__ users, int64_t n_users, int f,
                                         const int32_t* __restrict__ assign, int C, const float* __restrict__ scale,
                                         unsigned long long* __restrict__ sums, unsigned int* __restrict__ counts,
                                         int G) {
  extern __shared__ unsigned long long kw_acc[];  // [groups][C][f]
  const int ngb = (blockDim.x / 32) / G;          // groups per block
  const int64_t cf = (int64_t)C * f;
  unsigned int* kw_cnt = (unsigned int*)(kw_acc + ngb * cf);  // [groups][C]
  for (int64_t e = threadIdx.x; e < ngb * cf; e += blockDim.x) kw_acc[e] = 0ull;
  for (int e = threadIdx.x; e < ngb * C; e += blockDim.x) kw_cnt[e] = 0u;
  __syncthreads();
  const int w = threadIdx.x / 32, lane = threadIdx.x & 31;
  const int grp = w / G, gk = w - grp * G;
  const int k = 32 * gk + lane;  // this lane's dimension
  unsigned long long* acc = kw_acc + grp * cf;
  unsigned int* cnt = kw_cnt + grp * C;
  const float sc = scale[0];
  // each group takes 8 consecutive users at a time: their cluster ids and
  // row values are loaded before any add, so the loads overlap
  constexpr int kU = 8;
  const int64_t step = (int64_t)gridDim.x * ngb * kU;
  if (grp < ngb) {
    for (int64_t u0 = ((int64_t)blockIdx.x * ngb + grp) * kU; u0 < n_users; u0 += step) {
      int j[kU];
#pragma unroll
      for (int r = 0; r < kU; ++r) j[r] = u0 + r < n_users ? assign[u0 + r] : -1;
      if (k < f) {
        float x[kU];
#pragma unroll
        for (int r = 0; r < kU; ++r) x[r] = j[r] >= 0 ? users[(u0 + r) * f + k] : 0.f;
#pragma unroll
        for (int r = 0; r < kU; ++r)
          if (j[r] >= 0) acc[(int64_t)j[r] * f + k] += (unsigned long long)__float2ll_rn(x[r] * sc);
      }
      if (gk == 0 && lane == 0) {
#pragma unroll
        for (int r = 0; r < kU; ++r)
          if (j[r] >= 0) cnt[j[r]] += 1u;
      }
    }
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < cf; e += blockDim.x) {
    unsigned long long t = 0ull;
    for (int gg = 0; gg < ngb; ++gg) t += kw_acc[gg * cf + e];
    if (t) atomicAdd(&sums[e], t);
  }
  for (int e = threadIdx.x; e < C; e += blockDim.x) {
    unsigned int t = 0u;
    for (int gg = 0; gg < ngb; ++gg) t += kw_cnt[gg * C + e];
    if (t) atomicAdd(&counts[e], t);
  }
}

// Update step, part 2: mean of the members; an empty cluster keeps its centroid.
__global__ void kmeans_update_kernel(const unsigned long long* __restrict__ sums, const unsigned int* __restrict__ counts,
                                    int C, int f, const float* __restrict__ scale, float* __restrict__ cent) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= C * f) return;
  const int j = t / f;
  const unsigned int n = counts[j];
  if (n == 0) return;
  const double s = (double)(long long)sums[t];
  cent[t] = (float)(s * (double)scale[1] / (double)n);
}

// Spherical k-means (Sec. III-A: the clustering that minimises the user-
// centroid angles; the paper itself runs plain k-means as the faster one):
// centroids scaled to unit length after the draw and after every update, so
// the assignment step picks the largest cosine (||c_j||^2 / 2 is the same for
// every centroid).  A zero centroid stays zero.
__global__ void normalize_rows_kernel(float* __restrict__ cent, int C, int f) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= C) return;
  float* c = cent + (int64_t)j * f;
  float s = 0.f;
  for (int k = 0; k < f; ++k) s = __fmaf_rn(c[k], c[k], s);
  if (!(s > 0.f)) return;
  const float n = __fsqrt_rn(s);
  for (int k = 0; k < f; ++k) c[k] = __fdiv_rn(c[k], n);
}

// ---------------------------------------------------------------- bounds
// cos_b[j] (as order-preserving bits, initialised to +1): a lower bound of
// the smallest cosine between a member of cluster j and c_j.  Zero users are
// left out, and so are users whose FP32 ||u||^2 is below 2^-100, where
// subnormal squares make the computed cosine unreliable (the rescore scores
// those users exhaustively whatever the walk did); a centroid that small
// gives -1 (theta_b = pi).
//
// Eight lanes per user, four users per warp at a time: lane l of a group
// sums elements l, l + 8, ... with FMA and three shuffle steps add the
// group's partial sums (any summation order keeps each factor's relative
// error below the (f + 2) 2^-24 the margin allows).  The rescore decides
// "below 2^-100" from its own sequential sum, which can differ from this
// one in the last bits; a user is left out here only below 2^-100 (1 -
// 2^-8), so every user the rescore trusts is counted (one counted in
// addition only lowers the minimum).  Each block keeps its members' minima
// per cluster in shared memory (C <= kCosbShared) and sends one atomicMin
// per cluster it met.
constexpr int kCosbShared = 1024;

__global__ void __launch_bounds__(256)
    cosb_kernel(const float* __restrict__ users, int64_t n_users, int f, const int32_t* __restrict__ assign,
                const float* __restrict__ cent, int C, uint32_t* __restrict__ cosb_ord) {
  __shared__ uint32_t smin[kCosbShared];
  const bool in_smem = C <= kCosbShared;
  if (in_smem)
    for (int j = threadIdx.x; j < C; j += blockDim.x) smin[j] = 0xffffffffu;  // (above every cosine's bits)
  __syncthreads();
  const int lane = threadIdx.x & 31, sub = lane & 7;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t n_warps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t u4 = warp * 4; u4 < n_users; u4 += n_warps * 4) {  // (warp-uniform: the shuffles need every lane)
    const int64_t u = u4 + (lane >> 3);
    const bool valid = u < n_users;
    const int j = valid ? assign[u] : 0;
    const float* ur = users + (valid ? u : 0) * f;
    const float* cr = cent + (int64_t)j * f;
    float d = 0.f, su = 0.f, sc = 0.f;
    if (valid)
      for (int k = sub; k < f; k += 8) {
        const float x = ur[k], y = cr[k];
        d = __fmaf_rn(x, y, d);
        su = __fmaf_rn(x, x, su);
        sc = __fmaf_rn(y, y, sc);
      }
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) {
      d += __shfl_xor_sync(0xffffffffu, d, o);
      su += __shfl_xor_sync(0xffffffffu, su, o);
      sc += __shfl_xor_sync(0xffffffffu, sc, o);
    }
    if (!valid || sub != 0 || su < kTinySq * 0.99609375f) continue;
    float c;
    if (sc < kTinySq) {
      c = -1.f;
    } else {
      // each factor carries a relative error below (f + 2) 2^-24; |cos| <= 1
      c = __fdiv_rn(d, __fsqrt_rn(su) * __fsqrt_rn(sc)) - (float)(2 * f + 8) * 5.9604645e-08f * 2.f;
      c = fmaxf(c, -1.f);
    }
    if (in_smem) atomicMin(&smin[j], f2ord(c));
    else atomicMin(cosb_ord + j, f2ord(c));
  }
  if (in_smem) {
    __syncthreads();
    for (int j = threadIdx.x; j < C; j += blockDim.x)
      if (smin[j] != 0xffffffffu) atomicMin(cosb_ord + j, smin[j]);
  }
}

// CBound of every (cluster, item): key = float_desc_key(bound) (sorts
// descending), value = item position.  [C][n_items], cluster-major.
// One block: 128 items (one per thread, staged in shared memory as
// [f][129] to keep the banks apart) against a chunk of 32 centroids
// ([f][32], read eight at a time); every dot product, item norm and
// centroid norm is summed sequentially over k with FMA.
constexpr int kCbItems = 128, kCbChunk = 32;
static_assert(kCbChunk % 16 == 0, "the CBound kernel takes sixteen centroids at a time");

__host__ __device__ __forceinline__ size_t cb_items_floats(int f) {  // rounded to 4 floats (float4 reads after it)
  return ((size_t)f * (kCbItems + 1) + 3) & ~(size_t)3;
}

// ni: the item's norm bound from row_norm_ub_kernel (power-of-two scaled
// sums, valid at any magnitude; 0 only for the zero item).  rsc = sqrt(sc),
// rsi = sqrt(si) and sy = sqrt((1 - y)(1 + y)) depend only on the centroid
// or only on the item, so the caller computes them once (the same roundings
// as computing them here).
__device__ __forceinline__ float cbound_value(float d, float sc, float si, float ni, float y, int f, float rsc,
                                              float rsi, float sy) {
  float g;
  if (ni == 0.f) {
    g = 0.f;  // zero item: bound 0 = its score
  } else if (sc < kTinySq || si < kTinySq || y <= -1.f) {
    g = 1.f;  // theta_b = pi, or a cosine FP32 cannot evaluate reliably: no pruning
  } else {
    float x = __fdiv_rn(d, rsc * rsi) + (float)(2 * f + 8) * 5.9604645e-08f * 2.f;
    x = fminf(x, 1.f);
    if (x >= y) {
      g = 1.f;
    } else {
      const float sx = __fsqrt_rn((1.f - x) * (1.f + x));
      g = fminf(1.f, __fmaf_rn(x, y, sx * sy) + 9.5367432e-07f);  // + 2^-20
    }
  }
  // bound = ||i|| g: ni is an upper bound of ||i||, and ||i|| >= ni (1 - (2f + 4) 2^-23)
  return g >= 0.f ? ni * g * (1.f + 2.3841858e-07f)
                  : ni * (1.f - (float)(2 * f + 4) * 1.1920929e-07f) * g * (1.f - 2.3841858e-07f);
}

__global__ void __launch_bounds__(kCbItems)
    cbound_kernel(const float* __restrict__ cent, int C, int f, const float* __restrict__ items,
                  const float* __restrict__ item_nrm, int64_t n_items, const uint32_t* __restrict__ cosb_ord,
                  uint32_t* __restrict__ keys, int32_t* __restrict__ vals) {
  extern __shared__ __align__(16) float cb_smem[];
  float* it = cb_smem;                                  // [f][kCbItems + 1]
  float* ct = it + cb_items_floats(f);                  // [f][kCbChunk], 16-byte aligned
  float* cn2 = ct + (size_t)f * kCbChunk;               // [kCbChunk] ||c||^2
  float* crs = cn2 + kCbChunk;                          // [kCbChunk] sqrt(||c||^2)
  float* cy = crs + kCbChunk;                           // [kCbChunk] cos_b of the centroid's cluster
  float* csy = cy + kCbChunk;                           // [kCbChunk] sqrt((1 - y)(1 + y))
  const int t = threadIdx.x;
  const int64_t i0 = (int64_t)blockIdx.x * kCbItems;
  const int j0 = blockIdx.y * kCbChunk;
  const int rows = (int)min((int64_t)kCbItems, n_items - i0);
  const int nc = min(kCbChunk, C - j0);
  for (int e = t; e < kCbItems * f; e += kCbItems) {
    const int r = e / f, k = e - r * f;
    it[k * (kCbItems + 1) + r] = r < rows ? items[(i0 + r) * f + k] : 0.f;
  }
  for (int e = t; e < kCbChunk * f; e += kCbItems) {
    const int jj = e / f, k = e - jj * f;
    ct[k * kCbChunk + jj] = jj < nc ? cent[(int64_t)(j0 + jj) * f + k] : 0.f;
  }
  __syncthreads();
  if (t < kCbChunk) {
    float sc = 0.f;
    for (int k = 0; k < f; ++k) sc = __fmaf_rn(ct[k * kCbChunk + t], ct[k * kCbChunk + t], sc);
    cn2[t] = sc;
    crs[t] = __fsqrt_rn(sc);
    const float y = t < nc ? ord2f(cosb_ord[j0 + t]) : 1.f;
    cy[t] = y;
    csy[t] = __fsqrt_rn((1.f - y) * (1.f + y));
  }
  float si = 0.f;
  for (int k = 0; k < f; ++k) si = __fmaf_rn(it[k * (kCbItems + 1) + t], it[k * (kCbItems + 1) + t], si);
  const float rsi = __fsqrt_rn(si);
  __syncthreads();
  if (t >= rows) return;
  const int64_t i = i0 + t;
  const float ni = item_nrm[i];
  for (int jj = 0; jj < nc; jj += 16) {  // sixteen centroids at a time: sixteen independent sums
    float d[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) d[q] = 0.f;
    for (int k = 0; k < f; ++k) {
      const float v = it[k * (kCbItems + 1) + t];
#pragma unroll
      for (int h = 0; h < 4; ++h) {
        const float4 c4 = *reinterpret_cast<const float4*>(ct + k * kCbChunk + jj + 4 * h);
        d[4 * h + 0] = __fmaf_rn(c4.x, v, d[4 * h + 0]);
        d[4 * h + 1] = __fmaf_rn(c4.y, v, d[4 * h + 1]);
        d[4 * h + 2] = __fmaf_rn(c4.z, v, d[4 * h + 2]);
        d[4 * h + 3] = __fmaf_rn(c4.w, v, d[4 * h + 3]);
      }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) {
      if (jj + q < nc) {
        const int j = j0 + jj + q;
        const int64_t o = (int64_t)j * n_items + i;
        keys[o] = float_desc_key(
            cbound_value(d[q], cn2[jj + q], si, ni, cy[jj + q], f, crs[jj + q], rsi, csy[jj + q]));
        vals[o] = (int32_t)i;
      }
    }
  }
}

__global__ void cosb_init_kernel(uint32_t* __restrict__ cosb_ord, int C) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < C) cosb_ord[j] = f2ord(1.f);
}

__global__ void cosb_to_float_kernel(const uint32_t* __restrict__ cosb_ord, int C, float* __restrict__ out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < C) out[j] = ord2f(cosb_ord[j]);
}

// sorted key -> bound of the list rank.  The lists are sorted by the key's
// top 16 bits only (kListKeyBits), so each rank gets the largest bound its
// 16-bit bucket can hold: the key with the low bits cleared (keys ascend
// as bounds descend).  The result is non-increasing along the list and at
// least the bound of every item at that rank or later.
__global__ void keys_to_bounds_kernel(const uint32_t* __restrict__ keys, int64_t n, float* __restrict__ out) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  constexpr uint32_t mask = ~((1u << (32 - kListKeyBits)) - 1u);
  out[t] = ord2f(~(keys[t] & mask));
}

// ---------------------------------------------------------------- grouping
__global__ void iota_u32_kernel(const int32_t* __restrict__ assign, int64_t n, uint32_t* __restrict__ keys,
                                int32_t* __restrict__ ids) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  keys[t] = (uint32_t)assign[t];
  ids[t] = (int32_t)t;
}

// counts[j] += members of cluster j: a shared-memory histogram per block
// when C fits (use_smem), else global atomics.
__global__ void cluster_count_kernel(const int32_t* __restrict__ assign, int64_t n, int C, int use_smem,
                                     int* __restrict__ counts) {
  extern __shared__ int cc_hist[];
  if (use_smem) {
    for (int j = threadIdx.x; j < C; j += blockDim.x) cc_hist[j] = 0;
    __syncthreads();
  }
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(use_smem ? &cc_hist[assign[t]] : &counts[assign[t]], 1);
  if (use_smem) {
    __syncthreads();
    for (int j = threadIdx.x; j < C; j += blockDim.x)
      if (cc_hist[j]) atomicAdd(&counts[j], cc_hist[j]);
  }
}

// offsets[j] = users before cluster j; tile_off[j] = walk tiles before j
// (128 users per tile); tile_off[C] = total tiles.  One block.
__global__ void cluster_offsets_kernel(const int* __restrict__ counts, int C, int* __restrict__ offsets,
                                       int* __restrict__ tile_off) {
  if (threadIdx.x != 0) return;
  int o = 0, t = 0;
  for (int j = 0; j < C; ++j) {
    offsets[j] = o;
    tile_off[j] = t;
    o += counts[j];
    t += (counts[j] + kThreads - 1) / kThreads;
  }
  offsets[C] = o;
  tile_off[C] = t;
}

// ---------------------------------------------------------------- walk
// One block per work item (cluster j, tile of its users), taken from a
// global counter (persistent grid).  Each thread owns one user: its FP32
// vector in registers, the select state of common.cuh.  The cluster's
// sorted list is walked in shared-memory tiles of 32 items (rows gathered
// by position with cp.async); before each tile every thread checks the stop
// test of Algorithm 1 with the tile's leading bound (the largest bound of
// everything not yet visited, the list being sorted):
//     max(nhat_u * bound, 0)  <  tau_u   (strictly)
// (the clamp: a negative CBound times norm upper bounds is no upper bound
// on a negative score), and the block stops when it holds for all of its
// users.
template <int FP>
__global__ void __launch_bounds__(kThreads, 2)
    maximus_walk_kernel(const float* __restrict__ users, int f, const float* __restrict__ items,
                        const float* __restrict__ item_nrm, int64_t n_items, const int32_t* __restrict__ lists,
                        const float* __restrict__ bounds, const int32_t* __restrict__ user_perm,
                        const int* __restrict__ offsets, const int* __restrict__ tile_off, int C, int K,
                        SelectOut o, int32_t* __restrict__ visited, int* __restrict__ work_counter,
                        DevStats* stats, int* err) {
  extern __shared__ float4 smem4[];
  float* tiles = reinterpret_cast<float*>(smem4);     // [2][32][FP]
  float* nrms = tiles + 2 * kBlockItems * FP;          // [2][32]
  int32_t* poss = reinterpret_cast<int32_t*>(nrms + 2 * kBlockItems);  // [2][32]
  float* heap_base = reinterpret_cast<float*>(poss + 2 * kBlockItems); // [K][128]
  __shared__ int s_work;
  const int tid = threadIdx.x;
  const int total = tile_off[C];
  unsigned long long pairs = 0, blocks = 0;

  for (int e = tid; e < 2 * kBlockItems * FP; e += kThreads) tiles[e] = 0.f;

  while (true) {
    __syncthreads();
    if (tid == 0) s_work = atomicAdd(work_counter, 1);
    __syncthreads();
    const int w = s_work;
    if (w >= total) break;
    // cluster of work item w: the last j with tile_off[j] <= w
    int lo = 0, hi = C - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (tile_off[mid] <= w) lo = mid;
      else hi = mid - 1;
    }
    const int j = lo;
    const int r0 = offsets[j] + (w - tile_off[j]) * kThreads;
    const int r = r0 + tid;
    const bool active = r < offsets[j + 1];
    const int64_t u = active ? user_perm[r] : 0;
    float ur[FP];
    float ss = 0.f;
#pragma unroll
    for (int k = 0; k < FP; ++k) {
      ur[k] = (active && k < f) ? users[u * f + k] : 0.f;
      ss = __fmaf_rn(ur[k], ur[k], ss);
    }
    const float nu = __fsqrt_rn(ss) * (1.0f + (float)(f + 2) * 1.1920929e-07f);
    const float gu = fp32_score_gamma(f) * nu;
    UserSelect st;
    st.tau = active ? kNegInf : __int_as_float(0x7f800000);
    st.n_cand = 0;
    st.heap = heap_base + tid;
    st.stride = kThreads;
    st.K = K;
    st.cap = o.cap;
    st.cand_pos = o.cand_pos + u * (int64_t)o.cap;
    st.cand_ub = o.cand_ub + u * (int64_t)o.cap;
    heap_init(st.heap, st.stride, K);
    const int32_t* L = lists + (int64_t)j * n_items;
    const float* B = bounds + (int64_t)j * n_items;
    bool done = !active;
    int64_t seen = 0;
    const int64_t n_tiles = (n_items + kBlockItems - 1) / kBlockItems;

    auto load = [&](int buf, int64_t t0) {
      const int rows = (int)min((int64_t)kBlockItems, n_items - t0);
      float* tile = tiles + buf * kBlockItems * FP;
      for (int e = tid; e < rows * f; e += kThreads) {
        const int rr = e / f, k = e - rr * f;
        cp_async4(tile + rr * FP + k, items + (int64_t)L[t0 + rr] * f + k);
      }
      if (tid < rows) {
        const int32_t pos = L[t0 + tid];
        poss[buf * kBlockItems + tid] = pos;
        cp_async4(nrms + buf * kBlockItems + tid, item_nrm + pos);
      }
      cp_async_commit();
    };

    load(0, 0);
    for (int64_t t = 0; t < n_tiles; ++t) {
      const int buf = (int)(t & 1);
      const int64_t t0 = t * kBlockItems;
      // stop test with the leading bound of this tile (K items must be seen first)
      if (!done && seen >= K) {
        // a negative bound counts as 0: nhat_u, nhat_i exceed the true
        // norms, which would make a negative product too small
        float bnd = fmaxf(nu * B[t0], 0.f);
        bnd += bnd * 9.5367432e-07f;  // rounded up (2^-20)
        if (bnd < st.tau) done = true;
      }
      cp_async_wait_all();
      const int go = __syncthreads_or(!done);
      if (!go) break;
      if (t + 1 < n_tiles) load(buf ^ 1, t0 + kBlockItems);
      ++blocks;
      const int rows = (int)min((int64_t)kBlockItems, n_items - t0);
      if (!done) {
        const float* tile = tiles + buf * kBlockItems * FP;
        const float* nrm = nrms + buf * kBlockItems;
        const int32_t* pp = poss + buf * kBlockItems;
        for (int q = 0; q < rows; ++q) {
          float acc = 0.f;
          const float4* row = reinterpret_cast<const float4*>(tile + q * FP);
#pragma unroll
          for (int k4 = 0; k4 < FP / 4; ++k4) {
            const float4 a = row[k4];
            acc = __fmaf_rn(ur[4 * k4 + 0], a.x, acc);
            acc = __fmaf_rn(ur[4 * k4 + 1], a.y, acc);
            acc = __fmaf_rn(ur[4 * k4 + 2], a.z, acc);
            acc = __fmaf_rn(ur[4 * k4 + 3], a.w, acc);
          }
          const float h = __fmaf_rn(gu, nrm[q], acc);
          if (h >= st.tau) st.offer(h, __fmaf_rn(-gu, nrm[q], acc), pp[q]);
        }
        seen += rows;
      }
    }
    cp_async_wait_all();
    if (active) {
      o.tau[u] = st.tau;
      o.n_cand[u] = st.n_cand;
      visited[u] = (int32_t)seen;
      pairs += (unsigned long long)seen;
    }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, off);
  if ((tid & 31) == 0 && pairs) atomicAdd(&stats->pairs_scored, pairs);
  if (tid == 0 && blocks) atomicAdd(&stats->blocks_walked, blocks);
}

template <int FP>
cudaError_t launch_walk_fp(const float* users, int f, const float* items, const float* item_nrm, int64_t n_items,
                           const int32_t* lists, const float* bounds, const int32_t* user_perm, const int* offsets,
                           const int* tile_off, int C, int K, SelectOut o, int32_t* visited, int* work_counter,
                           DevStats* stats, int* err, int grid, cudaStream_t s) {
  const size_t smem = (size_t)(2 * kBlockItems * FP + 2 * kBlockItems + 2 * kBlockItems + K * kThreads) * 4;
  cudaError_t e = cudaFuncSetAttribute(maximus_walk_kernel<FP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  maximus_walk_kernel<FP><<<grid, kThreads, smem, s>>>(users, f, items, item_nrm, n_items, lists, bounds, user_perm,
                                                       offsets, tile_off, C, K, o, visited, work_counter, stats, err);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- tensor-core walk
// Cluster-ordered A rows: each cluster's users start at a 128-aligned row
// (pad_off), padding rows map to user -1.  One thread.
__global__ void mx_pad_layout_kernel(const int* __restrict__ counts, int C, int* __restrict__ pad_off) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  int o = 0;
  for (int j = 0; j < C; ++j) {
    pad_off[j] = o;
    o += (counts[j] + kThreads - 1) / kThreads * kThreads;
  }
  pad_off[C] = o;
}

__device__ __forceinline__ int find_segment(const int* __restrict__ off, int C, int x) {  // last j: off[j] <= x
  int lo = 0, hi = C - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) / 2;
    if (off[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// row_user[row] = user, user_row[user] = row, for every user (sorted rank r)
__global__ void mx_row_map_kernel(const int32_t* __restrict__ user_perm, int64_t n_users, const int* __restrict__ offsets,
                                  const int* __restrict__ pad_off, int C, int32_t* __restrict__ row_user,
                                  int32_t* __restrict__ user_row) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n_users) return;
  const int j = find_segment(offsets, C, (int)r);
  const int row = pad_off[j] + (int)(r - offsets[j]);
  const int32_t u = user_perm[r];
  row_user[row] = u;
  user_row[u] = row;
}

// dst[r] = src[map[r]] (BF16 rows of fp elements), zero rows for map < 0;
// 16-byte words.
__global__ void mx_gather_bf16_kernel(const uint4* __restrict__ src, const int32_t* __restrict__ map, int64_t n_rows,
                                      int words, uint4* __restrict__ dst) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_rows * words) return;
  const int64_t r = t / words;
  const int w = (int)(t - r * words);
  const int32_t m = map[r];
  dst[t] = m >= 0 ? src[(int64_t)m * words + w] : make_uint4(0, 0, 0, 0);
}

// Per-cluster item copies in list order (cluster j = blockIdx.y at rows
// j * n_pad + rank): BF16 operand rows, bound columns and positions for the
// list ranks [256 t_begin, 256 t_end_j), t_end_j = cl_end[j] (or t_end),
// capped at n_pad; ranks past the list are zero rows.  Only the ranks a walk
// reaches are copied.
__global__ void mx_items_by_cluster_kernel(const uint4* __restrict__ items_bf16, const float2* __restrict__ item_aux,
                                           const int32_t* __restrict__ lists, int64_t n_items, int64_t n_pad, int words,
                                           int t_begin, int t_end, const int* __restrict__ cl_end,
                                           uint4* __restrict__ b_rows, float2* __restrict__ aux_c,
                                           int32_t* __restrict__ pos_c) {
  const int64_t j = blockIdx.y;
  const int64_t r0 = (int64_t)t_begin * 256;
  const int64_t r1 = min(n_pad, (int64_t)(cl_end ? cl_end[j] : t_end) * 256);
  const int64_t n = (r1 - r0) * words;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t rank = r0 + e / words;
    const int w = (int)(e % words);
    const int64_t r = j * n_pad + rank;
    if (rank < n_items) {
      const int32_t pos = lists[j * n_items + rank];
      b_rows[r * words + w] = items_bf16[(int64_t)pos * words + w];
      if (w == 0) {
        aux_c[r] = item_aux[pos];
        pos_c[r] = pos;
      }
    } else {
      b_rows[r * words + w] = make_uint4(0, 0, 0, 0);
      if (w == 0) {
        aux_c[r] = make_float2(0.f, 0.f);
        pos_c[r] = 0;
      }
    }
  }
}

// Pass-1 work list: every 128-row user tile against the first t1 item tiles
// of its cluster's list.
__global__ void mx_work1_kernel(const int* __restrict__ pad_off, int C, int64_t n_pad, int t1, int* __restrict__ a_row,
                                int* __restrict__ b_row, int* __restrict__ tb, int* __restrict__ te,
                                int* __restrict__ n_work) {
  const int n = pad_off[C] / kThreads;
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w == 0) *n_work = n;
  if (w >= n) return;
  const int j = find_segment(pad_off, C, w * kThreads);
  a_row[w] = w * kThreads;
  b_row[w] = (int)(j * n_pad);
  tb[w] = 0;
  te[w] = t1;
}

// Item tiles every user needs after pass 1: ceil(r / 256) for the first list
// rank r >= r1 with max(nhat_u * bound(r), 0) < tau_u (rounded up), tau_u
// the K-th largest of the union of its two sub-lists' lower bounds (or
// their thresholds).  The list being sorted, no later item can reach tau_u
// either.  Users with no such rank need the whole list.  The sort key puts
// the users of a cluster in order of that need:
//   key = cluster << tile_bits | tiles.
__device__ __forceinline__ void mx_stop_user(const int32_t* __restrict__ assign, const float2* __restrict__ user_aux,
                                             const float* __restrict__ bounds, int64_t n_items, int r1, const SelectOut& o,
                                             int K, int tile_bits, int64_t u, int32_t* __restrict__ ustop,
                                             int* cl_max,  // shared or global per-cluster maxima
                                             uint32_t* __restrict__ keys, int32_t* __restrict__ vals) {
  const int64_t l0 = u * 2;
  float tau = fmaxf(o.tau[l0], o.tau[l0 + 1]);
  if (o.topl && o.topl_sorted) {
    const float* a = o.topl + l0 * K;
    const float* b = a + K;
    int ia = 0, ib = 0;
    float v = __int_as_float(0xff800000);
    for (int r = 0; r < K; ++r) {
      if (a[ia] >= b[ib]) v = a[ia++];
      else v = b[ib++];
    }
    tau = fmaxf(tau, v);
  }
  const float nu = user_aux[u].y;
  const int j = assign[u];
  const float* B = bounds + (int64_t)j * n_items;
  int64_t lo = r1 < n_items ? r1 : n_items, hi = n_items;  // first rank in [lo, hi) that stops; hi = none
  while (lo < hi) {
    const int64_t mid = (lo + hi) / 2;
    float bnd = fmaxf(nu * B[mid], 0.f);  // negative bounds count as 0, as in the walk
    bnd += bnd * 9.5367432e-07f;           // rounded up (2^-20)
    if (bnd < tau) hi = mid;
    else lo = mid + 1;
  }
  const int tiles = (int)((lo + 255) / 256);
  ustop[u] = tiles;
  atomicMax(&cl_max[j], tiles);
  keys[u] = ((uint32_t)j << tile_bits) | (uint32_t)tiles;
  vals[u] = (int32_t)u;
}

__global__ void mx_stop_kernel(const int32_t* __restrict__ assign, const float2* __restrict__ user_aux, int64_t n_users,
                               const float* __restrict__ bounds, int64_t n_items, int r1, SelectOut o, int K,
                               int tile_bits, int C, int use_smem, int32_t* __restrict__ ustop,
                               int* __restrict__ cl_end, uint32_t* __restrict__ keys, int32_t* __restrict__ vals) {
  extern __shared__ int st_clmax[];  // [C] per-block maxima (use_smem)
  if (use_smem) {
    for (int j = threadIdx.x; j < C; j += blockDim.x) st_clmax[j] = 0;
    __syncthreads();
  }
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u < n_users) mx_stop_user(assign, user_aux, bounds, n_items, r1, o, K, tile_bits, u, ustop,
                                use_smem ? st_clmax : cl_end, keys, vals);
  if (use_smem) {
    __syncthreads();
    for (int j = threadIdx.x; j < C; j += blockDim.x)
      if (st_clmax[j]) atomicMax(&cl_end[j], st_clmax[j]);
  }
}

// work_end[tile] = max item tiles over the users of the A tile.
__global__ void mx_tile_end_kernel(const int32_t* __restrict__ ustop, const int32_t* __restrict__ user_row,
                                   int64_t n_users, int* __restrict__ work_end) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n_users) return;
  atomicMax(&work_end[user_row[u] / kThreads], ustop[u]);
}

// Sort keys of the pass-2 work list: the A tiles that need more than t1
// item tiles, by cluster and within a cluster longest first
// (key = cluster << tile_bits | n_it - length), so that the CTAs running at
// one time read the same cluster's list through L2; the rest sort last.
__global__ void mx_work2_keys_kernel(const int* __restrict__ n_work1, const int* __restrict__ work_end,
                                     const int* __restrict__ b_row1, int64_t n_pad, int64_t max_work, int t1, int n_it,
                                     int tile_bits, uint32_t* __restrict__ keys, int32_t* __restrict__ vals,
                                     int* __restrict__ n_work2, DevStats* stats) {
  const int w = blockIdx.x * blockDim.x + threadIdx.x;
  if (w >= max_work) return;
  const bool real = w < *n_work1;
  const int end = real ? work_end[w] : 0;
  const uint32_t j = real ? (uint32_t)(b_row1[w] / n_pad) : 0u;
  keys[w] = end > t1 ? (j << tile_bits) | (uint32_t)(n_it - (end - t1)) : 0xffffffffu;
  vals[w] = w;
  if (end > t1) atomicAdd(n_work2, 1);
  if (real) atomicAdd(&stats->blocks_walked, (unsigned long long)(end > t1 ? end : t1));
}

__global__ void mx_work2_kernel(const int* __restrict__ n_work2, const int32_t* __restrict__ order,
                                const int* __restrict__ a_row1, const int* __restrict__ b_row1,
                                const int* __restrict__ work_end, int t1, int* __restrict__ a_row2,
                                int* __restrict__ b_row2, int* __restrict__ tb2, int* __restrict__ te2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= *n_work2) return;
  const int w = order[q];
  a_row2[q] = a_row1[w];
  b_row2[q] = b_row1[w];
  tb2[q] = t1;
  te2[q] = work_end[w];
}

// Items each user scored: the tiles its work item walked.
__global__ void mx_visited_kernel(const int32_t* __restrict__ user_row, int64_t n_users, const int* __restrict__ work_end,
                                  int t1, int64_t n_items, int32_t* __restrict__ visited,
                                  unsigned long long* __restrict__ pairs) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  unsigned long long v = 0;
  if (u < n_users) {
    const int end = max(t1, work_end[user_row[u] / kThreads]);
    v = (unsigned long long)min((int64_t)end * 256, n_items);
    visited[u] = (int32_t)v;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0 && v) atomicAdd(pairs, v);
}

unsigned copy_blocks(int C) {  // blocks per cluster of the list copies: about 64 per SM in all
  return (unsigned)std::max(1, sm_count() * 64 / std::max(C, 1));
}

int bits_for(int64_t x) {  // bits to hold 0..x
  int b = 0;
  while (b < 62 && (int64_t(1) << b) <= x) ++b;
  return b;
}

}  // namespace

bool mx_tc_regroup_fits(int C, int64_t n_items) {
  return bits_for(C - 1) + bits_for((n_items + 255) / 256) <= 32;
}

cudaError_t mx_tc_prepare(MxTc& m, const int32_t* user_perm, const void* items_bf16, const float2* item_aux,
                          const int32_t* lists, cudaStream_t s, int* launches) {
  m.items_bf16 = items_bf16;
  m.item_aux = item_aux;
  m.lists = lists;
  const int words = m.fp * m.esize / 16;
  mx_pad_layout_kernel<<<1, 32, 0, s>>>(m.counts, m.C, m.pad_off);
  cudaError_t e = cudaMemsetAsync(m.row_user, 0xff, sizeof(int32_t) * m.n_rows_max, s);
  if (e != cudaSuccess) return e;
  mx_row_map_kernel<<<(unsigned)((m.n_users + 255) / 256), 256, 0, s>>>(user_perm, m.n_users, m.offsets, m.pad_off, m.C,
                                                                        m.row_user, m.user_row);
  mx_gather_bf16_kernel<<<(unsigned)((m.n_rows_max * words + 255) / 256), 256, 0, s>>>(
      (const uint4*)m.users_bf16, m.row_user, m.n_rows_max, words, (uint4*)m.a_rows);
  const dim3 cgrid(copy_blocks(m.C), (unsigned)m.C);
  mx_items_by_cluster_kernel<<<cgrid, 256, 0, s>>>((const uint4*)items_bf16, item_aux, lists, m.n_items, m.n_pad, words,
                                                   0, m.t1, nullptr, (uint4*)m.b_rows, m.aux_c, m.pos_c);
  const int64_t mw = m.max_work;
  mx_work1_kernel<<<(unsigned)((mw + 255) / 256), 256, 0, s>>>(m.pad_off, m.C, m.n_pad, m.t1, m.w1, m.w1 + mw,
                                                                m.w1 + 2 * mw, m.w1 + 3 * mw, m.n_work);
  *launches += 5;
  return cudaGetLastError();
}

cudaError_t mx_tc_pass2(MxTc& m, const int32_t* assign, const float2* user_aux, const float* bounds, SelectOut o, int K,
                        int32_t** user_perm, int32_t* visited, DevStats* stats, cudaStream_t s, int* launches) {
  const int64_t mw = m.max_work, nU = m.n_users;
  const unsigned ub = (unsigned)((nU + 255) / 256), wb = (unsigned)((mw + 255) / 256);
  const int tile_bits = bits_for(m.n_it);
  const int key_bits = bits_for(m.C - 1) + tile_bits;
  cudaError_t e = cudaMemsetAsync(m.work_end, 0, sizeof(int) * mw, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m.n_work + 1, 0, sizeof(int), s);
  if (e == cudaSuccess) e = cudaMemsetAsync(m.cl_end, 0, sizeof(int) * m.C, s);
  if (e != cudaSuccess) return e;
  const int st_smem = m.C <= 8192;
  mx_stop_kernel<<<ub, 256, st_smem ? sizeof(int) * m.C : 0, s>>>(assign, user_aux, nU, bounds, m.n_items, m.t1 * 256,
                                                                   o, K, tile_bits, m.C, st_smem, m.ustop, m.cl_end,
                                                                   m.ukeys[0], m.uvals[0]);
  // the rest of each cluster's list that some member still needs
  const dim3 cgrid(copy_blocks(m.C), (unsigned)m.C);
  mx_items_by_cluster_kernel<<<cgrid, 256, 0, s>>>((const uint4*)m.items_bf16, m.item_aux, m.lists, m.n_items, m.n_pad,
                                                   (m.fp * m.esize / 16), m.t1, 0, m.cl_end, (uint4*)m.b_rows, m.aux_c, m.pos_c);
  *launches += 2;
  // regroup: the users of each cluster in order of the item tiles they
  // need, so that each A tile's walk is close to its users' own need
  uint32_t* k0 = m.ukeys[0];
  int32_t* v0 = m.uvals[0];
  uint32_t* k1 = m.ukeys[1];
  int32_t* v1 = m.uvals[1];
  e = radix_sort_pairs(k0, v0, k1, v1, nU, 1, 0, key_bits, m.temp, s, launches);
  if (e != cudaSuccess) return e;
  *user_perm = v0;
  mx_row_map_kernel<<<ub, 256, 0, s>>>(v0, nU, m.offsets, m.pad_off, m.C, m.row_user, m.user_row);
  mx_gather_bf16_kernel<<<(unsigned)((m.n_rows_max * ((m.fp * m.esize / 16)) + 255) / 256), 256, 0, s>>>(
      (const uint4*)m.users_bf16, m.row_user, m.n_rows_max, (m.fp * m.esize / 16), (uint4*)m.a_rows);
  mx_tile_end_kernel<<<ub, 256, 0, s>>>(m.ustop, m.user_row, nU, m.work_end);
  mx_work2_keys_kernel<<<wb, 256, 0, s>>>(m.n_work, m.work_end, m.w1 + mw, m.n_pad, mw, m.t1, m.n_it, tile_bits,
                                          m.wkeys[0], m.wvals[0], m.n_work + 1, stats);
  *launches += 4;
  uint32_t* wk0 = m.wkeys[0];
  int32_t* wv0 = m.wvals[0];
  uint32_t* wk1 = m.wkeys[1];
  int32_t* wv1 = m.wvals[1];
  e = radix_sort_pairs(wk0, wv0, wk1, wv1, mw, 1, 0, 32, m.temp, s, launches);
  if (e != cudaSuccess) return e;
  mx_work2_kernel<<<wb, 256, 0, s>>>(m.n_work + 1, wv0, m.w1, m.w1 + mw, m.work_end, m.t1, m.w2, m.w2 + mw,
                                     m.w2 + 2 * mw, m.w2 + 3 * mw);
  mx_visited_kernel<<<ub, 256, 0, s>>>(m.user_row, nU, m.work_end, m.t1, m.n_items, visited, &stats->pairs_scored);
  *launches += 2;
  return cudaGetLastError();
}

// k-means initial centroids: C distinct users drawn by Floyd's algorithm
// from SplitMix64 over a counter keyed by the seed (one thread; `chosen` is
// a zeroed bitmap of n bits).  For j = n - C .. n - 1: t = draw mod (j + 1);
// take t, or j if t was taken before.
namespace {

__device__ __forceinline__ uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void draw_init_ids_kernel(int64_t n, int C, uint64_t seed, uint32_t* __restrict__ chosen,
                                     int64_t* __restrict__ ids) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  uint64_t ctr = 0;
  int k = 0;
  for (int64_t j = n - C; j < n; ++j, ++k) {
    const int64_t t = (int64_t)(splitmix64(seed ^ splitmix64(++ctr)) % (uint64_t)(j + 1));
    const bool taken = (chosen[t >> 5] >> (t & 31)) & 1u;
    const int64_t pick = taken ? j : t;
    chosen[pick >> 5] |= 1u << (pick & 31);
    ids[k] = pick;
  }
}

}  // namespace

cudaError_t draw_init_ids(int64_t n, int C, uint64_t seed, uint32_t* chosen_bits, int64_t* ids, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(chosen_bits, 0, sizeof(uint32_t) * ((n + 31) / 32), s);
  if (e != cudaSuccess) return e;
  draw_init_ids_kernel<<<1, 32, 0, s>>>(n, C, seed, chosen_bits, ids);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- host side
namespace {

// One assignment step over n_users users and C centroids (hn2 = ||c_j||^2 / 2).
cudaError_t launch_kmeans_assign(const float* users, int64_t n_users, int f, const float* cent, const float* hn2,
                                 int C, int32_t* assign, cudaStream_t s) {
  const int fp = (int)round_up(f, 8);
  const unsigned blocks = (unsigned)((n_users + kThreads - 1) / kThreads);
  switch (fp) {
#define MIPS_KM_CASE(N) \
  case N:               \
    kmeans_assign_kernel<N><<<blocks, kThreads, 0, s>>>(users, n_users, f, cent, hn2, C, assign); \
    break;
    MIPS_KM_CASE(8) MIPS_KM_CASE(16) MIPS_KM_CASE(24) MIPS_KM_CASE(32) MIPS_KM_CASE(40) MIPS_KM_CASE(48)
    MIPS_KM_CASE(56) MIPS_KM_CASE(64) MIPS_KM_CASE(72) MIPS_KM_CASE(80) MIPS_KM_CASE(88) MIPS_KM_CASE(96)
    MIPS_KM_CASE(104) MIPS_KM_CASE(112) MIPS_KM_CASE(120) MIPS_KM_CASE(128)
#undef MIPS_KM_CASE
    default:
      return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

// Dynamic users (Sec. III-E, practical usage): a call's users are assigned to
// centroids fitted earlier, and only the clusters that receive users are
// kept.  used[j] marks cluster j.
__global__ void cluster_used_kernel(const int32_t* __restrict__ assign, int64_t n, int* __restrict__ used) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    used[assign[u]] = 1;
}

// One block of 1024 threads: the used clusters, in cluster order, get the
// slots 0, 1, ... (remap[j] = slot, or -1 for an unused cluster) and their
// centroids are packed into cent_out.  Slots past the last used cluster (up
// to C_eff) repeat the first packed centroid; no user is assigned to them.
__global__ void __launch_bounds__(1024) cluster_pack_kernel(const int* __restrict__ used, int C_fit,
                                                            const float* __restrict__ cent_fit, int f, int C_eff,
                                                            int* __restrict__ remap, float* __restrict__ cent_out) {
  __shared__ int s_warp[32];
  __shared__ int s_base;
  const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  if (tid == 0) s_base = 0;
  __syncthreads();
  for (int c0 = 0; c0 < C_fit; c0 += 1024) {
    const int j = c0 + tid;
    const int v = j < C_fit ? (used[j] != 0) : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int t = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
      int w = s_warp[lane], wi = w;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, wi, o);
        if (lane >= o) wi += t;
      }
      s_warp[lane] = wi - w;  // exclusive prefix of the warp totals
    }
    __syncthreads();
    const int slot = s_base + s_warp[wid] + incl - v;
    if (j < C_fit) remap[j] = v ? slot : -1;
    if (v)
      for (int k = 0; k < f; ++k) cent_out[(int64_t)slot * f + k] = cent_fit[(int64_t)j * f + k];
    __syncthreads();  // every thread has read s_base and s_warp
    if (tid == 1023) s_base = slot + v;
    __syncthreads();
  }
  const int n_used = s_base;
  for (int e = tid; e < (C_eff - n_used) * f; e += 1024) {
    const int d = n_used + e / f, k = e % f;
    cent_out[(int64_t)d * f + k] = cent_out[k];
  }
}

__global__ void cluster_remap_kernel(int32_t* __restrict__ assign, int64_t n, const int* __restrict__ remap) {
  for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
    assign[u] = remap[assign[u]];
}

}  // namespace

cudaError_t maximus_assign_fitted(const float* users, int64_t n_users, int f, const float* cent_fit, int C_fit,
                                  float* hn2_fit, int32_t* assign, int* used, int* remap, float* cent, int C_eff,
                                  const KmTc& tc, cudaStream_t s, int* launches) {
  half_norm2_kernel<<<(C_fit + 127) / 128, 128, 0, s>>>(cent_fit, C_fit, f, hn2_fit);
  cudaError_t e;
  if (tc.users_km) {
    e = km_tc_users(users, n_users, f, tc.users_km, s);
    if (e == cudaSuccess)
      e = km_tc_assign(tc.users_km, n_users, f, cent_fit, hn2_fit, C_fit, tc.cent_km, assign, tc.err, tc.max_smem, s);
    *launches += 3;
  } else {
    e = launch_kmeans_assign(users, n_users, f, cent_fit, hn2_fit, C_fit, assign, s);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(used, 0, sizeof(int) * C_fit, s);
  if (e != cudaSuccess) return e;
  const unsigned g = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_users + 255) / 256, (int64_t)sm_count() * 8));
  cluster_used_kernel<<<g, 256, 0, s>>>(assign, n_users, used);
  cluster_pack_kernel<<<1, 1024, 0, s>>>(used, C_fit, cent_fit, f, C_eff, remap, cent);
  cluster_remap_kernel<<<g, 256, 0, s>>>(assign, n_users, remap);
  *launches += 5;
  return cudaGetLastError();
}

cudaError_t maximus_kmeans(const float* users, int64_t n_users, int f, int C, int iters, const int64_t* init_ids_dev,
                           float* cent, float* hn2, int32_t* assign, unsigned long long* sums, unsigned int* counts,
                           uint32_t* absmax, float* scale, bool spherical, const KmTc& tc, cudaStream_t s,
                           int* launches) {
  gather_rows_i64<<<(unsigned)((C * f + 255) / 256), 256, 0, s>>>(users, init_ids_dev, C, f, cent);
  if (spherical) {
    normalize_rows_kernel<<<(C + 127) / 128, 128, 0, s>>>(cent, C, f);
    *launches += 1;
  }
  cudaError_t e = cudaMemsetAsync(absmax, 0, sizeof(uint32_t), s);
  if (e != cudaSuccess) return e;
  absmax_kernel<<<sm_count() * 4, 256, 0, s>>>(users, n_users * f, absmax);
  *launches += 2;
  kmeans_scale_kernel<<<1, 32, 0, s>>>(absmax, n_users, scale);
  *launches += 1;
  if (tc.users_km) {  // the users' BF16 operand rows, once
    e = km_tc_users(users, n_users, f, tc.users_km, s);
    if (e != cudaSuccess) return e;
    *launches += 1;
  }
  for (int it = 0; it < iters; ++it) {
    half_norm2_kernel<<<(C + 127) / 128, 128, 0, s>>>(cent, C, f, hn2);
    if (tc.users_km) {
      e = km_tc_assign(tc.users_km, n_users, f, cent, hn2, C, tc.cent_km, assign, tc.err, tc.max_smem, s);
      *launches += 1;
    } else {
      e = launch_kmeans_assign(users, n_users, f, cent, hn2, C, assign, s);
    }
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(sums, 0, sizeof(unsigned long long) * C * f, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(counts, 0, sizeof(unsigned int) * C, s);
    if (e != cudaSuccess) return e;
    // partial sums private to groups of G = ceil(f / 32) warps (each warp a
    // 32-dimension slice): 8, 4 or 2 groups per block, when they fit
    int max_smem = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int G = (f + 31) / 32;
    const size_t per_group = (size_t)C * f * 8 + (size_t)C * 4;
    int ngb = std::max(1, 8 / G);  // groups per block: at most 8 warps (f <= 32: one warp per group)
    while (ngb >= 2 && (size_t)ngb * per_group > (size_t)max_smem) ngb /= 2;
    if (ngb >= 2 || (ngb == 1 && G > 1 && per_group <= (size_t)max_smem)) {
      const size_t smem = (size_t)ngb * per_group;
      e = cudaFuncSetAttribute(kmeans_accum_warp_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      const int per_sm = std::max<int>(1, (int)((size_t)228 * 1024 / (smem + 1024)));
      const unsigned bx = (unsigned)std::max<int64_t>(
          1, std::min<int64_t>((n_users + 8 * ngb - 1) / (8 * ngb), (int64_t)sm_count() * std::min(per_sm, 8)));
      kmeans_accum_warp_kernel<<<bx, ngb * G * 32, smem, s>>>(users, n_users, f, assign, C, scale, sums, counts, G);
    } else if ((size_t)C * f * 8 + (size_t)C * 4 <= 96 * 1024) {
      // all partial sums fit one block's shared memory
      const size_t smem = (size_t)C * f * 8 + (size_t)C * 4;
      e = cudaFuncSetAttribute(kmeans_accum_smem_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      const unsigned bx = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_users * f + 255) / 256, (int64_t)sm_count() * 8));
      kmeans_accum_smem_kernel<<<dim3(bx, 1), 256, smem, s>>>(users, n_users, f, assign, C, C, scale, sums, counts);
    } else {  // many clusters: the global adds spread over C * f addresses
      kmeans_accum_kernel<<<(unsigned)((n_users * f + 255) / 256), 256, 0, s>>>(users, n_users, f, assign, C, scale,
                                                                              sums, counts);
    }
    kmeans_update_kernel<<<(C * f + 255) / 256, 256, 0, s>>>(sums, counts, C, f, scale, cent);
    *launches += 4;
    if (spherical) {
      normalize_rows_kernel<<<(C + 127) / 128, 128, 0, s>>>(cent, C, f);
      *launches += 1;
    }
  }
  return cudaGetLastError();
}

cudaError_t maximus_bounds(const float* users, int64_t n_users, int f, const int32_t* assign, const float* cent, int C,
                           const float* items, const float* item_nrm, int64_t n_items, uint32_t* cosb_ord,
                           uint32_t* keys, int32_t* vals, float* cosb_f, cudaStream_t s, int* launches) {
  cosb_init_kernel<<<(C + 127) / 128, 128, 0, s>>>(cosb_ord, C);
  {  // four users per warp; at most 8 blocks of 256 threads per SM, fewer for small inputs
    const int64_t blocks = std::min<int64_t>((n_users + 31) / 32, (int64_t)sm_count() * 8);
    cosb_kernel<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(users, n_users, f, assign, cent, C, cosb_ord);
  }
  const size_t smem = sizeof(float) * (cb_items_floats(f) + (size_t)f * kCbChunk + 4 * kCbChunk);
  cudaError_t e = cudaFuncSetAttribute(cbound_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const dim3 grid((unsigned)((n_items + kCbItems - 1) / kCbItems), (unsigned)((C + kCbChunk - 1) / kCbChunk));
  cbound_kernel<<<grid, kCbItems, smem, s>>>(cent, C, f, items, item_nrm, n_items, cosb_ord, keys, vals);
  cosb_to_float_kernel<<<(C + 127) / 128, 128, 0, s>>>(cosb_ord, C, cosb_f);
  *launches += 4;
  return cudaGetLastError();
}

cudaError_t maximus_group(const int32_t* assign, int64_t n_users, int C, uint32_t* keys, int32_t* ids, uint32_t* keys_alt,
                          int32_t* ids_alt, uint32_t* temp, int* counts, int* offsets, int* tile_off,
                          int32_t** user_perm, cudaStream_t s, int* launches) {
  iota_u32_kernel<<<(unsigned)((n_users + 255) / 256), 256, 0, s>>>(assign, n_users, keys, ids);
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(int) * C, s);
  if (e != cudaSuccess) return e;
  {
    const int use_smem = C <= 8192;
    const unsigned blocks = (unsigned)std::max<int64_t>(1, std::min<int64_t>((n_users + 255) / 256, (int64_t)sm_count() * 4));
    cluster_count_kernel<<<blocks, 256, use_smem ? sizeof(int) * C : 0, s>>>(assign, n_users, C, use_smem, counts);
  }
  cluster_offsets_kernel<<<1, 32, 0, s>>>(counts, C, offsets, tile_off);
  *launches += 3;
  int bits = 8;
  while ((1 << bits) < C) bits += 8;
  e = radix_sort_pairs(keys, ids, keys_alt, ids_alt, n_users, 1, 0, bits, temp, s, launches);
  *user_perm = ids;
  return e;
}

cudaError_t maximus_walk(const float* users, int f, const float* items, const float* item_nrm, int64_t n_items,
                         const int32_t* lists, const float* bounds, const int32_t* user_perm, const int* offsets,
                         const int* tile_off, int C, int K, SelectOut o, int32_t* visited, int* work_counter,
                         DevStats* stats, int* err, int num_sms, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(work_counter, 0, sizeof(int), s);
  if (e != cudaSuccess) return e;
  const int grid = num_sms * 4;
  switch ((int)round_up(f, 8)) {
#define MIPS_W_CASE(N) \
  case N:              \
    return launch_walk_fp<N>(users, f, items, item_nrm, n_items, lists, bounds, user_perm, offsets, tile_off, C, K, o, \
                             visited, work_counter, stats, err, grid, s);
    MIPS_W_CASE(8) MIPS_W_CASE(16) MIPS_W_CASE(24) MIPS_W_CASE(32) MIPS_W_CASE(40) MIPS_W_CASE(48) MIPS_W_CASE(56)
    MIPS_W_CASE(64) MIPS_W_CASE(72) MIPS_W_CASE(80) MIPS_W_CASE(88) MIPS_W_CASE(96) MIPS_W_CASE(104) MIPS_W_CASE(112)
    MIPS_W_CASE(120) MIPS_W_CASE(128)
#undef MIPS_W_CASE
    default:
      return cudaErrorInvalidValue;
  }
}

cudaError_t maximus_keys_to_bounds(const uint32_t* keys, int64_t n, float* out, cudaStream_t s) {
  keys_to_bounds_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(keys, n, out);
  return cudaGetLastError();
}

}  // namespace mips
