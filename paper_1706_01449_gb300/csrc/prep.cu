// Input preparation: row-norm upper bounds, BF16 operand rows with bound
// columns, row gathers.  The exact answer is Sec. II-B's top-K of u^T i per
// user; the blocked multiply (Sec. II-C) scores in BF16 here, and the bound
// columns keep every true top-K item above the select's threshold.
//
// BF16 operand layout (K-major rows of fp = round_up(f + 2, 16) bf16):
//   users (A operand): [ RN(u_0) .. RN(u_{f-1}) | beta_u | nhat_u | 0 ... ]
//   items (B operand): [ RN(i_0) .. RN(i_{f-1}) | nhat_i | alpha_i | 0 ... ]
// so that one tensor-core product of a user row with an item row yields
//   H = u~ . i~ + beta_u nhat_i + nhat_u alpha_i,
// an upper bound on the exact u^T i of the FP32 inputs, where
//   nhat_x  >= max(||x||, ||x~||)                      (rounded up to BF16)
//   beta_u  >= (||u - u~|| + g nhat_u)(1 + g)           (rounded up to BF16)
//   alpha_i >= (||i - i~|| + g nhat_i)(1 + g)           (rounded up to BF16)
// and g = (fp + 4) 2^-20 + f 2^-50 bounds the relative error of the FP32
// tensor-core accumulation over fp terms (taken far looser than any
// rounding or truncation accumulator of 23+ bits needs) together with the
// rounding of the FP64 definition.  Why H >= u^T i:
//   u^T i - u~.i~ = (u - u~)^T i + u~^T (i - i~)  <=  ||u-u~|| ||i|| + ||u~|| ||i-i~||,
// each bound column product covers one of those terms plus g nhat_u nhat_i,
// which exceeds the accumulation error g (||u~|| ||i~|| + bound terms).
// The matching lower bound used by the select is
//   L = H - 2 A - g (nhat_u nhat_i + A),   A = beta_u nhat_i + nhat_u alpha_i.
#include <cuda_bf16.h>
#include <cuda_fp8.h>

#include "common.cuh"

namespace mips {

namespace {

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ float warp_max(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// FP32 sum of squares of f terms has relative error below f 2^-24; the
// square root halves it.  This factor lifts the computed norm above the
// exact one with room to spare.  The sums are taken over rows scaled by a
// power of two (common.cuh: the largest |entry| in [1/2, 1)), so no term
// that matters is subnormal; `floor` covers the absolute error of those
// that are (below 2^-149 per entry and per square).
__device__ __forceinline__ float norm_ub(float sumsq, int f) {
  return __fsqrt_rn(sumsq) * (1.0f + (float)(f + 2) * 1.1920929e-07f);
}
__device__ __forceinline__ float tiny_floor(int f) { return (float)f * 1.1210388e-44f; }  // f 2^-146

__global__ void row_norm_ub_kernel(const float* __restrict__ x, int64_t n, int f,
                                   float* __restrict__ out, int* err) {
  int64_t row = (int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32;
  int lane = threadIdx.x & 31;
  if (row >= n) return;
  const float* r = x + row * f;
  float amax = 0.f;
  bool bad = false;
  for (int k = lane; k < f; k += 32) {
    amax = fmaxf(amax, fabsf(r[k]));
    bad |= !isfinite(r[k]);
  }
  amax = warp_max(amax);
  if (__any_sync(0xffffffffu, bad)) {
    if (lane == 0) {
      atomicOr(err, DEV_ERR_NONFINITE);
      out[row] = __int_as_float(0x7f800000);
    }
    return;
  }
  if (amax == 0.f) {  // the zero row: its norm is 0
    if (lane == 0) out[row] = 0.f;
    return;
  }
  const int e = norm_scale_exp(amax);
  float ss = 0.f;
  for (int k = lane; k < f; k += 32) {
    const float y = scale_pow2(r[k], e);
    ss = __fmaf_rn(y, y, ss);
  }
  ss = warp_sum(ss);
  if (lane == 0) {
    const float nb = unscale_pow2_ru(norm_ub(ss + tiny_floor(f), f), e);
    if (!isfinite(nb)) atomicOr(err, DEV_ERR_NONFINITE);
    out[row] = nb;
  }
}

// Rows per warp of the FP8 quantisation kernel: the loads of all of them
// are issued before any row's arithmetic (f <= 128: four elements per lane).
constexpr int kQuantRows = 4;

// BF16 operand rows, eight lanes per row (a warp quantises four rows at
// once; a whole warp per row spent most of its issue slots on the
// per-row reductions): lane s of a row's group holds elements s, s + 8, ..
// (up to 16 of them: f <= 128).  The sums are taken per lane and then over
// the group by three shuffle steps; the norm bounds allow a relative error
// of f 2^-24 for any order of summation.
__global__ void __launch_bounds__(256)
    quant_bf16_kernel(const float* __restrict__ x, int64_t n, int f, int fp, int role, __nv_bfloat16* __restrict__ out,
                      int64_t n_rows_out, float2* __restrict__ aux, int* err) {
  const int lane = threadIdx.x & 31, sub = lane & 7;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 3;
  if (row >= n_rows_out) return;  // (whole groups: a group's lanes share the row)
  const unsigned gm = 0xFFu << (lane & 24);  // this row's eight lanes
  __nv_bfloat16* o = out + row * fp;
  if (row >= n) {  // padding rows
    for (int k = sub; k < fp; k += 8) o[k] = __float2bfloat16_rn(0.f);
    return;
  }
  const float* r = x + row * f;
  float v[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int k = sub + 8 * j;
    v[j] = k < f ? r[k] : 0.f;
  }
  float amax = 0.f;
#pragma unroll
  for (int j = 0; j < 16; ++j) amax = fmaxf(amax, fabsf(v[j]));
#pragma unroll
  for (int o2 = 4; o2 > 0; o2 >>= 1) amax = fmaxf(amax, __shfl_xor_sync(gm, amax, o2));
  // sums over the row scaled by 2^e (largest |entry| in [1/2, 1)); a
  // non-finite or zero row keeps e = 0 (the non-finite check below flags it)
  const int e = (amax > 0.f && isfinite(amax)) ? norm_scale_exp(amax) : 0;
  float ss_x = 0.f, ss_t = 0.f, ss_d = 0.f;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    const int k = sub + 8 * j;
    if (k < f) {
      const float xv = v[j];
      const __nv_bfloat16 q = __float2bfloat16_rn(xv);
      const float t = __bfloat162float(q);
      const float d = __fsub_rn(xv, t);  // exact: t is xv rounded to 8 significant bits
      const float xs = scale_pow2(xv, e), ts = scale_pow2(t, e), ds = scale_pow2(d, e);
      ss_x = __fmaf_rn(xs, xs, ss_x);
      ss_t = __fmaf_rn(ts, ts, ss_t);
      ss_d = __fmaf_rn(ds, ds, ss_d);
      o[k] = q;
    }
  }
#pragma unroll
  for (int o2 = 4; o2 > 0; o2 >>= 1) {
    ss_x += __shfl_xor_sync(gm, ss_x, o2);
    ss_t += __shfl_xor_sync(gm, ss_t, o2);
    ss_d += __shfl_xor_sync(gm, ss_d, o2);
  }
  const float g = (float)(fp + 4) * 9.5367432e-07f + (float)f * 8.8817842e-16f;  // 2^-20, 2^-50
  // the zero row keeps 0 bounds (its scores are exactly 0); otherwise the
  // largest scaled square is at least 1/4, and the floor covers subnormal
  // squares of small entries and of the rounding errors d
  float nhat = 0.f, errn = 0.f;
  if (amax > 0.f) {
    nhat = unscale_pow2_ru(fmaxf(norm_ub(ss_x + tiny_floor(f), f), norm_ub(ss_t + tiny_floor(f), f)), e);
    errn = unscale_pow2_ru(norm_ub(ss_d + tiny_floor(f), f), e);
  }
  const __nv_bfloat16 nhat_b = __float2bfloat16_ru(nhat);
  const __nv_bfloat16 eb_b = __float2bfloat16_ru(__fmul_ru(__fmaf_ru(g, nhat, errn), 1.0f + g));
  if (sub == 0) {
    if (!isfinite(ss_x) || !isfinite(__bfloat162float(nhat_b))) atomicOr(err, DEV_ERR_NONFINITE);
    if (role == 0) {
      o[f] = eb_b;        // beta_u
      o[f + 1] = nhat_b;  // nhat_u
      aux[row] = make_float2(__bfloat162float(eb_b), __bfloat162float(nhat_b));
    } else {
      o[f] = nhat_b;    // nhat_i
      o[f + 1] = eb_b;  // alpha_i
      aux[row] = make_float2(__bfloat162float(nhat_b), __bfloat162float(eb_b));
    }
  }
  for (int k = f + 2 + sub; k < fp; k += 8) o[k] = __float2bfloat16_rn(0.f);
}

// ---------------------------------------------------------------- FP8 rows
// E4M3 operand layout (K-major rows of fp = tc_row_len8(f) bytes):
//   users: [ q(u_k / s_u) .. | RU(beta_u / s_u) | RU(nhat_u / s_u) | 0 .. ],  s_u = nhat_u / 384 per row
//   items: [ q(i_k / s_I) .. | RU(nhat_i / s_I) | RU(alpha_i / s_I) | 0 .. ], s_I = (max_i nhat_i) / 384
// q: round to nearest E4M3, saturating; RU: the quotient rounded up, then
// up to an E4M3 value.  The operands the MMA multiplies are, in input
// units, u~ = s_u q(u / s_u) and i~ = s_I q(i / s_I), and the bound columns
// are the BF16 layout's for these u~, i~ (nhat >= max(||x||, ||x~||),
// beta and alpha >= (||x - x~|| + g nhat)(1 + g)).  A rounded-up column
// times its scale is at least its input-unit value, so s_u s_I times the
// accumulator is H >= u~ . i~ + beta_u nhat_i + nhat_u alpha_i >= u^T i as in
// the BF16 case; aux receives those products (rounded up), so the select's
// A = beta_u nhat_i + nhat_u alpha_i from aux covers the folded columns and
// the quantisation error alike, and L = H - 2 A - g (nhat_u nhat_i + A)
// stays a lower bound.  The scales put every entry and every norm column at
// most 384 (times 1 + 2^-4 for nhat of a rounded row), below E4M3's 448.
constexpr float kFp8Inv = 2.6041666e-03f;  // 1 / 384

__device__ __forceinline__ uint8_t e4m3_rn(float x) {
  return (uint8_t)__nv_cvt_float_to_fp8(x, __NV_SATFINITE, __NV_E4M3);
}
__device__ __forceinline__ float e4m3_val(uint8_t q) {
  const __half_raw h = __nv_cvt_fp8_to_halfraw((__nv_fp8_storage_t)q, __NV_E4M3);
  return __half2float(__half(h));
}
// x >= 0 rounded up to an E4M3 value (positive encodings are ordered like
// their values; 0x7e = 448 is the largest finite one).
__device__ __forceinline__ uint8_t e4m3_ru(float x, int* err) {
  uint8_t q = e4m3_rn(x);
  if (e4m3_val(q) < x) {
    if (q >= 0x7e) atomicOr(err, DEV_ERR_INTERNAL);  // not reached: the scales keep x below 448
    else ++q;
  }
  return q;
}

// One row whose elements this lane holds in v (element lane + 32 j in v[j]).
// role 0 (users): the row's own scale, written to row_scale[row]; role 1
// (items): the scale *item_scale.
__device__ __forceinline__ void quant_fp8_row(const float (&v)[4], int64_t row, int64_t n, int f, int fp, int role,
                                              const float* __restrict__ item_scale, uint8_t* __restrict__ out,
                                              float2* __restrict__ aux, float* __restrict__ row_scale, int* err,
                                              int lane) {
  uint8_t* o = out + row * fp;
  if (row >= n) {  // padding rows
    for (int k = lane; k < fp; k += 32) o[k] = 0;
    return;
  }
  float amax = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (lane + 32 * j < f) amax = fmaxf(amax, fabsf(v[j]));
  amax = warp_max(amax);
  const int e = (amax > 0.f && isfinite(amax)) ? norm_scale_exp(amax) : 0;
  float ss_x = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j)
    if (lane + 32 * j < f) {
      const float xs = scale_pow2(v[j], e);
      ss_x = __fmaf_rn(xs, xs, ss_x);
    }
  ss_x = warp_sum(ss_x);
  const float nx = amax > 0.f ? unscale_pow2_ru(norm_ub(ss_x + tiny_floor(f), f), e) : 0.f;
  float sc = role == 0 ? __fmul_rn(nx, kFp8Inv) : *item_scale;
  if (!(sc > 0.f) || !isfinite(sc)) sc = 1.f;  // the zero row (every entry quantises to 0)
  float ss_t = 0.f, ss_d = 0.f;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int k = lane + 32 * j;
    if (k < f) {
      const float x = v[j];
      const uint8_t q = e4m3_rn(__fdiv_rn(x, sc));
      const float qv = e4m3_val(q);
      const float t = __fmul_rn(sc, qv);       // x~ (one rounding)
      const float d = __fmaf_rn(-sc, qv, x);   // x - x~ (one rounding)
      const float ts = scale_pow2(t, e), ds = scale_pow2(d, e);
      ss_t = __fmaf_rn(ts, ts, ss_t);
      ss_d = __fmaf_rn(ds, ds, ss_d);
      o[k] = q;
    }
  }
  ss_t = warp_sum(ss_t);
  ss_d = warp_sum(ss_d);
  const float g = (float)(fp + 4) * 9.5367432e-07f + (float)f * 8.8817842e-16f;  // 2^-20, 2^-50
  float nhat = 0.f, errn = 0.f;
  if (amax > 0.f) {
    nhat = fmaxf(nx, unscale_pow2_ru(norm_ub(ss_t + tiny_floor(f), f), e));
    errn = unscale_pow2_ru(norm_ub(ss_d + tiny_floor(f), f), e);
  }
  const float eb = __fmul_ru(__fmaf_ru(g, nhat, errn), 1.0f + g);
  if (lane == 0) {
    if (!isfinite(ss_x) || !isfinite(nhat)) atomicOr(err, DEV_ERR_NONFINITE);
    const float c0 = role == 0 ? eb : nhat, c1 = role == 0 ? nhat : eb;
    const uint8_t q0 = e4m3_ru(__fdiv_ru(c0, sc), err), q1 = e4m3_ru(__fdiv_ru(c1, sc), err);
    o[f] = q0;
    o[f + 1] = q1;
    aux[row] = make_float2(__fmul_ru(sc, e4m3_val(q0)), __fmul_ru(sc, e4m3_val(q1)));
    if (role == 0) row_scale[row] = sc;
  }
  for (int k = f + 2 + lane; k < fp; k += 32) o[k] = 0;
}

// A warp per kQuantRows consecutive rows.
__global__ void quant_fp8_kernel(const float* __restrict__ x, int64_t n, int f, int fp, int role,
                                 const float* __restrict__ item_scale, uint8_t* __restrict__ out, int64_t n_rows_out,
                                 float2* __restrict__ aux, float* __restrict__ row_scale, int* err) {
  const int lane = threadIdx.x & 31;
  const int64_t row0 = ((int64_t)blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32) * kQuantRows;
  if (row0 >= n_rows_out) return;
  float v[kQuantRows][4];
#pragma unroll
  for (int q = 0; q < kQuantRows; ++q) {
    const int64_t row = row0 + q;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int k = lane + 32 * j;
      v[q][j] = (row < n && k < f) ? x[row * f + k] : 0.f;
    }
  }
#pragma unroll
  for (int q = 0; q < kQuantRows; ++q)
    if (row0 + q < n_rows_out)
      quant_fp8_row(v[q], row0 + q, n, f, fp, role, item_scale, out, aux, row_scale, err, lane);
}

// s_I from the largest item norm bound (the sorted bounds' first entry).
__global__ void fp8_item_scale_kernel(const float* __restrict__ item_nrm, int64_t n, float* __restrict__ out) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const float m = n > 0 ? item_nrm[0] : 0.f;
  out[0] = (m > 0.f && isfinite(m)) ? __fmul_rn(m, kFp8Inv) : 1.f;
}

__global__ void gather_rows_kernel(const float* __restrict__ x, const int32_t* __restrict__ perm,
                                   int64_t n, int f, float* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * f) return;
  int64_t r = t / f;
  int k = (int)(t - r * f);
  out[t] = x[(int64_t)perm[r] * f + k];
}

__global__ void scatter_topk_kernel(const int32_t* __restrict__ src_idx, const double* __restrict__ src_sc,
                                    const int32_t* __restrict__ rows, int64_t n, int K, int32_t* __restrict__ dst_idx,
                                    double* __restrict__ dst_sc) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n * K) return;
  const int64_t r = t / K;
  const int k = (int)(t - r * K);
  dst_idx[(int64_t)rows[r] * K + k] = src_idx[t];
  dst_sc[(int64_t)rows[r] * K + k] = src_sc[t];
}

// Work list of the item-chunked blocked multiply: work item w = c * n_ut + t
// is user tile t against item tiles [c * tpc, min(n_it, (c + 1) tpc)) into
// sub-lists 2c, 2c + 1; identity row and position maps (padding rows -1).
__global__ void bmm_chunk_work_kernel(int n_ut, int nch, int tpc, int n_it, int64_t n_users, int64_t n_items_pad,
                                      int* __restrict__ a_row, int* __restrict__ b_row, int* __restrict__ tb,
                                      int* __restrict__ te, int* __restrict__ l_base, int* __restrict__ n_work,
                                      int32_t* __restrict__ row_user, int32_t* __restrict__ item_pos) {
  const int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x, stride = (int64_t)gridDim.x * blockDim.x;
  const int64_t nw = (int64_t)n_ut * nch;
  if (i0 == 0) *n_work = (int)nw;
  for (int64_t w = i0; w < nw; w += stride) {
    const int c = (int)(w / n_ut), t = (int)(w - (int64_t)c * n_ut);
    a_row[w] = t * 128;
    b_row[w] = 0;
    tb[w] = c * tpc;
    te[w] = min(n_it, (c + 1) * tpc);
    l_base[w] = 2 * c;
  }
  for (int64_t r = i0; r < (int64_t)n_ut * 128; r += stride) row_user[r] = r < n_users ? (int32_t)r : -1;
  for (int64_t r = i0; r < n_items_pad; r += stride) item_pos[r] = (int32_t)r;
}

// Sample split keys: 0 for the users whose image (a u + b) mod n is below
// ns, 1 for the rest; ids = u.
__global__ void sample_keys_kernel(int64_t n, uint64_t a, uint64_t b, int64_t ns, uint32_t* __restrict__ keys,
                                   int32_t* __restrict__ ids) {
  const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= n) return;
  const uint64_t img = (a * (uint64_t)u + b) % (uint64_t)n;  // a, u < 2^31: no overflow
  keys[u] = img < (uint64_t)ns ? 0u : 1u;
  ids[u] = (int32_t)u;
}

}  // namespace

void launch_sample_keys(int64_t n, uint64_t a, uint64_t b, int64_t ns, uint32_t* keys, int32_t* ids, cudaStream_t s) {
  if (n <= 0) return;
  sample_keys_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, a, b, ns, keys, ids);
}

int sm_count() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 1;
  if (dev < 0 || dev >= 64) {
    int n = 1;
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 1;
  }
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
    cached[dev] = n;
  }
  return cached[dev];
}

void launch_bmm_chunks(int n_ut, int nch, int tpc, int n_it, int64_t n_users, int64_t n_items_pad, int* work5,
                       int* n_work, int32_t* row_user, int32_t* item_pos, cudaStream_t s) {
  const int64_t nw = (int64_t)n_ut * nch;
  bmm_chunk_work_kernel<<<sm_count() * 2, 256, 0, s>>>(n_ut, nch, tpc, n_it, n_users, n_items_pad, work5, work5 + nw,
                                                work5 + 2 * nw, work5 + 3 * nw, work5 + 4 * nw, n_work, row_user,
                                                item_pos);
}

void launch_scatter_topk(const int32_t* src_idx, const double* src_sc, const int32_t* rows, int64_t n, int K,
                         int32_t* dst_idx, double* dst_sc, cudaStream_t s) {
  if (n <= 0) return;
  scatter_topk_kernel<<<(unsigned)((n * K + 255) / 256), 256, 0, s>>>(src_idx, src_sc, rows, n, K, dst_idx, dst_sc);
}

void launch_row_norm_ub(const float* x, int64_t n, int f, float* nrm_ub, int* err, cudaStream_t s) {
  if (n <= 0) return;
  int wpb = 8;
  row_norm_ub_kernel<<<(unsigned)((n + wpb - 1) / wpb), wpb * 32, 0, s>>>(x, n, f, nrm_ub, err);
}

void launch_quant_bf16(const float* x, int64_t n, int f, int fp, int role, void* out_bf16,
                       int64_t n_rows_out, float2* aux, int* err, cudaStream_t s) {
  if (n_rows_out <= 0) return;
  const int64_t rows_per_block = 256 / 8;  // eight lanes per row
  quant_bf16_kernel<<<(unsigned)((n_rows_out + rows_per_block - 1) / rows_per_block), 256, 0, s>>>(
      x, n, f, fp, role, (__nv_bfloat16*)out_bf16, n_rows_out, aux, err);
}

void launch_quant_fp8(const float* x, int64_t n, int f, int fp, int role, const float* item_scale, void* out,
                      int64_t n_rows_out, float2* aux, float* row_scale, int* err, cudaStream_t s) {
  if (n_rows_out <= 0) return;
  const int64_t rows_per_block = 8 * kQuantRows;
  quant_fp8_kernel<<<(unsigned)((n_rows_out + rows_per_block - 1) / rows_per_block), 8 * 32, 0, s>>>(
      x, n, f, fp, role, item_scale, (uint8_t*)out, n_rows_out, aux, row_scale, err);
}

void launch_fp8_item_scale(const float* item_nrm, int64_t n, float* item_scale, cudaStream_t s) {
  fp8_item_scale_kernel<<<1, 32, 0, s>>>(item_nrm, n, item_scale);
}

void launch_gather_rows(const float* x, const int32_t* perm, int64_t n, int f, float* out, cudaStream_t s) {
  int64_t total = n * f;
  if (total <= 0) return;
  gather_rows_kernel<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(x, perm, n, f, out);
}

}  // namespace mips
