// Stable LSD radix sort of (uint32 key, int32 value) pairs, batched over
// equal-length segments (segment s = elements [s n, (s + 1) n)).
//
// Used for the item order of the index (items by norm, descending) and for
// Maximus' per-cluster lists (items by CBound, descending; Algorithm 1,
// ConstructIndex).  Descending float order is obtained by sorting the key
// float_desc_key(x) ascending; stability keeps equal keys in input order.
//
// Each 8-bit pass is three kernels:
//   hist    one block per (tile of 4096 elements, segment): digit counts;
//   scan    in two steps, exclusive over [digit][tile] so that a digit's
//           elements from earlier tiles come first: one warp per (segment,
//           digit) row scans that digit's tile counts and keeps the row's
//           total, then one block per segment scans its 256 totals into
//           each digit's first output slot (the scatter adds the two);
//   scatter one block per (tile, segment): 16 rounds of 256 consecutive
//           elements; within a round each element's rank among equal digits
//           comes from __match_any_sync inside its warp plus the counts of
//           the warps before it, so the order of equal digits is kept.
#include "internal.h"

namespace mips {

namespace {

constexpr int kThreads = 256;
constexpr int kPerThread = 16;
constexpr int kTile = kThreads * kPerThread;  // 4096
constexpr int kDigits = 256;

__global__ void radix_hist_kernel(const uint32_t* __restrict__ keys, int64_t n, int shift,
                                  uint32_t* __restrict__ hist, int nb) {
  __shared__ uint32_t h[kDigits];
  const int b = blockIdx.x, seg = blockIdx.y;
  for (int d = threadIdx.x; d < kDigits; d += kThreads) h[d] = 0;
  __syncthreads();
  const uint32_t* k = keys + (int64_t)seg * n;
  const int64_t lo = (int64_t)b * kTile, hi = min(n, lo + kTile);
  for (int64_t i = lo + threadIdx.x; i < hi; i += kThreads) atomicAdd(&h[(k[i] >> shift) & 0xFF], 1u);
  __syncthreads();
  for (int d = threadIdx.x; d < kDigits; d += kThreads) hist[((int64_t)seg * kDigits + d) * nb + b] = h[d];
}

// Scan, step 1: warp per (segment, digit) row of nb tile counts, in place,
// exclusive within the row; the row's total goes to totals[seg][digit].
__global__ void radix_rowscan_kernel(uint32_t* __restrict__ hist, int nb, int n_rows, uint32_t* __restrict__ totals) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);  // seg * kDigits + digit
  const int lane = threadIdx.x & 31;
  if (row >= n_rows) return;
  uint32_t* h = hist + (int64_t)row * nb;
  uint32_t carry = 0;
  for (int b0 = 0; b0 < nb; b0 += 32) {
    const int b = b0 + lane;
    const uint32_t v = b < nb ? h[b] : 0u;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (b < nb) h[b] = carry + x - v;
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  if (lane == 0) totals[row] = carry;
}

// Scan, step 2: block (kDigits threads) per segment, exclusive scan of the
// digit totals in place: each digit's first output slot in the segment.
__global__ void radix_digitscan_kernel(uint32_t* __restrict__ totals) {
  __shared__ uint32_t warp_sums[kDigits / 32];
  uint32_t* t = totals + (int64_t)blockIdx.x * kDigits;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const uint32_t v = t[threadIdx.x];
  uint32_t x = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) warp_sums[w] = x;
  __syncthreads();
  uint32_t before = 0;
  for (int ww = 0; ww < w; ++ww) before += warp_sums[ww];
  t[threadIdx.x] = before + x - v;
}

__global__ void radix_scatter_kernel(const uint32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
                                     uint32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out, int64_t n,
                                     int shift, const uint32_t* __restrict__ offsets, int nb,
                                     const uint32_t* __restrict__ digit_base) {
  __shared__ uint32_t base[kDigits];                       // next output slot per digit
  __shared__ uint16_t warp_cnt[kThreads / 32][kDigits];    // this round's per-warp digit counts
  const int b = blockIdx.x, seg = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int d = threadIdx.x; d < kDigits; d += kThreads)
    base[d] = digit_base[seg * kDigits + d] + offsets[((int64_t)seg * kDigits + d) * nb + b];
  const int64_t off = (int64_t)seg * n;
  const int64_t lo = (int64_t)b * kTile, hi = min(n, lo + kTile);
  // the per-warp counts start at zero; after each round the lanes that set
  // an entry clear it again, so no round clears the whole array
  for (int e = threadIdx.x; e < (kThreads / 32) * kDigits; e += kThreads) (&warp_cnt[0][0])[e] = 0;
  __syncthreads();
  for (int64_t r0 = lo; r0 < hi; r0 += kThreads) {
    const int64_t i = r0 + threadIdx.x;
    const bool live = i < hi;
    uint32_t key = 0;
    int32_t val = 0;
    uint32_t d = kDigits;  // dead lanes get a digit of their own
    if (live) {
      key = keys_in[off + i];
      val = vals_in[off + i];
      d = (key >> shift) & 0xFF;
    }
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const int rank = __popc(peers & ((1u << lane) - 1));
    if (live && rank == 0) warp_cnt[w][d] = (uint16_t)__popc(peers);
    __syncthreads();
    if (live) {
      uint32_t before = 0;
      for (int ww = 0; ww < w; ++ww) before += warp_cnt[ww][d];
      const uint32_t pos = base[d] + before + rank;
      keys_out[off + pos] = key;
      vals_out[off + pos] = val;
    }
    __syncthreads();
    for (int dd = threadIdx.x; dd < kDigits; dd += kThreads) {
      uint32_t t = 0;
      for (int ww = 0; ww < kThreads / 32; ++ww) t += warp_cnt[ww][dd];
      base[dd] += t;
    }
    __syncthreads();
    if (live && rank == 0) warp_cnt[w][d] = 0;  // (read by all above)
    __syncwarp();  // the warp's next-round counts land after its resets
  }
}

__global__ void float_desc_keys_kernel(const float* __restrict__ x, int64_t n, uint32_t* __restrict__ keys,
                                       int32_t* __restrict__ iota, int64_t seg_len) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  keys[i] = float_desc_key(x[i]);
  if (iota) iota[i] = (int32_t)(i % seg_len);
}

}  // namespace

size_t radix_sort_temp_bytes(int64_t n, int n_seg) {
  const int nb = (int)((n + kTile - 1) / kTile);
  return sizeof(uint32_t) * (size_t)kDigits * (nb + 1) * n_seg;  // counts [seg][digit][tile], then totals [seg][digit]
}

cudaError_t radix_sort_pairs(uint32_t*& keys, int32_t*& vals, uint32_t*& keys_alt, int32_t*& vals_alt, int64_t n,
                             int n_seg, int begin_bit, int end_bit, uint32_t* temp, cudaStream_t s, int* launches) {
  if (n <= 0 || n_seg <= 0) return cudaSuccess;
  const int nb = (int)((n + kTile - 1) / kTile);
  dim3 grid(nb, n_seg);
  const int n_rows = n_seg * kDigits;
  uint32_t* totals = temp + (size_t)n_rows * nb;
  for (int shift = begin_bit; shift < end_bit; shift += 8) {
    radix_hist_kernel<<<grid, kThreads, 0, s>>>(keys, n, shift, temp, nb);
    radix_rowscan_kernel<<<(n_rows + 7) / 8, 256, 0, s>>>(temp, nb, n_rows, totals);
    radix_digitscan_kernel<<<n_seg, kDigits, 0, s>>>(totals);
    radix_scatter_kernel<<<grid, kThreads, 0, s>>>(keys, vals, keys_alt, vals_alt, n, shift, temp, nb, totals);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (launches) *launches += 4;
    uint32_t* tk = keys;
    keys = keys_alt;
    keys_alt = tk;
    int32_t* tv = vals;
    vals = vals_alt;
    vals_alt = tv;
  }
  return cudaSuccess;
}

cudaError_t make_float_desc_keys(const float* x, int64_t n, uint32_t* keys, int32_t* iota, int64_t seg_len,
                                 cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  float_desc_keys_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(x, n, keys, iota, seg_len);
  return cudaGetLastError();
}

}  // namespace mips
