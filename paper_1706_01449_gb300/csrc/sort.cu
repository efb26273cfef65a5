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
//   scatter one block per (tile, segment): a stable sort of the tile by
//           digit in shared memory (each warp ranks a contiguous eighth of
//           the tile with __match_any_sync and its own digit counters, so
//           the order of equal digits is kept), then the sorted tile goes
//           out in runs of equal digits, each contiguous in the output.
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

// Scatter of one tile of kTile elements: a stable local sort by digit in
// shared memory, then the copy out.  Warp w owns elements [512 w, 512 w +
// 512) of the tile (lane l: 512 w + 32 r + l, r = 0..15) and ranks them in
// order with __match_any_sync and warp-private digit counters (no block
// barrier); the counters, summed over the warps in order, give every warp
// its first slot per digit.  The sorted tile holds keys and tile indices;
// the copy out reads each value by its index (the tile's values are a
// 16 KB range) and writes runs of equal digits, each contiguous in the
// output, instead of one element per 32-byte sector.
constexpr int kScatterWarps = kThreads / 32;
constexpr int kPerWarp = kTile / kScatterWarps;  // 512
static_assert(kThreads == kDigits, "the scatter's digit pass runs a thread per digit");

__global__ void __launch_bounds__(kThreads, 3)
    radix_scatter_kernel(const uint32_t* __restrict__ keys_in, const int32_t* __restrict__ vals_in,
                         uint32_t* __restrict__ keys_out, int32_t* __restrict__ vals_out, int64_t n, int shift,
                         const uint32_t* __restrict__ offsets, int nb, const uint32_t* __restrict__ digit_base) {
  __shared__ uint32_t skeys[kTile];
  __shared__ uint16_t sidx[kTile];
  __shared__ uint16_t srank[16][kThreads];          // each element's rank among its warp's equal digits
  __shared__ uint32_t cnt[kScatterWarps][kDigits];  // counts, then each warp's first tile slot per digit
  __shared__ uint32_t lbase[kDigits];               // the digit's first slot in the sorted tile
  __shared__ uint32_t gbase[kDigits];               // the digit's first output slot of this tile
  __shared__ uint32_t wsum[kScatterWarps];
  const int b = blockIdx.x, seg = blockIdx.y;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t off = (int64_t)seg * n;
  const int64_t lo = (int64_t)b * kTile;
  const int len = (int)min((int64_t)kTile, n - lo);
  for (int d = lane; d < kDigits; d += 32) cnt[w][d] = 0u;
  __syncwarp();
  uint32_t key[16];
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int i = w * kPerWarp + 32 * r + lane;
    const bool live = i < len;
    key[r] = live ? keys_in[off + lo + i] : 0u;
  }
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int i = w * kPerWarp + 32 * r + lane;
    const bool live = i < len;
    const uint32_t d = live ? (key[r] >> shift) & 0xFFu : (uint32_t)kDigits;  // dead lanes: a digit of their own
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    const unsigned below = peers & ((1u << lane) - 1u);
    const uint32_t before = live ? cnt[w][d] : 0u;  // this warp's earlier elements of digit d
    srank[r][threadIdx.x] = (uint16_t)(before + __popc(below));
    __syncwarp();
    if (live && below == 0u) cnt[w][d] = before + __popc(peers);
    __syncwarp();
  }
  __syncthreads();
  // thread d: the tile's count of digit d, an exclusive scan over the digits,
  // then the warps' first slots in warp order
  const int d = threadIdx.x;
  uint32_t tc = 0;
#pragma unroll
  for (int ww = 0; ww < kScatterWarps; ++ww) tc += cnt[ww][d];
  uint32_t x = tc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) wsum[w] = x;
  __syncthreads();
  uint32_t lb = x - tc;
  for (int ww = 0; ww < w; ++ww) lb += wsum[ww];
  lbase[d] = lb;
  gbase[d] = digit_base[seg * kDigits + d] + offsets[((int64_t)seg * kDigits + d) * nb + b];
  uint32_t run = lb;
#pragma unroll
  for (int ww = 0; ww < kScatterWarps; ++ww) {
    const uint32_t c = cnt[ww][d];
    cnt[ww][d] = run;
    run += c;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < 16; ++r) {
    const int i = w * kPerWarp + 32 * r + lane;
    if (i < len) {
      const uint32_t pos = cnt[w][(key[r] >> shift) & 0xFFu] + srank[r][threadIdx.x];
      skeys[pos] = key[r];
      sidx[pos] = (uint16_t)i;
    }
  }
  __syncthreads();
  for (int p = threadIdx.x; p < len; p += kThreads) {
    const uint32_t k = skeys[p];
    const uint32_t dd = (k >> shift) & 0xFFu;
    const int64_t q = off + (int64_t)(gbase[dd] + ((uint32_t)p - lbase[dd]));
    keys_out[q] = k;
    vals_out[q] = vals_in[off + lo + sidx[p]];
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
