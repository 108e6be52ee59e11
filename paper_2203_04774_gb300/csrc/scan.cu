// Exclusive prefix sums (reduce-then-scan over tiles of 4096 elements).
#include "common.cuh"

namespace tl {
namespace {

constexpr int kScanThreads = 256;
constexpr int kScanItems = 16;
constexpr int kScanTile = kScanThreads * kScanItems;

__device__ __forceinline__ uint64_t warp_incl_scan(uint64_t v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint64_t o = __shfl_up_sync(0xffffffffu, v, d);
    if (lane >= d) v += o;
  }
  return v;
}

// Exclusive scan of one value per thread across the block; returns the
// exclusive prefix and writes the block total to *total.
__device__ __forceinline__ uint64_t block_excl_scan(uint64_t v, uint64_t *total) {
  __shared__ uint64_t warp_sums[kScanThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint64_t incl = warp_incl_scan(v);
  if (lane == 31) warp_sums[wid] = incl;
  __syncthreads();
  if (wid == 0) {
    uint64_t w = (lane < kScanThreads / 32) ? warp_sums[lane] : 0;
    uint64_t wi = warp_incl_scan(w);
    if (lane < kScanThreads / 32) warp_sums[lane] = wi - w;
    if (lane == kScanThreads / 32 - 1) *total = wi;
  }
  __syncthreads();
  return warp_sums[wid] + incl - v;
}

template <class T>
__global__ void __launch_bounds__(kScanThreads) k_tile_reduce(const T *__restrict__ in, uint64_t n,
                                                               uint64_t *__restrict__ partial) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    uint64_t idx = base + (uint64_t)i * kScanThreads + threadIdx.x;
    if (idx < n) s += (uint64_t)in[idx];
  }
  __shared__ uint64_t tot;
  uint64_t excl = block_excl_scan(s, &tot);
  (void)excl;
  __syncthreads();
  if (threadIdx.x == 0) partial[blockIdx.x] = tot;
}

// Tile element j lives at tile[pad(j)], one spare word after every 16: a
// thread's 16 consecutive elements then start 17 words apart, so its
// row-wise accesses hit distinct banks instead of one.
__device__ __forceinline__ int pad(int j) { return j + (j >> 4); }

template <class T>
__global__ void __launch_bounds__(kScanThreads)
    k_tile_scan(const T *__restrict__ in, uint64_t *__restrict__ out, uint64_t n,
                const uint64_t *__restrict__ tile_offset) {
  __shared__ uint64_t tile[kScanTile + kScanTile / 16];
  const uint64_t base = (uint64_t)blockIdx.x * kScanTile;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    uint64_t idx = base + (uint64_t)i * kScanThreads + threadIdx.x;
    tile[pad(i * kScanThreads + threadIdx.x)] = (idx < n) ? (uint64_t)in[idx] : 0;
  }
  __syncthreads();
  uint64_t v[kScanItems];
  uint64_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = tile[pad(threadIdx.x * kScanItems + i)];
    s += v[i];
  }
  __shared__ uint64_t tot;
  uint64_t run = block_excl_scan(s, &tot) + (tile_offset ? tile_offset[blockIdx.x] : 0);
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    tile[pad(threadIdx.x * kScanItems + i)] = run;
    run += v[i];
  }
  // out[n] = grand total, written by the thread holding element n-1.
  {
    uint64_t first = base + (uint64_t)threadIdx.x * kScanItems;
    if (n - 1 >= first && n - 1 < first + kScanItems) {
      int i = (int)(n - 1 - first);
      out[n] = tile[pad(threadIdx.x * kScanItems + i)] + v[i];
    }
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    uint64_t idx = base + (uint64_t)i * kScanThreads + threadIdx.x;
    if (idx < n) out[idx] = tile[pad(i * kScanThreads + threadIdx.x)];
  }
}

// Scratch (in uint64 words) needed to scan n elements.
uint64_t scan_scratch_words(uint64_t n) {
  uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles <= 1) return 0;
  return 2 * tiles + 1 + scan_scratch_words(tiles);
}

template <class T>
void scan_impl(const T *in, uint64_t *out, uint64_t n, uint64_t *scratch, cudaStream_t s) {
  if (n == 0) {
    TL_CUDA(cudaMemsetAsync(out, 0, sizeof(uint64_t), s));
    return;
  }
  uint64_t tiles = (n + kScanTile - 1) / kScanTile;
  if (tiles == 1) {
    k_tile_scan<T><<<1, kScanThreads, 0, s>>>(in, out, n, nullptr);
    TL_CHECK_LAUNCH();
    return;
  }
  // tile sums, their own scan (recursively), then the tile scans.
  uint64_t *partial = scratch;
  uint64_t *scanned = partial + tiles;
  k_tile_reduce<T><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, n, partial);
  TL_CHECK_LAUNCH();
  scan_impl<uint64_t>(partial, scanned, tiles, scanned + tiles + 1, s);
  k_tile_scan<T><<<(unsigned)tiles, kScanThreads, 0, s>>>(in, out, n, scanned);
  TL_CHECK_LAUNCH();
}

}  // namespace

void exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, DevBuf &tmp,
                        cudaStream_t s) {
  tmp.reserve(8 * (scan_scratch_words(n) + 1));
  scan_impl<uint64_t>(in, out, n, tmp.as<uint64_t>(), s);
}

void exclusive_scan_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t n, DevBuf &tmp,
                               cudaStream_t s) {
  tmp.reserve(8 * (scan_scratch_words(n) + 1));
  scan_impl<uint32_t>(in, out, n, tmp.as<uint64_t>(), s);
}

int bits_for(uint64_t v) {
  int b = 1;
  while (b < 64 && (v >> b)) ++b;
  return b;
}

}  // namespace tl
