// Stable LSD radix sort of uint64 keys, 8-bit digits.
//
// One pass = three launches: per-tile digit histograms, an exclusive scan of
// the digit-major histogram table, and a stable scatter in which each tile
// ranks its keys (warp match + per-warp digit counters, so equal digits keep
// their input order), reorders them in shared memory and writes runs of
// equal digits to their global offsets.
#include "common.cuh"

namespace tl {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 16;                         // keys per thread
constexpr int kSortTile = kSortThreads * kSortItems;   // 4096 keys per tile
constexpr int kRadix = 256;

__global__ void __launch_bounds__(kSortThreads)
    k_digit_hist(const uint64_t *__restrict__ keys, uint64_t n, int shift,
                 uint32_t *__restrict__ counts, uint32_t ntiles) {
  __shared__ uint32_t h[kRadix];
  for (int i = threadIdx.x; i < kRadix; i += kSortThreads) h[i] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
#pragma unroll 4
  for (int i = 0; i < kSortItems; ++i) {
    uint64_t idx = base + (uint64_t)i * kSortThreads + threadIdx.x;
    if (idx < n) atomicAdd(&h[(keys[idx] >> shift) & 0xFF], 1u);
  }
  __syncthreads();
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads)
    counts[(uint64_t)d * ntiles + blockIdx.x] = h[d];
}

// Three blocks per SM (at most 85 registers, no spills): two, at 99
// registers, left the memory pipe idle half the time.
__global__ void __launch_bounds__(kSortThreads, 3)
    k_scatter(const uint64_t *__restrict__ src, uint64_t *__restrict__ dst, uint64_t n,
              int shift, const uint64_t *__restrict__ offsets, uint32_t ntiles) {
  __shared__ uint32_t whist[kSortWarps][kRadix];  // per-warp counts, then offsets
  __shared__ uint32_t tile_start[kRadix];
  __shared__ uint64_t gbase[kRadix];
  __shared__ uint64_t sorted[kSortTile];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const uint64_t base = (uint64_t)blockIdx.x * kSortTile;
  for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads)
    (&whist[0][0])[i] = 0;
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads)
    gbase[d] = offsets[(uint64_t)d * ntiles + blockIdx.x];
  __syncthreads();

  // Warp w owns tile keys [w*512, (w+1)*512), read 32 at a time in order.
  uint64_t key[kSortItems];
  uint32_t rank[kSortItems];
  const unsigned lt_mask = (1u << lane) - 1u;
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    uint64_t idx = base + (uint64_t)wid * (32 * kSortItems) + it * 32 + lane;
    bool valid = idx < n;
    key[it] = valid ? src[idx] : 0;
    uint32_t d = valid ? (uint32_t)((key[it] >> shift) & 0xFF) : (0x100u + lane);
    unsigned peers = __match_any_sync(0xffffffffu, d);
    uint32_t before = 0;
    if (valid) before = whist[wid][d];
    __syncwarp();
    if (valid && (peers & lt_mask) == 0) whist[wid][d] = before + __popc(peers);
    __syncwarp();
    rank[it] = before + __popc(peers & lt_mask);
  }
  __syncthreads();
  // Per digit: exclusive scan over warps; digit totals -> tile_start.
  for (int d = threadIdx.x; d < kRadix; d += kSortThreads) {
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
      uint32_t c = whist[w][d];
      whist[w][d] = run;
      run += c;
    }
    tile_start[d] = run;  // total for now
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    // exclusive scan of the 256 digit totals by one warp (8 per lane)
    uint32_t v[8], s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      v[j] = tile_start[lane * 8 + j];
      s += v[j];
    }
    uint32_t incl = s;
#pragma unroll
    for (int dd = 1; dd < 32; dd <<= 1) {
      uint32_t o = __shfl_up_sync(0xffffffffu, incl, dd);
      if (lane >= dd) incl += o;
    }
    uint32_t run = incl - s;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      tile_start[lane * 8 + j] = run;
      run += v[j];
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < kSortItems; ++it) {
    uint64_t idx = base + (uint64_t)wid * (32 * kSortItems) + it * 32 + lane;
    if (idx < n) {
      uint32_t d = (uint32_t)((key[it] >> shift) & 0xFF);
      sorted[tile_start[d] + whist[wid][d] + rank[it]] = key[it];
    }
  }
  __syncthreads();
  const uint64_t valid_in_tile = (n - base < (uint64_t)kSortTile) ? (n - base) : kSortTile;
  for (uint32_t j = threadIdx.x; j < valid_in_tile; j += kSortThreads) {
    uint64_t k = sorted[j];
    uint32_t d = (uint32_t)((k >> shift) & 0xFF);
    dst[gbase[d] + (j - tile_start[d])] = k;
  }
}

}  // namespace

uint64_t *radix_sort_u64_impl(uint64_t *a, uint64_t *b, uint64_t n, int lo_bit, int lo_bits,
                              int hi_bit, int hi_bits, DevBuf &tmp, DevBuf &scan_tmp,
                              cudaStream_t s) {
  if (n <= 1) return a;
  const uint64_t ntiles64 = (n + kSortTile - 1) / kSortTile;
  if (ntiles64 > 0x7fffffffULL) fail(TL_EINVAL, "radix sort: too many keys");
  const uint32_t ntiles = (uint32_t)ntiles64;
  const uint64_t entries = (uint64_t)kRadix * ntiles;
  // tmp layout: counts (u32, entries) | offsets (u64, entries + 1) | scan scratch
  size_t counts_bytes = ((entries * 4 + 255) / 256) * 256;
  size_t offs_bytes = ((8 * (entries + 1) + 255) / 256) * 256;
  DevBuf &buf = tmp;
  buf.reserve(counts_bytes + offs_bytes);
  uint32_t *counts = buf.as<uint32_t>();
  uint64_t *offsets = reinterpret_cast<uint64_t *>(buf.as<char>() + counts_bytes);
  uint64_t *src = a, *dst = b;
  auto pass = [&](int shift) {
    k_digit_hist<<<ntiles, kSortThreads, 0, s>>>(src, n, shift, counts, ntiles);
    TL_CHECK_LAUNCH();
    exclusive_scan_u32_to_u64(counts, offsets, entries, scan_tmp, s);
    k_scatter<<<ntiles, kSortThreads, 0, s>>>(src, dst, n, shift, offsets, ntiles);
    TL_CHECK_LAUNCH();
    uint64_t *t = src;
    src = dst;
    dst = t;
  };
  for (int sh = lo_bit; sh < lo_bit + lo_bits; sh += 8) pass(sh);
  for (int sh = hi_bit; sh < hi_bit + hi_bits; sh += 8) pass(sh);
  return src;
}

void radix_sort_u64(uint64_t *keys, uint64_t *alt, uint64_t n, int lo_bit, int lo_bits,
                    int hi_bit, int hi_bits, DevBuf &tmp, DevBuf &scan_tmp, cudaStream_t s) {
  uint64_t *r =
      radix_sort_u64_impl(keys, alt, n, lo_bit, lo_bits, hi_bit, hi_bits, tmp, scan_tmp, s);
  if (r != keys) TL_CUDA(cudaMemcpyAsync(keys, r, n * sizeof(uint64_t), cudaMemcpyDeviceToDevice, s));
}

}  // namespace tl
