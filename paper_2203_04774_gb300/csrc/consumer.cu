// The device count + set-hash consumers (tl_count_hash, tl_count_hash_parts):
//   H = sum over triples of h(a, b, c) mod 2^64,
//   h(a, b, c) = mix(mix(mix(a + G) + b + G) + c + G),
// G = 0x9e3779b97f4a7c15, mix = the splitmix64 finaliser (Steele, Lea and
// Flood, OOPSLA 2014).  The sum does not depend on the order of the triples.
#include "hash.cuh"
#include "list.cuh"

namespace tl {
namespace {

// Four triples (48 bytes, three 16-byte loads) per thread when the buffer is
// 16-byte aligned; the remainder one by one.
__global__ void k_count_hash(const uint32_t *__restrict__ t, uint64_t n,
                             unsigned long long *__restrict__ acc) {
  unsigned long long h = 0;
  const uint64_t tid = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
  const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
  const bool aligned = (reinterpret_cast<uintptr_t>(t) & 15) == 0;
  const uint64_t groups = aligned ? n / 4 : 0;
  const uint4 *t4 = reinterpret_cast<const uint4 *>(t);
  for (uint64_t gi = tid; gi < groups; gi += stride) {
    const uint4 p = __ldcs(t4 + 3 * gi), q = __ldcs(t4 + 3 * gi + 1), r = __ldcs(t4 + 3 * gi + 2);
    h += triple_hash(p.x, p.y, p.z) + triple_hash(p.w, q.x, q.y) + triple_hash(q.z, q.w, r.x) +
         triple_hash(r.y, r.z, r.w);
  }
  for (uint64_t i = 4 * groups + tid; i < n; i += stride)
    h += triple_hash(t[3 * i], t[3 * i + 1], t[3 * i + 2]);
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) h += __shfl_down_sync(0xffffffffu, h, d);
  if ((threadIdx.x & 31) == 0) atomicAdd(acc, h);
}

// Per-part count and set hash of a disjoint union's triples: a triple's part
// is the one whose vertex range [vbase[p], vbase[p+1]) holds its ids, and it is
// hashed with part-local ids, so a part's (count, H) is the one it has alone.
// Each warp walks a contiguous range of the chunk (triples of one task, hence
// of one part, are contiguous) and keeps running sums while the part stays
// the same, adding them to the part's counters only when the part changes
// and at the end of its range.
__global__ void k_count_hash_parts(const uint32_t *__restrict__ t, uint64_t n,
                                   const uint64_t *__restrict__ vbase, uint32_t k,
                                   unsigned long long *__restrict__ counts,
                                   unsigned long long *__restrict__ hashes) {
  const int lane = threadIdx.x & 31;
  const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x >> 5);
  const uint64_t w = blockIdx.x * (uint64_t)(blockDim.x >> 5) + (threadIdx.x >> 5);
  const uint64_t per = ((n + warps - 1) / warps + 31) & ~31ull;
  const uint64_t r0 = w * per, r1 = r0 + per < n ? r0 + per : n;
  uint32_t cur = 0xffffffffu;  // the part of the running sums (the same in every lane)
  unsigned long long acc_c = 0, acc_h = 0;
  auto flush = [&]() {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
      acc_c += __shfl_down_sync(0xffffffffu, acc_c, d);
      acc_h += __shfl_down_sync(0xffffffffu, acc_h, d);
    }
    if (lane == 0 && cur != 0xffffffffu && acc_c) {
      atomicAdd(counts + cur, acc_c);
      atomicAdd(hashes + cur, acc_h);
    }
    acc_c = acc_h = 0;
  };
  for (uint64_t b = r0; b < r1; b += 32) {
    const uint64_t i = b + lane;
    const bool valid = i < r1;
    uint32_t p = 0xffffffffu;
    unsigned long long h = 0;
    if (valid) {
      const uint32_t a = __ldcs(t + 3 * i), bb = __ldcs(t + 3 * i + 1), c = __ldcs(t + 3 * i + 2);
      uint32_t lo = 0, hi = k - 1;
      while (lo < hi) {
        const uint32_t mid = (lo + hi + 1) >> 1;
        if (__ldg(vbase + mid) <= a) lo = mid; else hi = mid - 1;
      }
      p = lo;
      const uint32_t o = (uint32_t)__ldg(vbase + p);
      h = triple_hash(a - o, bb - o, c - o);
    }
    const uint32_t p0 = __shfl_sync(0xffffffffu, p, 0);
    if (__all_sync(0xffffffffu, !valid || p == p0)) {
      if (p0 != cur) {
        flush();
        cur = p0;
      }
      acc_c += valid ? 1 : 0;
      acc_h += h;
    } else {  // a part boundary inside these 32 triples
      flush();
      cur = 0xffffffffu;
      if (valid) {
        atomicAdd(counts + p, 1ull);
        atomicAdd(hashes + p, h);
      }
    }
  }
  flush();
}

}  // namespace

void launch_count_hash(const uint32_t *t, uint64_t n, unsigned long long *acc, cudaStream_t s) {
  if (n == 0) return;
  k_count_hash<<<grid_for(n, 256), 256, 0, s>>>(t, n, acc);
  TL_CHECK_LAUNCH();
}

void launch_count_hash_parts(const uint32_t *t, uint64_t n, const uint64_t *vbase, uint32_t k,
                             unsigned long long *counts, unsigned long long *hashes,
                             cudaStream_t s) {
  if (n == 0) return;
  k_count_hash_parts<<<grid_for(n, 256), 256, 0, s>>>(t, n, vbase, k, counts, hashes);
  TL_CHECK_LAUNCH();
}

}  // namespace tl
