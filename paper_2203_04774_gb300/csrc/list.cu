// Triangle listing: Algorithm 1 (A++) and Algorithm 2 (A+-) of Sec. 2.1.
//
// Both algorithms have the same shape once the "B vertex" x is fixed:
//   A++: x = w, probe set P_x = N-_w, scanned lists N+_y for y in P_x.
//   A+-: x = u, probe set P_x = N+_u, scanned lists N+_y for y in P_x.
// For every y in P_x and every z in N+_y, z in P_x reports triangle {x, y, z}
// (A++: u=y, v=z, w=x; A+-: u=x, v=y, w=z).  The number of membership tests
// is sum_{y in P_x} d+_y per x; summed over x it is C++ resp. C+- (Property 1).
//
// Work decomposition (a6).  Seed edge k = (x, y_k) is the k-th entry of the
// probe-side CSR; it owns the d+(y_k) work items [WP[k], WP[k+1]) of a global
// exclusive prefix WP.  Vertices with |P_x| <= 32 and little work are "small":
// a warp holds P_x in registers (one element per lane) and probes by binary
// search over the lanes.  The others are "large": a CTA holds P_x in shared
// memory (a bitmap over all ranks when n is small enough -- literally the
// boolean array B of Algorithms 1 and 2 -- else an open-addressing hash) and
// its work range is cut into pieces of at most kPieceWork items.
//
// Output (a9).  A CTA appends its triangles, as sorted original ids, to a
// private slab; at the end of a task it reserves room in the current output
// chunk with one atomic and copies the slab there.  If the chunk is full the
// task is queued for the next launch (after the consumer has drained the
// chunk) and nothing of it is written, so every chunk holds whole tasks and
// the listing resumes exactly where it stopped.
#include "list.cuh"

namespace tl {
namespace {

constexpr uint32_t kNone = 0xffffffffu;

__device__ __forceinline__ void sort3(uint32_t &a, uint32_t &b, uint32_t &c) {
  uint32_t t;
  if (a > b) t = a, a = b, b = t;
  if (b > c) t = b, b = c, c = t;
  if (a > b) t = a, a = b, b = t;
}

// Number of lanes j with v_j <= key (0..32), for v sorted ascending across
// the warp.  The five halving steps reach at most 31; the last lane is
// checked on its own.
__device__ __forceinline__ int warp_count_le(uint32_t v, uint32_t key) {
  int pos = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    uint32_t e = __shfl_sync(0xffffffffu, v, pos + step - 1);
    if (e <= key) pos += step;
  }
  const uint32_t last = __shfl_sync(0xffffffffu, v, 31);
  if (pos == 31 && last <= key) pos = 32;
  return pos;
}

// Task fetch shared by both kernels: returns the task id or -1.  Thread 0
// only; the caller broadcasts.
__device__ __forceinline__ int64_t fetch_task(ListCtl *ctl, const ListArgs &a) {
  if (*(volatile uint32_t *)&ctl->overflow) return -1;
  uint32_t idx = atomicAdd(&ctl->fetch, 1u);
  if (idx < a.n_retry) return a.retry_in[idx];
  uint64_t t = a.fresh_base + (idx - a.n_retry);
  return (t < a.n_tasks) ? (int64_t)t : -1;
}

// End of a task: reserve chunk room for the slab, copy it, or queue the task.
__device__ void commit_task(ListCtl *ctl, const ListArgs &a, int64_t t, const uint32_t *slab,
                            uint32_t cnt, unsigned long long probes, uint32_t *s_ok,
                            unsigned long long *s_pos) {
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t ok = 1;
    unsigned long long pos = 0;
    if (cnt > 0) {
      pos = atomicAdd(&ctl->cursor, (unsigned long long)cnt);
      if (pos + cnt > a.chunk_cap) ok = 0;
    }
    if (ok) {
      if (cnt > 0) {
        atomicMax(&ctl->valid_end, pos + cnt);
        atomicAdd(&ctl->triangles, (unsigned long long)cnt);
      }
      atomicAdd(&ctl->probes, probes);
    } else {
      atomicExch(&ctl->overflow, 1u);
      uint32_t r = atomicAdd(&ctl->n_retry_out, 1u);
      a.retry_out[r] = (uint32_t)t;
    }
    *s_ok = ok;
    *s_pos = pos;
  }
  __syncthreads();
  if (*s_ok && cnt > 0) {
    uint32_t *dst = a.chunk + 3ull * (*s_pos);
    const uint32_t words = 3u * cnt;
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) dst[i] = slab[i];
  }
  __syncthreads();
}

// ---- small vertices: one warp per x, P_x in registers ------------------------

__device__ __forceinline__ void list_small_x(const ListArgs &a, uint32_t x, uint32_t *slab,
                                             uint32_t *s_cnt, unsigned long long &probes) {
  const int lane = threadIdx.x & 31;
  const uint64_t pb = a.poff[x];
  const int p = (int)(a.poff[x + 1] - pb);
  const uint32_t P = (lane < p) ? a.padj[pb + lane] : kNone;  // ascending, padded
  uint32_t len = 0, invP = 0;
  uint64_t st = 0;
  if (lane < p) {
    st = a.out_off[P];
    len = (uint32_t)(a.out_off[P + 1] - st);
    invP = a.inv[P];
  }
  uint32_t end = len;  // inclusive scan of the scanned-list lengths
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    uint32_t o = __shfl_up_sync(0xffffffffu, end, d);
    if (lane >= d) end += o;
  }
  const uint32_t beg = end - len;
  const uint32_t W = __shfl_sync(0xffffffffu, end, 31);
  const uint32_t inv_x = a.inv[x];
  const unsigned lt = (1u << lane) - 1u;
  for (uint32_t base = 0; base < W; base += 32) {
    const uint32_t i = base + lane;
    const bool act = i < W;
    int seg = warp_count_le(end, i);  // first segment whose end > i
    seg = seg > 31 ? 31 : seg;
    const uint32_t sb = __shfl_sync(0xffffffffu, beg, seg);
    const uint64_t ss = __shfl_sync(0xffffffffu, st, seg);
    const uint32_t iy = __shfl_sync(0xffffffffu, invP, seg);
    uint32_t z = act ? a.out_adj[ss + (i - sb)] : 0u;
    const int q = warp_count_le(P, z);
    const uint32_t pz = __shfl_sync(0xffffffffu, P, q > 0 ? q - 1 : 0);
    const bool hit = act && q > 0 && pz == z;
    probes += act ? 1 : 0;
    const unsigned hm = __ballot_sync(0xffffffffu, hit);
    if (hm) {
      uint32_t basepos = 0;
      const int leader = __ffs(hm) - 1;
      if (lane == leader) basepos = atomicAdd(s_cnt, (uint32_t)__popc(hm));
      basepos = __shfl_sync(0xffffffffu, basepos, leader);
      if (hit) {
        uint32_t t0 = inv_x, t1 = iy, t2 = a.inv[z];
        sort3(t0, t1, t2);
        uint32_t r = basepos + __popc(hm & lt);
        slab[3 * r + 0] = t0;
        slab[3 * r + 1] = t1;
        slab[3 * r + 2] = t2;
      }
    }
  }
}

__device__ __forceinline__ uint64_t lower_bound_u64(const uint64_t *v, uint64_t n, uint64_t key) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (v[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ uint64_t upper_bound_u64(const uint64_t *v, uint64_t n, uint64_t key) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (v[mid] <= key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void __launch_bounds__(kSmallThreads) k_list_small(ListArgs a) {
  __shared__ int64_t s_t;
  __shared__ uint32_t s_x0, s_x1, s_next, s_cnt, s_ok;
  __shared__ unsigned long long s_pos, s_probes;
  uint32_t *slab = a.slabs + (uint64_t)blockIdx.x * a.slab_cap * 3;
  const int lane = threadIdx.x & 31;
  for (;;) {
    if (threadIdx.x == 0) {
      int64_t t = fetch_task(a.ctl, a);
      s_t = t;
      if (t >= 0) {
        // task t covers the small x whose work prefix lies in [t, t+1) * kSmallWork
        const uint64_t nr = a.x_end - a.x_begin;
        uint64_t r0 = lower_bound_u64(a.small_prefix, nr + 1, (uint64_t)t * kSmallWork);
        uint64_t r1 = lower_bound_u64(a.small_prefix, nr + 1, (uint64_t)(t + 1) * kSmallWork);
        s_x0 = a.x_begin + (uint32_t)(r0 < nr ? r0 : nr);
        s_x1 = a.x_begin + (uint32_t)(r1 < nr ? r1 : nr);
        s_next = s_x0;
        s_cnt = 0;
        s_probes = 0;
      }
    }
    __syncthreads();
    const int64_t t = s_t;
    if (t < 0) break;
    const uint32_t x1 = s_x1;
    unsigned long long probes = 0;
    for (;;) {
      uint32_t x = 0;
      if (lane == 0) x = atomicAdd(&s_next, 1u);
      x = __shfl_sync(0xffffffffu, x, 0);
      if (x >= x1) break;
      const uint64_t r = x - a.x_begin;
      if (a.small_prefix[r + 1] == a.small_prefix[r]) continue;  // not small (or no work)
      list_small_x(a, x, slab, &s_cnt, probes);
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) probes += __shfl_down_sync(0xffffffffu, probes, d);
    if (lane == 0) atomicAdd(&s_probes, probes);
    __syncthreads();
    commit_task(a.ctl, a, t, slab, s_cnt, s_probes, &s_ok, &s_pos);
  }
}

// ---- large vertices: one CTA per piece, P_x in shared memory -----------------

__device__ __forceinline__ uint32_t hash_slot(uint32_t r, uint32_t mask) {
  return (r * 0x9E3779B1u) & mask;
}

__global__ void __launch_bounds__(kLargeThreads, 1) k_list_large(ListArgs a) {
  extern __shared__ uint32_t sm[];  // bitmap or hash table
  __shared__ int64_t s_t;
  __shared__ uint32_t s_x, s_cnt, s_ok, s_mode, s_mask;
  __shared__ unsigned long long s_pos, s_probes, s_a, s_b;
  __shared__ uint64_t s_k0;
  uint32_t *slab = a.slabs + (uint64_t)blockIdx.x * a.slab_cap * 3;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nwarps = blockDim.x >> 5;
  const bool use_bitmap = a.n <= kBitmapMaxN;
  if (use_bitmap) {
    const uint32_t words = (a.n + 31) >> 5;
    for (uint32_t i = threadIdx.x; i < words; i += blockDim.x) sm[i] = 0;
  }
  const unsigned lt = (1u << lane) - 1u;
  for (;;) {
    if (threadIdx.x == 0) {
      int64_t t = fetch_task(a.ctl, a);
      s_t = t;
      if (t >= 0) {
        // x = the vertex whose piece range contains t
        const uint64_t nr = a.x_end - a.x_begin;
        uint64_t r = upper_bound_u64(a.piece_prefix, nr + 1, (uint64_t)t) - 1;
        const uint32_t x = a.x_begin + (uint32_t)r;
        const uint64_t piece = (uint64_t)t - a.piece_prefix[r];
        const uint64_t pb = a.poff[x], pe = a.poff[x + 1];
        const uint64_t w0 = a.WP[pb], w1 = a.WP[pe];
        const uint64_t ia = w0 + piece * kPieceWork;
        const uint64_t ib = (ia + kPieceWork < w1) ? ia + kPieceWork : w1;
        s_x = x;
        s_a = ia;
        s_b = ib;
        // first seed edge whose item range reaches past ia
        s_k0 = pb + upper_bound_u64(a.WP + pb, pe - pb, ia) - 1;
        s_cnt = 0;
        s_probes = 0;
        const uint64_t p = pe - pb;
        if (use_bitmap) {
          s_mode = 0;
        } else {
          uint32_t cap = 64;
          while (cap < 2 * p && cap < kHashMaxSlots) cap <<= 1;
          if (2 * p <= cap) {
            s_mode = 1;
            s_mask = cap - 1;
          } else {
            s_mode = 2;  // probe set too large for shared memory: binary search
          }
        }
      }
    }
    __syncthreads();
    const int64_t t = s_t;
    if (t < 0) break;
    const uint32_t x = s_x;
    const uint64_t pb = a.poff[x], pe = a.poff[x + 1];
    const uint32_t mode = s_mode, mask = s_mask;
    // build B: the probe set P_x
    if (mode == 0) {
      for (uint64_t k = pb + threadIdx.x; k < pe; k += blockDim.x) {
        uint32_t r = a.padj[k];
        atomicOr(&sm[r >> 5], 1u << (r & 31));
      }
    } else if (mode == 1) {
      for (uint32_t i = threadIdx.x; i <= mask; i += blockDim.x) sm[i] = kNone;
      __syncthreads();
      for (uint64_t k = pb + threadIdx.x; k < pe; k += blockDim.x) {
        uint32_t r = a.padj[k];
        uint32_t h = hash_slot(r, mask);
        while (atomicCAS(&sm[h], kNone, r) != kNone) h = (h + 1) & mask;
      }
    }
    __syncthreads();
    const uint64_t ia = s_a, ib = s_b;
    const uint32_t inv_x = a.inv[x];
    unsigned long long probes = 0;
    for (uint64_t k = s_k0 + wid; k < pe; k += nwarps) {
      const uint64_t wk = a.WP[k];
      if (wk >= ib) break;
      const uint64_t wk1 = a.WP[k + 1];
      const uint32_t y = a.padj[k];
      const uint64_t st = a.out_off[y];
      const uint64_t lo = (ia > wk ? ia : wk) - wk;
      const uint64_t hi = (ib < wk1 ? ib : wk1) - wk;
      const uint32_t iy = a.inv[y];
      for (uint64_t base = lo; base < hi; base += 32) {
        const uint64_t pos = base + lane;
        const bool act = pos < hi;
        bool hit = false;
        uint32_t z = 0;
        if (act) {
          z = a.out_adj[st + pos];
          ++probes;
          if (mode == 0) {
            hit = (sm[z >> 5] >> (z & 31)) & 1u;
          } else if (mode == 1) {
            uint32_t h = hash_slot(z, mask);
            for (;;) {
              uint32_t v = sm[h];
              if (v == z) { hit = true; break; }
              if (v == kNone) break;
              h = (h + 1) & mask;
            }
          } else {
            uint64_t lo2 = pb, hi2 = pe;
            while (lo2 < hi2) {
              uint64_t mid = (lo2 + hi2) >> 1;
              if (a.padj[mid] < z) lo2 = mid + 1; else hi2 = mid;
            }
            hit = lo2 < pe && a.padj[lo2] == z;
          }
        }
        const unsigned hm = __ballot_sync(0xffffffffu, hit);
        if (hm) {
          uint32_t basepos = 0;
          const int leader = __ffs(hm) - 1;
          if (lane == leader) basepos = atomicAdd(&s_cnt, (uint32_t)__popc(hm));
          basepos = __shfl_sync(0xffffffffu, basepos, leader);
          if (hit) {
            uint32_t t0 = inv_x, t1 = iy, t2 = a.inv[z];
            sort3(t0, t1, t2);
            uint32_t r = basepos + __popc(hm & lt);
            slab[3 * r + 0] = t0;
            slab[3 * r + 1] = t1;
            slab[3 * r + 2] = t2;
          }
        }
      }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) probes += __shfl_down_sync(0xffffffffu, probes, d);
    if (lane == 0) atomicAdd(&s_probes, probes);
    __syncthreads();
    // reset B
    if (mode == 0) {
      for (uint64_t k = pb + threadIdx.x; k < pe; k += blockDim.x) sm[a.padj[k] >> 5] = 0;
    }
    commit_task(a.ctl, a, t, slab, s_cnt, s_probes, &s_ok, &s_pos);
  }
}

// ---- bucketize (a6) -----------------------------------------------------------

// w[k] = d+(y_k) for every probe-side CSR entry k.
__global__ void k_seed_work(const uint32_t *__restrict__ padj, uint64_t m,
                            const uint64_t *__restrict__ out_off, uint32_t *__restrict__ w) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t y = padj[k];
    w[k] = (uint32_t)(out_off[y + 1] - out_off[y]);
  }
}

// Per x in the range: small work (W_x if small, else 0) and piece count (if
// large, else 0).
__global__ void k_classify(const uint64_t *__restrict__ poff, const uint64_t *__restrict__ WP,
                           uint32_t x_begin, uint32_t x_end, uint64_t *__restrict__ small_w,
                           uint64_t *__restrict__ pieces) {
  const uint64_t nr = x_end - x_begin;
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < nr;
       r += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = x_begin + (uint32_t)r;
    const uint64_t pb = poff[x], pe = poff[x + 1];
    const uint64_t W = WP[pe] - WP[pb];
    const uint64_t p = pe - pb;
    uint64_t sw = 0, np = 0;
    if (p > 0 && W > 0) {
      if (p <= 32 && W <= kSmallWork)
        sw = W;
      else
        np = (W + kPieceWork - 1) / kPieceWork;
    }
    small_w[r] = sw;
    pieces[r] = np;
  }
}

// ---- count + hash consumer ---------------------------------------------------

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void k_count_hash(const uint32_t *__restrict__ t, uint64_t n,
                             unsigned long long *__restrict__ acc) {
  const uint64_t G = 0x9e3779b97f4a7c15ull;
  unsigned long long h = 0;
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t v = mix64((uint64_t)t[3 * i] + G);
    v = mix64(v + (uint64_t)t[3 * i + 1] + G);
    v = mix64(v + (uint64_t)t[3 * i + 2] + G);
    h += v;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) h += __shfl_down_sync(0xffffffffu, h, d);
  if ((threadIdx.x & 31) == 0) atomicAdd(acc, h);
}

}  // namespace

// ---- host side ----------------------------------------------------------------

void launch_seed_work(const uint32_t *padj, uint64_t m, const uint64_t *out_off, uint32_t *w,
                      cudaStream_t s) {
  k_seed_work<<<grid_for(m, 256), 256, 0, s>>>(padj, m, out_off, w);
  TL_CHECK_LAUNCH();
}

void launch_classify(const uint64_t *poff, const uint64_t *WP, uint32_t x_begin, uint32_t x_end,
                     uint64_t *small_w, uint64_t *pieces, cudaStream_t s) {
  k_classify<<<grid_for((uint64_t)(x_end - x_begin), 256), 256, 0, s>>>(poff, WP, x_begin, x_end,
                                                                        small_w, pieces);
  TL_CHECK_LAUNCH();
}

int small_grid() {
  static int g = 0;
  if (!g) {
    int per_sm = 0;
    TL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_list_small, kSmallThreads, 0));
    g = num_sms() * (per_sm > 0 ? per_sm : 1);
  }
  return g;
}

int large_grid() {
  static int g = 0;
  if (!g) {
    TL_CUDA(cudaFuncSetAttribute(k_list_large, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kLargeSmemBytes));
    int per_sm = 0;
    TL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_list_large, kLargeThreads,
                                                          kLargeSmemBytes));
    g = num_sms() * (per_sm > 0 ? per_sm : 1);
  }
  return g;
}

void launch_list(int kind, const ListArgs &a, cudaStream_t s) {
  if (kind == 0) {
    k_list_small<<<small_grid(), kSmallThreads, 0, s>>>(a);
  } else {
    large_grid();
    k_list_large<<<large_grid(), kLargeThreads, kLargeSmemBytes, s>>>(a);
  }
  TL_CHECK_LAUNCH();
}

void launch_count_hash(const uint32_t *t, uint64_t n, unsigned long long *acc, cudaStream_t s) {
  if (n == 0) return;
  k_count_hash<<<grid_for(n, 256), 256, 0, s>>>(t, n, acc);
  TL_CHECK_LAUNCH();
}

}  // namespace tl
