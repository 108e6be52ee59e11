// Graph loading and the construction of the DAG G_pi (Sec. 1.3, Sec. 4.1).
//
//  a1  canonical keys (min << 32 | max), loops marked, radix sort, unique.
//  a2  rank check: a permutation of [0, n) or TL_EINVAL.
//  a3  relabel + orient: edge {a, b} -> (min(r_a, r_b), max(r_a, r_b)).
//  a4  radix sort by (src, dst) -> N+ CSR; stable re-sort by dst -> N- CSR.
//  a5  degrees -> C++ = sum d+^2, C+- = sum d+ d-, max degrees.
#include "graph.cuh"

namespace tl {
namespace {

constexpr uint64_t kLoop = ~0ull;
constexpr int kThreads = 256;

__global__ void k_canon(const uint32_t *__restrict__ edges, uint64_t m_in, uint32_t n,
                        uint64_t *__restrict__ keys, uint32_t *__restrict__ bad) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m_in;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t a = edges[2 * i], b = edges[2 * i + 1];
    if (a >= n || b >= n) {
      *bad = 1;
      keys[i] = kLoop;
      continue;
    }
    uint32_t lo = min(a, b), hi = max(a, b);
    keys[i] = (lo == hi) ? kLoop : ((uint64_t)lo << 32 | hi);
  }
}

// flags[i] = 1 if keys[i] starts a new distinct non-loop key (keys sorted).
__global__ void k_unique_flags(const uint64_t *__restrict__ keys, uint64_t m,
                               uint32_t *__restrict__ flags) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t k = keys[i];
    flags[i] = (k != kLoop && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
  }
}

__global__ void k_compact(const uint64_t *__restrict__ keys, const uint32_t *__restrict__ flags,
                          const uint64_t *__restrict__ pos, uint64_t m,
                          uint64_t *__restrict__ out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    if (flags[i]) out[pos[i]] = keys[i];
  }
}

__global__ void k_rank_hist(const uint32_t *__restrict__ rank, uint32_t n,
                            uint32_t *__restrict__ cnt, uint32_t *__restrict__ bad) {
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t r = rank[v];
    if (r >= n)
      *bad = 1;
    else
      atomicAdd(&cnt[r], 1u);
  }
}

__global__ void k_rank_check(const uint32_t *__restrict__ cnt, uint32_t n,
                             uint32_t *__restrict__ bad) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < n;
       r += (uint64_t)gridDim.x * blockDim.x) {
    if (cnt[r] != 1u) *bad = 1;
  }
}

__global__ void k_iota(uint32_t *__restrict__ v, uint32_t n) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
       i += (uint64_t)gridDim.x * blockDim.x)
    v[i] = (uint32_t)i;
}

__global__ void k_inverse(const uint32_t *__restrict__ rank, uint32_t n,
                          uint32_t *__restrict__ inv) {
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x)
    inv[rank[v]] = (uint32_t)v;
}

// Relabel by the ordering and orient from lower to higher rank (Sec. 1.3).
__global__ void k_orient(const uint64_t *__restrict__ E, uint64_t m,
                         const uint32_t *__restrict__ rank, uint64_t *__restrict__ keys) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t e = E[i];
    uint32_t ra = rank[(uint32_t)(e >> 32)], rb = rank[(uint32_t)e];
    uint32_t s = min(ra, rb), d = max(ra, rb);
    keys[i] = (uint64_t)s << 32 | d;
  }
}

__global__ void k_low_half(const uint64_t *__restrict__ keys, uint64_t m,
                           uint32_t *__restrict__ adj) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x)
    adj[i] = (uint32_t)keys[i];
}

__global__ void k_swap_halves(const uint64_t *__restrict__ in, uint64_t m,
                              uint64_t *__restrict__ out) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t k = in[i];
    out[i] = (k << 32) | (k >> 32);
  }
}

// CSR offsets from keys sorted by their high half: off[x] = first index whose
// high half is >= x, for x in [0, n]; off[n] = m.  One binary search per x,
// so long runs of empty rows cost nothing extra.
__global__ void k_offsets(const uint64_t *__restrict__ keys, uint64_t m, uint32_t n,
                          uint64_t *__restrict__ off) {
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x <= n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t lo = 0, hi = m;
    while (lo < hi) {
      const uint64_t mid = (lo + hi) >> 1;
      if ((keys[mid] >> 32) < x) lo = mid + 1; else hi = mid;
    }
    off[x] = lo;
  }
}

// acc[0] += sum d+^2 (C++), acc[1] += sum d+ d- (C+-), acc[2] = max d+,
// acc[3] = max d- (Definition of Sec. 3.1), acc[4] += sum d-^2 (C--, the
// cost of A--).
__global__ void k_cost(const uint64_t *__restrict__ out_off, const uint64_t *__restrict__ in_off,
                       uint32_t n, unsigned long long *__restrict__ acc) {
  unsigned long long s_pp = 0, s_pm = 0, s_mm = 0, mx_p = 0, mx_m = 0;
  for (uint64_t x = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; x < n;
       x += (uint64_t)gridDim.x * blockDim.x) {
    unsigned long long dp = out_off[x + 1] - out_off[x];
    unsigned long long dm = in_off[x + 1] - in_off[x];
    s_pp += dp * dp;
    s_pm += dp * dm;
    s_mm += dm * dm;
    mx_p = dp > mx_p ? dp : mx_p;
    mx_m = dm > mx_m ? dm : mx_m;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    s_pp += __shfl_down_sync(0xffffffffu, s_pp, d);
    s_pm += __shfl_down_sync(0xffffffffu, s_pm, d);
    s_mm += __shfl_down_sync(0xffffffffu, s_mm, d);
    unsigned long long a = __shfl_down_sync(0xffffffffu, mx_p, d);
    unsigned long long b = __shfl_down_sync(0xffffffffu, mx_m, d);
    mx_p = a > mx_p ? a : mx_p;
    mx_m = b > mx_m ? b : mx_m;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&acc[0], s_pp);
    atomicAdd(&acc[1], s_pm);
    atomicMax(&acc[2], mx_p);
    atomicMax(&acc[3], mx_m);
    atomicAdd(&acc[4], s_mm);
  }
}

// d_v of every vertex from the cleaned edge set (each key counts for both ends).
__global__ void k_degrees(const uint64_t *__restrict__ E, uint64_t m, uint32_t *__restrict__ deg) {
  for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < m;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t e = E[i];
    atomicAdd(&deg[(uint32_t)(e >> 32)], 1u);
    atomicAdd(&deg[(uint32_t)e], 1u);
  }
}

// key[v] = sort value << 32 | v, the sort value being d_v (ascending degree)
// or (2^bits - 1 - d_v) (descending degree); keys start in id order, so a
// stable sort on the high half breaks ties by increasing id.
__global__ void k_degree_keys(const uint32_t *__restrict__ deg, uint32_t n, int descending,
                              uint32_t top, uint64_t *__restrict__ keys) {
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t d = descending ? top - deg[v] : deg[v];
    keys[v] = (uint64_t)d << 32 | v;
  }
}

// Ranks from the sorted sequence: position p of vertex v gives rank p
// (degree ordering), or the Split rule of Sec. 3.3.3 on the 1-based position
// p+1 of the non-increasing degree sequence: p+1 = 2i+1 -> pi = i+1,
// p+1 = 2i -> pi = n+1-i (0-based rank = pi - 1).
__global__ void k_ranks_from_sequence(const uint64_t *__restrict__ keys, uint32_t n, int split,
                                      uint32_t *__restrict__ rank) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = (uint32_t)keys[p];
    uint64_t r = p;
    if (split) r = (p % 2 == 0) ? p / 2 : (uint64_t)n - (p + 1) / 2;
    rank[v] = (uint32_t)r;
  }
}

// Part-wise orderings of a disjoint union.  keys[p] (low half v, sorted by the
// ordering's sort value) -> part(v) << 32 | v, so that a stable sort on the
// high half groups the parts in order and keeps each part's sequence.
__global__ void k_part_keys(uint64_t *__restrict__ keys, uint32_t n,
                            const uint64_t *__restrict__ vbase, uint32_t k) {
  for (uint64_t p = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; p < n;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t v = (uint32_t)keys[p];
    uint32_t lo = 0, hi = k - 1;
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (vbase[mid] <= v) lo = mid; else hi = mid - 1;
    }
    keys[p] = (uint64_t)lo << 32 | v;
  }
}

// As k_ranks_from_sequence, within each part: the vertex at position p of
// part i's sequence (p counted from vbase[i]) gets rank vbase[i] + r(p, n_i).
__global__ void k_part_ranks(const uint64_t *__restrict__ keys, uint32_t n, int split,
                             const uint64_t *__restrict__ vbase, uint32_t *__restrict__ rank) {
  for (uint64_t q = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; q < n;
       q += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t key = keys[q];
    const uint32_t v = (uint32_t)key, part = (uint32_t)(key >> 32);
    const uint64_t b = vbase[part], np = vbase[part + 1] - b, p = q - b;
    uint64_t r = p;
    if (split) r = (p % 2 == 0) ? p / 2 : np - (p + 1) / 2;
    rank[v] = (uint32_t)(b + r);
  }
}

template <class T>
T read_scalar(const T *dev, cudaStream_t s) {
  T v;
  TL_CUDA(cudaMemcpyAsync(&v, dev, sizeof(T), cudaMemcpyDeviceToHost, s));
  TL_CUDA(cudaStreamSynchronize(s));
  return v;
}

}  // namespace

void build_edge_set(DeviceGraph &g, const uint32_t *edges, uint64_t m_in, bool on_device) {
  cudaStream_t s = g.stream;
  const uint32_t n = g.n;
  g.small.reserve(256);
  uint32_t *bad = g.small.as<uint32_t>();
  TL_CUDA(cudaMemsetAsync(bad, 0, 4, s));
  if (m_in == 0) {
    g.m = 0;
    g.E.reserve(8);
    return;
  }
  const uint32_t *dev_edges = edges;
  DevBuf staged(s);
  if (!on_device) {
    staged.reserve(m_in * 8);
    TL_CUDA(cudaMemcpyAsync(staged.p, edges, m_in * 8, cudaMemcpyHostToDevice, s));
    dev_edges = staged.as<uint32_t>();
  }
  g.keys_a.reserve(m_in * 8);
  g.keys_b.reserve(m_in * 8);
  uint64_t *ka = g.keys_a.as<uint64_t>();
  k_canon<<<grid_for(m_in, kThreads), kThreads, 0, s>>>(dev_edges, m_in, n, ka, bad);
  TL_CHECK_LAUNCH();
  if (read_scalar(bad, s)) fail(TL_EINVAL, "tl_graph_load: an edge has an id >= n");
  staged.release();
  finish_edge_set(g, m_in);
}

void finish_edge_set(DeviceGraph &g, uint64_t m_in) {
  cudaStream_t s = g.stream;
  const uint32_t n = g.n;
  uint64_t *ka = g.keys_a.as<uint64_t>(), *kb = g.keys_b.as<uint64_t>();
  const int b = bits_for(n > 1 ? n - 1 : 1);
  radix_sort_u64(ka, kb, m_in, 0, b, 32, b, g.sort_tmp, g.scan_tmp, s);
  // unique (flags in kb's storage as uint32, positions after them)
  DevBuf pos(s);
  pos.reserve((m_in + 1) * 8);
  uint32_t *flags = reinterpret_cast<uint32_t *>(kb);
  k_unique_flags<<<grid_for(m_in, kThreads), kThreads, 0, s>>>(ka, m_in, flags);
  TL_CHECK_LAUNCH();
  exclusive_scan_u32_to_u64(flags, pos.as<uint64_t>(), m_in, g.scan_tmp, s);
  const uint64_t m = read_scalar(pos.as<uint64_t>() + m_in, s);
  g.E.reserve((m ? m : 1) * 8);
  k_compact<<<grid_for(m_in, kThreads), kThreads, 0, s>>>(ka, flags, pos.as<uint64_t>(), m_in,
                                                          g.E.as<uint64_t>());
  TL_CHECK_LAUNCH();
  TL_CUDA(cudaStreamSynchronize(s));
  g.m = m;
  g.keys_a.release();
  g.keys_b.release();
  g.sort_tmp.release();
}

void csr_halves(const uint64_t *E, uint64_t m, uint32_t n, uint64_t *off_a, uint32_t *adj_a,
                uint64_t *off_b, uint32_t *adj_b, DevBuf &ka, DevBuf &kb, DevBuf &tmp,
                DevBuf &scan, cudaStream_t s) {
  if (m == 0) {
    TL_CUDA(cudaMemsetAsync(off_a, 0, ((uint64_t)n + 1) * 8, s));
    TL_CUDA(cudaMemsetAsync(off_b, 0, ((uint64_t)n + 1) * 8, s));
    return;
  }
  k_offsets<<<grid_for((uint64_t)n + 1, kThreads), kThreads, 0, s>>>(E, m, n, off_a);
  TL_CHECK_LAUNCH();
  k_low_half<<<grid_for(m, kThreads), kThreads, 0, s>>>(E, m, adj_a);
  TL_CHECK_LAUNCH();
  ka.reserve(m * 8);
  kb.reserve(m * 8);
  k_swap_halves<<<grid_for(m, kThreads), kThreads, 0, s>>>(E, m, ka.as<uint64_t>());
  TL_CHECK_LAUNCH();
  const int b = bits_for(n > 1 ? n - 1 : 1);
  radix_sort_u64(ka.as<uint64_t>(), kb.as<uint64_t>(), m, 0, 0, 32, b, tmp, scan, s);
  k_offsets<<<grid_for((uint64_t)n + 1, kThreads), kThreads, 0, s>>>(ka.as<uint64_t>(), m, n,
                                                                    off_b);
  TL_CHECK_LAUNCH();
  k_low_half<<<grid_for(m, kThreads), kThreads, 0, s>>>(ka.as<uint64_t>(), m, adj_b);
  TL_CHECK_LAUNCH();
}

bool is_permutation(const uint32_t *rank, uint32_t n, uint32_t *flag, cudaStream_t s) {
  DevBuf cnt(s);
  cnt.reserve((uint64_t)n * 4);
  TL_CUDA(cudaMemsetAsync(cnt.p, 0, (uint64_t)n * 4, s));
  TL_CUDA(cudaMemsetAsync(flag, 0, 4, s));
  k_rank_hist<<<grid_for(n, kThreads), kThreads, 0, s>>>(rank, n, cnt.as<uint32_t>(), flag);
  TL_CHECK_LAUNCH();
  k_rank_check<<<grid_for(n, kThreads), kThreads, 0, s>>>(cnt.as<uint32_t>(), n, flag);
  TL_CHECK_LAUNCH();
  return read_scalar(flag, s) == 0;
}

void build_dag(DeviceGraph &g, const uint32_t *rank, bool on_device) {
  cudaStream_t s = g.stream;
  const uint32_t n = g.n;
  const uint64_t m = g.m;
  g.small.reserve(256);
  uint32_t *bad = g.small.as<uint32_t>();
  unsigned long long *acc = reinterpret_cast<unsigned long long *>(g.small.as<char>() + 64);
  TL_CUDA(cudaMemsetAsync(g.small.p, 0, 256, s));

  // a2: the ordering must be a permutation of [0, n).
  DevBuf rank_new(s);
  rank_new.reserve((uint64_t)n * 4);
  if (rank) {
    TL_CUDA(cudaMemcpyAsync(rank_new.p, rank, (uint64_t)n * 4,
                            on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
  } else {  // the identity ordering
    k_iota<<<grid_for(n, kThreads), kThreads, 0, s>>>(rank_new.as<uint32_t>(), n);
    TL_CHECK_LAUNCH();
  }
  if (!is_permutation(rank_new.as<uint32_t>(), n, bad, s))
    fail(TL_EINVAL, "tl_order_apply: rank is not a permutation of [0, n)");

  g.rank.reserve((uint64_t)n * 4);
  g.inv.reserve((uint64_t)n * 4);
  TL_CUDA(cudaMemcpyAsync(g.rank.p, rank_new.p, (uint64_t)n * 4, cudaMemcpyDeviceToDevice, s));
  k_inverse<<<grid_for(n, kThreads), kThreads, 0, s>>>(g.rank.as<uint32_t>(), n,
                                                       g.inv.as<uint32_t>());
  TL_CHECK_LAUNCH();

  g.out_off.reserve(((uint64_t)n + 1) * 8);
  g.in_off.reserve(((uint64_t)n + 1) * 8);
  // +4 elements: the listing kernels read N+ lists with aligned 16-byte loads
  // that may extend up to 3 elements past the last list.
  g.out_adj.reserve((m + 4) * 4);
  g.in_adj.reserve((m + 4) * 4);  // scanned by A-- with the same 16-byte loads
  if (m > 0) {
    // a3: relabel + orient.
    g.keys_a.reserve(m * 8);
    g.keys_b.reserve(m * 8);
    uint64_t *ka = g.keys_a.as<uint64_t>(), *kb = g.keys_b.as<uint64_t>();
    k_orient<<<grid_for(m, kThreads), kThreads, 0, s>>>(g.E.as<uint64_t>(), m,
                                                        g.rank.as<uint32_t>(), ka);
    TL_CHECK_LAUNCH();
    // a4: sort by (src, dst) -> N+; then stable by dst -> N-.
    const int b = bits_for(n > 1 ? n - 1 : 1);
    radix_sort_u64(ka, kb, m, 0, b, 32, b, g.sort_tmp, g.scan_tmp, s);
    k_low_half<<<grid_for(m, kThreads), kThreads, 0, s>>>(ka, m, g.out_adj.as<uint32_t>());
    TL_CHECK_LAUNCH();
    k_offsets<<<grid_for((uint64_t)n + 1, kThreads), kThreads, 0, s>>>(ka, m, n,
                                                                      g.out_off.as<uint64_t>());
    TL_CHECK_LAUNCH();
    k_swap_halves<<<grid_for(m, kThreads), kThreads, 0, s>>>(ka, m, kb);
    TL_CHECK_LAUNCH();
    radix_sort_u64(kb, ka, m, 0, 0, 32, b, g.sort_tmp, g.scan_tmp, s);
    k_low_half<<<grid_for(m, kThreads), kThreads, 0, s>>>(kb, m, g.in_adj.as<uint32_t>());
    TL_CHECK_LAUNCH();
    k_offsets<<<grid_for((uint64_t)n + 1, kThreads), kThreads, 0, s>>>(kb, m, n,
                                                                      g.in_off.as<uint64_t>());
    TL_CHECK_LAUNCH();
  } else {
    TL_CUDA(cudaMemsetAsync(g.out_off.p, 0, ((uint64_t)n + 1) * 8, s));
    TL_CUDA(cudaMemsetAsync(g.in_off.p, 0, ((uint64_t)n + 1) * 8, s));
  }
  // a5: cost.
  k_cost<<<grid_for(n, kThreads), kThreads, 0, s>>>(g.out_off.as<uint64_t>(),
                                                    g.in_off.as<uint64_t>(), n, acc);
  TL_CHECK_LAUNCH();
  unsigned long long h[5];
  TL_CUDA(cudaMemcpyAsync(h, acc, sizeof(h), cudaMemcpyDeviceToHost, s));
  TL_CUDA(cudaStreamSynchronize(s));
  g.cost_app = h[0];
  g.cost_apm = h[1];
  g.cost_amm = h[4];
  g.max_out_deg = (uint32_t)h[2];
  g.max_in_deg = (uint32_t)h[3];
  g.ordered = true;
  // The sort buffers are dead until the next build; hand them back to the pool.
  g.keys_a.release();
  g.keys_b.release();
  g.sort_tmp.release();
}

}  // namespace tl

namespace tl {

void compute_order(DeviceGraph &g, int kind, uint32_t *rank, bool on_device) {
  cudaStream_t s = g.stream;
  const uint32_t n = g.n;
  DevBuf deg(s), ka(s), kb(s), out(s), tmp(s), scan(s);
  deg.reserve((uint64_t)n * 4);
  ka.reserve((uint64_t)n * 8);
  kb.reserve((uint64_t)n * 8);
  const int split = kind == TL_ORDER_SPLIT;
  if (kind == TL_ORDER_CORE) {
    // keys (round << 32 | v) of the level-synchronous peeling (core.cu)
    const uint32_t rounds = core_peel_keys(g, ka.as<uint64_t>());
    radix_sort_u64(ka.as<uint64_t>(), kb.as<uint64_t>(), n, 0, 0, 32, bits_for(rounds), tmp,
                   scan, s);
  } else {
    TL_CUDA(cudaMemsetAsync(deg.p, 0, (uint64_t)n * 4, s));
    if (g.m) {
      k_degrees<<<grid_for(g.m, kThreads), kThreads, 0, s>>>(g.E.as<uint64_t>(), g.m,
                                                             deg.as<uint32_t>());
      TL_CHECK_LAUNCH();
    }
    const int bits = bits_for(n);  // degrees are < n < 2^bits
    const uint32_t top = (uint32_t)((1ull << bits) - 1);
    k_degree_keys<<<grid_for(n, kThreads), kThreads, 0, s>>>(deg.as<uint32_t>(), n, split, top,
                                                             ka.as<uint64_t>());
    TL_CHECK_LAUNCH();
    radix_sort_u64(ka.as<uint64_t>(), kb.as<uint64_t>(), n, 0, 0, 32, bits, tmp, scan, s);
  }
  uint32_t *dst = rank;
  if (!on_device) {
    out.reserve((uint64_t)n * 4);
    dst = out.as<uint32_t>();
  }
  const uint32_t k = g.part_vbase.size() > 2 ? (uint32_t)(g.part_vbase.size() - 1) : 1;
  if (k > 1) {  // a union: the same ordering inside every part
    DevBuf vb(s);
    vb.reserve((uint64_t)(k + 1) * 8);
    TL_CUDA(cudaMemcpyAsync(vb.p, g.part_vbase.data(), (uint64_t)(k + 1) * 8,
                            cudaMemcpyHostToDevice, s));
    k_part_keys<<<grid_for(n, kThreads), kThreads, 0, s>>>(ka.as<uint64_t>(), n,
                                                           vb.as<uint64_t>(), k);
    TL_CHECK_LAUNCH();
    radix_sort_u64(ka.as<uint64_t>(), kb.as<uint64_t>(), n, 0, 0, 32, bits_for(k - 1), tmp, scan,
                   s);
    k_part_ranks<<<grid_for(n, kThreads), kThreads, 0, s>>>(ka.as<uint64_t>(), n, split,
                                                            vb.as<uint64_t>(), dst);
    TL_CHECK_LAUNCH();
    TL_CUDA(cudaStreamSynchronize(s));  // vb is read by the kernels above
  } else {
    k_ranks_from_sequence<<<grid_for(n, kThreads), kThreads, 0, s>>>(ka.as<uint64_t>(), n,
                                                                     split, dst);
    TL_CHECK_LAUNCH();
  }
  if (!on_device)
    TL_CUDA(cudaMemcpyAsync(rank, dst, (uint64_t)n * 4, cudaMemcpyDeviceToHost, s));
  TL_CUDA(cudaStreamSynchronize(s));
}

}  // namespace tl
