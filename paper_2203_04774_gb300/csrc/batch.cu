// Disjoint unions of graphs: many independent listing problems as one.
//
// No edge joins two parts, so every triangle of the union lies inside one part
// and the union's triangles are exactly the parts' triangles (Sec. 1.3: a
// triangle is three pairwise adjacent vertices).  Part i's vertex v is the
// union's vertex vbase[i] + v and its rank vbase[i] + rank_i[v]; the relative
// order of a part's vertices -- hence its DAG G_pi, its N+ / N- lists and its
// costs C++ and C+- (Sec. 3.1) -- is the part's own.  One build and one
// listing pass then serve all parts, whatever their number.
//
// The tables below are indexed by element (edge or vertex): part p holds the
// elements [base[p], base[p+1]).  A block of kTile elements finds the range of
// parts it spans once, then each thread binary-searches inside that range.
#include <vector>

#include "graph.cuh"

namespace tl {
namespace {

constexpr uint64_t kLoopKey = ~0ull;
constexpr int kThreads = 256;
constexpr int kTile = 2048;  // elements per block (8 per thread)

// Largest p in [lo, hi] with base[p] <= j.
__device__ __forceinline__ uint32_t part_of(const uint64_t *__restrict__ base, uint32_t lo,
                                            uint32_t hi, uint64_t j) {
  while (lo < hi) {
    const uint32_t mid = (lo + hi + 1) >> 1;
    if (__ldg(base + mid) <= j) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// The parts spanned by this block's tile [t0, t1) (t0 < t1 <= total).
__device__ __forceinline__ void tile_parts(const uint64_t *__restrict__ base, uint32_t k,
                                           uint64_t t0, uint64_t t1, uint32_t *s_lo,
                                           uint32_t *s_hi) {
  if (threadIdx.x == 0) {
    const uint32_t lo = part_of(base, 0, k - 1, t0);
    *s_lo = lo;
    *s_hi = part_of(base, lo, k - 1, t1 - 1);
  }
  __syncthreads();
}

// Canonical keys of concatenated part edge lists: ids are checked against the
// part's size, shifted by the part's vertex base, and loops become kLoopKey.
__global__ void k_parts_canon(const uint32_t *__restrict__ edges, uint64_t total, uint32_t k,
                              const uint64_t *__restrict__ ebase,
                              const uint64_t *__restrict__ vbase, uint64_t *__restrict__ keys,
                              uint32_t *__restrict__ bad) {
  __shared__ uint32_t s_lo, s_hi;
  const uint64_t t0 = (uint64_t)blockIdx.x * kTile;
  const uint64_t t1 = min(total, t0 + kTile);
  tile_parts(ebase, k, t0, t1, &s_lo, &s_hi);
  for (uint64_t j = t0 + threadIdx.x; j < t1; j += kThreads) {
    const uint32_t p = part_of(ebase, s_lo, s_hi, j);
    const uint64_t v0 = __ldg(vbase + p), np = __ldg(vbase + p + 1) - v0;
    const uint32_t a = edges[2 * j], b = edges[2 * j + 1];
    if (a >= np || b >= np) {
      *bad = 1;
      keys[j] = kLoopKey;
      continue;
    }
    const uint64_t lo = v0 + min(a, b), hi = v0 + max(a, b);
    keys[j] = (lo == hi) ? kLoopKey : (lo << 32 | hi);
  }
}

// E of the union: part p's (sorted) keys shifted by its vertex base; the
// concatenation in part order is sorted again.
__global__ void k_union_keys(const uint64_t *const *__restrict__ src, uint64_t total, uint32_t k,
                             const uint64_t *__restrict__ ebase,
                             const uint64_t *__restrict__ vbase, uint64_t *__restrict__ out) {
  __shared__ uint32_t s_lo, s_hi;
  const uint64_t t0 = (uint64_t)blockIdx.x * kTile;
  const uint64_t t1 = min(total, t0 + kTile);
  tile_parts(ebase, k, t0, t1, &s_lo, &s_hi);
  for (uint64_t j = t0 + threadIdx.x; j < t1; j += kThreads) {
    const uint32_t p = part_of(ebase, s_lo, s_hi, j);
    const uint64_t v0 = __ldg(vbase + p);
    out[j] = src[p][j - __ldg(ebase + p)] + (v0 << 32 | v0);
  }
}

// Ranks of the union: vbase[p] + rank_p[v] (identity where rank_p is null).
__global__ void k_union_ranks(const uint32_t *const *__restrict__ src, uint64_t total, uint32_t k,
                              const uint64_t *__restrict__ vbase, uint32_t *__restrict__ out) {
  __shared__ uint32_t s_lo, s_hi;
  const uint64_t t0 = (uint64_t)blockIdx.x * kTile;
  const uint64_t t1 = min(total, t0 + kTile);
  tile_parts(vbase, k, t0, t1, &s_lo, &s_hi);
  for (uint64_t j = t0 + threadIdx.x; j < t1; j += kThreads) {
    const uint32_t p = part_of(vbase, s_lo, s_hi, j);
    const uint64_t v0 = __ldg(vbase + p);
    const uint32_t *r = src[p];
    out[j] = (uint32_t)(v0 + (r ? r[j - v0] : (uint32_t)(j - v0)));
  }
}

// CSR offsets of the union: out[j] = ebase[p] + src[p][j - vbase[p]] for the
// part p holding vertex j (the entry off[n] is written by the host).
__global__ void k_union_offsets(const uint64_t *const *__restrict__ src, uint64_t total,
                                uint32_t k, const uint64_t *__restrict__ vbase,
                                const uint64_t *__restrict__ ebase, uint64_t *__restrict__ out) {
  __shared__ uint32_t s_lo, s_hi;
  const uint64_t t0 = (uint64_t)blockIdx.x * kTile;
  const uint64_t t1 = min(total, t0 + kTile);
  tile_parts(vbase, k, t0, t1, &s_lo, &s_hi);
  for (uint64_t j = t0 + threadIdx.x; j < t1; j += kThreads) {
    const uint32_t p = part_of(vbase, s_lo, s_hi, j);
    out[j] = __ldg(ebase + p) + src[p][j - __ldg(vbase + p)];
  }
}

// CSR lists of the union: out[j] = vbase[p] + src[p][j - ebase[p]] (ranks
// shifted into the part's range) for the part p holding entry j.
__global__ void k_union_adj(const uint32_t *const *__restrict__ src, uint64_t total, uint32_t k,
                            const uint64_t *__restrict__ ebase, const uint64_t *__restrict__ vbase,
                            uint32_t *__restrict__ out) {
  __shared__ uint32_t s_lo, s_hi;
  const uint64_t t0 = (uint64_t)blockIdx.x * kTile;
  const uint64_t t1 = min(total, t0 + kTile);
  tile_parts(ebase, k, t0, t1, &s_lo, &s_hi);
  for (uint64_t j = t0 + threadIdx.x; j < t1; j += kThreads) {
    const uint32_t p = part_of(ebase, s_lo, s_hi, j);
    out[j] = (uint32_t)__ldg(vbase + p) + src[p][j - __ldg(ebase + p)];
  }
}

template <class T>
T read_back(const T *dev, cudaStream_t s) {
  T v;
  TL_CUDA(cudaMemcpyAsync(&v, dev, sizeof(T), cudaMemcpyDeviceToHost, s));
  TL_CUDA(cudaStreamSynchronize(s));
  return v;
}

unsigned tiles(uint64_t total) { return (unsigned)((total + kTile - 1) / kTile); }

// Exclusive prefix of k sizes into k+1 entries; total must fit `limit`.
std::vector<uint64_t> prefix(uint32_t k, const uint64_t *sizes, uint64_t limit, const char *what) {
  std::vector<uint64_t> b(k + 1, 0);
  for (uint32_t i = 0; i < k; ++i) {
    b[i + 1] = b[i] + sizes[i];
    if (b[i + 1] > limit || b[i + 1] < b[i]) fail(TL_EINVAL, what);
  }
  return b;
}

}  // namespace

void build_edge_set_parts(DeviceGraph &g, uint32_t k, const uint32_t *n, const uint64_t *m_in,
                          const uint32_t *edges, bool on_device) {
  cudaStream_t s = g.stream;
  std::vector<uint64_t> nv(n, n + k);
  const std::vector<uint64_t> vb = prefix(k, nv.data(), 0xfffffffeull,
                                          "the parts hold more than 2^32 - 2 vertices");
  const std::vector<uint64_t> eb = prefix(k, m_in, ~0ull >> 4, "too many edges");
  g.n = (uint32_t)vb[k];
  g.part_vbase = vb;
  const uint64_t total = eb[k];
  g.small.reserve(256);
  uint32_t *bad = g.small.as<uint32_t>();
  TL_CUDA(cudaMemsetAsync(bad, 0, 4, s));
  if (total == 0) {
    g.m = 0;
    g.E.reserve(8);
    TL_CUDA(cudaStreamSynchronize(s));
    return;
  }
  DevBuf table(s), staged(s);
  table.reserve((2 * (uint64_t)k + 2) * 8);
  uint64_t *d_vb = table.as<uint64_t>(), *d_eb = d_vb + (k + 1);
  TL_CUDA(cudaMemcpyAsync(d_vb, vb.data(), (k + 1) * 8, cudaMemcpyHostToDevice, s));
  TL_CUDA(cudaMemcpyAsync(d_eb, eb.data(), (k + 1) * 8, cudaMemcpyHostToDevice, s));
  const uint32_t *dev_edges = edges;
  if (!on_device) {
    staged.reserve(total * 8);
    TL_CUDA(cudaMemcpyAsync(staged.p, edges, total * 8, cudaMemcpyHostToDevice, s));
    dev_edges = staged.as<uint32_t>();
  }
  g.keys_a.reserve(total * 8);
  g.keys_b.reserve(total * 8);
  k_parts_canon<<<tiles(total), kThreads, 0, s>>>(dev_edges, total, k, d_eb, d_vb,
                                                  g.keys_a.as<uint64_t>(), bad);
  TL_CHECK_LAUNCH();
  if (read_back(bad, s)) fail(TL_EINVAL, "tl_graph_load_parts: an edge has an id >= its part's n");
  staged.release();
  table.release();
  finish_edge_set(g, total);
}

namespace {

// The union of parts that all hold their DAG under the ordering to use:
// every array of the union is the parts' arrays concatenated, vertex ids and
// ranks shifted by vbase and list offsets by ebase; the costs add up.  Moves
// about 32 bytes per edge, against a full relabel-and-sort for build_dag.
void union_of_dags(DeviceGraph &u, uint32_t k, const DeviceGraph *const *parts,
                   const std::vector<uint64_t> &vb, const std::vector<uint64_t> &eb) {
  cudaStream_t s = u.stream;
  const uint32_t n = u.n;
  const uint64_t m = u.m;
  // table: vbase | ebase | pointers: E, rank, inv, out_off, in_off, out_adj, in_adj
  constexpr int kPtr = 7;
  std::vector<const void *> ptr((size_t)kPtr * k);
  uint64_t cpp = 0, cpm = 0, cmm = 0;
  uint32_t mxo = 0, mxi = 0;
  for (uint32_t i = 0; i < k; ++i) {
    const DeviceGraph &g = *parts[i];
    const void *p[kPtr] = {g.E.p, g.rank.p, g.inv.p, g.out_off.p, g.in_off.p, g.out_adj.p,
                           g.in_adj.p};
    for (int j = 0; j < kPtr; ++j) ptr[(size_t)j * k + i] = p[j];
    cpp += g.cost_app;
    cpm += g.cost_apm;
    cmm += g.cost_amm;
    mxo = g.max_out_deg > mxo ? g.max_out_deg : mxo;
    mxi = g.max_in_deg > mxi ? g.max_in_deg : mxi;
  }
  DevBuf table(s);
  table.reserve((2 * (uint64_t)k + 2 + (uint64_t)kPtr * k) * 8);
  uint64_t *d_vb = table.as<uint64_t>(), *d_eb = d_vb + (k + 1);
  const void **d_ptr = reinterpret_cast<const void **>(d_eb + (k + 1));
  TL_CUDA(cudaMemcpyAsync(d_vb, vb.data(), (k + 1) * 8, cudaMemcpyHostToDevice, s));
  TL_CUDA(cudaMemcpyAsync(d_eb, eb.data(), (k + 1) * 8, cudaMemcpyHostToDevice, s));
  TL_CUDA(cudaMemcpyAsync(d_ptr, ptr.data(), ptr.size() * 8, cudaMemcpyHostToDevice, s));
  auto col = [&](int j) { return d_ptr + (size_t)j * k; };
  u.E.reserve((m ? m : 1) * 8);
  u.rank.reserve((uint64_t)n * 4);
  u.inv.reserve((uint64_t)n * 4);
  u.out_off.reserve(((uint64_t)n + 1) * 8);
  u.in_off.reserve(((uint64_t)n + 1) * 8);
  u.out_adj.reserve((m + 4) * 4);
  u.in_adj.reserve((m + 4) * 4);
  if (m) {
    k_union_keys<<<tiles(m), kThreads, 0, s>>>(
        reinterpret_cast<const uint64_t *const *>(col(0)), m, k, d_eb, d_vb, u.E.as<uint64_t>());
    TL_CHECK_LAUNCH();
    for (int j = 5; j <= 6; ++j) {
      k_union_adj<<<tiles(m), kThreads, 0, s>>>(
          reinterpret_cast<const uint32_t *const *>(col(j)), m, k, d_eb, d_vb,
          (j == 5 ? u.out_adj : u.in_adj).as<uint32_t>());
      TL_CHECK_LAUNCH();
    }
  }
  for (int j = 1; j <= 2; ++j) {
    k_union_ranks<<<tiles(n), kThreads, 0, s>>>(reinterpret_cast<const uint32_t *const *>(col(j)),
                                                n, k, d_vb,
                                                (j == 1 ? u.rank : u.inv).as<uint32_t>());
    TL_CHECK_LAUNCH();
  }
  for (int j = 3; j <= 4; ++j) {
    uint64_t *off = (j == 3 ? u.out_off : u.in_off).as<uint64_t>();
    k_union_offsets<<<tiles(n), kThreads, 0, s>>>(
        reinterpret_cast<const uint64_t *const *>(col(j)), n, k, d_vb, d_eb, off);
    TL_CHECK_LAUNCH();
    TL_CUDA(cudaMemcpyAsync(off + n, &eb[k], 8, cudaMemcpyHostToDevice, s));
  }
  TL_CUDA(cudaStreamSynchronize(s));  // the host tables outlive their copies
  u.cost_app = cpp;
  u.cost_apm = cpm;
  u.cost_amm = cmm;
  u.max_out_deg = mxo;
  u.max_in_deg = mxi;
  u.ordered = true;
}

}  // namespace

void build_union(DeviceGraph &u, uint32_t k, const DeviceGraph *const *parts,
                 const uint32_t *const *rank) {
  cudaStream_t s = u.stream;
  std::vector<uint64_t> nv(k), mv(k);
  std::vector<const void *> esrc(k), rsrc(k);
  for (uint32_t i = 0; i < k; ++i) {
    nv[i] = parts[i]->n;
    mv[i] = parts[i]->m;
    esrc[i] = parts[i]->E.p;
    rsrc[i] = rank && rank[i] ? rank[i] : (parts[i]->ordered ? parts[i]->rank.p : nullptr);
  }
  const std::vector<uint64_t> vb = prefix(k, nv.data(), 0xfffffffeull,
                                          "the parts hold more than 2^32 - 2 vertices");
  const std::vector<uint64_t> eb = prefix(k, mv.data(), ~0ull >> 4, "too many edges");
  u.n = (uint32_t)vb[k];
  u.m = eb[k];
  bool dags = true;  // every part holds its DAG and keeps its ordering
  for (uint32_t i = 0; i < k && dags; ++i)
    dags = parts[i]->ordered && !(rank && rank[i]);
  if (dags) {
    union_of_dags(u, k, parts, vb, eb);
    u.part_vbase = vb;
    return;
  }
  // table: vbase[k+1] | ebase[k+1] | E pointers[k] | rank pointers[k]
  DevBuf table(s), rank_u(s);
  table.reserve((4 * (uint64_t)k + 2) * 8);
  uint64_t *d_vb = table.as<uint64_t>(), *d_eb = d_vb + (k + 1);
  const void **d_esrc = reinterpret_cast<const void **>(d_eb + (k + 1));
  const void **d_rsrc = d_esrc + k;
  TL_CUDA(cudaMemcpyAsync(d_vb, vb.data(), (k + 1) * 8, cudaMemcpyHostToDevice, s));
  TL_CUDA(cudaMemcpyAsync(d_eb, eb.data(), (k + 1) * 8, cudaMemcpyHostToDevice, s));
  TL_CUDA(cudaMemcpyAsync(d_esrc, esrc.data(), k * 8, cudaMemcpyHostToDevice, s));
  TL_CUDA(cudaMemcpyAsync(d_rsrc, rsrc.data(), k * 8, cudaMemcpyHostToDevice, s));
  u.E.reserve((u.m ? u.m : 1) * 8);
  if (u.m) {
    k_union_keys<<<tiles(u.m), kThreads, 0, s>>>(
        reinterpret_cast<const uint64_t *const *>(d_esrc), u.m, k, d_eb, d_vb,
        u.E.as<uint64_t>());
    TL_CHECK_LAUNCH();
  }
  rank_u.reserve((uint64_t)u.n * 4);
  k_union_ranks<<<tiles(u.n), kThreads, 0, s>>>(reinterpret_cast<const uint32_t *const *>(d_rsrc),
                                                 u.n, k, d_vb, rank_u.as<uint32_t>());
  TL_CHECK_LAUNCH();
  // The pageable host tables above must outlive their copies.
  TL_CUDA(cudaStreamSynchronize(s));
  // The union's rank is a permutation of [0, n) iff every part's is one of
  // [0, n_i): values below vbase[i+1] can only come from parts 0..i.
  build_dag(u, rank_u.as<uint32_t>(), true);
  u.part_vbase = vb;
}

}  // namespace tl
