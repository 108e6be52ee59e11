// The core ordering on the device (Sec. 1.3: the coreness c_v is the largest k
// such that v belongs to a subgraph of minimum degree k; the core ordering
// lists vertices by non-decreasing coreness, and the paper obtains it by
// repeatedly removing a vertex of minimum degree, Batagelj and Zaversnik).
//
// Level-synchronous peeling: at level k, every remaining vertex of degree <= k
// is removed in round r; removing it lowers its neighbours' degrees, and those
// that fall to k are removed in round r+1, and so on until none is left at
// level k; then k grows to the smallest remaining degree.  A vertex removed at
// level k has coreness k.  Vertices are ordered by (round, id); rounds grow
// with the levels, so coreness is non-decreasing along the ordering, and a
// vertex has at most k neighbours removed in its round or later (its degree
// when it was taken), hence d+_v <= c_v: the degeneracy property of the
// sequential peeling.  Ties differ from the sequential algorithm (a whole
// round is removed at once, by increasing id).
#include <vector>

#include "graph.cuh"

namespace tl {
namespace {

constexpr int kThreads = 256;

// Warp-aggregated slot reservation: returns this lane's slot when pred holds.
// All 32 lanes must call it.
__device__ __forceinline__ uint32_t warp_reserve(bool pred, uint32_t *counter) {
  const unsigned mask = __ballot_sync(0xffffffffu, pred);
  const int lane = threadIdx.x & 31;
  uint32_t base = 0;
  if (lane == 0 && mask) base = atomicAdd(counter, (uint32_t)__popc(mask));
  base = __shfl_sync(0xffffffffu, base, 0);
  return base + __popc(mask & ((1u << lane) - 1u));
}

// Undirected degree from the two CSR halves (N+ and N- of the identity order).
__global__ void k_core_degrees(const uint64_t *__restrict__ off_a,
                               const uint64_t *__restrict__ off_b, uint32_t n,
                               uint32_t *__restrict__ deg, uint32_t *__restrict__ active) {
  for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n;
       v += (uint64_t)gridDim.x * blockDim.x) {
    deg[v] = (uint32_t)((off_a[v + 1] - off_a[v]) + (off_b[v + 1] - off_b[v]));
    active[v] = (uint32_t)v;
  }
}

// Level start: the remaining vertices of degree <= k are removed now (frontier);
// the others stay (rest), and cnt[2] gets the smallest degree among them.
// cnt = {frontier size, rest size, min rest degree}.
__global__ void k_core_select(const uint32_t *__restrict__ active, uint32_t na,
                              const uint32_t *__restrict__ deg, uint32_t *__restrict__ removed,
                              uint32_t k, uint32_t *__restrict__ frontier,
                              uint32_t *__restrict__ rest, uint32_t *__restrict__ cnt) {
  const uint32_t stride = gridDim.x * blockDim.x;
  for (uint32_t base = blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < na;
       base += stride) {
    const uint32_t i = base + (threadIdx.x & 31);
    bool take = false, keep = false;
    uint32_t v = 0, d = 0;
    if (i < na) {
      v = active[i];
      if (!removed[v]) {
        d = deg[v];
        take = d <= k;
        keep = !take;
      }
    }
    if (take) removed[v] = 1;
    const uint32_t pf = warp_reserve(take, cnt);
    const uint32_t pr = warp_reserve(keep, cnt + 1);
    if (take) frontier[pf] = v;
    if (keep) {
      rest[pr] = v;
      atomicMin(cnt + 2, d);
    }
  }
}

// One round: a warp per frontier vertex v records key (round, v) and lowers
// the degree of each neighbour not yet removed; a neighbour whose degree
// falls from k+1 to k joins the next frontier (exactly once: one atomicSub
// sees k+1).
__global__ void k_core_peel(const uint32_t *__restrict__ frontier, uint32_t nf,
                            const uint64_t *__restrict__ off_a, const uint32_t *__restrict__ adj_a,
                            const uint64_t *__restrict__ off_b, const uint32_t *__restrict__ adj_b,
                            uint32_t *__restrict__ deg, uint32_t *__restrict__ removed,
                            uint64_t *__restrict__ key, uint32_t round, uint32_t k,
                            uint32_t *__restrict__ next, uint32_t *__restrict__ ncount) {
  const int lane = threadIdx.x & 31;
  const uint32_t warps = gridDim.x * (blockDim.x / 32);
  for (uint32_t w = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); w < nf; w += warps) {
    const uint32_t v = frontier[w];
    if (lane == 0) key[v] = (uint64_t)round << 32 | v;
    for (int half = 0; half < 2; ++half) {
      const uint64_t *off = half ? off_b : off_a;
      const uint32_t *adj = half ? adj_b : adj_a;
      const uint64_t b = off[v], e = off[v + 1];
      for (uint64_t j0 = b; j0 < e; j0 += 32) {
        const uint64_t j = j0 + lane;
        bool app = false;
        uint32_t u = 0;
        if (j < e) {
          u = adj[j];
          if (!*(volatile uint32_t *)(removed + u)) {
            const uint32_t old = atomicSub(deg + u, 1u);
            if (old == k + 1) {
              removed[u] = 1;
              app = true;
            }
          }
        }
        const uint32_t pos = warp_reserve(app, ncount);
        if (app) next[pos] = u;
      }
    }
  }
}

struct PinnedCounters {
  uint32_t *h = nullptr;
  PinnedCounters() { TL_CUDA(cudaMallocHost(&h, 16)); }
  ~PinnedCounters() {
    if (h) cudaFreeHost(h);
  }
};

}  // namespace

// Fills keys[v] = (round << 32 | v) for every vertex; returns the number of
// rounds.  The identity-order CSR halves are built from E here.
uint32_t core_peel_keys(DeviceGraph &g, uint64_t *keys) {
  cudaStream_t s = g.stream;
  const uint32_t n = g.n;
  const uint64_t m = g.m;
  DevBuf off_a(s), adj_a(s), off_b(s), adj_b(s), ka(s), kb(s), tmp(s), scan(s);
  off_a.reserve(((uint64_t)n + 1) * 8);
  off_b.reserve(((uint64_t)n + 1) * 8);
  adj_a.reserve((m ? m : 1) * 4);
  adj_b.reserve((m ? m : 1) * 4);
  csr_halves(g.E.as<uint64_t>(), m, n, off_a.as<uint64_t>(), adj_a.as<uint32_t>(),
             off_b.as<uint64_t>(), adj_b.as<uint32_t>(), ka, kb, tmp, scan, s);
  ka.release();
  kb.release();
  DevBuf deg(s), removed(s), act0(s), act1(s), fr0(s), fr1(s), cnt(s);
  for (DevBuf *b : {&deg, &removed, &act0, &act1, &fr0, &fr1}) b->reserve((uint64_t)n * 4);
  cnt.reserve(16);
  TL_CUDA(cudaMemsetAsync(removed.p, 0, (uint64_t)n * 4, s));
  k_core_degrees<<<grid_for(n, kThreads), kThreads, 0, s>>>(
      off_a.as<uint64_t>(), off_b.as<uint64_t>(), n, deg.as<uint32_t>(), act0.as<uint32_t>());
  TL_CHECK_LAUNCH();
  PinnedCounters hc;
  uint32_t *active = act0.as<uint32_t>(), *rest = act1.as<uint32_t>();
  uint32_t *front = fr0.as<uint32_t>(), *next = fr1.as<uint32_t>();
  uint32_t *dc = cnt.as<uint32_t>();
  uint32_t na = n, k = 0, round = 0;
  const uint32_t init[4] = {0, 0, 0xffffffffu, 0};
  while (na > 0) {
    TL_CUDA(cudaMemcpyAsync(dc, init, 16, cudaMemcpyHostToDevice, s));
    k_core_select<<<grid_for(na, kThreads), kThreads, 0, s>>>(active, na, deg.as<uint32_t>(),
                                                              removed.as<uint32_t>(), k, front,
                                                              rest, dc);
    TL_CHECK_LAUNCH();
    TL_CUDA(cudaMemcpyAsync(hc.h, dc, 16, cudaMemcpyDeviceToHost, s));
    TL_CUDA(cudaStreamSynchronize(s));
    uint32_t nf = hc.h[0];
    const uint32_t nr = hc.h[1], min_rest = hc.h[2];
    std::swap(active, rest);
    na = nr;
    if (nf == 0) {  // no vertex at this level: jump to the smallest remaining degree
      if (na > 0) k = min_rest > k ? min_rest : k + 1;
      continue;
    }
    while (nf > 0) {
      TL_CUDA(cudaMemsetAsync(dc + 3, 0, 4, s));
      const unsigned blocks = grid_for((uint64_t)nf * 32, kThreads);
      k_core_peel<<<blocks, kThreads, 0, s>>>(front, nf, off_a.as<uint64_t>(),
                                              adj_a.as<uint32_t>(), off_b.as<uint64_t>(),
                                              adj_b.as<uint32_t>(), deg.as<uint32_t>(),
                                              removed.as<uint32_t>(), keys, round, k, next,
                                              dc + 3);
      TL_CHECK_LAUNCH();
      ++round;
      TL_CUDA(cudaMemcpyAsync(hc.h + 3, dc + 3, 4, cudaMemcpyDeviceToHost, s));
      TL_CUDA(cudaStreamSynchronize(s));
      nf = hc.h[3];
      std::swap(front, next);
    }
    ++k;
  }
  TL_CUDA(cudaStreamSynchronize(s));
  return round;
}

}  // namespace tl
