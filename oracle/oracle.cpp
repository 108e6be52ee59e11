// CPU oracle for triangle listing with a given vertex ordering
// (Lecuyer, Jachiet, Magnien, Tabourier, arXiv:2203.04774).
//
// TEST INFRASTRUCTURE ONLY.  This file is a plain, slow, obviously correct
// restatement of the paper, used to check the CUDA path.  Only the test
// suite, the smoke check of __graft_entry__ and the CPU-baseline leg of
// bench.py may load it.  It shares no code, header or constant with the
// CUDA library: the hash below is written out again from its definition.
//
// Every function cites the passage it follows:
//   * graph model, ordering, DAG G_pi, N+ / N-, d+ / d-   : Sec. 1.3
//   * cleaning (loops removed, directions merged)         : Sec. 4.1
//   * Algorithm 1 (A++, "L+n") and Algorithm 2 (A+-, "S1+n"): Sec. 2.1
//   * Property 1 (operation counts)                       : Sec. 2.1
//   * cost C++ and C+- (Definition, "Cost induced by an ordering"): Sec. 3.1
//   * mere-listing task (ordering given)                  : Sec. 3.2
//
// Readings where the paper leaves a choice open:
//   * rank[v] = pi_v - 1 (0-based) instead of the 1-based pi of Sec. 1.3.
//   * A triangle is reported as its three ORIGINAL vertex ids sorted
//     a < b < c; the set of triangles is unique, their order is not.
//   * "probes" counts executions of the test "if B[v]" (Algorithm 1) or
//     "if B[w]" (Algorithm 2); Property 1 says this equals C++ resp. C+-.
//     The m set and m reset operations on B are counted separately.
//   * Set hash of a triangle set (not in the paper; an order-independent
//     checksum for large outputs):  H = sum over triangles of
//     h(a,b,c) = mix(mix(mix(a + G) + b + G) + c + G)  (mod 2^64), where
//     G = 0x9e3779b97f4a7c15 and mix is the splitmix64 finaliser (Steele,
//     Lea and Flood, OOPSLA 2014).
//
// Plain C++17 and the standard library only.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <utility>
#include <vector>

namespace {

constexpr uint64_t kGolden = 0x9e3779b97f4a7c15ULL;

uint64_t mix(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
  return z ^ (z >> 31);
}

uint64_t triple_hash(uint32_t a, uint32_t b, uint32_t c) {
  uint64_t t = mix(uint64_t(a) + kGolden);
  t = mix(t + uint64_t(b) + kGolden);
  return mix(t + uint64_t(c) + kGolden);
}

struct Graph {
  uint32_t n = 0;
  // Undirected simple edge set E as pairs (a, b), a < b, original ids.
  std::vector<std::pair<uint32_t, uint32_t>> E;
  // Ordering and the DAG G_pi in rank space (Sec. 1.3).
  std::vector<uint32_t> rank;  // rank[v] = pi_v - 1
  std::vector<uint32_t> inv;   // inv[rank[v]] = v
  // N+_x (successors of rank x) = out_adj[out_off[x] .. out_off[x+1]),
  // N-_x (predecessors) = in_adj[in_off[x] .. in_off[x+1]), each ascending.
  // Exact-size arrays, so that a graph of 2e9 edges fits in host memory.
  std::vector<uint64_t> out_off, in_off;
  std::vector<uint32_t> out_adj, in_adj;
  // The DAG is built on first use (so that loading a large graph and then
  // applying an ordering builds it once); the mutex guards that build.
  bool dag_ready = false;
  std::mutex dag_mu;
};

// A neighbour list as a range of ranks, for range-for loops.
struct Row {
  const uint32_t *b, *e;
  const uint32_t *begin() const { return b; }
  const uint32_t *end() const { return e; }
  uint64_t size() const { return uint64_t(e - b); }
};

Row Nplus(const Graph &g, uint32_t x) {
  return Row{g.out_adj.data() + g.out_off[x], g.out_adj.data() + g.out_off[x + 1]};
}
Row Nminus(const Graph &g, uint32_t x) {
  return Row{g.in_adj.data() + g.in_off[x], g.in_adj.data() + g.in_off[x + 1]};
}

// Where found triangles go: a buffer of triples (may be absent), a count and
// the set hash.
struct Sink {
  uint32_t *buf = nullptr;
  uint64_t cap = 0;
  uint64_t count = 0;
  uint64_t hash = 0;
  const Graph *g = nullptr;

  // Report triangle {u, v, w} given in rank space.
  void output(uint32_t u, uint32_t v, uint32_t w) {
    uint32_t t[3] = {g->inv[u], g->inv[v], g->inv[w]};
    std::sort(t, t + 3);
    if (buf && count < cap) {
      buf[3 * count + 0] = t[0];
      buf[3 * count + 1] = t[1];
      buf[3 * count + 2] = t[2];
    }
    ++count;
    hash += triple_hash(t[0], t[1], t[2]);
  }
};

// Orient every edge of E by the ordering (Sec. 1.3): (u, v) in E_pi iff
// pi_u < pi_v, stored as u -> v in rank space.  The rows are sized by
// counting d+ and d- first, filled, then sorted.
void build_dag(Graph &g) {
  const uint64_t m = g.E.size();
  g.out_off.assign(uint64_t(g.n) + 1, 0);
  g.in_off.assign(uint64_t(g.n) + 1, 0);
  for (const auto &e : g.E) {
    uint32_t ra = g.rank[e.first], rb = g.rank[e.second];
    ++g.out_off[std::min(ra, rb) + 1];  // d+ of the lower rank
    ++g.in_off[std::max(ra, rb) + 1];   // d- of the higher rank
  }
  for (uint32_t x = 0; x < g.n; ++x) {
    g.out_off[x + 1] += g.out_off[x];
    g.in_off[x + 1] += g.in_off[x];
  }
  g.out_adj.assign(m, 0);
  g.in_adj.assign(m, 0);
  std::vector<uint64_t> out_pos(g.out_off.begin(), g.out_off.end() - 1);
  std::vector<uint64_t> in_pos(g.in_off.begin(), g.in_off.end() - 1);
  for (const auto &e : g.E) {
    uint32_t ra = g.rank[e.first], rb = g.rank[e.second];
    uint32_t lo = std::min(ra, rb), hi = std::max(ra, rb);
    g.out_adj[out_pos[lo]++] = hi;
    g.in_adj[in_pos[hi]++] = lo;
  }
  for (uint32_t x = 0; x < g.n; ++x) {
    std::sort(g.out_adj.begin() + g.out_off[x], g.out_adj.begin() + g.out_off[x + 1]);
    std::sort(g.in_adj.begin() + g.in_off[x], g.in_adj.begin() + g.in_off[x + 1]);
  }
  g.dag_ready = true;
}

// The DAG of the current ordering, built if no call has needed it yet.
const Graph &with_dag(const void *h) {
  Graph *g = static_cast<Graph *>(const_cast<void *>(h));
  std::lock_guard<std::mutex> lock(g->dag_mu);
  if (!g->dag_ready) build_dag(*g);
  return *g;
}

// Algorithm 1 (A++), literally: for each vertex w, mark N-_w in B; for every
// u in N-_w and every v in N+_u, a set B[v] reports {u, v, w}; reset B.
// The outer loop runs over ranks [w_begin, w_end).
void list_app_literal(const Graph &g, uint32_t w_begin, uint32_t w_end, Sink &s,
                      uint64_t &probes) {
  std::vector<char> B(g.n, 0);
  for (uint32_t w = w_begin; w < w_end; ++w) {
    for (uint32_t v : Nminus(g, w)) B[v] = 1;
    for (uint32_t u : Nminus(g, w)) {
      for (uint32_t v : Nplus(g, u)) {
        ++probes;
        if (B[v]) s.output(u, v, w);
      }
    }
    for (uint32_t v : Nminus(g, w)) B[v] = 0;
  }
}

// Algorithm 2 (A+-), literally: for each vertex u, mark N+_u in B; for every
// v in N+_u and every w in N+_v, a set B[w] reports {u, v, w}; reset B.
void list_apm_literal(const Graph &g, uint32_t u_begin, uint32_t u_end, Sink &s,
                      uint64_t &probes) {
  std::vector<char> B(g.n, 0);
  for (uint32_t u = u_begin; u < u_end; ++u) {
    for (uint32_t w : Nplus(g, u)) B[w] = 1;
    for (uint32_t v : Nplus(g, u)) {
      for (uint32_t w : Nplus(g, v)) {
        ++probes;
        if (B[w]) s.output(u, v, w);
      }
    }
    for (uint32_t w : Nplus(g, u)) B[w] = 0;
  }
}

// A-- ("S2+n", the third variant the footnote of Sec. 2.1 names, seed edge
// S2 = (v, w)), in the same boolean-array form: for each vertex v, mark N-_v
// in B; for every w in N+_v and every u in N-_w, a set B[u] reports
// {u, v, w}; reset B.  Vertex w is scanned once per predecessor v, so the
// work is sum_w d-_w * d-_w = C-- (the mirror image of C++ under the reversed
// ordering, hence the footnote's "equivalent to A++").
void list_amm_literal(const Graph &g, uint32_t v_begin, uint32_t v_end, Sink &s,
                      uint64_t &probes) {
  std::vector<char> B(g.n, 0);
  for (uint32_t v = v_begin; v < v_end; ++v) {
    for (uint32_t u : Nminus(g, v)) B[u] = 1;
    for (uint32_t w : Nplus(g, v)) {
      for (uint32_t u : Nminus(g, w)) {
        ++probes;
        if (B[u]) s.output(u, v, w);
      }
    }
    for (uint32_t u : Nminus(g, v)) B[u] = 0;
  }
}

// The same algorithms written as one sorted-list intersection per seed
// edge (Sec. 2.1, "neighborhood intersection"): A++ seeds on the long edge
// L = (u, w) and intersects N+_u with N-_w; A+- seeds on the first short edge
// S1 = (u, v) and intersects N+_u with N+_v; A-- seeds on the second short
// edge S2 = (v, w) and intersects N-_v with N-_w.  std::set_intersection does
// the work; "probes" here counts the scanned list (N+_u, N+_v resp. N-_w) so
// that it is comparable with the literal form.
void list_app_sets(const Graph &g, uint32_t w_begin, uint32_t w_end, Sink &s,
                   uint64_t &probes) {
  std::vector<uint32_t> common;
  for (uint32_t w = w_begin; w < w_end; ++w) {
    for (uint32_t u : Nminus(g, w)) {
      common.clear();
      std::set_intersection(Nplus(g, u).begin(), Nplus(g, u).end(), Nminus(g, w).begin(),
                            Nminus(g, w).end(), std::back_inserter(common));
      probes += Nplus(g, u).size();
      for (uint32_t v : common) s.output(u, v, w);
    }
  }
}

void list_apm_sets(const Graph &g, uint32_t u_begin, uint32_t u_end, Sink &s,
                   uint64_t &probes) {
  std::vector<uint32_t> common;
  for (uint32_t u = u_begin; u < u_end; ++u) {
    for (uint32_t v : Nplus(g, u)) {
      common.clear();
      std::set_intersection(Nplus(g, u).begin(), Nplus(g, u).end(), Nplus(g, v).begin(),
                            Nplus(g, v).end(), std::back_inserter(common));
      probes += Nplus(g, v).size();
      for (uint32_t w : common) s.output(u, v, w);
    }
  }
}

void list_amm_sets(const Graph &g, uint32_t v_begin, uint32_t v_end, Sink &s,
                   uint64_t &probes) {
  std::vector<uint32_t> common;
  for (uint32_t v = v_begin; v < v_end; ++v) {
    for (uint32_t w : Nplus(g, v)) {
      common.clear();
      std::set_intersection(Nminus(g, v).begin(), Nminus(g, v).end(), Nminus(g, w).begin(),
                            Nminus(g, w).end(), std::back_inserter(common));
      probes += Nminus(g, w).size();
      for (uint32_t u : common) s.output(u, v, w);
    }
  }
}

}  // namespace

extern "C" {

// Status codes: 0 ok, 1 invalid argument, 2 output buffer too small (the
// count and hash are still complete).

// Load an undirected graph from a raw edge list edges[2*m_in] of ids in
// [0, n).  Loops are dropped and a pair listed several times, in either
// direction, is kept once (Sec. 4.1).  The ordering starts as the identity.
int or_graph_new(uint32_t n, const uint32_t *edges, uint64_t m_in, void **out) {
  *out = nullptr;
  Graph *g = new Graph;
  g->n = n;
  g->E.reserve(m_in);
  for (uint64_t i = 0; i < m_in; ++i) {
    uint32_t a = edges[2 * i], b = edges[2 * i + 1];
    if (a >= n || b >= n) {
      delete g;
      return 1;
    }
    if (a == b) continue;
    g->E.emplace_back(std::min(a, b), std::max(a, b));
  }
  std::sort(g->E.begin(), g->E.end());
  g->E.erase(std::unique(g->E.begin(), g->E.end()), g->E.end());
  g->rank.resize(n);
  g->inv.resize(n);
  for (uint32_t v = 0; v < n; ++v) g->rank[v] = g->inv[v] = v;
  *out = g;
  return 0;
}

void or_graph_free(void *h) { delete static_cast<Graph *>(h); }

uint64_t or_num_edges(const void *h) { return static_cast<const Graph *>(h)->E.size(); }

// Apply ordering rank[n] (rank[v] = pi_v - 1).  Not a permutation -> 1, and
// the previous ordering stays in force.
int or_order_apply(void *h, const uint32_t *rank) {
  Graph *g = static_cast<Graph *>(h);
  std::vector<char> seen(g->n, 0);
  for (uint32_t v = 0; v < g->n; ++v) {
    if (rank[v] >= g->n || seen[rank[v]]) return 1;
    seen[rank[v]] = 1;
  }
  for (uint32_t v = 0; v < g->n; ++v) {
    g->rank[v] = rank[v];
    g->inv[rank[v]] = v;
  }
  std::lock_guard<std::mutex> lock(g->dag_mu);
  build_dag(*g);
  return 0;
}

// Cost induced by the ordering (Definition of Sec. 3.1):
//   alg 0: C++ = sum_u d+_u * d+_u      alg 1: C+- = sum_u d+_u * d-_u
//   alg 2: C-- = sum_u d-_u * d-_u (A--, by the same counting as Property 1)
uint64_t or_cost(const void *h, int alg) {
  const Graph *g = &with_dag(h);
  uint64_t c = 0;
  for (uint32_t x = 0; x < g->n; ++x) {
    uint64_t dp = Nplus(*g, x).size(), dm = Nminus(*g, x).size();
    c += (alg == 0) ? dp * dp : (alg == 1 ? dp * dm : dm * dm);
  }
  return c;
}

// List triangles with Algorithm 1 (alg 0), Algorithm 2 (alg 1) or A-- (alg
// 2), in the literal boolean-array form (mode 0) or the set-intersection form
// (mode 1).  The outer loop runs over ranks [seed_begin, seed_end) (pass 0
// and n for the whole graph; a sub-range lists the triangles whose third
// vertex (A++), first vertex (A+-) or middle vertex (A--) lies in it).
// Triples go to buf[3*cap] when buf is not null.  Calls on one graph may run
// concurrently from several threads (each has its own B and sink).
int or_list(const void *h, int alg, int mode, uint32_t seed_begin, uint32_t seed_end,
            uint32_t *buf, uint64_t cap, uint64_t *count, uint64_t *hash,
            uint64_t *probes) {
  const Graph *g = &with_dag(h);
  if (alg < 0 || alg > 2 || mode < 0 || mode > 1) return 1;
  if (seed_end > g->n || seed_begin > seed_end) return 1;
  Sink s;
  s.buf = buf;
  s.cap = cap;
  s.g = g;
  uint64_t p = 0;
  if (alg == 0 && mode == 0) list_app_literal(*g, seed_begin, seed_end, s, p);
  if (alg == 0 && mode == 1) list_app_sets(*g, seed_begin, seed_end, s, p);
  if (alg == 1 && mode == 0) list_apm_literal(*g, seed_begin, seed_end, s, p);
  if (alg == 1 && mode == 1) list_apm_sets(*g, seed_begin, seed_end, s, p);
  if (alg == 2 && mode == 0) list_amm_literal(*g, seed_begin, seed_end, s, p);
  if (alg == 2 && mode == 1) list_amm_sets(*g, seed_begin, seed_end, s, p);
  if (count) *count = s.count;
  if (hash) *hash = s.hash;
  if (probes) *probes = p;
  return (buf && s.count > cap) ? 2 : 0;
}

// Export the DAG as CSR in rank space: dir 0 = N+ (out), dir 1 = N- (in).
// off[n+1] and adj[m] are caller-owned.
int or_csr(const void *h, int dir, uint64_t *off, uint32_t *adj) {
  const Graph *g = &with_dag(h);
  uint64_t k = 0;
  for (uint32_t x = 0; x < g->n; ++x) {
    off[x] = k;
    for (uint32_t y : (dir == 0 ? Nplus(*g, x) : Nminus(*g, x))) adj[k++] = y;
  }
  off[g->n] = k;
  return 0;
}

// Degree of every vertex of the simple graph (Sec. 1.3: its number of
// neighbours), counted over the cleaned edge set E, original ids.
int or_degrees(const void *h, uint32_t *deg) {
  const Graph *g = static_cast<const Graph *>(h);
  for (uint32_t v = 0; v < g->n; ++v) deg[v] = 0;
  for (const auto &e : g->E) {
    ++deg[e.first];
    ++deg[e.second];
  }
  return 0;
}

// The set hash of caller-given triples (each must already be sorted a<b<c).
uint64_t or_hash_triples(const uint32_t *t, uint64_t count) {
  uint64_t hsum = 0;
  for (uint64_t i = 0; i < count; ++i) hsum += triple_hash(t[3 * i], t[3 * i + 1], t[3 * i + 2]);
  return hsum;
}

uint64_t or_mix64(uint64_t z) { return mix(z); }

}  // extern "C"
