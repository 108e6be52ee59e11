/*
 * Host-side vertex orderings used as inputs of the listing path.
 *
 * Input graph: a simple undirected graph in symmetric CSR form (off[n+1],
 * adj[off[n]]), each row sorted by id.  Output: rank[v] in [0, n), a
 * permutation (rank[v] = pi_v - 1 with pi the 1-based index of Sec. 1.3).
 *
 *  - order_core:  degeneracy ordering by the bucket peeling of Batagelj and
 *                 Zaversnik (2003), which Sec. 1.3 names for core ordering.
 *  - order_check: the Check heuristic of Sec. 3.3.2.
 *  - order_neigh: the Neigh heuristic of Sec. 3.3.1 (Algorithm 3, Fig. 3),
 *                 minimising C+- as in the paper or C++ = sum of d+^2 (Sec.
 *                 3.3.1 notes that the heuristic serves other objectives,
 *                 C++ among them).
 *
 * Plain C99; no platform-specific code.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Batagelj-Zaversnik peeling: repeatedly remove a vertex of minimum current
 * degree; rank = removal index.  Initial bins are filled in increasing id
 * order, so the result is deterministic.  Returns the degeneracy c(G). */
int64_t tls_order_core(int64_t n, const int64_t *off, const uint32_t *adj,
                       uint32_t *rank) {
  if (n <= 0) return 0;
  int64_t *deg = (int64_t *)malloc(sizeof(int64_t) * n);
  int64_t *pos = (int64_t *)malloc(sizeof(int64_t) * n);
  int64_t *vert = (int64_t *)malloc(sizeof(int64_t) * n);
  int64_t md = 0;
  for (int64_t v = 0; v < n; ++v) {
    deg[v] = off[v + 1] - off[v];
    if (deg[v] > md) md = deg[v];
  }
  int64_t *bin = (int64_t *)calloc((size_t)md + 2, sizeof(int64_t));
  for (int64_t v = 0; v < n; ++v) bin[deg[v]]++;
  int64_t start = 0;
  for (int64_t d = 0; d <= md; ++d) {
    int64_t num = bin[d];
    bin[d] = start;
    start += num;
  }
  for (int64_t v = 0; v < n; ++v) {
    pos[v] = bin[deg[v]];
    vert[pos[v]] = v;
    bin[deg[v]]++;
  }
  for (int64_t d = md; d >= 1; --d) bin[d] = bin[d - 1];
  bin[0] = 0;
  int64_t degeneracy = 0;
  for (int64_t i = 0; i < n; ++i) {
    int64_t v = vert[i];
    rank[v] = (uint32_t)i;
    if (deg[v] > degeneracy) degeneracy = deg[v];
    for (int64_t k = off[v]; k < off[v + 1]; ++k) {
      int64_t u = adj[k];
      if (deg[u] > deg[v]) {
        int64_t du = deg[u], pu = pos[u], pw = bin[du], w = vert[pw];
        if (u != w) {
          pos[u] = pw;
          vert[pu] = w;
          pos[w] = pu;
          vert[pw] = u;
        }
        bin[du]++;
        deg[u]--;
      }
    }
  }
  free(deg);
  free(pos);
  free(vert);
  free(bin);
  return degeneracy;
}

/* Check heuristic (Sec. 3.3.2).  Vertices are taken by decreasing degree
 * (`by_degree_desc` gives that sequence).  Each vertex u goes either just
 * after the vertices already placed at the beginning, with cost
 * C_b = |N_b| (|N_e| + |N_?|), or just before those placed at the end, with
 * cost C_e = (|N_b| + |N_?|) |N_e|; the smaller cost wins, a tie goes to
 * the beginning. */
void tls_order_check(int64_t n, const int64_t *off, const uint32_t *adj,
                     const uint32_t *by_degree_desc, uint32_t *rank) {
  int64_t *nb = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  int64_t *ne = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  int64_t b = 0, e = n - 1;
  for (int64_t i = 0; i < n; ++i) {
    uint32_t u = by_degree_desc[i];
    int64_t d = off[u + 1] - off[u];
    int64_t Nb = nb[u], Ne = ne[u], Nq = d - Nb - Ne;
    int64_t Cb = Nb * (Ne + Nq), Ce = (Nb + Nq) * Ne;
    int at_begin = Cb <= Ce;
    rank[u] = (uint32_t)(at_begin ? b++ : e--);
    for (int64_t k = off[u]; k < off[u + 1]; ++k) {
      if (at_begin)
        nb[adj[k]]++;
      else
        ne[adj[k]]++;
    }
  }
  free(nb);
  free(ne);
}

/* ---- Neigh heuristic (Algorithm 3) -------------------------------------
 * The ordering is a doubly linked list; each vertex also carries a double
 * key that increases along the list, so two vertices compare in O(1).  A
 * vertex moved between two neighbours takes the midpoint key; when the
 * midpoint is no longer strictly between them, every key is renumbered
 * from the list (rare). */
typedef struct {
  int64_t n;
  int64_t *prev, *next;
  double *key;
  int64_t head, tail;
} olist;

static void ol_renumber(olist *L) {
  double k = 0.0;
  for (int64_t v = L->head; v >= 0; v = L->next[v]) L->key[v] = k, k += 1.0;
}

static void ol_unlink(olist *L, int64_t u) {
  int64_t p = L->prev[u], q = L->next[u];
  if (p >= 0) L->next[p] = q; else L->head = q;
  if (q >= 0) L->prev[q] = p; else L->tail = p;
}

/* Insert u right after x (x = -1 means at the head). */
static void ol_insert_after(olist *L, int64_t u, int64_t x) {
  int64_t q = (x >= 0) ? L->next[x] : L->head;
  L->prev[u] = x;
  L->next[u] = q;
  if (x >= 0) L->next[x] = u; else L->head = u;
  if (q >= 0) L->prev[q] = u; else L->tail = u;
  double lo = (x >= 0) ? L->key[x] : ((q >= 0) ? L->key[q] - 2.0 : 0.0);
  double hi = (q >= 0) ? L->key[q] : lo + 2.0;
  double mid = 0.5 * (lo + hi);
  if (!(mid > lo && mid < hi)) {
    ol_renumber(L);
  } else {
    L->key[u] = mid;
  }
}

static const double *g_sort_key;
static int cmp_by_key(const void *a, const void *b) {
  double ka = g_sort_key[*(const uint32_t *)a], kb = g_sort_key[*(const uint32_t *)b];
  return (ka > kb) - (ka < kb);
}

/* The cost Neigh minimises (Sec. 3.1): C+- = sum d+ d- (objective 0) or
 * C++ = sum d+^2 (objective 1). */
static int64_t neigh_cost(int64_t objective, int64_t n, const int64_t *dp, const int64_t *dm) {
  int64_t c = 0;
  for (int64_t v = 0; v < n; ++v) c += objective ? dp[v] * dp[v] : dp[v] * dm[v];
  return c;
}

/* Best slot of a vertex u of degree d whose neighbours nb[0..d) are sorted
 * in the current order, the first pcur of them before u.  Slot p puts u just
 * after nb[p-1] (p = 0: before nb[0]): u gets d- = p and d+ = d - p, and a
 * neighbour nb[j] has u as a successor iff j < p.  With dp'/dm' a
 * neighbour's degrees without its edge to u, the cost at slot p is a
 * constant plus
 *   C+-: p (d - p) + sum_{j<p} (dm'_j - dp'_j)
 *   C++: (d - p)^2 + sum_{j<p} (2 dp'_j + 1)     [(dp' + 1)^2 - dp'^2]
 * Among slots of equal cost the current one is kept, else the smallest p. */
static int64_t neigh_best_slot(int64_t objective, int64_t d, const uint32_t *nb, int64_t pcur,
                               const int64_t *dp, const int64_t *dm) {
  int64_t best_p = pcur, best = 0, cur_val = 0, run = 0;
  int have = 0;
  for (int64_t p = 0; p <= d; ++p) {
    int64_t val = (objective ? (d - p) * (d - p) : p * (d - p)) + run;
    if (p == pcur) cur_val = val;
    if (!have || val < best) best = val, best_p = p, have = 1;
    if (p < d) {
      uint32_t v = nb[p];
      int64_t before = p < pcur; /* v currently precedes u */
      int64_t dpv = dp[v] - before;
      int64_t dmv = dm[v] - (1 - before);
      run += objective ? 2 * dpv + 1 : dmv - dpv;
    }
  }
  return cur_val <= best ? pcur : best_p;
}

/* Neigh: starting from `rank` (updated in place), repeat passes over the
 * vertices in increasing id; each vertex u moves to the slot p* in [0, d_u]
 * (just after its p*-th neighbour in the current order, or before all of
 * them for p* = 0) that minimises the cost (C+- for objective 0, C++ for
 * objective 1).  A pass is repeated while it cut the cost by more than a
 * factor (1 - eps) (stopping rule of Algorithm 3; Neigh stops after
 * `max_iter` passes at most).  Among equal costs the current slot is kept,
 * else the smallest p.  cost_trace[i] = the cost before pass i and after
 * the last one.  Returns the number of passes. */
int64_t tls_order_neigh(int64_t n, const int64_t *off, const uint32_t *adj,
                        uint32_t *rank, double eps, int64_t max_iter,
                        int64_t *cost_trace, int64_t objective) {
  olist L;
  L.n = n;
  L.prev = (int64_t *)malloc(sizeof(int64_t) * n);
  L.next = (int64_t *)malloc(sizeof(int64_t) * n);
  L.key = (double *)malloc(sizeof(double) * n);
  int64_t *byrank = (int64_t *)malloc(sizeof(int64_t) * n);
  for (int64_t v = 0; v < n; ++v) byrank[rank[v]] = v;
  for (int64_t i = 0; i < n; ++i) {
    int64_t v = byrank[i];
    L.prev[v] = i ? byrank[i - 1] : -1;
    L.next[v] = (i + 1 < n) ? byrank[i + 1] : -1;
    L.key[v] = (double)i;
  }
  L.head = n ? byrank[0] : -1;
  L.tail = n ? byrank[n - 1] : -1;
  free(byrank);

  int64_t *dp = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  int64_t *dm = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  for (int64_t u = 0; u < n; ++u)
    for (int64_t k = off[u]; k < off[u + 1]; ++k) {
      if (L.key[adj[k]] > L.key[u]) dp[u]++; else dm[u]++;
    }
  int64_t maxd = 0;
  for (int64_t u = 0; u < n; ++u)
    if (off[u + 1] - off[u] > maxd) maxd = off[u + 1] - off[u];
  uint32_t *nb = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(maxd + 1));

  int64_t iters = 0;
  g_sort_key = L.key;
  while (iters < max_iter) {
    int64_t c0 = neigh_cost(objective, n, dp, dm);
    if (cost_trace) cost_trace[iters] = c0;
    for (int64_t u = 0; u < n; ++u) {
      int64_t d = off[u + 1] - off[u];
      if (d == 0) continue;
      memcpy(nb, adj + off[u], sizeof(uint32_t) * (size_t)d);
      qsort(nb, (size_t)d, sizeof(uint32_t), cmp_by_key);
      /* current slot of u = number of neighbours before it */
      int64_t pcur = 0;
      while (pcur < d && L.key[nb[pcur]] < L.key[u]) ++pcur;
      int64_t best_p = neigh_best_slot(objective, d, nb, pcur, dp, dm);
      if (best_p == pcur) continue;
      /* update degrees: neighbours before slot best_p are predecessors */
      for (int64_t j = 0; j < d; ++j) {
        uint32_t v = nb[j];
        int was_before = L.key[v] < L.key[u];
        int now_before = j < best_p;
        if (was_before != now_before) {
          if (now_before) { dp[v]++; dm[v]--; } else { dp[v]--; dm[v]++; }
        }
      }
      dm[u] = best_p;
      dp[u] = d - best_p;
      ol_unlink(&L, u);
      if (best_p == 0) ol_insert_after(&L, u, L.prev[nb[0]]);
      else ol_insert_after(&L, u, nb[best_p - 1]);
    }
    ++iters;
    int64_t c1 = neigh_cost(objective, n, dp, dm);
    if (!((double)c1 < (1.0 - eps) * (double)c0)) break;
  }
  if (cost_trace) cost_trace[iters] = neigh_cost(objective, n, dp, dm);
  int64_t i = 0;
  for (int64_t v = L.head; v >= 0; v = L.next[v]) rank[v] = (uint32_t)i++;
  free(nb);
  free(dp);
  free(dm);
  free(L.prev);
  free(L.next);
  free(L.key);
  return iters;
}

/* Single Neigh move of one vertex (the update of Fig. 3), for tests. */
void tls_neigh_move_one(int64_t n, const int64_t *off, const uint32_t *adj,
                        uint32_t *rank, int64_t u, int64_t objective) {
  (void)n;
  /* Build the same state as order_neigh, run the body for u only. */
  int64_t d = off[u + 1] - off[u];
  if (d == 0) return;
  int64_t *dp = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  int64_t *dm = (int64_t *)calloc((size_t)n, sizeof(int64_t));
  for (int64_t x = 0; x < n; ++x)
    for (int64_t k = off[x]; k < off[x + 1]; ++k) {
      if (rank[adj[k]] > rank[x]) dp[x]++; else dm[x]++;
    }
  uint32_t *nb = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)d);
  memcpy(nb, adj + off[u], sizeof(uint32_t) * (size_t)d);
  /* insertion sort by rank (d is small in tests) */
  for (int64_t i = 1; i < d; ++i) {
    uint32_t x = nb[i];
    int64_t j = i - 1;
    while (j >= 0 && rank[nb[j]] > rank[x]) nb[j + 1] = nb[j], --j;
    nb[j + 1] = x;
  }
  int64_t pcur = 0;
  while (pcur < d && rank[nb[pcur]] < rank[u]) ++pcur;
  int64_t best_p = neigh_best_slot(objective, d, nb, pcur, dp, dm);
  if (best_p != pcur) {
    /* new position: just after neighbour best_p-1, or just before nb[0] */
    uint32_t old = rank[u];
    int64_t target;
    if (best_p == 0) target = (int64_t)rank[nb[0]];      /* take nb[0]'s slot */
    else target = (int64_t)rank[nb[best_p - 1]] + 1;    /* slot after it */
    /* remove u, then insert at target (indices shift when removing) */
    for (int64_t x = 0; x < n; ++x)
      if (rank[x] > old) rank[x]--;
    if (target > (int64_t)old) target--;
    for (int64_t x = 0; x < n; ++x)
      if ((int64_t)rank[x] >= target && x != u) rank[x]++;
    rank[u] = (uint32_t)target;
  }
  free(nb);
  free(dp);
  free(dm);
}
