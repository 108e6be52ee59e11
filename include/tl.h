/*
 * tl.h -- triangle listing with a given vertex ordering on one GB300 GPU.
 *
 * C ABI of the hot path of Lecuyer, Jachiet, Magnien and Tabourier,
 * "Tailored vertex ordering for faster triangle listing in large graphs"
 * (arXiv:2203.04774): the "mere listing" task of Sec. 3.2 -- list every
 * triangle of an undirected graph once, the vertex ordering being given.
 *
 *   tl_graph_load      load an edge list; drop loops, merge duplicate and
 *                      reversed pairs (Sec. 4.1, dataset cleaning).
 *   tl_order_apply     relabel the vertices by an ordering pi and orient each
 *                      edge from lower to higher rank: the DAG G_pi of
 *                      Sec. 1.3, stored as a rank-space CSR of sorted
 *                      successor lists N+ and predecessor lists N-.
 *   tl_cost            C++(pi) = sum d+_u d+_u or C+-(pi) = sum d+_u d-_u
 *                      (Definition "Cost induced by an ordering", Sec. 3.1),
 *                      or C-- = sum d-_u d-_u of the third variant.
 *   tl_list_triangles  Algorithm 1 (A++), Algorithm 2 (A+-) or the third
 *                      variant A-- of Sec. 2.1; each triangle is reported
 *                      exactly once, in chunks of device memory handed to a
 *                      consumer callback.
 *
 * Conventions common to every call
 *   - Every call returns a tl_status; no C++ exception crosses the ABI.
 *     On failure tl_last_error() gives a message (thread-local, valid until
 *     the next call on the same thread).
 *   - Vertex ids are uint32 in [0, n).  Orderings are 0-based ranks:
 *     rank[v] = pi_v - 1, where pi is the 1-based index of Sec. 1.3.
 *   - A graph handle owns all of its device memory.  It is not thread-safe:
 *     use one handle per host thread.  Work is ordered on the handle's
 *     stream (the stream given to tl_graph_load).
 *   - "Host or device pointer" arguments say which with a flag; a device
 *     pointer must be device memory of the current CUDA device.
 *   - The library never falls back to the CPU: without a usable CUDA device
 *     every call that computes returns TL_ECUDA.
 */
#ifndef TL_H_
#define TL_H_

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define TL_EXPORT __attribute__((visibility("default")))
#else
#define TL_EXPORT
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tl_graph tl_graph; /* opaque */

typedef enum {
  TL_OK = 0,
  TL_EINVAL = 1,     /* bad argument: NULL, id >= n, rank not a permutation */
  TL_ENOMEM = 2,     /* device or pinned host allocation failed */
  TL_ECUDA = 3,      /* CUDA runtime error (see tl_last_error) */
  TL_ESTATE = 4,     /* call out of order, e.g. listing before order_apply */
  TL_ECALLBACK = 5,  /* the consumer returned non-zero; listing stopped */
  TL_ETIMEOUT = 6    /* a bounded device wait ran out */
} tl_status;

typedef enum {
  TL_APP = 0, /* Algorithm 1, A++ ("L+n"): seed edge L=(u,w), scan N+_u, probe N-_w */
  TL_APM = 1, /* Algorithm 2, A+- ("S1+n"): seed edge S1=(u,v), scan N+_v, probe N+_u */
  TL_AMM = 2  /* A-- ("S2+n", the third variant of the footnote of Sec. 2.1): seed
                 edge S2=(v,w), scan N-_w, probe N-_v; work C-- = sum d-_w d-_w */
} tl_alg;

/* Load an undirected graph.
 *   n          number of vertices (1 <= n < 2^32 - 1).
 *   edges      2*m_in uint32 ids, pairs (a_i, b_i) laid out a0 b0 a1 b1 ...;
 *              host pointer if edges_on_device == 0, else device pointer.
 *              The caller keeps ownership; the library copies what it needs.
 *   m_in       number of pairs (may be 0).
 *   stream     cudaStream_t (as void*) all of the handle's work is ordered
 *              on; NULL = the legacy default stream.
 * Loops (a == b) are dropped and a pair given several times, in either
 * direction, is kept once (Sec. 4.1).  An id >= n -> TL_EINVAL.  The
 * ordering starts as the identity (the "original ordering" of Sec. 2.2).
 * On success *out owns the graph; free it with tl_graph_free. */
TL_EXPORT tl_status tl_graph_load(tl_graph **out, uint32_t n, const uint32_t *edges,
                        uint64_t m_in, int edges_on_device, void *stream);

/* Disjoint unions: many independent graphs as one graph, so that one build
 * and one listing pass serve all of them.  The paper has no counterpart (it
 * lists one graph at a time); what makes it exact is that no edge joins two
 * parts, so each triangle of the union (three pairwise adjacent vertices,
 * Sec. 1.3) lies inside one part and the union's triangles are the parts'.
 * Layout: part i's vertex v is the union's vertex vbase_i + v, where
 * vbase_i = n_0 + ... + n_{i-1}; the union has n = n_0 + ... + n_{k-1}
 * vertices (< 2^32 - 1, else TL_EINVAL).  The union's triples carry union
 * ids; tl_count_hash_parts maps them back to (part, local ids).
 *
 * tl_graph_load_parts: k >= 1 graphs given as one concatenated edge list.
 *   n      host array of k part sizes, each >= 1.
 *   m_in   host array of k pair counts; part i's pairs follow part i-1's.
 *   edges  2 * sum(m_in) uint32 part-local ids (host or device pointer as in
 *          tl_graph_load); an id >= its part's n -> TL_EINVAL.
 * Cleaning as in tl_graph_load; the ordering starts as the identity.
 * On a union (from either call) tl_order_compute works part by part: part
 * i's vertices get the ranks vbase_i + (their ranks in the part's own
 * degree, Split or core ordering), so ranks [vbase_i, vbase_{i+1}) are part i's
 * and a tl_list_triangles_range over them lists part i alone. */
TL_EXPORT tl_status tl_graph_load_parts(tl_graph **out, uint32_t k, const uint32_t *n,
                                        const uint64_t *m_in, const uint32_t *edges,
                                        int edges_on_device, void *stream);

/* tl_graph_union: the disjoint union of k >= 1 loaded graphs, each under
 * rank[i] (device pointer, n_i part-local ranks) or, when rank or rank[i]
 * is NULL, under its current ordering (the identity if none was applied).
 * The union's ordering puts part i's vertex v at rank vbase_i + rank_i[v],
 * so each part keeps its DAG G_pi and its costs; C++, C+- and C-- of the
 * union are the sums over parts (Sec. 3.1).  The DAG is built before
 * returning: when no rank is given and every part already holds its DAG (an
 * ordering was applied to it), by concatenating the parts' DAGs (about 32
 * bytes moved per edge, no sort); otherwise by the relabel-and-sort of
 * tl_order_apply.
 * A rank[i] that is not a permutation of [0, n_i) -> TL_EINVAL.  The parts
 * are only read, and must not be modified or freed during the call; they
 * stay owned by the caller, and the union owns copies. */
TL_EXPORT tl_status tl_graph_union(tl_graph **out, const tl_graph *const *graphs,
                                   const uint32_t *const *rank, uint32_t k, void *stream);

/* Number of vertices and of undirected edges (after cleaning). */
TL_EXPORT tl_status tl_graph_size(const tl_graph *g, uint32_t *n, uint64_t *m);

/* Apply an ordering: rank[v] = pi_v - 1 for v in [0, n), host pointer if
 * rank_on_device == 0, else device pointer.  Builds G_pi (Sec. 1.3) as a
 * rank-space CSR: N+_x sorted ascending (successor ranks) and N-_x sorted
 * ascending (predecessor ranks).  Not a permutation of [0, n) ->
 * TL_EINVAL, and the previous ordering stays in force. */
TL_EXPORT tl_status tl_order_apply(tl_graph *g, const uint32_t *rank, int rank_on_device);

/* Orderings computed on the device from the loaded graph's degrees d_v
 * (Sec. 1.3), written as ranks (rank[v] = pi_v - 1) to `rank` (n uint32;
 * host pointer if rank_on_device == 0, else device pointer; caller-owned):
 *   TL_ORDER_DEGREE: non-decreasing degree, ties by increasing id -- the
 *                    degree ordering of Sec. 2.2;
 *   TL_ORDER_SPLIT:  the Split heuristic of Sec. 3.3.3 -- vertices by
 *                    non-increasing degree (ties by increasing id), the one at
 *                    1-based position 2i+1 gets pi = i+1, the one at 2i gets
 *                    pi = n+1-i;
 *   TL_ORDER_CORE:   a core ordering (Sec. 1.3, Sec. 2.2) by level-synchronous
 *                    peeling: at level k every remaining vertex of degree
 *                    <= k is removed in one round, the neighbours whose degree
 *                    falls to k in the next round, and so on; then k moves to
 *                    the smallest remaining degree.  Vertices are ranked by
 *                    (round, id): coreness is non-decreasing along the
 *                    ordering and d+_v <= c_v for every v (a degeneracy
 *                    ordering).  Ties differ from one-vertex-at-a-time
 *                    peeling (Batagelj and Zaversnik).
 * On a disjoint union each part is ordered on its own (see
 * tl_graph_load_parts).  The ordering is not applied; pass it to
 * tl_order_apply. */
typedef enum { TL_ORDER_DEGREE = 0, TL_ORDER_SPLIT = 1, TL_ORDER_CORE = 2 } tl_order_kind;
TL_EXPORT tl_status tl_order_compute(tl_graph *g, tl_order_kind kind, uint32_t *rank,
                                     int rank_on_device);

/* Cost of the current ordering (Sec. 3.1): TL_APP -> C++ = sum_u d+_u^2,
 * TL_APM -> C+- = sum_u d+_u d-_u, TL_AMM -> C-- = sum_u d-_u^2.  Exact,
 * uint64.  By Property 1 (and the same counting for A--) this is the number
 * of neighbour tests the chosen algorithm performs. */
TL_EXPORT tl_status tl_cost(const tl_graph *g, tl_alg alg, uint64_t *cost);

/* Consumer of one chunk of triangles.  dev_triples points to n_triples
 * records of three uint32 original vertex ids (a, b, c), a < b < c, in
 * device memory owned by the library and valid only during the call; the
 * consumer must have finished reading it (including device work it queued)
 * before it returns.  chunk_index counts chunks from 0.  Chunks hold no
 * particular order of triangles.  Return 0 to continue, non-zero to stop
 * listing with TL_ECALLBACK. */
typedef int (*tl_consumer)(const uint32_t *dev_triples, uint64_t n_triples,
                           uint64_t chunk_index, void *user);

/* List every triangle of the graph once (Sec. 2.1):
 *   TL_APP: for each oriented edge (u, w), every v in N+_u that is in N-_w
 *           gives triangle {u, v, w} (Algorithm 1);
 *   TL_APM: for each oriented edge (u, v), every w in N+_v that is in N+_u
 *           gives triangle {u, v, w} (Algorithm 2);
 *   TL_AMM: for each oriented edge (v, w), every u in N-_w that is in N-_v
 *           gives triangle {u, v, w} (A--).
 * Triangles are reported in original ids, sorted, in chunks of at most
 * chunk_bytes / 12 triples (chunk_bytes >= TL_MIN_CHUNK_BYTES; two chunk
 * buffers are allocated per call).  cb may be NULL (triangles are then only
 * counted).  *n_triangles (may be NULL) receives the number listed.  The
 * call returns when every chunk has been consumed. */
#define TL_MIN_CHUNK_BYTES ((size_t)12 << 20)
TL_EXPORT tl_status tl_list_triangles(tl_graph *g, tl_alg alg, size_t chunk_bytes,
                            tl_consumer cb, void *user, uint64_t *n_triangles);

/* Same, restricted to the seed vertices of rank [x_begin, x_end): the
 * vertex w of Algorithm 1's outer loop (A++), u of Algorithm 2's (A+-) or v
 * of A--'s.
 * Disjoint ranges list disjoint triangle sets whose union over a partition
 * of [0, n) is the full set; this is how independent replicas split one
 * graph.  Also returns the number of neighbour tests performed in
 * *n_probes (may be NULL); over the full range it equals tl_cost. */
TL_EXPORT tl_status tl_list_triangles_range(tl_graph *g, tl_alg alg, uint32_t x_begin,
                                  uint32_t x_end, size_t chunk_bytes,
                                  tl_consumer cb, void *user,
                                  uint64_t *n_triangles, uint64_t *n_probes);

/* The work split of the listing kernels: how the outer loop of Algorithms 1
 * and 2 (Sec. 2.1; for each vertex x, the seeds of x, each with its scanned
 * list) is cut into device tasks, and which kernel (which membership
 * structure for B) takes each vertex.  The paper runs that loop on one thread;
 * these are choices of the GPU path that change speed only, never the
 * triangles, their count or the probe count.  Each "B vertex" x (w for A++,
 * u for A+-, v for A--) with probe-set size p (the list marked in B) and W
 * membership tests goes to the first of five kernels that takes it:
 *   small   p <= small_max_p,  W <= warp_work: one warp, vertices grouped per task
 *   medium  p <= medium_max_p, W <= warp_work: one warp, vertices grouped per task
 *   narrow  p <= narrow_max_p: one-warp CTAs, pieces of narrow_piece tests
 *   mid     p <= mid_max_p:    256-thread CTAs, pieces of mid_piece tests
 *   large   any p:             1024-thread CTAs, pieces of
 *           clamp(large_per_p * p, large_min, large_max) tests (large_max is
 *           further capped at 1/16 of the listing's work per large CTA)
 * Every piece rebuilds B, so larger pieces amortise that build; smaller ones
 * balance the end of a launch.
 * narrow_keep_mib and narrow_cold_first set the L2 eviction priority of the
 * narrow kernel's loads in its short-list steps (four tests per lane spread
 * over lists shorter than 128 tests): the scanned lists of the highest ranks,
 * narrow_keep_mib MiB of them (under a degree ordering the most-scanned
 * lists), are loaded with evict_last, and with narrow_cold_first = 1 the
 * others with evict_first; 0 and 0 give no hint.
 * large_hash_max_p: on graphs of more than 2^20 ranks, a large vertex with
 * p <= large_hash_max_p is probed in a shared-memory bucketed hash table, a
 * larger one through a shared-memory filter whose candidates are checked
 * against the CTA's hash table in global memory when its warp flushes. */
typedef struct {
  uint32_t small_max_p;  /* <= 32   (per-warp table of 64 slots) */
  uint32_t medium_max_p; /* <= 1024 (per-warp table of 2048 slots) */
  uint32_t narrow_max_p; /* <= 256  (per-CTA table of 512 slots behind a filter) */
  uint32_t mid_max_p;    /* <= 2048 (per-CTA table of 8192 slots) */
  uint32_t warp_work;    /* 256 .. 4096 */
  uint32_t narrow_piece; /* >= 1024 */
  uint32_t mid_piece;    /* >= 1024 */
  uint32_t large_per_p;  /* >= 1 */
  uint32_t large_min;    /* >= 1024 */
  uint32_t large_max;    /* >= large_min */
  uint32_t narrow_keep_mib;   /* 0 .. 4096 */
  uint32_t narrow_cold_first; /* 0 or 1 */
  uint32_t large_hash_max_p;  /* <= 16384 (per-CTA table of 32768 slots) */
} tl_tuning;
/* The defaults (every graph starts with them). */
TL_EXPORT tl_status tl_default_tuning(tl_tuning *out);
/* Set the work split of later listings on g (NULL restores the defaults).
 * A value outside the ranges above -> TL_EINVAL, and g keeps its split. */
TL_EXPORT tl_status tl_set_tuning(tl_graph *g, const tl_tuning *t);
TL_EXPORT tl_status tl_get_tuning(const tl_graph *g, tl_tuning *out);

/* The work profile of a listing, the degree profile the work split is
 * chosen by (see paper_2203_04774_gb300/autotune.py): for the B vertices x
 * of rank [x_begin, x_end) (w for A++, u for A+-, v for A--), with probe-set
 * size p_x and W_x membership tests (so that the W_x add up to the cost of
 * Sec. 3.1 over the range, by Property 1),
 *   hist[bp * TL_PROFILE_BINS_W + bw] = sum of W_x over the x with
 *   bit_length(p_x) = bp and bit_length(W_x) = bw
 * (bit_length(0) = 0; larger values fall in the last bin).  hist is a host
 * array of TL_PROFILE_BINS_P * TL_PROFILE_BINS_W uint64, filled in full.
 * The paper has no counterpart. */
#define TL_PROFILE_BINS_P 33
#define TL_PROFILE_BINS_W 48
TL_EXPORT tl_status tl_work_profile(tl_graph *g, tl_alg alg, uint32_t x_begin, uint32_t x_end,
                                    uint64_t *hist);

/* A ready-made consumer: count the triples and add up their set hash
 *   H = sum over triples of h(a,b,c)  (mod 2^64),
 *   h(a,b,c) = mix(mix(mix(a + G) + b + G) + c + G),
 * G = 0x9e3779b97f4a7c15, mix = the splitmix64 finaliser (Steele, Lea and
 * Flood, OOPSLA 2014).  The sum does not depend on the order of triangles
 * or the chunking, so it checks a large output without storing it.
 * Pass a tl_count_hash_state* as `user`; zero it before listing.  The
 * reduction runs on the device on `stream` and is synchronised before the
 * consumer returns. */
typedef struct {
  uint64_t count;  /* out: triples seen */
  uint64_t hash;   /* out: H */
  void *stream;    /* in: cudaStream_t for the reduction (NULL = default) */
  void *scratch;   /* library-owned; leave NULL, release with tl_count_hash_release */
} tl_count_hash_state;
TL_EXPORT int tl_count_hash(const uint32_t *dev_triples, uint64_t n_triples,
                  uint64_t chunk_index, void *user);
TL_EXPORT void tl_count_hash_release(tl_count_hash_state *s);

/* The count + hash consumer per part of a disjoint union (tl_graph_load_parts,
 * tl_graph_union): each triple (a, b, c) belongs to the part p with
 * vbase[p] <= a < vbase[p+1] and is hashed with its part-local ids
 * (a - vbase[p], b - vbase[p], c - vbase[p]) by the H of tl_count_hash, so a
 * part's (count, hash) equals what tl_count_hash gives for that graph alone.
 * The paper has no counterpart: this demultiplexes batched listing.
 *   vbase   device, k+1 uint64 vertex offsets (vbase[0] = 0, vbase[k] = n).
 *   counts  device, k uint64; each call adds the chunk's per-part counts.
 *   hashes  device, k uint64; each call adds the chunk's per-part hashes.
 * All three are caller-owned (zero counts and hashes before listing); the
 * consumer allocates nothing.  The reduction runs on `stream` and is
 * synchronised before the call returns.  Returns 0 on success. */
typedef struct {
  const uint64_t *vbase; /* in: device */
  uint32_t k;            /* in: number of parts (>= 1) */
  uint64_t *counts;      /* in/out: device */
  uint64_t *hashes;      /* in/out: device */
  void *stream;          /* in: cudaStream_t for the reduction (NULL = default) */
} tl_count_hash_parts_state;
TL_EXPORT int tl_count_hash_parts(const uint32_t *dev_triples, uint64_t n_triples,
                                  uint64_t chunk_index, void *user);

/* The count + hash consumer again, for callers that cannot allocate device
 * memory.  The paper has no counterpart: this is a library convenience.
 * tl_count_hash allocates its accumulator with cudaMalloc on first use;
 * a consumer runs while the next listing kernel is in flight, and a caller
 * that keeps all device memory in its own pool, or must not incur the
 * implicit device synchronisation of cudaMalloc / cudaFree at that point,
 * cannot allocate there.  This variant calls no allocator: its scratch (one
 * partial hash per block of 16384 triples) lives in a fixed 128 KiB
 * file-scope device array that every GPU loading the library holds until
 * the process exits.
 *   - Same hash H and consumer signature as tl_count_hash.  Pass a
 *     tl_count_hash_noalloc_state* as `user`: dev_out is caller-owned device
 *     memory of two uint64 (count, hash); each call ADDS the chunk's count
 *     and hash to them (zero them before listing).  The reduction runs on
 *     `stream` and is synchronised before the call returns.
 *   - At most TL_NOALLOC_MAX_TRIPLES triples per call; a larger n_triples is
 *     rejected (non-zero return, message in tl_last_error) before any work.
 *   - All calls on a device share the scratch array and leave their partials
 *     in it; calls that overlap on the GPU race on it, so serialise them.
 *   - The first call on a device looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current; make that first call
 *     before any stream capture.
 * Returns 0 on success, non-zero on error. */
#define TL_NOALLOC_MAX_TRIPLES ((uint64_t)1 << 28)
typedef struct {
  uint64_t *dev_out; /* in: device pointer to {count, hash}; calls add to it */
  void *stream;      /* in: cudaStream_t for the reduction (NULL = default) */
} tl_count_hash_noalloc_state;
TL_EXPORT int tl_count_hash_noalloc(const uint32_t *dev_triples, uint64_t n_triples,
                                    uint64_t chunk_index, void *user);

/* ---- Serving: listing requests over device-resident graphs ----------------
 *
 * The paper has no counterpart (it lists one graph at a time); this is the
 * request loop around the same path.  Graphs and their orderings are
 * registered once and stay on the device: each registered ordering is kept
 * as a copy of the graph with its DAG built under it (16 m + 24 n bytes), so
 * that a batch is the concatenation of its requests' DAGs.  A request names a registered
 * graph, one of its registered orderings and an algorithm (TL_APP, TL_APM
 * or TL_AMM), and gets back the count and set hash H (as tl_count_hash) of the
 * graph's triangles.  Worker threads, one CUDA stream each, form batches:
 * a worker takes the oldest waiting requests, as many as fit (at most
 * max_batch, their estimated device footprint within what the budget has
 * left), lists them as one disjoint union (tl_graph_union; the requests
 * grouped by algorithm, one listing range per group) and completes them
 * together.  With workers >= 2, requests that arrive while one batch is on
 * the GPU are admitted into the next as soon as a worker and memory are
 * free, and the two batches overlap on the device.  max_batch = 1 serves
 * one request per pass (the unbatched baseline).
 *
 * Footprint: a request on a graph with n vertices and m edges is charged
 * 40 m + 160 n bytes (its share of the union's edge set, sort buffers,
 * CSR and listing work arrays), and each batch the fixed buffers of one
 * listing call (output chunks and staging).  A request that cannot fit in
 * an empty server fails with TL_ENOMEM; otherwise it waits (first come,
 * first served: a request never overtakes an older one).
 *
 * Thread safety: submit and wait may be called from any threads.  The
 * registered graphs must stay alive, and must not be modified or freed,
 * until tl_server_free returns; tl_server_free waits for every submitted
 * request to finish. */
typedef struct tl_server tl_server; /* opaque */
typedef struct {
  size_t hbm_budget_bytes; /* device bytes admitted batches may hold (estimate) */
  uint32_t max_batch;      /* requests per batch, >= 1 */
  uint32_t workers;        /* batches in flight, >= 1 (one host thread + stream each) */
  size_t chunk_bytes;      /* output chunk of each listing, >= TL_MIN_CHUNK_BYTES */
} tl_server_config;
typedef struct {
  tl_status status;      /* TL_OK, or why the request failed */
  uint32_t batch_size;   /* requests listed in the same pass */
  uint64_t triangles;    /* number of triangles of the graph */
  uint64_t hash;         /* their set hash H */
  uint64_t t_submit_ns;  /* tl_server_now_ns() at submit, admission and completion */
  uint64_t t_admit_ns;
  uint64_t t_done_ns;
  int32_t tuning_entry;  /* entry of the tuning table used for its group, -1 = defaults */
} tl_request_result;
TL_EXPORT tl_status tl_server_create(tl_server **out, const tl_server_config *cfg);
/* Register g (caller-owned, loaded on the current device) -> *graph_id. */
TL_EXPORT tl_status tl_server_add_graph(tl_server *s, const tl_graph *g, uint32_t *graph_id);
/* Register an ordering of a registered graph: rank[v] = pi_v - 1, n uint32,
 * host or device pointer (read during the call).  The server builds and keeps
 * a copy of the graph with its DAG under this ordering (16 m + 24 n bytes of
 * device memory until tl_server_free).  Not a permutation -> TL_EINVAL. */
TL_EXPORT tl_status tl_server_add_ordering(tl_server *s, uint32_t graph_id, const uint32_t *rank,
                                           int rank_on_device, uint32_t *ordering_id);
/* Work splits by degree profile for the server's batches (see tl_tuning and
 * tl_work_profile): before each algorithm group of a batch is listed, its
 * work profile is computed on the device and the group takes the tuning of
 * the nearest entry of the same algorithm, the distance being the L1
 * distance of the normalised profile marginals (by bit length of p and of
 * W) plus |log2 m - log2_m| / 8, m the batch's edge count.  count = 0 (or
 * entries NULL) restores the defaults.  The table is copied; it applies to
 * batches that start after the call.  Entries are those of
 * paper_2203_04774_gb300/tuning_table.json (autotune.py). */
typedef struct {
  tl_alg alg;
  double profile_p[TL_PROFILE_BINS_P];
  double profile_w[TL_PROFILE_BINS_W];
  double log2_m;
  tl_tuning tuning;
} tl_tuning_entry;
TL_EXPORT tl_status tl_server_set_tuning_table(tl_server *s, const tl_tuning_entry *entries,
                                               uint32_t count);
/* Queue a request; returns at once with its id. */
TL_EXPORT tl_status tl_server_submit(tl_server *s, uint32_t graph_id, uint32_t ordering_id,
                                     tl_alg alg, uint64_t *request_id);
/* Block until the request has finished and return its result (each id can
 * be waited for once, by one thread).  An unknown id, or an id another
 * thread is already waiting for -> TL_EINVAL. */
TL_EXPORT tl_status tl_server_wait(tl_server *s, uint64_t request_id, tl_request_result *out);
/* Finish every submitted request, stop the workers, release the server's
 * device memory.  NULL is a no-op. */
TL_EXPORT void tl_server_free(tl_server *s);
/* The admission charges: *request_bytes for one request on graph_id (may be
 * NULL) and *batch_bytes for every batch (may be NULL). */
TL_EXPORT tl_status tl_server_footprint(const tl_server *s, uint32_t graph_id,
                                        uint64_t *request_bytes, uint64_t *batch_bytes);
/* The monotonic clock of the result timestamps, in nanoseconds. */
TL_EXPORT uint64_t tl_server_now_ns(void);

/* Device copies of the DAG (rank space), for inspection and tests.
 *   dir 0: N+ (out) lists, dir 1: N- (in) lists.
 *   off: n+1 uint64 offsets, adj: m uint32 neighbour ranks, both host
 *   pointers owned by the caller; rows sorted ascending. */
TL_EXPORT tl_status tl_graph_csr(const tl_graph *g, int dir, uint64_t *off, uint32_t *adj);

/* Counters of the last tl_list_triangles* call on this graph, for benches
 * and profiling.  kernel_ms are CUDA-event durations of the listing kernels
 * (index 0: small-, 1: medium-, 2: narrow-, 3: mid-, 4: large-vertex
 * kernel; see tl_tuning), recorded on the handle's stream around each
 * launch. */
#define TL_KERNELS 5
typedef struct {
  uint64_t launches;     /* listing kernel launches */
  uint64_t chunks;       /* chunks handed to the consumer */
  uint64_t triangles;    /* triangles listed */
  uint64_t probes;       /* membership tests performed */
  uint64_t tasks[TL_KERNELS];     /* tasks of each kernel */
  double kernel_ms[TL_KERNELS];   /* summed device time of each kernel */
  uint64_t kernel_probes[TL_KERNELS];     /* membership tests done by each kernel */
  uint64_t kernel_triangles[TL_KERNELS];  /* triangles found by each kernel */
  double bucketize_ms;           /* host wall time of the work split (a6) */
  double consumer_ms;            /* host wall time inside the consumer */
  double wall_ms;                /* host wall time of the whole call */
} tl_list_stats;
TL_EXPORT tl_status tl_last_list_stats(const tl_graph *g, tl_list_stats *out);

/* Number of CUDA kernels this library has launched since it was loaded
 * (all threads, all graphs). */
TL_EXPORT uint64_t tl_kernel_launches(void);

/* Release the graph and all of its device memory.  NULL is a no-op. */
TL_EXPORT void tl_graph_free(tl_graph *g);

/* Message of the last failed call on this thread ("" if none). */
TL_EXPORT const char *tl_last_error(void);

/* Library version string. */
TL_EXPORT const char *tl_version(void);

#ifdef __cplusplus
}
#endif
#endif /* TL_H_ */
