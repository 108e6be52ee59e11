// C ABI of libtl (declared in include/tl.h).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "list.cuh"

namespace tl {

namespace {
thread_local std::string g_last_error;
std::atomic<uint64_t> g_launches{0};
}

void set_error(const std::string &msg) { g_last_error = msg; }
void clear_error() { g_last_error.clear(); }
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

cudaMemPool_t device_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  TL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) fail(TL_EINVAL, "device index out of range");
  cudaMemPool_t p;
  {
    std::lock_guard<std::mutex> lock(mu);
    if (!pools[dev]) TL_CUDA(cudaDeviceGetDefaultMemPool(&pools[dev], dev));
    p = pools[dev];
  }
  // The threshold counts every reserved byte, in use or not: keep it 32 GiB
  // above what is in use, so that up to 32 GiB of freed buffers stay cached
  // for the next call however much long-lived memory (resident graphs) the
  // pool holds, and the rest goes back to the driver at sync points.
  uint64_t used = 0;
  TL_CUDA(cudaMemPoolGetAttribute(p, cudaMemPoolAttrUsedMemCurrent, &used));
  uint64_t keep = used + (32ull << 30);
  TL_CUDA(cudaMemPoolSetAttribute(p, cudaMemPoolAttrReleaseThreshold, &keep));
  return p;
}

namespace {

// Pinned host copy of the control block (one per graph).
struct PinnedCtl {
  ListCtl *h = nullptr;
  PinnedCtl() {
    TL_CUDA(cudaMallocHost(&h, sizeof(ListCtl)));
    std::memset(h, 0, sizeof(ListCtl));
  }
  ~PinnedCtl() {
    if (h) cudaFreeHost(h);
  }
};

}  // namespace
}  // namespace tl

namespace {
tl_tuning tl_default_tuning_value() {
  tl_tuning t;
  t.small_max_p = tl::kSmallMaxP;
  t.medium_max_p = tl::kMediumMaxP;
  t.narrow_max_p = tl::kNarrowMaxP;
  t.mid_max_p = tl::kMidMaxP;
  t.warp_work = (uint32_t)tl::kWarpWorkMax;
  t.narrow_piece = 1u << 14;
  t.mid_piece = 1u << 16;
  t.large_per_p = 64;
  t.large_min = 1u << 16;
  t.large_max = 1u << 22;
  t.narrow_keep_mib = 0;
  t.narrow_cold_first = 0;
  t.large_hash_max_p = tl::kHashMaxSlots / 2;
  return t;
}
}  // namespace

struct tl_graph {
  tl::DeviceGraph g;
  // listing workspace
  tl::DevBuf wseed, WP, ctl, chunks, slabs, retry, rretry, ghash;
  uint64_t rretry_cap = 0;  // RetryPiece records per half of rretry
  // per-vertex classification (tiers 0, 1: weights and flags; tiers 2, 3: pieces),
  // their prefixes, and the compacted vertex lists of tiers 0 and 1
  tl::DevBuf tw[2], tf[2], tpref[2], tpos[2], tx[2], twp[2], tstart[2], pieces[3],
      piece_prefix[3], task_x[3];
  tl::PinnedCtl *pctl = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr};
  tl_list_stats stats{};
  int cached_alg = -1;
  int wp_alg = -1;  // the algorithm WP was computed for (-1: none)
  uint32_t cached_xb = 0, cached_xe = 0;
  uint64_t n_tasks[tl::kTiers] = {0, 0, 0, 0, 0};
  // the work split: as set by tl_set_tuning, and as used by the cached tables
  tl_tuning tuning = tl_default_tuning_value();
  tl::Tuning used_tu{};
  uint64_t tier_count[2] = {0, 0};
  void bind(cudaStream_t s) {
    g.bind(s);
    for (tl::DevBuf *b : {&wseed, &WP, &ctl, &chunks, &slabs, &retry, &rretry, &ghash})
      b->stream = s;
    for (int t = 0; t < 2; ++t)
      for (tl::DevBuf *b : {&tw[t], &tf[t], &tpref[t], &tpos[t], &tx[t], &twp[t], &tstart[t]})
        b->stream = s;
    for (int t = 0; t < 3; ++t)
      for (tl::DevBuf *b : {&pieces[t], &piece_prefix[t], &task_x[t]}) b->stream = s;
  }
  ~tl_graph() {
    delete pctl;
    for (auto &e : ev)
      if (e) cudaEventDestroy(e);
  }
};

#define TL_API_BEGIN \
  try {              \
    tl::clear_error();
#define TL_API_END                                           \
  }                                                          \
  catch (const tl::Error &e) {                               \
    tl::set_error(e.msg);                                    \
    return e.status;                                         \
  }                                                          \
  catch (const std::bad_alloc &) {                           \
    tl::set_error("host allocation failed");                 \
    return TL_ENOMEM;                                        \
  }                                                          \
  catch (...) {                                              \
    tl::set_error("unexpected internal error");              \
    return TL_ECUDA;                                         \
  }                                                          \
  return TL_OK;

namespace {

// Build the DAG of the identity ordering if no ordering has been applied yet.
void ensure_ordered(tl_graph *G) {
  if (!G->g.ordered) {
    G->cached_alg = -1;
    G->wp_alg = -1;
    tl::build_dag(G->g, nullptr, true);
  }
}

void require_device() {
  int count = 0;
  cudaError_t e = cudaGetDeviceCount(&count);
  if (e != cudaSuccess || count == 0)
    tl::fail(TL_ECUDA, std::string("no usable CUDA device: ") +
                           (e != cudaSuccess ? cudaGetErrorString(e) : "device count is 0"));
}

// The three CSR roles of one algorithm (Sec. 2.1): the probe set P_x put in
// B, the seeds y of x, and the list scanned for each seed.
//   A++ (seed edge L):  P_x = N-_x, seeds N-_x, scan N+_y
//   A+- (seed edge S1): P_x = N+_x, seeds N+_x, scan N+_y
//   A-- (seed edge S2): P_x = N-_x, seeds N+_x, scan N-_y
struct Sides {
  const uint64_t *poff, *soff, *scan_off;
  const uint32_t *padj, *sadj, *scan_adj;
};
Sides sides(const tl::DeviceGraph &g, int alg) {
  const uint64_t *io = g.in_off.as<uint64_t>(), *oo = g.out_off.as<uint64_t>();
  const uint32_t *ia = g.in_adj.as<uint32_t>(), *oa = g.out_adj.as<uint32_t>();
  if (alg == TL_APP) return Sides{io, io, oo, ia, ia, oa};
  if (alg == TL_APM) return Sides{oo, oo, oo, oa, oa, oa};
  return Sides{io, oo, io, ia, oa, ia};
}

template <class T>
T read_dev(const T *p, cudaStream_t s) {
  T v;
  TL_CUDA(cudaMemcpyAsync(&v, p, sizeof(T), cudaMemcpyDeviceToHost, s));
  TL_CUDA(cudaStreamSynchronize(s));
  return v;
}

// The work split used for one listing: the caller's tuning, with large pieces
// capped at 1/16 of an even share of the range's work per large-vertex CTA,
// so that no single piece holds up the end of the launch on a small graph.
tl::Tuning effective_tuning(const tl_tuning &t, uint64_t range_work) {
  tl::Tuning tu;
  tu.small_max_p = t.small_max_p;
  tu.medium_max_p = t.medium_max_p;
  tu.narrow_max_p = t.narrow_max_p;
  tu.mid_max_p = t.mid_max_p;
  tu.warp_work = t.warp_work;
  tu.narrow_piece = t.narrow_piece;
  tu.mid_piece = t.mid_piece;
  tu.large_per_p = t.large_per_p;
  tu.large_min = t.large_min;
  tu.narrow_keep_mib = t.narrow_keep_mib;
  tu.narrow_cold_first = t.narrow_cold_first;
  tu.large_hash_max_p = t.large_hash_max_p;
  const uint64_t cap = range_work / (16ull * (uint64_t)tl::tier_grid(tl::kTierLarge));
  uint64_t mx = std::min<uint64_t>(t.large_max, std::max<uint64_t>(cap, t.large_min));
  tu.large_max = (uint32_t)mx;
  return tu;
}

bool same_tuning(const tl::Tuning &a, const tl::Tuning &b) {
  return a.small_max_p == b.small_max_p && a.medium_max_p == b.medium_max_p &&
         a.narrow_max_p == b.narrow_max_p && a.mid_max_p == b.mid_max_p &&
         a.warp_work == b.warp_work && a.narrow_piece == b.narrow_piece &&
         a.mid_piece == b.mid_piece && a.large_per_p == b.large_per_p &&
         a.large_min == b.large_min && a.large_max == b.large_max &&
         a.large_hash_max_p == b.large_hash_max_p;
}

// WP, the exclusive prefix of the scanned-list lengths over all seed-side
// entries of one algorithm (the flat work space; kept until the DAG changes).
void ensure_wp(tl_graph *G, int alg) {
  if (G->wp_alg == alg) return;
  tl::DeviceGraph &g = G->g;
  cudaStream_t s = g.stream;
  const uint64_t m = g.m;
  const Sides sd = sides(g, alg);
  G->wseed.reserve((m ? m : 1) * 4);
  G->WP.reserve((m + 1) * 8);
  if (m) tl::launch_seed_work(sd.sadj, m, sd.scan_off, G->wseed.as<uint32_t>(), s);
  tl::exclusive_scan_u32_to_u64(G->wseed.as<uint32_t>(), G->WP.as<uint64_t>(), m, g.scan_tmp, s);
  G->wp_alg = alg;
  G->cached_alg = -1;  // task tables of another algorithm used the old WP
}

// a6: per-seed-edge work prefix and the task counts of every kernel.
void bucketize(tl_graph *G, int alg, uint32_t xb, uint32_t xe) {
  tl::DeviceGraph &g = G->g;
  cudaStream_t s = g.stream;
  const Sides sd = sides(g, alg);
  ensure_wp(G, alg);
  G->ctl.reserve(sizeof(tl::ListCtl));
  uint64_t *rw = reinterpret_cast<uint64_t *>(G->ctl.p);  // scratch before the launches
  tl::launch_range_work(sd.soff, G->WP.as<uint64_t>(), xb, xe, rw, s);
  const uint64_t range_work = read_dev(rw, s);
  const tl::Tuning tu = effective_tuning(G->tuning, range_work);
  if (G->cached_alg == alg && G->cached_xb == xb && G->cached_xe == xe &&
      same_tuning(tu, G->used_tu))
    return;
  const uint64_t nr = xe - xb;
  const uint64_t nr1 = nr ? nr : 1;
  for (int t = 0; t < 2; ++t) {
    G->tw[t].reserve(nr1 * 8);
    G->tf[t].reserve(nr1 * 4);
    G->tpref[t].reserve((nr + 1) * 8);
    G->tpos[t].reserve((nr + 1) * 8);
    G->tx[t].reserve(nr1 * 4);
    G->twp[t].reserve((nr + 1) * 8);
  }
  for (int t = 0; t < 3; ++t) {
    G->pieces[t].reserve(nr1 * 8);
    G->piece_prefix[t].reserve((nr + 1) * 8);
  }
  if (nr)
    tl::launch_classify(sd.poff, sd.soff, G->WP.as<uint64_t>(), xb, xe, tu,
                        G->tw[0].as<uint64_t>(), G->tw[1].as<uint64_t>(),
                        G->tf[0].as<uint32_t>(), G->tf[1].as<uint32_t>(),
                        G->pieces[0].as<uint64_t>(), G->pieces[1].as<uint64_t>(),
                        G->pieces[2].as<uint64_t>(), s);
  for (int t = 0; t < 2; ++t) {
    tl::exclusive_scan_u64(G->tw[t].as<uint64_t>(), G->tpref[t].as<uint64_t>(), nr, g.scan_tmp, s);
    tl::exclusive_scan_u32_to_u64(G->tf[t].as<uint32_t>(), G->tpos[t].as<uint64_t>(), nr,
                                  g.scan_tmp, s);
    tl::launch_compact_tier(G->tf[t].as<uint32_t>(), G->tpos[t].as<uint64_t>(),
                            G->tpref[t].as<uint64_t>(), xb, nr, G->tx[t].as<uint32_t>(),
                            G->twp[t].as<uint64_t>(), s);
  }
  for (int t = 0; t < 3; ++t)
    tl::exclusive_scan_u64(G->pieces[t].as<uint64_t>(), G->piece_prefix[t].as<uint64_t>(), nr,
                           g.scan_tmp, s);
  // totals: weights of tiers 0 and 1, their vertex counts, pieces of tiers 2, 3 and 4
  uint64_t tot[7];
  TL_CUDA(cudaMemcpyAsync(&tot[0], G->tpref[0].as<uint64_t>() + nr, 8, cudaMemcpyDeviceToHost, s));
  TL_CUDA(cudaMemcpyAsync(&tot[1], G->tpref[1].as<uint64_t>() + nr, 8, cudaMemcpyDeviceToHost, s));
  TL_CUDA(cudaMemcpyAsync(&tot[2], G->tpos[0].as<uint64_t>() + nr, 8, cudaMemcpyDeviceToHost, s));
  TL_CUDA(cudaMemcpyAsync(&tot[3], G->tpos[1].as<uint64_t>() + nr, 8, cudaMemcpyDeviceToHost, s));
  for (int t = 0; t < 3; ++t)
    TL_CUDA(cudaMemcpyAsync(&tot[4 + t], G->piece_prefix[t].as<uint64_t>() + nr, 8,
                            cudaMemcpyDeviceToHost, s));
  TL_CUDA(cudaStreamSynchronize(s));
  G->n_tasks[0] = (tot[0] + tu.warp_work - 1) / tu.warp_work;
  G->n_tasks[1] = (tot[1] + tu.warp_work - 1) / tu.warp_work;
  for (int t = 0; t < 3; ++t) G->n_tasks[2 + t] = tot[4 + t];
  G->tier_count[0] = tot[2];
  G->tier_count[1] = tot[3];
  for (int t = 0; t < 2; ++t) {
    G->tstart[t].reserve((G->n_tasks[t] + 1) * 4);
    tl::launch_task_bounds(G->twp[t].as<uint64_t>(), G->tier_count[t], G->n_tasks[t],
                           tu.warp_work, G->tstart[t].as<uint32_t>(), s);
  }
  for (int t = 0; t < 3; ++t) {
    G->task_x[t].reserve((G->n_tasks[2 + t] ? G->n_tasks[2 + t] : 1) * 4);
    tl::launch_task_owner(G->piece_prefix[t].as<uint64_t>(), xb, nr, G->task_x[t].as<uint32_t>(),
                          s);
  }
  G->cached_alg = alg;
  G->cached_xb = xb;
  G->cached_xe = xe;
  G->used_tu = tu;
}

struct Phase {
  int kind;
  uint64_t n_tasks;
  uint64_t fresh = 0;
  uint32_t n_retry = 0;
};

tl_status list_impl(tl_graph *G, int alg, uint32_t xb, uint32_t xe, size_t chunk_bytes,
                    tl_consumer cb, void *user, uint64_t *n_triangles, uint64_t *n_probes) {
  TL_API_BEGIN
  if (!G) tl::fail(TL_EINVAL, "graph is NULL");
  if (alg != TL_APP && alg != TL_APM && alg != TL_AMM)
    tl::fail(TL_EINVAL, "alg must be TL_APP, TL_APM or TL_AMM");
  tl::DeviceGraph &g = G->g;
  ensure_ordered(G);
  if (xb > xe || xe > g.n) tl::fail(TL_EINVAL, "seed range outside [0, n]");
  if (chunk_bytes < TL_MIN_CHUNK_BYTES) tl::fail(TL_EINVAL, "chunk_bytes below TL_MIN_CHUNK_BYTES");
  const uint64_t cap = chunk_bytes / 12;
  if (cap < tl::kSlabCap) tl::fail(TL_EINVAL, "chunk too small for one task");
  cudaStream_t s = g.stream;
  const auto t_call = std::chrono::steady_clock::now();
  auto ms_since = [](std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0)
        .count();
  };
  bucketize(G, alg, xb, xe);
  const double bucketize_ms = ms_since(t_call);

  uint64_t slab_words = 0, max_tasks = 1;
  for (int t = 0; t < 2; ++t) {  // warp tiers: one global slab per warp
    const uint64_t w = (uint64_t)tl::tier_grid(t) * (tl::kWarpThreads / 32) * tl::slab_cap(t);
    slab_words = w > slab_words ? w : slab_words;
    max_tasks = G->n_tasks[t] > max_tasks ? G->n_tasks[t] : max_tasks;
  }
  G->chunks.reserve(2 * cap * 12);
  G->slabs.reserve(slab_words * 12);
  // hub tables in global memory, needed only when the bitmap over all ranks
  // does not fit in shared memory
  const bool need_ghash = g.n > tl::kBitmapMaxN && G->n_tasks[tl::kTierLarge] > 0;
  if (need_ghash)
    G->ghash.reserve((uint64_t)tl::tier_grid(tl::kTierLarge) * tl::kGHashSlots * 4);
  G->retry.reserve(2 * max_tasks * 4);
  G->ctl.reserve(sizeof(tl::ListCtl));
  if (!G->pctl) G->pctl = new tl::PinnedCtl();
  tl::ListCtl *hc = G->pctl->h;
  uint32_t *chunk[2] = {G->chunks.as<uint32_t>(), G->chunks.as<uint32_t>() + 3 * cap};
  uint32_t *retry[2] = {G->retry.as<uint32_t>(), G->retry.as<uint32_t>() + max_tasks};
  // CTA tiers: a launch queues at most one record per CTA and piece, and a
  // CTA runs at most two pieces after the chunk fills (the current one and
  // the one it had already fetched); plus the records it did not fetch
  const uint64_t warps_cta =
      2 * std::max<uint64_t>({(uint64_t)tl::tier_grid(tl::kTierNarrow),
                              (uint64_t)tl::tier_grid(tl::kTierMid),
                              (uint64_t)tl::tier_grid(tl::kTierLarge)});
  auto rr_half = [&](int h) { return G->rretry.as<tl::RetryPiece>() + h * G->rretry_cap; };
  auto reserve_ranges = [&](int in_half, uint64_t n_in, uint64_t need) {
    if (need <= G->rretry_cap) return;
    const uint64_t cap2 = std::max<uint64_t>(need, 2 * G->rretry_cap);
    tl::DevBuf nb(s);
    nb.reserve(2 * cap2 * sizeof(tl::RetryPiece));
    if (n_in)
      TL_CUDA(cudaMemcpyAsync(nb.as<tl::RetryPiece>() + in_half * cap2, rr_half(in_half),
                              n_in * sizeof(tl::RetryPiece), cudaMemcpyDeviceToDevice, s));
    std::swap(G->rretry.p, nb.p);
    std::swap(G->rretry.bytes, nb.bytes);
    G->rretry_cap = cap2;
  };

  tl::ListArgs a{};
  a.n = g.n;
  a.x_begin = xb;
  a.x_end = xe;
  const Sides sd = sides(g, alg);
  a.poff = sd.poff;
  a.padj = sd.padj;
  a.soff = sd.soff;
  a.sadj = sd.sadj;
  a.scan_off = sd.scan_off;
  a.scan_adj = sd.scan_adj;
  a.inv = g.inv.as<uint32_t>();
  a.WP = G->WP.as<uint64_t>();
  a.ctl = G->ctl.as<tl::ListCtl>();
  a.chunk_cap = cap;
  a.slabs = G->slabs.as<uint32_t>();
  a.ghash = need_ghash ? G->ghash.as<uint32_t>() : nullptr;
  a.tu = G->used_tu;
  {
    // L2 priority of the narrow kernel's short-step loads; the scanned CSR
    // holds m entries in rank order, so the highest ranks' lists end it
    const uint64_t keep = (uint64_t)G->tuning.narrow_keep_mib << 18;  // 4-byte entries
    a.l2_keep_from = keep == 0 ? ~0ull : (g.m > keep ? g.m - keep : 0);
    a.l2_cold_first = G->tuning.narrow_cold_first;
  }

  if (!G->ev[0]) {
    TL_CUDA(cudaEventCreate(&G->ev[0]));
    TL_CUDA(cudaEventCreate(&G->ev[1]));
  }
  tl_list_stats st{};
  for (int t = 0; t < tl::kTiers; ++t) st.tasks[t] = G->n_tasks[t];
  G->stats = st;
  constexpr int kPhases = tl::kTiers;
  Phase phases[kPhases] = {{0, G->n_tasks[0]},
                           {1, G->n_tasks[1]},
                           {2, G->n_tasks[2]},
                           {3, G->n_tasks[3]},
                           {4, G->n_tasks[4]}};
  int cur = 0, rsel = 0;
  uint64_t filled = 0, chunk_idx = 0, total_tri = 0, total_probes = 0;
  int pending = -1;
  uint64_t pending_n = 0;
  bool stopped = false;
  int ph = 0;
  double consumer_ms = 0;
  auto deliver = [&](int which, uint64_t cnt) {
    if (cb && cnt > 0 && !stopped) {
      const auto t0 = std::chrono::steady_clock::now();
      if (cb(chunk[which], cnt, chunk_idx, user) != 0) stopped = true;
      consumer_ms += ms_since(t0);
    }
    if (cnt > 0) ++chunk_idx;
    st.chunks = chunk_idx;
  };
  for (;;) {
    while (ph < kPhases && phases[ph].fresh >= phases[ph].n_tasks && phases[ph].n_retry == 0) ++ph;
    const bool launch = ph < kPhases && !stopped;
    Phase *P = launch ? &phases[ph] : nullptr;
    if (launch) {
      std::memset(hc, 0, sizeof(*hc));
      hc->cursor = filled;
      hc->first_fail = ~0ull;
      TL_CUDA(cudaMemcpyAsync(a.ctl, hc, sizeof(*hc), cudaMemcpyHostToDevice, s));
      a.chunk = chunk[cur];
      a.n_retry = P->n_retry;
      if (P->kind < 2) {
        a.retry_in = retry[rsel];
        a.retry_out = retry[rsel ^ 1];
      } else {
        reserve_ranges(rsel, P->n_retry, P->n_retry + warps_cta);
        a.rr_in = rr_half(rsel);
        a.rr_out = rr_half(rsel ^ 1);
      }
      a.fresh_base = P->fresh;
      a.n_tasks = P->n_tasks;
      a.slab_cap = tl::slab_cap(P->kind);
      a.tier = P->kind;
      if (P->kind >= 2) {
        a.piece_prefix = G->piece_prefix[P->kind - 2].as<uint64_t>();
        a.task_x = G->task_x[P->kind - 2].as<uint32_t>();
      }
      if (P->kind < 2) {
        a.tier_x = G->tx[P->kind].as<uint32_t>();
        a.tier_wp = G->twp[P->kind].as<uint64_t>();
        a.task_start = G->tstart[P->kind].as<uint32_t>();
        a.tier_count = G->tier_count[P->kind];
      }
      TL_CUDA(cudaEventRecord(G->ev[0], s));
      tl::launch_list(P->kind, a, s);
      TL_CUDA(cudaEventRecord(G->ev[1], s));
      ++st.launches;
      TL_CUDA(cudaMemcpyAsync(hc, a.ctl, sizeof(*hc), cudaMemcpyDeviceToHost, s));
    }
    if (pending >= 0) {  // consumer runs while the next launch is in flight
      deliver(pending, pending_n);
      pending = -1;
    }
    if (!launch) break;
    TL_CUDA(cudaStreamSynchronize(s));
    {
      float ms = 0.f;
      TL_CUDA(cudaEventElapsedTime(&ms, G->ev[0], G->ev[1]));
      st.kernel_ms[P->kind] += ms;
    }
    // the reservations that fit are the chunk prefix [filled, valid_end)
    const uint64_t valid_end = hc->overflow ? std::min<uint64_t>(hc->first_fail, hc->cursor)
                                            : hc->cursor;
    const uint64_t launch_tri = valid_end - filled;
    total_tri += launch_tri;
    total_probes += hc->probes;
    st.kernel_triangles[P->kind] += launch_tri;
    st.kernel_probes[P->kind] += hc->probes;
    const uint32_t fetched = hc->fetch;
    const uint32_t used_retry = fetched < P->n_retry ? fetched : P->n_retry;
    uint64_t fresh_fetched = fetched > P->n_retry ? (uint64_t)(fetched - P->n_retry) : 0;
    if (fresh_fetched > P->n_tasks - P->fresh) fresh_fetched = P->n_tasks - P->fresh;
    uint32_t nr_out = hc->n_retry_out;
    if (used_retry < P->n_retry) {  // retry entries nobody fetched carry over
      const uint64_t left = P->n_retry - used_retry;
      if (P->kind < 2) {
        TL_CUDA(cudaMemcpyAsync(retry[rsel ^ 1] + nr_out, retry[rsel] + used_retry, left * 4,
                                cudaMemcpyDeviceToDevice, s));
      } else {
        TL_CUDA(cudaMemcpyAsync(rr_half(rsel ^ 1) + nr_out, rr_half(rsel) + used_retry,
                                left * sizeof(tl::RetryPiece), cudaMemcpyDeviceToDevice, s));
      }
      nr_out += (uint32_t)left;
    }
    const bool progress = valid_end > filled || fresh_fetched > 0 ||
                          nr_out < P->n_retry + fresh_fetched || hc->probes > 0;
    P->fresh += fresh_fetched;
    P->n_retry = nr_out;
    rsel ^= 1;
    filled = valid_end;
    if (hc->overflow) {
      if (filled == 0 && !progress) tl::fail(TL_ECUDA, "listing made no progress");
      pending = cur;
      pending_n = filled;
      cur ^= 1;
      filled = 0;
    }
  }
  if (!stopped && filled > 0) deliver(cur, filled);
  TL_CUDA(cudaStreamSynchronize(s));
  if (n_triangles) *n_triangles = total_tri;
  if (n_probes) *n_probes = total_probes;
  st.triangles = total_tri;
  st.probes = total_probes;
  st.bucketize_ms = bucketize_ms;
  st.consumer_ms = consumer_ms;
  st.wall_ms = ms_since(t_call);
  G->stats = st;
  if (stopped) tl::fail(TL_ECALLBACK, "the consumer asked to stop");
  TL_API_END
}

}  // namespace

extern "C" {

tl_status tl_graph_load(tl_graph **out, uint32_t n, const uint32_t *edges, uint64_t m_in,
                        int edges_on_device, void *stream) {
  TL_API_BEGIN
  if (!out) tl::fail(TL_EINVAL, "out is NULL");
  *out = nullptr;
  if (n == 0 || n == 0xffffffffu) tl::fail(TL_EINVAL, "n must be in [1, 2^32 - 2]");
  if (m_in > 0 && !edges) tl::fail(TL_EINVAL, "edges is NULL");
  require_device();
  tl_graph *G = new tl_graph();
  try {
    G->g.n = n;
    G->bind(static_cast<cudaStream_t>(stream));
    tl::build_edge_set(G->g, edges, m_in, edges_on_device != 0);
    // The identity ordering (the dataset's original one) is built lazily, on
    // the first call that needs a DAG before any tl_order_apply.
  } catch (...) {
    delete G;
    throw;
  }
  *out = G;
  TL_API_END
}

tl_status tl_graph_load_parts(tl_graph **out, uint32_t k, const uint32_t *n,
                              const uint64_t *m_in, const uint32_t *edges, int edges_on_device,
                              void *stream) {
  TL_API_BEGIN
  if (!out) tl::fail(TL_EINVAL, "out is NULL");
  *out = nullptr;
  if (k == 0 || !n || !m_in) tl::fail(TL_EINVAL, "k must be >= 1 and n, m_in non-NULL");
  uint64_t total = 0;
  for (uint32_t i = 0; i < k; ++i) {
    if (n[i] == 0) tl::fail(TL_EINVAL, "every part needs n >= 1");
    total += m_in[i];
  }
  if (total > 0 && !edges) tl::fail(TL_EINVAL, "edges is NULL");
  require_device();
  tl_graph *G = new tl_graph();
  try {
    G->bind(static_cast<cudaStream_t>(stream));
    tl::build_edge_set_parts(G->g, k, n, m_in, edges, edges_on_device != 0);
  } catch (...) {
    delete G;
    throw;
  }
  *out = G;
  TL_API_END
}

tl_status tl_graph_union(tl_graph **out, const tl_graph *const *graphs,
                         const uint32_t *const *rank, uint32_t k, void *stream) {
  TL_API_BEGIN
  if (!out) tl::fail(TL_EINVAL, "out is NULL");
  *out = nullptr;
  if (k == 0 || !graphs) tl::fail(TL_EINVAL, "k must be >= 1 and graphs non-NULL");
  std::vector<const tl::DeviceGraph *> parts(k);
  for (uint32_t i = 0; i < k; ++i) {
    if (!graphs[i]) tl::fail(TL_EINVAL, "a graph is NULL");
    parts[i] = &graphs[i]->g;
  }
  require_device();
  tl_graph *G = new tl_graph();
  try {
    G->bind(static_cast<cudaStream_t>(stream));
    tl::build_union(G->g, k, parts.data(), rank);
  } catch (...) {
    delete G;
    throw;
  }
  *out = G;
  TL_API_END
}

tl_status tl_graph_size(const tl_graph *G, uint32_t *n, uint64_t *m) {
  TL_API_BEGIN
  if (!G) tl::fail(TL_EINVAL, "graph is NULL");
  if (n) *n = G->g.n;
  if (m) *m = G->g.m;
  TL_API_END
}

tl_status tl_order_apply(tl_graph *G, const uint32_t *rank, int rank_on_device) {
  TL_API_BEGIN
  if (!G || !rank) tl::fail(TL_EINVAL, "graph or rank is NULL");
  G->cached_alg = -1;
  G->wp_alg = -1;
  tl::build_dag(G->g, rank, rank_on_device != 0);
  TL_API_END
}

tl_status tl_order_compute(tl_graph *G, tl_order_kind kind, uint32_t *rank, int rank_on_device) {
  TL_API_BEGIN
  if (!G || !rank) tl::fail(TL_EINVAL, "graph or rank is NULL");
  if (kind != TL_ORDER_DEGREE && kind != TL_ORDER_SPLIT && kind != TL_ORDER_CORE)
    tl::fail(TL_EINVAL, "kind must be TL_ORDER_DEGREE, TL_ORDER_SPLIT or TL_ORDER_CORE");
  tl::compute_order(G->g, kind, rank, rank_on_device != 0);
  TL_API_END
}

tl_status tl_cost(const tl_graph *G, tl_alg alg, uint64_t *cost) {
  TL_API_BEGIN
  if (!G || !cost) tl::fail(TL_EINVAL, "graph or cost is NULL");
  if (alg != TL_APP && alg != TL_APM && alg != TL_AMM)
    tl::fail(TL_EINVAL, "alg must be TL_APP, TL_APM or TL_AMM");
  ensure_ordered(const_cast<tl_graph *>(G));
  *cost = alg == TL_APP ? G->g.cost_app : (alg == TL_APM ? G->g.cost_apm : G->g.cost_amm);
  TL_API_END
}

tl_status tl_list_triangles(tl_graph *G, tl_alg alg, size_t chunk_bytes, tl_consumer cb,
                            void *user, uint64_t *n_triangles) {
  uint32_t n = G ? G->g.n : 0;
  return list_impl(G, alg, 0, n, chunk_bytes, cb, user, n_triangles, nullptr);
}

tl_status tl_list_triangles_range(tl_graph *G, tl_alg alg, uint32_t x_begin, uint32_t x_end,
                                  size_t chunk_bytes, tl_consumer cb, void *user,
                                  uint64_t *n_triangles, uint64_t *n_probes) {
  return list_impl(G, alg, x_begin, x_end, chunk_bytes, cb, user, n_triangles, n_probes);
}

int tl_count_hash(const uint32_t *dev_triples, uint64_t n_triples, uint64_t chunk_index,
                  void *user) {
  (void)chunk_index;
  tl_count_hash_state *st = static_cast<tl_count_hash_state *>(user);
  if (!st) return 1;
  cudaStream_t s = static_cast<cudaStream_t>(st->stream);
  if (!st->scratch) {
    if (cudaMalloc(&st->scratch, 64) != cudaSuccess) return 1;
  }
  unsigned long long *acc = static_cast<unsigned long long *>(st->scratch);
  unsigned long long h = 0;
  try {
    TL_CUDA(cudaMemsetAsync(acc, 0, 8, s));
    tl::launch_count_hash(dev_triples, n_triples, acc, s);
    TL_CUDA(cudaMemcpyAsync(&h, acc, 8, cudaMemcpyDeviceToHost, s));
    TL_CUDA(cudaStreamSynchronize(s));
  } catch (const tl::Error &e) {
    tl::set_error(e.msg);
    return 1;
  }
  st->count += n_triples;
  st->hash += h;
  return 0;
}

int tl_count_hash_parts(const uint32_t *dev_triples, uint64_t n_triples, uint64_t chunk_index,
                        void *user) {
  (void)chunk_index;
  tl_count_hash_parts_state *st = static_cast<tl_count_hash_parts_state *>(user);
  if (!st || !st->vbase || st->k == 0 || !st->counts || !st->hashes) {
    tl::set_error("tl_count_hash_parts: state needs vbase, k >= 1, counts and hashes");
    return 1;
  }
  cudaStream_t s = static_cast<cudaStream_t>(st->stream);
  try {
    tl::launch_count_hash_parts(dev_triples, n_triples, st->vbase, st->k,
                                reinterpret_cast<unsigned long long *>(st->counts),
                                reinterpret_cast<unsigned long long *>(st->hashes), s);
    TL_CUDA(cudaStreamSynchronize(s));
  } catch (const tl::Error &e) {
    tl::set_error(e.msg);
    return 1;
  }
  return 0;
}

void tl_count_hash_release(tl_count_hash_state *s) {
  if (s && s->scratch) {
    cudaFree(s->scratch);
    s->scratch = nullptr;
  }
}

tl_status tl_work_profile(tl_graph *G, tl_alg alg, uint32_t x_begin, uint32_t x_end,
                          uint64_t *hist) {
  TL_API_BEGIN
  if (!G || !hist) tl::fail(TL_EINVAL, "graph or hist is NULL");
  if (alg != TL_APP && alg != TL_APM && alg != TL_AMM)
    tl::fail(TL_EINVAL, "alg must be TL_APP, TL_APM or TL_AMM");
  ensure_ordered(G);
  tl::DeviceGraph &g = G->g;
  if (x_begin > x_end || x_end > g.n) tl::fail(TL_EINVAL, "seed range outside [0, n]");
  cudaStream_t s = g.stream;
  ensure_wp(G, alg);
  const Sides sd = sides(g, alg);
  constexpr uint64_t kBins = (uint64_t)tl::kProfileBinsP * tl::kProfileBinsW;
  tl::DevBuf h(s);
  h.reserve(kBins * 8);
  TL_CUDA(cudaMemsetAsync(h.p, 0, kBins * 8, s));
  tl::launch_work_profile(sd.poff, sd.soff, G->WP.as<uint64_t>(), x_begin, x_end,
                          h.as<unsigned long long>(), s);
  TL_CUDA(cudaMemcpyAsync(hist, h.p, kBins * 8, cudaMemcpyDeviceToHost, s));
  TL_CUDA(cudaStreamSynchronize(s));
  TL_API_END
}

tl_status tl_default_tuning(tl_tuning *out) {
  TL_API_BEGIN
  if (!out) tl::fail(TL_EINVAL, "out is NULL");
  *out = tl_default_tuning_value();
  TL_API_END
}

tl_status tl_set_tuning(tl_graph *G, const tl_tuning *t) {
  TL_API_BEGIN
  if (!G) tl::fail(TL_EINVAL, "graph is NULL");
  const tl_tuning v = t ? *t : tl_default_tuning_value();
  if (v.small_max_p > tl::kSmallMaxP || v.medium_max_p > tl::kMediumMaxP ||
      v.narrow_max_p > tl::kNarrowMaxP || v.mid_max_p > tl::kMidMaxP)
    tl::fail(TL_EINVAL, "a probe-set threshold is above what its kernel's table holds "
                        "(32, 1024, 256, 2048)");
  if (v.warp_work < 256 || v.warp_work > tl::kWarpWorkMax)
    tl::fail(TL_EINVAL, "warp_work must be in [256, 4096]");
  if (v.narrow_piece < 1024 || v.mid_piece < 1024 || v.large_min < 1024)
    tl::fail(TL_EINVAL, "narrow_piece, mid_piece and large_min must be >= 1024");
  if (v.large_per_p < 1 || v.large_max < v.large_min)
    tl::fail(TL_EINVAL, "large_per_p must be >= 1 and large_max >= large_min");
  if (v.narrow_keep_mib > 4096 || v.narrow_cold_first > 1)
    tl::fail(TL_EINVAL, "narrow_keep_mib must be <= 4096 and narrow_cold_first 0 or 1");
  if (v.large_hash_max_p > tl::kHashMaxSlots / 2)
    tl::fail(TL_EINVAL, "large_hash_max_p must be <= 16384");
  G->tuning = v;
  TL_API_END
}

tl_status tl_get_tuning(const tl_graph *G, tl_tuning *out) {
  TL_API_BEGIN
  if (!G || !out) tl::fail(TL_EINVAL, "NULL argument");
  *out = G->tuning;
  TL_API_END
}

tl_status tl_graph_csr(const tl_graph *G, int dir, uint64_t *off, uint32_t *adj) {
  TL_API_BEGIN
  if (!G || !off || !adj) tl::fail(TL_EINVAL, "NULL argument");
  if (dir != 0 && dir != 1) tl::fail(TL_EINVAL, "dir must be 0 (N+) or 1 (N-)");
  ensure_ordered(const_cast<tl_graph *>(G));
  const tl::DeviceGraph &g = G->g;
  const tl::DevBuf &o = dir == 0 ? g.out_off : g.in_off;
  const tl::DevBuf &d = dir == 0 ? g.out_adj : g.in_adj;
  TL_CUDA(cudaMemcpyAsync(off, o.p, ((uint64_t)g.n + 1) * 8, cudaMemcpyDeviceToHost, g.stream));
  if (g.m) TL_CUDA(cudaMemcpyAsync(adj, d.p, g.m * 4, cudaMemcpyDeviceToHost, g.stream));
  TL_CUDA(cudaStreamSynchronize(g.stream));
  TL_API_END
}

tl_status tl_last_list_stats(const tl_graph *G, tl_list_stats *out) {
  TL_API_BEGIN
  if (!G || !out) tl::fail(TL_EINVAL, "NULL argument");
  *out = G->stats;
  TL_API_END
}

uint64_t tl_kernel_launches(void) { return tl::g_launches.load(); }

void tl_graph_free(tl_graph *G) { delete G; }

const char *tl_last_error(void) { return tl::g_last_error.c_str(); }

const char *tl_version(void) { return "tl 0.1 (sm_103a)"; }

}  // extern "C"
