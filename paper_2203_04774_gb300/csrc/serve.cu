// Serving: a request loop with admission by device footprint and continuous
// batching of requests into disjoint unions (declared in include/tl.h).
//
// Host code only.  Each worker thread owns a CUDA stream (plus one for the
// consumer's reductions) and runs one batch at a time: union of the batch's
// graphs under the requested orderings (tl_graph_union), one listing range per
// algorithm, per-part count + hash (tl_count_hash_parts), results.  Workers
// take requests from one FIFO queue under a mutex; admission charges an
// estimated footprint against the budget and releases it when the batch ends.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <memory>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "list.cuh"

namespace {

uint64_t now_ns() {
  return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

struct Request {
  uint64_t id = 0;
  const tl_graph *g = nullptr;  // the prepared handle, copied from the registry at
  uint32_t n = 0;               // submit so that workers never read the registry
  tl_alg alg = TL_APP;
  uint64_t footprint = 0;
  bool done = false;
  bool waited = false;  // a thread is waiting for it (at most one may)
  tl_request_result res{};
};

struct GraphEntry {
  const tl_graph *g = nullptr;
  uint32_t n = 0;
  uint64_t m = 0;
  // one handle per registered ordering, owned by the server: a copy of the
  // graph with its DAG built under that ordering, so that a batch's union
  // only concatenates the parts' arrays
  std::vector<tl_graph *> prepared;
};

struct Worker {
  std::thread th;
  cudaStream_t stream = nullptr, cstream = nullptr;
  uint64_t *d_vbase = nullptr, *d_counts = nullptr, *d_hashes = nullptr;  // max_batch (+1)
};

}  // namespace

struct tl_server {
  tl_server_config cfg{};
  int device = 0;
  uint64_t batch_fixed = 0;  // bytes one listing call holds whatever the graphs
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request *> pending;
  std::unordered_map<uint64_t, Request *> requests;
  std::vector<GraphEntry> graphs;
  cudaStream_t reg_stream = nullptr;  // prepared handles are built (and freed) on it
  std::mutex reg_mu;                  // one registration at a time on reg_stream
  uint64_t in_use = 0, next_id = 1;
  bool stop = false;
  std::vector<Worker> workers;
  // work splits by degree profile; replaced whole, read by workers under mu
  std::shared_ptr<const std::vector<tl_tuning_entry>> tuning;
};

namespace {

uint64_t footprint(uint32_t n, uint64_t m) { return 40 * m + 160 * (uint64_t)n; }

// The entry of `table` for `alg` nearest to the work profile of ranks
// [xb, xe) of u (see tl_server_set_tuning_table), or -1.
int nearest_entry(tl_graph *u, tl_alg alg, uint32_t xb, uint32_t xe,
                  const std::vector<tl_tuning_entry> &table, tl_status &st) {
  bool any = false;
  for (const auto &e : table) any = any || e.alg == alg;
  if (!any) return -1;
  std::vector<uint64_t> h((size_t)TL_PROFILE_BINS_P * TL_PROFILE_BINS_W);
  st = tl_work_profile(u, alg, xb, xe, h.data());
  if (st != TL_OK) return -1;
  double p[TL_PROFILE_BINS_P] = {}, w[TL_PROFILE_BINS_W] = {}, tot = 0;
  for (int i = 0; i < TL_PROFILE_BINS_P; ++i)
    for (int j = 0; j < TL_PROFILE_BINS_W; ++j) {
      const double v = (double)h[(size_t)i * TL_PROFILE_BINS_W + j];
      p[i] += v;
      w[j] += v;
      tot += v;
    }
  if (tot > 0) {
    for (double &v : p) v /= tot;
    for (double &v : w) v /= tot;
  }
  uint32_t n = 0;
  uint64_t m = 0;
  tl_graph_size(u, &n, &m);
  const double lm = std::log2((double)(m ? m : 1));
  int best = -1;
  double bd = 0;
  for (size_t k = 0; k < table.size(); ++k) {
    const tl_tuning_entry &e = table[k];
    if (e.alg != alg) continue;
    double d = std::fabs(lm - e.log2_m) / 8.0;
    for (int i = 0; i < TL_PROFILE_BINS_P; ++i) d += std::fabs(p[i] - e.profile_p[i]);
    for (int j = 0; j < TL_PROFILE_BINS_W; ++j) d += std::fabs(w[j] - e.profile_w[j]);
    if (best < 0 || d < bd) {
      best = (int)k;
      bd = d;
    }
  }
  return best;
}

// Runs one batch on worker W; fills every request's result (not `done`).
void run_batch(tl_server *S, Worker &W, std::vector<Request *> &batch) {
  std::stable_sort(batch.begin(), batch.end(),
                   [](const Request *a, const Request *b) { return a->alg < b->alg; });
  const uint32_t k = (uint32_t)batch.size();
  std::vector<const tl_graph *> parts(k);
  std::vector<uint64_t> vb(k + 1, 0);
  for (uint32_t i = 0; i < k; ++i) {
    parts[i] = batch[i]->g;
    vb[i + 1] = vb[i] + batch[i]->n;
  }
  tl_status st = TL_OK;
  std::vector<uint64_t> counts(k, 0), hashes(k, 0);
  tl_graph *u = nullptr;
  if (cudaSetDevice(S->device) != cudaSuccess) st = TL_ECUDA;
  // the parts keep their own orderings: the union concatenates their DAGs
  if (st == TL_OK) st = tl_graph_union(&u, parts.data(), nullptr, k, W.stream);
  if (st == TL_OK) {
    tl_count_hash_parts_state cs{W.d_vbase, k, W.d_counts, W.d_hashes, W.cstream};
    bool ok = cudaMemcpyAsync(W.d_vbase, vb.data(), (k + 1) * 8, cudaMemcpyHostToDevice,
                              W.cstream) == cudaSuccess &&
              cudaMemsetAsync(W.d_counts, 0, k * 8, W.cstream) == cudaSuccess &&
              cudaMemsetAsync(W.d_hashes, 0, k * 8, W.cstream) == cudaSuccess &&
              cudaStreamSynchronize(W.cstream) == cudaSuccess;
    if (!ok) st = TL_ECUDA;
    std::shared_ptr<const std::vector<tl_tuning_entry>> table;
    {
      std::lock_guard<std::mutex> lk(S->mu);
      table = S->tuning;
    }
    // one listing range per run of requests with the same algorithm, under
    // the work split of the table entry nearest to that range's profile
    for (uint32_t i = 0; st == TL_OK && i < k;) {
      uint32_t j = i;
      while (j < k && batch[j]->alg == batch[i]->alg) ++j;
      int e = -1;
      if (table && !table->empty())
        e = nearest_entry(u, batch[i]->alg, (uint32_t)vb[i], (uint32_t)vb[j], *table, st);
      if (st == TL_OK) st = tl_set_tuning(u, e >= 0 ? &(*table)[e].tuning : nullptr);
      for (uint32_t q = i; q < j; ++q) batch[q]->res.tuning_entry = e;
      if (st == TL_OK)
        st = tl_list_triangles_range(u, batch[i]->alg, (uint32_t)vb[i], (uint32_t)vb[j],
                                     S->cfg.chunk_bytes, tl_count_hash_parts, &cs, nullptr,
                                     nullptr);
      i = j;
    }
    if (st == TL_OK) {
      ok = cudaMemcpyAsync(counts.data(), W.d_counts, k * 8, cudaMemcpyDeviceToHost,
                           W.cstream) == cudaSuccess &&
           cudaMemcpyAsync(hashes.data(), W.d_hashes, k * 8, cudaMemcpyDeviceToHost,
                           W.cstream) == cudaSuccess &&
           cudaStreamSynchronize(W.cstream) == cudaSuccess;
      if (!ok) st = TL_ECUDA;
    }
  }
  if (u) tl_graph_free(u);
  for (uint32_t i = 0; i < k; ++i) {
    batch[i]->res.status = st;
    batch[i]->res.batch_size = k;
    batch[i]->res.triangles = st == TL_OK ? counts[i] : 0;
    batch[i]->res.hash = st == TL_OK ? hashes[i] : 0;
  }
}

void worker_main(tl_server *S, Worker *W) {
  cudaSetDevice(S->device);
  const uint64_t budget = S->cfg.hbm_budget_bytes;
  for (;;) {
    std::vector<Request *> batch;
    uint64_t charged = 0;
    {
      std::unique_lock<std::mutex> lk(S->mu);
      for (;;) {
        if (S->pending.empty()) {
          if (S->stop) return;
          S->cv_work.wait(lk);
          continue;
        }
        Request *head = S->pending.front();
        if (head->footprint + S->batch_fixed > budget) {  // cannot fit even alone
          S->pending.pop_front();
          head->res.status = TL_ENOMEM;
          head->res.t_admit_ns = head->res.t_done_ns = now_ns();
          head->done = true;
          S->cv_done.notify_all();
          continue;
        }
        if (S->in_use + head->footprint + S->batch_fixed > budget) {
          S->cv_work.wait(lk);  // wait for a batch to release memory
          continue;
        }
        charged = S->batch_fixed;
        while (!S->pending.empty() && batch.size() < S->cfg.max_batch) {
          Request *r = S->pending.front();
          if (S->in_use + charged + r->footprint > budget) break;
          charged += r->footprint;
          batch.push_back(r);
          S->pending.pop_front();
        }
        S->in_use += charged;
        break;
      }
    }
    const uint64_t t_admit = now_ns();
    for (Request *r : batch) r->res.t_admit_ns = t_admit;
    run_batch(S, *W, batch);
    const uint64_t t_done = now_ns();
    {
      std::lock_guard<std::mutex> lk(S->mu);
      S->in_use -= charged;
      for (Request *r : batch) {
        r->res.t_done_ns = t_done;
        r->done = true;
      }
    }
    S->cv_done.notify_all();
    S->cv_work.notify_all();
  }
}

void destroy(tl_server *S) {
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  for (Worker &W : S->workers)
    if (W.th.joinable()) W.th.join();
  cudaSetDevice(S->device);
  for (Worker &W : S->workers) {
    if (W.d_vbase) cudaFree(W.d_vbase);
    if (W.d_counts) cudaFree(W.d_counts);
    if (W.d_hashes) cudaFree(W.d_hashes);
    if (W.stream) cudaStreamDestroy(W.stream);
    if (W.cstream) cudaStreamDestroy(W.cstream);
  }
  for (GraphEntry &ge : S->graphs)
    for (tl_graph *h : ge.prepared) tl_graph_free(h);
  if (S->reg_stream) {
    cudaStreamSynchronize(S->reg_stream);
    cudaStreamDestroy(S->reg_stream);
  }
  for (auto &kv : S->requests) delete kv.second;
  delete S;
}

}  // namespace

#define TL_SERVE_BEGIN \
  try {                \
    tl::clear_error();
#define TL_SERVE_END                              \
  }                                               \
  catch (const tl::Error &e) {                    \
    tl::set_error(e.msg);                         \
    return e.status;                              \
  }                                               \
  catch (const std::bad_alloc &) {                \
    tl::set_error("host allocation failed");      \
    return TL_ENOMEM;                             \
  }                                               \
  catch (...) {                                   \
    tl::set_error("unexpected internal error");   \
    return TL_ECUDA;                              \
  }                                               \
  return TL_OK;

extern "C" {

uint64_t tl_server_now_ns(void) { return now_ns(); }

tl_status tl_server_create(tl_server **out, const tl_server_config *cfg) {
  TL_SERVE_BEGIN
  if (!out || !cfg) tl::fail(TL_EINVAL, "out or cfg is NULL");
  *out = nullptr;
  if (cfg->max_batch == 0 || cfg->workers == 0)
    tl::fail(TL_EINVAL, "max_batch and workers must be >= 1");
  if (cfg->chunk_bytes < TL_MIN_CHUNK_BYTES)
    tl::fail(TL_EINVAL, "chunk_bytes below TL_MIN_CHUNK_BYTES");
  tl_server *S = new tl_server();
  S->cfg = *cfg;
  try {
    TL_CUDA(cudaGetDevice(&S->device));
    TL_CUDA(cudaStreamCreateWithFlags(&S->reg_stream, cudaStreamNonBlocking));
    S->batch_fixed = tl::list_fixed_bytes(cfg->chunk_bytes);
    S->workers.resize(cfg->workers);
    for (Worker &W : S->workers) {
      TL_CUDA(cudaStreamCreateWithFlags(&W.stream, cudaStreamNonBlocking));
      TL_CUDA(cudaStreamCreateWithFlags(&W.cstream, cudaStreamNonBlocking));
      TL_CUDA(cudaMalloc(&W.d_vbase, ((uint64_t)cfg->max_batch + 1) * 8));
      TL_CUDA(cudaMalloc(&W.d_counts, (uint64_t)cfg->max_batch * 8));
      TL_CUDA(cudaMalloc(&W.d_hashes, (uint64_t)cfg->max_batch * 8));
    }
    for (Worker &W : S->workers) W.th = std::thread(worker_main, S, &W);
  } catch (...) {
    destroy(S);
    throw;
  }
  *out = S;
  TL_SERVE_END
}

tl_status tl_server_add_graph(tl_server *S, const tl_graph *g, uint32_t *graph_id) {
  TL_SERVE_BEGIN
  if (!S || !g || !graph_id) tl::fail(TL_EINVAL, "NULL argument");
  GraphEntry ge;
  ge.g = g;
  tl_status st = tl_graph_size(g, &ge.n, &ge.m);
  if (st != TL_OK) return st;
  std::lock_guard<std::mutex> lk(S->mu);
  S->graphs.push_back(ge);
  *graph_id = (uint32_t)(S->graphs.size() - 1);
  TL_SERVE_END
}

tl_status tl_server_add_ordering(tl_server *S, uint32_t graph_id, const uint32_t *rank,
                                 int rank_on_device, uint32_t *ordering_id) {
  TL_SERVE_BEGIN
  if (!S || !rank || !ordering_id) tl::fail(TL_EINVAL, "NULL argument");
  const tl_graph *g = nullptr;
  uint32_t n = 0;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (graph_id >= S->graphs.size()) tl::fail(TL_EINVAL, "unknown graph_id");
    g = S->graphs[graph_id].g;
    n = S->graphs[graph_id].n;
  }
  TL_CUDA(cudaSetDevice(S->device));
  std::lock_guard<std::mutex> reg(S->reg_mu);
  cudaStream_t s = S->reg_stream;
  tl::DevBuf d(s);  // host ranks are staged on the device
  const uint32_t *dev_rank = rank;
  if (!rank_on_device) {
    d.reserve((uint64_t)n * 4);
    TL_CUDA(cudaMemcpyAsync(d.p, rank, (uint64_t)n * 4, cudaMemcpyHostToDevice, s));
    dev_rank = d.as<uint32_t>();
  }
  // a one-part union: a copy of the graph with its DAG under this ordering
  // (not a permutation -> TL_EINVAL)
  tl_graph *h = nullptr;
  const tl_status st = tl_graph_union(&h, &g, &dev_rank, 1, s);
  if (st != TL_OK) return st;
  std::lock_guard<std::mutex> lk(S->mu);
  GraphEntry &ge = S->graphs[graph_id];
  ge.prepared.push_back(h);
  *ordering_id = (uint32_t)(ge.prepared.size() - 1);
  TL_SERVE_END
}

tl_status tl_server_submit(tl_server *S, uint32_t graph_id, uint32_t ordering_id, tl_alg alg,
                           uint64_t *request_id) {
  TL_SERVE_BEGIN
  if (!S || !request_id) tl::fail(TL_EINVAL, "NULL argument");
  if (alg != TL_APP && alg != TL_APM && alg != TL_AMM)
    tl::fail(TL_EINVAL, "alg must be TL_APP, TL_APM or TL_AMM");
  Request *r = new Request();
  r->res.t_submit_ns = now_ns();
  r->res.tuning_entry = -1;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    if (graph_id >= S->graphs.size() || ordering_id >= S->graphs[graph_id].prepared.size()) {
      delete r;
      tl::fail(TL_EINVAL, "unknown graph_id or ordering_id");
    }
    const GraphEntry &ge = S->graphs[graph_id];
    r->id = S->next_id++;
    r->g = ge.prepared[ordering_id];
    r->n = ge.n;
    r->alg = alg;
    r->footprint = footprint(ge.n, ge.m);
    S->requests[r->id] = r;
    S->pending.push_back(r);
    *request_id = r->id;
  }
  S->cv_work.notify_one();
  TL_SERVE_END
}

tl_status tl_server_set_tuning_table(tl_server *S, const tl_tuning_entry *entries,
                                     uint32_t count) {
  TL_SERVE_BEGIN
  if (!S) tl::fail(TL_EINVAL, "server is NULL");
  auto t = std::make_shared<std::vector<tl_tuning_entry>>();
  if (entries && count) {
    t->assign(entries, entries + count);
    for (const auto &e : *t)
      if (e.alg != TL_APP && e.alg != TL_APM && e.alg != TL_AMM)
        tl::fail(TL_EINVAL, "a tuning entry names an unknown algorithm");
  }
  std::lock_guard<std::mutex> lk(S->mu);
  S->tuning = t;
  TL_SERVE_END
}

tl_status tl_server_wait(tl_server *S, uint64_t request_id, tl_request_result *out) {
  TL_SERVE_BEGIN
  if (!S || !out) tl::fail(TL_EINVAL, "NULL argument");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->requests.find(request_id);
  if (it == S->requests.end()) tl::fail(TL_EINVAL, "unknown request id");
  Request *r = it->second;
  if (r->waited) tl::fail(TL_EINVAL, "another thread is already waiting for this request");
  r->waited = true;
  S->cv_done.wait(lk, [r] { return r->done; });
  *out = r->res;
  S->requests.erase(it);
  delete r;
  TL_SERVE_END
}

tl_status tl_server_footprint(const tl_server *S, uint32_t graph_id, uint64_t *request_bytes,
                              uint64_t *batch_bytes) {
  TL_SERVE_BEGIN
  if (!S) tl::fail(TL_EINVAL, "server is NULL");
  tl_server *W = const_cast<tl_server *>(S);
  std::lock_guard<std::mutex> lk(W->mu);
  if (graph_id >= S->graphs.size()) tl::fail(TL_EINVAL, "unknown graph_id");
  if (request_bytes) *request_bytes = footprint(S->graphs[graph_id].n, S->graphs[graph_id].m);
  if (batch_bytes) *batch_bytes = S->batch_fixed;
  TL_SERVE_END
}

void tl_server_free(tl_server *S) {
  if (S) destroy(S);
}

}  // extern "C"
