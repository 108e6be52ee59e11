// The device-resident graph and the internal entry points of each step.
#pragma once

#include <vector>

#include "common.cuh"

namespace tl {

// Everything a graph handle owns on the device.
//   E        undirected simple edges, key = min_id << 32 | max_id, sorted.
//   rank/inv current ordering: rank[v] = pi_v - 1, inv[rank[v]] = v.
//   out_*    N+ lists (successor ranks) as CSR over ranks, rows ascending.
//   in_*     N- lists (predecessor ranks), rows ascending.
struct DeviceGraph {
  uint32_t n = 0;
  uint64_t m = 0;
  cudaStream_t stream = nullptr;
  bool ordered = false;
  DevBuf E, rank, inv, out_off, out_adj, in_off, in_adj;
  // workspaces (kept between calls so repeated calls do not reallocate)
  DevBuf keys_a, keys_b, sort_tmp, scan_tmp, small;  // small: flags/counters
  uint64_t cost_app = 0, cost_apm = 0, cost_amm = 0;
  uint32_t max_out_deg = 0, max_in_deg = 0;
  // A disjoint union's part table: part i holds vertices [vbase[i], vbase[i+1]);
  // empty for a graph loaded whole.
  std::vector<uint64_t> part_vbase;
  // Order every buffer's allocation and release on stream s.
  void bind(cudaStream_t s) {
    stream = s;
    for (DevBuf *b : {&E, &rank, &inv, &out_off, &out_adj, &in_off, &in_adj, &keys_a, &keys_b,
                      &sort_tmp, &scan_tmp, &small})
      b->stream = s;
  }
};

// a1: copy + canonicalise + dedup (build.cu).  Throws tl::Error.
void build_edge_set(DeviceGraph &g, const uint32_t *edges, uint64_t m_in, bool on_device);
// The tail of a1: sort the m_in canonical keys in g.keys_a (loops = ~0),
// drop loops and duplicates into g.E, set g.m.
void finish_edge_set(DeviceGraph &g, uint64_t m_in);
// Disjoint unions (batch.cu).  Part i holds n[i] vertices and becomes
// vertices [vbase[i], vbase[i] + n[i]) of the union.
//   Concatenated edge lists with part-local ids (host arrays n, m_in of k entries).
void build_edge_set_parts(DeviceGraph &g, uint32_t k, const uint32_t *n, const uint64_t *m_in,
                          const uint32_t *edges, bool on_device);
//   Loaded graphs, each under rank[i] (device, part-local) or, if null, its
//   current ordering (identity when none was applied); builds the union's DAG.
void build_union(DeviceGraph &u, uint32_t k, const DeviceGraph *const *parts,
                 const uint32_t *const *rank);
// N+ / N- halves of the CSR of keys sorted by (high, low) half: off_a/adj_a by
// high half, off_b/adj_b by low half (rows ascending); ka, kb: m-key scratch.
void csr_halves(const uint64_t *E, uint64_t m, uint32_t n, uint64_t *off_a, uint32_t *adj_a,
                uint64_t *off_b, uint32_t *adj_b, DevBuf &ka, DevBuf &kb, DevBuf &tmp,
                DevBuf &scan, cudaStream_t s);
// Level-synchronous core peeling (core.cu): keys[v] = round << 32 | v; returns
// the number of rounds.
uint32_t core_peel_keys(DeviceGraph &g, uint64_t *keys);
// True iff rank[0..n) (device) is a permutation of [0, n); `flag` is one
// device uint32 of scratch.  Synchronises s.
bool is_permutation(const uint32_t *rank, uint32_t n, uint32_t *flag, cudaStream_t s);
// a2-a5: validate the permutation, relabel, orient, CSR out/in, cost.
// rank == nullptr applies the identity ordering.
void build_dag(DeviceGraph &g, const uint32_t *rank, bool on_device);
// Degree (kind 0), Split (kind 1) or core (kind 2) ordering of the loaded graph into rank[n];
// on a union, part by part (part i's ranks are vbase[i] + its own ranks).
void compute_order(DeviceGraph &g, int kind, uint32_t *rank, bool on_device);

}  // namespace tl
