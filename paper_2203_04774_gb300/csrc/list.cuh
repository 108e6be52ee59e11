// Listing kernels: shared definitions between list.cu and api.cu.
#pragma once

#include "graph.cuh"

namespace tl {

constexpr int kSmallThreads = 256;
constexpr int kLargeThreads = 1024;
// Work (membership tests) of one task: a small task groups small vertices
// up to about kSmallWork tests (at most 2 * kSmallWork); a large vertex is
// cut into pieces of at most kPieceWork tests.
constexpr uint64_t kSmallWork = 1u << 16;
constexpr uint64_t kPieceWork = 1u << 16;
// Shared-memory probe structures of the large kernel.
constexpr uint32_t kBitmapMaxN = 1572864u;              // 192 KiB bitmap over ranks
constexpr uint32_t kHashMaxSlots = 32768u;              // 128 KiB hash table
constexpr int kLargeSmemBytes = (int)(kBitmapMaxN / 8);  // >= kHashMaxSlots * 4
// Triangles a task can produce (bounded by its work).
constexpr uint64_t kSlabCap = 2 * kSmallWork > kPieceWork ? 2 * kSmallWork : kPieceWork;

// Device control block of one listing launch.
struct ListCtl {
  unsigned long long cursor;     // chunk slots reserved (may pass the capacity)
  unsigned long long valid_end;  // end of the committed prefix of the chunk
  unsigned long long triangles;  // triangles committed
  unsigned long long probes;     // membership tests of committed tasks
  uint32_t overflow;             // a reservation did not fit
  uint32_t fetch;                // task fetch counter
  uint32_t n_retry_out;          // tasks queued for the next launch
  uint32_t pad;
};

struct ListArgs {
  uint32_t n, x_begin, x_end;
  const uint64_t *poff;          // probe-side CSR: A++ -> N-, A+- -> N+
  const uint32_t *padj;
  const uint64_t *out_off;       // scanned lists N+
  const uint32_t *out_adj;
  const uint32_t *inv;           // rank -> original id
  const uint64_t *WP;            // work prefix over probe-side entries [m+1]
  const uint64_t *small_prefix;  // over x in range [nr+1]
  const uint64_t *piece_prefix;  // over x in range [nr+1]
  ListCtl *ctl;
  uint32_t *chunk;               // output chunk, 3 uint32 per triangle
  uint64_t chunk_cap;            // triangles
  uint32_t *slabs;               // per-CTA staging, slab_cap triangles each
  uint64_t slab_cap;
  const uint32_t *retry_in;      // tasks left over by the previous launch
  uint32_t n_retry;
  uint32_t *retry_out;
  uint64_t fresh_base;           // first task not yet fetched
  uint64_t n_tasks;
};

void launch_seed_work(const uint32_t *padj, uint64_t m, const uint64_t *out_off, uint32_t *w,
                      cudaStream_t s);
void launch_classify(const uint64_t *poff, const uint64_t *WP, uint32_t x_begin, uint32_t x_end,
                     uint64_t *small_w, uint64_t *pieces, cudaStream_t s);
// kind 0: small-vertex kernel, kind 1: large-vertex kernel.
void launch_list(int kind, const ListArgs &a, cudaStream_t s);
int small_grid();
int large_grid();
void launch_count_hash(const uint32_t *t, uint64_t n, unsigned long long *acc, cudaStream_t s);

}  // namespace tl
