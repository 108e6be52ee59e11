// Listing kernels: shared definitions between list.cu and api.cu.
#pragma once

#include "graph.cuh"

namespace tl {

// Tiers of B vertices x (by probe-set size p = |P_x| and work W_x, the
// number of membership tests of x; ww = Tuning::warp_work):
//   0 small:  p <= 32,   W <= ww  -- one warp per x, 64-slot hash per warp
//   1 medium: p <= 1024, W <= ww  -- one warp per x, 2048-slot hash per warp
//   2 narrow: p <= 256,  W >  ww  -- one-warp CTA per piece, 2^14-bit filter in
//                                    front of a 512-slot bucketed hash
//   3 mid:    p <= 2048, W >  ww  -- 256-thread CTA per piece, 8192-slot bucketed hash
//   4 large:  p >  2048           -- 1024-thread CTA per piece, bitmap / hash
constexpr int kTiers = 5;
constexpr int kTierSmall = 0, kTierMedium = 1, kTierNarrow = 2, kTierMid = 3, kTierLarge = 4;
constexpr int kWarpThreads = 256;
constexpr int kNarrowThreads = 32;
constexpr int kMidThreads = 256;
constexpr int kLargeThreads = 1024;
constexpr uint32_t kSmallMaxP = 32, kMediumMaxP = 1024, kNarrowMaxP = 256, kMidMaxP = 2048;
constexpr int kSmallSlots = 64, kMediumSlots = 2048;  // per warp, >= 2p (load <= 1/2)
constexpr int kNarrowSlots = 512;                      // per one-warp CTA, >= 2p
constexpr int kNarrowFilterWords = 512;                // 2^14 filter bits before the table
constexpr int kMidSlots = 8192;                        // per CTA, >= 4p
// Work (membership tests) per task: a warp-tier task is owned by one warp
// and groups vertices up to about warp_work units, a vertex weighing its
// tests plus kVertexCost (its setup is a chain of dependent loads); each
// vertex has <= warp_work tests, so a task has < 2 warp_work tests.  A
// narrow, mid or large vertex is cut into pieces of piece_work(tier, p)
// tests, each run by one CTA.
constexpr uint64_t kWarpWorkMax = 1u << 12;
constexpr uint64_t kVertexCost = 256;

// Run-time choices of the work split (tl_tuning in the C ABI).
struct Tuning {
  uint32_t small_max_p;  // tier thresholds on p, at most the table sizes allow:
  uint32_t medium_max_p; //   small <= kSmallMaxP, medium <= kMediumMaxP,
  uint32_t narrow_max_p; //   narrow <= kNarrowMaxP, mid <= kMidMaxP
  uint32_t mid_max_p;
  uint32_t warp_work;    // warp-tier task size, tests (256 .. kWarpWorkMax)
  uint32_t narrow_piece; // tests per piece of a narrow vertex
  uint32_t mid_piece;    // tests per piece of a mid vertex
  uint32_t large_per_p;  // large pieces: clamp(large_per_p * p, large_min, large_max)
  uint32_t large_min;
  uint32_t large_max;
  uint32_t narrow_keep_mib;   // L2 priority of the narrow kernel's short-step loads
  uint32_t narrow_cold_first; //   (see l2_keep_from / l2_cold_first in ListArgs)
  uint32_t large_hash_max_p;  // n > kBitmapMaxN: larger large vertices take filter + global table
};
__host__ __device__ inline uint64_t piece_work(const Tuning &tu, int tier, uint64_t p) {
  if (tier == kTierNarrow) return tu.narrow_piece;
  if (tier == kTierMid) return tu.mid_piece;
  uint64_t w = (uint64_t)tu.large_per_p * p;
  w = w < tu.large_min ? tu.large_min : w;
  return w > tu.large_max ? tu.large_max : w;
}
// Shared-memory probe structures of the large kernel.
constexpr uint32_t kBitmapMaxN = 1u << 20;               // 128 KiB bitmap over ranks
constexpr uint32_t kHashMaxSlots = 32768u;               // 128 KiB hash table
// Hubs too large for the shared-memory table when n > kBitmapMaxN: a 2^20-bit
// shared-memory filter over hashed ranks in front of a per-CTA hash table of
// kGHashSlots slots in global memory (p <= kGHashSlots / 2).
constexpr uint32_t kFilterWords = 1u << 15;
constexpr uint32_t kGHashSlots = 1u << 18;
// Output of the CTA tiers: each warp stages its hits as (original id of y,
// rank of z) pairs in a shared-memory buffer of kWarpBuf entries and copies
// them to the chunk itself when fewer than kWarpStep free entries are left
// (one step adds at most kWarpStep hits) and at the end of its range.
constexpr uint32_t kWarpBuf = 352;  // 4 mid CTAs (56 KiB each) per SM
constexpr uint32_t kWarpStep = 128;
constexpr int kNarrowProbeBytes = (kNarrowFilterWords + kNarrowSlots) * 4;
constexpr int kMidProbeBytes = kMidSlots * 4;
constexpr int kLargeProbeBytes = (int)(kBitmapMaxN / 8);  // = kHashMaxSlots * 4 = kFilterWords * 4
constexpr int kNarrowSmemBytes = kNarrowProbeBytes + (kNarrowThreads / 32) * (int)kWarpBuf * 8;
constexpr int kMidSmemBytes = kMidProbeBytes + (kMidThreads / 32) * (int)kWarpBuf * 8;
constexpr int kLargeSmemBytes = kLargeProbeBytes + (kLargeThreads / 32) * (int)kWarpBuf * 8;
// Triangles a warp-tier task can produce (bounded by its work): the size of
// each warp's global slab.  A chunk must hold at least that many.
constexpr uint64_t kSlabCapWarp = 2 * kWarpWorkMax;
constexpr uint64_t kSlabCap = kSlabCapWarp;
__host__ __device__ inline uint64_t slab_cap(int tier) { return tier < 2 ? kSlabCapWarp : 0; }

// Device control block of one listing launch.  Reservations are atomic adds
// to `cursor`, so the successful ones form the prefix [start, first_fail) of
// the chunk (or [start, cursor) when none failed).
// The cursor, hit by every reservation, has a 128-byte line of its own.
struct ListCtl {
  unsigned long long cursor;      // chunk slots reserved (may pass the capacity)
  unsigned long long pad0[15];
  unsigned long long first_fail;  // smallest position of a reservation that did not fit
  unsigned long long probes;      // membership tests of committed work
  uint32_t overflow;              // a reservation did not fit
  uint32_t fetch;                 // task fetch counter
  uint32_t n_retry_out;           // tasks / ranges queued for the next launch
  uint32_t pad1;
};

// Retry record of the CTA tiers: the tests of B vertex x that a CTA's warps
// could not commit because the chunk was full, one range [r[i][0], r[i][1])
// per warp that stopped.  A retry runs them as one piece (one build of B),
// warp i taking range i.
constexpr int kMaxRanges = kLargeThreads / 32;
struct RetryPiece {
  uint32_t x, n;
  uint64_t r[kMaxRanges][2];
};

struct ListArgs {
  uint32_t n, x_begin, x_end;
  // For B vertex x: probe set P_x = padj[poff[x], poff[x+1]); seeds y =
  // sadj[soff[x], soff[x+1]); for each seed, the list scan_adj[scan_off[y],
  // scan_off[y+1]) is scanned.  A++: N-, N-, N+;  A+-: N+, N+, N+;
  // A--: N-, N+, N-.
  const uint64_t *poff;
  const uint32_t *padj;
  const uint64_t *soff;
  const uint32_t *sadj;
  const uint64_t *scan_off;
  const uint32_t *scan_adj;      // read 16 bytes at a time: padded by 4 elements
  const uint32_t *inv;           // rank -> original id
  const uint64_t *WP;            // work prefix over seed-side entries [m+1]
  // warp tiers: the tier's vertices in rank order and their work prefix
  // [count+1]; task t holds vertices [task_start[t], task_start[t+1])
  const uint32_t *tier_x;
  const uint64_t *tier_wp;
  const uint32_t *task_start;
  uint64_t tier_count;
  // narrow / mid / large tier: piece prefix over x in [x_begin, x_end) [nr+1]
  // and the vertex of every task [n_tasks]; CTAs take tasks from the last
  // (highest ranks, the largest vertices under a degree ordering) down
  const uint64_t *piece_prefix;
  const uint32_t *task_x;
  uint32_t *ghash;               // large tier, n > kBitmapMaxN: kGHashSlots per CTA (or null)
  Tuning tu;                     // the work split the task tables were built with
  // narrow kernel, short-list steps: loads of scan_adj entries at index >=
  // l2_keep_from take L2 evict_last, the others evict_first when
  // l2_cold_first is set (~0 and 0: no hint)
  uint64_t l2_keep_from;
  uint32_t l2_cold_first;
  int tier;
  ListCtl *ctl;
  uint32_t *chunk;               // output chunk, 3 uint32 per triangle
  uint64_t chunk_cap;            // triangles
  uint32_t *slabs;               // warp tiers: per-warp staging, slab_cap triangles each
  uint64_t slab_cap;
  const uint32_t *retry_in;      // warp tiers: tasks left over by the previous launch
  uint32_t n_retry;              // entries in retry_in / rr_in
  uint32_t *retry_out;
  const RetryPiece *rr_in;       // CTA tiers: pieces left over by the previous launch
  RetryPiece *rr_out;
  uint64_t fresh_base;           // first task not yet fetched
  uint64_t n_tasks;
};

void launch_seed_work(const uint32_t *sadj, uint64_t m, const uint64_t *scan_off, uint32_t *w,
                      cudaStream_t s);
// Per x in [x_begin, x_end): weight in tier 0 / 1 (0 if not in the tier),
// the membership flags, and the piece counts of tiers 2, 3 and 4.
void launch_classify(const uint64_t *poff, const uint64_t *soff, const uint64_t *WP,
                     uint32_t x_begin, uint32_t x_end, const Tuning &tu,
                     uint64_t *w0, uint64_t *w1, uint32_t *f0, uint32_t *f1, uint64_t *pieces2,
                     uint64_t *pieces3, uint64_t *pieces4, cudaStream_t s);
// Compact the vertices of one warp tier: x_list[pos[r]] = x, wp_list[pos[r]] = pref[r].
void launch_compact_tier(const uint32_t *flags, const uint64_t *pos, const uint64_t *pref,
                         uint32_t x_begin, uint64_t nr, uint32_t *x_list, uint64_t *wp_list,
                         cudaStream_t s);
// task_start[t] = first tier vertex whose work prefix is >= t * warp_work
// (clamped to count), t in [0, n_tasks].
void launch_task_bounds(const uint64_t *wp_list, uint64_t count, uint64_t n_tasks,
                        uint64_t warp_work, uint32_t *task_start, cudaStream_t s);
// task_x[t] = the vertex owning task t of a narrow, mid or large tier.
// Work profile of the B vertices x in [x_begin, x_end): hist[bp * kProfileBinsW
// + bw] += W_x, bp = bit length of p_x, bw = bit length of W_x (hist is
// kProfileBinsP * kProfileBinsW uint64 on the device, zeroed by the caller).
constexpr int kProfileBinsP = TL_PROFILE_BINS_P, kProfileBinsW = TL_PROFILE_BINS_W;
void launch_work_profile(const uint64_t *poff, const uint64_t *soff, const uint64_t *WP,
                         uint32_t x_begin, uint32_t x_end, unsigned long long *hist,
                         cudaStream_t s);
// *out = WP[soff[x_end]] - WP[soff[x_begin]]: the tests of a seed range.
void launch_range_work(const uint64_t *soff, const uint64_t *WP, uint32_t x_begin,
                       uint32_t x_end, uint64_t *out, cudaStream_t s);
void launch_task_owner(const uint64_t *piece_prefix, uint32_t x_begin, uint64_t nr,
                       uint32_t *task_x, cudaStream_t s);
// tier 0, 1: warp kernels; tier 2: narrow (one-warp) CTA kernel; tier 3: mid
// CTA kernel; tier 4: large CTA kernel.
void launch_list(int tier, const ListArgs &a, cudaStream_t s);
int tier_grid(int tier);
// Device bytes one listing call holds whatever the graph: two output chunks,
// the staging slabs and (at most) the hub hash tables.
uint64_t list_fixed_bytes(uint64_t chunk_bytes);
void launch_count_hash(const uint32_t *t, uint64_t n, unsigned long long *acc, cudaStream_t s);
void launch_count_hash_parts(const uint32_t *t, uint64_t n, const uint64_t *vbase, uint32_t k,
                             unsigned long long *counts, unsigned long long *hashes,
                             cudaStream_t s);

}  // namespace tl
