// Triangle listing: Algorithm 1 (A++), Algorithm 2 (A+-) and the third
// variant A-- of Sec. 2.1.
//
// The three algorithms have the same shape once the "B vertex" x is fixed:
//   A++: x = w, probe set P_x = N-_w, seeds y in N-_w, scanned lists N+_y;
//   A+-: x = u, probe set P_x = N+_u, seeds y in N+_u, scanned lists N+_y;
//   A--: x = v, probe set P_x = N-_v, seeds y in N+_v, scanned lists N-_y.
// For every seed y and every z in its scanned list, z in P_x reports a
// triangle {x, y, z} (A++: u=y, v=z, w=x; A+-: u=x, v=y, w=z; A--: u=z, v=x,
// w=y).  The membership tests of x number the sum of its seeds' list
// lengths; summed over x they are C++, C+- resp. C-- (Property 1).
//
// Work space (a6).  Seed edge k = (x, y_k) is the k-th entry of the seed-side
// CSR; it owns the tests [WP[k], WP[k+1]) of a global exclusive prefix WP.
// Every kernel walks the tests of a range with the same warp-level mapping
// (scan_items): a window of 32 consecutive seed edges is held one per lane;
// a list of at least 32 tests is streamed with 16-byte loads, shorter ones
// share 128-test steps (four tests per lane) in which each lane finds the
// seed edge of each of its tests by a shuffle binary search over the window,
// so all lanes work whatever the lengths.
// The seed edge of a range's first test is found by the whole warp (32
// samples of WP and a ballot per round).
//
// B (the boolean array of the algorithms) per tier:
//   small/medium x: a per-warp hash table in shared memory (load <= 1/2), one
//   warp per x, vertices grouped into tasks of about warp_work tests;
//   mid/large x: one structure per CTA -- a bucketed hash, a bitmap over all
//   ranks when n is small enough (literally B, bit-packed), a shared filter in
//   front of a global hash for hubs of large graphs, or binary search in the
//   sorted row -- and the work cut into pieces shared by the CTA's warps.
//
// Output (a9).  Warp tiers: a task's hits go to the warp's global slab; at its
// end one atomic reserves room in the current chunk and the warp copies them,
// or the whole task is queued for the next launch.  CTA tiers: each warp
// stages hits in shared memory and copies them to the chunk itself (one
// atomic per flush); a warp whose reservation fails stops, and the exact test
// ranges whose hits were not written go to the next launch, one record per
// piece.  Either way every chunk holds complete output for the tests it
// covers, and the listing resumes exactly where it stopped.

#include "list.cuh"

namespace tl {
namespace {

constexpr uint32_t kEmpty = 0xffffffffu;

__device__ __forceinline__ void sort3(uint32_t &a, uint32_t &b, uint32_t &c) {
  uint32_t t;
  if (a > b) t = a, a = b, b = t;
  if (b > c) t = b, b = c, c = t;
  if (a > b) t = a, a = b, b = t;
}

// Number of lanes j with v_j <= key (0..32), for v ascending across the
// warp.  The five halving steps reach at most 31; the last lane is checked
// on its own.
__device__ __forceinline__ int warp_count_le(uint32_t v, uint32_t key) {
  int pos = 0;
#pragma unroll
  for (int step = 16; step >= 1; step >>= 1) {
    uint32_t e = __shfl_sync(0xffffffffu, v, pos + step - 1);
    if (e <= key) pos += step;
  }
  const uint32_t last = __shfl_sync(0xffffffffu, v, 31);
  if (pos == 31 && last <= key) pos = 32;
  return pos;
}

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src) {
  uint32_t lo = __shfl_sync(0xffffffffu, (uint32_t)v, src);
  uint32_t hi = __shfl_sync(0xffffffffu, (uint32_t)(v >> 32), src);
  return ((uint64_t)hi << 32) | lo;
}

// Number of elements <= key in the sorted v[0, n), by the whole warp (every
// lane calls it with the same arguments and gets the result): each round the
// lanes sample 32 evenly spaced elements and one ballot narrows the range
// 32-fold, so a search takes about log32(n) + 1 dependent loads instead of
// log2(n).  Invariant: every element before `base` is <= key and the count
// lies in [base, base + cnt].
__device__ __forceinline__ uint64_t warp_upper_bound_u64(const uint64_t *v, uint64_t n,
                                                         uint64_t key) {
  const int lane = threadIdx.x & 31;
  uint64_t base = 0, cnt = n;
  while (cnt > 32) {
    const uint64_t step = (cnt + 31) >> 5;  // 32 step >= cnt
    const uint64_t idx = base + (uint64_t)lane * step;
    const bool le = idx < base + cnt && v[idx] <= key;
    const uint32_t c = __popc(__ballot_sync(0xffffffffu, le));  // samples <= key: a prefix
    if (c == 0) return base;
    // sample c-1 is <= key; sample c (if any) is > key or past the range
    const uint64_t lo = base + (uint64_t)(c - 1) * step + 1;
    const uint64_t hi = base + (uint64_t)c * step < base + cnt ? base + (uint64_t)c * step
                                                               : base + cnt;
    base = lo;
    cnt = hi - lo;
  }
  const bool le = (uint64_t)lane < cnt && v[base + lane] <= key;
  return base + __popc(__ballot_sync(0xffffffffu, le));
}

__device__ __forceinline__ uint64_t lower_bound_u64(const uint64_t *v, uint64_t n, uint64_t key) {
  uint64_t lo = 0, hi = n;
  while (lo < hi) {
    uint64_t mid = (lo + hi) >> 1;
    if (v[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Multiplicative hash into a table of 2^lg slots.
__device__ __forceinline__ uint32_t hslot(uint32_t r, int lg) {
  return (r * 0x9E3779B1u) >> (32 - lg);
}

__device__ __forceinline__ void hash_insert(uint32_t *H, int lg, uint32_t r) {
  const uint32_t mask = (1u << lg) - 1u;
  uint32_t h = hslot(r, lg);
  while (atomicCAS(&H[h], kEmpty, r) != kEmpty) h = (h + 1) & mask;
}

__device__ __forceinline__ bool hash_find(const uint32_t *H, int lg, uint32_t z) {
  const uint32_t mask = (1u << lg) - 1u;
  uint32_t h = hslot(z, lg);
  for (;;) {
    uint32_t v = H[h];
    if (v == z) return true;
    if (v == kEmpty) return false;
    h = (h + 1) & mask;
  }
}

// Bucketed table for the CTA tiers: 2^lgb buckets of four slots, key r in
// bucket bslot(r) or, when that is full, the next ones (linear probing by
// bucket).  A thread writes slot s of a bucket only after finding slots
// 0..s-1 taken, so the taken slots of a bucket are always a prefix: a bucket
// whose last slot is empty ends a search.  A lookup reads one bucket with a
// single 16-byte shared-memory load.
__device__ __forceinline__ uint32_t bslot(uint32_t r, int lgb) {
  return (r * 0x9E3779B1u) >> (32 - lgb);
}

__device__ __forceinline__ void bucket_insert(uint32_t *H, int lgb, uint32_t r) {
  const uint32_t mask = (1u << lgb) - 1u;
  uint32_t b = bslot(r, lgb);
  for (;;) {
#pragma unroll
    for (int s = 0; s < 4; ++s)
      if (atomicCAS(&H[4 * b + s], kEmpty, r) == kEmpty) return;
    b = (b + 1) & mask;
  }
}

__device__ __forceinline__ bool bucket_find(const uint32_t *H, int lgb, uint32_t z) {
  const uint32_t mask = (1u << lgb) - 1u;
  uint32_t b = bslot(z, lgb);
  for (;;) {
    const uint4 q = reinterpret_cast<const uint4 *>(H)[b];
    if (q.x == z || q.y == z || q.z == z || q.w == z) return true;
    if (q.w == kEmpty) return false;
    b = (b + 1) & mask;
  }
}

// Filter bit of rank r (2^20 bits) for the hub tier's shared-memory filter.
__device__ __forceinline__ uint32_t fslot(uint32_t r) { return (r * 0x85EBCA77u) >> 12; }

// Membership tests of the walk, four keys at a time (check4): the keys of a
// lane's 16-byte load, or its four tests of a short-list step.  Where a probe
// can miss its first slot, the four first probes are issued before any
// result is used and the rare longer searches follow one by one.
struct WarpHashMember {  // linear probing, per-warp table of 2^lg slots
  const uint32_t *H;
  int lg;
  __device__ bool one(uint32_t z) const { return hash_find(H, lg, z); }
  __device__ void check4(const uint32_t z[4], bool r[4]) const {
#pragma unroll
    for (int u = 0; u < 4; ++u) r[u] = one(z[u]);
  }
};

struct BucketMember {  // four-slot buckets, 2^lgb buckets
  const uint32_t *H;
  int lgb;
  __device__ void check4(const uint32_t z[4], bool r[4]) const {
    uint4 q[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) q[u] = reinterpret_cast<const uint4 *>(H)[bslot(z[u], lgb)];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      r[u] = q[u].x == z[u] || q[u].y == z[u] || q[u].z == z[u] || q[u].w == z[u];
      if (!r[u] && q[u].w != kEmpty) r[u] = bucket_find(H, lgb, z[u]);
    }
  }
};

struct BitmapMember {  // one bit per rank (the boolean array B, bit-packed)
  const uint32_t *B;
  __device__ bool one(uint32_t z) const { return ((B[z >> 5] >> (z & 31)) & 1u) != 0; }
  __device__ void check4(const uint32_t z[4], bool r[4]) const {
#pragma unroll
    for (int u = 0; u < 4; ++u) r[u] = one(z[u]);
  }
};

struct FilterMember {  // one bit per hashed rank: may answer yes wrongly
  const uint32_t *F;
  __device__ bool one(uint32_t z) const {
    const uint32_t f = fslot(z);
    return ((F[f >> 5] >> (f & 31)) & 1u) != 0;
  }
  __device__ void check4(const uint32_t z[4], bool r[4]) const {
#pragma unroll
    for (int u = 0; u < 4; ++u) r[u] = one(z[u]);
  }
};

struct SmallFilterMember {  // 2^14 bits, one hashed bit per key: may answer yes wrongly
  const uint32_t *F;
  __device__ static uint32_t bit(uint32_t z) { return (z * 0x85EBCA77u) >> 18; }
  __device__ bool one(uint32_t z) const {
    const uint32_t f = bit(z);
    return ((F[f >> 5] >> (f & 31)) & 1u) != 0;
  }
  __device__ void check4(const uint32_t z[4], bool r[4]) const {
#pragma unroll
    for (int u = 0; u < 4; ++u) r[u] = one(z[u]);
  }
};

struct SortedRowMember {  // binary search in the sorted probe list
  const uint32_t *P;
  uint64_t n;
  __device__ bool one(uint32_t z) const {
    uint64_t lo = 0, hi = n;
    while (lo < hi) {
      const uint64_t mid = (lo + hi) >> 1;
      if (P[mid] < z) lo = mid + 1; else hi = mid;
    }
    return lo < n && P[lo] == z;
  }
  __device__ void check4(const uint32_t z[4], bool r[4]) const {
#pragma unroll
    for (int u = 0; u < 4; ++u) r[u] = one(z[u]);
  }
};

// Task fetch shared by all kernels: returns the task id or -1.  Thread 0
// only; the caller broadcasts.
__device__ __forceinline__ int64_t fetch_task(ListCtl *ctl, const ListArgs &a) {
  if (*(volatile uint32_t *)&ctl->overflow) return -1;
  uint32_t idx = atomicAdd(&ctl->fetch, 1u);
  if (idx < a.n_retry) return a.retry_in[idx];
  uint64_t t = a.fresh_base + (idx - a.n_retry);
  return (t < a.n_tasks) ? (int64_t)t : -1;
}

// Copy a warp-tier task's slab to the chunk: each entry is (original id of x,
// original id of y, rank of z); z is translated and the triple sorted here,
// four triples per thread per round with their gathers issued together.
__device__ __forceinline__ void copy_out(const uint32_t *__restrict__ inv, const uint32_t *slab,
                                         uint32_t cnt, uint32_t *dst, uint32_t tid,
                                         uint32_t nthreads) {
  for (uint32_t i0 = tid; i0 < cnt; i0 += 4 * nthreads) {
    uint32_t t[4][3];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t i = i0 + u * nthreads;
      if (i < cnt) {
        t[u][0] = slab[3 * i];
        t[u][1] = slab[3 * i + 1];
        t[u][2] = slab[3 * i + 2];
      }
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (i0 + u * nthreads < cnt) t[u][2] = __ldg(inv + t[u][2]);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t i = i0 + u * nthreads;
      if (i < cnt) {
        sort3(t[u][0], t[u][1], t[u][2]);
        // streaming stores: the chunk is read once by the consumer, so it
        // should not evict the adjacency lists from L2
        __stcs(dst + 3 * i, t[u][0]);
        __stcs(dst + 3 * i + 1, t[u][1]);
        __stcs(dst + 3 * i + 2, t[u][2]);
      }
    }
  }
}

// Output state of one warp of a CTA tier (see kWarpBuf).
struct WarpOut {
  uint32_t *buf;                   // shared memory: kWarpBuf (original id of y, rank of z)
  uint32_t cnt;                    // entries in buf (the same in every lane)
  uint64_t safe;                   // the warp's tests before `safe` are committed
  unsigned long long probes_safe;  // this lane's tests before `safe`
  bool failed;                     // a reservation did not fit: the warp stopped
};

// Exact-membership checks applied to a warp's staged entries before they are
// written.  NoVerify: the walk's test was exact already.  GlobalHashVerify:
// the walk tested a shared-memory filter only; the CTA's hash table in global
// memory decides, four keys per lane in flight.  SharedBucketVerify: the walk
// tested a small shared filter; the bucketed table behind it decides, in a
// function of its own so that the walk keeps its registers.
struct NoVerify {
  static constexpr bool kActive = false;
  __device__ void prefetch(uint32_t) const {}
};

__device__ __noinline__ uint32_t verify_bucket(uint32_t *buf, uint32_t cnt, const uint32_t *H,
                                               int lgb) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  uint2 *b2 = reinterpret_cast<uint2 *>(buf);
  uint32_t out = 0;
  for (uint32_t i0 = 0; i0 < cnt; i0 += 32) {
    const uint32_t i = i0 + lane;
    uint2 e = make_uint2(0, 0);
    bool keep = false;
    if (i < cnt) {
      e = b2[i];
      keep = bucket_find(H, lgb, e.y);
    }
    const unsigned km = __ballot_sync(0xffffffffu, keep);
    __syncwarp();  // every entry of this round is read before any is moved
    if (keep) b2[out + __popc(km & lt)] = e;
    out += __popc(km);
    __syncwarp();
  }
  return out;
}

struct SharedBucketVerify {
  static constexpr bool kActive = true, kOutOfLine = true;
  const uint32_t *H;
  int lgb;
  __device__ void prefetch(uint32_t) const {}
  __device__ uint32_t run(uint32_t *buf, uint32_t cnt) const {
    return verify_bucket(buf, cnt, H, lgb);
  }
};

struct GlobalHashVerify {
  static constexpr bool kActive = true, kOutOfLine = false;
  const uint32_t *H;
  int lg;
  // a candidate's first slot is asked into L2 when the candidate is staged,
  // so that the check at flush finds it there
  __device__ void prefetch(uint32_t z) const {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(H + hslot(z, lg)));
  }
  __device__ void check4(const uint32_t z[4], const bool valid[4], bool res[4]) const {
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t h[4];
    bool open[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      h[u] = hslot(z[u], lg);
      res[u] = false;
      open[u] = valid[u];
    }
    for (;;) {  // linear probing; the four searches advance together
      uint32_t v[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) v[u] = open[u] ? __ldcg(H + h[u]) : 0u;
      bool more = false;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (!open[u]) continue;
        if (v[u] == z[u]) {
          res[u] = true;
          open[u] = false;
        } else if (v[u] == kEmpty) {
          open[u] = false;
        } else {
          h[u] = (h[u] + 1) & mask;
          more = true;
        }
      }
      if (!more) break;
    }
  }
};

// Keep the staged entries (original id of y, rank of z) whose z passes the
// exact check, compacted in place; returns how many are left.
template <class Verify>
__device__ __forceinline__ uint32_t warp_verify_4(uint32_t *buf, uint32_t cnt, const Verify &vf) {
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  uint2 *b2 = reinterpret_cast<uint2 *>(buf);
  uint32_t out = 0;
  for (uint32_t i0 = 0; i0 < cnt; i0 += 128) {
    uint2 e[4];
    uint32_t z[4];
    bool valid[4], keep[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t i = i0 + 32 * u + lane;
      valid[u] = i < cnt;
      e[u] = valid[u] ? b2[i] : make_uint2(0, 0);
      z[u] = e[u].y;
    }
    vf.check4(z, valid, keep);
    __syncwarp();  // every entry of this round is read before any is moved
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const unsigned km = __ballot_sync(0xffffffffu, keep[u]);
      if (keep[u]) b2[out + __popc(km & lt)] = e[u];
      out += __popc(km);
    }
    __syncwarp();
  }
  return out;
}

template <class Verify>
__device__ __forceinline__ uint32_t warp_verify(uint32_t *buf, uint32_t cnt, const Verify &vf) {
  if constexpr (!Verify::kActive) {
    return cnt;
  } else if constexpr (Verify::kOutOfLine) {
    return vf.run(buf, cnt);
  } else {
    return warp_verify_4(buf, cnt, vf);
  }
}

// Copy a warp's buffer of cnt > 0 entries (original id of y, rank of z) to
// the chunk as sorted original-id triples with x, after reserving room with
// one atomic.  The triples are written with 16-byte streaming stores, four
// triples (three uint4) per lane, after a head of at most three single
// triples that brings the destination to a 16-byte boundary; each lane's
// four z gathers are issued together.  Returns false if the chunk is full.
// Scalar arguments only, so that the caller's state stays in registers.
__device__ __noinline__ bool warp_flush(ListCtl *ctl, uint32_t *chunk, uint64_t chunk_cap,
                                        const uint32_t *__restrict__ inv, const uint32_t *buf,
                                        uint32_t cnt, uint32_t inv_x) {
  const int lane = threadIdx.x & 31;
  unsigned long long pos = 0;
  uint32_t ok = 1;
  if (lane == 0) {
    // once one reservation has failed every later one fails too (the cursor
    // only grows), so the result of the add alone decides
    pos = atomicAdd(&ctl->cursor, (unsigned long long)cnt);
    if (pos + cnt > chunk_cap) {
      ok = 0;
      atomicMin(&ctl->first_fail, pos);
      atomicExch(&ctl->overflow, 1u);
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  if (!ok) return false;
  pos = (unsigned long long)__shfl_sync(0xffffffffu, (long long)pos, 0);
  uint32_t *dst = chunk + 3ull * pos;
  const uint2 *b2 = reinterpret_cast<const uint2 *>(buf);
  // dst sits `mis` words past a 16-byte boundary; triple i starts 3 i words
  // later, on a boundary when mis + 3 i = 0 mod 4, i.e. for i = mis mod 4
  const uint32_t mis = (uint32_t)((reinterpret_cast<uintptr_t>(dst) >> 2) & 3u);
  const uint32_t head = mis < cnt ? mis : cnt;
  const uint32_t groups = (cnt - head) >> 2;
  const uint32_t tail0 = head + 4 * groups;
  // head and tail (at most three triples each): one triple per lane
  auto one = [&](uint32_t i) {
    const uint2 e = b2[i];
    uint32_t p = inv_x, q = e.x, r = __ldg(inv + e.y);
    sort3(p, q, r);
    __stcs(dst + 3 * i, p);
    __stcs(dst + 3 * i + 1, q);
    __stcs(dst + 3 * i + 2, r);
  };
  if ((uint32_t)lane < head) one(lane);
  if ((uint32_t)lane < cnt - tail0) one(tail0 + lane);
  // body: four consecutive triples per lane, three aligned 16-byte stores
  uint4 *d4 = reinterpret_cast<uint4 *>(dst + 3 * head);
  for (uint32_t gi = lane; gi < groups; gi += 32) {
    const uint32_t i = head + 4 * gi;
    uint2 e[4];
    uint32_t t[4][3];
#pragma unroll
    for (int u = 0; u < 4; ++u) e[u] = b2[i + u];
#pragma unroll
    for (int u = 0; u < 4; ++u) t[u][2] = __ldg(inv + e[u].y);
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      t[u][0] = inv_x;
      t[u][1] = e[u].x;
      sort3(t[u][0], t[u][1], t[u][2]);
    }
    __stcs(d4 + 3 * gi, make_uint4(t[0][0], t[0][1], t[0][2], t[1][0]));
    __stcs(d4 + 3 * gi + 1, make_uint4(t[1][1], t[1][2], t[2][0], t[2][1]));
    __stcs(d4 + 3 * gi + 2, make_uint4(t[2][2], t[3][0], t[3][1], t[3][2]));
  }
  __syncwarp();
  return true;
}

// Commit a warp's buffer: afterwards every test before `cur` is committed.
// On a full chunk sets o.failed and leaves o.safe where it was.
template <class Verify>
__device__ __forceinline__ bool warp_commit(const ListArgs &a, WarpOut &o, uint32_t inv_x,
                                            uint64_t cur, unsigned long long probes,
                                            const Verify &vf) {
  if (o.cnt > 0) o.cnt = warp_verify(o.buf, o.cnt, vf);
  if (o.cnt > 0) {
    if (!warp_flush(a.ctl, a.chunk, a.chunk_cap, a.inv, o.buf, o.cnt, inv_x)) {
      o.failed = true;
      return false;
    }
    o.cnt = 0;
  }
  o.safe = cur;
  o.probes_safe = probes;
  return true;
}

// A piece's tests split evenly (32-aligned) over kWarps warps.
template <int kWarps, class T>
__device__ __forceinline__ void split_piece(uint64_t ia, uint64_t ib, T r[][2]) {
  const uint64_t per = (((ib - ia) + kWarps - 1) / kWarps + 31) & ~31ull;
  for (int w = 0; w < kWarps; ++w) {
    const uint64_t u = ia + (uint64_t)w * per, v = u + per;
    r[w][0] = u < ib ? u : ib;
    r[w][1] = v < ib ? v : ib;
  }
}

// Next piece of work of a CTA tier (thread 0): a retry piece (*retry set to
// its record), else the next fresh task's piece [ia, ib) of B vertex x.
// False when the chunk is full or no work is left.
__device__ __forceinline__ bool fetch_piece(const ListArgs &a, uint32_t &x, uint64_t &ia,
                                            uint64_t &ib, const RetryPiece *&retry) {
  retry = nullptr;
  if (*(volatile uint32_t *)&a.ctl->overflow) return false;
  const uint32_t idx = atomicAdd(&a.ctl->fetch, 1u);
  if (idx < a.n_retry) {
    retry = a.rr_in + idx;
    x = retry->x;
    return true;
  }
  const uint64_t f = a.fresh_base + (idx - a.n_retry);
  if (f >= a.n_tasks) return false;
  // fresh tasks from the last down: under a degree ordering the largest
  // vertices have the highest ranks, and starting with them keeps the end of
  // the launch from waiting on one big piece
  const uint64_t t = a.n_tasks - 1 - f;
  x = a.task_x[t];
  const uint64_t piece = t - a.piece_prefix[x - a.x_begin];
  const uint64_t w1 = a.WP[a.soff[x + 1]];
  const uint64_t pw = piece_work(a.tu, a.tier, a.poff[x + 1] - a.poff[x]);
  ia = a.WP[a.soff[x]] + piece * pw;
  ib = ia + pw < w1 ? ia + pw : w1;
  return true;
}

// Warp-level end of a warp-tier task: reserve chunk room for the warp's slab
// and copy it, or queue the task.
__device__ void commit_warp(ListCtl *ctl, const ListArgs &a, int64_t t, const uint32_t *slab,
                            uint32_t cnt, unsigned long long probes) {
  const int lane = threadIdx.x & 31;
  uint32_t ok = 1;
  unsigned long long pos = 0;
  if (lane == 0) {
    if (cnt > 0) {
      pos = atomicAdd(&ctl->cursor, (unsigned long long)cnt);
      if (pos + cnt > a.chunk_cap) ok = 0;
    }
    if (ok) {
      atomicAdd(&ctl->probes, probes);
    } else {
      atomicMin(&ctl->first_fail, pos);
      atomicExch(&ctl->overflow, 1u);
      const uint32_t r = atomicAdd(&ctl->n_retry_out, 1u);
      a.retry_out[r] = (uint32_t)t;
    }
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  pos = (unsigned long long)__shfl_sync(0xffffffffu, (long long)pos, 0);
  if (ok && cnt > 0) {
    copy_out(a.inv, slab, cnt, a.chunk + 3ull * pos, lane, 32);
  }
  __syncwarp();
}

// Load of one scanned element in a short-list step.  With kHint (the narrow
// kernel) it can carry an L2 eviction priority: evict_last for the kept
// lists (keep), evict_first for the others when cold_first is set; with
// neither it is a plain load.
template <bool kHint>
__device__ __forceinline__ uint32_t load_scanned(const uint32_t *q, bool keep,
                                                 uint32_t cold_first) {
  uint32_t v;
  if (kHint && (keep || cold_first)) {
    uint64_t pol;
    if (keep)
      asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    else
      asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    asm volatile("ld.global.nc.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(v) : "l"(q), "l"(pol));
  } else {
    v = *q;
  }
  return v;
}

// Warp-level walk of the tests [i0, i1) of B vertex x, whose seed row is
// [pb, pe) (entries of sadj); k0 is the seed edge holding test i0 (found by
// binary search when ~0).  For each test: z = the scanned element, and
// member (one key, or four at a time) answers B[z].  Hits
// go to the warp's own global slab as (original id of x, original id of y,
// rank of z) at positions counted by wcnt (kEmit 0, warp tiers), or to the
// warp's shared-memory buffer as (original id of y, rank of z), flushed to the
// chunk whenever it could overflow in the next step (kEmit 1, CTA tiers: on a
// failed flush the walk stops with o.failed set).  kHint: the short-list
// steps' loads take the L2 priorities of a.l2_keep_from / a.l2_cold_first.
template <int kEmit, bool kPrefetch, bool kHint, class Member, class Verify = NoVerify>
__device__ __forceinline__ void scan_items(const ListArgs &a, uint64_t pb, uint64_t pe, uint64_t k0,
                                           uint64_t i0, uint64_t i1, uint32_t inv_x,
                                           Member member, uint32_t *slab, WarpOut &o,
                                           uint32_t &wcnt, unsigned long long &probes,
                                           const Verify &vf = Verify()) {
  if (i0 >= i1) return;
  const int lane = threadIdx.x & 31;
  const unsigned lt = (1u << lane) - 1u;
  // seed edge holding test i0
  uint64_t k = (k0 != ~0ull) ? k0 : pb + warp_upper_bound_u64(a.WP + pb, pe - pb, i0) - 1;
  uint64_t E = 0, A = 0, Elast = 0, S = 0;  // S, E: first test and end of the lane's edge
  uint32_t iy = 0;
  auto load_window = [&](uint64_t kw) {
    const uint64_t kk = kw + lane;
    const bool valid = kk < pe;
    uint64_t B = ~0ull;
    E = ~0ull;
    A = 0;
    iy = 0;
    if (valid) {
      B = a.WP[kk];
      E = a.WP[kk + 1];
      const uint32_t y = a.sadj[kk];
      A = a.scan_off[y] - B;  // scanned element of test i is scan_adj[A + i]
      iy = a.inv[y];
    }
    S = B;
    Elast = shfl_u64(E, 31);
  };
  load_window(k);
  uint64_t base = i0;
  while (base < i1) {
    // j0 = the window's seed edge holding test `base` (32: window exhausted)
    const int j0 = __popc(__ballot_sync(0xffffffffu, E <= base));
    if (j0 == 32) {
      k += 32;
      load_window(k);
      continue;
    }
    const uint64_t Ej0 = shfl_u64(E, j0);
    if (Ej0 - base >= 32) {
      // Long run: every test up to min(Ej0, i1) scans the same list N+_y (at
      // most 2^31 tests per run, so that offsets within it fit 32 bits).
      const uint64_t Aj = shfl_u64(A, j0) + base;
      const uint32_t iyj = __shfl_sync(0xffffffffu, iy, j0);
      const uint64_t rest = (Ej0 < i1 ? Ej0 : i1) - base;
      const uint32_t run = rest < (1ull << 31) ? (uint32_t)rest : (1u << 31);
      // Each lane takes 4 consecutive elements with one aligned 16-byte load
      // (scan_adj is 256-byte aligned and padded by 4 elements), and the warp
      // reserves slab room for the 128 tests of an iteration at once.  Offsets
      // count from the aligned element before the run's first test, which
      // sits `lead` elements in: element e is a test of the run iff
      // lead <= e < lead + run.
      const uint32_t *src = a.scan_adj + (Aj & ~3ull);
      const uint32_t lead = (uint32_t)(Aj & 3), span = lead + run;
      // With kPrefetch (kernels with registers to spare) the next iteration's
      // 16 bytes are loaded one iteration ahead.  Only a run's first and last
      // iterations hold elements outside the run; their tests are masked, and
      // probes are counted once per run.
      uint4 vn = make_uint4(0, 0, 0, 0);
      if (kPrefetch && 4u * lane < span) vn = *reinterpret_cast<const uint4 *>(src + 4 * lane);
      for (uint32_t e0 = 0; e0 < span; e0 += 128) {
        if (kEmit == 1 && o.cnt > kWarpBuf - kWarpStep) {
          // every test before this iteration's first one has its hits in buf
          const uint32_t done = e0 > lead ? e0 - lead : 0;
          if (!warp_commit(a, o, inv_x, base + done, probes + (lane == 0 ? done : 0), vf))
            return;
        }
        const uint32_t e = e0 + 4 * lane;
        uint4 v = vn;
        if (kPrefetch) {
          if (e + 128 < span) vn = *reinterpret_cast<const uint4 *>(src + e + 128);
        } else if (e < span) {
          v = *reinterpret_cast<const uint4 *>(src + e);
        }
        const uint32_t z[4] = {v.x, v.y, v.z, v.w};
        bool hit[4];
        member.check4(z, hit);
        if (e0 < lead || e0 + 128 > span) {  // the same for the whole warp
#pragma unroll
          for (int u = 0; u < 4; ++u) hit[u] = hit[u] && e + u - lead < run;
        }
        // positions: the hits of element u of all lanes, u = 0..3, one after
        // the other (the order of triangles is free)
        unsigned hm[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) hm[u] = __ballot_sync(0xffffffffu, hit[u]);
        const uint32_t c0 = __popc(hm[0]), c1 = __popc(hm[1]), c2 = __popc(hm[2]);
        const uint32_t total = c0 + c1 + c2 + __popc(hm[3]);
        if (total == 0) continue;
        uint32_t basepos;
        if (kEmit == 0) {
          basepos = wcnt;
          wcnt += total;
        } else {
          basepos = o.cnt;
          o.cnt += total;
        }
        const uint32_t start[4] = {basepos, basepos + c0, basepos + c0 + c1,
                                   basepos + c0 + c1 + c2};
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          if (hit[u]) {
            // z stays a rank here; the copy to the chunk translates it
            const uint32_t r = start[u] + __popc(hm[u] & lt);
            if (kEmit == 0) {
              slab[3 * r + 0] = inv_x;
              slab[3 * r + 1] = iyj;
              slab[3 * r + 2] = z[u];
            } else {
              reinterpret_cast<uint2 *>(o.buf)[r] = make_uint2(iyj, z[u]);
              vf.prefetch(z[u]);
            }
          }
        }
      }
      if (lane == 0) probes += run;
      base += run;
      continue;
    }
    // Short segments: one step of up to 128 tests spread over several lists,
    // test base + 32 u + lane on lane `lane` (u = 0..3), so that each group of
    // 32 is coalesced and every lane has four independent loads in flight.
    // The step stops where a long list (>= 128 tests) starts, which the
    // streaming path takes next.
    if (kEmit == 1 && o.cnt > kWarpBuf - kWarpStep) {
      if (!warp_commit(a, o, inv_x, base, probes, vf)) return;
    }
    uint64_t lim = base + 128;
    if (lim > i1) lim = i1;
    if (lim > Elast) lim = Elast;
    {
      const bool long_after = E != ~0ull && S > base && E - S >= 128;
      const unsigned lm = __ballot_sync(0xffffffffu, long_after);
      if (lm) {
        const uint64_t s0 = shfl_u64(S, __ffs(lm) - 1);
        if (s0 < lim) lim = s0;
      }
    }
    // segment ends relative to base, clamped to [0, 160]
    const uint32_t D = (E <= base) ? 0u : (uint32_t)((E - base) < 160 ? (E - base) : 160);
    uint32_t z[4], iyj[4];
    bool act[4], hit[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const uint32_t off = lane + 32 * u;
      act[u] = base + off < lim;
      const int j = warp_count_le(D, off);  // seed edge of test base + off (< 32 when act)
      const int jj = j < 31 ? j : 31;
      const uint64_t Aj = shfl_u64(A, jj);
      iyj[u] = __shfl_sync(0xffffffffu, iy, jj);
      const uint64_t q = Aj + base + off;
      z[u] = act[u] ? load_scanned<kHint>(a.scan_adj + q, kHint && q >= a.l2_keep_from,
                                          a.l2_cold_first)
                    : 0u;
    }
    member.check4(z, hit);
    unsigned hm[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      hit[u] = hit[u] && act[u];
      hm[u] = __ballot_sync(0xffffffffu, hit[u]);
      probes += act[u] ? 1 : 0;
    }
    const uint32_t c0 = __popc(hm[0]), c1 = __popc(hm[1]), c2 = __popc(hm[2]);
    const uint32_t total = c0 + c1 + c2 + __popc(hm[3]);
    if (total > 0) {
      uint32_t basepos;
      if (kEmit == 0) {
        basepos = wcnt;
        wcnt += total;
      } else {
        basepos = o.cnt;
        o.cnt += total;
      }
      const uint32_t startpos[4] = {basepos, basepos + c0, basepos + c0 + c1,
                                    basepos + c0 + c1 + c2};
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        if (hit[u]) {
          const uint32_t r = startpos[u] + __popc(hm[u] & lt);
          if (kEmit == 0) {
            slab[3 * r + 0] = inv_x;
            slab[3 * r + 1] = iyj[u];
            slab[3 * r + 2] = z[u];
          } else {
            reinterpret_cast<uint2 *>(o.buf)[r] = make_uint2(iyj[u], z[u]);
            vf.prefetch(z[u]);
          }
        }
      }
    }
    base = lim;
  }
}

// ---- small and medium vertices: one warp per x, B = per-warp hash ----------

template <int SLOTS>
__global__ void __launch_bounds__(kWarpThreads, 4) k_list_warp(ListArgs a) {
  extern __shared__ uint32_t sm[];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  uint32_t *H = sm + wid * SLOTS;
  const uint64_t gwarp = (uint64_t)blockIdx.x * (kWarpThreads / 32) + wid;
  uint32_t *slab = a.slabs + gwarp * a.slab_cap * 3;
  WarpOut nout{nullptr, 0, 0, 0, false};  // unused by the global-slab path
  for (;;) {
    int64_t t = 0;
    if (lane == 0) t = fetch_task(a.ctl, a);
    t = __shfl_sync(0xffffffffu, (long long)t, 0);
    if (t < 0) break;
    const uint32_t i0 = a.task_start[t], i1 = a.task_start[t + 1];
    unsigned long long probes = 0;
    uint32_t cnt = 0;
    for (uint32_t idx = i0; idx < i1; ++idx) {
      const uint32_t x = a.tier_x[idx];
      const uint64_t pb = a.poff[x], pe = a.poff[x + 1];
      const uint64_t sb = a.soff[x], se = a.soff[x + 1];
      const uint32_t p = (uint32_t)(pe - pb);
      int lg = 6;
      while ((1u << lg) < 2 * p) ++lg;  // 2p <= SLOTS by the tier's definition
      const uint32_t cap = 1u << lg;
      for (uint32_t i = lane; i < cap; i += 32) H[i] = kEmpty;
      __syncwarp();
      for (uint64_t q = pb + lane; q < pe; q += 32) hash_insert(H, lg, a.padj[q]);
      __syncwarp();
      scan_items<0, false, false>(a, sb, se, sb, a.WP[sb], a.WP[se], a.inv[x], WarpHashMember{H, lg},
                           slab, nout, cnt, probes);
      __syncwarp();
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) probes += __shfl_down_sync(0xffffffffu, probes, d);
    commit_warp(a.ctl, a, t, slab, cnt, probes);
  }
}

// ---- narrow, mid and large vertices: one CTA per piece, B shared by the CTA
//   narrow (p <= 256, one warp per CTA) and mid (p <= 2048): bucketed hash of
//   <= 1024 resp. 8192 slots (load <= 1/4).
//   large: a bitmap over all ranks when n <= kBitmapMaxN (mode 0), else a
//   hash of <= kHashMaxSlots slots (mode 1), else a filter in shared memory +
//   the CTA's hash table in global memory (mode 3), else binary search in the
//   sorted row (mode 2).

template <int THREADS, int TIER>
__global__ void __launch_bounds__(THREADS, TIER == kTierLarge ? 1 : (TIER == kTierMid ? 4 : 28))
    k_list_cta(ListArgs a) {
  // probe structure (bitmap, hash or filter) | one output buffer per warp
  extern __shared__ __align__(16) uint32_t sm[];
  constexpr uint32_t kProbeWords =
      (TIER == kTierNarrow ? kNarrowProbeBytes
                           : (TIER == kTierMid ? kMidProbeBytes : kLargeProbeBytes)) / 4;
  // the next piece of work (one test range per warp), fetched by the first
  // warp done with the current one while the others finish (or by thread 0
  // before the first); the ranges of warps stopped by a full chunk
  constexpr int kWarps = THREADS / 32;
  __shared__ unsigned long long s_rng[kWarps][2], s_fail[kWarps][2];
  __shared__ uint32_t s_x, s_ok, s_mode, s_lg, s_fetcher, s_nfail;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  WarpOut o{sm + kProbeWords + (uint32_t)wid * 2 * kWarpBuf, 0, 0, 0, false};
  uint32_t unused = 0;
  const bool use_bitmap = TIER == kTierLarge && a.n <= kBitmapMaxN;
  if (use_bitmap) {
    const uint32_t words = (a.n + 31) >> 5;
    for (uint32_t i = threadIdx.x; i < words; i += THREADS) sm[i] = 0;
  }
  auto fetch_next = [&]() {  // one thread
    uint32_t x = 0;
    uint64_t ia = 0, ib = 0;
    const RetryPiece *rp = nullptr;
    const bool ok = fetch_piece(a, x, ia, ib, rp);
    s_ok = ok;
    if (!ok) return;
    if (rp) {  // the recorded ranges, one per warp
      const uint32_t nr = rp->n;
      for (int w = 0; w < kWarps; ++w) {
        s_rng[w][0] = w < (int)nr ? rp->r[w][0] : 0;
        s_rng[w][1] = w < (int)nr ? rp->r[w][1] : 0;
      }
    } else {  // the piece's tests, split evenly (32-aligned) over the warps
      split_piece<kWarps>(ia, ib, s_rng);
    }
    const uint64_t p = a.poff[x + 1] - a.poff[x];
    s_x = x;
    s_lg = 6;
    if (use_bitmap) {
      s_mode = 0;
      return;
    }
    // narrow and mid tiers: load <= 1/4, so most lookups end at the first bucket
    const uint32_t max_slots = TIER == kTierNarrow ? (uint32_t)kNarrowSlots
                               : (TIER == kTierMid ? (uint32_t)kMidSlots : kHashMaxSlots);
    const uint64_t want = TIER == kTierLarge ? 2 * p : 4 * p;
    uint32_t lg = 6;
    while ((1ull << lg) < want && (1u << lg) < max_slots) ++lg;
    s_lg = lg;
    s_mode = (2 * p <= (1ull << lg)) ? 1 : 2;  // 2: too large, binary search
    if (TIER == kTierLarge && (s_mode == 2 || p > a.tu.large_hash_max_p) && a.ghash &&
        2 * p <= kGHashSlots) {
      // 3: shared-memory filter + this CTA's hash table in global memory
      lg = 6;
      while ((1ull << lg) < 2 * p) ++lg;
      s_lg = lg;
      s_mode = 3;
    }
  };
  if (threadIdx.x == 0) {
    s_fetcher = 0;
    s_nfail = 0;
    fetch_next();
  }
  for (;;) {
    __syncthreads();
    if (!s_ok) break;
    const uint32_t x = s_x;
    const uint64_t pb = a.poff[x], pe = a.poff[x + 1];  // probe set P_x
    const uint64_t sb = a.soff[x], se = a.soff[x + 1];  // seeds
    const uint32_t mode = s_mode;
    const int lg = (int)s_lg;
    const uint64_t wa = s_rng[wid][0], wb = s_rng[wid][1];  // this warp's tests
    // build B: the probe set P_x (narrow and mid vertices always take mode
    // 1, so the other modes are compiled for the large kernel only)
    constexpr bool kLarge = TIER == kTierLarge;
    constexpr bool kPf = TIER == kTierNarrow;  // registers allow the walk's prefetch
    if (kLarge && mode == 0) {
      for (uint64_t q = pb + threadIdx.x; q < pe; q += THREADS) {
        const uint32_t r = a.padj[q];
        atomicOr(&sm[r >> 5], 1u << (r & 31));
      }
    } else if (TIER == kTierNarrow) {  // filter words, then the buckets
      for (uint32_t i = threadIdx.x; i < (uint32_t)kNarrowFilterWords; i += THREADS) sm[i] = 0;
      for (uint32_t i = threadIdx.x; i < (1u << lg); i += THREADS)
        sm[kNarrowFilterWords + i] = kEmpty;
      __syncthreads();
      for (uint64_t q = pb + threadIdx.x; q < pe; q += THREADS) {
        const uint32_t r = a.padj[q];
        const uint32_t f = SmallFilterMember::bit(r);
        atomicOr(&sm[f >> 5], 1u << (f & 31));
        bucket_insert(sm + kNarrowFilterWords, lg - 2, r);
      }
    } else if (mode == 1) {  // lg = log2(slots); buckets of four
      for (uint32_t i = threadIdx.x; i < (1u << lg); i += THREADS) sm[i] = kEmpty;
      __syncthreads();
      for (uint64_t q = pb + threadIdx.x; q < pe; q += THREADS)
        bucket_insert(sm, lg - 2, a.padj[q]);
    } else if (kLarge && mode == 3) {
      uint32_t *gh = a.ghash + (uint64_t)blockIdx.x * kGHashSlots;
      for (uint32_t i = threadIdx.x; i < kFilterWords; i += THREADS) sm[i] = 0;
      for (uint32_t i = threadIdx.x; i < (1u << lg); i += THREADS) gh[i] = kEmpty;
      __syncthreads();
      for (uint64_t q = pb + threadIdx.x; q < pe; q += THREADS) {
        const uint32_t r = a.padj[q];
        const uint32_t f = fslot(r);
        atomicOr(&sm[f >> 5], 1u << (f & 31));
        hash_insert(gh, lg, r);
      }
    }
    __syncthreads();
    const uint32_t inv_x = a.inv[x];
    unsigned long long probes = 0;
    o.cnt = 0;
    o.safe = wa;
    o.probes_safe = 0;
    o.failed = false;
    if (TIER == kTierNarrow) {
      // the walk tests the filter; staged candidates meet the table at flush
      const SharedBucketVerify vf{sm + kNarrowFilterWords, lg - 2};
      scan_items<1, kPf, kPf>(a, sb, se, ~0ull, wa, wb, inv_x, SmallFilterMember{sm}, nullptr, o,
                         unused, probes, vf);
      if (!o.failed) warp_commit(a, o, inv_x, wb, probes, vf);
    } else if (kLarge && mode == 0) {
      scan_items<1, kPf, kPf>(a, sb, se, ~0ull, wa, wb, inv_x, BitmapMember{sm}, nullptr, o, unused,
                         probes);
    } else if (!kLarge || mode == 1) {
      scan_items<1, kPf, kPf>(a, sb, se, ~0ull, wa, wb, inv_x, BucketMember{sm, lg - 2}, nullptr, o,
                         unused, probes);
    } else if (mode == 3) {
      // the walk tests the shared filter only; the staged candidates are
      // checked against the CTA's global hash table when the warp flushes
      const GlobalHashVerify vf{a.ghash + (uint64_t)blockIdx.x * kGHashSlots, lg};
      scan_items<1, kPf, kPf>(a, sb, se, ~0ull, wa, wb, inv_x, FilterMember{sm}, nullptr, o, unused,
                         probes, vf);
      if (!o.failed) warp_commit(a, o, inv_x, wb, probes, vf);
    } else {
      scan_items<1, kPf, kPf>(a, sb, se, ~0ull, wa, wb, inv_x,
                         SortedRowMember{a.padj + pb, pe - pb}, nullptr, o, unused, probes);
    }
    if (!o.failed && TIER != kTierNarrow && (!kLarge || mode != 3))
      warp_commit(a, o, inv_x, wb, probes, NoVerify());
    // commit the warp's tests before o.safe; queue the rest for the next launch
    unsigned long long done = o.probes_safe;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) done += __shfl_down_sync(0xffffffffu, done, d);
    if (lane == 0) {
      if (done) atomicAdd(&a.ctl->probes, done);
      if (o.failed && o.safe < wb) {
        const uint32_t f = atomicAdd(&s_nfail, 1u);
        s_fail[f][0] = o.safe;
        s_fail[f][1] = wb;
      }
      // every thread has read the current piece's s_* (before the barrier
      // that ended the build); the first warp here fetches the next piece
      if (atomicExch(&s_fetcher, 1u) == 0) fetch_next();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      s_fetcher = 0;
      const uint32_t nf = s_nfail;
      if (nf) {  // one record for the piece's uncommitted ranges
        RetryPiece *rp = a.rr_out + atomicAdd(&a.ctl->n_retry_out, 1u);
        rp->x = x;
        rp->n = nf;
        for (uint32_t f = 0; f < nf; ++f) {
          rp->r[f][0] = s_fail[f][0];
          rp->r[f][1] = s_fail[f][1];
        }
        s_nfail = 0;
      }
    }
    if (kLarge && mode == 0) {  // reset B
      for (uint64_t q = pb + threadIdx.x; q < pe; q += THREADS) sm[a.padj[q] >> 5] = 0;
    }
  }
}

// ---- bucketize (a6) -----------------------------------------------------------

// w[k] = length of the list scanned for seed entry k (d+ of y_k, or d- for A--).
__global__ void k_seed_work(const uint32_t *__restrict__ sadj, uint64_t m,
                            const uint64_t *__restrict__ scan_off, uint32_t *__restrict__ w) {
  for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < m;
       k += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t y = sadj[k];
    w[k] = (uint32_t)(scan_off[y + 1] - scan_off[y]);
  }
}

__global__ void k_classify(const uint64_t *__restrict__ poff, const uint64_t *__restrict__ soff,
                           const uint64_t *__restrict__ WP,
                           uint32_t x_begin, uint32_t x_end, Tuning tu, uint64_t *__restrict__ w0,
                           uint64_t *__restrict__ w1, uint32_t *__restrict__ f0,
                           uint32_t *__restrict__ f1, uint64_t *__restrict__ pieces2,
                           uint64_t *__restrict__ pieces3, uint64_t *__restrict__ pieces4) {
  const uint64_t nr = x_end - x_begin;
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < nr;
       r += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = x_begin + (uint32_t)r;
    const uint64_t W = WP[soff[x + 1]] - WP[soff[x]];
    const uint64_t p = poff[x + 1] - poff[x];
    uint64_t a0 = 0, a1 = 0, n2 = 0, n3 = 0, n4 = 0;
    // every prescribed test runs, also when P_x is empty (possible for A--,
    // whose seeds are not its probe set): the work then equals the cost
    if (W > 0) {
      if (p <= tu.small_max_p && W <= tu.warp_work) {
        a0 = W + kVertexCost;
      } else if (p <= tu.medium_max_p && W <= tu.warp_work) {
        a1 = W + kVertexCost;
      } else {
        const int tier =
            p <= tu.narrow_max_p ? kTierNarrow : (p <= tu.mid_max_p ? kTierMid : kTierLarge);
        const uint64_t pw = piece_work(tu, tier, p);
        const uint64_t np = (W + pw - 1) / pw;
        if (tier == kTierNarrow) n2 = np; else if (tier == kTierMid) n3 = np; else n4 = np;
      }
    }
    w0[r] = a0;
    w1[r] = a1;
    f0[r] = a0 ? 1u : 0u;
    f1[r] = a1 ? 1u : 0u;
    pieces2[r] = n2;
    pieces3[r] = n3;
    pieces4[r] = n4;
  }
}

__global__ void k_compact_tier(const uint32_t *__restrict__ flags, const uint64_t *__restrict__ pos,
                               const uint64_t *__restrict__ pref, uint32_t x_begin, uint64_t nr,
                               uint32_t *__restrict__ x_list, uint64_t *__restrict__ wp_list) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r <= nr;
       r += (uint64_t)gridDim.x * blockDim.x) {
    if (r == nr) {
      wp_list[pos[nr]] = pref[nr];  // total work after the last vertex
    } else if (flags[r]) {
      x_list[pos[r]] = x_begin + (uint32_t)r;
      wp_list[pos[r]] = pref[r];
    }
  }
}

__global__ void k_task_bounds(const uint64_t *__restrict__ wp, uint64_t count, uint64_t n_tasks,
                              uint64_t warp_work, uint32_t *__restrict__ task_start) {
  for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t <= n_tasks;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t i = lower_bound_u64(wp, count + 1, t * warp_work);
    task_start[t] = (uint32_t)(i < count ? i : count);
  }
}

__global__ void k_task_owner(const uint64_t *__restrict__ prefix, uint32_t x_begin, uint64_t nr,
                             uint32_t *__restrict__ task_x) {
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < nr;
       r += (uint64_t)gridDim.x * blockDim.x) {
    for (uint64_t t = prefix[r]; t < prefix[r + 1]; ++t) task_x[t] = x_begin + (uint32_t)r;
  }
}

__global__ void k_range_work(const uint64_t *__restrict__ soff, const uint64_t *__restrict__ WP,
                             uint32_t x_begin, uint32_t x_end, uint64_t *__restrict__ out) {
  *out = WP[soff[x_end]] - WP[soff[x_begin]];
}

// Per-block bins in shared memory, added to the global histogram at the end.
__global__ void k_work_profile(const uint64_t *__restrict__ poff, const uint64_t *__restrict__ soff,
                               const uint64_t *__restrict__ WP, uint32_t x_begin, uint32_t x_end,
                               unsigned long long *__restrict__ hist) {
  __shared__ unsigned long long bins[kProfileBinsP * kProfileBinsW];
  for (int i = threadIdx.x; i < kProfileBinsP * kProfileBinsW; i += blockDim.x) bins[i] = 0;
  __syncthreads();
  const uint64_t nr = x_end - x_begin;
  for (uint64_t r = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; r < nr;
       r += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t x = x_begin + (uint32_t)r;
    const uint64_t W = WP[soff[x + 1]] - WP[soff[x]];
    if (W == 0) continue;
    const uint64_t p = poff[x + 1] - poff[x];
    const int bp = 64 - __clzll((long long)p), bw = 64 - __clzll((long long)W);
    atomicAdd(&bins[(bp < kProfileBinsP ? bp : kProfileBinsP - 1) * kProfileBinsW +
                    (bw < kProfileBinsW ? bw : kProfileBinsW - 1)],
              (unsigned long long)W);
  }
  __syncthreads();
  for (int i = threadIdx.x; i < kProfileBinsP * kProfileBinsW; i += blockDim.x)
    if (bins[i]) atomicAdd(&hist[i], bins[i]);
}

template <class K>
int occupancy_grid(K kernel, int threads, int smem) {
  if (smem > 48 * 1024)
    TL_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  int per_sm = 0;
  TL_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem));
  return num_sms() * (per_sm > 0 ? per_sm : 1);
}

constexpr int kSmemSmall = kSmallSlots * 4 * (kWarpThreads / 32);
constexpr int kSmemMedium = kMediumSlots * 4 * (kWarpThreads / 32);
constexpr int kSmemMid = kMidSmemBytes;

}  // namespace

// ---- host side ----------------------------------------------------------------

void launch_seed_work(const uint32_t *sadj, uint64_t m, const uint64_t *scan_off, uint32_t *w,
                      cudaStream_t s) {
  k_seed_work<<<grid_for(m, 256), 256, 0, s>>>(sadj, m, scan_off, w);
  TL_CHECK_LAUNCH();
}

void launch_classify(const uint64_t *poff, const uint64_t *soff, const uint64_t *WP,
                     uint32_t x_begin, uint32_t x_end, const Tuning &tu,
                     uint64_t *w0, uint64_t *w1, uint32_t *f0, uint32_t *f1, uint64_t *pieces2,
                     uint64_t *pieces3, uint64_t *pieces4, cudaStream_t s) {
  k_classify<<<grid_for((uint64_t)(x_end - x_begin), 256), 256, 0, s>>>(
      poff, soff, WP, x_begin, x_end, tu, w0, w1, f0, f1, pieces2, pieces3, pieces4);
  TL_CHECK_LAUNCH();
}

void launch_compact_tier(const uint32_t *flags, const uint64_t *pos, const uint64_t *pref,
                         uint32_t x_begin, uint64_t nr, uint32_t *x_list, uint64_t *wp_list,
                         cudaStream_t s) {
  k_compact_tier<<<grid_for(nr + 1, 256), 256, 0, s>>>(flags, pos, pref, x_begin, nr, x_list,
                                                       wp_list);
  TL_CHECK_LAUNCH();
}

void launch_task_bounds(const uint64_t *wp_list, uint64_t count, uint64_t n_tasks,
                        uint64_t warp_work, uint32_t *task_start, cudaStream_t s) {
  k_task_bounds<<<grid_for(n_tasks + 1, 256), 256, 0, s>>>(wp_list, count, n_tasks, warp_work,
                                                           task_start);
  TL_CHECK_LAUNCH();
}

void launch_task_owner(const uint64_t *piece_prefix, uint32_t x_begin, uint64_t nr,
                       uint32_t *task_x, cudaStream_t s) {
  if (nr == 0) return;
  k_task_owner<<<grid_for(nr, 256), 256, 0, s>>>(piece_prefix, x_begin, nr, task_x);
  TL_CHECK_LAUNCH();
}

void launch_range_work(const uint64_t *soff, const uint64_t *WP, uint32_t x_begin,
                       uint32_t x_end, uint64_t *out, cudaStream_t s) {
  k_range_work<<<1, 1, 0, s>>>(soff, WP, x_begin, x_end, out);
  TL_CHECK_LAUNCH();
}

void launch_work_profile(const uint64_t *poff, const uint64_t *soff, const uint64_t *WP,
                         uint32_t x_begin, uint32_t x_end, unsigned long long *hist,
                         cudaStream_t s) {
  if (x_end <= x_begin) return;
  k_work_profile<<<grid_for((uint64_t)(x_end - x_begin), 256, (unsigned)num_sms() * 2), 256, 0,
                   s>>>(poff, soff, WP, x_begin, x_end, hist);
  TL_CHECK_LAUNCH();
}

int tier_grid(int tier) {
  // initialised once, thread-safely (a throw leaves it for the next call)
  struct Grids {
    int g[kTiers];
  };
  static const Grids grids = [] {
    Grids r;
    r.g[0] = occupancy_grid(k_list_warp<kSmallSlots>, kWarpThreads, kSmemSmall);
    r.g[1] = occupancy_grid(k_list_warp<kMediumSlots>, kWarpThreads, kSmemMedium);
    r.g[2] = occupancy_grid(k_list_cta<kNarrowThreads, kTierNarrow>, kNarrowThreads,
                            kNarrowSmemBytes);
    r.g[3] = occupancy_grid(k_list_cta<kMidThreads, kTierMid>, kMidThreads, kSmemMid);
    r.g[4] = occupancy_grid(k_list_cta<kLargeThreads, kTierLarge>, kLargeThreads,
                            kLargeSmemBytes);
    return r;
  }();
  return grids.g[tier];
}

uint64_t list_fixed_bytes(uint64_t chunk_bytes) {
  uint64_t slab = 0;
  for (int t = 0; t < 2; ++t) {  // the warp tiers' global slabs
    const uint64_t w = (uint64_t)tier_grid(t) * (kWarpThreads / 32) * slab_cap(t);
    slab = w > slab ? w : slab;
  }
  return 2 * (chunk_bytes / 12) * 12 + slab * 12 +
         (uint64_t)tier_grid(kTierLarge) * kGHashSlots * 4;
}

void launch_list(int tier, const ListArgs &a, cudaStream_t s) {
  const int grid = tier_grid(tier);
  if (tier == 0) {
    k_list_warp<kSmallSlots><<<grid, kWarpThreads, kSmemSmall, s>>>(a);
  } else if (tier == 1) {
    k_list_warp<kMediumSlots><<<grid, kWarpThreads, kSmemMedium, s>>>(a);
  } else if (tier == kTierNarrow) {
    k_list_cta<kNarrowThreads, kTierNarrow><<<grid, kNarrowThreads, kNarrowSmemBytes, s>>>(a);
  } else if (tier == kTierMid) {
    k_list_cta<kMidThreads, kTierMid><<<grid, kMidThreads, kSmemMid, s>>>(a);
  } else {
    k_list_cta<kLargeThreads, kTierLarge><<<grid, kLargeThreads, kLargeSmemBytes, s>>>(a);
  }
  TL_CHECK_LAUNCH();
}

}  // namespace tl
