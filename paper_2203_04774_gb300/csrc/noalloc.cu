// tl_count_hash_noalloc: the count + set-hash consumer without any device
// allocation.
//
// Why it exists.  tl_count_hash allocates its accumulator with cudaMalloc
// on first use.  Some callers cannot allocate at that point: a consumer runs
// in the middle of tl_list_triangles while the next listing kernel is in
// flight, and a caller that keeps every byte of device memory in its own
// pool (or that must not trigger the implicit device synchronisation of a
// cudaMalloc / cudaFree there) needs a consumer that touches no allocator.
// This variant keeps its scratch -- one partial hash per block of triples --
// in a fixed file-scope device array instead.
//
// Limits and sharing.
//   * Scratch: kNoallocBlocks partials of 8 bytes (128 KiB), in a static
//     __device__ array that every GPU which loads the library holds until
//     the process exits.
//   * One call handles at most TL_NOALLOC_MAX_TRIPLES triples (one partial
//     per block of kNoallocPerBlock triples); larger calls are rejected
//     before any device work.
//   * Every call on a device shares the array and leaves its own partials
//     in it.  Each call writes every partial it later reads, so nothing
//     needs clearing, but calls that overlap on the GPU (two streams, two
//     threads) race on the array and must be serialised by the caller.
//   * The array's device address is looked up once per device, with that
//     device current, on the first call made on it (cudaGetSymbolAddress).
//     Make that first call before any stream capture.
#include <mutex>

#include "common.cuh"
#include "hash.cuh"

namespace {

constexpr int kNoallocThreads = 256;
constexpr uint64_t kNoallocPerBlock = 16384;  // triples per block (64 per thread)
constexpr uint64_t kNoallocBlocks = 16384;
static_assert(kNoallocBlocks * kNoallocPerBlock == TL_NOALLOC_MAX_TRIPLES,
              "the header's limit must match the scratch layout");

static __device__ __align__(256) unsigned long long g_noalloc_partials[kNoallocBlocks];

__device__ __forceinline__ unsigned long long block_sum(unsigned long long v) {
  __shared__ unsigned long long warp_sums[kNoallocThreads / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_down_sync(0xffffffffu, v, d);
  if (lane == 0) warp_sums[wid] = v;
  __syncthreads();
  unsigned long long s = 0;
  if (wid == 0) {
    s = (lane < kNoallocThreads / 32) ? warp_sums[lane] : 0;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) s += __shfl_down_sync(0xffffffffu, s, d);
  }
  return s;  // valid in thread 0
}

// Block b hashes triples [b * kNoallocPerBlock, ...) and stores its partial.
__global__ void __launch_bounds__(kNoallocThreads)
    k_noalloc_partials(const uint32_t *__restrict__ t, uint64_t n,
                       unsigned long long *__restrict__ partials) {
  const uint64_t begin = (uint64_t)blockIdx.x * kNoallocPerBlock;
  const uint64_t end = (begin + kNoallocPerBlock < n) ? begin + kNoallocPerBlock : n;
  unsigned long long h = 0;
  for (uint64_t i = begin + threadIdx.x; i < end; i += kNoallocThreads)
    h += tl::triple_hash(t[3 * i], t[3 * i + 1], t[3 * i + 2]);
  h = block_sum(h);
  if (threadIdx.x == 0) partials[blockIdx.x] = h;
}

// One block adds the first `blocks` partials to out[1] and n to out[0].
__global__ void __launch_bounds__(kNoallocThreads)
    k_noalloc_finish(const unsigned long long *__restrict__ partials, uint32_t blocks,
                     uint64_t n, uint64_t *__restrict__ out) {
  unsigned long long h = 0;
  for (uint32_t i = threadIdx.x; i < blocks; i += kNoallocThreads) h += partials[i];
  h = block_sum(h);
  if (threadIdx.x == 0) {
    out[0] += n;
    out[1] += h;
  }
}

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mu;
unsigned long long *g_noalloc_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
unsigned long long *noalloc_scratch() {
  int dev = 0;
  TL_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) tl::fail(TL_EINVAL, "device index out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void *p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_partials);
    if (e != cudaSuccess || !p)
      tl::fail(TL_ECUDA, std::string("cudaGetSymbolAddress(noalloc scratch): ") +
                             cudaGetErrorString(e));
    g_noalloc_addr[dev] = static_cast<unsigned long long *>(p);
  }
  return g_noalloc_addr[dev];
}

}  // namespace

extern "C" int tl_count_hash_noalloc(const uint32_t *dev_triples, uint64_t n_triples,
                                     uint64_t chunk_index, void *user) {
  (void)chunk_index;
  try {
    tl::clear_error();
    auto *st = static_cast<tl_count_hash_noalloc_state *>(user);
    if (!st || !st->dev_out) tl::fail(TL_EINVAL, "tl_count_hash_noalloc: state or dev_out is NULL");
    if (n_triples > TL_NOALLOC_MAX_TRIPLES)
      tl::fail(TL_EINVAL, "tl_count_hash_noalloc: more than TL_NOALLOC_MAX_TRIPLES triples "
                          "in one call; split the buffer");
    if (n_triples > 0 && !dev_triples)
      tl::fail(TL_EINVAL, "tl_count_hash_noalloc: dev_triples is NULL");
    cudaStream_t s = static_cast<cudaStream_t>(st->stream);
    unsigned long long *scratch = noalloc_scratch();
    const uint32_t blocks = (uint32_t)((n_triples + kNoallocPerBlock - 1) / kNoallocPerBlock);
    if (blocks > 0) {
      k_noalloc_partials<<<blocks, kNoallocThreads, 0, s>>>(dev_triples, n_triples, scratch);
      TL_CHECK_LAUNCH();
    }
    k_noalloc_finish<<<1, kNoallocThreads, 0, s>>>(scratch, blocks, n_triples, st->dev_out);
    TL_CHECK_LAUNCH();
    TL_CUDA(cudaStreamSynchronize(s));
    return 0;
  } catch (const tl::Error &e) {
    tl::set_error(e.msg);
    return 1;
  } catch (...) {
    tl::set_error("tl_count_hash_noalloc: unexpected internal error");
    return 1;
  }
}
