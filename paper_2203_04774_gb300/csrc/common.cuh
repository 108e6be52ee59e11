// Internal declarations shared by the translation units of libtl.
// Nothing here is part of the C ABI (include/tl.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "../../include/tl.h"

namespace tl {

// ---- error reporting --------------------------------------------------------

void set_error(const std::string &msg);
void clear_error();

struct Error {
  tl_status status;
  std::string msg;
};

// Throws tl::Error on a CUDA failure; the C-ABI wrappers catch it.
#define TL_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess) {                                                       \
      throw ::tl::Error{e_ == cudaErrorMemoryAllocation ? TL_ENOMEM : TL_ECUDA,    \
                        std::string(#call) + ": " + cudaGetErrorString(e_)};       \
    }                                                                              \
  } while (0)

// Every kernel launch site is followed by TL_CHECK_LAUNCH(), which also
// counts the launch (tl_kernel_launches).
void count_launch();
#define TL_CHECK_LAUNCH()          \
  do {                             \
    ::tl::count_launch();          \
    TL_CUDA(cudaGetLastError());   \
  } while (0)

inline void fail(tl_status s, const std::string &msg) { throw Error{s, msg}; }

// ---- device buffer (RAII, stream-ordered) ------------------------------------

// The current device's default memory pool; each call sets its release
// threshold to the bytes in use + 8 GiB, so that up to 8 GiB of freed memory
// stays cached and buffers of repeated calls are recycled without driver
// round trips.
cudaMemPool_t device_pool();

// Allocations come from the device pool in stream order on `stream` (the
// owning graph's stream; it must outlive the buffer).
struct DevBuf {
  void *p = nullptr;
  size_t bytes = 0;
  cudaStream_t stream = nullptr;
  DevBuf() = default;
  explicit DevBuf(cudaStream_t s) : stream(s) {}
  DevBuf(const DevBuf &) = delete;
  DevBuf &operator=(const DevBuf &) = delete;
  ~DevBuf() { release(); }
  void release() {
    if (p) cudaFreeAsync(p, stream);
    p = nullptr;
    bytes = 0;
  }
  // Grow to at least `b` bytes (contents are not preserved).
  void reserve(size_t b) {
    if (b <= bytes && p) return;
    release();
    size_t want = b ? b : 16;
    TL_CUDA(cudaMallocFromPoolAsync(&p, want, device_pool(), stream));
    bytes = want;
  }
  template <class T> T *as() const { return static_cast<T *>(p); }
};

constexpr int kWarp = 32;

inline int num_sms() {
  // initialised once, thread-safely (a throw leaves it for the next call)
  static const int sms = [] {
    int dev = 0, v = 0;
    TL_CUDA(cudaGetDevice(&dev));
    TL_CUDA(cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev));
    return v;
  }();
  return sms;
}

inline unsigned grid_for(uint64_t items, int block, unsigned cap = 0) {
  uint64_t g = (items + block - 1) / block;
  if (g == 0) g = 1;
  unsigned c = cap ? cap : (unsigned)num_sms() * 16u;
  return (unsigned)(g < c ? g : c);
}

// ---- primitives (scan.cu, sort.cu) ------------------------------------------

// Exclusive prefix sum of uint64 values in place-or-out: out[i] = sum in[0..i),
// out[n] = total (out has n+1 entries).  `tmp` is scratch owned by the caller.
void exclusive_scan_u64(const uint64_t *in, uint64_t *out, uint64_t n, DevBuf &tmp,
                        cudaStream_t s);
// Same for uint32 inputs widened to uint64 sums.
void exclusive_scan_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t n, DevBuf &tmp,
                               cudaStream_t s);

// Stable LSD radix sort of uint64 keys on bit ranges [lo_bit, lo_bit+lo_bits)
// then [hi_bit, hi_bit+hi_bits) (either may be empty).  Result ends in `keys`
// (the alternate buffer `alt` is used as ping-pong storage, same size).
void radix_sort_u64(uint64_t *keys, uint64_t *alt, uint64_t n, int lo_bit, int lo_bits,
                    int hi_bit, int hi_bits, DevBuf &tmp, DevBuf &scan_tmp, cudaStream_t s);

int bits_for(uint64_t max_value);  // number of bits to represent max_value (>= 1)

}  // namespace tl
