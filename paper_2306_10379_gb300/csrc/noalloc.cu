// An allocation-free variant of the df64 Gram product, for callers that may
// not allocate device memory at call time: code running while a CUDA graph is
// being captured into a pool it does not own, real-time or embedded callers
// that forbid allocation after start-up, or hosts whose allocator is not
// reachable from the calling thread. The per-block partial sums live in one
// file-scope __device__ array instead of a cudaMalloc'd buffer.
#include <atomic>

#include "oz.cuh"

namespace gsi {

// 8 MiB of partial sums: at most (number of SMs) x 4096 df64 values are used
// for any p, q <= 128 (the split count times the output blocks never exceeds
// the SM count), i.e. 4.75 MiB on a 152-SM GB300. Every device that loads the
// library holds this array until the process exits.
constexpr size_t NOALLOC_SCRATCH_BYTES = (size_t)8 << 20;
static __device__ __align__(256) float2 g_gram_scratch[NOALLOC_SCRATCH_BYTES / sizeof(float2)];

namespace {
constexpr int kMaxDevices = 64;
// Device address of g_gram_scratch per device. Threads making their first
// call on a device at the same time all store the same value, so relaxed
// atomics suffice. The cache assumes the device's primary context lives until
// the process exits: after a cudaDeviceReset the next context places the
// array anew, and the cached address would be stale.
std::atomic<void*> g_scratch_addr[kMaxDevices] = {};
}  // namespace

}  // namespace gsi

using namespace gsi;

extern "C" gsi_status gsi_oz_gram_noalloc(int64_t n, int32_t p, int32_t q, const float* U,
                                          const float* V, int32_t sym, double* G, void* stream) {
  if (n < 0 || p < 1 || q < 1 || p > 128 || q > 128 || !G || (n > 0 && (!U || !V)) ||
      (sym && (p != q || U != V)))
    return GSI_ERR_ARG;
  if (oz_gram_scratch_bytes(n, p, q, sym != 0) > NOALLOC_SCRATCH_BYTES) {
    set_last_error("gsi_oz_gram_noalloc: partial sums exceed the 8 MiB static scratch");
    return GSI_ERR_ARG;
  }
  int dev = 0;
  GSI_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return GSI_ERR_ARG;
  // The array's name is a host-side stand-in in host code; the device address
  // is looked up once per device, with that device current.
  void* ptr = g_scratch_addr[dev].load(std::memory_order_relaxed);
  if (!ptr) {
    GSI_CUDA_TRY(cudaGetSymbolAddress(&ptr, g_gram_scratch));
    g_scratch_addr[dev].store(ptr, std::memory_order_relaxed);
  }
  return oz_gram(n, p, q, reinterpret_cast<const float2*>(U), reinterpret_cast<const float2*>(V),
                 sym != 0, G, reinterpret_cast<float2*>(ptr), (cudaStream_t)stream);
}
