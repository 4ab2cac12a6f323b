// kdfmm_total_momentum_noalloc: the total-momentum reduction with its scratch
// in a fixed device array of this library instead of memory allocated per
// call.  For callers that must not allocate device memory while they run:
// cudaMalloc and cudaFree can synchronise the whole device, can fail or stall
// when another allocator already holds the memory, and are not allowed by
// callers that work inside a fixed memory budget.
//
// The array holds the per-block partial sums of one call (at most
// kMomentumMaxBlocks blocks, 6 doubles each: 48 KiB), and every GPU that loads
// the library keeps it until the process exits.  All calls share it: each call
// overwrites every partial it later reads, so nothing has to be cleared
// between calls, but calls whose work overlaps on the GPU (for example on two
// streams at once) race on it.
#include <mutex>

#include "kdfmm_internal.cuh"

namespace kdfmm {

int64_t momentum_blocks(int64_t n);

namespace {

constexpr int kMomentumMaxBlocks = 1024;            // momentum_blocks() never exceeds this
constexpr int64_t kNoallocMaxN = int64_t(1) << 30;  // same particle limit as the tree build
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_momentum_scratch[kMomentumMaxBlocks * 6];

// Device address of g_momentum_scratch per device, looked up once: in host
// code the symbol itself is only a host-side stand-in.
std::mutex g_lock;
double* g_scratch_ptr[kMaxDevices] = {};

int scratch_for_current_device(double** out) {
  int dev = 0;
  int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  if (dev < 0 || dev >= kMaxDevices)
    return set_error(KDFMM_ERR_INVALID_ARG, "device %d beyond the %d supported", dev, kMaxDevices);
  std::lock_guard<std::mutex> guard(g_lock);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    rc = check_cuda(cudaGetSymbolAddress(&p, g_momentum_scratch), "cudaGetSymbolAddress");
    if (rc) return rc;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return KDFMM_OK;
}

bool on_device(const void* p) {
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace kdfmm

extern "C" int kdfmm_total_momentum_noalloc(const double* m, const double* v, int64_t n,
                                            double* out, void* stream) {
  using namespace kdfmm;
  if (n < 1 || n > kNoallocMaxN)
    return set_error(KDFMM_ERR_INVALID_ARG,
                     "n must lie in [1, %lld] for the allocation-free reduction (got %lld)",
                     (long long)kNoallocMaxN, (long long)n);
  if (momentum_blocks(n) > kMomentumMaxBlocks)
    return set_error(KDFMM_ERR_INVALID_ARG, "n = %lld needs more than %d partial sums",
                     (long long)n, kMomentumMaxBlocks);
  if (!m || !v || !out || !on_device(m) || !on_device(v) || !on_device(out))
    return set_error(KDFMM_ERR_INVALID_ARG, "m, v and out must be device pointers");
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc) return rc;
  return momentum(m, v, n, out, scratch, static_cast<cudaStream_t>(stream));
}
