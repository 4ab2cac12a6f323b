// Kick and drift of a kick-drift-kick leapfrog, the integrator that carries
// the force evaluation through time (Sec. 4 follows the centre of mass over
// many steps; the paper's own runs rebuild the tree every step).
//   v += dt_kick * a;  x += dt_drift * v   (after the kick)
#include <algorithm>
#include <cmath>

#include "kdfmm_internal.cuh"

namespace kdfmm {
namespace {

__global__ void k_kick_drift(double* __restrict__ x, double* __restrict__ v,
                             const double* __restrict__ a, int64_t n3, double dt_kick,
                             double dt_drift) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n3;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double vi = __dadd_rn(v[i], __dmul_rn(dt_kick, a[i]));
    v[i] = vi;
    if (dt_drift != 0.0) x[i] = __dadd_rn(x[i], __dmul_rn(dt_drift, vi));
  }
}

}  // namespace
}  // namespace kdfmm

using namespace kdfmm;

extern "C" int kdfmm_kick_drift(double* x, double* v, const double* a, int64_t n, double dt_kick,
                                double dt_drift, void* stream) {
  if (n < 1 || n > (int64_t(1) << 30))
    return set_error(KDFMM_ERR_INVALID_ARG, "n must lie in [1, 2^30] (got %lld)", (long long)n);
  if (!(std::isfinite(dt_kick) && std::isfinite(dt_drift)))
    return set_error(KDFMM_ERR_INVALID_ARG, "time steps must be finite");
  if (!x || !v || !a) return set_error(KDFMM_ERR_INVALID_ARG, "x, v and a must not be NULL");
  cudaPointerAttributes at{};
  for (const void* p : {(const void*)x, (const void*)v, (const void*)a}) {
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess ||
        (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)) {
      cudaGetLastError();
      return set_error(KDFMM_ERR_INVALID_ARG, "x, v and a must be device pointers");
    }
  }
  const int64_t n3 = 3 * n;
  const unsigned blocks = (unsigned)std::min<int64_t>((n3 + 255) / 256, grid_blocks(16));
  k_kick_drift<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(x, v, a, n3, dt_kick,
                                                                       dt_drift);
  return check_cuda(cudaGetLastError(), "kick_drift launch");
}
