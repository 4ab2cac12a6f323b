// Measured arithmetic throughput of the current device: float32 and float64
// fused multiply-adds (the units that bound the P2P and M2L kernels) and the
// derived float32 peak from the device's SM count and maximum clock.  These
// are the denominators of the ALU roofline; the paper has no counterpart.
#include <algorithm>

#include "kdfmm_internal.cuh"

namespace kdfmm {
namespace {

constexpr int kPeakIters = 4096;   // FMA rounds per chain
constexpr int kPeakThreads = 256;
constexpr int kPeakBlocksPerSm = 8;

// 16 independent float32 FMA chains per thread (enough to cover the FMA
// latency at full occupancy); the sum is stored so nothing is dead code.
__global__ void __launch_bounds__(kPeakThreads) k_ffma_peak(float* out, float a, float b) {
  float c[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) c[i] = (float)threadIdx.x * 1e-3f + (float)i;
  for (int it = 0; it < kPeakIters; ++it) {
#pragma unroll
    for (int i = 0; i < 16; ++i) c[i] = fmaf(c[i], a, b);
  }
  float s = 0.0f;
#pragma unroll
  for (int i = 0; i < 16; ++i) s += c[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

// 8 independent float64 FMA chains per thread, an eighth of the rounds.
__global__ void __launch_bounds__(kPeakThreads) k_dfma_peak(double* out, double a, double b) {
  double c[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) c[i] = (double)threadIdx.x * 1e-3 + (double)i;
  for (int it = 0; it < kPeakIters / 8; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) c[i] = fma(c[i], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += c[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace
}  // namespace kdfmm

using namespace kdfmm;

extern "C" int kdfmm_measure_peaks(double* out, void* stream) {
  if (!out) return set_error(KDFMM_ERR_INVALID_ARG, "out is NULL");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0, clk_khz = 0;
  int rc = check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
  if (rc) return rc;
  rc = check_cuda(cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev), "clock rate");
  if (rc) return rc;
  const int sms = sm_count();
  const unsigned blocks = (unsigned)(sms * kPeakBlocksPerSm);
  const size_t nthr = (size_t)blocks * kPeakThreads;
  double* sink = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaMalloc(&sink, nthr * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(KDFMM_ERR_OOM, "peak probe buffer");
  }
  rc = check_cuda(cudaEventCreate(&e0), "event");
  if (!rc) rc = check_cuda(cudaEventCreate(&e1), "event");
  float best32 = 1e30f, best64 = 1e30f;
  for (int rep = 0; rep < 4 && !rc; ++rep) {       // the first round warms up
    float ms = 0.0f;
    cudaEventRecord(e0, s);
    k_ffma_peak<<<blocks, kPeakThreads, 0, s>>>(reinterpret_cast<float*>(sink), 0.999f, 1e-3f);
    cudaEventRecord(e1, s);
    rc = check_cuda(cudaEventSynchronize(e1), "ffma probe");
    if (rc) break;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best32 = std::min(best32, ms);
    cudaEventRecord(e0, s);
    k_dfma_peak<<<blocks, kPeakThreads, 0, s>>>(sink, 0.999, 1e-3);
    cudaEventRecord(e1, s);
    rc = check_cuda(cudaEventSynchronize(e1), "dfma probe");
    if (rc) break;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best64 = std::min(best64, ms);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(sink);
  if (rc) return rc;
  out[0] = (double)nthr * 16.0 * kPeakIters * 2.0 / (best32 * 1e-3) / 1e12;
  out[1] = (double)nthr * 8.0 * (kPeakIters / 8) * 2.0 / (best64 * 1e-3) / 1e12;
  out[2] = (double)sms;
  out[3] = clk_khz / 1e3;
  out[4] = (double)sms * 128.0 * 2.0 * (clk_khz * 1e3) / 1e12;
  return KDFMM_OK;
}
