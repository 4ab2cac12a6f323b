// Device-wide exclusive scans (build finalisation, list offsets) and the total
// momentum reduction sum_i m_i v_i (Sec. 4, Eq. 30: the total force the
// leaf-only walk fails to cancel).
#include "kdfmm_internal.cuh"

namespace kdfmm {

namespace {

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

template <class T>
__device__ __forceinline__ T warp_incl_scan(T v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T w = __shfl_up_sync(0xffffffffu, v, o);
    if (lane >= o) v += w;
  }
  return v;
}

// Exclusive scan of one tile per block; the block total goes to tot[block].
// n_dev, when given, holds the element count (at most n); the launch is sized
// for n.
template <class TO>
__global__ void k_scan_tile(const int32_t* __restrict__ in, TO* __restrict__ out, int64_t n,
                            const int32_t* __restrict__ n_dev, TO* __restrict__ tot) {
  __shared__ TO warp_tot[kScanThreads / 32];
  if (n_dev) n = *n_dev;
  const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
  TO v[kScanPer];
  TO run = 0;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    int64_t i = base + k;
    TO e = i < n ? (TO)in[i] : (TO)0;
    v[k] = run;
    run += e;
  }
  TO incl = warp_incl_scan<TO>(run);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 31) warp_tot[w] = incl;
  __syncthreads();
  if (w == 0) {
    TO t = lane < kScanThreads / 32 ? warp_tot[lane] : (TO)0;
    TO ti = warp_incl_scan<TO>(t);
    if (lane < kScanThreads / 32) warp_tot[lane] = ti - t;
    if (lane == kScanThreads / 32 - 1) tot[blockIdx.x] = ti;
  }
  __syncthreads();
  TO off = warp_tot[w] + incl - run;
#pragma unroll
  for (int k = 0; k < kScanPer; ++k) {
    int64_t i = base + k;
    if (i < n) out[i] = off + v[k];
  }
}

// Exclusive scan of the nb block totals in place, tot[nb] = grand total.
template <class TO>
__global__ void k_scan_top(TO* tot, int64_t nb) {
  __shared__ TO warp_tot[32];
  __shared__ TO carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int64_t base = 0; base < nb; base += blockDim.x) {
    int64_t i = base + threadIdx.x;
    TO e = i < nb ? tot[i] : (TO)0;
    TO incl = warp_incl_scan<TO>(e);
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
      TO t = lane < (int)(blockDim.x / 32) ? warp_tot[lane] : (TO)0;
      TO ti = warp_incl_scan<TO>(t);
      warp_tot[lane] = ti - t;
    }
    __syncthreads();
    TO excl = carry + warp_tot[w] + incl - e;
    __syncthreads();
    if (i < nb) tot[i] = excl;
    if (threadIdx.x == blockDim.x - 1) carry = excl + e;
    __syncthreads();
  }
  if (threadIdx.x == 0) tot[nb] = carry;
}

template <class TO>
__global__ void k_scan_add(TO* __restrict__ out, int64_t n, const int32_t* __restrict__ n_dev,
                           const TO* __restrict__ tot, int64_t nb) {
  if (n_dev) n = *n_dev;
  const int64_t base = (int64_t)blockIdx.x * kScanTile;
  const TO off = tot[blockIdx.x];
  for (int k = threadIdx.x; k < kScanTile; k += blockDim.x) {
    int64_t i = base + k;
    if (i < n) out[i] += off;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) out[n] = tot[nb];
}

template <class TO>
void scan_impl(const int32_t* in, TO* out, int64_t n, const int32_t* n_dev, TO* tmp,
               cudaStream_t s) {
  int64_t nb = (n + kScanTile - 1) / kScanTile;
  if (nb == 0) {
    cudaMemsetAsync(out, 0, sizeof(TO), s);
    return;
  }
  k_scan_tile<TO><<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, n_dev, tmp);
  k_scan_top<TO><<<1, 1024, 0, s>>>(tmp, nb);
  k_scan_add<TO><<<(unsigned)nb, kScanThreads, 0, s>>>(out, n, n_dev, tmp, nb);
}

// ---------------------------------------------------------------------------
// total momentum
// ---------------------------------------------------------------------------
constexpr int kMomThreads = 256;

// Each block sums its contiguous range in plain float64 per thread, then
// combines its threads with two-sum in a fixed order: partial = (hi, lo) x 3.
__global__ void k_momentum_blocks(const double* __restrict__ m, const double* __restrict__ v,
                                  int64_t n, int64_t per_block, double* __restrict__ part) {
  __shared__ double sh[kMomThreads][6];
  const int64_t lo = (int64_t)blockIdx.x * per_block;
  const int64_t hi = min(n, lo + per_block);
  double ax = 0.0, ay = 0.0, az = 0.0;
  for (int64_t i = lo + threadIdx.x; i < hi; i += kMomThreads) {
    double mi = m[i];
    ax = __dadd_rn(ax, __dmul_rn(mi, v[3 * i + 0]));
    ay = __dadd_rn(ay, __dmul_rn(mi, v[3 * i + 1]));
    az = __dadd_rn(az, __dmul_rn(mi, v[3 * i + 2]));
  }
  sh[threadIdx.x][0] = ax; sh[threadIdx.x][1] = 0.0;
  sh[threadIdx.x][2] = ay; sh[threadIdx.x][3] = 0.0;
  sh[threadIdx.x][4] = az; sh[threadIdx.x][5] = 0.0;
  __syncthreads();
  for (int stride = kMomThreads / 2; stride > 0; stride >>= 1) {
    if (threadIdx.x < stride) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double s, e;
        two_sum_d(sh[threadIdx.x][2 * c], sh[threadIdx.x + stride][2 * c], s, e);
        sh[threadIdx.x][2 * c] = s;
        sh[threadIdx.x][2 * c + 1] =
            __dadd_rn(__dadd_rn(sh[threadIdx.x][2 * c + 1], sh[threadIdx.x + stride][2 * c + 1]), e);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < 6) part[6 * blockIdx.x + threadIdx.x] = sh[0][threadIdx.x];
}

// Combines the partials: thread t folds partials t, t + 256, ... with two-sum,
// then a fixed-order tree over the threads.  Deterministic for a given count.
__global__ void k_momentum_final(const double* __restrict__ part, int nb, double* __restrict__ out) {
  __shared__ double sh[kMomThreads][6];
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (int b = threadIdx.x; b < nb; b += kMomThreads) {
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      double s, e;
      two_sum_d(v[2 * c], part[6 * b + 2 * c], s, e);
      v[2 * c] = s;
      v[2 * c + 1] = __dadd_rn(__dadd_rn(v[2 * c + 1], part[6 * b + 2 * c + 1]), e);
    }
  }
  for (int j = 0; j < 6; ++j) sh[threadIdx.x][j] = v[j];
  __syncthreads();
  for (int stride = kMomThreads / 2; stride > 0; stride >>= 1) {
    if (threadIdx.x < stride) {
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        double s, e;
        two_sum_d(sh[threadIdx.x][2 * c], sh[threadIdx.x + stride][2 * c], s, e);
        sh[threadIdx.x][2 * c] = s;
        sh[threadIdx.x][2 * c + 1] =
            __dadd_rn(__dadd_rn(sh[threadIdx.x][2 * c + 1], sh[threadIdx.x + stride][2 * c + 1]), e);
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < 3) out[threadIdx.x] = __dadd_rn(sh[0][2 * threadIdx.x], sh[0][2 * threadIdx.x + 1]);
}

}  // namespace

int64_t scan_tmp_elems(int64_t n) { return (n + kScanTile - 1) / kScanTile + 2; }

void scan_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, cudaStream_t s) {
  scan_impl<int32_t>(in, out, n, nullptr, tmp, s);
}

void scan_i32_dev(const int32_t* in, int32_t* out, const int32_t* n_dev, int64_t cap, int32_t* tmp,
                  cudaStream_t s) {
  scan_impl<int32_t>(in, out, cap, n_dev, tmp, s);
}

void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s) {
  scan_impl<int64_t>(in, out, n, nullptr, tmp, s);
}

int64_t momentum_blocks(int64_t n) {
  int64_t nb = (n + 4095) / 4096;
  if (nb > 1024) nb = 1024;
  if (nb < 1) nb = 1;
  return nb;
}

int momentum(const double* m, const double* v, int64_t n, double* out, double* scratch,
             cudaStream_t s) {
  int64_t nb = momentum_blocks(n);
  int64_t per = (n + nb - 1) / nb;
  k_momentum_blocks<<<(unsigned)nb, kMomThreads, 0, s>>>(m, v, n, per, scratch);
  k_momentum_final<<<1, kMomThreads, 0, s>>>(scratch, (int)nb, out);
  return check_cuda(cudaGetLastError(), "momentum launch");
}

}  // namespace kdfmm
