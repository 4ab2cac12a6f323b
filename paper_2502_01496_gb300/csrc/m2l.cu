// M2L (Sec. 2, Eq. 6): the field of a source cell beta (mass M, traceless
// quadrupole Q of Eq. 7) about the sink leaf's centre of mass, r = com_alpha -
// com_beta, expanded so that L2P (Eq. 8) can evaluate it at the particles.
//
// The local expansion is stored as the Cartesian derivatives of the potential
//   Phi(R) = -M/R - Q_jk R_j R_k / (2 R^5) = -M D0 - (1/6) Q_jk D2_jk,
// D_n = grad^n (1/R), up to third order (20 numbers): C0 = Phi, C1 = grad Phi,
// C2, C3.  Eq. 6 is a = -C1 and the Taylor terms of Eq. 8 are -C2 x and
// -(1/2) C3 x x.  With g_n the n-th derivative of (2 rho)^(-1/2) at rho =
// R^2/2 (g_n = (-1)^n (2n-1)!! / R^(2n+1)), q = R.Q.R and u = Q.R:
//   C0    = -M g0 - g2 q / 6
//   C1_i  = s1 R_i + t2 u_i
//   C2_ab = s2 R_a R_b + s1 d_ab + t3 (R_a u_b + R_b u_a) + t2 Q_ab
//   C3_abc= s3 R_a R_b R_c + s2 (d_ab R_c + d_ac R_b + d_bc R_a)
//         + t4 (R_b R_c u_a + R_a R_c u_b + R_a R_b u_c)
//         + t3 (R_a Q_bc + R_b Q_ac + R_c Q_ab + d_ab u_c + d_ac u_b + d_bc u_a)
// with s_n = -M g_n - g_(n+2) q / 6 and t_n = -g_n / 3.
//
// The standard p = 3 series (sink and source orders adding up to at most 2 in
// the acceleration, the multipole section of the paper) differs only in
// dropping the quadrupole's C2 and C3 terms (template flag STD).
//
// One warp per sink leaf; its lanes take the far cells in turn.  Mixed mode
// works in float32, except the monopole's share of C0 and C1 (-M/R and
// M R/R^3, the terms that carry the forces between cells and so the total
// force of Sec. 4): those are formed in float-float arithmetic (error-free
// products with FMA, compensated R^2, one Newton step on the reciprocal
// square root) from R = com_alpha - com_beta taken exactly from the (high,
// low) float centres, and C0 and C1 are summed with compensation.  Plain
// float32 there left a total force 1e-3 off the float64 one at theta = 0.3.
// FP64 mode works in float64 throughout.
#include <algorithm>
#include <climits>

#include "kdfmm_internal.cuh"

namespace kdfmm {

namespace {

template <class T>
__device__ __forceinline__ T rsqrt_t(T v);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float v) { return rsqrtf(v); }
template <>
__device__ __forceinline__ double rsqrt_t<double>(double v) { return rsqrt(v); }

// Error-free transforms (float32): a * b = p + e exactly (FMA), and the
// float-float monopole of a far cell: C0 = -M / R and C1 = M R / R^3 as
// (high, low) pairs from R = (Rh + Rl).
__device__ __forceinline__ void two_prod(float a, float b, float& p, float& e) {
  p = a * b;
  e = fmaf(a, b, -p);
}
__device__ __forceinline__ void fast_two_sum(float a, float b, float& s, float& e) {
  s = a + b;
  e = b - (s - a);
}
__device__ __forceinline__ void monopole_ff(const float Rh[3], const float Rl[3], float M,
                                            float C0[2], float C1[3][2]) {
  // R^2 = S + sl
  float p0, e0, p1, e1, p2, e2;
  two_prod(Rh[0], Rh[0], p0, e0);
  two_prod(Rh[1], Rh[1], p1, e1);
  two_prod(Rh[2], Rh[2], p2, e2);
  float S, t, S2, t2;
  two_sum(p0, p1, S, t);
  two_sum(S, p2, S2, t2);
  const float sl = (t + t2) + (e0 + e1 + e2) +
                   2.0f * fmaf(Rh[0], Rl[0], fmaf(Rh[1], Rl[1], Rh[2] * Rl[2]));
  // y = 1 / sqrt(S2 + sl) = yh + yl: one Newton step on the hardware estimate
  const float y0 = rsqrtf(S2);
  float q, qe;
  two_prod(y0, y0, q, qe);
  const float res = fmaf(-S2, q, 1.0f) - (S2 * qe + sl * q);   // 1 - R^2 y0^2
  const float yl = 0.5f * y0 * res;
  float yh, yl2;
  fast_two_sum(y0, yl, yh, yl2);
  // y^3 = (y^2) y
  float y2, y2e;
  two_prod(yh, yh, y2, y2e);
  y2e += 2.0f * yh * yl2;
  float y3, y3e;
  two_prod(y2, yh, y3, y3e);
  y3e += y2 * yl2 + y2e * yh;
  // M y^3 and M y
  float my3, my3e, my, mye;
  two_prod(M, y3, my3, my3e);
  my3e = fmaf(M, y3e, my3e);
  two_prod(M, yh, my, mye);
  mye = fmaf(M, yl2, mye);
  C0[0] = -my; C0[1] = -mye;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    float c, ce;
    two_prod(my3, Rh[i], c, ce);
    C1[i][0] = c;
    C1[i][1] = ce + fmaf(my3, Rl[i], my3e * Rh[i]);
  }
}

template <class T>
__device__ __forceinline__ T c2e(int a, int b, const T R[3], const T u[3], const T Qm[3][3], T s1,
                                 T s2, T t2, T t3) {
  T v = s2 * R[a] * R[b] + t3 * (R[a] * u[b] + R[b] * u[a]) + t2 * Qm[a][b];
  if (a == b) v += s1;
  return v;
}

template <class T>
__device__ __forceinline__ T c3e(int a, int b, int c, const T R[3], const T u[3], const T Qm[3][3],
                                 T s2, T s3, T t3, T t4) {
  T d = (a == b ? R[c] : T(0)) + (a == c ? R[b] : T(0)) + (b == c ? R[a] : T(0));
  T du = (a == b ? u[c] : T(0)) + (a == c ? u[b] : T(0)) + (b == c ? u[a] : T(0));
  return s3 * R[a] * R[b] * R[c] + s2 * d +
         t4 * (R[b] * R[c] * u[a] + R[a] * R[c] * u[b] + R[a] * R[b] * u[c]) +
         t3 * (R[a] * Qm[b][c] + R[b] * Qm[a][c] + R[c] * Qm[a][b] + du);
}

// Local coefficients of one source: out[0] C0; [1..3] C1 x y z; [4..9] C2 xx
// xy xz yy yz zz; [10..19] C3 xxx xxy xxz xyy xyz xzz yyy yyz yzz zzz.
// STD: the standard p = 3 series (sink and source orders add up to at most
// p - 1 = 2 for the acceleration): the quadrupole keeps only its C0 and C1
// terms, C2 and C3 come from the monopole alone.
// NOMONO01: leave the monopole's share out of C0 and C1 (added separately).
template <class T, bool STD = false, bool NOMONO01 = false>
__device__ __forceinline__ void m2l_coeffs(T Rx, T Ry, T Rz, T M, const T Q[6], T out[20]) {
  const T R[3] = {Rx, Ry, Rz};
  const T Qm[3][3] = {{Q[0], Q[1], Q[2]}, {Q[1], Q[3], Q[4]}, {Q[2], Q[4], Q[5]}};
  const T R2 = Rx * Rx + Ry * Ry + Rz * Rz;
  const T g0 = rsqrt_t<T>(R2);
  const T i2 = g0 * g0;
  const T g1 = -g0 * i2;
  const T g2 = T(-3) * g1 * i2;
  const T g3 = T(-5) * g2 * i2;
  const T g4 = T(-7) * g3 * i2;
  const T g5 = T(-9) * g4 * i2;
  T u[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) u[i] = Qm[i][0] * Rx + Qm[i][1] * Ry + Qm[i][2] * Rz;
  const T q = Rx * u[0] + Ry * u[1] + Rz * u[2];
  const T sixth = T(1) / T(6), third = T(1) / T(3);
  const T qs = q * sixth;
  const T s1 = -M * g1 - g3 * qs;
  const T t2 = -g2 * third;
  out[0] = (NOMONO01 ? T(0) : -M * g0) - g2 * qs;
#pragma unroll
  for (int i = 0; i < 3; ++i) out[1 + i] = (NOMONO01 ? -g3 * qs : s1) * R[i] + t2 * u[i];
  // second and third order: both parts, or the monopole alone (STD)
  const T s1h = STD ? -M * g1 : s1;
  const T s2 = STD ? -M * g2 : -M * g2 - g4 * qs;
  const T s3 = STD ? -M * g3 : -M * g3 - g5 * qs;
  const T t2h = STD ? T(0) : t2;
  const T t3 = STD ? T(0) : -g3 * third, t4 = STD ? T(0) : -g4 * third;
  out[4] = c2e<T>(0, 0, R, u, Qm, s1h, s2, t2h, t3);
  out[5] = c2e<T>(0, 1, R, u, Qm, s1h, s2, t2h, t3);
  out[6] = c2e<T>(0, 2, R, u, Qm, s1h, s2, t2h, t3);
  out[7] = c2e<T>(1, 1, R, u, Qm, s1h, s2, t2h, t3);
  out[8] = c2e<T>(1, 2, R, u, Qm, s1h, s2, t2h, t3);
  out[9] = c2e<T>(2, 2, R, u, Qm, s1h, s2, t2h, t3);
  out[10] = c3e<T>(0, 0, 0, R, u, Qm, s2, s3, t3, t4);
  out[11] = c3e<T>(0, 0, 1, R, u, Qm, s2, s3, t3, t4);
  out[12] = c3e<T>(0, 0, 2, R, u, Qm, s2, s3, t3, t4);
  out[13] = c3e<T>(0, 1, 1, R, u, Qm, s2, s3, t3, t4);
  out[14] = c3e<T>(0, 1, 2, R, u, Qm, s2, s3, t3, t4);
  out[15] = c3e<T>(0, 2, 2, R, u, Qm, s2, s3, t3, t4);
  out[16] = c3e<T>(1, 1, 1, R, u, Qm, s2, s3, t3, t4);
  out[17] = c3e<T>(1, 1, 2, R, u, Qm, s2, s3, t3, t4);
  out[18] = c3e<T>(1, 2, 2, R, u, Qm, s2, s3, t3, t4);
  out[19] = c3e<T>(2, 2, 2, R, u, Qm, s2, s3, t3, t4);
}

struct M2LArgs {
  const int32_t* leaf_cells;
  const int32_t* counters;   // counters[C_LEAVES]: leaves
  int64_t cap_far;           // entries a list may hold (slot size, or no limit)
  int max_leaves;            // leaves the lists were made for
  int nsinks;                // > 0: sinks are cells 0 .. nsinks-1 (leaf_cells unused)
  const int32_t* far_cnt;
  const int32_t* far_idx;
  const int64_t* far_off;
  const float4* src32;
  const double* src64;
  float* lexp32;
  double* lexp64;
};

// Blocks of 128 threads: at ~96 registers a thread, 256-thread blocks fit two
// per SM (16 warps), 128-thread blocks five (20 warps); the extra warps hide
// the two dependent loads per far cell (index, then moments) -- 18 % less
// time on the benchmark workload (1.16 -> 0.95 ms).  Prefetching the next far
// cell instead cost registers and so warps, and was slower.
template <bool STD>
__global__ void __launch_bounds__(128) k_m2l_mixed(M2LArgs A) {
  const int lane = threadIdx.x & 31;
  const int nleaves = A.nsinks > 0 ? A.nsinks : min(A.counters[C_LEAVES], A.max_leaves);
  for (int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); k < nleaves;
       k += (int)((gridDim.x * blockDim.x) >> 5)) {
  const int a = A.nsinks > 0 ? k : A.leaf_cells[k];
  const float4 ah = A.src32[4 * a], al = A.src32[4 * a + 1];
  float acc[20], lo[4];
#pragma unroll
  for (int j = 0; j < 20; ++j) acc[j] = 0.0f;
#pragma unroll
  for (int j = 0; j < 4; ++j) lo[j] = 0.0f;
  const int64_t off = A.far_off[k], nf = min((int64_t)A.far_cnt[k], A.cap_far);
  // the next far cell's index is loaded an iteration ahead, so that each
  // iteration waits on one L2 round trip (the moments) instead of two (6 % off
  // the kernel; loading the next moments ahead too cost more registers than
  // it saved)
  int bn = lane < nf ? A.far_idx[off + lane] : 0;
  for (int64_t e = lane; e < nf; e += 32) {
    const int b = bn;
    if (e + 32 < nf) bn = A.far_idx[off + e + 32];
    const float4 b0 = A.src32[4 * b], b1 = A.src32[4 * b + 1], b2 = A.src32[4 * b + 2],
                 b3 = A.src32[4 * b + 3];
    // R = com_alpha - com_beta as (high, low) from the (high, low) centres
    float Rh[3], Rl[3];
    {
      const float ahv[3] = {ah.x, ah.y, ah.z}, alv[3] = {al.x, al.y, al.z};
      const float bhv[3] = {b0.x, b0.y, b0.z}, blv[3] = {b1.x, b1.y, b1.z};
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        float d, e;
        two_sum(ahv[i], -bhv[i], d, e);
        fast_two_sum(d, (alv[i] - blv[i]) + e, Rh[i], Rl[i]);
      }
    }
    const float Q[6] = {b2.x, b2.y, b2.z, b2.w, b3.x, b3.y};
    float C[20];
    m2l_coeffs<float, STD, true>(Rh[0], Rh[1], Rh[2], b0.w, Q, C);
    float C0[2], C1[3][2];
    monopole_ff(Rh, Rl, b0.w, C0, C1);
    df_add2(acc[0], lo[0], C0[0], C0[1]);
    df_add(acc[0], lo[0], C[0]);
#pragma unroll
    for (int j = 1; j < 4; ++j) {
      df_add2(acc[j], lo[j], C1[j - 1][0], C1[j - 1][1]);
      df_add(acc[j], lo[j], C[j]);
    }
#pragma unroll
    for (int j = 4; j < 20; ++j) acc[j] += C[j];
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      float bh = __shfl_xor_sync(0xffffffffu, acc[j], o);
      float bl = __shfl_xor_sync(0xffffffffu, lo[j], o);
      df_add2(acc[j], lo[j], bh, bl);
    }
#pragma unroll
    for (int j = 4; j < 20; ++j) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
  }
  float* out = A.lexp32 + 24 * (int64_t)k;
  if (lane < 20) {
    float v = acc[0];
#pragma unroll
    for (int j = 1; j < 20; ++j) v = lane == j ? acc[j] : v;
    out[lane] = v;
  } else if (lane < 24) {
    float v = lo[0];
#pragma unroll
    for (int j = 1; j < 4; ++j) v = lane - 20 == j ? lo[j] : v;
    out[lane] = v;
  }
  }
}

template <bool STD>
__global__ void __launch_bounds__(256) k_m2l_fp64(M2LArgs A) {
  const int lane = threadIdx.x & 31;
  const int nleaves = A.nsinks > 0 ? A.nsinks : min(A.counters[C_LEAVES], A.max_leaves);
  for (int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); k < nleaves;
       k += (int)((gridDim.x * blockDim.x) >> 5)) {
  const int a = A.nsinks > 0 ? k : A.leaf_cells[k];
  const double* sa = A.src64 + 10 * (int64_t)a;
  const double ax = sa[0], ay = sa[1], az = sa[2];
  double acc[20];
#pragma unroll
  for (int j = 0; j < 20; ++j) acc[j] = 0.0;
  const int64_t off = A.far_off[k], nf = min((int64_t)A.far_cnt[k], A.cap_far);
  for (int64_t e = lane; e < nf; e += 32) {
    const int b = A.far_idx[off + e];
    const double* sb = A.src64 + 10 * (int64_t)b;
    double C[20];
    m2l_coeffs<double, STD>(ax - sb[0], ay - sb[1], az - sb[2], sb[3], sb + 4, C);
#pragma unroll
    for (int j = 0; j < 20; ++j) acc[j] += C[j];
  }
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
#pragma unroll
    for (int j = 0; j < 20; ++j) acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], o);
  }
  double* out = A.lexp64 + 20 * (int64_t)k;
  if (lane < 20) {
    double v = acc[0];
#pragma unroll
    for (int j = 1; j < 20; ++j) v = lane == j ? acc[j] : v;
    out[lane] = v;
  }
  }
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

int run_m2l(kdfmm_tree_s* t, cudaStream_t s) {
  M2LArgs A{};
  A.leaf_cells = t->leaf_cells;
  A.counters = t->counters;
  A.cap_far = t->L.exact ? INT64_MAX : t->L.cap_far;
  A.max_leaves = std::max(t->grid_leaves, 1);
  A.far_cnt = t->L.far_cnt;
  A.far_off = t->L.far_off;
  A.far_idx = t->L.far_idx;
  A.src32 = t->c.src32;
  A.src64 = t->c.src64;
  A.lexp32 = t->lexp32;
  A.lexp64 = t->lexp64;
  const unsigned g = blocks_for((int64_t)std::max(t->grid_leaves, 1) * 32, 256);
  const unsigned gm = blocks_for((int64_t)std::max(t->grid_leaves, 1) * 32, 128);
  const bool std_exp = t->p.expansion == KDFMM_EXPANSION_STANDARD;
  if (t->p.precision == KDFMM_MIXED) {
    if (std_exp) k_m2l_mixed<true><<<gm, 128, 0, s>>>(A);
    else k_m2l_mixed<false><<<gm, 128, 0, s>>>(A);
  } else {
    if (std_exp) k_m2l_fp64<true><<<g, 256, 0, s>>>(A);
    else k_m2l_fp64<false><<<g, 256, 0, s>>>(A);
  }
  t->launches += 1;
  return check_cuda(cudaGetLastError(), "m2l launch");
}

// M2L into every cell from per-cell far lists (the dual walk): sink cell c's
// list is far_idx[far_off[c] ...) with far_cnt[c] entries; the coefficients go
// to out32 (24 floats per cell) or out64 (20 doubles per cell).
int run_m2l_cells(kdfmm_tree_s* t, const int32_t* far_cnt, const int64_t* far_off,
                  const int32_t* far_idx, float* out32, double* out64, cudaStream_t s) {
  M2LArgs A{};
  A.leaf_cells = nullptr;
  A.counters = t->counters;
  A.cap_far = INT64_MAX;
  A.max_leaves = t->ncells;
  A.nsinks = t->ncells;
  A.far_cnt = far_cnt;
  A.far_off = far_off;
  A.far_idx = far_idx;
  A.src32 = t->c.src32;
  A.src64 = t->c.src64;
  A.lexp32 = out32;
  A.lexp64 = out64;
  const unsigned g = blocks_for((int64_t)std::max(t->ncells, 1) * 32, 256);
  const unsigned gm = blocks_for((int64_t)std::max(t->ncells, 1) * 32, 128);
  const bool std_exp = t->p.expansion == KDFMM_EXPANSION_STANDARD;
  if (t->p.precision == KDFMM_MIXED) {
    if (std_exp) k_m2l_mixed<true><<<gm, 128, 0, s>>>(A);
    else k_m2l_mixed<false><<<gm, 128, 0, s>>>(A);
  } else {
    if (std_exp) k_m2l_fp64<true><<<g, 256, 0, s>>>(A);
    else k_m2l_fp64<false><<<g, 256, 0, s>>>(A);
  }
  t->launches += 1;
  return check_cuda(cudaGetLastError(), "m2l (cells) launch");
}

}  // namespace kdfmm
