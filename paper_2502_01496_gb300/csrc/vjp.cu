// Vector-Jacobian product of one force evaluation with respect to positions
// and masses, through the same tree and interaction lists (topology, lists
// and smoothing lengths held fixed).  The paper has no adjoint; this is the
// derivative of the evaluation of Sec. 2 (Eqs. 3, 6, 7, 8, 13).  FP64 mode
// runs every step in float64; mixed mode runs the M2L and P2P reverses with
// float32 terms (as its forward does) and float64 sums.
//
// a_i = sum_{j in near(leaf i), j != i} m_j K(x_i - x_j)            (P2P)
//     + L(C_alpha, x_i - com_alpha)                                (L2P, Eq. 8)
// C_alpha = sum_{beta in far(alpha)} C(com_alpha - com_beta, M_beta, Q_beta)   (M2L, Eq. 6)
// with M, com = S/M (S = sum m x) and Q (Eq. 7) functions of the particles.
//
// Reverse order: L2P (cotangents of each leaf's expansion and of x_i, com),
// M2L (cotangents of r = com_alpha - com_beta, M_beta, Q_beta: C is linear in M
// and Q, its r-derivatives come from dual numbers), P2P on the target side and
// on the source side, then the moments: per cell the
// cotangents (M_bar, com_bar, Q_bar) give m_bar_i and x_bar_i as a quadratic
// polynomial in x_i, summed over the leaf's chain of ancestors.
#include <algorithm>
#include <climits>

#include "kdfmm_internal.cuh"

namespace kdfmm {

namespace {

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// ---------------------------------------------------------------------------
// M2L coefficients (same closed forms as the forward) on a dual-number type
// ---------------------------------------------------------------------------
// S: the scalar (double, or float in mixed mode); d holds the derivatives
// with respect to the three components of r.
template <class S>
struct DualT {
  S v, d[3];
};
template <class S>
__device__ __forceinline__ DualT<S> operator+(const DualT<S>& a, const DualT<S>& b) {
  return DualT<S>{a.v + b.v, {a.d[0] + b.d[0], a.d[1] + b.d[1], a.d[2] + b.d[2]}};
}
template <class S>
__device__ __forceinline__ DualT<S> operator-(const DualT<S>& a, const DualT<S>& b) {
  return DualT<S>{a.v - b.v, {a.d[0] - b.d[0], a.d[1] - b.d[1], a.d[2] - b.d[2]}};
}
template <class S>
__device__ __forceinline__ DualT<S> operator-(const DualT<S>& a) {
  return DualT<S>{-a.v, {-a.d[0], -a.d[1], -a.d[2]}};
}
template <class S>
__device__ __forceinline__ DualT<S> operator*(const DualT<S>& a, const DualT<S>& b) {
  return DualT<S>{a.v * b.v,
                  {a.d[0] * b.v + a.v * b.d[0], a.d[1] * b.v + a.v * b.d[1],
                   a.d[2] * b.v + a.v * b.d[2]}};
}
template <class S>
__device__ __forceinline__ DualT<S>& operator+=(DualT<S>& a, const DualT<S>& b) { return a = a + b; }

__device__ __forceinline__ double rsq(double v) { return 1.0 / sqrt(v); }
__device__ __forceinline__ float rsq(float v) { return rsqrtf(v); }

template <class S>
__device__ __forceinline__ DualT<S> rsqrt_dual(const DualT<S>& a) {
  const S r = rsq(a.v);
  const S dr = S(-0.5) * r / a.v;
  return DualT<S>{r, {dr * a.d[0], dr * a.d[1], dr * a.d[2]}};
}

template <class T>
__device__ __forceinline__ T tc(double v);
template <>
__device__ __forceinline__ double tc<double>(double v) { return v; }
template <>
__device__ __forceinline__ float tc<float>(double v) { return (float)v; }
template <>
__device__ __forceinline__ DualT<double> tc<DualT<double>>(double v) {
  return DualT<double>{v, {0.0, 0.0, 0.0}};
}
template <>
__device__ __forceinline__ DualT<float> tc<DualT<float>>(double v) {
  return DualT<float>{(float)v, {0.0f, 0.0f, 0.0f}};
}

__device__ __forceinline__ double rs(double v) { return rsq(v); }
__device__ __forceinline__ float rs(float v) { return rsq(v); }
template <class S>
__device__ __forceinline__ DualT<S> rs(const DualT<S>& v) { return rsqrt_dual(v); }

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
  T d = tc<T>(0.0), du = tc<T>(0.0);
  if (a == b) { d += R[c]; du += u[c]; }
  if (a == c) { d += R[b]; du += u[b]; }
  if (b == c) { d += R[a]; du += u[a]; }
  return s3 * R[a] * R[b] * R[c] + s2 * d +
         t4 * (R[b] * R[c] * u[a] + R[a] * R[c] * u[b] + R[a] * R[b] * u[c]) +
         t3 * (R[a] * Qm[b][c] + R[b] * Qm[a][c] + R[c] * Qm[a][b] + du);
}

// sum_j w_j C_j over the 20 compact coefficients C0, C1 (3), C2 (6), C3 (10)
// of the potential Phi = -M/R - Q_jk R_j R_k / (2 R^5) and its derivatives
// (the closed forms of m2l.cu); contracting as each coefficient is formed
// keeps one accumulator instead of twenty.
// STD: the standard p = 3 series -- the quadrupole keeps only its C0 and C1
// terms (as in m2l.cu).
template <class T, bool STD>
__device__ T m2l_contract(const T R[3], double M, const double Q[6], const double w[20]) {
  const T Qm[3][3] = {{tc<T>(Q[0]), tc<T>(Q[1]), tc<T>(Q[2])},
                      {tc<T>(Q[1]), tc<T>(Q[3]), tc<T>(Q[4])},
                      {tc<T>(Q[2]), tc<T>(Q[4]), tc<T>(Q[5])}};
  const T R2 = R[0] * R[0] + R[1] * R[1] + R[2] * R[2];
  const T g0 = rs(R2);
  const T i2 = g0 * g0;
  const T g1 = -(g0 * i2);
  const T g2 = tc<T>(-3.0) * g1 * i2;
  const T g3 = tc<T>(-5.0) * g2 * i2;
  const T g4 = tc<T>(-7.0) * g3 * i2;
  const T g5 = tc<T>(-9.0) * g4 * i2;
  T u[3];
  for (int i = 0; i < 3; ++i) u[i] = Qm[i][0] * R[0] + Qm[i][1] * R[1] + Qm[i][2] * R[2];
  const T q = R[0] * u[0] + R[1] * u[1] + R[2] * u[2];
  const T qs = q * tc<T>(1.0 / 6.0);
  const T Mt = tc<T>(M);
  const T s1 = -(Mt * g1) - g3 * qs;
  const T t2 = g2 * tc<T>(-1.0 / 3.0);
  T acc = tc<T>(w[0]) * (-(Mt * g0) - g2 * qs);
  for (int i = 0; i < 3; ++i) acc += tc<T>(w[1 + i]) * (s1 * R[i] + t2 * u[i]);
  const T s1h = STD ? -(Mt * g1) : s1;
  const T s2 = STD ? -(Mt * g2) : -(Mt * g2) - g4 * qs;
  const T s3 = STD ? -(Mt * g3) : -(Mt * g3) - g5 * qs;
  const T t2h = STD ? tc<T>(0.0) : t2;
  const T t3 = STD ? tc<T>(0.0) : g3 * tc<T>(-1.0 / 3.0);
  const T t4 = STD ? tc<T>(0.0) : g4 * tc<T>(-1.0 / 3.0);
  const int c2a[6] = {0, 0, 0, 1, 1, 2}, c2b[6] = {0, 1, 2, 1, 2, 2};
#pragma unroll
  for (int k = 0; k < 6; ++k)
    acc += tc<T>(w[4 + k]) * c2e<T>(c2a[k], c2b[k], R, u, Qm, s1h, s2, t2h, t3);
  const int c3a[10] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 2}, c3b[10] = {0, 0, 0, 1, 1, 2, 1, 1, 2, 2},
            c3c[10] = {0, 1, 2, 1, 2, 2, 1, 2, 2, 2};
#pragma unroll
  for (int k = 0; k < 10; ++k)
    acc += tc<T>(w[10 + k]) * c3e<T>(c3a[k], c3b[k], c3c[k], R, u, Qm, s2, s3, t3, t4);
  return acc;
}

// index of the compact C2 entry (a, b) and C3 entry (a, b, c)
__device__ __forceinline__ int c2i(int a, int b) {
  if (a > b) { int t = a; a = b; b = t; }
  return a == 0 ? 4 + b : (a == 1 ? 6 + b : 9);
}
__device__ __forceinline__ int c3i(int a, int b, int c) {
  // sort a <= b <= c
  if (a > b) { int t = a; a = b; b = t; }
  if (b > c) { int t = b; b = c; c = t; }
  if (a > b) { int t = a; a = b; b = t; }
  if (a == 0) return b == 0 ? 10 + c : (b == 1 ? 12 + c : 15);
  if (a == 1) return b == 1 ? 15 + c : 18;
  return 19;
}

// ---------------------------------------------------------------------------
// kernels
// ---------------------------------------------------------------------------
struct VjpArgs {
  int64_t n;
  int nleaves, ncells;
  int soft_kind;
  bool mixed;
  const int32_t* leaf_sys;
  const double* sys_eps;
  const int32_t* leaf_cells;
  const int32_t* leaf_rank;
  Cells c;
  PCols tp;
  const float* lexp32;
  const double* lexp64;
  const int32_t *far_cnt, *far_idx, *near_cnt, *near_idx;
  const int64_t *far_off, *near_off;
  int64_t cap_far, cap_near;            // entries a list may hold
  double* ab;                           // cotangent in tree order (N x 3)
  double* xbar;                         // tree order (N x 3)
  double* mbar;                         // tree order (N)
  double* xsrc;                         // P2P source-side part of x_bar (N x 3, atomics)
  double* msrc;                         // P2P source-side part of m_bar (N, atomics)
  double* cbar;                         // per leaf: 20 expansion cotangents
  double* cell_bar;                     // per cell: M_bar, com_bar (3), Q_bar (6)
  // the evaluation's split of long near lists (segment items after the
  // leaves; their target-side partial sums are added in segment order)
  const int32_t* counters;
  const int32_t *seg_first, *seg_leaf;
  double* seg_part;
  int64_t seg_cap;
};

__global__ void k_gather_abar(const double* __restrict__ abar, VjpArgs V) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= V.n) return;
  const int64_t i = V.tp.idx[p];
  V.ab[3 * p] = abar[3 * i];
  V.ab[3 * p + 1] = abar[3 * i + 1];
  V.ab[3 * p + 2] = abar[3 * i + 2];
  V.xbar[3 * p] = V.xbar[3 * p + 1] = V.xbar[3 * p + 2] = 0.0;
  V.xsrc[3 * p] = V.xsrc[3 * p + 1] = V.xsrc[3 * p + 2] = 0.0;
  V.mbar[p] = V.msrc[p] = 0.0;
}

__device__ __forceinline__ void load_coeffs(const VjpArgs& V, int k, double C[20]) {
  if (V.mixed) {
    const float* f = V.lexp32 + 24 * (int64_t)k;
    for (int j = 0; j < 20; ++j) C[j] = (double)f[j];
    for (int j = 0; j < 4; ++j) C[j] += (double)f[20 + j];
  } else {
    const double* d = V.lexp64 + 20 * (int64_t)k;
    for (int j = 0; j < 20; ++j) C[j] = d[j];
  }
}

// L2P reverse: warp per leaf, lane per particle.  a_i = -(C1 + C2 x + C3 x x / 2)
// with x = x_i - com_alpha.
__global__ void k_vjp_l2p(VjpArgs V) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= V.nleaves) return;
  const int a = V.leaf_cells[k];
  const int f = V.c.first[a], cnt = V.c.count[a];
  double C[20];
  load_coeffs(V, k, C);
  double cb[20];
  for (int j = 0; j < 20; ++j) cb[j] = 0.0;
  double gx = 0.0, gy = 0.0, gz = 0.0;             // sum of (d a / d x)^T a_bar
  if (lane < cnt) {
    const int64_t p = (int64_t)f + lane;
    const double x[3] = {V.tp.x[p] - V.c.cx[a], V.tp.y[p] - V.c.cy[a], V.tp.z[p] - V.c.cz[a]};
    const double b[3] = {V.ab[3 * p], V.ab[3 * p + 1], V.ab[3 * p + 2]};
    // (d a_i / d x_j) = -(C2_ij + C3_ijk x_k): g_j = sum_i b_i (d a_i / d x_j)
    double g[3];
    for (int jj = 0; jj < 3; ++jj) {
      double s = 0.0;
      for (int ii = 0; ii < 3; ++ii) {
        double t = C[c2i(ii, jj)];
        for (int kk = 0; kk < 3; ++kk) t += C[c3i(ii, jj, kk)] * x[kk];
        s += b[ii] * t;
      }
      g[jj] = -s;
    }
    V.xbar[3 * p] += g[0];
    V.xbar[3 * p + 1] += g[1];
    V.xbar[3 * p + 2] += g[2];
    gx = g[0]; gy = g[1]; gz = g[2];
    // expansion cotangents: a_i depends on C1_i, C2_ij x_j, 1/2 C3_ijk x_j x_k
    for (int ii = 0; ii < 3; ++ii) {
      cb[1 + ii] -= b[ii];
      for (int jj = 0; jj < 3; ++jj) {
        cb[c2i(ii, jj)] -= b[ii] * x[jj];
        for (int kk = 0; kk < 3; ++kk) cb[c3i(ii, jj, kk)] -= 0.5 * b[ii] * x[jj] * x[kk];
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    for (int j = 0; j < 20; ++j) cb[j] += __shfl_xor_sync(0xffffffffu, cb[j], o);
    gx += __shfl_xor_sync(0xffffffffu, gx, o);
    gy += __shfl_xor_sync(0xffffffffu, gy, o);
    gz += __shfl_xor_sync(0xffffffffu, gz, o);
  }
  if (lane == 0) {
    for (int j = 0; j < 20; ++j) V.cbar[20 * (int64_t)k + j] = cb[j];
    // x = x_i - com_alpha: the com receives minus the particles' share
    double* cbc = V.cell_bar + 10 * (int64_t)a;
    atomicAdd(&cbc[1], -gx);
    atomicAdd(&cbc[2], -gy);
    atomicAdd(&cbc[3], -gz);
  }
}

// M2L reverse: warp per sink leaf, lanes over its far cells.  S: arithmetic
// of the coefficients (float in mixed mode, as in the forward); r is formed
// in float64 and every sum is kept in float64.
template <bool STD, class S>
__global__ void k_vjp_m2l(VjpArgs V) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= V.nleaves) return;
  const int a = V.leaf_cells[k];
  double cb[20];
  for (int j = 0; j < 20; ++j) cb[j] = V.cbar[20 * (int64_t)k + j];
  const double ax = V.c.cx[a], ay = V.c.cy[a], az = V.c.cz[a];
  double rx = 0.0, ry = 0.0, rz = 0.0;
  const int64_t off = V.far_off[k];
  const int nf = (int)min((int64_t)V.far_cnt[k], V.cap_far);
  const double zq[6] = {0, 0, 0, 0, 0, 0};
  for (int e = lane; e < nf; e += 32) {
    const int b = V.far_idx[off + e];
    const S r[3] = {(S)(ax - V.c.cx[b]), (S)(ay - V.c.cy[b]), (S)(az - V.c.cz[b])};
    const double* Qb = V.c.Q + 6 * (int64_t)b;
    // r-derivatives of sum_j cb_j C_j by dual numbers; M and Q enter linearly
    const DualT<S> R[3] = {DualT<S>{r[0], {S(1), S(0), S(0)}}, DualT<S>{r[1], {S(0), S(1), S(0)}},
                           DualT<S>{r[2], {S(0), S(0), S(1)}}};
    const DualT<S> cr = m2l_contract<DualT<S>, STD>(R, V.c.M[b], Qb, cb);
    const double gr[3] = {(double)cr.d[0], (double)cr.d[1], (double)cr.d[2]};
    const double mbar = (double)m2l_contract<S, STD>(r, 1.0, zq, cb);
    double qbar[6];
    for (int qq = 0; qq < 6; ++qq) {
      double eq[6] = {0, 0, 0, 0, 0, 0};
      eq[qq] = 1.0;
      qbar[qq] = (double)m2l_contract<S, STD>(r, 0.0, eq, cb);
    }
    rx += gr[0]; ry += gr[1]; rz += gr[2];
    double* cbb = V.cell_bar + 10 * (int64_t)b;
    atomicAdd(&cbb[0], mbar);
    atomicAdd(&cbb[1], -gr[0]);
    atomicAdd(&cbb[2], -gr[1]);
    atomicAdd(&cbb[3], -gr[2]);
    for (int q = 0; q < 6; ++q) atomicAdd(&cbb[4 + q], qbar[q]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    rx += __shfl_xor_sync(0xffffffffu, rx, o);
    ry += __shfl_xor_sync(0xffffffffu, ry, o);
    rz += __shfl_xor_sync(0xffffffffu, rz, o);
  }
  if (lane == 0) {
    double* cba = V.cell_bar + 10 * (int64_t)a;
    atomicAdd(&cba[1], rx);
    atomicAdd(&cba[2], ry);
    atomicAdd(&cba[3], rz);
  }
}

// Pair kernel K (a_i += m_j K(d), d = x_i - x_j) and (J b) for J = dK/dd.
// M4 mass fraction F(q) for 1 <= q < 2, and 4 pi w(q) (the M4 kernel times 4 pi).
template <class S>
__device__ __forceinline__ S m4_F_outer(S q) {
  const S t = S(2) - q;
  return S(1) - t * t * t * t * (S(1) - S(0.8) * t + t * t / S(6));
}
template <class S>
__device__ __forceinline__ S m4_w4pi(S q) {
  if (q < S(1)) return S(4) * (S(1) - S(1.5) * q * q + S(0.75) * q * q * q);
  if (q < S(2)) { const S t = S(2) - q; return t * t * t; }
  return S(0);
}
// K(d) = -f(r) d with J = dK/dd = -f I - g d d^T, g = f'(r) / r.  Plummer:
// f = (r^2 + eps^2)^(-3/2), g = -3 (r^2 + eps^2)^(-5/2).  M4 (Eq. 13,
// symmetrised): the mean of the two sides' terms; one side, q = r/h:
//   q < 1:       f = (4/3 - 6/5 q^2 + q^3/2) / h^3,   g = (-12/5 + 3/2 q) / h^5
//   1 <= q < 2:  f = F(q) / (q^3 h^3),  g = (F'(q) q - 3 F(q)) / (q^5 h^5), F' = 4 pi w q^2
//   q >= 2:      f = 1 / r^3,           g = -3 / r^5
// (the q < 1 forms are the polynomials themselves, finite at r = 0, where g
// multiplies d = 0).
template <class S>
__device__ __forceinline__ void pair_fg(int kind, S r2, S eps2, S hi, S hj, S& f, S& g) {
  if (kind == KDFMM_SOFT_PLUMMER) {
    const S inv = rsq(r2 + eps2);
    const S inv3 = inv * inv * inv;
    f = inv3;
    g = S(-3) * inv3 * inv * inv;
    return;
  }
  const S r = sqrt(r2);
  S fs = S(0), gs = S(0);
  const S hs[2] = {hi, hj};
  for (int side = 0; side < 2; ++side) {
    const S h = hs[side];
    const S hinv = S(1) / h;
    const S q = r * hinv;
    const S h3inv = hinv * hinv * hinv;
    if (q >= S(2)) {
      const S rinv = S(1) / r;
      const S r3inv = rinv * rinv * rinv;
      fs += r3inv;
      gs += S(-3) * r3inv * rinv * rinv;
    } else if (q < S(1)) {
      fs += (S(4) / S(3) + q * q * (S(-1.2) + S(0.5) * q)) * h3inv;
      gs += (S(-2.4) + S(1.5) * q) * h3inv * hinv * hinv;
    } else {
      const S q2 = q * q, F = m4_F_outer(q);
      fs += F / (q2 * q) * h3inv;
      gs += (m4_w4pi(q) * q2 * q - S(3) * F) / (q2 * q2 * q) * h3inv * hinv * hinv;
    }
  }
  f = S(0.5) * fs;
  g = S(0.5) * gs;
}

// P2P reverse, warp per target leaf, lanes = (target, slice) as in the
// forward: the target side x_bar_i += sum_j m_j J(d) a_bar_i stays in the
// lane; the source side (x_bar_j -= m_j J(d) a_bar_i, m_bar_j += K(d).a_bar_i)
// is summed over the leaf's targets by shuffles and added with one float64
// atomic per source into separate arrays.
// S: arithmetic of the pair terms (float in mixed mode); differences of
// positions are formed in float64 first and every sum is kept in float64.
template <class S>
__global__ void k_vjp_p2p(VjpArgs V) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  const int nitems = V.nleaves + (int)min((int64_t)V.counters[C_SEGS], V.seg_cap);
  for (int item = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); item < nitems;
       item += (int)((gridDim.x * blockDim.x) >> 5)) {
  const bool seg = item >= V.nleaves;
  const int g = item - V.nleaves;
  const int k = seg ? V.seg_leaf[g] : item;
  if (k < 0) continue;
  const int a = V.leaf_cells[k];
  const int fa = V.c.first[a], nt = V.c.count[a];
  const int K = 32 / nt, t = lane % nt, sl = lane / nt;
  const bool act = sl < K;
  const int64_t pi = (int64_t)fa + t;
  const double xi = V.tp.x[pi], yi = V.tp.y[pi], zi = V.tp.z[pi], hi = V.tp.h[pi];
  const S bS[3] = {(S)V.ab[3 * pi], (S)V.ab[3 * pi + 1], (S)V.ab[3 * pi + 2]};
  const double eps = V.sys_eps[V.leaf_sys[k]], eps2 = eps * eps;
  double gx = 0.0, gy = 0.0, gz = 0.0;
  const int64_t nall = min((int64_t)V.near_cnt[k], V.cap_near);
  const int64_t sidx = seg ? (int64_t)(g - V.seg_first[k] + 1) : 0;
  const int64_t e0 = V.near_off[k] + sidx * kSegEntries;
  const int nn = (int)(min(nall, (sidx + 1) * kSegEntries) - sidx * kSegEntries);
  for (int e = 0; e < nn; ++e) {
    const int bc = V.near_idx[e0 + e];
    const int fb = V.c.first[bc], nb = V.c.count[bc];
    const int iters = (nb + K - 1) / K;
    for (int it = 0; it < iters; ++it) {
      const int j = sl + K * it;
      const int64_t pj = (int64_t)fb + j;
      S sx = S(0), sy = S(0), sz = S(0), sm = S(0);
      if (act && j < nb && pj != pi) {
        const S d[3] = {(S)(xi - V.tp.x[pj]), (S)(yi - V.tp.y[pj]), (S)(zi - V.tp.z[pj])};
        const S r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
        S f, g;
        pair_fg<S>(V.soft_kind, r2, (S)eps2, (S)hi, (S)V.tp.h[pj], f, g);
        const S db = d[0] * bS[0] + d[1] * bS[1] + d[2] * bS[2];
        const S mj = (S)V.tp.m[pj];
        // J b = -f b - (f'/r) d (d.b)
        const S jx = -f * bS[0] - g * d[0] * db;
        const S jy = -f * bS[1] - g * d[1] * db;
        const S jz = -f * bS[2] - g * d[2] * db;
        gx += (double)(mj * jx); gy += (double)(mj * jy); gz += (double)(mj * jz);
        sx = -mj * jx; sy = -mj * jy; sz = -mj * jz;
        sm = -f * db;                                          // K(d) . a_bar_i
      }
      for (int o = 1; o < nt; o <<= 1) {                       // over the slice's targets
        const S ox = __shfl_down_sync(full, sx, o), oy = __shfl_down_sync(full, sy, o);
        const S oz = __shfl_down_sync(full, sz, o), om = __shfl_down_sync(full, sm, o);
        if (t + o < nt) { sx += ox; sy += oy; sz += oz; sm += om; }
      }
      if (t == 0 && act && j < nb) {
        atomicAdd(&V.xsrc[3 * pj], (double)sx);
        atomicAdd(&V.xsrc[3 * pj + 1], (double)sy);
        atomicAdd(&V.xsrc[3 * pj + 2], (double)sz);
        atomicAdd(&V.msrc[pj], (double)sm);
      }
    }
  }
  for (int s = 1; s < K; ++s) {
    const int src = t + s * nt;
    const double ox = __shfl_sync(full, gx, src), oy = __shfl_sync(full, gy, src),
                 oz = __shfl_sync(full, gz, src);
    if (sl == 0) { gx += ox; gy += oy; gz += oz; }
  }
  if (act && sl == 0) {
    if (seg) {
      double* P = V.seg_part + (int64_t)g * 128 + 4 * t;
      P[0] = gx; P[1] = gy; P[2] = gz;
    } else {
      V.xbar[3 * pi] += gx;
      V.xbar[3 * pi + 1] += gy;
      V.xbar[3 * pi + 2] += gz;
    }
  }
  }
}

// Adds the extra segments' target-side sums to x_bar, warp per leaf (the
// warp of its first extra segment), lane per target, in segment order.
__global__ void k_vjp_seg_combine(VjpArgs V) {
  const int lane = threadIdx.x & 31;
  const int nseg = (int)min((int64_t)V.counters[C_SEGS], V.seg_cap);
  for (int g = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); g < nseg;
       g += (int)((gridDim.x * blockDim.x) >> 5)) {
    const int k = V.seg_leaf[g];
    if (k < 0) continue;
    const int f = V.seg_first[k];
    if (g != f) continue;
    const int a = V.leaf_cells[k];
    if (lane >= V.c.count[a]) continue;
    const int x = extra_segments(min((int64_t)V.near_cnt[k], V.cap_near));
    double s0 = 0.0, s1 = 0.0, s2 = 0.0;
    for (int q = 0; q < x; ++q) {
      const double* P = V.seg_part + (int64_t)(f + q) * 128 + 4 * lane;
      s0 += P[0]; s1 += P[1]; s2 += P[2];
    }
    const int64_t pi = (int64_t)V.c.first[a] + lane;
    V.xbar[3 * pi] += s0;
    V.xbar[3 * pi + 1] += s1;
    V.xbar[3 * pi + 2] += s2;
  }
}

// Moments reverse.  For a cell with cotangents (M_bar, com_bar, Q_bar):
// com = S / M gives S_bar = com_bar / M and M_bar' = M_bar - com_bar.com / M;
// Q (Eq. 7) gives, with G = [[4q0-2q3-2q5, 3q1, 3q2], [., 4q3-2q0-2q5, 3q4],
// [., ., 4q5-2q0-2q3]] and y = x - com:
//   m_bar_i += M_bar' + x.S_bar + y^T G y / 2,   x_bar_i += m_i (S_bar + G y).
// As polynomials in x: a0 + a1.x + x^T (G/2) x and m_i (a1 + G x), with
// a1 = S_bar - G com, a0 = M_bar' + com^T G com / 2; summed over ancestors.
__global__ void k_vjp_moments(VjpArgs V) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= V.nleaves) return;
  const int leaf = V.leaf_cells[k];
  double a0 = 0.0, a1[3] = {0.0, 0.0, 0.0}, G[6] = {0, 0, 0, 0, 0, 0};   // G: xx xy xz yy yz zz
  for (int c = leaf; c >= 0; c = V.c.parent[c]) {
    const double* cb = V.cell_bar + 10 * (int64_t)c;
    const double M = V.c.M[c];
    const double com[3] = {V.c.cx[c], V.c.cy[c], V.c.cz[c]};
    const double Sb[3] = {cb[1] / M, cb[2] / M, cb[3] / M};
    const double Mb = cb[0] - (cb[1] * com[0] + cb[2] * com[1] + cb[3] * com[2]) / M;
    const double q0 = cb[4], q1 = cb[5], q2 = cb[6], q3 = cb[7], q4 = cb[8], q5 = cb[9];
    const double g[6] = {4 * q0 - 2 * q3 - 2 * q5, 3 * q1, 3 * q2, 4 * q3 - 2 * q0 - 2 * q5, 3 * q4,
                         4 * q5 - 2 * q0 - 2 * q3};
    const double Gc[3] = {g[0] * com[0] + g[1] * com[1] + g[2] * com[2],
                          g[1] * com[0] + g[3] * com[1] + g[4] * com[2],
                          g[2] * com[0] + g[4] * com[1] + g[5] * com[2]};
    a0 += Mb + 0.5 * (com[0] * Gc[0] + com[1] * Gc[1] + com[2] * Gc[2]);
    for (int d = 0; d < 3; ++d) a1[d] += Sb[d] - Gc[d];
    for (int d = 0; d < 6; ++d) G[d] += g[d];
  }
  const int f = V.c.first[leaf], cnt = V.c.count[leaf];
  for (int j = 0; j < cnt; ++j) {
    const int64_t p = (int64_t)f + j;
    const double x[3] = {V.tp.x[p], V.tp.y[p], V.tp.z[p]};
    const double Gx[3] = {G[0] * x[0] + G[1] * x[1] + G[2] * x[2],
                          G[1] * x[0] + G[3] * x[1] + G[4] * x[2],
                          G[2] * x[0] + G[4] * x[1] + G[5] * x[2]};
    const double mi = V.tp.m[p];
    V.mbar[p] += a0 + a1[0] * x[0] + a1[1] * x[1] + a1[2] * x[2] +
                 0.5 * (x[0] * Gx[0] + x[1] * Gx[1] + x[2] * Gx[2]);
    V.xbar[3 * p] += mi * (a1[0] + Gx[0]);
    V.xbar[3 * p + 1] += mi * (a1[1] + Gx[1]);
    V.xbar[3 * p + 2] += mi * (a1[2] + Gx[2]);
  }
}

__global__ void k_scatter_bar(VjpArgs V, double* __restrict__ x_bar, double* __restrict__ m_bar) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= V.n) return;
  const int64_t i = V.tp.idx[p];
  x_bar[3 * i] = V.xbar[3 * p] + V.xsrc[3 * p];
  x_bar[3 * i + 1] = V.xbar[3 * p + 1] + V.xsrc[3 * p + 1];
  x_bar[3 * i + 2] = V.xbar[3 * p + 2] + V.xsrc[3 * p + 2];
  m_bar[i] = V.mbar[p] + V.msrc[p];
}

}  // namespace

int run_vjp(kdfmm_tree_s* t, const double* a_bar, double* x_bar, double* m_bar, cudaStream_t s) {
  const int64_t n = t->n;
  const int nl = t->nleaves, nc = t->ncells;
  // scratch: a_bar, x_bar (two parts), m_bar (two parts) in tree order, then
  // the leaves' expansion cotangents and the cells' moment cotangents
  const size_t bytes = (size_t)n * 11 * sizeof(double) + (size_t)nl * 20 * sizeof(double) +
                       (size_t)nc * 10 * sizeof(double);
  char* buf = nullptr;
  int rc = check_cuda(cudaMallocAsync((void**)&buf, bytes, s), "adjoint scratch");
  if (rc) return rc;
  VjpArgs V{};
  V.n = n;
  V.nleaves = nl;
  V.ncells = nc;
  V.soft_kind = t->p.soft_kind;
  V.leaf_sys = t->leaf_sys;
  V.sys_eps = t->sys_eps;
  V.mixed = t->p.precision == KDFMM_MIXED;
  V.leaf_cells = t->leaf_cells;
  V.leaf_rank = t->leaf_rank;
  V.c = t->c;
  V.tp = t->tp;
  V.lexp32 = t->lexp32;
  V.lexp64 = t->lexp64;
  V.far_cnt = t->L.far_cnt; V.far_idx = t->L.far_idx;
  V.near_cnt = t->L.near_cnt; V.near_idx = t->L.near_idx;
  V.far_off = t->L.far_off; V.near_off = t->L.near_off;
  V.cap_far = t->L.exact ? INT64_MAX : t->L.cap_far;
  V.cap_near = t->L.exact ? INT64_MAX : t->L.cap_near;
  V.counters = t->counters;
  V.seg_first = t->L.seg_first;
  V.seg_leaf = t->L.seg_leaf;
  V.seg_part = t->L.seg_part;
  V.seg_cap = t->L.seg_cap;
  double* dp = reinterpret_cast<double*>(buf);
  V.ab = dp; dp += 3 * n;
  V.xbar = dp; dp += 3 * n;
  V.xsrc = dp; dp += 3 * n;
  V.mbar = dp; dp += n;
  V.msrc = dp; dp += n;
  V.cbar = dp; dp += 20 * (int64_t)nl;
  V.cell_bar = dp;
  cudaMemsetAsync(V.cell_bar, 0, (size_t)nc * 10 * sizeof(double), s);
  k_gather_abar<<<blocks_for(n, 256), 256, 0, s>>>(a_bar, V);
  k_vjp_l2p<<<blocks_for((int64_t)nl * 32, 128), 128, 0, s>>>(V);
  const unsigned gw = blocks_for((int64_t)nl * 32, 128);
  const bool std_exp = t->p.expansion == KDFMM_EXPANSION_STANDARD;
  if (V.mixed) {
    if (std_exp) k_vjp_m2l<true, float><<<gw, 128, 0, s>>>(V);
    else k_vjp_m2l<false, float><<<gw, 128, 0, s>>>(V);
    k_vjp_p2p<float><<<gw, 128, 0, s>>>(V);
  } else {
    if (std_exp) k_vjp_m2l<true, double><<<gw, 128, 0, s>>>(V);
    else k_vjp_m2l<false, double><<<gw, 128, 0, s>>>(V);
    k_vjp_p2p<double><<<gw, 128, 0, s>>>(V);
  }
  k_vjp_seg_combine<<<grid_blocks(2), 256, 0, s>>>(V);
  k_vjp_moments<<<blocks_for(nl, 128), 128, 0, s>>>(V);
  k_scatter_bar<<<blocks_for(n, 256), 256, 0, s>>>(V, x_bar, m_bar);
  t->launches += 7;
  rc = check_cuda(cudaGetLastError(), "adjoint launch");
  cudaFreeAsync(buf, s);
  return rc;
}

}  // namespace kdfmm
