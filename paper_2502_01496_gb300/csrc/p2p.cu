// Short-range direct summation (P2P) over each leaf's near list, L2P (Eq. 8)
// of its local expansion, and the assembly a = a_short + a_long (Eq. 3) in
// the caller's particle order.
//
// Pair interaction on particle i from j (d = x_i - x_j, j != i):
//   Plummer:   a = -m_j d / (d^2 + eps^2)^(3/2),  phi = -m_j / sqrt(d^2 + eps^2);
//   M4 kernel: the symmetrised Green's function of Eq. 13,
//              a = -m_j [g(r,h_i) + g(r,h_j)]/2 d/r,  phi = -m_j [psi(r,h_i) + psi(r,h_j)]/2,
//              with g = F(q)/r^2 (F the mass fraction of the cubic spline inside
//              q = r/h) and psi = P(q)/h; outside q = 2 they are 1/r^2 and 1/r
//              (Eq. 15).  Written here as g/r = h^-3 F(q)/q^3.
//
// One warp per target leaf.  A leaf of n_t <= 32 targets uses K = 32 / n_t
// source slices: lane = target + n_t * slice, slice k takes sources k, k+K, ...
// of every near leaf, and the slices are combined at the end.  A near list
// longer than kSegEntries leaves (a large leaf in the sparse outskirts of a
// centrally condensed system can have most of the system in it) is split
// into segments of kSegEntries: the leaf's warp takes the first, the others
// are separate work items, and their partial sums are added afterwards in
// segment order, so the result does not depend on scheduling.
//
// Mixed mode: positions are float32 offsets from each particle's own leaf
// centre of mass; the target is shifted by the difference of the two leaf
// centres (from (high, low) float pairs), so no large coordinate enters the
// float32 arithmetic.  Each near leaf's contribution is summed in float32 and
// folded into a (high, low) accumulator with two-sum; the long-range part is
// added to the (high, low) pairs and the result converted to float64 once.
// FP64 mode uses float64 absolute positions.
#include <algorithm>
#include <climits>

#include "kdfmm_internal.cuh"

namespace kdfmm {

namespace {

struct P2PArgs {
  const int32_t* leaf_cells;
  const int32_t* counters;   // counters[C_LEAVES]: leaves
  int64_t cap_near;          // entries a list may hold (slot size, or no limit)
  int max_leaves;            // leaves the lists were made for
  const int32_t *cfirst, *ccount;
  const int32_t* near_cnt;
  const int32_t* near_idx;
  const int64_t* near_off;
  const float4* src32;       // cell (hi, M), (lo, 0), ...
  const float4* pf;          // (x - com_leaf, m)
  const float4* ph;          // (1/h, 1/h^3, h, (2h)^2)
  PCols tp;                  // float64 tree-order particles
  const double* cx;
  const double *cy, *cz;
  const float* lexp32;
  const double* lexp64;
  const float4* walk;        // cell (com, s) float32
  const float4* walk2;       // cell (h_max, skip, count, 0)
  const int32_t* leaf_sys;   // system of each leaf
  const double* sys_eps;     // Plummer softening length of each system
  double* a;
  double* phi;
  // near lists longer than kSegEntries: segment 0 is the leaf's own work
  // item, the others (counters[C_SEGS], at most seg_cap) are items after the
  // leaves, whose partial sums seg_part k_seg_combine adds in segment order
  const int32_t* seg_first;
  const int32_t* seg_leaf;
  double* seg_part;
  int64_t seg_cap;
};

// M4 cubic spline, q = r/h < 2: F(q)/q^3 and P(q) (qi = 1/q).
__device__ __forceinline__ float m4_fq3(float q, float qi) {
  if (q < 1.0f) return 1.3333333f + q * q * (-1.2f + 0.5f * q);
  return 2.6666667f + q * (-3.0f + q * (1.2f - 0.16666667f * q)) - 0.06666667f * qi * qi * qi;
}
__device__ __forceinline__ float m4_pot(float q, float qi) {
  const float q2 = q * q;
  if (q < 1.0f) return 1.4f + q2 * (-0.6666667f + q2 * (0.3f - 0.1f * q));
  return 1.6f + q2 * (-1.3333333f + q * (1.0f + q * (-0.3f + 0.033333335f * q))) - 0.06666667f * qi;
}
__device__ __forceinline__ double m4_fq3_d(double q, double qi) {
  if (q < 1.0) return 4.0 / 3.0 + q * q * (-1.2 + 0.5 * q);
  return 8.0 / 3.0 + q * (-3.0 + q * (1.2 - q * (1.0 / 6.0))) - qi * qi * qi * (1.0 / 15.0);
}
__device__ __forceinline__ double m4_pot_d(double q, double qi) {
  const double q2 = q * q;
  if (q < 1.0) return 1.4 + q2 * (-2.0 / 3.0 + q2 * (0.3 - 0.1 * q));
  return 1.6 + q2 * (-4.0 / 3.0 + q * (1.0 + q * (-0.3 + q * (1.0 / 30.0)))) - qi * (1.0 / 15.0);
}

// Reciprocal square root, flush-to-zero form of the hardware approximation
// (relative error below 2^-22).  Its arguments here are 0 (coincident
// particles, selected away) or far above the subnormal range, where the
// flush changes nothing and the subnormal fix-up of rsqrtf is dead weight.
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float y;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

// Interaction of one target with one source, float32, accumulated into f*.
template <int SOFT>
__device__ __forceinline__ void pair32(float rx, float ry, float rz, float mj, const float4& hi,
                                       const float4& hj, float eps2, float& fx, float& fy,
                                       float& fz, float& fp) {
  if (SOFT == KDFMM_SOFT_PLUMMER) {
    const float r2 = rx * rx + ry * ry + rz * rz + eps2;
    const float inv = rsqrt_ftz(r2);
    const float minv = mj * inv;
    const float f = minv * inv * inv;
    fx -= f * rx; fy -= f * ry; fz -= f * rz;
    fp -= minv;
  } else {
    const float r2 = fmaxf(rx * rx + ry * ry + rz * rz, 1e-30f);
    const float inv = rsqrt_ftz(r2);
    const float r = r2 * inv;
    const float qa = r * hi.x, qb = r * hj.x;
    float f, p;
    if (qa < 2.0f || qb < 2.0f) {
      const float inv3 = inv * inv * inv;
      const float fa = qa < 2.0f ? hi.y * m4_fq3(qa, inv * hi.z) : inv3;
      const float fb = qb < 2.0f ? hj.y * m4_fq3(qb, inv * hj.z) : inv3;
      const float pa = qa < 2.0f ? hi.x * m4_pot(qa, inv * hi.z) : inv;
      const float pb = qb < 2.0f ? hj.x * m4_pot(qb, inv * hj.z) : inv;
      f = 0.5f * (fa + fb);
      p = 0.5f * (pa + pb);
    } else {
      f = inv * inv * inv;
      p = inv;
    }
    const float mf = mj * f;
    fx -= mf * rx; fy -= mf * ry; fz -= mf * rz;
    fp -= mj * p;
  }
}

// One side of the symmetrised M4 pair, branch-free: returns g/r (force per
// unit displacement and mass) and psi for smoothing length h (hinv = 1/h,
// hinv3 = 1/h^3), at distance r (inv = 1/r, inv3 = 1/r^3).
//   q < 1     : g/r = h^-3 (4/3 - 6/5 q^2 + 1/2 q^3),
//               psi = h^-1 (7/5 - 2/3 q^2 + 3/10 q^4 - 1/10 q^5)
//   1 <= q < 2: g/r = r^-3 (1 - t^4 (1 - 4/5 t + t^2/6)),  t = 2 - q
//               psi = r^-1 (1 - t^5 (1/10 - t/30))
//   q >= 2    : g/r = r^-3, psi = 1/r  (t clamped to 0)
// The [1,2) force is the enclosed mass 1 - int_q^2 (2-u)^3 u^2 du written in
// t; the [1,2) potential is 1/r + h^-1 R(q) with R = 8/5 - 4/3 q^2 + q^3 -
// 3/10 q^4 + q^5/30 - 16/(15 q), and q R(q) = -t^5 (1/10 - t/30) exactly.
__device__ __forceinline__ void m4_side(float r, float inv, float inv3, float hinv, float hinv3,
                                        float& f, float& p) {
  const float q = r * hinv;
  const float q2 = q * q;
  const float t = fmaxf(2.0f - q, 0.0f);
  const float t2 = t * t;
  const float t4 = t2 * t2;
  const float g = 1.0f + t * (-0.8f + 0.16666667f * t);
  const float f_out = inv3 * fmaf(-t4, g, 1.0f);
  const float f_in = hinv3 * (1.3333334f + q2 * (-1.2f + 0.5f * q));
  f = q < 1.0f ? f_in : f_out;
  const float p_in = hinv * (1.4f + q2 * (-0.6666667f + q2 * (0.3f - 0.1f * q)));
  const float p_out = inv * fmaf(-t4 * t, fmaf(-0.033333335f, t, 0.1f), 1.0f);
  p = q < 1.0f ? p_in : p_out;
}

// Symmetrised M4 pair (Eq. 13), branch-free; hi / hj = (1/h, 1/h^3, h, -).
__device__ __forceinline__ void m4pair32(float rx, float ry, float rz, float mj, const float4& hi,
                                         const float4& hj, float& fx, float& fy, float& fz,
                                         float& fp) {
  const float r2 = fmaxf(rx * rx + ry * ry + rz * rz, 1e-30f);
  const float inv = rsqrt_ftz(r2);
  const float r = r2 * inv;
  const float inv3 = inv * inv * inv;
  float fa, pa, fb, pb;
  m4_side(r, inv, inv3, hi.x, hi.y, fa, pa);
  m4_side(r, inv, inv3, hj.x, hj.y, fb, pb);
  const float mf = 0.5f * mj * (fa + fb);
  fx -= mf * rx; fy -= mf * ry; fz -= mf * rz;
  fp -= 0.5f * mj * (pa + pb);
}

// L2P of the 20 coefficients at x: a = -(C1 + C2 x + C3 x x / 2),
// phi = C0 + C1.x + x.C2.x/2 + C3 x x x / 6.  Returns the parts beyond the
// leading C0 / C1 terms (which the caller adds in higher precision).
template <class T>
__device__ __forceinline__ void l2p_tail(const T* C, T x, T y, T z, T& ax, T& ay, T& az, T& p) {
  const T v0 = C[4] * x + C[5] * y + C[6] * z;
  const T v1 = C[5] * x + C[7] * y + C[8] * z;
  const T v2 = C[6] * x + C[8] * y + C[9] * z;
  const T xx = x * x, yy = y * y, zz = z * z, xy = x * y, xz = x * z, yz = y * z;
  const T w0 = C[10] * xx + C[13] * yy + C[15] * zz + T(2) * (C[11] * xy + C[12] * xz + C[14] * yz);
  const T w1 = C[11] * xx + C[16] * yy + C[18] * zz + T(2) * (C[13] * xy + C[14] * xz + C[17] * yz);
  const T w2 = C[12] * xx + C[17] * yy + C[19] * zz + T(2) * (C[14] * xy + C[15] * xz + C[18] * yz);
  ax = -(v0 + T(0.5) * w0);
  ay = -(v1 + T(0.5) * w1);
  az = -(v2 + T(0.5) * w2);
  p = (C[1] * x + C[2] * y + C[3] * z) + T(0.5) * (x * v0 + y * v1 + z * v2) +
      (x * w0 + y * w1 + z * w2) / T(6);
}

template <int SOFT, bool SELF>
__device__ __forceinline__ void near_leaf32(const P2PArgs& A, int fb, int nb, int sl, int K, int t,
                                            float xs, float ys, float zs, const float4& hi,
                                            float eps2f, float& fx, float& fy, float& fz,
                                            float& fp) {
  for (int j = sl; j < nb; j += K) {
    if (SELF && j == t) continue;
    const float4 s = A.pf[fb + j];
    if (SOFT == KDFMM_SOFT_M4)     // own leaf: nearly every pair is inside a support
      m4pair32(xs - s.x, ys - s.y, zs - s.z, s.w, hi, A.ph[fb + j], fx, fy, fz, fp);
    else
      pair32<SOFT>(xs - s.x, ys - s.y, zs - s.z, s.w, hi, hi, eps2f, fx, fy, fz, fp);
  }
}

// Newtonian pair (no kernel softening, optional Plummer eps^2), float32.
__device__ __forceinline__ void newton32(float rx, float ry, float rz, float mj, float eps2,
                                         float& fx, float& fy, float& fz, float& fp) {
  const float r2 = rx * rx + ry * ry + rz * rz + eps2;
  const float inv = rsqrt_ftz(r2);
  const float minv = mj * inv;
  const float f = minv * inv * inv;
  fx -= f * rx; fy -= f * ry; fz -= f * rz;
  fp -= minv;
}

// Newtonian pair for r2 > 0 outside both kernel supports; contributes
// nothing when `inside` (that pair is evaluated with the kernel instead).
__device__ __forceinline__ void newton32_outside(float rx, float ry, float rz, float r2, float mj,
                                                 bool inside, float& fx, float& fy, float& fz,
                                                 float& fp) {
  const float inv = rsqrt_ftz(r2);              // infinite for coincident pairs: selected away
  const float m1 = mj * inv;
  const float minv = inside ? 0.0f : m1;
  const float f = inside ? 0.0f : m1 * inv * inv;
  fx -= f * rx; fy -= f * ry; fz -= f * rz;
  fp -= minv;
}

constexpr int kStageCap = 256;     // staged sources per warp and chunk
constexpr int kStageRounds = 4;    // staging loads in flight per lane (half with M4 data)
constexpr int kP2PWarps = 4;

// Mixed precision.  Per chunk of near leaves the warp stages their particles
// in shared memory, shifted to the target leaf's centre of mass, and splits
// them into sources that lie outside the kernel support of every target
// (|s| - s_alpha >= 2 max(h_max,alpha, h_j): plain 1/r^2, Eq. 15) and sources
// that may not (full M4 pair).  The split only selects the instruction path:
// the M4 pair reduces to the same 1/r^2 outside the support.  The target's
// own leaf is summed separately so that j = i is skipped exactly.
template <int SOFT>
__global__ void __launch_bounds__(kP2PWarps * 32, 6) k_p2p_mixed(P2PArgs A) {
  constexpr bool M4 = SOFT == KDFMM_SOFT_M4;
  constexpr int R = M4 ? kStageRounds / 2 : kStageRounds;
  __shared__ float4 s_pos[kP2PWarps][kStageCap];
  __shared__ float4 s_ker[M4 ? kP2PWarps : 1][M4 ? kStageCap : 1];
  __shared__ int s_tbeg[kP2PWarps][32], s_tfirst[kP2PWarps][32];   // chunk's leaves: staged start, first
  __shared__ float4 s_toff[kP2PWarps][32];                          // and offset to the target com
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nleaves = min(A.counters[C_LEAVES], A.max_leaves);
  const int nitems = nleaves + (int)min((int64_t)A.counters[C_SEGS], A.seg_cap);
  for (int item = blockIdx.x * kP2PWarps + warp; item < nitems; item += gridDim.x * kP2PWarps) {
  const bool seg = item >= nleaves;
  const int g = item - nleaves;
  const int k = seg ? A.seg_leaf[g] : item;
  if (k < 0) continue;
  float4* sp = s_pos[warp];
  float4* sk = s_ker[M4 ? warp : 0];
  int* tb = s_tbeg[warp];
  int* tf = s_tfirst[warp];
  float4* toff = s_toff[warp];
  const int a = A.leaf_cells[k];
  const int fa = A.cfirst[a], nt = A.ccount[a];
  const int K = 32 / nt;
  const int t = lane % nt, sl = lane / nt;
  const bool act = sl < K;
  const float4 xa = A.pf[fa + t];
  float4 hi = make_float4(0.f, 0.f, 0.f, 0.f);
  if (M4) hi = A.ph[fa + t];
  const float4 ca = A.src32[4 * a], cal = A.src32[4 * a + 1];
  const float sa = A.walk[a].w, hmax_a = A.walk2[a].x;
  const double eps = A.sys_eps[A.leaf_sys[k]];
  float eps2f = (float)(eps * eps);
  asm("" : "+f"(eps2f));   // opaque: not recomputed in float64 at every pair
  float axh = 0.f, axl = 0.f, ayh = 0.f, ayl = 0.f, azh = 0.f, azl = 0.f, ph_ = 0.f, pl = 0.f;
  if (!seg) {
    float fx = 0.f, fy = 0.f, fz = 0.f, fp = 0.f;
    if (act)
      near_leaf32<SOFT, true>(A, fa, nt, sl, K, t, xa.x, xa.y, xa.z, hi, eps2f, fx, fy, fz, fp);
    df_add(axh, axl, fx); df_add(ayh, ayl, fy); df_add(azh, azl, fz); df_add(ph_, pl, fp);
  }
  const unsigned full = 0xffffffffu, lt = (1u << lane) - 1u;
  const int64_t nall = min((int64_t)A.near_cnt[k], A.cap_near);
  const int64_t sidx = seg ? (int64_t)(g - A.seg_first[k] + 1) : 0;
  const int64_t e1 = A.near_off[k] + min(nall, (sidx + 1) * kSegEntries);
  for (int64_t e = A.near_off[k] + sidx * kSegEntries; e < e1;) {
    // up to 32 candidate leaves, one per lane
    const int64_t my = e + lane;
    int cnt = 0, first = 0;
    float dx = 0.f, dy = 0.f, dz = 0.f;
    if (my < e1) {
      const int b = A.near_idx[my];
      if (b != a) {
        cnt = A.ccount[b];
        first = A.cfirst[b];
        const float4 cb = A.src32[4 * b], cbl = A.src32[4 * b + 1];
        dx = (cb.x - ca.x) + (cbl.x - cal.x);
        dy = (cb.y - ca.y) + (cbl.y - cal.y);
        dz = (cb.z - ca.z) + (cbl.z - cal.z);
      }
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int w = __shfl_up_sync(full, incl, o);
      if (lane >= o) incl += w;
    }
    const int L = __popc(__ballot_sync(full, my < e1 && incl <= kStageCap));
    // stage the chunk's sources with flat indexing: lane r*32 + lane of a
    // batch of R rounds takes staged index idx, finds its leaf by
    // binary search over the leaves' starts, and every load of the batch is
    // issued before any is used (the loads are L2 gathers: latency-bound)
    if (lane < L) {
      tb[lane] = incl - cnt;
      tf[lane] = first;
      toff[lane] = make_float4(dx, dy, dz, 0.0f);
    }
    __syncwarp();
    const int total = __shfl_sync(full, incl, L - 1);
    int nN = 0, nK = 0;
    for (int r0 = 0; r0 < total; r0 += 32 * R) {
      float4 pv[R], hv[R];
      int lv[R];
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int idx = r0 + 32 * r + lane;
        int l = 0;
#pragma unroll
        for (int step = 16; step > 0; step >>= 1)
          if (l + step < L && tb[l + step] <= idx) l += step;
        lv[r] = l;
        pv[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        hv[r] = make_float4(0.f, 0.f, 0.f, 0.f);
        if (idx < total) {
          const int src = tf[l] + idx - tb[l];
          pv[r] = A.pf[src];
          if (M4) hv[r] = A.ph[src];
        }
      }
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const bool v = r0 + 32 * r + lane < total;
        const float4 o = toff[lv[r]];
        float4 p = pv[r];
        p.x += o.x; p.y += o.y; p.z += o.z;
        bool need = false;
        if (M4 && v) {
          // d - s_a < X  <=>  d^2 < (s_a + X)^2 (both sides >= 0)
          const float d2 = p.x * p.x + p.y * p.y + p.z * p.z;
          const float reach = sa + 2.0f * fmaxf(hmax_a, hv[r].z) * 1.0001f + 1e-20f;
          need = d2 < reach * reach;
        }
        const unsigned vm = __ballot_sync(full, v), nm = __ballot_sync(full, v && need);
        if (v) {
          if (need) {
            const int pos = kStageCap - 1 - (nK + __popc(nm & lt));
            sp[pos] = p;
            sk[pos] = hv[r];
          } else {
            sp[nN + __popc(vm & ~nm & lt)] = p;
          }
        }
        nK += __popc(nm);
        nN += __popc(vm & ~nm);
      }
    }
    __syncwarp();
    float fx = 0.f, fy = 0.f, fz = 0.f, fp = 0.f;
    if (act) {
#pragma unroll 4
      for (int j = sl; j < nN; j += K) {
        const float4 s = sp[j];
        newton32(xa.x - s.x, xa.y - s.y, xa.z - s.z, s.w, eps2f, fx, fy, fz, fp);
      }
      if (M4) {
        // Two passes over the lane's pairs of the kernel segment, 128 at a
        // time.  Pass 1: every pair as a plain 1/r^2 pair, except those
        // inside either smoothing kernel's support (r < 2 max(h_i, h_j)),
        // which are marked in a bit mask instead; pass 2 visits only the
        // marked pairs with the full symmetrised M4 pair.  Only a sixth of the
        // segment's pairs is inside, and a lane's marked pairs are dense work.
        const float h2i = hi.w;                                   // (2 h_i)^2
        const int j0 = kStageCap - nK + sl;
        const int npair = j0 < kStageCap ? (kStageCap - j0 + K - 1) / K : 0;
        for (int i0 = 0; i0 < npair; i0 += 128) {
          const int nb = min(128, npair - i0);
          const int jb = j0 + K * i0;
          uint32_t in[4] = {0u, 0u, 0u, 0u};
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            const int nbw = min(32, nb - 32 * w);
#pragma unroll 4
            for (int b = 0; b < nbw; ++b) {
              const int j = jb + K * (32 * w + b);
              const float4 s = sp[j];
              const float rx = xa.x - s.x, ry = xa.y - s.y, rz = xa.z - s.z;
              const float r2 = rx * rx + ry * ry + rz * rz;
              const bool inside = r2 < fmaxf(h2i, sk[j].w);        // inside (2 max(h_i, h_j))
              in[w] |= (uint32_t)inside << b;
              newton32_outside(rx, ry, rz, r2, s.w, inside, fx, fy, fz, fp);
            }
          }
#pragma unroll
          for (int w = 0; w < 4; ++w) {
            uint32_t msk = in[w];
            while (msk != 0u) {
              const int b = __ffs(msk) - 1;
              msk &= msk - 1u;
              const int j = jb + K * (32 * w + b);
              const float4 s = sp[j];
              m4pair32(xa.x - s.x, xa.y - s.y, xa.z - s.z, s.w, hi, sk[j], fx, fy, fz, fp);
            }
          }
        }
      }
    }
    df_add(axh, axl, fx); df_add(ayh, ayl, fy); df_add(azh, azl, fz); df_add(ph_, pl, fp);
    __syncwarp();
    e += L;
  }
  // combine the source slices of each target
  for (int s = 1; s < K; ++s) {
    const int src = t + s * nt;
    const float bxh = __shfl_sync(full, axh, src), bxl = __shfl_sync(full, axl, src);
    const float byh = __shfl_sync(full, ayh, src), byl = __shfl_sync(full, ayl, src);
    const float bzh = __shfl_sync(full, azh, src), bzl = __shfl_sync(full, azl, src);
    const float bph = __shfl_sync(full, ph_, src), bpl = __shfl_sync(full, pl, src);
    if (sl == 0) {
      df_add2(axh, axl, bxh, bxl);
      df_add2(ayh, ayl, byh, byl);
      df_add2(azh, azl, bzh, bzl);
      df_add2(ph_, pl, bph, bpl);
    }
  }
  if (sl != 0 || !act) continue;
  if (seg) {
    double* P = A.seg_part + (int64_t)g * 128 + 4 * t;
    P[0] = (double)axh + (double)axl;
    P[1] = (double)ayh + (double)ayl;
    P[2] = (double)azh + (double)azl;
    P[3] = (double)ph_ + (double)pl;
    continue;
  }
  const float* C = A.lexp32 + 24 * (int64_t)k;
  float tx, ty, tz, tp_;
  l2p_tail<float>(C, xa.x, xa.y, xa.z, tx, ty, tz, tp_);
  // a = a_short + a_long (Eq. 3) and phi likewise, summed as (high, low)
  // float pairs and converted to float64 once (the FP64 pipe runs at 1/64 rate)
  df_add2(axh, axl, -C[1], -C[21]);
  df_add2(ayh, ayl, -C[2], -C[22]);
  df_add2(azh, azl, -C[3], -C[23]);
  df_add2(ph_, pl, C[0], C[20]);
  df_add(axh, axl, tx); df_add(ayh, ayl, ty); df_add(azh, azl, tz); df_add(ph_, pl, tp_);
  const int64_t ci = A.tp.idx[fa + t];
  A.a[3 * ci + 0] = (double)axh + (double)axl;
  A.a[3 * ci + 1] = (double)ayh + (double)ayl;
  A.a[3 * ci + 2] = (double)azh + (double)azl;
  if (A.phi) A.phi[ci] = (double)ph_ + (double)pl;
  }
}

constexpr int kStage64 = 128;      // staged sources per warp and chunk (float64 path)
constexpr int kP2P64Warps = 4;

// Float64 pair on target i from source j, d = x_i - x_j; hinv = 1/h and
// hinv3 = 1/h^3 of each side (M4 kernel), eps2 (Plummer).
template <int SOFT>
__device__ __forceinline__ void pair64(double rx, double ry, double rz, double mj, double hi,
                                       double hinv_i, double hinv3_i, double hj, double hinv_j,
                                       double hinv3_j, double eps2, double& fx, double& fy,
                                       double& fz, double& fp) {
  if (SOFT == KDFMM_SOFT_PLUMMER) {
    const double r2 = rx * rx + ry * ry + rz * rz + eps2;
    const double inv = rsqrt(r2);
    const double minv = mj * inv;
    const double f = minv * inv * inv;
    fx -= f * rx; fy -= f * ry; fz -= f * rz;
    fp -= minv;
  } else {
    const double r2 = rx * rx + ry * ry + rz * rz;
    if (r2 == 0.0) {
      fp -= mj * 0.7 * (hinv_i + hinv_j);        // P(0) = 7/5 on both sides, halved
      return;
    }
    const double inv = rsqrt(r2);
    const double r = r2 * inv;
    const double qa = r * hinv_i, qb = r * hinv_j;
    double f, p;
    if (qa < 2.0 || qb < 2.0) {
      const double inv3 = inv * inv * inv;
      const double fa = qa < 2.0 ? hinv3_i * m4_fq3_d(qa, hi * inv) : inv3;
      const double fb = qb < 2.0 ? hinv3_j * m4_fq3_d(qb, hj * inv) : inv3;
      const double pa = qa < 2.0 ? hinv_i * m4_pot_d(qa, hi * inv) : inv;
      const double pb = qb < 2.0 ? hinv_j * m4_pot_d(qb, hj * inv) : inv;
      f = 0.5 * (fa + fb);
      p = 0.5 * (pa + pb);
    } else {
      f = inv * inv * inv;
      p = inv;
    }
    const double mf = mj * f;
    fx -= mf * rx; fy -= mf * ry; fz -= mf * rz;
    fp -= mj * p;
  }
}

// Float64 mode: lanes = (target, source slice) as K = 32 / n_t slices;
// per chunk of near leaves (at most kStage64 sources) the warp stages the
// sources' float64 positions, masses and smoothing lengths (with (2h)^2) in
// shared memory, then every lane sums its slice; the target's own leaf is
// summed separately (j != i).  The slices are added in slice order.
template <int SOFT>
__global__ void __launch_bounds__(kP2P64Warps * 32) k_p2p_fp64(P2PArgs A) {
  constexpr bool M4 = SOFT == KDFMM_SOFT_M4;
  __shared__ double s_x[kP2P64Warps][kStage64], s_y[kP2P64Warps][kStage64];
  __shared__ double s_z[kP2P64Warps][kStage64], s_m[kP2P64Warps][kStage64];
  __shared__ double s_h[M4 ? kP2P64Warps : 1][M4 ? kStage64 : 1];
  __shared__ double s_h2[M4 ? kP2P64Warps : 1][M4 ? kStage64 : 1];   // (2 h)^2, rounded up
  __shared__ uint8_t s_leaf[kP2P64Warps][kStage64];
  __shared__ int s_tbeg[kP2P64Warps][32], s_tfirst[kP2P64Warps][32];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const unsigned full = 0xffffffffu;
  const int nleaves = min(A.counters[C_LEAVES], A.max_leaves);
  const int nitems = nleaves + (int)min((int64_t)A.counters[C_SEGS], A.seg_cap);
  double *sx = s_x[warp], *sy = s_y[warp], *sz = s_z[warp], *sm = s_m[warp];
  double* sh = s_h[M4 ? warp : 0];
  double* sh2 = s_h2[M4 ? warp : 0];
  uint8_t* sl_of = s_leaf[warp];
  int* tb = s_tbeg[warp];
  int* tf = s_tfirst[warp];
  for (int item = blockIdx.x * kP2P64Warps + warp; item < nitems; item += gridDim.x * kP2P64Warps) {
  const bool seg = item >= nleaves;
  const int g = item - nleaves;
  const int k = seg ? A.seg_leaf[g] : item;
  if (k < 0) continue;
  const int a = A.leaf_cells[k];
  const int fa = A.cfirst[a], nt = A.ccount[a];
  const int K = 32 / nt;
  const int t = lane % nt, sl = lane / nt;
  const bool act = sl < K;
  const int64_t it = (int64_t)fa + t;
  const double xi = A.tp.x[it], yi = A.tp.y[it], zi = A.tp.z[it];
  const double hi = M4 ? A.tp.h[it] : 0.0;
  const double hinv_i = M4 ? 1.0 / hi : 0.0;
  const double hinv3_i = hinv_i * hinv_i * hinv_i;
  const double h2i = 4.0 * hi * hi * (1.0 + 1e-12);
  const double eps = A.sys_eps[A.leaf_sys[k]];
  const double eps2 = eps * eps;
  double fx = 0.0, fy = 0.0, fz = 0.0, fp = 0.0;
  if (!seg && act) {
    for (int j = sl; j < nt; j += K) {
      if (j == t) continue;
      const int64_t js = (int64_t)fa + j;
      const double hj = M4 ? A.tp.h[js] : 0.0;
      const double hinv_j = M4 ? 1.0 / hj : 0.0;
      pair64<SOFT>(xi - A.tp.x[js], yi - A.tp.y[js], zi - A.tp.z[js], A.tp.m[js], hi, hinv_i,
                   hinv3_i, hj, hinv_j, hinv_j * hinv_j * hinv_j, eps2, fx, fy, fz, fp);
    }
  }
  const int64_t nall = min((int64_t)A.near_cnt[k], A.cap_near);
  const int64_t sidx = seg ? (int64_t)(g - A.seg_first[k] + 1) : 0;
  const int64_t e1 = A.near_off[k] + min(nall, (sidx + 1) * kSegEntries);
  for (int64_t e = A.near_off[k] + sidx * kSegEntries; e < e1;) {
    const int64_t my = e + lane;
    int cnt = 0, first = 0;
    if (my < e1) {
      const int b = A.near_idx[my];
      if (b != a) {
        cnt = A.ccount[b];
        first = A.cfirst[b];
      }
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int w = __shfl_up_sync(full, incl, o);
      if (lane >= o) incl += w;
    }
    const int L = __popc(__ballot_sync(full, my < e1 && incl <= kStage64));
    if (lane < L) {
      const int beg = incl - cnt;
      tb[lane] = beg;
      tf[lane] = first;
      for (int q = 0; q < cnt; ++q) sl_of[beg + q] = (uint8_t)lane;
    }
    __syncwarp();
    const int total = __shfl_sync(full, incl, L - 1);
    for (int idx = lane; idx < total; idx += 32) {
      const int l = sl_of[idx];
      const int64_t src = (int64_t)tf[l] + idx - tb[l];
      sx[idx] = A.tp.x[src];
      sy[idx] = A.tp.y[src];
      sz[idx] = A.tp.z[src];
      sm[idx] = A.tp.m[src];
      if (M4) {
        const double h = A.tp.h[src];
        sh[idx] = h;
        sh2[idx] = 4.0 * h * h * (1.0 + 1e-12);
      }
    }
    __syncwarp();
    if (act && !M4) {
      for (int j = sl; j < total; j += K)
        pair64<SOFT>(xi - sx[j], yi - sy[j], zi - sz[j], sm[j], 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, eps2,
                     fx, fy, fz, fp);
    } else if (act) {
      // M4 kernel, 32 sources of the lane's slice at a time.  Pass 1: every
      // pair as 1/r^2 except those that may lie inside either support
      // (r^2 < (2 max(h_i, h_j))^2, thresholds rounded up), which are marked;
      // pass 2: the marked pairs with the full symmetrised pair.  A warp
      // branching per pair instead ran the kernel path for all its lanes
      // whenever one lane needed it.
      for (int j0 = sl; j0 < total; j0 += 32 * K) {
        uint32_t in = 0u;
        for (int b = 0; b < 32; ++b) {
          const int j = j0 + b * K;
          if (j >= total) break;
          const double rx = xi - sx[j], ry = yi - sy[j], rz = zi - sz[j];
          const double r2 = rx * rx + ry * ry + rz * rz;
          const bool inside = r2 < fmax(h2i, sh2[j]);
          in |= (uint32_t)inside << b;
          const double inv = rsqrt(inside ? 1.0 : r2);
          const double minv = (inside ? 0.0 : sm[j]) * inv;
          const double f = minv * inv * inv;
          fx -= f * rx; fy -= f * ry; fz -= f * rz;
          fp -= minv;
        }
        while (in != 0u) {
          const int b = __ffs(in) - 1;
          in &= in - 1u;
          const int j = j0 + b * K;
          const double hj = sh[j], hinv_j = 1.0 / hj;
          pair64<SOFT>(xi - sx[j], yi - sy[j], zi - sz[j], sm[j], hi, hinv_i, hinv3_i, hj, hinv_j,
                       hinv_j * hinv_j * hinv_j, eps2, fx, fy, fz, fp);
        }
      }
    }
    __syncwarp();
    e += L;
  }
  for (int s = 1; s < K; ++s) {
    const int src = t + s * nt;
    const double bx = __shfl_sync(full, fx, src), by = __shfl_sync(full, fy, src);
    const double bz = __shfl_sync(full, fz, src), bp = __shfl_sync(full, fp, src);
    if (sl == 0) { fx += bx; fy += by; fz += bz; fp += bp; }
  }
  if (sl != 0 || !act) continue;
  if (seg) {
    double* P = A.seg_part + (int64_t)g * 128 + 4 * t;
    P[0] = fx; P[1] = fy; P[2] = fz; P[3] = fp;
    continue;
  }
  const double* C = A.lexp64 + 20 * (int64_t)k;
  const double x = xi - A.cx[a], y = yi - A.cy[a], z = zi - A.cz[a];
  double tx, ty, tz, tp_;
  l2p_tail<double>(C, x, y, z, tx, ty, tz, tp_);
  const int64_t ci = A.tp.idx[it];
  A.a[3 * ci + 0] = fx + (tx - C[1]);
  A.a[3 * ci + 1] = fy + (ty - C[2]);
  A.a[3 * ci + 2] = fz + (tz - C[3]);
  if (A.phi) A.phi[ci] = fp + (C[0] + tp_);
  }
}

// Reserves the extra segments of every leaf (any order: a leaf's segments
// are contiguous and combined in segment order).  More than seg_cap flags
// ST_LISTS and drops the leaf's extra segments (the evaluation is redone);
// their entries below seg_cap are marked -1, which every consumer skips.
__global__ void k_seg_plan(const int32_t* __restrict__ near_cnt, int64_t cap_near,
                           int max_leaves, int32_t* counters, int32_t* seg_first,
                           int32_t* seg_leaf, int64_t seg_cap, int32_t* status) {
  const int nleaves = min(counters[C_LEAVES], max_leaves);
  KD_GRID_STRIDE(k, nleaves) {
    const int x = extra_segments(min((int64_t)near_cnt[k], cap_near));
    int first = -1;
    if (x > 0) {
      const int base = atomicAdd(&counters[C_SEGS], x);
      if ((int64_t)base + x <= seg_cap) {
        first = base;
        for (int q = 0; q < x; ++q) seg_leaf[base + q] = k;
      } else {
        atomicOr(status, ST_LISTS);
        for (int q = 0; q < x && (int64_t)base + q < seg_cap; ++q) seg_leaf[base + q] = -1;
      }
    }
    seg_first[k] = first;
  }
}

// Adds the extra segments' partial sums to a and phi (caller order), warp
// per leaf (the warp of its first extra segment), lane per target.
__global__ void k_seg_combine(P2PArgs A) {
  const int lane = threadIdx.x & 31;
  const int nseg = (int)min((int64_t)A.counters[C_SEGS], A.seg_cap);
  for (int g = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); g < nseg;
       g += (int)((gridDim.x * blockDim.x) >> 5)) {
    const int k = A.seg_leaf[g];
    if (k < 0) continue;
    const int f = A.seg_first[k];
    if (g != f) continue;
    const int a = A.leaf_cells[k];
    if (lane >= A.ccount[a]) continue;
    const int x = extra_segments(min((int64_t)A.near_cnt[k], A.cap_near));
    double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
    for (int q = 0; q < x; ++q) {
      const double* P = A.seg_part + (int64_t)(f + q) * 128 + 4 * lane;
      s0 += P[0]; s1 += P[1]; s2 += P[2]; s3 += P[3];
    }
    const int64_t ci = A.tp.idx[A.cfirst[a] + lane];
    A.a[3 * ci + 0] += s0;
    A.a[3 * ci + 1] += s1;
    A.a[3 * ci + 2] += s2;
    if (A.phi) A.phi[ci] += s3;
  }
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

int ensure_segments(kdfmm_tree_s* t, int64_t need) {
  Lists& L = t->L;
  if (L.seg_cap >= need && L.seg_leaf != nullptr) return KDFMM_OK;
  // the plan of the last evaluation is kept (the adjoint reuses it)
  const int64_t cap = std::max<int64_t>(need, 64);
  int32_t* leaf = nullptr;
  double* part = nullptr;
  if (cudaMalloc(&leaf, (size_t)cap * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&part, (size_t)cap * 128 * sizeof(double)) != cudaSuccess) {
    cudaFree(leaf);
    cudaGetLastError();
    return set_error(KDFMM_ERR_OOM, "P2P segments (%lld)", (long long)cap);
  }
  if (L.seg_leaf != nullptr && L.seg_cap > 0 &&
      cudaMemcpy(leaf, L.seg_leaf, (size_t)L.seg_cap * sizeof(int32_t), cudaMemcpyDeviceToDevice) !=
          cudaSuccess) {
    cudaFree(leaf);
    cudaFree(part);
    return check_cuda(cudaGetLastError(), "segment copy");
  }
  cudaFree(L.seg_leaf);
  cudaFree(L.seg_part);
  L.seg_leaf = leaf;
  L.seg_part = part;
  L.seg_cap = cap;
  return KDFMM_OK;
}

int64_t segments_bound(const kdfmm_tree_s* t) {
  const Lists& L = t->L;
  const int64_t entries = L.exact ? L.near_cap : t->host_stats[KDFMM_STAT_NNEAR];
  return entries / kSegEntries + 64;
}

int plan_segments(kdfmm_tree_s* t, cudaStream_t s) {
  const int gl = std::max(t->grid_leaves, 1);
  cudaMemsetAsync(t->counters + C_SEGS, 0, sizeof(int32_t), s);
  k_seg_plan<<<std::min<unsigned>(blocks_for(gl, 256), grid_blocks()), 256, 0, s>>>(
      t->L.near_cnt, t->L.exact ? INT64_MAX : t->L.cap_near, gl, t->counters, t->L.seg_first,
      t->L.seg_leaf, t->L.seg_cap, t->status);
  t->launches += 1;
  return check_cuda(cudaGetLastError(), "segment plan");
}

int run_p2p(kdfmm_tree_s* t, double* a, double* phi, cudaStream_t s) {
  P2PArgs A{};
  A.leaf_cells = t->leaf_cells;
  A.counters = t->counters;
  A.cap_near = t->L.exact ? INT64_MAX : t->L.cap_near;
  A.max_leaves = std::max(t->grid_leaves, 1);
  A.cfirst = t->c.first;
  A.ccount = t->c.count;
  A.near_cnt = t->L.near_cnt;
  A.near_off = t->L.near_off;
  A.near_idx = t->L.near_idx;
  A.src32 = t->c.src32;
  A.pf = t->pf;
  A.ph = t->ph;
  A.tp = t->tp;
  A.cx = t->c.cx; A.cy = t->c.cy; A.cz = t->c.cz;
  A.lexp32 = t->lexp32;
  A.lexp64 = t->lexp64;
  A.walk = t->c.walk;
  A.walk2 = t->c.walk2;
  A.leaf_sys = t->leaf_sys;
  A.sys_eps = t->sys_eps;
  A.a = a;
  A.phi = phi;
  A.seg_first = t->L.seg_first;
  A.seg_leaf = t->L.seg_leaf;
  A.seg_part = t->L.seg_part;
  A.seg_cap = t->L.seg_cap;
  int rc = plan_segments(t, s);
  if (rc) return rc;
  const int gl = std::max(t->grid_leaves, 1);
  const bool m4 = t->p.soft_kind == KDFMM_SOFT_M4;
  if (t->p.precision == KDFMM_MIXED) {
    const unsigned gm = blocks_for(gl, kP2PWarps);
    if (m4) k_p2p_mixed<KDFMM_SOFT_M4><<<gm, kP2PWarps * 32, 0, s>>>(A);
    else k_p2p_mixed<KDFMM_SOFT_PLUMMER><<<gm, kP2PWarps * 32, 0, s>>>(A);
  } else {
    const unsigned g64 = blocks_for(gl, kP2P64Warps);
    if (m4) k_p2p_fp64<KDFMM_SOFT_M4><<<g64, kP2P64Warps * 32, 0, s>>>(A);
    else k_p2p_fp64<KDFMM_SOFT_PLUMMER><<<g64, kP2P64Warps * 32, 0, s>>>(A);
  }
  k_seg_combine<<<grid_blocks(2), 256, 0, s>>>(A);
  t->launches += 2;
  return check_cuda(cudaGetLastError(), "p2p launch");
}

}  // namespace kdfmm
