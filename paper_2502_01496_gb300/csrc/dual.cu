// Symmetric dual-tree walk (KDFMM_WALK_DUAL): the correction the paper's
// conclusions point to (mutually interacting cells, after Dehnen), as a
// separate mode next to the paper's leaf-only walk.
//
// interact(A, B), processed level by level from each system's (root, root):
//   A == B, a leaf     -> near pair (A, A)
//   A == B, super-cell -> (L, L), (R, R), (L, R)
//   well separated     -> far pair (A, B): M2L into A from B and into B from A
//   two leaves         -> near pair (A, B): P2P both ways
//   otherwise          -> split the larger cell (by s; never a leaf; ties A)
// Well separated: theta r > s_A + s_B (the symmetric form of Eq. 4) and
// r >= s_A + s_B + R_kern max(h_A, h_B) (the smoothing spheres of Eq. 5 cannot
// meet); decided in float32 with rigorous margins, and inside the margins in
// float64 in the oracle's order, no contraction.
//
// Every cell then gets a local expansion from its far list (M2L, Eq. 6 or the
// standard series), and each leaf the sum of its ancestors' expansions (and
// its own) translated exactly to its centre of mass -- the potential
// expansion is a cubic polynomial, so moving its centre changes nothing but
// rounding.  P2P runs on the leaf's near list.  Within a mutual pair the
// expansions' Newton's third law (Sec. 3) holds, so the total force vanishes
// to rounding.  Lists are filled by atomics: their entry order, and so the
// last bits of the sums, may vary run to run.
#include <algorithm>
#include <climits>

#include "kdfmm_internal.cuh"

namespace kdfmm {

namespace {

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

constexpr int kLevelsPerSync = 8;

enum { DQ_OUT = 0, DQ_FAR = 1, DQ_NEAR = 2, DQ_OVER = 3, DQ_IN = 4 };

struct DualArgs {
  Cells c;
  const int64_t* sys_off;
  const double* sys_theta;
  int n_sys;
  double r_kern;
  const float* com_bound;    // max |com component| over the cells (float32 error bounds)
  const int2* in;            // this level's pairs: ctr[DQ_IN] of them
  int2 *out, *far, *near;
  int64_t cap_out, cap_far, cap_near;
  int32_t* ctr;
  unsigned long long* np2p;
};

__device__ __forceinline__ bool well_separated(const Cells& c, int A, int B, double theta,
                                               double rk) {
  if (theta == 0.0) return false;
  const double dx = __dsub_rn(c.cx[A], c.cx[B]);
  const double dy = __dsub_rn(c.cy[A], c.cy[B]);
  const double dz = __dsub_rn(c.cz[A], c.cz[B]);
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  const double ss = __dadd_rn(c.s[A], c.s[B]);
  if (!(__dmul_rn(__dmul_rn(theta, theta), r2) > __dmul_rn(ss, ss))) return false;
  const double hm = c.hmax[A] > c.hmax[B] ? c.hmax[A] : c.hmax[B];
  const double rr = __dadd_rn(ss, __dmul_rn(rk, hm));
  return r2 >= __dmul_rn(rr, rr);
}

// The separation test first in float32 (centres of mass, sizes and h_max as
// float32, with rigorous error margins as in the leaf walk's filter): 1
// certainly separated, 0 certainly not, -1 too close to call (float64 then).
__device__ __forceinline__ int separated_filter(float4 a, float ha, float4 b, float hb, float thf,
                                                float rkf, float bound) {
  const float u = 5.9604645e-8f;   // 2^-24
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  const float r = sqrtf(dx * dx + dy * dy + dz * dz);
  const float dr = 16.0f * u * (3.5f * bound + 3.0f * r) + 1e-30f;
  const float ss = a.w + b.w;
  const float rhs = ss + rkf * fmaxf(ha, hb);
  if (thf * (r + dr) < ss * (1.0f - 16.0f * u) || r + dr < rhs * (1.0f - 32.0f * u)) return 0;
  if (thf * fmaxf(r - dr, 0.0f) > ss * (1.0f + 16.0f * u) && r - dr > rhs * (1.0f + 32.0f * u))
    return 1;
  return -1;
}

// Reserves n entries of queue `slot` for each lane (one atomic per warp);
// returns the lane's first entry, or -1 when the queue is full (flagged).
__device__ __forceinline__ int64_t warp_reserve(int32_t* ctr, int slot, int n, int64_t cap) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(full, incl, o);
    if (lane >= o) incl += v;
  }
  const int tot = __shfl_sync(full, incl, 31);
  int base = 0;
  if (lane == 0 && tot > 0) base = atomicAdd(&ctr[slot], tot);
  base = __shfl_sync(full, base, 0);
  if ((int64_t)base + tot > cap) {
    if (lane == 0) atomicOr(&ctr[DQ_OVER], 1);
    return -1;
  }
  return (int64_t)base + incl - n;
}

// One level of the pair recursion: thread per pair, warp-aggregated queue
// pushes, grid-stride over the ctr[DQ_IN] pairs of the level.
__global__ void k_dual_level(DualArgs D) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31;
  // after an overflow the level's results are discarded (the walk is redone
  // with larger queues); the count never exceeds the queue's entries
  if (D.ctr[DQ_OVER]) return;
  const int n_in = (int)min((int64_t)D.ctr[DQ_IN], D.cap_out);
  const Cells& c = D.c;
  const float bound = *D.com_bound;
  const int stride = gridDim.x * blockDim.x;
  for (int base = blockIdx.x * blockDim.x + (threadIdx.x & ~31); base < n_in; base += stride) {
    const int p = base + lane;
    int n_out = 0, n_far = 0, n_near = 0;
    int2 o0 = make_int2(0, 0), o1 = o0, o2 = o0, fp = o0, np = o0;
    unsigned long long pairs = 0;
    if (p < n_in) {
      const int A = D.in[p].x, B = D.in[p].y;
      const bool leafA = c.left[A] < 0, leafB = c.left[B] < 0;
      if (A == B) {
        if (leafA) {
          n_near = 1;
          np = make_int2(A, A);
          const unsigned long long na = (unsigned long long)c.count[A];
          pairs = na * na - na;
        } else {
          const int L = c.left[A], R = c.right[A];
          n_out = 3;
          o0 = make_int2(L, L);
          o1 = make_int2(R, R);
          o2 = make_int2(L, R);
        }
      } else {
        const double theta = D.sys_theta[system_of(D.sys_off, D.n_sys, c.first[A])];
        int sep = 0;
        if (theta != 0.0) {
          sep = separated_filter(c.walk[A], c.walk2[A].x, c.walk[B], c.walk2[B].x, (float)theta,
                                 (float)D.r_kern, bound);
          if (sep < 0) sep = well_separated(c, A, B, theta, D.r_kern);
        }
        if (sep) {
          n_far = 1;
          fp = make_int2(A, B);
        } else if (leafA && leafB) {
          n_near = 1;
          np = make_int2(A, B);
          pairs = 2ull * (unsigned long long)c.count[A] * (unsigned long long)c.count[B];
        } else {
          n_out = 2;
          const bool split_a = !leafA && (leafB || c.s[A] >= c.s[B]);
          o0 = split_a ? make_int2(c.left[A], B) : make_int2(A, c.left[B]);
          o1 = split_a ? make_int2(c.right[A], B) : make_int2(A, c.right[B]);
        }
      }
    }
    const int64_t po = warp_reserve(D.ctr, DQ_OUT, n_out, D.cap_out);
    const int64_t pf = warp_reserve(D.ctr, DQ_FAR, n_far, D.cap_far);
    const int64_t pn = warp_reserve(D.ctr, DQ_NEAR, n_near, D.cap_near);
    if (po >= 0 && n_out > 0) {
      D.out[po] = o0;
      D.out[po + 1] = o1;
      if (n_out == 3) D.out[po + 2] = o2;
    }
    if (pf >= 0 && n_far) D.far[pf] = fp;
    if (pn >= 0 && n_near) D.near[pn] = np;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) pairs += __shfl_xor_sync(full, pairs, o);
    if (lane == 0 && pairs) atomicAdd(D.np2p, pairs);
  }
}

// Makes the last level's output the next level's input.
__global__ void k_dual_advance(int32_t* ctr) {
  ctr[DQ_IN] = ctr[DQ_OUT];
  ctr[DQ_OUT] = 0;
}

__global__ void k_dual_roots(const int32_t* __restrict__ sys_root, int n_sys, int2* q) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < n_sys) q[k] = make_int2(sys_root[k], sys_root[k]);
}

// Far pairs act both ways: counts per cell, then fill (after a scan).
__global__ void k_far_count(const int2* __restrict__ far, int nfar, int32_t* cnt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nfar) return;
  atomicAdd(&cnt[far[e].x], 1);
  atomicAdd(&cnt[far[e].y], 1);
}
__global__ void k_far_fill(const int2* __restrict__ far, int nfar, const int64_t* __restrict__ off,
                           int32_t* cursor, int32_t* idx) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nfar) return;
  const int A = far[e].x, B = far[e].y;
  idx[off[A] + atomicAdd(&cursor[A], 1)] = B;
  idx[off[B] + atomicAdd(&cursor[B], 1)] = A;
}

// Near pairs act both ways (a leaf with itself once), per leaf ordinal.
__global__ void k_near_count(const int2* __restrict__ near, int nnear,
                             const int32_t* __restrict__ leaf_rank, int32_t* cnt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnear) return;
  const int A = near[e].x, B = near[e].y;
  atomicAdd(&cnt[leaf_rank[A]], 1);
  if (A != B) atomicAdd(&cnt[leaf_rank[B]], 1);
}
__global__ void k_near_fill(const int2* __restrict__ near, int nnear,
                            const int32_t* __restrict__ leaf_rank, const int64_t* __restrict__ off,
                            int32_t* cursor, int32_t* idx) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= nnear) return;
  const int A = near[e].x, B = near[e].y;
  const int ra = leaf_rank[A];
  idx[off[ra] + atomicAdd(&cursor[ra], 1)] = B;
  if (A != B) {
    const int rb = leaf_rank[B];
    idx[off[rb] + atomicAdd(&cursor[rb], 1)] = A;
  }
}

// ---------------------------------------------------------------------------
// L2L: each leaf's expansion is the sum over the leaf and its ancestors of
// their expansions re-centred at the leaf's centre of mass.  Re-centring a
// cubic polynomial is exact up to rounding and re-centrings compose, so the
// sum is formed top-down, one tree level per launch: a cell's total is its
// own expansion plus its parent's total re-centred at the cell's centre of
// mass.  With d the shift from the old centre to the new one (the polynomial
// in x = p - old written in x' = p - new = x - d):
//   C0' = C0 + C1.d + d.C2.d / 2 + C3[d,d,d] / 6
//   C1' = C1 + C2 d + C3[d,d] / 2,   C2' = C2 + C3 d,   C3' = C3.
// Compact indices: C1 (1..3), C2 xx xy xz yy yz zz (4..9), C3 xxx xxy xxz xyy
// xyz xzz yyy yyz yzz zzz (10..19).
// ---------------------------------------------------------------------------
// Written out term by term (indices as above).
__device__ __forceinline__ void recentre_add(const double C[20], const double d[3], double acc[20]) {
  const double dx = d[0], dy = d[1], dz = d[2];
  // C3 unchanged
  acc[10] += C[10];
  acc[11] += C[11];
  acc[12] += C[12];
  acc[13] += C[13];
  acc[14] += C[14];
  acc[15] += C[15];
  acc[16] += C[16];
  acc[17] += C[17];
  acc[18] += C[18];
  acc[19] += C[19];
  // C2' = C2 + C3 d
  acc[4] += C[4] + C[10] * dx + C[11] * dy + C[12] * dz;
  acc[5] += C[5] + C[11] * dx + C[13] * dy + C[14] * dz;
  acc[6] += C[6] + C[12] * dx + C[14] * dy + C[15] * dz;
  acc[7] += C[7] + C[13] * dx + C[16] * dy + C[17] * dz;
  acc[8] += C[8] + C[14] * dx + C[17] * dy + C[18] * dz;
  acc[9] += C[9] + C[15] * dx + C[18] * dy + C[19] * dz;
  // C1' = C1 + C2 d + C3[d,d] / 2
  acc[1] += C[1] + (C[4] * dx + C[5] * dy + C[6] * dz) + 0.5 * (C[10] * dx * dx + C[11] * dx * dy
      + C[12] * dx * dz + C[11] * dy * dx + C[13] * dy * dy + C[14] * dy * dz + C[12] * dz * dx
      + C[14] * dz * dy + C[15] * dz * dz);
  acc[2] += C[2] + (C[5] * dx + C[7] * dy + C[8] * dz) + 0.5 * (C[11] * dx * dx + C[13] * dx * dy
      + C[14] * dx * dz + C[13] * dy * dx + C[16] * dy * dy + C[17] * dy * dz + C[14] * dz * dx
      + C[17] * dz * dy + C[18] * dz * dz);
  acc[3] += C[3] + (C[6] * dx + C[8] * dy + C[9] * dz) + 0.5 * (C[12] * dx * dx + C[14] * dx * dy
      + C[15] * dx * dz + C[14] * dy * dx + C[17] * dy * dy + C[18] * dy * dz + C[15] * dz * dx
      + C[18] * dz * dy + C[19] * dz * dz);
  // C0' = C0 + C1.d + d.C2.d / 2 + C3[d,d,d] / 6
  acc[0] += C[0] + (C[1] * dx + C[2] * dy + C[3] * dz) + 0.5 * (C[4] * dx * dx + C[5] * dx * dy
      + C[6] * dx * dz + C[5] * dy * dx + C[7] * dy * dy + C[8] * dy * dz + C[6] * dz * dx + C[8] * dz * dy
      + C[9] * dz * dz)
      + (1.0 / 6.0) * (C[10] * dx * dx * dx + C[11] * dx * dx * dy + C[12] * dx * dx * dz
      + C[11] * dx * dy * dx + C[13] * dx * dy * dy + C[14] * dx * dy * dz + C[12] * dx * dz * dx
      + C[14] * dx * dz * dy + C[15] * dx * dz * dz + C[11] * dy * dx * dx + C[13] * dy * dx * dy
      + C[14] * dy * dx * dz + C[13] * dy * dy * dx + C[16] * dy * dy * dy + C[17] * dy * dy * dz
      + C[14] * dy * dz * dx + C[17] * dy * dz * dy + C[18] * dy * dz * dz + C[12] * dz * dx * dx
      + C[14] * dz * dx * dy + C[15] * dz * dx * dz + C[14] * dz * dy * dx + C[17] * dz * dy * dy
      + C[18] * dz * dy * dz + C[15] * dz * dz * dx + C[18] * dz * dz * dy + C[19] * dz * dz * dz);
}

struct L2LArgs {
  Cells c;
  const int32_t* leaf_rank;
  int ncells;
  int level;
  bool mixed;
  const float* cell32;
  const double* cell64;
  double* tot;
  float* leaf32;
  double* leaf64;
};

// The cells of one tree level (all systems): total = own + parent's total
// re-centred; leaves also write their expansion in the evaluation's format.
__global__ void k_l2l_level(L2LArgs A) {
  KD_GRID_STRIDE(cell, A.ncells) {
    if (A.c.depth[cell] != A.level) continue;
    double acc[20];
    if (A.mixed) {
      const float* f = A.cell32 + 24 * (int64_t)cell;
#pragma unroll
      for (int j = 0; j < 20; ++j) acc[j] = (double)f[j];
#pragma unroll
      for (int j = 0; j < 4; ++j) acc[j] += (double)f[20 + j];
    } else {
      const double* d = A.cell64 + 20 * (int64_t)cell;
#pragma unroll
      for (int j = 0; j < 20; ++j) acc[j] = d[j];
    }
    const int p = A.c.parent[cell];
    if (p >= 0) {
      double P[20];
      const double* tp = A.tot + 20 * (int64_t)p;
#pragma unroll
      for (int j = 0; j < 20; ++j) P[j] = tp[j];
      const double d[3] = {A.c.cx[cell] - A.c.cx[p], A.c.cy[cell] - A.c.cy[p],
                           A.c.cz[cell] - A.c.cz[p]};
      recentre_add(P, d, acc);
    }
    double* to = A.tot + 20 * (int64_t)cell;
#pragma unroll
    for (int j = 0; j < 20; ++j) to[j] = acc[j];
    const int k = A.leaf_rank[cell];
    if (k < 0) continue;
    if (A.mixed) {
      float* out = A.leaf32 + 24 * (int64_t)k;
#pragma unroll
      for (int j = 0; j < 20; ++j) out[j] = (float)acc[j];
#pragma unroll
      for (int j = 0; j < 4; ++j) out[20 + j] = (float)(acc[j] - (double)out[j]);
    } else {
      double* out = A.leaf64 + 20 * (int64_t)k;
#pragma unroll
      for (int j = 0; j < 20; ++j) out[j] = acc[j];
    }
  }
}

template <class T>
int grow(T** p, int64_t* have, int64_t need, const char* what) {
  if (*have >= need) return KDFMM_OK;
  cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc(p, (size_t)std::max<int64_t>(need, 1) * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(KDFMM_ERR_OOM, "%s (%lld entries)", what, (long long)need);
  }
  *have = need;
  return KDFMM_OK;
}

}  // namespace

void free_dual(kdfmm_tree_s* t) {
  auto& D = t->dual;
  cudaFree(D.q[0]); cudaFree(D.q[1]); cudaFree(D.far); cudaFree(D.near); cudaFree(D.ctr);
  cudaFree(D.far_cnt); cudaFree(D.far_off); cudaFree(D.far_idx); cudaFree(D.cursor);
  cudaFree(D.lcell32); cudaFree(D.lcell64); cudaFree(D.ltot);
  D = kdfmm_tree_s::Dual{};
}

int run_dual_walk(kdfmm_tree_s* t, cudaStream_t s) {
  auto& D = t->dual;
  Lists& L = t->L;
  const int nc = t->ncells, nl = t->nleaves;
  int rc;
  if (!D.ctr && (rc = check_cuda(cudaMalloc(&D.ctr, 8 * sizeof(int32_t)), "dual counters")))
    return rc;
  // the three per-cell arrays always share one capacity
  int64_t cap = D.cells_cap;
  if ((rc = grow(&D.far_cnt, &cap, (int64_t)nc + 2, "dual far counts"))) return rc;
  cap = D.cells_cap;
  if ((rc = grow(&D.cursor, &cap, (int64_t)nc + 2, "dual cursors"))) return rc;
  cap = D.cells_cap;
  if ((rc = grow(&D.far_off, &cap, (int64_t)nc + 2, "dual far offsets"))) return rc;
  D.cells_cap = cap;
  int64_t qc = std::max<int64_t>(D.q_cap, 4 * (int64_t)nc + 1024);
  int64_t fc = std::max<int64_t>(D.far_cap, 8 * (int64_t)nc + 1024);
  int64_t ncap = std::max<int64_t>(D.near_cap, 8 * (int64_t)nl + 1024);
  int32_t* hc = t->host_counters;
  int64_t nfar = 0, nnear = 0;
  for (int attempt = 0;; ++attempt) {
    if (attempt > 8) return set_error(KDFMM_ERR_CAPACITY, "dual walk kept outgrowing its queues");
    int64_t h0 = D.q_cap, h1 = D.q_cap, h2 = D.far_cap, h3 = D.near_cap;
    if ((rc = grow(&D.q[0], &h0, qc, "pair queue"))) return rc;
    if ((rc = grow(&D.q[1], &h1, qc, "pair queue"))) return rc;
    if ((rc = grow(&D.far, &h2, fc, "far pairs"))) return rc;
    if ((rc = grow(&D.near, &h3, ncap, "near pairs"))) return rc;
    D.q_cap = qc; D.far_cap = fc; D.near_cap = ncap;
    cudaMemsetAsync(D.ctr, 0, 8 * sizeof(int32_t), s);
    cudaMemsetAsync(L.near_np, 0, 4 * sizeof(int64_t), s);
    cudaMemcpyAsync(D.ctr + DQ_OUT, &t->n_sys, sizeof(int32_t), cudaMemcpyHostToDevice, s);
    k_dual_roots<<<blocks_for(t->n_sys, 128), 128, 0, s>>>(t->sys_root, t->n_sys, D.q[0]);
    t->launches += 1;
    DualArgs A{};
    A.c = t->c;
    A.sys_off = t->sys_off;
    A.sys_theta = t->sys_theta;
    A.n_sys = t->n_sys;
    A.r_kern = t->p.r_kern;
    A.far = D.far;
    A.near = D.near;
    A.cap_out = qc; A.cap_far = fc; A.cap_near = ncap;
    A.ctr = D.ctr;
    A.com_bound = t->com_bound;
    A.np2p = reinterpret_cast<unsigned long long*>(L.near_np);
    // levels in batches of kLevelsPerSync: the launches read their pair
    // counts on the device, the host looks at the queue between batches
    int cur = 0;
    bool over = false;
    for (;;) {
      for (int l = 0; l < kLevelsPerSync; ++l) {
        A.in = D.q[cur];
        A.out = D.q[cur ^ 1];
        k_dual_advance<<<1, 1, 0, s>>>(D.ctr);
        k_dual_level<<<grid_blocks(), 256, 0, s>>>(A);
        t->launches += 2;
        cur ^= 1;
      }
      cudaMemcpyAsync(hc + 40, D.ctr, 5 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
      if ((rc = check_cuda(cudaStreamSynchronize(s), "dual walk levels"))) return rc;
      if (hc[40 + DQ_OVER]) { over = true; break; }
      if (hc[40 + DQ_OUT] == 0) break;
    }
    if (!over) {
      nfar = hc[40 + DQ_FAR];
      nnear = hc[40 + DQ_NEAR];
      break;
    }
    qc *= 2; fc *= 2; ncap *= 2;
  }
  // per-cell far lists (both directions)
  cudaMemsetAsync(D.far_cnt, 0, (size_t)(nc + 1) * sizeof(int32_t), s);
  cudaMemsetAsync(D.cursor, 0, (size_t)(nc + 1) * sizeof(int32_t), s);
  if (nfar > 0) k_far_count<<<blocks_for(nfar, 256), 256, 0, s>>>(D.far, (int)nfar, D.far_cnt);
  scan_i32_to_i64(D.far_cnt, D.far_off, nc, reinterpret_cast<int64_t*>(t->scan_tmp), s);
  if ((rc = grow(&D.far_idx, &D.far_idx_cap, 2 * nfar, "dual far lists"))) return rc;
  if (nfar > 0)
    k_far_fill<<<blocks_for(nfar, 256), 256, 0, s>>>(D.far, (int)nfar, D.far_off, D.cursor,
                                                      D.far_idx);
  // per-leaf near lists (both directions, a leaf with itself once)
  cudaMemsetAsync(L.near_cnt, 0, (size_t)(nl + 1) * sizeof(int32_t), s);
  cudaMemsetAsync(D.cursor, 0, (size_t)(nc + 1) * sizeof(int32_t), s);
  k_near_count<<<blocks_for(std::max<int64_t>(nnear, 1), 256), 256, 0, s>>>(D.near, (int)nnear,
                                                                            t->leaf_rank, L.near_cnt);
  scan_i32_to_i64(L.near_cnt, L.near_off, nl, reinterpret_cast<int64_t*>(t->scan_tmp), s);
  const int64_t entries = 2 * nnear - nl;      // every leaf meets itself exactly once
  if ((rc = grow(&L.near_idx, &L.near_cap, std::max<int64_t>(entries, 2 * nnear), "dual near lists")))
    return rc;
  k_near_fill<<<blocks_for(std::max<int64_t>(nnear, 1), 256), 256, 0, s>>>(
      D.near, (int)nnear, t->leaf_rank, L.near_off, D.cursor, L.near_idx);
  t->launches += 10;
  L.exact = true;
  D.nfar = 2 * nfar;
  D.nnear = entries;
  t->host_stats[KDFMM_STAT_NFAR] = D.nfar;
  t->host_stats[KDFMM_STAT_NNEAR] = D.nnear;
  return check_cuda(cudaGetLastError(), "dual walk launch");
}

int run_dual_local(kdfmm_tree_s* t, cudaStream_t s) {
  auto& D = t->dual;
  const bool mixed = t->p.precision == KDFMM_MIXED;
  int rc;
  int64_t have = 0;
  if (mixed) {
    have = D.lcell32 ? t->cap_cells * 24 : 0;
    if ((rc = grow(&D.lcell32, &have, t->cap_cells * 24, "cell expansions"))) return rc;
  } else {
    have = D.lcell64 ? t->cap_cells * 20 : 0;
    if ((rc = grow(&D.lcell64, &have, t->cap_cells * 20, "cell expansions"))) return rc;
  }
  if ((rc = run_m2l_cells(t, D.far_cnt, D.far_off, D.far_idx, D.lcell32, D.lcell64, s))) return rc;
  if ((rc = grow(&D.ltot, &D.ltot_cap, t->cap_cells * 20, "cell expansion totals"))) return rc;
  L2LArgs A{};
  A.c = t->c;
  A.leaf_rank = t->leaf_rank;
  A.ncells = t->ncells;
  A.mixed = mixed;
  A.cell32 = D.lcell32;
  A.cell64 = D.lcell64;
  A.tot = D.ltot;
  A.leaf32 = t->lexp32;
  A.leaf64 = t->lexp64;
  const unsigned grid = std::min<unsigned>(blocks_for(std::max(t->ncells, 1), 128), grid_blocks());
  for (int level = 0; level <= t->depth; ++level) {
    A.level = level;
    k_l2l_level<<<grid, 128, 0, s>>>(A);
  }
  t->launches += t->depth + 1;
  return check_cuda(cudaGetLastError(), "l2l launch");
}

}  // namespace kdfmm
