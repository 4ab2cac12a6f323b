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
// meet); evaluated in float64 in the oracle's order, no contraction.
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

enum { DQ_OUT = 0, DQ_FAR = 1, DQ_NEAR = 2, DQ_OVER = 3 };

struct DualArgs {
  Cells c;
  const int64_t* sys_off;
  const double* sys_theta;
  int n_sys;
  double r_kern;
  const int2* in;
  int n_in;
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

__device__ __forceinline__ void push(int2* buf, int64_t cap, int32_t* ctr, int slot, int2 v,
                                     int32_t* over) {
  const int k = atomicAdd(&ctr[slot], 1);
  if (k < cap) buf[k] = v; else atomicOr(over, 1);
}

// One level of the pair recursion: thread per pair of the level.
__global__ void k_dual_level(DualArgs D) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= D.n_in) return;
  const int A = D.in[p].x, B = D.in[p].y;
  const Cells& c = D.c;
  int32_t* over = &D.ctr[DQ_OVER];
  const bool leafA = c.left[A] < 0, leafB = c.left[B] < 0;
  if (A == B) {
    if (leafA) {
      push(D.near, D.cap_near, D.ctr, DQ_NEAR, make_int2(A, A), over);
      const unsigned long long na = (unsigned long long)c.count[A];
      atomicAdd(D.np2p, na * na - na);
    } else {
      const int L = c.left[A], R = c.right[A];
      push(D.out, D.cap_out, D.ctr, DQ_OUT, make_int2(L, L), over);
      push(D.out, D.cap_out, D.ctr, DQ_OUT, make_int2(R, R), over);
      push(D.out, D.cap_out, D.ctr, DQ_OUT, make_int2(L, R), over);
    }
    return;
  }
  const double theta = D.sys_theta[system_of(D.sys_off, D.n_sys, c.first[A])];
  if (well_separated(c, A, B, theta, D.r_kern)) {
    push(D.far, D.cap_far, D.ctr, DQ_FAR, make_int2(A, B), over);
    return;
  }
  if (leafA && leafB) {
    push(D.near, D.cap_near, D.ctr, DQ_NEAR, make_int2(A, B), over);
    atomicAdd(D.np2p, 2ull * (unsigned long long)c.count[A] * (unsigned long long)c.count[B]);
    return;
  }
  const bool split_a = !leafA && (leafB || c.s[A] >= c.s[B]);
  if (split_a) {
    push(D.out, D.cap_out, D.ctr, DQ_OUT, make_int2(c.left[A], B), over);
    push(D.out, D.cap_out, D.ctr, DQ_OUT, make_int2(c.right[A], B), over);
  } else {
    push(D.out, D.cap_out, D.ctr, DQ_OUT, make_int2(A, c.left[B]), over);
    push(D.out, D.cap_out, D.ctr, DQ_OUT, make_int2(A, c.right[B]), over);
  }
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
// their expansions re-centred at the leaf's centre of mass.  With d the
// shift from the old centre to the new one (the polynomial in x = p - old
// written in x' = p - new = x - d):
//   C0' = C0 + C1.d + d.C2.d / 2 + C3[d,d,d] / 6
//   C1' = C1 + C2 d + C3[d,d] / 2,   C2' = C2 + C3 d,   C3' = C3.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int c2i(int a, int b) {
  if (a > b) { const int t = a; a = b; b = t; }
  return a == 0 ? 4 + b : (a == 1 ? 6 + b : 9);
}
__device__ __forceinline__ int c3i(int a, int b, int c) {
  if (a > b) { const int t = a; a = b; b = t; }
  if (b > c) { const int t = b; b = c; c = t; }
  if (a > b) { const int t = a; a = b; b = t; }
  if (a == 0) return b == 0 ? 10 + c : (b == 1 ? 12 + c : 15);
  if (a == 1) return b == 1 ? 15 + c : 18;
  return 19;
}

struct L2LArgs {
  Cells c;
  const int32_t* leaf_cells;
  int nleaves;
  bool mixed;
  const float* cell32;
  const double* cell64;
  float* leaf32;
  double* leaf64;
};

__global__ void k_l2l(L2LArgs A) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= A.nleaves) return;
  const int leaf = A.leaf_cells[k];
  const double lx = A.c.cx[leaf], ly = A.c.cy[leaf], lz = A.c.cz[leaf];
  double acc[20];
  for (int j = 0; j < 20; ++j) acc[j] = 0.0;
  for (int cell = leaf; cell >= 0; cell = A.c.parent[cell]) {
    double C[20];
    if (A.mixed) {
      const float* f = A.cell32 + 24 * (int64_t)cell;
      for (int j = 0; j < 20; ++j) C[j] = (double)f[j];
      for (int j = 0; j < 4; ++j) C[j] += (double)f[20 + j];
    } else {
      const double* d = A.cell64 + 20 * (int64_t)cell;
      for (int j = 0; j < 20; ++j) C[j] = d[j];
    }
    const double d[3] = {lx - A.c.cx[cell], ly - A.c.cy[cell], lz - A.c.cz[cell]};
    // C3 unchanged
    for (int j = 10; j < 20; ++j) acc[j] += C[j];
    // C2' = C2 + C3 d
    for (int a = 0; a < 3; ++a)
      for (int b = a; b < 3; ++b) {
        double v = C[c2i(a, b)];
        for (int e = 0; e < 3; ++e) v += C[c3i(a, b, e)] * d[e];
        acc[c2i(a, b)] += v;
      }
    // C1' = C1 + C2 d + C3[d,d] / 2
    for (int a = 0; a < 3; ++a) {
      double v = C[1 + a];
      for (int b = 0; b < 3; ++b) {
        v += C[c2i(a, b)] * d[b];
        for (int e = 0; e < 3; ++e) v += 0.5 * C[c3i(a, b, e)] * d[b] * d[e];
      }
      acc[1 + a] += v;
    }
    // C0' = C0 + C1.d + d.C2.d / 2 + C3[d,d,d] / 6
    double v = C[0];
    for (int a = 0; a < 3; ++a) {
      v += C[1 + a] * d[a];
      for (int b = 0; b < 3; ++b) {
        v += 0.5 * C[c2i(a, b)] * d[a] * d[b];
        for (int e = 0; e < 3; ++e) v += C[c3i(a, b, e)] * d[a] * d[b] * d[e] / 6.0;
      }
    }
    acc[0] += v;
  }
  if (A.mixed) {
    float* out = A.leaf32 + 24 * (int64_t)k;
    for (int j = 0; j < 20; ++j) out[j] = (float)acc[j];
    for (int j = 0; j < 4; ++j) out[20 + j] = (float)(acc[j] - (double)out[j]);
  } else {
    double* out = A.leaf64 + 20 * (int64_t)k;
    for (int j = 0; j < 20; ++j) out[j] = acc[j];
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
  cudaFree(D.lcell32); cudaFree(D.lcell64);
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
    A.np2p = reinterpret_cast<unsigned long long*>(L.near_np);
    int n_in = t->n_sys, cur = 0;
    bool over = false;
    while (n_in > 0) {
      A.in = D.q[cur];
      A.n_in = n_in;
      A.out = D.q[cur ^ 1];
      cudaMemsetAsync(D.ctr + DQ_OUT, 0, sizeof(int32_t), s);
      k_dual_level<<<blocks_for(n_in, 256), 256, 0, s>>>(A);
      t->launches += 1;
      cudaMemcpyAsync(hc + 40, D.ctr, 4 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
      if ((rc = check_cuda(cudaStreamSynchronize(s), "dual walk level"))) return rc;
      if (hc[40 + DQ_OVER]) { over = true; break; }
      n_in = hc[40 + DQ_OUT];
      cur ^= 1;
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
  L2LArgs A{};
  A.c = t->c;
  A.leaf_cells = t->leaf_cells;
  A.nleaves = t->nleaves;
  A.mixed = mixed;
  A.cell32 = D.lcell32;
  A.cell64 = D.lcell64;
  A.leaf32 = t->lexp32;
  A.leaf64 = t->lexp64;
  k_l2l<<<blocks_for(t->nleaves, 128), 128, 0, s>>>(A);
  t->launches += 1;
  return check_cuda(cudaGetLastError(), "l2l launch");
}

}  // namespace kdfmm
