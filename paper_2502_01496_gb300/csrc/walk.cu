// Leaf-only tree walk (Sec. 2 and Sec. 4): for every leaf alpha, descend from
// the root; a cell beta is opened when Eq. 4 (theta^2 < (s_beta / r)^2) or
// Eq. 5 (r^2 < [s_alpha + s_beta + R_kern max(h_alpha, h_beta)]^2) holds, r
// the distance between the centres of mass.  An opened leaf joins alpha's
// near (P2P) list, an opened super-cell is descended, a cell that is not
// opened joins the far (M2L) list.  Super-cells never walk, so the pairs
// "super-cell <- leaf" are never formed: the asymmetry the paper analyses.
//
// Cells are in pre-order, so the depth-first walk needs no stack: after an
// opened cell comes id + 1, after a closed one its skip pointer.  Lists come
// out in ascending id.
//
// Decisions must match the float64 reference bit for bit.  Each is first
// tried in float32 with a rigorous error margin (rounding of the centres of
// mass, the sizes, theta and every operation); only a decision inside the
// margin (about 1e-6 relative) is re-evaluated in float64 with the reference's
// expression order and no contraction.
#include "kdfmm_internal.cuh"

namespace kdfmm {

namespace {

struct WalkArgs {
  const float4* walk;
  const float2* walk2;
  const double *cx, *cy, *cz, *s, *hmax;
  const int32_t* count;
  const int32_t* leaf_cells;
  int nleaves, ncells;
  const float* com_bound;
  double theta, r_kern;
  int32_t *far_cnt, *near_cnt;
  const int64_t *far_off, *near_off;
  int32_t *far_idx, *near_idx;
  unsigned long long* stats;   // [0] P2P interactions, [1] float64 decisions
};

__device__ __forceinline__ bool open_exact(double ax, double ay, double az, double sa, double ha,
                                           double bx, double by, double bz, double sb, double hb,
                                           double theta, double rk) {
  const double dx = __dsub_rn(ax, bx), dy = __dsub_rn(ay, by), dz = __dsub_rn(az, bz);
  const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
  if (r2 == 0.0) return true;
  if (theta == 0.0) return true;
  if (__dmul_rn(__dmul_rn(theta, theta), r2) < __dmul_rn(sb, sb)) return true;
  const double hm = ha > hb ? ha : hb;
  const double rr = __dadd_rn(__dadd_rn(sa, sb), __dmul_rn(rk, hm));
  return r2 < __dmul_rn(rr, rr);
}

// 1: certainly opened, 0: certainly not, -1: too close to call in float32.
__device__ __forceinline__ int open_filter(float4 a, float ha, float4 b, float hb, float thf,
                                           float rkf, float bound) {
  const float u = 5.9604645e-8f;   // 2^-24
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  const float r = sqrtf(dx * dx + dy * dy + dz * dz);
  const float dr = 16.0f * u * (3.5f * bound + 3.0f * r) + 1e-30f;
  const float sb = b.w;
  if (thf * (r + dr) < sb * (1.0f - 16.0f * u)) return 1;                       // Eq. 4
  const float rhs = a.w + sb + rkf * fmaxf(ha, hb);
  if (r + dr < rhs * (1.0f - 32.0f * u)) return 1;                              // Eq. 5
  if (thf * fmaxf(r - dr, 0.0f) > sb * (1.0f + 16.0f * u) && r - dr > rhs * (1.0f + 32.0f * u))
    return 0;
  return -1;
}

template <bool FILL>
__global__ void __launch_bounds__(128) k_walk(WalkArgs W) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= W.nleaves) return;
  const int a = W.leaf_cells[k];
  const float4 wa = W.walk[a];
  const float ha = W.walk2[a].x;
  const double ax = W.cx[a], ay = W.cy[a], az = W.cz[a], sa = W.s[a], ha64 = W.hmax[a];
  const float bound = *W.com_bound;
  const float thf = (float)W.theta, rkf = (float)W.r_kern;
  const bool always = W.theta == 0.0;
  int64_t fo = 0, no = 0;
  if (FILL) { fo = W.far_off[k]; no = W.near_off[k]; }
  int nf = 0, nn = 0, nex = 0;
  long long np = 0;
  int i = 0;
  while (i < W.ncells) {
    const float4 wb = W.walk[i];
    const float2 w2 = W.walk2[i];
    const int skip = __float_as_int(w2.y);
    int o = always ? 1 : open_filter(wa, ha, wb, w2.x, thf, rkf, bound);
    if (o < 0) {
      o = open_exact(ax, ay, az, sa, ha64, W.cx[i], W.cy[i], W.cz[i], W.s[i], W.hmax[i], W.theta,
                     W.r_kern);
      ++nex;
    }
    if (o) {
      if (skip == i + 1) {                    // opened leaf: short range
        if (FILL) W.near_idx[no + nn] = i;
        else np += W.count[i];
        ++nn;
      }
      i = i + 1;
    } else {                                  // closed: long range, skip its subtree
      if (FILL) W.far_idx[fo + nf] = i;
      ++nf;
      i = skip;
    }
  }
  if (!FILL) {
    W.far_cnt[k] = nf;
    W.near_cnt[k] = nn;
    const long long na = W.count[a];
    atomicAdd(&W.stats[0], (unsigned long long)(na * np - na));
    if (nex) atomicAdd(&W.stats[1], (unsigned long long)nex);
  }
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

int ensure_lists(kdfmm_tree_s* t, int64_t nfar, int64_t nnear) {
  Lists& L = t->L;
  if (L.far_cap < nfar) {
    cudaFree(L.far_idx);
    L.far_idx = nullptr;
    int64_t cap = nfar + nfar / 4 + 1024;
    if (cudaMalloc(&L.far_idx, cap * sizeof(int32_t)) != cudaSuccess)
      return set_error(KDFMM_ERR_OOM, "far list allocation (%lld entries)", (long long)cap);
    L.far_cap = cap;
  }
  if (L.near_cap < nnear) {
    cudaFree(L.near_idx);
    L.near_idx = nullptr;
    int64_t cap = nnear + nnear / 4 + 1024;
    if (cudaMalloc(&L.near_idx, cap * sizeof(int32_t)) != cudaSuccess)
      return set_error(KDFMM_ERR_OOM, "near list allocation (%lld entries)", (long long)cap);
    L.near_cap = cap;
  }
  return KDFMM_OK;
}

int run_walk(kdfmm_tree_s* t, cudaStream_t s) {
  const int nl = t->nleaves;
  WalkArgs W{};
  W.walk = t->c.walk;
  W.walk2 = t->c.walk2;
  W.cx = t->c.cx; W.cy = t->c.cy; W.cz = t->c.cz; W.s = t->c.s; W.hmax = t->c.hmax;
  W.count = t->c.count;
  W.leaf_cells = t->leaf_cells;
  W.nleaves = nl;
  W.ncells = t->ncells;
  W.com_bound = t->com_bound;
  W.theta = t->p.theta;
  W.r_kern = t->p.r_kern;
  W.far_cnt = t->L.far_cnt;
  W.near_cnt = t->L.near_cnt;
  W.far_off = t->L.far_off;
  W.near_off = t->L.near_off;
  W.stats = reinterpret_cast<unsigned long long*>(t->L.near_np);
  cudaMemsetAsync(t->L.near_np, 0, 4 * sizeof(int64_t), s);
  k_walk<false><<<blocks_for(nl, 128), 128, 0, s>>>(W);
  int64_t* tmp64 = reinterpret_cast<int64_t*>(t->scan_tmp);
  scan_i32_to_i64(t->L.far_cnt, t->L.far_off, nl, tmp64, s);
  scan_i32_to_i64(t->L.near_cnt, t->L.near_off, nl, tmp64, s);
  int64_t* hs = t->host_stats;
  cudaMemcpyAsync(hs + 16, t->L.far_off + nl, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(hs + 17, t->L.near_off + nl, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  int rc = check_cuda(cudaStreamSynchronize(s), "walk count");
  if (rc) return rc;
  const int64_t nfar = hs[16], nnear = hs[17];
  if ((rc = ensure_lists(t, nfar, nnear))) return rc;
  W.far_idx = t->L.far_idx;
  W.near_idx = t->L.near_idx;
  k_walk<true><<<blocks_for(nl, 128), 128, 0, s>>>(W);
  t->launches += 8;
  t->host_stats[KDFMM_STAT_NFAR] = nfar;
  t->host_stats[KDFMM_STAT_NNEAR] = nnear;
  return check_cuda(cudaGetLastError(), "walk launch");
}

}  // namespace kdfmm
