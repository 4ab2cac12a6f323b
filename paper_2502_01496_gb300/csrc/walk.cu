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
#include <algorithm>
#include <climits>
#include <cstdlib>
#include <cstring>

#include "kdfmm_internal.cuh"

namespace kdfmm {

namespace {

struct WalkArgs {
  const float4* walk;
  const float2* walk2;
  const double *cx, *cy, *cz, *s, *hmax;
  const int32_t* count;
  const int32_t* leaf_cells;
  const int32_t* counters;         // counters[C_LEAVES]: leaves to walk
  int slot_leaves;                 // slot mode: leaves the slots were allocated for
  int32_t* status;
  const float* com_bound;
  const int32_t* leaf_sys;         // system of each leaf
  const int32_t* sys_root;         // first cell of each system (+ end)
  const double* sys_theta;
  double r_kern;
  int32_t *far_cnt, *near_cnt;
  int64_t *far_off, *near_off;     // where leaf k's lists start
  int32_t *far_idx, *near_idx;
  int64_t cap_far, cap_near;       // slot mode: entries per leaf (k * cap is the start)
  bool exact;                      // exact mode: far_off / near_off are given, no limit
  int32_t* maxc;                   // [0] longest far list, [1] longest near list
  unsigned long long* stats;       // [0] P2P interactions, [1] float64 decisions, [2] far, [3] near
  int budget;                      // cells one thread visits before handing its leaf on
  int32_t* heavy;                  // queue of the leaves handed on
  int32_t* heavy_n;                // its length (counters[C_HEAVY])
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

// One thread per leaf.  Slot mode: the lists go to fixed-capacity slots of
// the leaf (entries beyond the capacity are counted, not stored; the host
// then grows the slots and walks again, or switches to exact mode).  Exact
// mode: the counts of a previous pass, scanned, give each leaf's start.
// A leaf whose walk visits more than W.budget cells (a large leaf in the
// sparse outskirts of a centrally condensed system opens most of the tree)
// is queued for k_walk_heavy, which redoes it with a whole block.
__global__ void __launch_bounds__(128, 10) k_walk(WalkArgs W) {
  // the grid covers slot_leaves leaves; more leaves than slots is flagged and
  // the evaluation is redone by the host
  const int nleaves = W.counters[C_LEAVES];
  if (!W.exact && nleaves > W.slot_leaves && blockIdx.x == 0 && threadIdx.x == 0)
    atomicOr(W.status, ST_LISTS);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nleaves || (!W.exact && k >= W.slot_leaves)) return;
  {
  const int a = W.leaf_cells[k];
  const float4 wa = W.walk[a];
  const float ha = W.walk2[a].x;
  const double ax = W.cx[a], ay = W.cy[a], az = W.cz[a], sa = W.s[a], ha64 = W.hmax[a];
  const float bound = *W.com_bound;
  const int sys = W.leaf_sys[k];
  const double theta = W.sys_theta[sys];
  const int i_end = W.sys_root[sys + 1];
  const float thf = (float)theta, rkf = (float)W.r_kern;
  const bool always = theta == 0.0;
  int64_t fo, no;
  if (W.exact) {
    fo = W.far_off[k];
    no = W.near_off[k];
  } else {
    fo = (int64_t)k * W.cap_far;
    no = (int64_t)k * W.cap_near;
    W.far_off[k] = fo;
    W.near_off[k] = no;
  }
  int32_t* far = W.far_idx + fo;
  int32_t* near = W.near_idx + no;
  const int64_t cap_far = W.exact ? INT64_MAX : W.cap_far;
  const int64_t cap_near = W.exact ? INT64_MAX : W.cap_near;
  int nf = 0, nn = 0, nex = 0;
  long long np = 0;
  int i = W.sys_root[sys];              // the walk stays inside the leaf's own tree
  int visits = 0;
  while (i < i_end) {
    if (++visits > W.budget) {
      W.heavy[atomicAdd(W.heavy_n, 1)] = k;
      return;
    }
    const float4 wb = W.walk[i];
    const float2 w2 = W.walk2[i];
    const int skip = __float_as_int(w2.y);
    int o = always ? 1 : open_filter(wa, ha, wb, w2.x, thf, rkf, bound);
    if (o < 0) {
      o = open_exact(ax, ay, az, sa, ha64, W.cx[i], W.cy[i], W.cz[i], W.s[i], W.hmax[i], theta,
                     W.r_kern);
      ++nex;
    }
    if (o) {
      if (skip == i + 1) {                    // opened leaf: short range
        if (nn < cap_near) near[nn] = i;
        np += W.count[i];
        ++nn;
      }
      i = i + 1;
    } else {                                  // closed: long range, skip its subtree
      if (nf < cap_far) far[nf] = i;
      ++nf;
      i = skip;
    }
  }
  W.far_cnt[k] = nf;
  W.near_cnt[k] = nn;
  atomicMax(&W.maxc[0], nf);
  atomicMax(&W.maxc[1], nn);
  const long long na = W.count[a];
  atomicAdd(&W.stats[0], (unsigned long long)(na * np - na));
  atomicAdd(&W.stats[2], (unsigned long long)nf);
  atomicAdd(&W.stats[3], (unsigned long long)nn);
  if (nex) atomicAdd(&W.stats[1], (unsigned long long)nex);
  }
}

// Block-wide walk of the queued leaves.  The depth-first walk visits cell i
// unless a cell p < i with i < skip(p) -- an ancestor of i in pre-order --
// was closed; so with every cell of the system decided at once, i is visited
// iff the largest skip pointer of the closed cells before i does not exceed
// i (a prefix maximum).  A visited closed cell joins the far list, a visited
// opened leaf the near list; a block scan keeps them in ascending id, as the
// thread walk emits them.  Tiles of kHeavyTile cells advance past the subtrees
// closed so far, so closed regions are not read.
constexpr int kHeavyThreads = 256;
constexpr int kHeavyPer = 4;                        // consecutive cells per thread
constexpr int kHeavyTile = kHeavyThreads * kHeavyPer;
constexpr int kHeavyWarps = kHeavyThreads / 32;
constexpr int kHeavyGrid = 152 * 2;

// Exclusive block scan (maximum) of v; *total gets the block's maximum.
__device__ __forceinline__ int block_excl_max(int v, int* total, int* sh) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int u = __shfl_up_sync(full, inc, o);
    if (lane >= o) inc = max(inc, u);
  }
  int ex = __shfl_up_sync(full, inc, 1);
  if (lane == 0) ex = 0;
  if (lane == 31) sh[w] = inc;
  __syncthreads();
  int pre = 0, tot = 0;
#pragma unroll
  for (int q = 0; q < kHeavyWarps; ++q) {
    if (q < w) pre = max(pre, sh[q]);
    tot = max(tot, sh[q]);
  }
  __syncthreads();
  *total = tot;
  return max(pre, ex);
}

// Exclusive block scan (sum) of (a, b); *ta, *tb get the block's sums.
__device__ __forceinline__ int2 block_excl_sum2(int a, int b, int* ta, int* tb, int2* sh) {
  const unsigned full = 0xffffffffu;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int ia = a, ib = b;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int ua = __shfl_up_sync(full, ia, o), ub = __shfl_up_sync(full, ib, o);
    if (lane >= o) { ia += ua; ib += ub; }
  }
  if (lane == 31) sh[w] = make_int2(ia, ib);
  __syncthreads();
  int pa = 0, pb = 0, sa = 0, sb = 0;
#pragma unroll
  for (int q = 0; q < kHeavyWarps; ++q) {
    const int2 v = sh[q];
    if (q < w) { pa += v.x; pb += v.y; }
    sa += v.x; sb += v.y;
  }
  __syncthreads();
  *ta = sa;
  *tb = sb;
  return make_int2(pa + ia - a, pb + ib - b);
}

__global__ void __launch_bounds__(kHeavyThreads) k_walk_heavy(WalkArgs W) {
  __shared__ int sh_max[kHeavyWarps];
  __shared__ int2 sh_sum[kHeavyWarps];
  __shared__ long long sh_np[kHeavyWarps];
  __shared__ int sh_nex[kHeavyWarps];
  const int nq = *W.heavy_n;
  for (int q = blockIdx.x; q < nq; q += gridDim.x) {
    const int k = W.heavy[q];
    const int a = W.leaf_cells[k];
    const float4 wa = W.walk[a];
    const float ha = W.walk2[a].x;
    const double ax = W.cx[a], ay = W.cy[a], az = W.cz[a], sa = W.s[a], ha64 = W.hmax[a];
    const float bound = *W.com_bound;
    const int sys = W.leaf_sys[k];
    const double theta = W.sys_theta[sys];
    const int i0 = W.sys_root[sys], i_end = W.sys_root[sys + 1];
    const float thf = (float)theta, rkf = (float)W.r_kern;
    const bool always = theta == 0.0;
    const int64_t fo = W.exact ? W.far_off[k] : (int64_t)k * W.cap_far;
    const int64_t no = W.exact ? W.near_off[k] : (int64_t)k * W.cap_near;
    int32_t* far = W.far_idx + fo;
    int32_t* near = W.near_idx + no;
    const int64_t cap_far = W.exact ? INT64_MAX : W.cap_far;
    const int64_t cap_near = W.exact ? INT64_MAX : W.cap_near;
    int nf = 0, nn = 0, carry = 0, nex = 0;
    long long np = 0;
    for (int t0 = i0; t0 < i_end;) {
      const int c0 = t0 + kHeavyPer * (int)threadIdx.x;
      int o[kHeavyPer], sk[kHeavyPer];
      bool ex[kHeavyPer];
      int tmax = 0;
#pragma unroll
      for (int j = 0; j < kHeavyPer; ++j) {
        const int c = c0 + j;
        o[j] = 1;
        sk[j] = 0;
        ex[j] = false;
        if (c < i_end) {
          const float4 wb = W.walk[c];
          const float2 w2 = W.walk2[c];
          sk[j] = __float_as_int(w2.y);
          o[j] = always ? 1 : open_filter(wa, ha, wb, w2.x, thf, rkf, bound);
          if (o[j] < 0) {
            o[j] = open_exact(ax, ay, az, sa, ha64, W.cx[c], W.cy[c], W.cz[c], W.s[c], W.hmax[c],
                              theta, W.r_kern);
            ex[j] = true;
          }
          if (!o[j]) tmax = max(tmax, sk[j]);
        }
      }
      int tile_max;
      int pre = max(carry, block_excl_max(tmax, &tile_max, sh_max));
      int mf = 0, mn = 0;
      bool ef[kHeavyPer], en[kHeavyPer];
#pragma unroll
      for (int j = 0; j < kHeavyPer; ++j) {
        const int c = c0 + j;
        const bool vis = c < i_end && pre <= c;
        ef[j] = vis && !o[j];
        en[j] = vis && o[j] && sk[j] == c + 1;
        mf += ef[j];
        mn += en[j];
        if (en[j]) np += W.count[c];
        if (vis && ex[j]) ++nex;
        if (c < i_end && !o[j]) pre = max(pre, sk[j]);
      }
      int tf, tn;
      const int2 pos = block_excl_sum2(mf, mn, &tf, &tn, sh_sum);
      int pf = nf + pos.x, pn = nn + pos.y;
#pragma unroll
      for (int j = 0; j < kHeavyPer; ++j) {
        if (ef[j]) { if (pf < cap_far) far[pf] = c0 + j; ++pf; }
        if (en[j]) { if (pn < cap_near) near[pn] = c0 + j; ++pn; }
      }
      nf += tf;
      nn += tn;
      carry = max(carry, tile_max);
      t0 = max(t0 + kHeavyTile, carry);
    }
    // block sums of the pair count and the float64 decisions
    const unsigned full = 0xffffffffu;
#pragma unroll
    for (int o2 = 16; o2 > 0; o2 >>= 1) {
      np += __shfl_xor_sync(full, np, o2);
      nex += __shfl_xor_sync(full, nex, o2);
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { sh_np[w] = np; sh_nex[w] = nex; }
    __syncthreads();
    if (threadIdx.x == 0) {
      long long npt = 0;
      int nxt = 0;
      for (int q2 = 0; q2 < kHeavyWarps; ++q2) { npt += sh_np[q2]; nxt += sh_nex[q2]; }
      if (!W.exact) {
        W.far_off[k] = fo;
        W.near_off[k] = no;
      }
      W.far_cnt[k] = nf;
      W.near_cnt[k] = nn;
      atomicMax(&W.maxc[0], nf);
      atomicMax(&W.maxc[1], nn);
      const long long na = W.count[a];
      atomicAdd(&W.stats[0], (unsigned long long)(na * npt - na));
      atomicAdd(&W.stats[2], (unsigned long long)nf);
      atomicAdd(&W.stats[3], (unsigned long long)nn);
      if (nxt) atomicAdd(&W.stats[1], (unsigned long long)nxt);
    }
    __syncthreads();
  }
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Cells one thread walks before its leaf goes to the block-wide walk
// (KDFMM_WALK_BUDGET overrides it; the lists do not depend on it).
static int walk_budget() {
  const char* v = getenv("KDFMM_WALK_BUDGET");
  if (v != nullptr) {
    const long b = strtol(v, nullptr, 10);
    if (b >= 1 && b <= INT_MAX) return (int)b;
  }
  return 4096;
}

}  // namespace

// Grows a list buffer to `need` entries; with `keep` the entries already
// there are copied over (the slot layout does not depend on the size).
static int ensure_idx(int32_t** idx, int64_t* have, int64_t need, const char* what,
                      bool keep = false) {
  if (*have >= need) return KDFMM_OK;
  int32_t* fresh = nullptr;
  if (cudaMalloc(&fresh, (size_t)std::max<int64_t>(need, 1) * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(KDFMM_ERR_OOM, "%s (%lld entries)", what, (long long)need);
  }
  if (keep && *idx != nullptr && *have > 0 &&
      cudaMemcpy(fresh, *idx, (size_t)*have * sizeof(int32_t), cudaMemcpyDeviceToDevice) !=
          cudaSuccess) {
    cudaFree(fresh);
    return check_cuda(cudaGetLastError(), "list copy");
  }
  cudaFree(*idx);
  *idx = fresh;
  *have = need;
  return KDFMM_OK;
}

// Slots waste memory when a few leaves have far longer lists than the rest
// (small theta on a centrally condensed system): when grown slots would take
// more than this many bytes and more than twice the bytes of the entries
// themselves, the lists are stored exactly instead.  The environment variable
// KDFMM_LIST_MODE=exact forces exact lists (one extra walk pass).
constexpr int64_t kSlotBudgetBytes = int64_t(1) << 30;

static bool force_exact_lists() {
  const char* v = getenv("KDFMM_LIST_MODE");
  return v != nullptr && strcmp(v, "exact") == 0;
}

static WalkArgs walk_args(kdfmm_tree_s* t) {
  Lists& L = t->L;
  WalkArgs W{};
  W.walk = t->c.walk;
  W.walk2 = t->c.walk2;
  W.cx = t->c.cx; W.cy = t->c.cy; W.cz = t->c.cz; W.s = t->c.s; W.hmax = t->c.hmax;
  W.count = t->c.count;
  W.leaf_cells = t->leaf_cells;
  W.counters = t->counters;
  W.status = t->status;
  W.com_bound = t->com_bound;
  W.leaf_sys = t->leaf_sys;
  W.sys_root = t->sys_root;
  W.sys_theta = t->sys_theta;
  W.r_kern = t->p.r_kern;
  W.far_cnt = L.far_cnt;
  W.near_cnt = L.near_cnt;
  W.far_off = L.far_off;
  W.near_off = L.near_off;
  W.maxc = t->counters + C_MAXFAR;
  W.stats = reinterpret_cast<unsigned long long*>(L.near_np);
  W.budget = walk_budget();
  W.heavy = L.heavy;
  W.heavy_n = t->counters + C_HEAVY;
  return W;
}

// One walk into the current slots (or exact lists), no synchronisation.
static void walk_launch(kdfmm_tree_s* t, WalkArgs W, bool exact, int64_t cf, int64_t cn,
                        int slot_leaves, cudaStream_t s) {
  Lists& L = t->L;
  W.exact = exact;
  W.far_idx = L.far_idx;
  W.near_idx = L.near_idx;
  W.cap_far = cf;
  W.cap_near = cn;
  W.slot_leaves = slot_leaves;
  cudaMemsetAsync(L.near_np, 0, 4 * sizeof(int64_t), s);
  cudaMemsetAsync(t->counters + C_MAXFAR, 0, 2 * sizeof(int32_t), s);
  cudaMemsetAsync(t->counters + C_HEAVY, 0, sizeof(int32_t), s);
  k_walk<<<blocks_for(std::max(slot_leaves, 1), 128), 128, 0, s>>>(W);
  k_walk_heavy<<<kHeavyGrid, kHeavyThreads, 0, s>>>(W);
  t->launches += 2;
}

int ensure_slots(kdfmm_tree_s* t, int slot_leaves) {
  Lists& L = t->L;
  int rc;
  if ((rc = ensure_idx(&L.far_idx, &L.far_cap, (int64_t)slot_leaves * L.cap_far, "far list slots",
                       true)))
    return rc;
  return ensure_idx(&L.near_idx, &L.near_cap, (int64_t)slot_leaves * L.cap_near,
                    "near list slots", true);
}

int walk_fixed(kdfmm_tree_s* t, int slot_leaves, cudaStream_t s) {
  Lists& L = t->L;
  if (L.far_cap < (int64_t)slot_leaves * L.cap_far || L.near_cap < (int64_t)slot_leaves * L.cap_near)
    return set_error(KDFMM_ERR_INTERNAL, "list slots not allocated for %d leaves", slot_leaves);
  L.exact = false;
  walk_launch(t, walk_args(t), false, L.cap_far, L.cap_near, slot_leaves, s);
  return check_cuda(cudaGetLastError(), "walk launch");
}

int run_walk(kdfmm_tree_s* t, cudaStream_t s) {
  const int nl = t->nleaves;
  Lists& L = t->L;
  int64_t cf = L.cap_far > 0 ? L.cap_far : 512, cn = L.cap_near > 0 ? L.cap_near : 128;
  WalkArgs W = walk_args(t);
  int32_t* hc = t->host_counters;
  int rc;
  auto launch = [&](bool exact) {
    walk_launch(t, W, exact, cf, cn, nl, s);
    cudaMemcpyAsync(hc + C_MAXFAR, t->counters + C_MAXFAR, 2 * sizeof(int32_t),
                    cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(t->host_stats + 16, L.near_np, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    return check_cuda(cudaStreamSynchronize(s), "walk");
  };
  const bool force_exact = force_exact_lists();
  for (int attempt = 0; attempt < 4; ++attempt) {
    if ((rc = ensure_idx(&L.far_idx, &L.far_cap, (int64_t)nl * cf, "far list slots"))) return rc;
    if ((rc = ensure_idx(&L.near_idx, &L.near_cap, (int64_t)nl * cn, "near list slots"))) return rc;
    if ((rc = launch(false))) return rc;
    const int64_t mf = hc[C_MAXFAR], mn = hc[C_MAXNEAR];
    const int64_t tot_far = t->host_stats[16 + 2], tot_near = t->host_stats[16 + 3];
    if (mf <= cf && mn <= cn && !force_exact) {
      L.cap_far = cf;
      L.cap_near = cn;
      L.exact = false;
      t->host_stats[KDFMM_STAT_NFAR] = tot_far;
      t->host_stats[KDFMM_STAT_NNEAR] = tot_near;
      return check_cuda(cudaGetLastError(), "walk launch");
    }
    const int64_t cf2 = std::max<int64_t>(cf, mf + mf / 4 + 16);
    const int64_t cn2 = std::max<int64_t>(cn, mn + mn / 4 + 16);
    const int64_t slot_bytes = (int64_t)nl * (cf2 + cn2) * 4;
    if (force_exact || (slot_bytes > kSlotBudgetBytes && slot_bytes > 8 * (tot_far + tot_near))) {
      // exact lists from this pass's counts: one more pass fills them
      scan_i32_to_i64(L.far_cnt, L.far_off, nl, reinterpret_cast<int64_t*>(t->scan_tmp), s);
      scan_i32_to_i64(L.near_cnt, L.near_off, nl, reinterpret_cast<int64_t*>(t->scan_tmp), s);
      t->launches += 6;
      if ((rc = ensure_idx(&L.far_idx, &L.far_cap, tot_far, "far lists"))) return rc;
      if ((rc = ensure_idx(&L.near_idx, &L.near_cap, tot_near, "near lists"))) return rc;
      if ((rc = launch(true))) return rc;
      if (t->host_stats[16 + 2] != tot_far || t->host_stats[16 + 3] != tot_near)
        return set_error(KDFMM_ERR_INTERNAL, "the two walk passes disagree");
      L.exact = true;
      t->host_stats[KDFMM_STAT_NFAR] = tot_far;
      t->host_stats[KDFMM_STAT_NNEAR] = tot_near;
      return check_cuda(cudaGetLastError(), "walk launch");
    }
    cf = cf2;
    cn = cn2;
  }
  return set_error(KDFMM_ERR_CAPACITY, "interaction lists kept outgrowing their slots");
}

}  // namespace kdfmm
