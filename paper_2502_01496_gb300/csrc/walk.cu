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
  const float4* walk2;            // (h_max, skip, count, 0)
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
  bool arena;                      // arena mode: each leaf's lists are placed where room is
                                   // reserved for them (far_off / near_off say where)
  int64_t far_cap, near_cap;       // arena mode: entries the list buffers hold
  int32_t* temp;                   // arena mode: budget entries per thread of the grid
  int64_t heavy_scratch;           // arena mode: entries of temp each k_walk_heavy block may use
  bool exact;                      // two-pass mode: far_off / near_off are given (the scanned
                                   // counts of a first pass), no limit
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

// The depth-first walk of leaf k (`valid` false: no leaf, the lane only
// keeps the warp company), emitting far entries with far(nf, cell) and near
// entries with near(nn, cell).  Must be called by all 32 lanes of the warp.
// Returns false for an invalid lane and for a leaf whose walk passes W.budget
// visited cells (a large leaf in the sparse outskirts of a centrally
// condensed system opens most of the tree): that leaf is queued for
// k_walk_heavy, which redoes it with a block.  Within the budget a walk emits
// at most W.budget entries.
//
// The cell's record is loaded first in a step, ahead of the budget test, so
// that its latency overlaps the test (loads behind that branch made the walk
// 8 to 13 % slower).  SYNC makes the loop warp-synchronous (a vote at its
// head), so the lanes reconverge at every step and a record load is one
// instruction for all walking lanes: 3 % faster on the slot-mode walk of a
// binary polytrope, 4 % slower on the arena walk of a Plummer sphere, whose
// lanes' walks differ more in length (the slot walk syncs, the arena walk
// runs free).
// The float32 copies of theta and R_kern and the theta = 0 flag go through
// an empty asm, which makes them opaque values: otherwise the compiler, short
// of registers, recomputes them from the float64 values at every step, and on
// this part a float64 conversion or comparison occupies the float64 pipe 64
// cycles a warp instruction (two such instructions a step kept it 43 % busy).
template <bool SYNC, class Far, class Near>
__device__ __forceinline__ bool walk_leaf(const WalkArgs& W, int k, bool valid, Far far, Near near,
                                          int& nf, int& nn, long long& np, int& nex) {
  const unsigned full = 0xffffffffu;
  float4 wa = make_float4(0.f, 0.f, 0.f, 0.f);
  float ha = 0.f;
  double ax = 0., ay = 0., az = 0., sa = 0., ha64 = 0., theta = 0.;
  int i = 0, i_end = 0;
  if (valid) {
    const int a = W.leaf_cells[k];
    wa = W.walk[a];
    ha = W.walk2[a].x;
    ax = W.cx[a]; ay = W.cy[a]; az = W.cz[a]; sa = W.s[a]; ha64 = W.hmax[a];
    const int sys = W.leaf_sys[k];
    theta = W.sys_theta[sys];
    i = W.sys_root[sys];                // the walk stays inside the leaf's own tree
    i_end = W.sys_root[sys + 1];
  }
  const float bound = *W.com_bound;
  float thf = (float)theta, rkf = (float)W.r_kern;
  int always = theta == 0.0;
  asm("" : "+f"(thf), "+f"(rkf), "+r"(always));
  bool ok = valid;
  int visits = 0;
  for (;;) {
    if (SYNC) {
      if (!__any_sync(full, i < i_end)) break;
      if (i >= i_end) continue;
    } else if (i >= i_end) {
      break;
    }
    const float4 wb = W.walk[i];
    const float4 w2 = W.walk2[i];
    if (++visits > W.budget) {
      W.heavy[atomicAdd(W.heavy_n, 1)] = k;
      ok = false;
      i_end = 0;
      continue;
    }
    const int skip = __float_as_int(w2.y);
    int o = always ? 1 : open_filter(wa, ha, wb, w2.x, thf, rkf, bound);
    if (o < 0) {
      o = open_exact(ax, ay, az, sa, ha64, W.cx[i], W.cy[i], W.cz[i], W.s[i], W.hmax[i], theta,
                     W.r_kern);
      ++nex;
    }
    if (o) {
      if (skip == i + 1) {                    // opened leaf: short range
        near(nn, i);
        np += __float_as_int(w2.z);
        ++nn;
      }
      i = i + 1;
    } else {                                  // closed: long range, skip its subtree
      far(nf, i);
      ++nf;
      i = skip;
    }
  }
  return ok;
}

__device__ __forceinline__ void walk_stats(const WalkArgs& W, int k, int nf, int nn, long long np,
                                           int nex) {
  atomicMax(&W.maxc[0], nf);
  atomicMax(&W.maxc[1], nn);
  const long long na = W.count[W.leaf_cells[k]];
  atomicAdd(&W.stats[0], (unsigned long long)(na * np - na));
  if (nex) atomicAdd(&W.stats[1], (unsigned long long)nex);
}

// One thread per leaf.  Slot mode: the lists go to fixed-capacity slots of
// the leaf (entries beyond the capacity are counted, not stored; the host
// then grows the slots and walks again, or changes mode).  Two-pass mode: the
// counts of a previous pass, scanned, give each leaf's start.  A leaf whose
// walk passes W.budget visited cells is queued for k_walk_heavy, which writes
// its lists and counts.
__global__ void __launch_bounds__(128, 10) k_walk(WalkArgs W) {
  // the grid covers slot_leaves leaves; more leaves than slots is flagged and
  // the evaluation is redone by the host
  const int nleaves = W.counters[C_LEAVES];
  if (!W.exact && nleaves > W.slot_leaves && blockIdx.x == 0 && threadIdx.x == 0)
    atomicOr(W.status, ST_LISTS);
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k - (int)(threadIdx.x & 31) >= nleaves) return;       // the whole warp is past the leaves
  const bool valid = k < nleaves && (W.exact || k < W.slot_leaves);
  int64_t fo = 0, no = 0;
  if (valid && W.exact) {
    fo = W.far_off[k];
    no = W.near_off[k];
  } else if (valid) {
    fo = (int64_t)k * W.cap_far;
    no = (int64_t)k * W.cap_near;
    W.far_off[k] = fo;
    W.near_off[k] = no;
  }
  int32_t* const far_l = W.far_idx + fo;
  int32_t* const near_l = W.near_idx + no;
  const int64_t cap_far = W.exact ? INT64_MAX : W.cap_far;
  const int64_t cap_near = W.exact ? INT64_MAX : W.cap_near;
  int nf = 0, nn = 0, nex = 0;
  long long np = 0;
  if (!walk_leaf<true>(
          W, k, valid, [&](int e, int c) { if (e < cap_far) far_l[e] = c; },
          [&](int e, int c) { if (e < cap_near) near_l[e] = c; }, nf, nn, np, nex))
    return;
  W.far_cnt[k] = nf;
  W.near_cnt[k] = nn;
  walk_stats(W, k, nf, nn, np, nex);
  atomicAdd(&W.stats[2], (unsigned long long)nf);
  atomicAdd(&W.stats[3], (unsigned long long)nn);
}

// Copies n entries of a list from a thread's scratch (DOWN: stored backwards
// from src) to dst, by the 32 lanes of a warp: coalesced, kCopyBatch loads a
// lane in flight before the stores (the copy is latency-bound otherwise).
constexpr int kCopyBatch = 8;
template <bool DOWN>
__device__ __forceinline__ void warp_copy_list(const int32_t* __restrict__ src, int n,
                                               int32_t* __restrict__ dst, int lane) {
  for (int e0 = 0; e0 < n; e0 += 32 * kCopyBatch) {
    int32_t v[kCopyBatch];
#pragma unroll
    for (int u = 0; u < kCopyBatch; ++u) {
      const int e = e0 + 32 * u + lane;
      v[u] = e < n ? src[DOWN ? -e : e] : 0;
    }
#pragma unroll
    for (int u = 0; u < kCopyBatch; ++u) {
      const int e = e0 + 32 * u + lane;
      if (e < n) dst[e] = v[u];
    }
  }
}

// Copies the warp's 32 lists (lane l's list: pre[l + 1] - pre[l] entries of
// thread tid0 + l's scratch, to dst + pre[l]) list by list.
template <bool DOWN>
__device__ __forceinline__ void warp_copy(const int32_t* __restrict__ temp, int64_t tid0, int B,
                                          const int* pre, int32_t* __restrict__ dst) {
  const int lane = threadIdx.x & 31;
  for (int l = 0; l < 32; ++l) {
    const int32_t* src = temp + (tid0 + l) * B + (DOWN ? B - 1 : 0);
    warp_copy_list<DOWN>(src, pre[l + 1] - pre[l], dst + pre[l], lane);
  }
}

// Arena mode (lists of very different lengths, where fixed slots would waste
// memory): a persistent grid, warp per 32 consecutive leaves, thread per
// leaf.  Each thread walks into its own scratch of W.budget entries (far
// from the front, near from the back: a walk within the budget emits at most
// one entry per visited cell); the warp then reserves room for its 32 leaves'
// lists with one atomic per list kind on the running totals (stats[2],
// stats[3]) and copies them there, coalesced.  Totals beyond the buffers
// flag ST_LISTS and store nothing (counts 0); the host grows and walks again.
// SYNC is walk_leaf's loop form: free-running for one round of threads,
// synchronous for several (the host picks it from its leaf count).
template <bool SYNC>
__global__ void __launch_bounds__(128, 10) k_walk_arena(WalkArgs W) {
  __shared__ int s_pre[4][2][33];         // per warp: exclusive prefixes of the far and near counts
  const unsigned full = 0xffffffffu;
  const int nleaves = W.counters[C_LEAVES];
  const int lane = threadIdx.x & 31;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tid0 = tid - lane;
  const int B = W.budget;
  int32_t* temp = W.temp + tid * B;
  // one round (every leaf has a thread): leaf k's scratch is thread k's and
  // k_arena_copy moves the lists afterwards, with all of the GPU's loads in
  // flight at once; with more rounds each warp copies before its next round
  const bool deferred = (int64_t)gridDim.x * blockDim.x >= nleaves;
  for (int64_t kb = tid0; kb < nleaves; kb += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)kb + lane;
    int nf = 0, nn = 0, nex = 0;
    long long np = 0;
    int32_t* const near_l = temp + (B - 1);
    const bool ok = walk_leaf<SYNC>(
        W, k, k < nleaves, [&](int e, int c) { temp[e] = c; }, [&](int e, int c) { near_l[-e] = c; },
        nf, nn, np, nex);
    if (!ok) nf = nn = 0;
    int fi = nf, ni = nn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int uf = __shfl_up_sync(full, fi, o), un = __shfl_up_sync(full, ni, o);
      if (lane >= o) { fi += uf; ni += un; }
    }
    const int ftot = __shfl_sync(full, fi, 31), ntot = __shfl_sync(full, ni, 31);
    unsigned long long fb = 0, nb = 0;
    if (lane == 0) {
      fb = atomicAdd(&W.stats[2], (unsigned long long)ftot);
      nb = atomicAdd(&W.stats[3], (unsigned long long)ntot);
    }
    fb = __shfl_sync(full, fb, 0);
    nb = __shfl_sync(full, nb, 0);
    const bool fits = (int64_t)(fb + ftot) <= W.far_cap && (int64_t)(nb + ntot) <= W.near_cap;
    if (!fits && lane == 0) atomicOr(W.status, ST_LISTS);
    const int64_t myf = (int64_t)fb + fi - nf, myn = (int64_t)nb + ni - nn;
    if (ok) {
      W.far_off[k] = myf;
      W.near_off[k] = myn;
      W.far_cnt[k] = fits ? nf : 0;
      W.near_cnt[k] = fits ? nn : 0;
      walk_stats(W, k, nf, nn, np, nex);
    } else if (k < nleaves) {         // queued: k_walk_heavy writes its lists and counts
      W.far_cnt[k] = 0;
      W.near_cnt[k] = 0;
    }
    int* pf = s_pre[threadIdx.x >> 5][0];
    int* pn = s_pre[threadIdx.x >> 5][1];
    pf[lane] = fi - nf;
    pn[lane] = ni - nn;
    if (lane == 31) { pf[32] = fi; pn[32] = ni; }
    __syncwarp();
    if (fits && !deferred) {
      warp_copy<false>(W.temp, tid0, B, pf, W.far_idx + fb);
      warp_copy<true>(W.temp, tid0, B, pn, W.near_idx + nb);
    }
    __syncwarp();
  }
}

// The deferred copy of a one-round arena walk (k_walk_arena's `deferred`):
// warp per leaf, lanes over its entries; leaf k's lists are in the scratch of
// thread k.  Runs before k_walk_heavy, while the queued leaves' counts are 0.
__global__ void k_arena_copy(WalkArgs W, int64_t walk_threads) {
  const int nleaves = W.counters[C_LEAVES];
  if (nleaves > walk_threads) return;            // the walk copied its lists itself
  const int lane = threadIdx.x & 31;
  const int B = W.budget;
  for (int k = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5); k < nleaves;
       k += (int)((gridDim.x * blockDim.x) >> 5)) {
    const int32_t* src = W.temp + (int64_t)k * B;
    warp_copy_list<false>(src, W.far_cnt[k], W.far_idx + W.far_off[k], lane);
    warp_copy_list<true>(src + (B - 1), W.near_cnt[k], W.near_idx + W.near_off[k], lane);
  }
}

// Block-wide walk of the queued leaves.  The depth-first walk visits cell i
// unless a cell p < i with i < skip(p) -- an ancestor of i in pre-order --
// was closed; so with every cell of the system decided at once, i is visited
// iff the largest skip pointer of the closed cells before i does not exceed
// i (a prefix maximum).  A visited closed cell joins the far list, a visited
// opened leaf the near list; a block scan keeps them in ascending id, as the
// thread walk emits them.  Tiles of kHeavyTile cells advance past the subtrees
// closed so far, so closed regions are not read.  A queued leaf's walk is a
// chain of tiles, so the block is wide (512 threads, two blocks per SM: 5 %
// faster over the Plummer 2^20 walk than 256 threads, which take twice the
// tiles).
constexpr int kHeavyThreads = 512;
constexpr int kHeavyPer = 4;                        // consecutive cells per thread
constexpr int kHeavyTile = kHeavyThreads * kHeavyPer;
constexpr int kHeavyWarps = kHeavyThreads / 32;

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

__global__ void __launch_bounds__(kHeavyThreads, 2) k_walk_heavy(WalkArgs W) {
  __shared__ int sh_max[kHeavyWarps];
  __shared__ int2 sh_sum[kHeavyWarps];
  __shared__ long long sh_np[kHeavyWarps];
  __shared__ int sh_nex[kHeavyWarps];
  __shared__ long long sh_base[2];
  __shared__ int sh_fits;
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
    float thf = (float)theta, rkf = (float)W.r_kern;
    int always = theta == 0.0;
    asm("" : "+f"(thf), "+f"(rkf), "+r"(always));   // opaque: see walk_leaf
    int64_t fo = W.exact ? W.far_off[k] : (int64_t)k * W.cap_far;
    int64_t no = W.exact ? W.near_off[k] : (int64_t)k * W.cap_near;
    int64_t cap_far = W.exact ? INT64_MAX : W.cap_far;
    int64_t cap_near = W.exact ? INT64_MAX : W.cap_near;
    bool fits = true;
    int nf = 0, nn = 0, carry = 0, nex = 0;
    long long np = 0;
    // reserves room for the (block-uniform) nf + nn entries on the running totals
    auto reserve = [&]() {
      if (threadIdx.x == 0) {
        const unsigned long long fb = atomicAdd(&W.stats[2], (unsigned long long)nf);
        const unsigned long long nb = atomicAdd(&W.stats[3], (unsigned long long)nn);
        const int ok = (int64_t)(fb + nf) <= W.far_cap && (int64_t)(nb + nn) <= W.near_cap;
        if (!ok) atomicOr(W.status, ST_LISTS);
        sh_base[0] = (long long)fb;
        sh_base[1] = (long long)nb;
        sh_fits = ok;
      }
      __syncthreads();
      fo = sh_base[0];
      no = sh_base[1];
      fits = sh_fits != 0;
      __syncthreads();
    };
    // Slot and two-pass modes: one pass emitting at the leaf's offsets.
    // Arena mode: one pass into this block's slice of the thread walk's
    // scratch (idle by now), far entries from its front and near entries from
    // its back -- a walk emits at most one entry per cell of its system, so
    // the two never meet -- then room is reserved and the block copies the
    // lists there.  A system with more cells than the slice holds takes a
    // counting pass, the reservation and an emitting pass instead.
    const bool staged = W.arena && (int64_t)(i_end - i0) <= W.heavy_scratch;
    int32_t* const scr = W.temp + (int64_t)blockIdx.x * W.heavy_scratch;
    if (staged) cap_far = cap_near = INT64_MAX;
    for (int pass = (W.arena && !staged) ? 0 : 1; pass < 2; ++pass) {
    const bool emit = pass == 1;
    int32_t* far = staged ? scr : W.far_idx + fo;
    int32_t* near = staged ? scr + (W.heavy_scratch - 1) : W.near_idx + no;
    const int nstep = staged ? -1 : 1;                 // near entries run backwards in the slice
    nf = nn = carry = nex = 0;
    np = 0;
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
          const float4 w2 = W.walk2[c];
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
      if (emit) {
#pragma unroll
        for (int j = 0; j < kHeavyPer; ++j) {
          if (ef[j]) { if (pf < cap_far) far[pf] = c0 + j; ++pf; }
          if (en[j]) { if (pn < cap_near) near[(int64_t)nstep * pn] = c0 + j; ++pn; }
        }
      }
      nf += tf;
      nn += tn;
      carry = max(carry, tile_max);
      t0 = max(t0 + kHeavyTile, carry);
    }
    if (!emit) {
      reserve();
      cap_far = cap_near = INT64_MAX;
      if (!fits) break;
    }
    }
    if (staged) {
      __syncthreads();                                 // the slice is written
      reserve();
      if (fits) {
        for (int e = threadIdx.x; e < nf; e += kHeavyThreads) W.far_idx[fo + e] = scr[e];
        for (int e = threadIdx.x; e < nn; e += kHeavyThreads)
          W.near_idx[no + e] = scr[W.heavy_scratch - 1 - e];
      }
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
      W.far_off[k] = fo;
      W.near_off[k] = no;
      W.far_cnt[k] = fits ? nf : 0;
      W.near_cnt[k] = fits ? nn : 0;
      atomicMax(&W.maxc[0], nf);
      atomicMax(&W.maxc[1], nn);
      const long long na = W.count[a];
      atomicAdd(&W.stats[0], (unsigned long long)(na * npt - na));
      if (!W.arena) {
        atomicAdd(&W.stats[2], (unsigned long long)nf);
        atomicAdd(&W.stats[3], (unsigned long long)nn);
      }
      if (nxt) atomicAdd(&W.stats[1], (unsigned long long)nxt);
    }
    __syncthreads();
  }
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

// Cells one thread walks before its leaf goes to the block-wide walk: the
// handle's setting (kdfmm_tree_set_walk_budget), else KDFMM_WALK_BUDGET, else
// 4096 (the lists do not depend on it).
static int walk_budget(const kdfmm_tree_s* t) {
  if (t->walk_budget > 0) return t->walk_budget;
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
// themselves, the handle switches to arena mode for good, or, when the arena
// walk's scratch cannot be allocated, to two-pass lists (a counting walk,
// a scan, a filling walk) for that evaluation.  The environment variable
// KDFMM_LIST_MODE=exact starts a handle in arena mode with small buffers
// (which then grow); KDFMM_LIST_MODE=two_pass always takes two passes.
constexpr int64_t kSlotBudgetBytes = int64_t(1) << 30;

static bool list_mode_is(const char* want) {
  const char* v = getenv("KDFMM_LIST_MODE");
  return v != nullptr && strcmp(v, want) == 0;
}

// Persistent grid of the arena walk: the resident blocks, at most one thread
// per leaf.
static int arena_grid_for(int leaves) {
  static int per_sm = 0;
  const int sms = sm_count();
  if (per_sm == 0) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk_arena<true>, 128, 0) != cudaSuccess ||
        per_sm < 1) {
      cudaGetLastError();
      per_sm = 1;
    }
  }
  return (int)std::max<int64_t>(1, std::min<int64_t>(blocks_for(std::max(leaves, 1), 128),
                                                     (int64_t)per_sm * sms));
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
  W.budget = walk_budget(t);
  W.heavy = L.heavy;
  W.heavy_n = t->counters + C_HEAVY;
  return W;
}

// One walk into the current slots or arena, no synchronisation.
enum class ListMode { kSlots, kArena, kTwoPass };

static void walk_launch(kdfmm_tree_s* t, WalkArgs W, ListMode mode, int64_t cf, int64_t cn,
                        int slot_leaves, cudaStream_t s) {
  Lists& L = t->L;
  const bool arena = mode == ListMode::kArena;
  W.arena = arena;
  W.exact = mode == ListMode::kTwoPass;
  W.far_idx = L.far_idx;
  W.near_idx = L.near_idx;
  W.cap_far = cf;
  W.cap_near = cn;
  W.far_cap = L.far_cap;
  W.near_cap = L.near_cap;
  W.temp = L.temp;
  W.heavy_scratch = arena ? L.temp_cap / grid_blocks(2) : 0;
  W.slot_leaves = slot_leaves;
  cudaMemsetAsync(L.near_np, 0, 4 * sizeof(int64_t), s);
  cudaMemsetAsync(t->counters + C_MAXFAR, 0, 2 * sizeof(int32_t), s);
  cudaMemsetAsync(t->counters + C_HEAVY, 0, sizeof(int32_t), s);
  if (arena) {
    // one round (no more leaves than threads): the walk is latency-bound and
    // its lanes run free; several rounds fill the GPU and the synchronous loop
    // wins (3 % slower on a Plummer sphere of 2^20, 9 % faster on 256
    // Plummer systems).  The host's leaf count picks the form; the kernel
    // handles any count.
    if (slot_leaves <= (int64_t)L.arena_grid * 128)
      k_walk_arena<false><<<L.arena_grid, 128, 0, s>>>(W);
    else
      k_walk_arena<true><<<L.arena_grid, 128, 0, s>>>(W);
    k_arena_copy<<<grid_blocks(), 256, 0, s>>>(W, (int64_t)L.arena_grid * 128);
    t->launches += 1;
  } else {
    k_walk<<<blocks_for(std::max(slot_leaves, 1), 128), 128, 0, s>>>(W);
  }
  k_walk_heavy<<<grid_blocks(2), kHeavyThreads, 0, s>>>(W);
  t->launches += 2;
}

// Scratch of the arena walk over `leaves` leaves (budget entries per thread).
static int ensure_temp(kdfmm_tree_s* t, int leaves) {
  Lists& L = t->L;
  L.arena_grid = arena_grid_for(leaves);
  const int64_t need = (int64_t)L.arena_grid * 128 * walk_budget(t);
  if (L.temp_cap >= need && L.temp != nullptr) return KDFMM_OK;
  cudaFree(L.temp);
  L.temp = nullptr;
  L.temp_cap = 0;
  if (cudaMalloc(&L.temp, (size_t)need * sizeof(int32_t)) != cudaSuccess) {
    cudaGetLastError();
    return set_error(KDFMM_ERR_OOM, "walk scratch (%lld entries)", (long long)need);
  }
  L.temp_cap = need;
  return KDFMM_OK;
}

int ensure_arena(kdfmm_tree_s* t, int leaves, double extra) {
  Lists& L = t->L;
  const int64_t nf = t->host_stats[KDFMM_STAT_NFAR], nn = t->host_stats[KDFMM_STAT_NNEAR];
  int rc;
  if ((rc = ensure_idx(&L.far_idx, &L.far_cap, (int64_t)(nf * extra) + 1024, "far lists", true)))
    return rc;
  if ((rc = ensure_idx(&L.near_idx, &L.near_cap, (int64_t)(nn * extra) + 1024, "near lists", true)))
    return rc;
  return ensure_temp(t, leaves);
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
  if (L.arena) {
    if (L.temp == nullptr) return set_error(KDFMM_ERR_INTERNAL, "arena walk scratch not allocated");
    walk_launch(t, walk_args(t), ListMode::kArena, 0, 0, slot_leaves, s);
    return check_cuda(cudaGetLastError(), "walk launch");
  }
  if (L.far_cap < (int64_t)slot_leaves * L.cap_far || L.near_cap < (int64_t)slot_leaves * L.cap_near)
    return set_error(KDFMM_ERR_INTERNAL, "list slots not allocated for %d leaves", slot_leaves);
  L.exact = false;
  walk_launch(t, walk_args(t), ListMode::kSlots, L.cap_far, L.cap_near, slot_leaves, s);
  return check_cuda(cudaGetLastError(), "walk launch");
}

int run_walk(kdfmm_tree_s* t, cudaStream_t s) {
  const int nl = t->nleaves;
  Lists& L = t->L;
  int64_t cf = L.cap_far > 0 ? L.cap_far : 512, cn = L.cap_near > 0 ? L.cap_near : 128;
  WalkArgs W = walk_args(t);
  int32_t* hc = t->host_counters;
  int rc;
  auto launch = [&](ListMode mode) {
    walk_launch(t, W, mode, cf, cn, nl, s);
    cudaMemcpyAsync(hc + C_MAXFAR, t->counters + C_MAXFAR, 2 * sizeof(int32_t),
                    cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(t->host_stats + 16, L.near_np, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
    return check_cuda(cudaStreamSynchronize(s), "walk");
  };
  auto done = [&](ListMode mode) {
    L.arena = mode == ListMode::kArena;
    L.exact = mode != ListMode::kSlots;
    t->host_stats[KDFMM_STAT_NFAR] = t->host_stats[16 + 2];
    t->host_stats[KDFMM_STAT_NNEAR] = t->host_stats[16 + 3];
    return check_cuda(cudaGetLastError(), "walk launch");
  };
  // two passes: counts only (slots of size 0), scanned into offsets, then
  // the lists at those offsets
  auto two_pass = [&]() {
    cf = cn = 0;
    if ((rc = launch(ListMode::kSlots))) return rc;
    const int64_t tf = t->host_stats[16 + 2], tn = t->host_stats[16 + 3];
    scan_i32_to_i64(L.far_cnt, L.far_off, nl, reinterpret_cast<int64_t*>(t->scan_tmp), s);
    scan_i32_to_i64(L.near_cnt, L.near_off, nl, reinterpret_cast<int64_t*>(t->scan_tmp), s);
    t->launches += 6;
    if ((rc = ensure_idx(&L.far_idx, &L.far_cap, tf, "far lists"))) return rc;
    if ((rc = ensure_idx(&L.near_idx, &L.near_cap, tn, "near lists"))) return rc;
    if ((rc = launch(ListMode::kTwoPass))) return rc;
    if (t->host_stats[16 + 2] != tf || t->host_stats[16 + 3] != tn)
      return set_error(KDFMM_ERR_INTERNAL, "the two walk passes disagree");
    return done(ListMode::kTwoPass);
  };
  // arena mode: one pass; a first pass whose lists outgrow the buffers
  // (counts 0, totals complete) is repeated once with room for the totals
  auto arena_walk = [&](int64_t want_far, int64_t want_near) {
    for (int attempt = 0; attempt < 2; ++attempt) {
      if ((rc = ensure_idx(&L.far_idx, &L.far_cap, want_far, "far lists"))) return rc;
      if ((rc = ensure_idx(&L.near_idx, &L.near_cap, want_near, "near lists"))) return rc;
      if (ensure_temp(t, nl) != KDFMM_OK) {
        L.arena = false;
        return two_pass();
      }
      if ((rc = launch(ListMode::kArena))) return rc;
      const int64_t tf = t->host_stats[16 + 2], tn = t->host_stats[16 + 3];
      if (tf <= L.far_cap && tn <= L.near_cap) return done(ListMode::kArena);
      want_far = tf + tf / 8 + 1024;
      want_near = tn + tn / 8 + 1024;
    }
    return set_error(KDFMM_ERR_CAPACITY, "interaction lists kept outgrowing their buffers");
  };
  if (list_mode_is("two_pass")) return two_pass();
  if (L.arena) return arena_walk(L.far_cap, L.near_cap);
  if (list_mode_is("exact")) return arena_walk((int64_t)nl * 64, (int64_t)nl * 16);
  for (int attempt = 0; attempt < 4; ++attempt) {
    if ((rc = ensure_idx(&L.far_idx, &L.far_cap, (int64_t)nl * cf, "far list slots"))) return rc;
    if ((rc = ensure_idx(&L.near_idx, &L.near_cap, (int64_t)nl * cn, "near list slots"))) return rc;
    if ((rc = launch(ListMode::kSlots))) return rc;
    const int64_t mf = hc[C_MAXFAR], mn = hc[C_MAXNEAR];
    const int64_t tot_far = t->host_stats[16 + 2], tot_near = t->host_stats[16 + 3];
    if (mf <= cf && mn <= cn) {
      L.cap_far = cf;
      L.cap_near = cn;
      return done(ListMode::kSlots);
    }
    const int64_t cf2 = std::max<int64_t>(cf, mf + mf / 4 + 16);
    const int64_t cn2 = std::max<int64_t>(cn, mn + mn / 4 + 16);
    const int64_t slot_bytes = (int64_t)nl * (cf2 + cn2) * 4;
    if (slot_bytes > kSlotBudgetBytes && slot_bytes > 8 * (tot_far + tot_near))
      return arena_walk(tot_far + tot_far / 8 + 1024, tot_near + tot_near / 8 + 1024);
    cf = cf2;
    cn = cn2;
  }
  return set_error(KDFMM_ERR_CAPACITY, "interaction lists kept outgrowing their slots");
}

}  // namespace kdfmm
