// kd-tree construction and cell moments (Sec. 2; Eq. 7).
//
// Each cell is cut through its centre of mass across the longest side of its
// bounding box; a cell with more than n_leaf particles is split.  The centre
// of mass is the pairwise (perfect binary tree) sum of m and m x over the
// cell's particles in ascending caller index, zero-padded to a power of two,
// divided by the pairwise sum of m -- every float64 operation that decides a
// cut is correctly rounded and uncontracted, so the tree is reproducible bit
// for bit on any device and on the host.
//
// Phase A: cells larger than kSubtreeMax are split level by level in global
//          memory, each cell tiled into 2048-element chunks aligned to the
//          cell's first particle (chunk sums are the subtrees of the pairwise
//          tree, so the tiling does not change the result).
// Phase B: a cell of at most kSubtreeMax particles is finished by one CTA with
//          its particles held in shared memory; each warp splits one cell.
// Then the cells are renumbered in pre-order from their particle ranges, the
// quadrupoles and h_max are accumulated bottom-up, and float32 views for the
// walk, the M2L and the P2P are derived.
#include <algorithm>
#include <climits>

#include "kdfmm_internal.cuh"

namespace kdfmm {

namespace {

struct BuildArgs {
  PCols src, dst;
  TmpCells tmp;
  int32_t* counters;
  int32_t* status;
  const int64_t* sys_off;          // forest: particle offsets of the systems
  const int32_t* sys_nleaf;        // forest: leaf size of each system
  int32_t n_sys;
  int64_t capA, capB, capL, cap_cells;
};

__device__ __forceinline__ int nleaf_at(const BuildArgs& A, int64_t first) {
  return A.sys_nleaf[system_of(A.sys_off, A.n_sys, first)];
}

__device__ __forceinline__ double coord(const PCols& p, int axis, int64_t i) {
  return axis == 0 ? p.x[i] : (axis == 1 ? p.y[i] : p.z[i]);
}

__device__ __forceinline__ void set_status(int32_t* status, int bits) { atomicOr(status, bits); }

// ---------------------------------------------------------------------------
// initial gather: caller order -> SoA buffer 0, with validation
// ---------------------------------------------------------------------------
__global__ void k_init(const double* __restrict__ x, const double* __restrict__ m,
                       const double* __restrict__ h, int64_t n, const int64_t* __restrict__ sys_off,
                       int n_sys, const double* __restrict__ sys_eps, int soft_kind, PCols b,
                       int32_t* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2], mi = m[i];
  double hi = (h != nullptr && soft_kind == KDFMM_SOFT_M4) ? h[i]
                                                           : sys_eps[system_of(sys_off, n_sys, i)];
  bool ok = isfinite(xi) && isfinite(yi) && isfinite(zi) && isfinite(mi) && isfinite(hi) &&
            mi > 0.0 && (soft_kind == KDFMM_SOFT_M4 ? hi > 0.0 : hi >= 0.0);
  if (!ok) set_status(status, ST_NONFINITE);
  b.x[i] = xi; b.y[i] = yi; b.z[i] = zi; b.m[i] = mi; b.h[i] = hi;
  b.idx[i] = (int32_t)i;
}

// One root segment per system (build-order cell k for system k).
__global__ void k_roots(BuildArgs A, Seg* segA, Seg* segB, Seg* segL) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k == 0) atomicAdd(&A.counters[0], A.n_sys);
  if (k >= A.n_sys) return;
  const int64_t f = A.sys_off[k], cnt = A.sys_off[k + 1] - f;
  const Seg g{(int32_t)f, (int32_t)cnt, k, 0};
  if (cnt > kSubtreeMax) {
    const int i = atomicAdd(&A.counters[1], 1);
    if (i < A.capA) segA[i] = g; else set_status(A.status, ST_CAPACITY);
  } else if (cnt > A.sys_nleaf[k]) {
    const int i = atomicAdd(&A.counters[2], 1);
    if (i < A.capB) segB[i] = g; else set_status(A.status, ST_CAPACITY);
  } else {
    const int i = atomicAdd(&A.counters[3], 1);
    if (i < A.capL) segL[i] = g; else set_status(A.status, ST_CAPACITY);
  }
}

// Pushes a new segment onto the list that will process it.
__device__ void push_child(const BuildArgs& A, Seg c, Seg* nextA, Seg* segB, Seg* segL) {
  if (c.count > kSubtreeMax) {
    int k = atomicAdd(&A.counters[1], 1);
    if (k < A.capA) nextA[k] = c; else set_status(A.status, ST_CAPACITY);
  } else if (c.count > nleaf_at(A, c.first)) {
    int k = atomicAdd(&A.counters[2], 1);
    if (k < A.capB) segB[k] = c; else set_status(A.status, ST_CAPACITY);
  } else {
    int k = atomicAdd(&A.counters[3], 1);
    if (k < A.capL) segL[k] = c; else set_status(A.status, ST_CAPACITY);
  }
}

// ---------------------------------------------------------------------------
// phase A
// ---------------------------------------------------------------------------
__device__ __forceinline__ int nchunks_of(int count) { return (count + kChunk - 1) / kChunk; }

// Start of a phase-A level: the segments pushed by the previous level are
// this level's (counters[C_NA]); the push counter restarts.
__global__ void k_level_begin(int32_t* counters, int64_t capA, int32_t* status) {
  int na = counters[C_NEXT_A];
  if (na > capA) {
    set_status(status, ST_CAPACITY);
    na = (int)capA;
  }
  counters[C_NA] = na;
  counters[C_NEXT_A] = 0;
}

// After the last phase-A level: segments still waiting for a split mean the
// fixed number of levels was too small.
__global__ void k_levels_done(const int32_t* counters, int32_t* status) {
  if (counters[C_NEXT_A] > 0) set_status(status, ST_UNFINISHED);
}

// Chunk offsets of the nA segments (single block) and the chunk -> segment map.
__global__ void k_chunk_map(const Seg* __restrict__ segs, const int32_t* __restrict__ nA_dev, int32_t* __restrict__ seg_off,
                            int32_t* __restrict__ chunk_seg, int32_t* counters) {
  const int nA = *nA_dev;
  __shared__ int32_t warp_tot[32];
  __shared__ int32_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int base = 0; base < nA; base += blockDim.x) {
    int s = base + threadIdx.x;
    int e = s < nA ? nchunks_of(segs[s].count) : 0;
    int incl = e;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    if (lane == 31) warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
      int t = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
      int ti = t;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int v = __shfl_up_sync(0xffffffffu, ti, o);
        if (lane >= o) ti += v;
      }
      warp_tot[lane] = ti - t;
    }
    __syncthreads();
    int excl = carry + warp_tot[w] + incl - e;
    __syncthreads();
    if (s < nA) {
      seg_off[s] = excl;
      for (int c = 0; c < e; ++c) chunk_seg[excl + c] = s;
    }
    if (threadIdx.x == blockDim.x - 1) carry = excl + e;
    __syncthreads();
  }
  if (threadIdx.x == 0) counters[4] = carry;
}

// Chunk partial sums (pairwise subtree of kChunk elements) and bounding box keys.
__global__ void __launch_bounds__(kChunkThreads)
k_chunk_reduce(const Seg* __restrict__ segs, const int32_t* __restrict__ chunk_seg,
               const int32_t* __restrict__ seg_off, const int32_t* __restrict__ counters,
               PCols p, double* __restrict__ csum, long long* __restrict__ ckey) {
  const int b = blockIdx.x;
  if (b >= counters[4]) return;
  const int s = chunk_seg[b];
  const Seg g = segs[s];
  const int rel0 = (b - seg_off[s]) * kChunk;
  const int cnt = g.count - rel0;               // valid elements from the chunk start
  const int64_t base = (int64_t)g.first + rel0;
  // the bounding-box keys come with the same loads (get runs once per element)
  long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
  auto get = [&](int k) {
    int64_t i = base + k;
    const double x = p.x[i], y = p.y[i], z = p.z[i];
    const long long kx = dkey(x), ky = dkey(y), kz = dkey(z);
    lo[0] = min(lo[0], kx); hi[0] = max(hi[0], kx);
    lo[1] = min(lo[1], ky); hi[1] = max(hi[1], ky);
    lo[2] = min(lo[2], kz); hi[2] = max(hi[2], kz);
    return elem4(p.m[i], x, y, z);
  };
  Sum4 v = block_tree<3>(8 * threadIdx.x, cnt, get);
  v = warp_tree4(v);
#pragma unroll
  for (int d = 0; d < 3; ++d) { lo[d] = warp_min_ll(lo[d]); hi[d] = warp_max_ll(hi[d]); }
  __shared__ Sum4 ws[kChunkThreads / 32];
  __shared__ long long wk[kChunkThreads / 32][6];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) {
    ws[w] = v;
    for (int d = 0; d < 3; ++d) { wk[w][d] = lo[d]; wk[w][3 + d] = hi[d]; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // perfect tree over the warps' subtrees (the top levels of the chunk's tree)
    constexpr int kW = kChunkThreads / 32;
    Sum4 t4[kW];
#pragma unroll
    for (int q = 0; q < kW; ++q) t4[q] = ws[q];
#pragma unroll
    for (int width = kW; width > 1; width >>= 1)
#pragma unroll
      for (int q = 0; q < width / 2; ++q) t4[q] = add4(t4[2 * q], t4[2 * q + 1]);
    const Sum4 t = t4[0];
    csum[4 * b + 0] = t.m; csum[4 * b + 1] = t.x; csum[4 * b + 2] = t.y; csum[4 * b + 3] = t.z;
    for (int d = 0; d < 6; ++d) {
      long long r = wk[0][d];
      for (int q = 1; q < kChunkThreads / 32; ++q) r = d < 3 ? min(r, wk[q][d]) : max(r, wk[q][d]);
      ckey[6 * b + d] = r;
    }
  }
}

// Warp per segment: pairwise tree over its chunk sums, centre of mass, axis, cut.
__global__ void k_decide(const Seg* __restrict__ segs, const int32_t* __restrict__ nA_dev, const int32_t* __restrict__ seg_off,
                         const double* __restrict__ csum, const long long* __restrict__ ckey,
                         TmpCells tmp, int32_t* __restrict__ seg_axis, double* __restrict__ seg_cut,
                         float* __restrict__ seg_xb, long long* __restrict__ seg_s2) {
  const int nA = *nA_dev;
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= nA) return;
  const Seg g = segs[s];
  const int C = nchunks_of(g.count);
  const int off = seg_off[s];
  int P = 1;
  while (P < C) P <<= 1;
  const int B = P > 32 ? P >> 5 : 1;
  auto chunk = [&](int c) {
    return c < C ? Sum4{csum[4 * (off + c)], csum[4 * (off + c) + 1], csum[4 * (off + c) + 2],
                        csum[4 * (off + c) + 3]}
                 : zero4();
  };
  Sum4 v;
  if (B == 1) {
    v = chunk(lane);
  } else {
    // sequential perfect tree over this lane's B chunks (carry stack)
    Sum4 st[16];
    int top = 0;
    for (int k = 0; k < B; ++k) {
      Sum4 e = chunk(lane * B + k);
      for (int kk = k; kk & 1; kk >>= 1) e = add4(st[--top], e);
      st[top++] = e;
    }
    v = st[0];
  }
  v = warp_tree4(v);
  long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
  for (int c = lane; c < C; c += 32)
    for (int d = 0; d < 3; ++d) {
      lo[d] = min(lo[d], ckey[6 * (off + c) + d]);
      hi[d] = max(hi[d], ckey[6 * (off + c) + 3 + d]);
    }
  double dlo[3], dhi[3];
  for (int d = 0; d < 3; ++d) {
    dlo[d] = dunkey(warp_min_ll(lo[d]));
    dhi[d] = dunkey(warp_max_ll(hi[d]));
  }
  if (lane == 0) {
    const double M = v.m;
    const double cx = __ddiv_rn(v.x, M), cy = __ddiv_rn(v.y, M), cz = __ddiv_rn(v.z, M);
    const int axis = longest_axis(dlo, dhi);
    const int c = g.cell;
    tmp.first[c] = g.first; tmp.count[c] = g.count; tmp.depth[c] = g.dbuf >> 1;
    tmp.M[c] = M; tmp.cx[c] = cx; tmp.cy[c] = cy; tmp.cz[c] = cz;
    seg_axis[s] = axis;
    seg_cut[s] = axis == 0 ? cx : (axis == 1 ? cy : cz);
    double X = 0.0;
    for (int d = 0; d < 3; ++d) X = fmax(X, fmax(fabs(dlo[d]), fabs(dhi[d])));
    seg_xb[s] = (float)X * 1.000001f;
    seg_s2[s] = 0;
  }
}

// Per chunk: particles left of the cut, and the largest float32 estimate of
// the squared distance to the centre of mass (coordinates truncated to
// float32 with integer operations; the exact size follows in the scatter).
__global__ void __launch_bounds__(kChunkThreads)
k_chunk_count(const Seg* __restrict__ segs, const int32_t* __restrict__ chunk_seg,
              const int32_t* __restrict__ seg_off, const int32_t* __restrict__ counters, PCols p,
              TmpCells tmp, const int32_t* __restrict__ seg_axis, const double* __restrict__ seg_cut,
              int32_t* __restrict__ cleft, float* __restrict__ cs2) {
  const int b = blockIdx.x;
  if (b >= counters[4]) return;
  const int s = chunk_seg[b];
  const Seg g = segs[s];
  const int rel0 = (b - seg_off[s]) * kChunk;
  const int cnt = min(kChunk, g.count - rel0);
  const int64_t base = (int64_t)g.first + rel0;
  const int axis = seg_axis[s];
  const long long ckey = dkey(seg_cut[s]);
  const float cx = trunc_to_float(tmp.cx[g.cell]), cy = trunc_to_float(tmp.cy[g.cell]),
              cz = trunc_to_float(tmp.cz[g.cell]);
  int nl = 0;
  float s2 = 0.0f;
#pragma unroll
  for (int pass = 0; pass < kChunk / kChunkThreads; ++pass) {   // all loads in flight
    const int k = pass * kChunkThreads + threadIdx.x;
    if (k >= cnt) continue;
    int64_t i = base + k;
    const double px = p.x[i], py = p.y[i], pz = p.z[i];
    const double a = axis == 0 ? px : (axis == 1 ? py : pz);
    nl += dkey(a) < ckey;
    const float dx = trunc_to_float(px) - cx, dy = trunc_to_float(py) - cy, dz = trunc_to_float(pz) - cz;
    s2 = fmaxf(s2, dx * dx + dy * dy + dz * dz);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nl += __shfl_xor_sync(0xffffffffu, nl, o);
    s2 = fmaxf(s2, __shfl_xor_sync(0xffffffffu, s2, o));
  }
  __shared__ int wn[kChunkThreads / 32];
  __shared__ float ws2[kChunkThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { wn[w] = nl; ws2[w] = s2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    float m2 = 0.0f;
    for (int q = 0; q < kChunkThreads / 32; ++q) { t += wn[q]; m2 = fmaxf(m2, ws2[q]); }
    cleft[b] = t;
    cs2[b] = m2;
  }
}

// Warp per segment: offsets of the left particles per chunk, the split point,
// s, and the two children.
__global__ void k_split(const Seg* __restrict__ segs, const int32_t* __restrict__ nA_dev, const int32_t* __restrict__ seg_off,
                        const int32_t* __restrict__ cleft, const float* __restrict__ cs2,
                        int32_t* __restrict__ cloff, int32_t* __restrict__ seg_nl,
                        const float* __restrict__ seg_xb, float* __restrict__ seg_thr2, BuildArgs A,
                        Seg* nextA, Seg* segB, Seg* segL, int dst_buf) {
  const int nA = *nA_dev;
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= nA) return;
  const Seg g = segs[s];
  const int C = nchunks_of(g.count);
  const int off = seg_off[s];
  int run = 0;
  float s2 = 0.0f;
  for (int base = 0; base < C; base += 32) {
    int c = base + lane;
    int v = c < C ? cleft[off + c] : 0;
    if (c < C) s2 = fmaxf(s2, cs2[off + c]);
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int w = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += w;
    }
    if (c < C) cloff[off + c] = run + incl - v;
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s2 = fmaxf(s2, __shfl_xor_sync(0xffffffffu, s2, o));
  if (lane != 0) return;
  {
    const float Dm = sqrtf(s2);
    const float thr = Dm - 2.0f * dist_err_bound(seg_xb[s], Dm);
    seg_thr2[s] = thr > 0.0f ? thr * thr * (1.0f - 1e-6f) : -1.0f;
  }
  int nl = run;
  const bool fallback = (nl == 0 || nl == g.count);
  if (fallback) {
    nl = g.count / 2;
    atomicAdd(&A.counters[5], 1);
  }
  seg_nl[s] = fallback ? -nl - 1 : nl;
  const int c = g.cell;
  int cid = atomicAdd(&A.counters[0], 2);
  if (cid + 2 > A.cap_cells) { set_status(A.status, ST_CAPACITY); return; }
  A.tmp.left[c] = cid;
  A.tmp.right[c] = cid + 1;
  const int depth = (g.dbuf >> 1) + 1;
  atomicMax(&A.counters[6], depth);
  push_child(A, Seg{g.first, nl, cid, depth << 1 | dst_buf}, nextA, segB, segL);
  push_child(A, Seg{g.first + nl, g.count - nl, cid + 1, depth << 1 | dst_buf}, nextA, segB, segL);
}

// Stable scatter of one chunk into the other buffer.  Element k of the chunk
// (pass k / kChunkThreads, thread k % kChunkThreads) goes to the left child at
// its rank among the segment's left elements, else to the right child.  The
// flags of all the chunk's elements are taken first (their coordinate loads in
// flight together), one block barrier publishes the passes' warp counts, and
// the moves follow with kMoveBatch elements' loads in flight per thread.  Pass
// by pass, with two barriers each, the kernel waited on one load at a time:
// this form took the benchmark's build 3.72 -> 3.56 ms (batches of 1, 2 or 4
// elements, rolled or unrolled, measured within 1 % of each other).
constexpr int kScatterPasses = kChunk / kChunkThreads;
constexpr int kMoveBatch = 2;
__global__ void __launch_bounds__(kChunkThreads)
k_chunk_scatter(const Seg* __restrict__ segs, const int32_t* __restrict__ chunk_seg,
                const int32_t* __restrict__ seg_off, const int32_t* __restrict__ counters, PCols src,
                PCols dst, const int32_t* __restrict__ seg_axis, const double* __restrict__ seg_cut,
                const int32_t* __restrict__ cloff, const int32_t* __restrict__ seg_nl,
                TmpCells tmp, const float* __restrict__ seg_thr2, long long* __restrict__ seg_s2) {
  const int b = blockIdx.x;
  if (b >= counters[4]) return;
  const int s = chunk_seg[b];
  const Seg g = segs[s];
  const int rel0 = (b - seg_off[s]) * kChunk;
  const int code = seg_nl[s];
  const bool fallback = code < 0;
  const int nl = fallback ? -code - 1 : code;
  const int axis = seg_axis[s];
  const long long ckey = dkey(seg_cut[s]);
  __shared__ int wcount[kScatterPasses][kChunkThreads / 32];
  __shared__ long long ws2[kChunkThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const unsigned lt = (1u << lane) - 1u;
  bool flag[kScatterPasses];
  int rank[kScatterPasses];
#pragma unroll
  for (int pass = 0; pass < kScatterPasses; ++pass) {
    const int k = rel0 + pass * kChunkThreads + threadIdx.x;   // position within the segment
    flag[pass] = false;
    if (k < g.count)
      flag[pass] = fallback ? (k < nl) : (dkey(coord(src, axis, (int64_t)g.first + k)) < ckey);
  }
#pragma unroll
  for (int pass = 0; pass < kScatterPasses; ++pass) {
    const unsigned mask = __ballot_sync(0xffffffffu, flag[pass]);
    rank[pass] = __popc(mask & lt);
    if (lane == 0) wcount[pass][w] = __popc(mask);
  }
  __syncthreads();
  int before = fallback ? min(rel0, nl) : cloff[b];          // left elements before the pass
#pragma unroll
  for (int pass = 0; pass < kScatterPasses; ++pass) {
    int woff = 0, tot = 0;
#pragma unroll
    for (int q = 0; q < kChunkThreads / 32; ++q) {
      const int c = wcount[pass][q];
      woff += q < w ? c : 0;
      tot += c;
    }
    rank[pass] += before + woff;                               // left elements before this one
    before += tot;
  }
  const double cx = tmp.cx[g.cell], cy = tmp.cy[g.cell], cz = tmp.cz[g.cell];
  const float cxf = trunc_to_float(cx), cyf = trunc_to_float(cy), czf = trunc_to_float(cz);
  const float thr2 = seg_thr2[s];
  long long s2 = 0;
#pragma unroll 1
  for (int p0 = 0; p0 < kScatterPasses; p0 += kMoveBatch) {
    double px[kMoveBatch], py[kMoveBatch], pz[kMoveBatch], pm[kMoveBatch], ph[kMoveBatch];
    int32_t pi[kMoveBatch];
#pragma unroll
    for (int u = 0; u < kMoveBatch; ++u) {
      const int k = rel0 + (p0 + u) * kChunkThreads + threadIdx.x;
      px[u] = py[u] = pz[u] = pm[u] = ph[u] = 0.0;
      pi[u] = 0;
      if (k < g.count) {
        const int64_t i = (int64_t)g.first + k;
        px[u] = src.x[i]; py[u] = src.y[i]; pz[u] = src.z[i];
        pm[u] = src.m[i]; ph[u] = src.h[i]; pi[u] = src.idx[i];
      }
    }
#pragma unroll
    for (int u = 0; u < kMoveBatch; ++u) {
      const int k = rel0 + (p0 + u) * kChunkThreads + threadIdx.x;
      if (k >= g.count) continue;
      const int lb = rank[p0 + u];
      const int64_t d = flag[p0 + u] ? (int64_t)g.first + lb : (int64_t)g.first + nl + (k - lb);
      dst.x[d] = px[u]; dst.y[d] = py[u]; dst.z[d] = pz[u];
      dst.m[d] = pm[u]; dst.h[d] = ph[u]; dst.idx[d] = pi[u];
      const float ex = trunc_to_float(px[u]) - cxf, ey = trunc_to_float(py[u]) - cyf,
                  ez = trunc_to_float(pz[u]) - czf;
      if (ex * ex + ey * ey + ez * ez >= thr2)
        s2 = max(s2, __double_as_longlong(dist2_rn(px[u], py[u], pz[u], cx, cy, cz)));
    }
  }
  s2 = warp_max_ll(s2);
  if (lane == 0) ws2[w] = s2;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long m2 = 0;
    for (int q = 0; q < kChunkThreads / 32; ++q) m2 = max(m2, ws2[q]);
    if (m2 > 0) atomicMax(reinterpret_cast<unsigned long long*>(&seg_s2[s]), (unsigned long long)m2);
  }
}

// Size of each phase-A cell from the exact squared maximum of its candidates.
__global__ void k_seg_size(const Seg* __restrict__ segs, const int32_t* __restrict__ nA_dev, const long long* __restrict__ seg_s2,
                           TmpCells tmp) {
  const int nA = *nA_dev;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < nA) tmp.s[segs[s].cell] = sqrt(__longlong_as_double(seg_s2[s]));
}

// ---------------------------------------------------------------------------
// phase B: one CTA finishes a subtree in shared memory
// ---------------------------------------------------------------------------
struct SubArgs {
  BuildArgs A;
  PCols buf0, buf1, out;
  const Seg* segB;
  int qcap;
};

// Cells of at least kBlockSeg particles are split by the whole CTA, one after
// the other; smaller ones by one warp each, in parallel (1024 measured 4 %
// faster over the build than 256, where a level of 8 cells of 256 took 8
// CTA-wide splits in a row).
constexpr int kBlockSeg = 1024;
constexpr int kSubWarps = kSubtreeThreads / 32;

// Shared-memory views of one subtree: float64 particles, float32 shadows of
// the positions (for the size filter), local index and scratch index arrays,
// and the two segment queues.
struct SubSmem {
  double *x, *y, *z, *m;
  float *xf, *yf, *zf;
  uint16_t *idx, *scr;
  int4* q[2];
};

__device__ __forceinline__ float dist2_f(const SubSmem& S, int q, float cx, float cy, float cz) {
  const float dx = S.xf[q] - cx, dy = S.yf[q] - cy, dz = S.zf[q] - cz;
  return dx * dx + dy * dy + dz * dz;
}

__device__ __forceinline__ float abs_bound(const double lo[3], const double hi[3]) {
  double X = 0.0;
  for (int d = 0; d < 3; ++d) X = fmax(X, fmax(fabs(lo[d]), fabs(hi[d])));
  return (float)X * 1.0000005f;
}

constexpr int kThreadSeg = 64;                      // split by one thread at this size

// Canonical pairwise sum of the cnt (<= 2^7) particles idx[lf..lf+cnt) by one
// thread: a carry stack builds the perfect binary tree over the sequence
// zero-padded to a power of two.  The padded zeros are not added: a subtree
// of zeros contributes nothing and x + 0 = x, so folding the stack from its
// top after the last element gives the same tree value.
__device__ __forceinline__ Sum4 thread_pairwise(const SubSmem& L, int lf, int cnt) {
  Sum4 st[8];
  int top = 0;
  for (int k = 0; k < cnt; ++k) {
    const int q = L.idx[lf + k];
    Sum4 e = elem4(L.m[q], L.x[q], L.y[q], L.z[q]);
    for (int kk = k; kk & 1; kk >>= 1) e = add4(st[--top], e);
    st[top++] = e;
  }
  Sum4 v = st[top - 1];
  for (int i = top - 2; i >= 0; --i) v = add4(st[i], v);
  return v;
}

// Exact squared size of a cell held in shared memory, by one thread: float32
// distances over the shadow coordinates select the particles that may hold the
// maximum, and only those are evaluated in float64.
__device__ __forceinline__ long long thread_size2(const SubSmem& L, int lf, int cnt, double cx,
                                                  double cy, double cz) {
  const float cxf = (float)cx, cyf = (float)cy, czf = (float)cz;
  float d2m = 0.0f, X = fmaxf(fabsf(cxf), fmaxf(fabsf(cyf), fabsf(czf)));
  for (int k = 0; k < cnt; ++k) {
    const int q = L.idx[lf + k];
    d2m = fmaxf(d2m, dist2_f(L, q, cxf, cyf, czf));
    X = fmaxf(X, fmaxf(fabsf(L.xf[q]), fmaxf(fabsf(L.yf[q]), fabsf(L.zf[q]))));
  }
  const float Dm = sqrtf(d2m);
  const float thr = Dm - 2.0f * dist_err_bound(X * 1.0000005f, Dm);
  const float thr2 = thr > 0.0f ? thr * thr * (1.0f - 1e-6f) : -1.0f;
  long long s2 = 0;
  for (int k = 0; k < cnt; ++k) {
    const int q = L.idx[lf + k];
    if (dist2_f(L, q, cxf, cyf, czf) >= thr2)
      s2 = max(s2, __double_as_longlong(dist2_rn(L.x[q], L.y[q], L.z[q], cx, cy, cz)));
  }
  return s2;
}

// Moments of a leaf in shared memory, computed by one thread.
__device__ void leaf_thread(const SubArgs& S, const SubSmem& L, int lf, int cnt, int cell,
                            int depth, int gfirst) {
  const Sum4 v = thread_pairwise(L, lf, cnt);
  const double M = v.m;
  const double cx = __ddiv_rn(v.x, M), cy = __ddiv_rn(v.y, M), cz = __ddiv_rn(v.z, M);
  const long long s2 = thread_size2(L, lf, cnt, cx, cy, cz);
  TmpCells t = S.A.tmp;
  t.first[cell] = gfirst + lf; t.count[cell] = cnt; t.depth[cell] = depth;
  t.M[cell] = M; t.cx[cell] = cx; t.cy[cell] = cy; t.cz[cell] = cz;
  t.s[cell] = sqrt(__longlong_as_double(s2));
  t.left[cell] = -1; t.right[cell] = -1;
}

// Queues of one level of a subtree: cells to split next, leaves to finish.
struct Queues {
  int* qn_next;
  int4* q_next;
  int* nleaf;
  int4* leaves;
  int leafcap;
  int n_leaf;      // leaf size of the subtree's system
};

// Pushes child `c` (local first, count, cell, depth) onto the queue that will
// process it; called by one thread.
__device__ __forceinline__ void push_local(const SubArgs& S, const Queues& Q, int4 c) {
  if (c.y > Q.n_leaf) {
    int pos = atomicAdd(Q.qn_next, 1);
    if (pos < S.qcap) Q.q_next[pos] = c; else set_status(S.A.status, ST_CAPACITY);
  } else {
    int pos = atomicAdd(Q.nleaf, 1);
    if (pos < Q.leafcap) Q.leaves[pos] = c; else set_status(S.A.status, ST_CAPACITY);
  }
}

// Allocates the two children of `cell` and queues them (lane 0 of the calling
// warp).  Returns false if the cell table is full.
__device__ bool make_children(const SubArgs& S, const Queues& Q, int lf, int cnt, int nl, int cell,
                              int depth) {
  const int lane = threadIdx.x & 31;
  const BuildArgs& A = S.A;
  int ok = 1;
  if (lane == 0) {
    const int cid = atomicAdd(&A.counters[0], 2);
    if (cid + 2 > A.cap_cells) {
      set_status(A.status, ST_CAPACITY);
      ok = 0;
    } else {
      A.tmp.left[cell] = cid;
      A.tmp.right[cell] = cid + 1;
      push_local(S, Q, make_int4(lf, nl, cid, depth + 1));
      push_local(S, Q, make_int4(lf + nl, cnt - nl, cid + 1, depth + 1));
    }
  }
  return __shfl_sync(0xffffffffu, ok, 0) != 0;
}

// A segment split by one thread (small cells): sums, bounding box, centre of
// mass, exact size, serial stable partition; leaf children are finished at
// once by the same thread.
__device__ void split_thread(const SubArgs& S, const SubSmem& L, const Queues& Q, int4 e, int gfirst,
                             int& depth_max) {
  const int lf = e.x, cnt = e.y, cell = e.z, depth = e.w;
  const BuildArgs& A = S.A;
  const Sum4 v = thread_pairwise(L, lf, cnt);
  long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
  for (int k = 0; k < cnt; ++k) {
    const int q = L.idx[lf + k];
    const long long kx = dkey(L.x[q]), ky = dkey(L.y[q]), kz = dkey(L.z[q]);
    lo[0] = min(lo[0], kx); hi[0] = max(hi[0], kx);
    lo[1] = min(lo[1], ky); hi[1] = max(hi[1], ky);
    lo[2] = min(lo[2], kz); hi[2] = max(hi[2], kz);
  }
  double dlo[3], dhi[3];
  for (int d = 0; d < 3; ++d) { dlo[d] = dunkey(lo[d]); dhi[d] = dunkey(hi[d]); }
  const double M = v.m;
  const double cx = __ddiv_rn(v.x, M), cy = __ddiv_rn(v.y, M), cz = __ddiv_rn(v.z, M);
  const int axis = longest_axis(dlo, dhi);
  const long long ckey = dkey(axis == 0 ? cx : (axis == 1 ? cy : cz));
  const double* sa = axis == 0 ? L.x : (axis == 1 ? L.y : L.z);
  const long long s2 = thread_size2(L, lf, cnt, cx, cy, cz);
  int nl = 0;
  for (int k = 0; k < cnt; ++k) nl += dkey(sa[L.idx[lf + k]]) < ckey;
  if (nl == 0 || nl == cnt) {
    nl = cnt / 2;
    atomicAdd(&A.counters[5], 1);
  } else {
    int l = 0, r = nl;
    for (int k = 0; k < cnt; ++k) {
      const int q = L.idx[lf + k];
      L.scr[lf + (dkey(sa[q]) < ckey ? l++ : r++)] = (uint16_t)q;
    }
    for (int k = 0; k < cnt; ++k) L.idx[lf + k] = L.scr[lf + k];
  }
  TmpCells t = A.tmp;
  t.first[cell] = gfirst + lf; t.count[cell] = cnt; t.depth[cell] = depth;
  t.M[cell] = M; t.cx[cell] = cx; t.cy[cell] = cy; t.cz[cell] = cz;
  t.s[cell] = sqrt(__longlong_as_double(s2));
  const int cid = atomicAdd(&A.counters[0], 2);
  if (cid + 2 > A.cap_cells) {
    set_status(A.status, ST_CAPACITY);
    return;
  }
  t.left[cell] = cid;
  t.right[cell] = cid + 1;
  depth_max = max(depth_max, depth + 1);
  const int clf[2] = {lf, lf + nl}, ccnt[2] = {nl, cnt - nl};
  for (int side = 0; side < 2; ++side) {
    if (ccnt[side] > Q.n_leaf) {
      int pos = atomicAdd(Q.qn_next, 1);
      if (pos < S.qcap) Q.q_next[pos] = make_int4(clf[side], ccnt[side], cid + side, depth + 1);
      else set_status(A.status, ST_CAPACITY);
    } else {
      leaf_thread(S, L, clf[side], ccnt[side], cid + side, depth + 1, gfirst);
    }
  }
}

// A segment split by one warp.
__device__ void split_warp(const SubArgs& S, const SubSmem& L, const Queues& Q, int4 e, int gfirst,
                           int& depth_max) {
  const int lane = threadIdx.x & 31;
  const int lf = e.x, cnt = e.y, cell = e.z, depth = e.w;
  const BuildArgs& A = S.A;
  auto get = [&](int k) {
    int qq = L.idx[lf + k];
    return elem4(L.m[qq], L.x[qq], L.y[qq], L.z[qq]);
  };
  Sum4 v = warp_pairwise(cnt, get);
  long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
  for (int k = lane; k < cnt; k += 32) {
    int qq = L.idx[lf + k];
    long long kx = dkey(L.x[qq]), ky = dkey(L.y[qq]), kz = dkey(L.z[qq]);
    lo[0] = min(lo[0], kx); hi[0] = max(hi[0], kx);
    lo[1] = min(lo[1], ky); hi[1] = max(hi[1], ky);
    lo[2] = min(lo[2], kz); hi[2] = max(hi[2], kz);
  }
  double dlo[3], dhi[3];
  for (int d = 0; d < 3; ++d) { dlo[d] = dunkey(warp_min_ll(lo[d])); dhi[d] = dunkey(warp_max_ll(hi[d])); }
  const double M = v.m;
  // the three divisions run once, on lanes 0, 1, 2
  const double quo = __ddiv_rn(lane == 1 ? v.y : (lane == 2 ? v.z : v.x), M);
  const double cx = __shfl_sync(0xffffffffu, quo, 0), cy = __shfl_sync(0xffffffffu, quo, 1),
               cz = __shfl_sync(0xffffffffu, quo, 2);
  const int axis = longest_axis(dlo, dhi);
  const long long ckey = dkey(axis == 0 ? cx : (axis == 1 ? cy : cz));
  const double* sa = axis == 0 ? L.x : (axis == 1 ? L.y : L.z);
  // size: float32 filter, then exact float64 for the candidates
  const float cxf = (float)cx, cyf = (float)cy, czf = (float)cz, X = abs_bound(dlo, dhi);
  float d2m = 0.0f;
  int nl = 0;
  for (int k = lane; k < cnt; k += 32) {
    int qq = L.idx[lf + k];
    d2m = fmaxf(d2m, dist2_f(L, qq, cxf, cyf, czf));
    nl += dkey(sa[qq]) < ckey;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d2m = fmaxf(d2m, __shfl_xor_sync(0xffffffffu, d2m, o));
    nl += __shfl_xor_sync(0xffffffffu, nl, o);
  }
  const float Dm = sqrtf(d2m);
  const float thr = Dm - 2.0f * dist_err_bound(X, Dm);
  const float thr2 = thr > 0.0f ? thr * thr * (1.0f - 1e-6f) : -1.0f;
  long long s2 = 0;
  for (int k = lane; k < cnt; k += 32) {
    int qq = L.idx[lf + k];
    if (dist2_f(L, qq, cxf, cyf, czf) >= thr2)
      s2 = max(s2, __double_as_longlong(dist2_rn(L.x[qq], L.y[qq], L.z[qq], cx, cy, cz)));
  }
  s2 = warp_max_ll(s2);
  const bool fallback = (nl == 0 || nl == cnt);
  if (fallback) {
    nl = cnt / 2;
    if (lane == 0) atomicAdd(&A.counters[5], 1);
  } else {
    int offl = 0, offr = nl;
    for (int base = 0; base < cnt; base += 32) {
      int k = base + lane;
      bool valid = k < cnt;
      int qq = valid ? L.idx[lf + k] : 0;
      bool f = valid && dkey(sa[qq]) < ckey;
      unsigned ml = __ballot_sync(0xffffffffu, f);
      unsigned mr = __ballot_sync(0xffffffffu, valid && !f);
      unsigned lt = (1u << lane) - 1u;
      if (valid) L.scr[lf + (f ? offl + __popc(ml & lt) : offr + __popc(mr & lt))] = (uint16_t)qq;
      offl += __popc(ml);
      offr += __popc(mr);
    }
    __syncwarp();
    for (int k = lane; k < cnt; k += 32) L.idx[lf + k] = L.scr[lf + k];
    __syncwarp();
  }
  if (lane == 0) {
    TmpCells t = A.tmp;
    t.first[cell] = gfirst + lf; t.count[cell] = cnt; t.depth[cell] = depth;
    t.M[cell] = M; t.cx[cell] = cx; t.cy[cell] = cy; t.cz[cell] = cz;
    t.s[cell] = sqrt(__longlong_as_double(s2));
  }
  if (make_children(S, Q, lf, cnt, nl, cell, depth)) depth_max = max(depth_max, depth + 1);
}

// Block-wide helpers (all kSubtreeThreads threads call them).
struct BlockScratch {
  Sum4 ws[kSubWarps];
  long long wk[kSubWarps][6];
  float wf[kSubWarps];
  int wi[kSubWarps];
  double com[3];
  double bb[6];
  float thr2;
  int nl;
  int axis;
};

// A segment split by the whole CTA.  The pairwise sum splits the padded
// sequence into kSubWarps aligned sub-blocks, one per warp (the top levels of
// the same perfect tree).
__device__ void split_block(const SubArgs& S, const SubSmem& L, BlockScratch& B, const Queues& Q,
                            int4 e, int gfirst, int& depth_max) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int lf = e.x, cnt = e.y, cell = e.z, depth = e.w;
  const BuildArgs& A = S.A;
  int P = 1;
  while (P < cnt) P <<= 1;                         // P >= kBlockSeg
  const int Pw = P / kSubWarps;                    // per warp, >= 32
  const int base = w * Pw + lane * (Pw >> 5);
  auto get = [&](int k) {
    int qq = L.idx[lf + k];
    return elem4(L.m[qq], L.x[qq], L.y[qq], L.z[qq]);
  };
  Sum4 v;
  switch (Pw >> 5) {
    case 1: v = block_tree<0>(base, cnt, get); break;
    case 2: v = block_tree<1>(base, cnt, get); break;
    case 4: v = block_tree<2>(base, cnt, get); break;
    default: v = block_tree<3>(base, cnt, get); break;
  }
  v = warp_tree4(v);
  long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
  for (int k = threadIdx.x; k < cnt; k += kSubtreeThreads) {
    int qq = L.idx[lf + k];
    long long kx = dkey(L.x[qq]), ky = dkey(L.y[qq]), kz = dkey(L.z[qq]);
    lo[0] = min(lo[0], kx); hi[0] = max(hi[0], kx);
    lo[1] = min(lo[1], ky); hi[1] = max(hi[1], ky);
    lo[2] = min(lo[2], kz); hi[2] = max(hi[2], kz);
  }
  for (int d = 0; d < 3; ++d) { lo[d] = warp_min_ll(lo[d]); hi[d] = warp_max_ll(hi[d]); }
  if (lane == 0) {
    B.ws[w] = v;
    for (int d = 0; d < 3; ++d) { B.wk[w][d] = lo[d]; B.wk[w][3 + d] = hi[d]; }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    Sum4 t = add4(add4(add4(B.ws[0], B.ws[1]), add4(B.ws[2], B.ws[3])),
                  add4(add4(B.ws[4], B.ws[5]), add4(B.ws[6], B.ws[7])));
    double dlo[3], dhi[3];
    for (int d = 0; d < 3; ++d) {
      long long l = B.wk[0][d], h = B.wk[0][3 + d];
      for (int q = 1; q < kSubWarps; ++q) { l = min(l, B.wk[q][d]); h = max(h, B.wk[q][3 + d]); }
      dlo[d] = dunkey(l);
      dhi[d] = dunkey(h);
    }
    B.com[0] = t.x; B.com[1] = t.y; B.com[2] = t.z; B.bb[0] = t.m;
    B.axis = longest_axis(dlo, dhi);
  }
  __syncthreads();
  if (w == 0) {                                    // the three divisions on lanes 0, 1, 2
    const double quo = __ddiv_rn(B.com[lane < 3 ? lane : 0], B.bb[0]);
    const double Mc = B.bb[0];
    __syncwarp();
    if (lane < 3) B.com[lane] = quo;
    if (lane == 0) {
      TmpCells tc = A.tmp;
      tc.first[cell] = gfirst + lf; tc.count[cell] = cnt; tc.depth[cell] = depth;
      tc.M[cell] = Mc; tc.cx[cell] = quo;
    }
    const double qy = __shfl_sync(0xffffffffu, quo, 1), qz = __shfl_sync(0xffffffffu, quo, 2);
    if (lane == 0) { A.tmp.cy[cell] = qy; A.tmp.cz[cell] = qz; }
  }
  __syncthreads();
  const double cx = B.com[0], cy = B.com[1], cz = B.com[2];
  const int axis = B.axis;
  const long long ckey = dkey(B.com[axis]);
  const double* sa = axis == 0 ? L.x : (axis == 1 ? L.y : L.z);
  const float cxf = (float)cx, cyf = (float)cy, czf = (float)cz;
  float d2m = 0.0f;
  int nl = 0;
  for (int k = threadIdx.x; k < cnt; k += kSubtreeThreads) {
    int qq = L.idx[lf + k];
    d2m = fmaxf(d2m, dist2_f(L, qq, cxf, cyf, czf));
    nl += dkey(sa[qq]) < ckey;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d2m = fmaxf(d2m, __shfl_xor_sync(0xffffffffu, d2m, o));
    nl += __shfl_xor_sync(0xffffffffu, nl, o);
  }
  if (lane == 0) { B.wf[w] = d2m; B.wi[w] = nl; }
  __syncthreads();
  if (threadIdx.x == 0) {
    float m2 = 0.0f;
    int t = 0;
    for (int q = 0; q < kSubWarps; ++q) { m2 = fmaxf(m2, B.wf[q]); t += B.wi[q]; }
    double blo[3], bhi[3];
    for (int d = 0; d < 3; ++d) {
      long long l = B.wk[0][d], h = B.wk[0][3 + d];
      for (int q = 1; q < kSubWarps; ++q) { l = min(l, B.wk[q][d]); h = max(h, B.wk[q][3 + d]); }
      blo[d] = dunkey(l);
      bhi[d] = dunkey(h);
    }
    const float Dm = sqrtf(m2);
    const float thr = Dm - 2.0f * dist_err_bound(abs_bound(blo, bhi), Dm);
    B.thr2 = thr > 0.0f ? thr * thr * (1.0f - 1e-6f) : -1.0f;
    B.nl = t;
  }
  __syncthreads();
  const float thr2 = B.thr2;
  nl = B.nl;
  long long s2 = 0;
  for (int k = threadIdx.x; k < cnt; k += kSubtreeThreads) {
    int qq = L.idx[lf + k];
    if (dist2_f(L, qq, cxf, cyf, czf) >= thr2)
      s2 = max(s2, __double_as_longlong(dist2_rn(L.x[qq], L.y[qq], L.z[qq], cx, cy, cz)));
  }
  s2 = warp_max_ll(s2);
  __syncthreads();                                 // B.wk reused below
  if (lane == 0) B.wk[w][0] = s2;
  const bool fallback = (nl == 0 || nl == cnt);
  if (!fallback) {
    // stable partition in rounds of one element per thread
    int offl = 0;
    for (int r0 = 0; r0 < cnt; r0 += kSubtreeThreads) {
      const int k = r0 + threadIdx.x;
      const bool valid = k < cnt;
      const int qq = valid ? L.idx[lf + k] : 0;
      const bool f = valid && dkey(sa[qq]) < ckey;
      const unsigned ml = __ballot_sync(0xffffffffu, f);
      if (lane == 0) B.wi[w] = __popc(ml);
      __syncthreads();
      int woff = 0, tot = 0;
      for (int q = 0; q < kSubWarps; ++q) {
        if (q < w) woff += B.wi[q];
        tot += B.wi[q];
      }
      if (valid) {
        const int lb = offl + woff + __popc(ml & ((1u << lane) - 1u));
        L.scr[lf + (f ? lb : nl + (k - lb))] = (uint16_t)qq;
      }
      offl += tot;
      __syncthreads();
    }
    for (int k = threadIdx.x; k < cnt; k += kSubtreeThreads) L.idx[lf + k] = L.scr[lf + k];
  }
  __syncthreads();
  if (w == 0) {
    long long m2 = lane < kSubWarps ? B.wk[lane][0] : 0;
    m2 = warp_max_ll(m2);
    if (lane == 0) A.tmp.s[cell] = sqrt(__longlong_as_double(m2));
    if (fallback) {
      nl = cnt / 2;
      if (lane == 0) atomicAdd(&A.counters[5], 1);
    }
    if (make_children(S, Q, lf, cnt, nl, cell, depth)) depth_max = max(depth_max, depth + 1);
  }
  __syncthreads();
}

__global__ void __launch_bounds__(kSubtreeThreads)
k_subtree(SubArgs S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ BlockScratch B;
  __shared__ int qn[2];
  __shared__ int nleaf;
  SubSmem L;
  L.x = reinterpret_cast<double*>(smem_raw);
  L.y = L.x + kSubtreeMax;
  L.z = L.y + kSubtreeMax;
  L.m = L.z + kSubtreeMax;
  L.xf = reinterpret_cast<float*>(L.m + kSubtreeMax);
  L.yf = L.xf + kSubtreeMax;
  L.zf = L.yf + kSubtreeMax;
  L.idx = reinterpret_cast<uint16_t*>(L.zf + kSubtreeMax);
  L.scr = L.idx + kSubtreeMax;
  L.q[0] = reinterpret_cast<int4*>(L.scr + kSubtreeMax);
  L.q[1] = L.q[0] + S.qcap;
  int4* leaves = L.q[1] + S.qcap;
  const int leafcap = 2 * S.qcap;

  // persistent: the CTA takes segments from a work counter until none is left
  __shared__ int s_seg;
  const int nB = min(S.A.counters[C_NB], (int)S.A.capB);
  for (;;) {
  __syncthreads();
  if (threadIdx.x == 0) s_seg = atomicAdd(&S.A.counters[C_WORK], 1);
  __syncthreads();
  if (s_seg >= nB) break;
  const Seg g = S.segB[s_seg];
  const PCols in = (g.dbuf & 1) ? S.buf1 : S.buf0;
  const int n = g.count;
  const int gfirst = g.first;
  const int n_leaf = nleaf_at(S.A, gfirst);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    const double x = in.x[gfirst + k], y = in.y[gfirst + k], z = in.z[gfirst + k];
    L.x[k] = x; L.y[k] = y; L.z[k] = z;
    L.m[k] = in.m[gfirst + k];
    L.xf[k] = trunc_to_float(x); L.yf[k] = trunc_to_float(y); L.zf[k] = trunc_to_float(z);
    L.idx[k] = (uint16_t)k;
  }
  int cur = 0;
  if (threadIdx.x == 0) {
    L.q[0][0] = make_int4(0, n, g.cell, g.dbuf >> 1);
    qn[0] = 1;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  int depth_max = 0;
  while (qn[cur] > 0) {
    const int nxt = cur ^ 1;
    if (threadIdx.x == 0) { qn[nxt] = 0; nleaf = 0; }
    __syncthreads();
    const int nq = qn[cur];
    const Queues Q{&qn[nxt], L.q[nxt], &nleaf, leaves, leafcap, n_leaf};
    // large cells: the whole CTA, one after the other
    for (int qi = 0; qi < nq; ++qi) {
      const int4 e = L.q[cur][qi];
      if (e.y >= kBlockSeg) split_block(S, L, B, Q, e, gfirst, depth_max);
    }
    // medium cells: one warp each
    for (int qi = warp; qi < nq; qi += nwarps) {
      const int4 e = L.q[cur][qi];
      if (e.y > kThreadSeg && e.y < kBlockSeg) split_warp(S, L, Q, e, gfirst, depth_max);
    }
    // small cells: one thread each (with their leaf children)
    for (int qi = threadIdx.x; qi < nq; qi += blockDim.x) {
      const int4 e = L.q[cur][qi];
      if (e.y <= kThreadSeg) split_thread(S, L, Q, e, gfirst, depth_max);
    }
    __syncthreads();
    // leaves split off by the CTA and warp passes: one thread each
    const int nlv = min(nleaf, leafcap);
    for (int li = threadIdx.x; li < nlv; li += blockDim.x) {
      const int4 e = leaves[li];
      leaf_thread(S, L, e.x, e.y, e.z, e.w, gfirst);
    }
    __syncthreads();
    cur ^= 1;
  }
  depth_max = max(depth_max, __shfl_xor_sync(0xffffffffu, depth_max, 16));
  depth_max = max(depth_max, __shfl_xor_sync(0xffffffffu, depth_max, 8));
  depth_max = max(depth_max, __shfl_xor_sync(0xffffffffu, depth_max, 4));
  depth_max = max(depth_max, __shfl_xor_sync(0xffffffffu, depth_max, 2));
  depth_max = max(depth_max, __shfl_xor_sync(0xffffffffu, depth_max, 1));
  if ((threadIdx.x & 31) == 0 && depth_max > 0) atomicMax(&S.A.counters[6], depth_max);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    int src = L.idx[k];
    int64_t p = (int64_t)gfirst + k;
    S.out.x[p] = L.x[src]; S.out.y[p] = L.y[src]; S.out.z[p] = L.z[src]; S.out.m[p] = L.m[src];
    S.out.h[p] = in.h[gfirst + src];
    S.out.idx[p] = in.idx[gfirst + src];
  }
  }
}

// Leaves produced directly by phase A (or a root that is already a leaf): one
// thread per leaf, pairwise sums by a carry stack.
__global__ void k_leaf_segs(SubArgs S, const Seg* __restrict__ segL) {
  const int nL = min(S.A.counters[C_NL], (int)S.A.capL);
  KD_GRID_STRIDE(sidx, nL) {
  const Seg g = segL[sidx];
  const PCols in = (g.dbuf & 1) ? S.buf1 : S.buf0;
  const int cnt = g.count;
  int P = 1;
  while (P < cnt) P <<= 1;
  Sum4 st[8];
  int top = 0;
  for (int k = 0; k < P; ++k) {
    Sum4 e = zero4();
    if (k < cnt) {
      const int64_t i = (int64_t)g.first + k;
      e = elem4(in.m[i], in.x[i], in.y[i], in.z[i]);
    }
    for (int kk = k; kk & 1; kk >>= 1) e = add4(st[--top], e);
    st[top++] = e;
  }
  const Sum4 v = st[0];
  const double M = v.m;
  const double cx = __ddiv_rn(v.x, M), cy = __ddiv_rn(v.y, M), cz = __ddiv_rn(v.z, M);
  long long s2 = 0;
  for (int k = 0; k < cnt; ++k) {
    const int64_t i = (int64_t)g.first + k;
    s2 = max(s2, __double_as_longlong(dist2_rn(in.x[i], in.y[i], in.z[i], cx, cy, cz)));
    S.out.x[i] = in.x[i]; S.out.y[i] = in.y[i]; S.out.z[i] = in.z[i];
    S.out.m[i] = in.m[i]; S.out.h[i] = in.h[i]; S.out.idx[i] = in.idx[i];
  }
  TmpCells t = S.A.tmp;
  const int c = g.cell;
  t.first[c] = g.first; t.count[c] = cnt; t.depth[c] = g.dbuf >> 1;
  t.M[c] = M; t.cx[c] = cx; t.cy[c] = cy; t.cz[c] = cz;
  t.s[c] = sqrt(__longlong_as_double(s2));
  t.left[c] = -1; t.right[c] = -1;
  }
}

// ---------------------------------------------------------------------------
// pre-order numbering: a cell's id is the number of cells starting before its
// first particle plus its depth below the topmost cell starting there.
// ---------------------------------------------------------------------------
__global__ void k_fill2(int32_t* a, int32_t va, int32_t* b, int32_t vb, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) { a[i] = va; b[i] = vb; }
}

__global__ void k_count_starts(TmpCells tmp, const int32_t* __restrict__ counters,
                               int32_t* cnt_start, int32_t* min_depth) {
  const int ncells = counters[C_CELLS];
  KD_GRID_STRIDE(c, ncells) {
    const int f = tmp.first[c];
    atomicAdd(&cnt_start[f], 1);
    atomicMin(&min_depth[f], tmp.depth[c]);
  }
}

__device__ __forceinline__ int preorder_id(const int32_t* start_off, const int32_t* min_depth,
                                           int first, int depth) {
  return start_off[first] + depth - min_depth[first];
}

__global__ void k_remap(TmpCells tmp, const int32_t* __restrict__ counters, const int32_t* __restrict__ start_off,
                        const int32_t* __restrict__ min_depth, Cells c, int32_t* status) {
  const int t_n = counters[C_CELLS];
  KD_GRID_STRIDE(t, t_n) {
  const int f = tmp.first[t], cnt = tmp.count[t], d = tmp.depth[t];
  const int id = preorder_id(start_off, min_depth, f, d);
  c.first[id] = f; c.count[id] = cnt; c.depth[id] = d;
  c.skip[id] = start_off[f + cnt];
  c.M[id] = tmp.M[t]; c.cx[id] = tmp.cx[t]; c.cy[id] = tmp.cy[t]; c.cz[id] = tmp.cz[t];
  c.s[id] = tmp.s[t];
  const int lt = tmp.left[t];
  if (lt >= 0) {
    const int rt = tmp.right[t];
    const int idl = preorder_id(start_off, min_depth, tmp.first[lt], tmp.depth[lt]);
    const int idr = preorder_id(start_off, min_depth, tmp.first[rt], tmp.depth[rt]);
    if (idl != id + 1) atomicOr(status, ST_INTERNAL);
    c.left[id] = idl; c.right[id] = idr;
    c.parent[idl] = id; c.parent[idr] = id;
  } else {
    c.left[id] = -1; c.right[id] = -1;
  }
  if (d == 0) c.parent[id] = -1;               // a system's root
  }
}

// Pre-order id of each system's root; sys_root[n_sys] = number of cells.
__global__ void k_sys_roots(const int64_t* __restrict__ sys_off, int n_sys,
                            const int32_t* __restrict__ start_off, int32_t* sys_root) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k <= n_sys) sys_root[k] = start_off[sys_off[k]];
}

// Leaves: h_max and Q (Eq. 7) from their particles (one thread per leaf);
// then each parent, once its second child has finished, from its children
// (parallel-axis shift of Q).  Every sum runs in a fixed order.
__global__ void k_upward(Cells c, const int32_t* __restrict__ leaf_cells, const int32_t* __restrict__ counters, PCols tp) {
  const int k_n = counters[C_LEAVES];
  KD_GRID_STRIDE(k, k_n) {
  const int t = leaf_cells[k];
  double q[6], hm = 0.0;
  {
    // S_jk = sum m y_j y_k (9 float64 operations a particle), then
    // Q = 3 S - tr(S) I (Eq. 7) once for the leaf
    const int f = c.first[t], cnt = c.count[t];
    const double cx = c.cx[t], cy = c.cy[t], cz = c.cz[t];
    double S[6] = {0, 0, 0, 0, 0, 0};
    for (int j = 0; j < cnt; ++j) {
      const int64_t i = (int64_t)f + j;
      const double m = tp.m[i];
      const double y0 = tp.x[i] - cx, y1 = tp.y[i] - cy, y2 = tp.z[i] - cz;
      const double my0 = m * y0, my1 = m * y1, my2 = m * y2;
      S[0] = fma(my0, y0, S[0]); S[1] = fma(my0, y1, S[1]); S[2] = fma(my0, y2, S[2]);
      S[3] = fma(my1, y1, S[3]); S[4] = fma(my1, y2, S[4]); S[5] = fma(my2, y2, S[5]);
      hm = fmax(hm, tp.h[i]);
    }
    const double tr = S[0] + S[3] + S[5];
    q[0] = 3.0 * S[0] - tr; q[1] = 3.0 * S[1]; q[2] = 3.0 * S[2];
    q[3] = 3.0 * S[3] - tr; q[4] = 3.0 * S[4]; q[5] = 3.0 * S[5] - tr;
  }
  for (int j = 0; j < 6; ++j) c.Q[6 * t + j] = q[j];
  c.hmax[t] = hm;
  int cur = t;
  while (true) {
    const int p = c.parent[cur];
    if (p < 0) break;
    __threadfence();
    if (atomicAdd(&c.ready[p], 1) == 0) break;      // the sibling finishes the parent
    __threadfence();
    const double px = c.cx[p], py = c.cy[p], pz = c.cz[p];
    double qp[6] = {0, 0, 0, 0, 0, 0}, hp = 0.0;
    const int ch[2] = {c.left[p], c.right[p]};
    for (int side = 0; side < 2; ++side) {
      // parallel-axis shift of the child's Q to the parent's centre of mass:
      // + M (3 d d - |d|^2 I)
      const int kc = ch[side];
      const double mk = c.M[kc];
      const double d0 = c.cx[kc] - px, d1 = c.cy[kc] - py, d2 = c.cz[kc] - pz;
      const double m0 = 3.0 * mk * d0, m1 = 3.0 * mk * d1;
      const double mdd = mk * (d0 * d0 + d1 * d1 + d2 * d2);
      qp[0] += __ldcg(&c.Q[6 * kc + 0]) + fma(m0, d0, -mdd);
      qp[1] += __ldcg(&c.Q[6 * kc + 1]) + m0 * d1;
      qp[2] += __ldcg(&c.Q[6 * kc + 2]) + m0 * d2;
      qp[3] += __ldcg(&c.Q[6 * kc + 3]) + fma(m1, d1, -mdd);
      qp[4] += __ldcg(&c.Q[6 * kc + 4]) + m1 * d2;
      qp[5] += __ldcg(&c.Q[6 * kc + 5]) + fma(3.0 * mk * d2, d2, -mdd);
      hp = fmax(hp, __ldcg(&c.hmax[kc]));
    }
    for (int j = 0; j < 6; ++j) c.Q[6 * p + j] = qp[j];
    c.hmax[p] = hp;
    cur = p;
  }
  }
}

__global__ void k_leaf_flags(const Cells c, const int32_t* __restrict__ counters, int32_t* flag) {
  const int t_n = counters[C_CELLS];
  KD_GRID_STRIDE(t, t_n) flag[t] = c.left[t] < 0 ? 1 : 0;
}

// float32 views of the cells.
__global__ void k_derive_cells(Cells c, const int32_t* __restrict__ counters, float* com_bound) {
  const int t_n = counters[C_CELLS];
  KD_GRID_STRIDE(t, t_n) {
  const double cx = c.cx[t], cy = c.cy[t], cz = c.cz[t];
  c.walk[t] = make_float4((float)cx, (float)cy, (float)cz, (float)c.s[t]);
  c.walk2[t] = make_float4((float)c.hmax[t], __int_as_float(c.skip[t]), __int_as_float(c.count[t]),
                          0.0f);
  const float hx = (float)cx, hy = (float)cy, hz = (float)cz;
  c.src32[4 * t + 0] = make_float4(hx, hy, hz, (float)c.M[t]);
  c.src32[4 * t + 1] = make_float4((float)(cx - (double)hx), (float)(cy - (double)hy),
                                   (float)(cz - (double)hz), 0.0f);
  c.src32[4 * t + 2] = make_float4((float)c.Q[6 * t + 0], (float)c.Q[6 * t + 1],
                                   (float)c.Q[6 * t + 2], (float)c.Q[6 * t + 3]);
  c.src32[4 * t + 3] = make_float4((float)c.Q[6 * t + 4], (float)c.Q[6 * t + 5], 0.0f, 0.0f);
  double* s64 = c.src64 + 10 * (int64_t)t;
  s64[0] = cx; s64[1] = cy; s64[2] = cz; s64[3] = c.M[t];
  for (int k = 0; k < 6; ++k) s64[4 + k] = c.Q[6 * t + k];
  float b = fmaxf(fabsf((float)cx), fmaxf(fabsf((float)cy), fabsf((float)cz)));
  atomicMax(reinterpret_cast<int*>(com_bound), __float_as_int(b));
  }
}

// Leaf ordinal -> cell and system; the leaf count goes to counters[C_LEAVES].
__global__ void k_leaf_list(const Cells c, int32_t* counters, int32_t* leaf_rank,
                            int32_t* leaf_cells, const int64_t* __restrict__ sys_off, int n_sys,
                            int32_t* leaf_sys) {
  const int t_n = counters[C_CELLS];
  if (blockIdx.x == 0 && threadIdx.x == 0) counters[C_LEAVES] = leaf_rank[t_n];
  KD_GRID_STRIDE(t, t_n) {
  if (c.left[t] < 0) {
    const int r = leaf_rank[t];
    leaf_cells[r] = t;
    leaf_sys[r] = system_of(sys_off, n_sys, c.first[t]);
  } else {
    leaf_rank[t] = -1;
  }
  }
}

// Per-particle float32 data relative to the centre of mass of its leaf.
__global__ void k_particles32(const Cells c, const int32_t* __restrict__ leaf_cells,
                              const int32_t* __restrict__ counters, PCols tp, float4* pf,
                              float4* ph) {
  const int nleaves = counters[C_LEAVES];
  const int lane = threadIdx.x & 31;
  const int w0 = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
  const int nw = (int)((gridDim.x * blockDim.x) >> 5);
  for (int k = w0; k < nleaves; k += nw) {
    const int cell = leaf_cells[k];
    const int f = c.first[cell], cnt = c.count[cell];
    if (lane >= cnt) continue;
    const int64_t i = (int64_t)f + lane;
    pf[i] = make_float4((float)(tp.x[i] - c.cx[cell]), (float)(tp.y[i] - c.cy[cell]),
                        (float)(tp.z[i] - c.cz[cell]), (float)tp.m[i]);
    const float h = (float)tp.h[i];
    const float hi = h > 0.0f ? 1.0f / h : 0.0f;
    ph[i] = make_float4(hi, hi * hi * hi, h, 4.0f * h * h);   // 1/h, 1/h^3, h, (2h)^2
  }
}

inline unsigned blocks_for(int64_t n, int threads) { return (unsigned)((n + threads - 1) / threads); }

}  // namespace

// ---------------------------------------------------------------------------
// host orchestration
// ---------------------------------------------------------------------------
static int alloc_cols(PCols* c, int64_t n) {
  if (cudaMalloc(&c->x, n * sizeof(double)) != cudaSuccess) return -1;
  if (cudaMalloc(&c->y, n * sizeof(double)) != cudaSuccess) return -1;
  if (cudaMalloc(&c->z, n * sizeof(double)) != cudaSuccess) return -1;
  if (cudaMalloc(&c->m, n * sizeof(double)) != cudaSuccess) return -1;
  if (cudaMalloc(&c->h, n * sizeof(double)) != cudaSuccess) return -1;
  if (cudaMalloc(&c->idx, n * sizeof(int32_t)) != cudaSuccess) return -1;
  return 0;
}
static void free_cols(PCols* c) {
  cudaFree(c->x); cudaFree(c->y); cudaFree(c->z); cudaFree(c->m); cudaFree(c->h); cudaFree(c->idx);
  *c = PCols{};
}

void free_build_buffers(kdfmm_tree_s* t) {
  for (int k = 0; k < 2; ++k) { free_cols(&t->buf[k]); cudaFree(t->segA[k]); t->segA[k] = nullptr; }
  free_cols(&t->tp);
  void* ptrs[] = {t->segB, t->segL, t->chunk_seg, t->seg_chunk_off, t->chunk_sum, t->chunk_key,
                  t->chunk_left, t->chunk_loff, t->chunk_s2, t->seg_axis, t->seg_cut, t->seg_nl,
                  t->seg_xb, t->seg_thr2, t->seg_s2,
                  t->tmp.first, t->tmp.count, t->tmp.left, t->tmp.right, t->tmp.depth, t->tmp.M,
                  t->tmp.cx, t->tmp.cy, t->tmp.cz, t->tmp.s, t->cnt_start, t->min_depth,
                  t->start_off, t->scan_tmp, t->pf, t->ph, t->c.first, t->c.count, t->c.left,
                  t->c.right, t->c.parent, t->c.skip, t->c.depth, t->c.M, t->c.cx, t->c.cy,
                  t->c.cz, t->c.s, t->c.hmax, t->c.Q, t->c.walk, t->c.walk2, t->c.src32,
                  t->c.src64, t->c.ready, t->leaf_cells, t->leaf_rank, t->leaf_sys, t->lexp64,
                  t->lexp32};
  for (void* p : ptrs) cudaFree(p);
  t->segB = t->segL = nullptr;
  t->chunk_seg = t->seg_chunk_off = t->chunk_left = t->chunk_loff = t->seg_axis = t->seg_nl = nullptr;
  t->chunk_sum = t->seg_cut = nullptr;
  t->chunk_key = nullptr;
  t->chunk_s2 = t->seg_xb = t->seg_thr2 = nullptr;
  t->seg_s2 = nullptr;
  t->tmp = TmpCells{};
  t->cnt_start = t->min_depth = t->start_off = t->scan_tmp = nullptr;
  t->pf = t->ph = nullptr;
  t->c = Cells{};
  t->leaf_cells = t->leaf_rank = t->leaf_sys = nullptr;
  t->lexp64 = nullptr;
  t->lexp32 = nullptr;
  t->cap_n = 0;
}

#define KD_ALLOC(ptr, count)                                                        \
  do {                                                                              \
    if (cudaMalloc((void**)&(ptr), (size_t)(count) * sizeof(*(ptr))) != cudaSuccess) \
      return set_error(KDFMM_ERR_OOM, "device allocation of %s failed", #ptr);      \
  } while (0)

static int ensure_build_buffers(kdfmm_tree_s* t, int64_t n) {
  if (t->cap_n >= n) return KDFMM_OK;
  cudaDeviceSynchronize();
  free_build_buffers(t);
  cudaGetLastError();
  for (int k = 0; k < 2; ++k)
    if (alloc_cols(&t->buf[k], n)) return set_error(KDFMM_ERR_OOM, "particle buffers");
  if (alloc_cols(&t->tp, n)) return set_error(KDFMM_ERR_OOM, "tree-order particles");
  t->capA = n / kSubtreeMax + 4;
  t->capB = n / 2 + 4;
  t->capL = n / 4 + 64;
  KD_ALLOC(t->segA[0], t->capA);
  KD_ALLOC(t->segA[1], t->capA);
  KD_ALLOC(t->segB, t->capB);
  KD_ALLOC(t->segL, t->capL);
  t->cap_chunks = n / kChunk + t->capA + 4;
  KD_ALLOC(t->chunk_seg, t->cap_chunks);
  KD_ALLOC(t->chunk_sum, 4 * t->cap_chunks);
  KD_ALLOC(t->chunk_key, 6 * t->cap_chunks);
  KD_ALLOC(t->chunk_left, t->cap_chunks);
  KD_ALLOC(t->chunk_loff, t->cap_chunks);
  KD_ALLOC(t->chunk_s2, t->cap_chunks);
  KD_ALLOC(t->seg_chunk_off, t->capA);
  KD_ALLOC(t->seg_axis, t->capA);
  KD_ALLOC(t->seg_cut, t->capA);
  KD_ALLOC(t->seg_nl, t->capA);
  KD_ALLOC(t->seg_xb, t->capA);
  KD_ALLOC(t->seg_thr2, t->capA);
  KD_ALLOC(t->seg_s2, t->capA);
  t->cap_cells = 2 * n + 2;
  const int64_t nc = t->cap_cells;
  KD_ALLOC(t->tmp.first, nc); KD_ALLOC(t->tmp.count, nc); KD_ALLOC(t->tmp.left, nc);
  KD_ALLOC(t->tmp.right, nc); KD_ALLOC(t->tmp.depth, nc); KD_ALLOC(t->tmp.M, nc);
  KD_ALLOC(t->tmp.cx, nc); KD_ALLOC(t->tmp.cy, nc); KD_ALLOC(t->tmp.cz, nc); KD_ALLOC(t->tmp.s, nc);
  KD_ALLOC(t->cnt_start, n + 2);
  KD_ALLOC(t->min_depth, n + 2);
  KD_ALLOC(t->start_off, n + 2);
  t->cap_scan = scan_tmp_elems(nc > n + 2 ? nc : n + 2) * 2 + 16;
  KD_ALLOC(t->scan_tmp, t->cap_scan);
  KD_ALLOC(t->pf, n);
  KD_ALLOC(t->ph, n);
  Cells& c = t->c;
  KD_ALLOC(c.first, nc); KD_ALLOC(c.count, nc); KD_ALLOC(c.left, nc); KD_ALLOC(c.right, nc);
  KD_ALLOC(c.parent, nc); KD_ALLOC(c.skip, nc); KD_ALLOC(c.depth, nc);
  KD_ALLOC(c.M, nc); KD_ALLOC(c.cx, nc); KD_ALLOC(c.cy, nc); KD_ALLOC(c.cz, nc);
  KD_ALLOC(c.s, nc); KD_ALLOC(c.hmax, nc); KD_ALLOC(c.Q, 6 * nc);
  KD_ALLOC(c.walk, nc); KD_ALLOC(c.walk2, nc); KD_ALLOC(c.src32, 4 * nc); KD_ALLOC(c.src64, 10 * nc);
  KD_ALLOC(c.ready, nc);
  KD_ALLOC(t->leaf_cells, nc);
  KD_ALLOC(t->leaf_rank, nc + 1);
  KD_ALLOC(t->leaf_sys, nc);
  KD_ALLOC(t->lexp64, 20 * (n + 1));
  KD_ALLOC(t->lexp32, 24 * (n + 1));
  t->cap_n = n;
  return KDFMM_OK;
}

// Launch sizes of the persistent subtree kernel (host calls only; made once
// per handle and shared-memory size, outside any stream capture).
static int subtree_setup(kdfmm_tree_s* t, size_t smem) {
  if (t->subtree_smem == smem) return KDFMM_OK;
  int rc = check_cuda(cudaFuncSetAttribute(k_subtree, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem),
                      "subtree smem attribute");
  if (rc) return rc;
  int per_sm = 0, sms = 0;
  rc = check_cuda(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_subtree,
                                                                 kSubtreeThreads, smem),
                  "subtree occupancy");
  if (rc) return rc;
  rc = check_cuda(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, t->device), "SMs");
  if (rc) return rc;
  t->subtree_grid = std::max(1, per_sm) * std::max(1, sms);
  t->subtree_smem = smem;
  return KDFMM_OK;
}

// Builds the tree (or forest).  fixed_levels <= 0: the host follows the
// device counters (a synchronisation after the first step, each phase-A
// level, the subtrees and the numbering) and records the number of phase-A
// levels in t->levels_used.  fixed_levels > 0: the same launches with no
// synchronisation -- exactly that many phase-A levels, every launch sized
// from capacities and reading its count on the device -- so the sequence can
// be captured in a CUDA graph; a phase A that needed more levels, or any
// capacity overflow, is left in the status word for the caller to check.
int build_tree(kdfmm_tree_s* t, const double* x, const double* m, const double* h, cudaStream_t s,
               int fixed_levels) {
  const int64_t n = t->n;
  const bool deferred = fixed_levels > 0;
  int rc = ensure_build_buffers(t, n);
  if (rc) return rc;
  const kdfmm_params& P = t->p;
  cudaMemsetAsync(t->counters, 0, 32 * sizeof(int32_t), s);
  cudaMemsetAsync(t->status, 0, sizeof(int32_t), s);
  cudaMemsetAsync(t->com_bound, 0, sizeof(float), s);
  BuildArgs A{};
  A.tmp = t->tmp;
  A.counters = t->counters;
  A.status = t->status;
  A.sys_off = t->sys_off;
  A.sys_nleaf = t->sys_nleaf;
  A.n_sys = t->n_sys;
  A.capA = t->capA; A.capB = t->capB; A.capL = t->capL; A.cap_cells = t->cap_cells;
  k_init<<<blocks_for(n, 256), 256, 0, s>>>(x, m, h, n, t->sys_off, t->n_sys, t->sys_eps,
                                            P.soft_kind, t->buf[0], t->status);
  k_roots<<<blocks_for(t->n_sys, 128), 128, 0, s>>>(A, t->segA[0], t->segB, t->segL);
  t->launches += 2;

  int32_t* hc = t->host_counters;
  auto read_back = [&](const char* what) {
    cudaMemcpyAsync(hc, t->counters, 32 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&hc[32], t->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    return check_cuda(cudaStreamSynchronize(s), what);
  };
  if (!deferred) {
    if ((rc = read_back("build init"))) return rc;
    if (hc[32] & ST_NONFINITE)
      return set_error(KDFMM_ERR_NONFINITE, "non-finite position or non-positive mass / h");
  }
  // phase A: cells above kSubtreeMax, one level per pass
  const unsigned maxc = (unsigned)(n / kChunk + t->capA + 1);
  const unsigned segw = blocks_for(t->capA * 32, 256);
  int cur = 0, level = 0;
  while (deferred ? level < fixed_levels : hc[C_NEXT_A] > 0) {
    const int src = level & 1, dst = src ^ 1;
    A.src = t->buf[src];
    A.dst = t->buf[dst];
    const Seg* segs = t->segA[cur];
    Seg* next = t->segA[cur ^ 1];
    const int32_t* nA = t->counters + C_NA;
    k_level_begin<<<1, 1, 0, s>>>(t->counters, t->capA, t->status);
    k_chunk_map<<<1, 1024, 0, s>>>(segs, nA, t->seg_chunk_off, t->chunk_seg, t->counters);
    k_chunk_reduce<<<maxc, kChunkThreads, 0, s>>>(segs, t->chunk_seg, t->seg_chunk_off, t->counters,
                                                  t->buf[src], t->chunk_sum, t->chunk_key);
    k_decide<<<segw, 256, 0, s>>>(segs, nA, t->seg_chunk_off, t->chunk_sum, t->chunk_key, t->tmp,
                                  t->seg_axis, t->seg_cut, t->seg_xb, t->seg_s2);
    k_chunk_count<<<maxc, kChunkThreads, 0, s>>>(segs, t->chunk_seg, t->seg_chunk_off, t->counters,
                                                 t->buf[src], t->tmp, t->seg_axis, t->seg_cut,
                                                 t->chunk_left, t->chunk_s2);
    k_split<<<segw, 256, 0, s>>>(segs, nA, t->seg_chunk_off, t->chunk_left, t->chunk_s2,
                                 t->chunk_loff, t->seg_nl, t->seg_xb, t->seg_thr2, A, next, t->segB,
                                 t->segL, dst);
    k_chunk_scatter<<<maxc, kChunkThreads, 0, s>>>(segs, t->chunk_seg, t->seg_chunk_off, t->counters,
                                                   t->buf[src], t->buf[dst], t->seg_axis, t->seg_cut,
                                                   t->chunk_loff, t->seg_nl, t->tmp, t->seg_thr2,
                                                   t->seg_s2);
    k_seg_size<<<blocks_for(t->capA, 128), 128, 0, s>>>(segs, nA, t->seg_s2, t->tmp);
    t->launches += 8;
    cur ^= 1;
    ++level;
    if (!deferred) {
      if ((rc = read_back("build level"))) return rc;
      if (hc[32] & ST_CAPACITY) return set_error(KDFMM_ERR_CAPACITY, "segment lists overflow");
      if (level > 200) return set_error(KDFMM_ERR_INTERNAL, "phase A did not terminate");
    }
  }
  if (deferred) {
    k_levels_done<<<1, 1, 0, s>>>(t->counters, t->status);
    t->launches += 1;
  } else {
    t->levels_used = level;
  }

  // phase B: the remaining cells in shared memory, persistent CTAs
  SubArgs S{};
  S.A = A;
  S.buf0 = t->buf[0];
  S.buf1 = t->buf[1];
  S.out = t->tp;
  S.segB = t->segB;
  S.qcap = kSubtreeMax / (t->min_nleaf + 1) + 2;
  const size_t smem = 4 * kSubtreeMax * sizeof(double) + 3 * kSubtreeMax * sizeof(float) +
                      2 * kSubtreeMax * sizeof(uint16_t) + 4 * (size_t)S.qcap * sizeof(int4);
  if ((rc = subtree_setup(t, smem))) return rc;
  const int gsub = deferred ? t->subtree_grid : std::max(1, std::min(t->subtree_grid, hc[C_NB]));
  k_subtree<<<gsub, kSubtreeThreads, smem, s>>>(S);
  k_leaf_segs<<<grid_blocks(2), 128, 0, s>>>(S, t->segL);
  t->launches += 2;
  if (!deferred) {
    if ((rc = read_back("build subtrees"))) return rc;
    if (hc[32] & ST_NONFINITE)
      return set_error(KDFMM_ERR_NONFINITE, "non-finite position or non-positive mass / h");
    if (hc[32] & ST_CAPACITY) return set_error(KDFMM_ERR_CAPACITY, "build capacity exceeded");
    t->ncells = hc[C_CELLS];
    t->nfallback = hc[C_FALLBACK];
    t->depth = hc[C_DEPTH];
  }

  // pre-order numbering, counts read on the device
  k_fill2<<<blocks_for(n + 1, 256), 256, 0, s>>>(t->cnt_start, 0, t->min_depth, INT_MAX, n + 1);
  k_count_starts<<<grid_blocks(), 256, 0, s>>>(t->tmp, t->counters, t->cnt_start, t->min_depth);
  scan_i32(t->cnt_start, t->start_off, n, t->scan_tmp, s);
  k_remap<<<grid_blocks(), 256, 0, s>>>(t->tmp, t->counters, t->start_off, t->min_depth, t->c,
                                      t->status);
  k_leaf_flags<<<grid_blocks(), 256, 0, s>>>(t->c, t->counters, t->c.ready);
  scan_i32_dev(t->c.ready, t->leaf_rank, t->counters + C_CELLS,
               deferred ? t->cap_cells : (int64_t)t->ncells, t->scan_tmp, s);
  k_leaf_list<<<grid_blocks(), 256, 0, s>>>(t->c, t->counters, t->leaf_rank, t->leaf_cells,
                                          t->sys_off, t->n_sys, t->leaf_sys);
  k_sys_roots<<<blocks_for(t->n_sys + 1, 128), 128, 0, s>>>(t->sys_off, t->n_sys, t->start_off,
                                                            t->sys_root);
  if (!deferred) {
    if ((rc = read_back("build finalise"))) return rc;
    t->nleaves = hc[C_LEAVES];
    if (hc[32] & ST_INTERNAL) return set_error(KDFMM_ERR_INTERNAL, "pre-order numbering inconsistent");
  }
  cudaMemsetAsync(t->c.ready, 0,
                  (size_t)(deferred ? t->cap_cells : (int64_t)t->ncells) * sizeof(int32_t), s);
  // one thread per leaf (the climb is latency-bound): the grid follows the last
  // known leaf count with a margin; more leaves than threads loop
  const int64_t up_threads = std::max<int64_t>(t->nleaves, 1) + t->nleaves / 4 + 128;
  k_upward<<<blocks_for(up_threads, 128), 128, 0, s>>>(t->c, t->leaf_cells, t->counters, t->tp);
  k_derive_cells<<<grid_blocks(), 256, 0, s>>>(t->c, t->counters, t->com_bound);
  k_particles32<<<grid_blocks(), 256, 0, s>>>(t->c, t->leaf_cells, t->counters, t->tp, t->pf, t->ph);
  t->launches += 15;
  return check_cuda(cudaGetLastError(), "build launch");
}

// ---------------------------------------------------------------------------
// Frozen topology: new positions / masses / smoothing lengths for the same
// particles, the tree's cells and the last interaction lists kept.  Leaf sums
// are pairwise over the leaf's particles (tree order = ascending caller index
// within a leaf); a parent's M and sum m x are its left child's plus its right
// child's; s is the exact maximum distance; Q the parallel-axis shift.
// ---------------------------------------------------------------------------
namespace {

__global__ void k_gather_frozen(const double* __restrict__ x, const double* __restrict__ m,
                                const double* __restrict__ h, int64_t n,
                                const int64_t* __restrict__ sys_off, int n_sys,
                                const double* __restrict__ sys_eps, int soft_kind, PCols tp,
                                int32_t* status) {
  const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const int64_t i = tp.idx[p];
  const double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2], mi = m[i];
  const double hi = (h != nullptr && soft_kind == KDFMM_SOFT_M4)
                        ? h[i]
                        : sys_eps[system_of(sys_off, n_sys, i)];
  const bool ok = isfinite(xi) && isfinite(yi) && isfinite(zi) && isfinite(mi) && isfinite(hi) &&
                  mi > 0.0 && (soft_kind == KDFMM_SOFT_M4 ? hi > 0.0 : hi >= 0.0);
  if (!ok) atomicOr(status, ST_NONFINITE);
  tp.x[p] = xi; tp.y[p] = yi; tp.z[p] = zi; tp.m[p] = mi; tp.h[p] = hi;
}

// Leaves: pairwise sums (carry stack), centre of mass, exact size, h_max, Q.
__global__ void k_leaf_frozen(Cells c, const int32_t* __restrict__ leaf_cells, int nleaves, PCols tp,
                              double* Sx, double* Sy, double* Sz) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nleaves) return;
  const int t = leaf_cells[k];
  const int f = c.first[t], cnt = c.count[t];
  Sum4 st[8];
  int top = 0;
  for (int j = 0; j < cnt; ++j) {
    const int64_t i = (int64_t)f + j;
    Sum4 e = elem4(tp.m[i], tp.x[i], tp.y[i], tp.z[i]);
    for (int kk = j; kk & 1; kk >>= 1) e = add4(st[--top], e);
    st[top++] = e;
  }
  Sum4 v = st[top - 1];
  for (int i = top - 2; i >= 0; --i) v = add4(st[i], v);
  const double cx = __ddiv_rn(v.x, v.m), cy = __ddiv_rn(v.y, v.m), cz = __ddiv_rn(v.z, v.m);
  long long s2 = 0;
  double q[6] = {0, 0, 0, 0, 0, 0}, hm = 0.0;
  for (int j = 0; j < cnt; ++j) {
    const int64_t i = (int64_t)f + j;
    s2 = max(s2, __double_as_longlong(dist2_rn(tp.x[i], tp.y[i], tp.z[i], cx, cy, cz)));
    const double mi = tp.m[i];
    const double y0 = tp.x[i] - cx, y1 = tp.y[i] - cy, y2 = tp.z[i] - cz;
    const double y2s = y0 * y0 + y1 * y1 + y2 * y2;
    q[0] += mi * (3.0 * y0 * y0 - y2s);
    q[1] += mi * (3.0 * y0 * y1);
    q[2] += mi * (3.0 * y0 * y2);
    q[3] += mi * (3.0 * y1 * y1 - y2s);
    q[4] += mi * (3.0 * y1 * y2);
    q[5] += mi * (3.0 * y2 * y2 - y2s);
    hm = fmax(hm, tp.h[i]);
  }
  c.M[t] = v.m; c.cx[t] = cx; c.cy[t] = cy; c.cz[t] = cz;
  Sx[t] = v.x; Sy[t] = v.y; Sz[t] = v.z;
  c.s[t] = sqrt(__longlong_as_double(s2));
  c.hmax[t] = hm;
  for (int j = 0; j < 6; ++j) c.Q[6 * t + j] = q[j];
}

// Parents from their children, bottom-up (the second child to finish goes on).
__global__ void k_upward_frozen(Cells c, const int32_t* __restrict__ leaf_cells, int nleaves,
                                double* Sx, double* Sy, double* Sz) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= nleaves) return;
  int cur = leaf_cells[k];
  while (true) {
    const int p = c.parent[cur];
    if (p < 0) break;
    __threadfence();
    if (atomicAdd(&c.ready[p], 1) == 0) break;
    __threadfence();
    const int L = c.left[p], R = c.right[p];
    const double M = __dadd_rn(__ldcg(&c.M[L]), __ldcg(&c.M[R]));
    const double sx = __dadd_rn(__ldcg(&Sx[L]), __ldcg(&Sx[R]));
    const double sy = __dadd_rn(__ldcg(&Sy[L]), __ldcg(&Sy[R]));
    const double sz = __dadd_rn(__ldcg(&Sz[L]), __ldcg(&Sz[R]));
    const double px = __ddiv_rn(sx, M), py = __ddiv_rn(sy, M), pz = __ddiv_rn(sz, M);
    double q[6] = {0, 0, 0, 0, 0, 0}, hm = 0.0;
    const int ch[2] = {L, R};
    for (int side = 0; side < 2; ++side) {
      const int kc = ch[side];
      const double mk = __ldcg(&c.M[kc]);
      const double d0 = __ldcg(&c.cx[kc]) - px, d1 = __ldcg(&c.cy[kc]) - py, d2 = __ldcg(&c.cz[kc]) - pz;
      const double dd = d0 * d0 + d1 * d1 + d2 * d2;
      q[0] += __ldcg(&c.Q[6 * kc + 0]) + mk * (3.0 * d0 * d0 - dd);
      q[1] += __ldcg(&c.Q[6 * kc + 1]) + mk * (3.0 * d0 * d1);
      q[2] += __ldcg(&c.Q[6 * kc + 2]) + mk * (3.0 * d0 * d2);
      q[3] += __ldcg(&c.Q[6 * kc + 3]) + mk * (3.0 * d1 * d1 - dd);
      q[4] += __ldcg(&c.Q[6 * kc + 4]) + mk * (3.0 * d1 * d2);
      q[5] += __ldcg(&c.Q[6 * kc + 5]) + mk * (3.0 * d2 * d2 - dd);
      hm = fmax(hm, __ldcg(&c.hmax[kc]));
    }
    c.M[p] = M; c.cx[p] = px; c.cy[p] = py; c.cz[p] = pz;
    Sx[p] = sx; Sy[p] = sy; Sz[p] = sz;
    for (int j = 0; j < 6; ++j) c.Q[6 * p + j] = q[j];
    c.hmax[p] = hm;
    cur = p;
  }
}

// Exact size of every super-cell: one warp per cell, float32 filter over
// truncated coordinates, float64 for the candidates.
__global__ void k_size_frozen(Cells c, int ncells, PCols tp) {
  const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (t >= ncells || c.left[t] < 0) return;
  const int64_t f = c.first[t];
  const int cnt = c.count[t];
  const double cx = c.cx[t], cy = c.cy[t], cz = c.cz[t];
  const float cxf = trunc_to_float(cx), cyf = trunc_to_float(cy), czf = trunc_to_float(cz);
  float d2m = 0.0f, X = fmaxf(fabsf(cxf), fmaxf(fabsf(cyf), fabsf(czf)));
  for (int j = lane; j < cnt; j += 32) {
    const float dx = trunc_to_float(tp.x[f + j]) - cxf, dy = trunc_to_float(tp.y[f + j]) - cyf,
                dz = trunc_to_float(tp.z[f + j]) - czf;
    d2m = fmaxf(d2m, dx * dx + dy * dy + dz * dz);
    X = fmaxf(X, fmaxf(fabsf(trunc_to_float(tp.x[f + j])),
                       fmaxf(fabsf(trunc_to_float(tp.y[f + j])), fabsf(trunc_to_float(tp.z[f + j])))));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    d2m = fmaxf(d2m, __shfl_xor_sync(0xffffffffu, d2m, o));
    X = fmaxf(X, __shfl_xor_sync(0xffffffffu, X, o));
  }
  const float Dm = sqrtf(d2m);
  const float thr = Dm - 2.0f * dist_err_bound(X * 1.000001f, Dm);
  const float thr2 = thr > 0.0f ? thr * thr * (1.0f - 1e-6f) : -1.0f;
  long long s2 = 0;
  for (int j = lane; j < cnt; j += 32) {
    const double px = tp.x[f + j], py = tp.y[f + j], pz = tp.z[f + j];
    const float dx = trunc_to_float(px) - cxf, dy = trunc_to_float(py) - cyf,
                dz = trunc_to_float(pz) - czf;
    if (dx * dx + dy * dy + dz * dz >= thr2)
      s2 = max(s2, __double_as_longlong(dist2_rn(px, py, pz, cx, cy, cz)));
  }
  s2 = warp_max_ll(s2);
  if (lane == 0) c.s[t] = sqrt(__longlong_as_double(s2));
}

}  // namespace

int recompute_moments(kdfmm_tree_s* t, const double* x, const double* m, const double* h,
                      cudaStream_t s) {
  const int64_t n = t->n;
  const int ncells = t->ncells, nl = t->nleaves;
  cudaMemsetAsync(t->status, 0, sizeof(int32_t), s);
  cudaMemsetAsync(t->com_bound, 0, sizeof(float), s);
  k_gather_frozen<<<blocks_for(n, 256), 256, 0, s>>>(x, m, h, n, t->sys_off, t->n_sys, t->sys_eps,
                                                     t->p.soft_kind, t->tp, t->status);
  double *Sx = t->tmp.cx, *Sy = t->tmp.cy, *Sz = t->tmp.cz;     // free after the build
  k_leaf_frozen<<<blocks_for(nl, 128), 128, 0, s>>>(t->c, t->leaf_cells, nl, t->tp, Sx, Sy, Sz);
  cudaMemsetAsync(t->c.ready, 0, (size_t)ncells * sizeof(int32_t), s);
  k_upward_frozen<<<blocks_for(nl, 128), 128, 0, s>>>(t->c, t->leaf_cells, nl, Sx, Sy, Sz);
  k_size_frozen<<<blocks_for((int64_t)ncells * 32, 256), 256, 0, s>>>(t->c, ncells, t->tp);
  k_derive_cells<<<grid_blocks(), 256, 0, s>>>(t->c, t->counters, t->com_bound);
  k_particles32<<<grid_blocks(), 256, 0, s>>>(t->c, t->leaf_cells, t->counters, t->tp,
                                                                  t->pf, t->ph);
  t->launches += 6;
  cudaMemcpyAsync(&t->host_counters[16], t->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  int rc = check_cuda(cudaStreamSynchronize(s), "frozen moments");
  if (rc) return rc;
  if (t->host_counters[16] & ST_NONFINITE)
    return set_error(KDFMM_ERR_NONFINITE, "non-finite position or non-positive mass / h");
  return check_cuda(cudaGetLastError(), "frozen moments launch");
}

}  // namespace kdfmm
