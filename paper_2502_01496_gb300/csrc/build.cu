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
#include <climits>

#include "kdfmm_internal.cuh"

namespace kdfmm {

namespace {

struct BuildArgs {
  PCols src, dst;
  TmpCells tmp;
  int32_t* counters;
  int32_t* status;
  int32_t n_leaf;
  int64_t capA, capB, capL, cap_cells;
};

__device__ __forceinline__ double coord(const PCols& p, int axis, int64_t i) {
  return axis == 0 ? p.x[i] : (axis == 1 ? p.y[i] : p.z[i]);
}

__device__ __forceinline__ void set_status(int32_t* status, int bits) { atomicOr(status, bits); }

// ---------------------------------------------------------------------------
// initial gather: caller order -> SoA buffer 0, with validation
// ---------------------------------------------------------------------------
__global__ void k_init(const double* __restrict__ x, const double* __restrict__ m,
                       const double* __restrict__ h, int64_t n, double eps, int soft_kind,
                       PCols b, int32_t* status) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double xi = x[3 * i], yi = x[3 * i + 1], zi = x[3 * i + 2], mi = m[i];
  double hi = (h != nullptr && soft_kind == KDFMM_SOFT_M4) ? h[i] : eps;
  bool ok = isfinite(xi) && isfinite(yi) && isfinite(zi) && isfinite(mi) && isfinite(hi) &&
            mi > 0.0 && (soft_kind == KDFMM_SOFT_M4 ? hi > 0.0 : hi >= 0.0);
  if (!ok) set_status(status, ST_NONFINITE);
  b.x[i] = xi; b.y[i] = yi; b.z[i] = zi; b.m[i] = mi; b.h[i] = hi;
  b.idx[i] = (int32_t)i;
}

__global__ void k_root(int64_t n, int32_t n_leaf, Seg* segA, Seg* segB, Seg* segL,
                       int32_t* counters) {
  Seg g{0, (int32_t)n, 0, 0};
  counters[0] = 1;
  if (n > kSubtreeMax) { segA[0] = g; counters[1] = 1; }
  else if (n > n_leaf) { segB[0] = g; counters[2] = 1; }
  else { segL[0] = g; counters[3] = 1; }
}

// Pushes a new segment onto the list that will process it.
__device__ void push_child(const BuildArgs& A, Seg c, Seg* nextA, Seg* segB, Seg* segL) {
  if (c.count > kSubtreeMax) {
    int k = atomicAdd(&A.counters[1], 1);
    if (k < A.capA) nextA[k] = c; else set_status(A.status, ST_CAPACITY);
  } else if (c.count > A.n_leaf) {
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

// Chunk offsets of the nA segments (single block) and the chunk -> segment map.
__global__ void k_chunk_map(const Seg* __restrict__ segs, int nA, int32_t* __restrict__ seg_off,
                            int32_t* __restrict__ chunk_seg, int32_t* counters) {
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

// Chunk partial sums (pairwise subtree of 2048 elements) and bounding box keys.
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
  auto get = [&](int k) {
    int64_t i = base + k;
    return elem4(p.m[i], p.x[i], p.y[i], p.z[i]);
  };
  Sum4 v = block_tree<3>(8 * threadIdx.x, cnt, get);
  long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
  for (int k = threadIdx.x; k < kChunk && k < cnt; k += kChunkThreads) {
    int64_t i = base + k;
    long long kx = dkey(p.x[i]), ky = dkey(p.y[i]), kz = dkey(p.z[i]);
    lo[0] = min(lo[0], kx); hi[0] = max(hi[0], kx);
    lo[1] = min(lo[1], ky); hi[1] = max(hi[1], ky);
    lo[2] = min(lo[2], kz); hi[2] = max(hi[2], kz);
  }
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
    Sum4 t = add4(add4(add4(ws[0], ws[1]), add4(ws[2], ws[3])),
                  add4(add4(ws[4], ws[5]), add4(ws[6], ws[7])));
    csum[4 * b + 0] = t.m; csum[4 * b + 1] = t.x; csum[4 * b + 2] = t.y; csum[4 * b + 3] = t.z;
    for (int d = 0; d < 6; ++d) {
      long long r = wk[0][d];
      for (int q = 1; q < kChunkThreads / 32; ++q) r = d < 3 ? min(r, wk[q][d]) : max(r, wk[q][d]);
      ckey[6 * b + d] = r;
    }
  }
}

// Warp per segment: pairwise tree over its chunk sums, centre of mass, axis, cut.
__global__ void k_decide(const Seg* __restrict__ segs, int nA, const int32_t* __restrict__ seg_off,
                         const double* __restrict__ csum, const long long* __restrict__ ckey,
                         TmpCells tmp, int32_t* __restrict__ seg_axis, double* __restrict__ seg_cut) {
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
  }
}

// Per chunk: particles left of the cut, and the exact max squared distance to
// the centre of mass.
__global__ void __launch_bounds__(kChunkThreads)
k_chunk_count(const Seg* __restrict__ segs, const int32_t* __restrict__ chunk_seg,
              const int32_t* __restrict__ seg_off, const int32_t* __restrict__ counters, PCols p,
              TmpCells tmp, const int32_t* __restrict__ seg_axis, const double* __restrict__ seg_cut,
              int32_t* __restrict__ cleft, long long* __restrict__ cs2) {
  const int b = blockIdx.x;
  if (b >= counters[4]) return;
  const int s = chunk_seg[b];
  const Seg g = segs[s];
  const int rel0 = (b - seg_off[s]) * kChunk;
  const int cnt = min(kChunk, g.count - rel0);
  const int64_t base = (int64_t)g.first + rel0;
  const int axis = seg_axis[s];
  const double cut = seg_cut[s];
  const double cx = tmp.cx[g.cell], cy = tmp.cy[g.cell], cz = tmp.cz[g.cell];
  int nl = 0;
  long long s2 = 0;
  for (int k = threadIdx.x; k < cnt; k += kChunkThreads) {
    int64_t i = base + k;
    double px = p.x[i], py = p.y[i], pz = p.z[i];
    double a = axis == 0 ? px : (axis == 1 ? py : pz);
    nl += a < cut;
    long long d2 = __double_as_longlong(dist2_rn(px, py, pz, cx, cy, cz));
    s2 = max(s2, d2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    nl += __shfl_xor_sync(0xffffffffu, nl, o);
    long long w2 = __shfl_xor_sync(0xffffffffu, s2, o);
    s2 = max(s2, w2);
  }
  __shared__ int wn[kChunkThreads / 32];
  __shared__ long long ws2[kChunkThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) { wn[w] = nl; ws2[w] = s2; }
  __syncthreads();
  if (threadIdx.x == 0) {
    int t = 0;
    long long m2 = 0;
    for (int q = 0; q < kChunkThreads / 32; ++q) { t += wn[q]; m2 = max(m2, ws2[q]); }
    cleft[b] = t;
    cs2[b] = m2;
  }
}

// Warp per segment: offsets of the left particles per chunk, the split point,
// s, and the two children.
__global__ void k_split(const Seg* __restrict__ segs, int nA, const int32_t* __restrict__ seg_off,
                        const int32_t* __restrict__ cleft, const long long* __restrict__ cs2,
                        int32_t* __restrict__ cloff, int32_t* __restrict__ seg_nl, BuildArgs A,
                        Seg* nextA, Seg* segB, Seg* segL, int dst_buf) {
  const int s = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= nA) return;
  const Seg g = segs[s];
  const int C = nchunks_of(g.count);
  const int off = seg_off[s];
  int run = 0;
  long long s2 = 0;
  for (int base = 0; base < C; base += 32) {
    int c = base + lane;
    int v = c < C ? cleft[off + c] : 0;
    if (c < C) s2 = max(s2, cs2[off + c]);
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      int w = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += w;
    }
    if (c < C) cloff[off + c] = run + incl - v;
    run += __shfl_sync(0xffffffffu, incl, 31);
  }
  s2 = warp_max_ll(s2);
  if (lane != 0) return;
  int nl = run;
  const bool fallback = (nl == 0 || nl == g.count);
  if (fallback) {
    nl = g.count / 2;
    atomicAdd(&A.counters[5], 1);
  }
  seg_nl[s] = fallback ? -nl - 1 : nl;
  const int c = g.cell;
  A.tmp.s[c] = sqrt(__longlong_as_double(s2));
  int cid = atomicAdd(&A.counters[0], 2);
  if (cid + 2 > A.cap_cells) { set_status(A.status, ST_CAPACITY); return; }
  A.tmp.left[c] = cid;
  A.tmp.right[c] = cid + 1;
  const int depth = (g.dbuf >> 1) + 1;
  atomicMax(&A.counters[6], depth);
  push_child(A, Seg{g.first, nl, cid, depth << 1 | dst_buf}, nextA, segB, segL);
  push_child(A, Seg{g.first + nl, g.count - nl, cid + 1, depth << 1 | dst_buf}, nextA, segB, segL);
}

// Stable scatter of one chunk into the other buffer.
__global__ void __launch_bounds__(kChunkThreads)
k_chunk_scatter(const Seg* __restrict__ segs, const int32_t* __restrict__ chunk_seg,
                const int32_t* __restrict__ seg_off, const int32_t* __restrict__ counters, PCols src,
                PCols dst, const int32_t* __restrict__ seg_axis, const double* __restrict__ seg_cut,
                const int32_t* __restrict__ cloff, const int32_t* __restrict__ seg_nl) {
  const int b = blockIdx.x;
  if (b >= counters[4]) return;
  const int s = chunk_seg[b];
  const Seg g = segs[s];
  const int rel0 = (b - seg_off[s]) * kChunk;
  const int code = seg_nl[s];
  const bool fallback = code < 0;
  const int nl = fallback ? -code - 1 : code;
  const int axis = seg_axis[s];
  const double cut = seg_cut[s];
  int lefts_before = fallback ? min(rel0, nl) : cloff[b];
  __shared__ int wcount[kChunkThreads / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int pass = 0; pass < kChunk / kChunkThreads; ++pass) {
    const int k = rel0 + pass * kChunkThreads + threadIdx.x;   // position within the segment
    const bool valid = k < g.count;
    const int64_t i = (int64_t)g.first + k;
    bool flag = false;
    if (valid) flag = fallback ? (k < nl) : (coord(src, axis, i) < cut);
    unsigned mask = __ballot_sync(0xffffffffu, flag);
    int rank = __popc(mask & ((1u << lane) - 1u));
    if (lane == 0) wcount[w] = __popc(mask);
    __syncthreads();
    int woff = 0, tot = 0;
    for (int q = 0; q < kChunkThreads / 32; ++q) {
      if (q < w) woff += wcount[q];
      tot += wcount[q];
    }
    if (valid) {
      const int lb = lefts_before + woff + rank;             // left particles before k
      const int64_t d = flag ? (int64_t)g.first + lb : (int64_t)g.first + nl + (k - lb);
      dst.x[d] = src.x[i]; dst.y[d] = src.y[i]; dst.z[d] = src.z[i];
      dst.m[d] = src.m[i]; dst.h[d] = src.h[i]; dst.idx[d] = src.idx[i];
    }
    lefts_before += tot;
    __syncthreads();
  }
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

// Moments of a leaf that lives in shared memory (count <= 32): one lane per
// particle.
__device__ void leaf_in_smem(const SubArgs& S, const double* sx, const double* sy,
                             const double* sz, const double* sm, const uint16_t* lidx, int lf,
                             int cnt, int cell, int depth, int gfirst) {
  const int lane = threadIdx.x & 31;
  auto get = [&](int k) {
    int q = lidx[lf + k];
    return elem4(sm[q], sx[q], sy[q], sz[q]);
  };
  Sum4 v = warp_pairwise(cnt, get);
  const double M = v.m;
  const double cx = __ddiv_rn(v.x, M), cy = __ddiv_rn(v.y, M), cz = __ddiv_rn(v.z, M);
  long long s2 = 0;
  if (lane < cnt) {
    int q = lidx[lf + lane];
    s2 = __double_as_longlong(dist2_rn(sx[q], sy[q], sz[q], cx, cy, cz));
  }
  s2 = warp_max_ll(s2);
  if (lane == 0) {
    TmpCells t = S.A.tmp;
    t.first[cell] = gfirst + lf; t.count[cell] = cnt; t.depth[cell] = depth;
    t.M[cell] = M; t.cx[cell] = cx; t.cy[cell] = cy; t.cz[cell] = cz;
    t.s[cell] = sqrt(__longlong_as_double(s2));
    t.left[cell] = -1; t.right[cell] = -1;
  }
}

__global__ void __launch_bounds__(kSubtreeThreads)
k_subtree(SubArgs S) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sx = reinterpret_cast<double*>(smem_raw);
  double* sy = sx + kSubtreeMax;
  double* sz = sy + kSubtreeMax;
  double* sm = sz + kSubtreeMax;
  uint16_t* lidx = reinterpret_cast<uint16_t*>(sm + kSubtreeMax);
  uint16_t* lscr = lidx + kSubtreeMax;
  int4* q[2];
  q[0] = reinterpret_cast<int4*>(lscr + kSubtreeMax);
  q[1] = q[0] + S.qcap;
  __shared__ int qn[2];

  const Seg g = S.segB[blockIdx.x];
  const PCols in = (g.dbuf & 1) ? S.buf1 : S.buf0;
  const int n = g.count;
  const int gfirst = g.first;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    sx[k] = in.x[gfirst + k]; sy[k] = in.y[gfirst + k]; sz[k] = in.z[gfirst + k];
    sm[k] = in.m[gfirst + k];
    lidx[k] = (uint16_t)k;
  }
  int cur = 0;
  if (threadIdx.x == 0) {
    q[0][0] = make_int4(0, n, g.cell, g.dbuf >> 1);
    qn[0] = 1;
  }
  __syncthreads();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const BuildArgs& A = S.A;
  int depth_max = 0;
  while (qn[cur] > 0) {
    const int nxt = cur ^ 1;
    if (threadIdx.x == 0) qn[nxt] = 0;
    __syncthreads();
    const int nq = qn[cur];
    for (int qi = warp; qi < nq; qi += nwarps) {
      const int4 e = q[cur][qi];
      const int lf = e.x, cnt = e.y, cell = e.z, depth = e.w;
      auto get = [&](int k) {
        int qq = lidx[lf + k];
        return elem4(sm[qq], sx[qq], sy[qq], sz[qq]);
      };
      Sum4 v = warp_pairwise(cnt, get);
      long long lo[3] = {LLONG_MAX, LLONG_MAX, LLONG_MAX}, hi[3] = {LLONG_MIN, LLONG_MIN, LLONG_MIN};
      for (int k = lane; k < cnt; k += 32) {
        int qq = lidx[lf + k];
        long long kx = dkey(sx[qq]), ky = dkey(sy[qq]), kz = dkey(sz[qq]);
        lo[0] = min(lo[0], kx); hi[0] = max(hi[0], kx);
        lo[1] = min(lo[1], ky); hi[1] = max(hi[1], ky);
        lo[2] = min(lo[2], kz); hi[2] = max(hi[2], kz);
      }
      double dlo[3], dhi[3];
      for (int d = 0; d < 3; ++d) { dlo[d] = dunkey(warp_min_ll(lo[d])); dhi[d] = dunkey(warp_max_ll(hi[d])); }
      const double M = v.m;
      const double cx = __ddiv_rn(v.x, M), cy = __ddiv_rn(v.y, M), cz = __ddiv_rn(v.z, M);
      const int axis = longest_axis(dlo, dhi);
      const double cut = axis == 0 ? cx : (axis == 1 ? cy : cz);
      const double* sa = axis == 0 ? sx : (axis == 1 ? sy : sz);
      // exact size and the number of particles left of the cut
      long long s2 = 0;
      int nl = 0;
      for (int k = lane; k < cnt; k += 32) {
        int qq = lidx[lf + k];
        s2 = max(s2, __double_as_longlong(dist2_rn(sx[qq], sy[qq], sz[qq], cx, cy, cz)));
        nl += sa[qq] < cut;
      }
      s2 = warp_max_ll(s2);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) nl += __shfl_xor_sync(0xffffffffu, nl, o);
      const bool fallback = (nl == 0 || nl == cnt);
      if (fallback) {
        nl = cnt / 2;
        if (lane == 0) atomicAdd(&A.counters[5], 1);
      } else {
        // stable partition through the scratch index array
        int offl = 0, offr = nl;
        for (int base = 0; base < cnt; base += 32) {
          int k = base + lane;
          bool valid = k < cnt;
          int qq = valid ? lidx[lf + k] : 0;
          bool f = valid && sa[qq] < cut;
          unsigned ml = __ballot_sync(0xffffffffu, f);
          unsigned mr = __ballot_sync(0xffffffffu, valid && !f);
          unsigned lt = (1u << lane) - 1u;
          if (valid) lscr[lf + (f ? offl + __popc(ml & lt) : offr + __popc(mr & lt))] = (uint16_t)qq;
          offl += __popc(ml);
          offr += __popc(mr);
        }
        __syncwarp();
        for (int k = lane; k < cnt; k += 32) lidx[lf + k] = lscr[lf + k];
        __syncwarp();
      }
      int cid = 0;
      if (lane == 0) {
        TmpCells t = A.tmp;
        t.first[cell] = gfirst + lf; t.count[cell] = cnt; t.depth[cell] = depth;
        t.M[cell] = M; t.cx[cell] = cx; t.cy[cell] = cy; t.cz[cell] = cz;
        t.s[cell] = sqrt(__longlong_as_double(s2));
        cid = atomicAdd(&A.counters[0], 2);
        if (cid + 2 > A.cap_cells) {
          set_status(A.status, ST_CAPACITY);
          cid = -1;
        } else {
          t.left[cell] = cid;
          t.right[cell] = cid + 1;
        }
      }
      cid = __shfl_sync(0xffffffffu, cid, 0);
      if (cid < 0) continue;
      depth_max = max(depth_max, depth + 1);
      const int clf[2] = {lf, lf + nl}, ccnt[2] = {nl, cnt - nl};
      for (int side = 0; side < 2; ++side) {
        if (ccnt[side] > A.n_leaf) {
          if (lane == 0) {
            int pos = atomicAdd(&qn[nxt], 1);
            if (pos < S.qcap) q[nxt][pos] = make_int4(clf[side], ccnt[side], cid + side, depth + 1);
            else set_status(A.status, ST_CAPACITY);
          }
        } else {
          leaf_in_smem(S, sx, sy, sz, sm, lidx, clf[side], ccnt[side], cid + side, depth + 1, gfirst);
        }
      }
    }
    __syncthreads();
    cur ^= 1;
  }
  if (lane == 0 && depth_max > 0) atomicMax(&A.counters[6], depth_max);
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    int src = lidx[k];
    int64_t p = (int64_t)gfirst + k;
    S.out.x[p] = sx[src]; S.out.y[p] = sy[src]; S.out.z[p] = sz[src]; S.out.m[p] = sm[src];
    S.out.h[p] = in.h[gfirst + src];
    S.out.idx[p] = in.idx[gfirst + src];
  }
}

// Leaves produced directly by phase A (or a root that is already a leaf).
__global__ void k_leaf_segs(SubArgs S, const Seg* __restrict__ segL, int nL) {
  const int sidx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (sidx >= nL) return;
  const Seg g = segL[sidx];
  const PCols in = (g.dbuf & 1) ? S.buf1 : S.buf0;
  const int cnt = g.count;
  auto get = [&](int k) {
    int64_t i = (int64_t)g.first + k;
    return elem4(in.m[i], in.x[i], in.y[i], in.z[i]);
  };
  Sum4 v = warp_pairwise(cnt, get);
  const double M = v.m;
  const double cx = __ddiv_rn(v.x, M), cy = __ddiv_rn(v.y, M), cz = __ddiv_rn(v.z, M);
  long long s2 = 0;
  if (lane < cnt) {
    int64_t i = (int64_t)g.first + lane;
    s2 = __double_as_longlong(dist2_rn(in.x[i], in.y[i], in.z[i], cx, cy, cz));
    S.out.x[i] = in.x[i]; S.out.y[i] = in.y[i]; S.out.z[i] = in.z[i];
    S.out.m[i] = in.m[i]; S.out.h[i] = in.h[i]; S.out.idx[i] = in.idx[i];
  }
  s2 = warp_max_ll(s2);
  if (lane == 0) {
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

__global__ void k_count_starts(TmpCells tmp, int ncells, int32_t* cnt_start, int32_t* min_depth) {
  int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  int f = tmp.first[c];
  atomicAdd(&cnt_start[f], 1);
  atomicMin(&min_depth[f], tmp.depth[c]);
}

__device__ __forceinline__ int preorder_id(const int32_t* start_off, const int32_t* min_depth,
                                           int first, int depth) {
  return start_off[first] + depth - min_depth[first];
}

__global__ void k_remap(TmpCells tmp, int ncells, const int32_t* __restrict__ start_off,
                        const int32_t* __restrict__ min_depth, Cells c, int32_t* status) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncells) return;
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
  if (id == 0) c.parent[0] = -1;
}

// Leaves: h_max and Q (Eq. 7) from their particles; then each parent, once its
// second child has finished, from its children (parallel-axis shift of Q).
__global__ void k_upward(Cells c, int ncells, PCols tp) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncells || c.left[t] >= 0) return;
  {
    const int f = c.first[t], cnt = c.count[t];
    const double cx = c.cx[t], cy = c.cy[t], cz = c.cz[t];
    double q[6] = {0, 0, 0, 0, 0, 0}, hm = 0.0;
    for (int k = 0; k < cnt; ++k) {
      int64_t i = (int64_t)f + k;
      double m = tp.m[i];
      double y0 = tp.x[i] - cx, y1 = tp.y[i] - cy, y2 = tp.z[i] - cz;
      double y2s = y0 * y0 + y1 * y1 + y2 * y2;
      q[0] += m * (3.0 * y0 * y0 - y2s);
      q[1] += m * (3.0 * y0 * y1);
      q[2] += m * (3.0 * y0 * y2);
      q[3] += m * (3.0 * y1 * y1 - y2s);
      q[4] += m * (3.0 * y1 * y2);
      q[5] += m * (3.0 * y2 * y2 - y2s);
      hm = fmax(hm, tp.h[i]);
    }
    for (int k = 0; k < 6; ++k) c.Q[6 * t + k] = q[k];
    c.hmax[t] = hm;
  }
  int cur = t;
  while (true) {
    const int p = c.parent[cur];
    if (p < 0) break;
    __threadfence();
    if (atomicAdd(&c.ready[p], 1) == 0) break;      // the sibling finishes the parent
    __threadfence();
    const double px = c.cx[p], py = c.cy[p], pz = c.cz[p];
    double q[6] = {0, 0, 0, 0, 0, 0}, hm = 0.0;
    const int ch[2] = {c.left[p], c.right[p]};
    for (int side = 0; side < 2; ++side) {
      const int k = ch[side];
      const double mk = c.M[k];
      const double d0 = c.cx[k] - px, d1 = c.cy[k] - py, d2 = c.cz[k] - pz;
      const double dd = d0 * d0 + d1 * d1 + d2 * d2;
      q[0] += __ldcg(&c.Q[6 * k + 0]) + mk * (3.0 * d0 * d0 - dd);
      q[1] += __ldcg(&c.Q[6 * k + 1]) + mk * (3.0 * d0 * d1);
      q[2] += __ldcg(&c.Q[6 * k + 2]) + mk * (3.0 * d0 * d2);
      q[3] += __ldcg(&c.Q[6 * k + 3]) + mk * (3.0 * d1 * d1 - dd);
      q[4] += __ldcg(&c.Q[6 * k + 4]) + mk * (3.0 * d1 * d2);
      q[5] += __ldcg(&c.Q[6 * k + 5]) + mk * (3.0 * d2 * d2 - dd);
      hm = fmax(hm, __ldcg(&c.hmax[k]));
    }
    for (int k = 0; k < 6; ++k) c.Q[6 * p + k] = q[k];
    c.hmax[p] = hm;
    cur = p;
  }
}

// float32 views of the cells; leaf flags for the leaf ranking.
__global__ void k_derive_cells(Cells c, int ncells, int32_t* leaf_flag, float* com_bound) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncells) return;
  const double cx = c.cx[t], cy = c.cy[t], cz = c.cz[t];
  c.walk[t] = make_float4((float)cx, (float)cy, (float)cz, (float)c.s[t]);
  c.walk2[t] = make_float2((float)c.hmax[t], __int_as_float(c.skip[t]));
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
  leaf_flag[t] = c.left[t] < 0 ? 1 : 0;
  float b = fmaxf(fabsf((float)cx), fmaxf(fabsf((float)cy), fabsf((float)cz)));
  atomicMax(reinterpret_cast<int*>(com_bound), __float_as_int(b));
}

__global__ void k_leaf_list(const Cells c, int ncells, int32_t* leaf_rank, int32_t* leaf_cells) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ncells) return;
  if (c.left[t] < 0) leaf_cells[leaf_rank[t]] = t;
  else leaf_rank[t] = -1;
}

// Per-particle float32 data relative to the centre of mass of its leaf.
__global__ void k_particles32(const Cells c, const int32_t* __restrict__ leaf_cells, int nleaves,
                              PCols tp, float4* pf, float4* ph) {
  const int k = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (k >= nleaves) return;
  const int cell = leaf_cells[k];
  const int f = c.first[cell], cnt = c.count[cell];
  if (lane >= cnt) return;
  const int64_t i = (int64_t)f + lane;
  pf[i] = make_float4((float)(tp.x[i] - c.cx[cell]), (float)(tp.y[i] - c.cy[cell]),
                      (float)(tp.z[i] - c.cz[cell]), (float)tp.m[i]);
  const float h = (float)tp.h[i];
  const float hi = h > 0.0f ? 1.0f / h : 0.0f;
  ph[i] = make_float4(hi, hi * hi * hi, h, 0.0f);
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
                  t->tmp.first, t->tmp.count, t->tmp.left, t->tmp.right, t->tmp.depth, t->tmp.M,
                  t->tmp.cx, t->tmp.cy, t->tmp.cz, t->tmp.s, t->cnt_start, t->min_depth,
                  t->start_off, t->scan_tmp, t->pf, t->ph, t->c.first, t->c.count, t->c.left,
                  t->c.right, t->c.parent, t->c.skip, t->c.depth, t->c.M, t->c.cx, t->c.cy,
                  t->c.cz, t->c.s, t->c.hmax, t->c.Q, t->c.walk, t->c.walk2, t->c.src32,
                  t->c.src64, t->c.ready, t->leaf_cells, t->leaf_rank, t->lexp64, t->lexp32};
  for (void* p : ptrs) cudaFree(p);
  t->segB = t->segL = nullptr;
  t->chunk_seg = t->seg_chunk_off = t->chunk_left = t->chunk_loff = t->seg_axis = t->seg_nl = nullptr;
  t->chunk_sum = t->seg_cut = nullptr;
  t->chunk_key = t->chunk_s2 = nullptr;
  t->tmp = TmpCells{};
  t->cnt_start = t->min_depth = t->start_off = t->scan_tmp = nullptr;
  t->pf = t->ph = nullptr;
  t->c = Cells{};
  t->leaf_cells = t->leaf_rank = nullptr;
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
  KD_ALLOC(t->lexp64, 20 * (n + 1));
  KD_ALLOC(t->lexp32, 24 * (n + 1));
  t->cap_n = n;
  return KDFMM_OK;
}

int build_tree(kdfmm_tree_s* t, const double* x, const double* m, const double* h, cudaStream_t s) {
  const int64_t n = t->n;
  int rc = ensure_build_buffers(t, n);
  if (rc) return rc;
  const kdfmm_params& P = t->p;
  cudaMemsetAsync(t->counters, 0, 16 * sizeof(int32_t), s);
  cudaMemsetAsync(t->status, 0, sizeof(int32_t), s);
  cudaMemsetAsync(t->com_bound, 0, sizeof(float), s);
  k_init<<<blocks_for(n, 256), 256, 0, s>>>(x, m, h, n, P.eps, P.soft_kind, t->buf[0], t->status);
  k_root<<<1, 1, 0, s>>>(n, P.n_leaf, t->segA[0], t->segB, t->segL, t->counters);
  t->launches += 2;

  BuildArgs A{};
  A.tmp = t->tmp;
  A.counters = t->counters;
  A.status = t->status;
  A.n_leaf = P.n_leaf;
  A.capA = t->capA; A.capB = t->capB; A.capL = t->capL; A.cap_cells = t->cap_cells;

  int32_t* hc = t->host_counters;
  rc = check_cuda(cudaMemcpyAsync(hc, t->counters, 16 * sizeof(int32_t), cudaMemcpyDeviceToHost, s),
                  "counters");
  if (rc) return rc;
  cudaMemcpyAsync(&t->host_counters[16], t->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if ((rc = check_cuda(cudaStreamSynchronize(s), "build init"))) return rc;
  if (t->host_counters[16] & ST_NONFINITE)
    return set_error(KDFMM_ERR_NONFINITE, "non-finite position or non-positive mass / h");
  int nA = hc[1];
  int cur = 0, level = 0;
  while (nA > 0) {
    const int src = level & 1, dst = src ^ 1;
    A.src = t->buf[src];
    A.dst = t->buf[dst];
    const Seg* segs = t->segA[cur];
    Seg* next = t->segA[cur ^ 1];
    cudaMemsetAsync(t->counters + 1, 0, sizeof(int32_t), s);
    k_chunk_map<<<1, 1024, 0, s>>>(segs, nA, t->seg_chunk_off, t->chunk_seg, t->counters);
    const unsigned maxc = (unsigned)(n / kChunk + nA + 1);
    k_chunk_reduce<<<maxc, kChunkThreads, 0, s>>>(segs, t->chunk_seg, t->seg_chunk_off, t->counters,
                                                  t->buf[src], t->chunk_sum, t->chunk_key);
    k_decide<<<blocks_for((int64_t)nA * 32, 256), 256, 0, s>>>(segs, nA, t->seg_chunk_off,
                                                               t->chunk_sum, t->chunk_key, t->tmp,
                                                               t->seg_axis, t->seg_cut);
    k_chunk_count<<<maxc, kChunkThreads, 0, s>>>(segs, t->chunk_seg, t->seg_chunk_off, t->counters,
                                                 t->buf[src], t->tmp, t->seg_axis, t->seg_cut,
                                                 t->chunk_left, t->chunk_s2);
    k_split<<<blocks_for((int64_t)nA * 32, 256), 256, 0, s>>>(
        segs, nA, t->seg_chunk_off, t->chunk_left, t->chunk_s2, t->chunk_loff, t->seg_nl, A, next,
        t->segB, t->segL, dst);
    k_chunk_scatter<<<maxc, kChunkThreads, 0, s>>>(segs, t->chunk_seg, t->seg_chunk_off, t->counters,
                                                   t->buf[src], t->buf[dst], t->seg_axis, t->seg_cut,
                                                   t->chunk_loff, t->seg_nl);
    t->launches += 6;
    rc = check_cuda(cudaMemcpyAsync(hc, t->counters, 16 * sizeof(int32_t), cudaMemcpyDeviceToHost, s),
                    "counters");
    if (rc) return rc;
    if ((rc = check_cuda(cudaStreamSynchronize(s), "build level"))) return rc;
    nA = hc[1];
    if (nA > t->capA || hc[2] > t->capB || hc[3] > t->capL)
      return set_error(KDFMM_ERR_CAPACITY, "segment lists overflow");
    cur ^= 1;
    ++level;
    if (level > 200) return set_error(KDFMM_ERR_INTERNAL, "phase A did not terminate");
  }
  const int nB = hc[2], nL = hc[3];
  if (nB > t->capB || nL > t->capL) return set_error(KDFMM_ERR_CAPACITY, "segment lists overflow");

  SubArgs S{};
  S.A = A;
  S.buf0 = t->buf[0];
  S.buf1 = t->buf[1];
  S.out = t->tp;
  S.segB = t->segB;
  S.qcap = kSubtreeMax / (P.n_leaf + 1) + 2;
  if (nB > 0) {
    size_t smem = 4 * kSubtreeMax * sizeof(double) + 2 * kSubtreeMax * sizeof(uint16_t) +
                  2 * (size_t)S.qcap * sizeof(int4);
    rc = check_cuda(cudaFuncSetAttribute(k_subtree, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem),
                    "subtree smem attribute");
    if (rc) return rc;
    k_subtree<<<nB, kSubtreeThreads, smem, s>>>(S);
    t->launches += 1;
  }
  if (nL > 0) {
    k_leaf_segs<<<blocks_for((int64_t)nL * 32, 256), 256, 0, s>>>(S, t->segL, nL);
    t->launches += 1;
  }
  rc = check_cuda(cudaMemcpyAsync(hc, t->counters, 16 * sizeof(int32_t), cudaMemcpyDeviceToHost, s),
                  "counters");
  if (rc) return rc;
  int32_t status = 0;
  cudaMemcpyAsync(&t->host_counters[16], t->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if ((rc = check_cuda(cudaStreamSynchronize(s), "build subtrees"))) return rc;
  status = t->host_counters[16];
  if (status & ST_NONFINITE)
    return set_error(KDFMM_ERR_NONFINITE, "non-finite position or non-positive mass / h");
  if (status & ST_CAPACITY) return set_error(KDFMM_ERR_CAPACITY, "build capacity exceeded");
  const int ncells = hc[0];
  t->ncells = ncells;
  t->nfallback = hc[5];
  t->depth = hc[6];

  // pre-order numbering
  k_fill2<<<blocks_for(n + 1, 256), 256, 0, s>>>(t->cnt_start, 0, t->min_depth, INT_MAX, n + 1);
  k_count_starts<<<blocks_for(ncells, 256), 256, 0, s>>>(t->tmp, ncells, t->cnt_start, t->min_depth);
  scan_i32(t->cnt_start, t->start_off, n, t->scan_tmp, s);
  k_remap<<<blocks_for(ncells, 256), 256, 0, s>>>(t->tmp, ncells, t->start_off, t->min_depth, t->c,
                                                  t->status);
  cudaMemsetAsync(t->c.ready, 0, (size_t)ncells * sizeof(int32_t), s);
  k_upward<<<blocks_for(ncells, 128), 128, 0, s>>>(t->c, ncells, t->tp);
  // the arrival counters are free again: reuse them for the leaf flags
  k_derive_cells<<<blocks_for(ncells, 256), 256, 0, s>>>(t->c, ncells, t->c.ready, t->com_bound);
  scan_i32(t->c.ready, t->leaf_rank, ncells, t->scan_tmp, s);
  cudaMemcpyAsync(&t->host_counters[17], t->leaf_rank + ncells, sizeof(int32_t),
                  cudaMemcpyDeviceToHost, s);
  k_leaf_list<<<blocks_for(ncells, 256), 256, 0, s>>>(t->c, ncells, t->leaf_rank, t->leaf_cells);
  t->launches += 12;
  cudaMemcpyAsync(&t->host_counters[16], t->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  if ((rc = check_cuda(cudaStreamSynchronize(s), "build finalise"))) return rc;
  t->nleaves = t->host_counters[17];
  if (t->host_counters[16] & ST_INTERNAL)
    return set_error(KDFMM_ERR_INTERNAL, "pre-order numbering inconsistent");
  k_particles32<<<blocks_for((int64_t)t->nleaves * 32, 256), 256, 0, s>>>(
      t->c, t->leaf_cells, t->nleaves, t->tp, t->pf, t->ph);
  t->launches += 1;
  return check_cuda(cudaGetLastError(), "build launch");
}

// Frozen-topology moments are not provided by this build.
int recompute_moments(kdfmm_tree_s* t, const double* x, const double* m, const double* h,
                      cudaStream_t s) {
  (void)t; (void)x; (void)m; (void)h; (void)s;
  return set_error(KDFMM_ERR_INVALID_ARG, "frozen-topology moments not available in this build");
}

}  // namespace kdfmm
