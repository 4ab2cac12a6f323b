// Internal declarations of the kdfmm CUDA library (sm_103a).  Not part of the
// public ABI; include/kdfmm.h is.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "kdfmm.h"

namespace kdfmm {

// ---------------------------------------------------------------------------
// Tunables
// ---------------------------------------------------------------------------
constexpr int kChunk = 2048;           // phase-A reduction chunk (elements)
constexpr int kChunkThreads = 256;     // 8 consecutive elements per thread
static_assert(kChunk == 8 * kChunkThreads, "the chunk reduce sums 8 elements per thread");
constexpr int kSubtreeMax = 2048;      // cells this small finish in shared memory
constexpr int kSubtreeThreads = 256;
constexpr int kNumStatus = 4;

// Device-side status bits (OR-ed into a device word, read after a sync).
enum : int {
  ST_NONFINITE = 1,
  ST_CAPACITY = 2,
  ST_INTERNAL = 4,
  ST_TIMEOUT = 8,
  ST_UNFINISHED = 16,   // phase A still held segments after its fixed number of levels
  ST_LISTS = 32,        // the leaves or an interaction list outgrew a fixed capacity
};

// Slots of the handle's device counter block (32 int32).  Kernels read the
// sizes they work on from here, so a launch needs no host-side count.
enum : int {
  C_CELLS = 0,      // cells allocated
  C_NEXT_A = 1,     // segments pushed for the next phase-A level
  C_NB = 2,         // phase-B segments
  C_NL = 3,         // leaf segments finished by phase A
  C_CHUNKS = 4,     // chunks of the current phase-A level
  C_FALLBACK = 5,   // degenerate cuts
  C_DEPTH = 6,      // deepest level
  C_MAXFAR = 8,     // longest far list of the last walk
  C_MAXNEAR = 9,    // longest near list of the last walk
  C_NA = 10,        // segments of the current phase-A level
  C_LEAVES = 11,    // leaves
  C_WORK = 12,      // dynamic work counter of the persistent subtree kernel
  C_HEAVY = 13,     // leaves whose walk outgrew the per-thread budget (queued)
  C_SEGS = 14,      // extra P2P segments of leaves with long near lists
};

// Streaming multiprocessors of the current device (queried once per device).
int sm_count();
// Grid of the grid-stride (persistent) kernels: per_sm blocks on every SM.
inline unsigned grid_blocks(int per_sm = 8) { return (unsigned)(sm_count() * per_sm); }
#define KD_GRID_STRIDE(i, n)                                                             \
  for (int i = (int)(blockIdx.x * blockDim.x + threadIdx.x); i < (n); i += (int)(gridDim.x * blockDim.x))

// A contiguous run of tree positions that belongs to one cell during the build.
struct Seg {
  int32_t first;   // first tree position
  int32_t count;   // particles
  int32_t cell;    // build-order (temporary) cell id
  int32_t dbuf;    // depth << 1 | buffer holding the particles
};

// Particle columns, float64, in one tree order.
struct PCols {
  double *x, *y, *z, *m, *h;
  int32_t* idx;    // caller index
};

// Cells in build (temporary) order.
struct TmpCells {
  int32_t *first, *count, *left, *right, *depth;
  double *M, *cx, *cy, *cz, *s;
};

// Cells in final pre-order.
struct Cells {
  int32_t *first, *count, *left, *right, *parent, *skip, *depth;
  double *M, *cx, *cy, *cz, *s, *hmax;
  double* Q;                 // 6 per cell: xx xy xz yy yz zz
  // derived views
  float4* walk;              // (com x y z, s) in float32 for the walk's filter
  float4* walk2;             // (h_max, skip, particle count as int bits, 0)
  float4* src32;             // 4 per cell: (hi xyz, M), (lo xyz, 0), (Q xx xy xz yy), (Q yz zz, 0, 0)
  double* src64;             // 10 per cell: com xyz, M, Q[6]
  int32_t* ready;            // bottom-up arrival counters
};

// Interaction lists: leaf k's far (M2L) list is far_idx[far_off[k] ...] with
// far_cnt[k] entries, its near (P2P) list likewise; entries in ascending id.
// Slot mode: far_off[k] = k * cap_far (fixed-size slots); exact mode: the
// scanned counts (used when a few lists are far longer than the rest).
struct Lists {
  int32_t *far_cnt, *near_cnt;
  int64_t *far_off, *near_off;     // nleaves + 1
  int32_t *far_idx, *near_idx;
  int64_t far_cap, near_cap;       // allocated entries
  int64_t cap_far, cap_near;       // slot size per leaf (slot mode)
  bool exact;                      // offsets are per leaf, counts unlimited (arena or dual walk)
  bool arena;                      // leaf walk into reserved room (one pass, see walk.cu)
  int32_t* temp;                   // arena walk: per-thread scratch
  int64_t temp_cap;                // its entries
  int32_t arena_grid;              // blocks of the arena walk
  int64_t* near_np;                // device statistics of the walk (4)
  int32_t* heavy;                  // leaves queued for the block-wide walk (nleaves)
  // near lists longer than kSegEntries are split: segment 0 stays with the
  // leaf, the others are work items of their own whose partial sums
  // (seg_part, 32 targets x 4 doubles each) are added in segment order
  int32_t* seg_first;              // per leaf: first extra segment, or -1
  int32_t* seg_leaf;               // per extra segment: its leaf
  double* seg_part;                // per extra segment: partial sums
  int64_t seg_cap;                 // extra segments allocated
};

// Near entries per P2P segment.
constexpr int kSegEntries = 256;

// Extra segments of a near list of n entries.
__host__ __device__ __forceinline__ int extra_segments(int64_t n) {
  return n > kSegEntries ? (int)((n - 1) / kSegEntries) : 0;
}

}  // namespace kdfmm

struct kdfmm_tree_s {
  int device = 0;
  int64_t n = 0, cap_n = 0;
  int32_t ncells = 0, nleaves = 0, depth = 0, nfallback = 0;
  int32_t grid_leaves = 0;         // leaves the launches of an evaluation are sized for
  int32_t levels_used = 0;         // phase-A levels of the last host-followed build
  int32_t subtree_grid = 0;        // persistent grid of the subtree kernel
  size_t subtree_smem = 0;
  int64_t cap_cells = 0;
  kdfmm_params p{};
  bool built = false, evaluated = false, lists_frozen = false;

  // build scratch
  kdfmm::PCols buf[2]{};
  kdfmm::Seg* segA[2]{};
  kdfmm::Seg *segB = nullptr, *segL = nullptr;
  int64_t capA = 0, capB = 0, capL = 0;
  int32_t* counters = nullptr;     // device: [0] cells, [1] nextA, [2] nB, [3] nL, [4] chunks, [5] nfallback, [6] depth, [7] nexact
  int32_t* status = nullptr;       // device status word
  int32_t* chunk_seg = nullptr;
  int32_t* seg_chunk_off = nullptr;
  double* chunk_sum = nullptr;     // 4 per chunk
  long long* chunk_key = nullptr;  // 6 per chunk: min xyz, max xyz
  int32_t* chunk_left = nullptr;
  int32_t* chunk_loff = nullptr;
  float* chunk_s2 = nullptr;         // per chunk: largest float32 squared distance
  float* seg_xb = nullptr;           // per segment: bound on |coordinates|
  float* seg_thr2 = nullptr;         // per segment: candidate threshold for the exact size
  long long* seg_s2 = nullptr;       // per segment: exact squared size (as int64 bits)
  int32_t* seg_axis = nullptr;
  double* seg_cut = nullptr;
  int32_t* seg_nl = nullptr;
  int64_t cap_chunks = 0, cap_segA = 0;
  kdfmm::TmpCells tmp{};
  int32_t *cnt_start = nullptr, *min_depth = nullptr, *start_off = nullptr;
  int32_t* scan_tmp = nullptr;
  int64_t cap_scan = 0;

  // final tree
  kdfmm::PCols tp{};               // tree order: x y z m h, idx = caller index
  float4* pf = nullptr;            // (x - com_leaf, m) float32
  float4* ph = nullptr;            // (1/h, 1/h^3, h, (2h)^2) float32
  kdfmm::Cells c{};
  int32_t* leaf_cells = nullptr;   // pre-order ids of the leaves
  int32_t* leaf_rank = nullptr;    // cell -> leaf ordinal (-1 for super-cells)
  float* com_bound = nullptr;      // device: max |com component| over cells
  kdfmm::Lists L{};
  double* lexp64 = nullptr;        // 20 per leaf
  float* lexp32 = nullptr;         // 24 per leaf (20 coefficients + 4 low parts)

  // systems: a forest of independent trees (one system for a single tree);
  // system k owns particles [sys_off[k], sys_off[k + 1]) in caller order and
  // cells [sys_root[k], sys_root[k + 1]) in pre-order
  int32_t n_sys = 0, cap_sys = 0;
  int32_t min_nleaf = 0;
  int64_t* sys_off = nullptr;      // device, n_sys + 1
  double* sys_theta = nullptr;     // device, n_sys
  double* sys_eps = nullptr;       // device, n_sys
  int32_t* sys_nleaf = nullptr;    // device, n_sys
  int32_t* sys_root = nullptr;     // device, n_sys + 1
  int32_t* leaf_sys = nullptr;     // device, system of each leaf ordinal
  int64_t* host_sys_off = nullptr; // pinned host copy of sys_off

  double* mom_partial = nullptr;   // total_momentum scratch
  int64_t cap_mom = 0;
  int64_t* host_stats = nullptr;   // pinned host mirror
  int32_t* host_counters = nullptr;
  int64_t launches = 0;            // kernels launched by this handle
  int32_t walk_budget = 0;         // cells a walk thread visits before its leaf goes to the
                                   // block-wide walk (0: the default)

  // symmetric dual-tree walk (KDFMM_WALK_DUAL): pair queues, the far and near
  // pair lists, per-cell far lists and per-cell local expansions
  struct Dual {
    int2 *q[2] = {nullptr, nullptr}, *far = nullptr, *near = nullptr;
    int64_t q_cap = 0, far_cap = 0, near_cap = 0;
    int32_t* ctr = nullptr;              // device: [0] queue out, [1] far pairs, [2] near pairs, [3] overflow
    int64_t* np2p = nullptr;             // device: particle pairs of the near list
    int32_t* far_cnt = nullptr;          // per cell
    int64_t* far_off = nullptr;          // per cell + 1
    int32_t* far_idx = nullptr;
    int64_t far_idx_cap = 0, cells_cap = 0;
    int32_t* cursor = nullptr;           // per cell (fill cursors)
    float* lcell32 = nullptr;            // 24 per cell
    double* lcell64 = nullptr;           // 20 per cell
    double* ltot = nullptr;              // 20 per cell: own + ancestors' expansions, at its com
    int64_t ltot_cap = 0;
    int64_t nfar = 0, nnear = 0;         // entries (both directions)
  } dual;

  // captured evaluation (kdfmm_fmm_accel_batched): valid for the arguments
  // and buffers it was captured with
  struct GraphKey {
    const void *x, *m, *h;
    void *a, *phi;
    int64_t n, cap_n, cap_far, cap_near, far_cap, near_cap, seg_cap, temp_cap;
    int32_t n_sys, cap_sys, min_nleaf, soft_kind, precision, expansion, walk, arena_grid, budget;
    bool arena;
    double r_kern;
    bool operator==(const GraphKey& o) const {
      return x == o.x && m == o.m && h == o.h && a == o.a && phi == o.phi && n == o.n &&
             expansion == o.expansion && walk == o.walk && budget == o.budget &&
             cap_n == o.cap_n && cap_far == o.cap_far && cap_near == o.cap_near &&
             far_cap == o.far_cap && near_cap == o.near_cap && seg_cap == o.seg_cap &&
             temp_cap == o.temp_cap && arena == o.arena && arena_grid == o.arena_grid &&
             n_sys == o.n_sys &&
             cap_sys == o.cap_sys && min_nleaf == o.min_nleaf && soft_kind == o.soft_kind &&
             precision == o.precision && r_kern == o.r_kern;
    }
  };
  GraphKey graph_key{};
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t capture_stream = nullptr;
  int32_t graph_levels = 0, graph_leaves = 0;
  int64_t graph_launches = 0;      // kernels in the captured graph
  bool timing = false;
  cudaEvent_t ev[2 * KDFMM_NPHASES]{};
  bool ev_used[KDFMM_NPHASES]{};
};

namespace kdfmm {

// ---------------------------------------------------------------------------
// Device helpers
// ---------------------------------------------------------------------------

// Order-preserving int64 key of a double (min / max / < with integer ops):
// for non-NaN a, b: a < b exactly when dkey(a) < dkey(b) (-0 is keyed as +0).
__device__ __forceinline__ long long dkey(double v) {
  long long b = __double_as_longlong(v);
  if (b == (long long)0x8000000000000000ULL) b = 0;
  return b ^ ((b >> 63) & 0x7fffffffffffffffLL);
}
__device__ __forceinline__ double dunkey(long long k) {
  return __longlong_as_double(k ^ ((k >> 63) & 0x7fffffffffffffffLL));
}

// float32 value of a double by truncating the mantissa, with integer
// operations only: |result| <= |v| and |v - result| < 2^-23 |v| for normal
// results; magnitudes below 2^-126 become zero, above the float range infinity.
// Used where a float32 estimate with a known error bound is enough.
__device__ __forceinline__ float trunc_to_float(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const unsigned hi = (unsigned)(b >> 32), lo = (unsigned)b;
  const unsigned sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu) - 1023 + 127;
  if (e <= 0) return __uint_as_float(sign);
  if (e >= 255) return __uint_as_float(sign | 0x7f800000u);
  const unsigned mant = ((hi & 0xfffffu) << 3) | (lo >> 29);
  return __uint_as_float(sign | ((unsigned)e << 23) | mant);
}

// Bound on |d_float32 - d| for a distance d whose coordinates and centre lie
// within X of the origin, the coordinates taken as float32 by rounding or by
// trunc_to_float (per component 2 x 2^-23 X, the difference, squares, sum and
// square root), with a safety factor of more than 2.
__device__ __forceinline__ float dist_err_bound(float X, float d) {
  const float u = 5.9604645e-8f;
  return 16.0f * u * (X + d) + 1e-37f;
}

struct Sum4 {
  double m, x, y, z;
};
__device__ __forceinline__ Sum4 zero4() { return Sum4{0.0, 0.0, 0.0, 0.0}; }
__device__ __forceinline__ Sum4 add4(const Sum4& a, const Sum4& b) {
  return Sum4{__dadd_rn(a.m, b.m), __dadd_rn(a.x, b.x), __dadd_rn(a.y, b.y), __dadd_rn(a.z, b.z)};
}
__device__ __forceinline__ Sum4 shfl_xor4(const Sum4& a, int o) {
  return Sum4{__shfl_xor_sync(0xffffffffu, a.m, o), __shfl_xor_sync(0xffffffffu, a.x, o),
              __shfl_xor_sync(0xffffffffu, a.y, o), __shfl_xor_sync(0xffffffffu, a.z, o)};
}
// Butterfly over the 32 lanes: lane l holds the sum of an aligned block l;
// pairing (2j, 2j+1), then pairs of pairs... is the perfect binary tree, and
// every lane ends with the full sum.
__device__ __forceinline__ Sum4 warp_tree4(Sum4 v) {
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) v = add4(v, shfl_xor4(v, o));
  return v;
}
// The element (m, m x, m y, m z) of one particle, products correctly rounded.
__device__ __forceinline__ Sum4 elem4(double m, double x, double y, double z) {
  return Sum4{m, __dmul_rn(m, x), __dmul_rn(m, y), __dmul_rn(m, z)};
}

// Perfect binary tree over 2^LOGB consecutive elements starting at `base`,
// entries at or beyond `count` reading as zero.
template <int LOGB, class F>
__device__ __forceinline__ Sum4 block_tree(int base, int count, const F& get) {
  if constexpr (LOGB == 0) {
    return base < count ? get(base) : zero4();
  } else {
    if (base >= count) return zero4();
    constexpr int H = 1 << (LOGB - 1);
    Sum4 l = block_tree<LOGB - 1>(base, count, get);
    Sum4 r = block_tree<LOGB - 1>(base + H, count, get);
    return add4(l, r);
  }
}

// Canonical pairwise sum of `count` elements (count <= 2048) by one warp: the
// sequence is padded to P = 2^ceil(log2 count); lane l sums its aligned block
// of P/32 elements as a perfect tree, the butterfly combines the lanes.
template <class F>
__device__ __forceinline__ Sum4 warp_pairwise(int count, const F& get) {
  const int lane = threadIdx.x & 31;
  int P = 1;
  while (P < count) P <<= 1;
  Sum4 v;
  if (P <= 32) {
    v = lane < count ? get(lane) : zero4();
  } else {
    const int B = P >> 5;
    const int base = lane * B;
    switch (B) {
      case 2: v = block_tree<1>(base, count, get); break;
      case 4: v = block_tree<2>(base, count, get); break;
      case 8: v = block_tree<3>(base, count, get); break;
      case 16: v = block_tree<4>(base, count, get); break;
      case 32: v = block_tree<5>(base, count, get); break;
      default: v = block_tree<6>(base, count, get); break;
    }
  }
  return warp_tree4(v);
}

__device__ __forceinline__ long long warp_min_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w < v ? w : v;
  }
  return v;
}
__device__ __forceinline__ long long warp_max_ll(long long v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    long long w = __shfl_xor_sync(0xffffffffu, v, o);
    v = w > v ? w : v;
  }
  return v;
}

// Squared distance exactly as dx*dx + dy*dy + dz*dz (no contraction).
__device__ __forceinline__ double dist2_rn(double x, double y, double z, double cx, double cy,
                                           double cz) {
  double dx = __dsub_rn(x, cx), dy = __dsub_rn(y, cy), dz = __dsub_rn(z, cz);
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Longest side of a bounding box; ties go to the lowest axis.
__device__ __forceinline__ int longest_axis(const double lo[3], const double hi[3]) {
  double e0 = __dsub_rn(hi[0], lo[0]), e1 = __dsub_rn(hi[1], lo[1]), e2 = __dsub_rn(hi[2], lo[2]);
  int axis = 0;
  double best = e0;
  if (e1 > best) { axis = 1; best = e1; }
  if (e2 > best) { axis = 2; }
  return axis;
}

// Error-free transformation a + b = s + e (Knuth two-sum), float32.
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (hi, lo) += v with the rounding error of the high part carried in lo.
__device__ __forceinline__ void df_add(float& hi, float& lo, float v) {
  float s, e;
  two_sum(hi, v, s, e);
  hi = s;
  lo = __fadd_rn(lo, e);
}
// (hi, lo) += (bh, bl)
__device__ __forceinline__ void df_add2(float& hi, float& lo, float bh, float bl) {
  float s, e;
  two_sum(hi, bh, s, e);
  hi = s;
  lo = __fadd_rn(__fadd_rn(lo, bl), e);
}
__device__ __forceinline__ void two_sum_d(double a, double b, double& s, double& e) {
  s = __dadd_rn(a, b);
  double bb = __dsub_rn(s, a);
  e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
}

// System holding particle position p (caller order) of a forest: the largest
// k with off[k] <= p (every system holds at least one particle).
__device__ __forceinline__ int system_of(const int64_t* __restrict__ off, int n_sys, int64_t p) {
  int lo = 0, hi = n_sys - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (off[mid] <= p) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// ---------------------------------------------------------------------------
// Host-side launchers (defined in the .cu files)
// ---------------------------------------------------------------------------
int build_tree(kdfmm_tree_s* t, const double* x, const double* m, const double* h,
               cudaStream_t s, int fixed_levels);
int recompute_moments(kdfmm_tree_s* t, const double* x, const double* m, const double* h,
                      cudaStream_t s);
int run_walk(kdfmm_tree_s* t, cudaStream_t s);
// walk into the current slot capacities without synchronising or allocating
// (ensure_slots first; overflow is flagged in the status word)
int ensure_slots(kdfmm_tree_s* t, int slot_leaves);
int walk_fixed(kdfmm_tree_s* t, int slot_leaves, cudaStream_t s);
// Arena mode: list buffers for `extra` times the last walk's entries and the
// scratch of an arena walk over `leaves` leaves (before a capture).
int ensure_arena(kdfmm_tree_s* t, int leaves, double extra);
int run_m2l(kdfmm_tree_s* t, cudaStream_t s);
int run_m2l_cells(kdfmm_tree_s* t, const int32_t* far_cnt, const int64_t* far_off,
                  const int32_t* far_idx, float* out32, double* out64, cudaStream_t s);
// symmetric dual-tree walk: lists (per-cell far, per-leaf near), then the
// per-cell M2L and the translation of every cell's expansion to its leaves
int run_dual_walk(kdfmm_tree_s* t, cudaStream_t s);
int run_dual_local(kdfmm_tree_s* t, cudaStream_t s);
void free_dual(kdfmm_tree_s* t);
int run_p2p(kdfmm_tree_s* t, double* a, double* phi, cudaStream_t s);
// Extra P2P segments: storage for `need`, an upper bound from the last walk's
// list sizes, and the plan (run by run_p2p; the adjoint reuses it).
int ensure_segments(kdfmm_tree_s* t, int64_t need);
int64_t segments_bound(const kdfmm_tree_s* t);
int plan_segments(kdfmm_tree_s* t, cudaStream_t s);
int run_vjp(kdfmm_tree_s* t, const double* a_bar, double* x_bar, double* m_bar, cudaStream_t s);
int momentum(const double* m, const double* v, int64_t n, double* out, double* scratch,
             cudaStream_t s);
// exclusive scan of n int32 (out may alias in); returns the total in *total_dev
void scan_i32(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, cudaStream_t s);
// the same with the count read from device memory (*n_dev <= cap)
void scan_i32_dev(const int32_t* in, int32_t* out, const int32_t* n_dev, int64_t cap, int32_t* tmp,
                  cudaStream_t s);
void scan_i32_to_i64(const int32_t* in, int64_t* out, int64_t n, int64_t* tmp, cudaStream_t s);
int64_t scan_tmp_elems(int64_t n);

// tracing (api.cu): CUDA events around a phase when timing is enabled
void phase_begin(kdfmm_tree_s* t, int phase, cudaStream_t s);
void phase_end(kdfmm_tree_s* t, int phase, cudaStream_t s);

// error plumbing (api.cu)
int set_error(int code, const char* fmt, ...);
int check_cuda(cudaError_t e, const char* what);

}  // namespace kdfmm
