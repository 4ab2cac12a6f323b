// C ABI of the kdfmm library (declared in include/kdfmm.h): argument
// checking, device buffers owned by the handle, and the order of the steps of
// one force evaluation.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <vector>

#include "kdfmm_internal.cuh"

namespace kdfmm {

void free_build_buffers(kdfmm_tree_s* t);
int64_t momentum_blocks(int64_t n);

namespace {
thread_local char g_err[512] = "";

bool is_device_ptr(const void* p) {
  if (p == nullptr) return false;
  cudaPointerAttributes attr;
  if (cudaPointerGetAttributes(&attr, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return attr.type == cudaMemoryTypeDevice || attr.type == cudaMemoryTypeManaged;
}

int check_params(const kdfmm_params* p, const double* h) {
  if (!p) return set_error(KDFMM_ERR_INVALID_ARG, "params is NULL");
  if (!(p->theta >= 0.0 && p->theta <= 1.0))
    return set_error(KDFMM_ERR_INVALID_ARG, "theta must lie in [0, 1] (got %g)", p->theta);
  if (p->n_leaf < 1 || p->n_leaf > KDFMM_MAX_LEAF)
    return set_error(KDFMM_ERR_INVALID_ARG, "n_leaf must lie in [1, %d] (got %d)", KDFMM_MAX_LEAF,
                     p->n_leaf);
  if (p->soft_kind != KDFMM_SOFT_PLUMMER && p->soft_kind != KDFMM_SOFT_M4)
    return set_error(KDFMM_ERR_INVALID_ARG, "unknown soft_kind %d", p->soft_kind);
  if (p->precision != KDFMM_FP64 && p->precision != KDFMM_MIXED)
    return set_error(KDFMM_ERR_INVALID_ARG, "unknown precision %d", p->precision);
  if (!(std::isfinite(p->eps) && p->eps >= 0.0))
    return set_error(KDFMM_ERR_INVALID_ARG, "eps must be finite and >= 0");
  if (!(std::isfinite(p->r_kern) && p->r_kern >= 0.0))
    return set_error(KDFMM_ERR_INVALID_ARG, "r_kern must be finite and >= 0");
  if (p->expansion != KDFMM_EXPANSION_PHANTOM && p->expansion != KDFMM_EXPANSION_STANDARD)
    return set_error(KDFMM_ERR_INVALID_ARG, "unknown expansion %d", p->expansion);
  if (p->walk != KDFMM_WALK_LEAF && p->walk != KDFMM_WALK_DUAL)
    return set_error(KDFMM_ERR_INVALID_ARG, "unknown walk %d", p->walk);
  if (p->reserved != 0) return set_error(KDFMM_ERR_INVALID_ARG, "reserved must be 0");
  if (p->soft_kind == KDFMM_SOFT_M4 && h == nullptr)
    return set_error(KDFMM_ERR_INVALID_ARG, "M4 kernel softening needs smoothing lengths h");
  return KDFMM_OK;
}

}  // namespace

int set_error(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

int sm_count() {
  static int cached[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return 1;
  }
  if (cached[dev] == 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) {
      cudaGetLastError();
      n = 1;
    }
    cached[dev] = n;
  }
  return cached[dev];
}

int check_cuda(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return KDFMM_OK;
  return set_error(KDFMM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

void phase_begin(kdfmm_tree_s* t, int phase, cudaStream_t s) {
  if (!t->timing) return;
  if (!t->ev[2 * phase]) {
    cudaEventCreate(&t->ev[2 * phase]);
    cudaEventCreate(&t->ev[2 * phase + 1]);
  }
  cudaEventRecord(t->ev[2 * phase], s);
}

void phase_end(kdfmm_tree_s* t, int phase, cudaStream_t s) {
  if (!t->timing || !t->ev[2 * phase + 1]) return;
  cudaEventRecord(t->ev[2 * phase + 1], s);
  t->ev_used[phase] = true;
}

static int grow_eval_buffers(kdfmm_tree_s* t, int64_t cap) {
  Lists& L = t->L;
  cudaFree(L.far_cnt); cudaFree(L.near_cnt); cudaFree(L.far_off); cudaFree(L.near_off);
  cudaFree(L.heavy); cudaFree(L.seg_first);
  L.far_cnt = L.near_cnt = L.heavy = L.seg_first = nullptr;
  L.far_off = L.near_off = nullptr;
  if (cudaMalloc(&L.far_cnt, (cap + 1) * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&L.near_cnt, (cap + 1) * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&L.far_off, (cap + 2) * sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc(&L.near_off, (cap + 2) * sizeof(int64_t)) != cudaSuccess ||
      cudaMalloc(&L.heavy, (cap + 1) * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&L.seg_first, (cap + 1) * sizeof(int32_t)) != cudaSuccess)
    return set_error(KDFMM_ERR_OOM, "interaction list offsets");
  // leaves that a walk skipped keep empty lists
  cudaMemset(L.far_cnt, 0, (cap + 1) * sizeof(int32_t));
  cudaMemset(L.near_cnt, 0, (cap + 1) * sizeof(int32_t));
  cudaMemset(L.far_off, 0, (cap + 2) * sizeof(int64_t));
  cudaMemset(L.near_off, 0, (cap + 2) * sizeof(int64_t));
  return KDFMM_OK;
}

// Per-system parameters on the device (a single tree is a forest of one).
// Host arrays are staged through pinned memory owned by the handle.
static int set_systems(kdfmm_tree_s* t, const int64_t* off, int32_t n_sys, const double* theta,
                       const double* eps, const int32_t* nleaf, const kdfmm_params* p,
                       cudaStream_t s) {
  if (n_sys > t->cap_sys) {
    cudaStreamSynchronize(s);
    cudaFree(t->sys_off); cudaFree(t->sys_theta); cudaFree(t->sys_eps); cudaFree(t->sys_nleaf);
    cudaFree(t->sys_root);
    if (t->host_sys_off) cudaFreeHost(t->host_sys_off);
    t->sys_off = nullptr; t->sys_theta = t->sys_eps = nullptr;
    t->sys_nleaf = t->sys_root = nullptr;
    t->host_sys_off = nullptr;
    t->cap_sys = 0;
    t->n_sys = 0;
    const size_t k = (size_t)n_sys + 1;
    if (cudaMalloc(&t->sys_off, k * sizeof(int64_t)) != cudaSuccess ||
        cudaMalloc(&t->sys_theta, k * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&t->sys_eps, k * sizeof(double)) != cudaSuccess ||
        cudaMalloc(&t->sys_nleaf, k * sizeof(int32_t)) != cudaSuccess ||
        cudaMalloc(&t->sys_root, k * sizeof(int32_t)) != cudaSuccess ||
        cudaHostAlloc(&t->host_sys_off, k * (2 * sizeof(int64_t) + 2 * sizeof(double)), 0) !=
            cudaSuccess)
      return set_error(KDFMM_ERR_OOM, "system tables (%d systems)", n_sys);
    t->cap_sys = n_sys;
  }
  const size_t k = (size_t)t->cap_sys + 1;
  int64_t* ho = t->host_sys_off;
  double* ht = reinterpret_cast<double*>(ho + k);
  double* he = ht + k;
  int32_t* hn = reinterpret_cast<int32_t*>(he + k);
  // the staged copy of the previous call has completed (every build synchronises)
  bool same = t->n_sys == n_sys;
  for (int32_t i = 0; same && i <= n_sys; ++i) same = ho[i] == off[i];
  for (int32_t i = 0; same && i < n_sys; ++i)
    same = ht[i] == (theta ? theta[i] : p->theta) && he[i] == (eps ? eps[i] : p->eps) &&
           hn[i] == (nleaf ? nleaf[i] : p->n_leaf);
  if (same) return KDFMM_OK;
  int32_t mn = KDFMM_MAX_LEAF;
  for (int32_t i = 0; i <= n_sys; ++i) ho[i] = off[i];
  for (int32_t i = 0; i < n_sys; ++i) {
    ht[i] = theta ? theta[i] : p->theta;
    he[i] = eps ? eps[i] : p->eps;
    hn[i] = nleaf ? nleaf[i] : p->n_leaf;
    mn = std::min(mn, hn[i]);
  }
  t->n_sys = n_sys;
  t->min_nleaf = mn;
  int rc = check_cuda(cudaMemcpyAsync(t->sys_off, ho, k * sizeof(int64_t), cudaMemcpyHostToDevice, s),
                      "system offsets");
  if (!rc) rc = check_cuda(cudaMemcpyAsync(t->sys_theta, ht, n_sys * sizeof(double),
                                           cudaMemcpyHostToDevice, s), "system theta");
  if (!rc) rc = check_cuda(cudaMemcpyAsync(t->sys_eps, he, n_sys * sizeof(double),
                                           cudaMemcpyHostToDevice, s), "system eps");
  if (!rc) rc = check_cuda(cudaMemcpyAsync(t->sys_nleaf, hn, n_sys * sizeof(int32_t),
                                           cudaMemcpyHostToDevice, s), "system n_leaf");
  return rc;
}

static int check_systems(const int64_t* off, int32_t n_sys, const double* theta, const double* eps,
                         const int32_t* nleaf) {
  if (n_sys < 1) return set_error(KDFMM_ERR_INVALID_ARG, "n_sys must be >= 1 (got %d)", n_sys);
  if (!off) return set_error(KDFMM_ERR_INVALID_ARG, "sys_offset is NULL");
  if (off[0] != 0) return set_error(KDFMM_ERR_INVALID_ARG, "sys_offset[0] must be 0");
  for (int32_t i = 0; i < n_sys; ++i) {
    if (off[i + 1] <= off[i])
      return set_error(KDFMM_ERR_INVALID_ARG, "system %d is empty or sys_offset decreases", i);
    if (theta && !(theta[i] >= 0.0 && theta[i] <= 1.0))
      return set_error(KDFMM_ERR_INVALID_ARG, "theta[%d] must lie in [0, 1] (got %g)", i, theta[i]);
    if (eps && !(std::isfinite(eps[i]) && eps[i] >= 0.0))
      return set_error(KDFMM_ERR_INVALID_ARG, "eps[%d] must be finite and >= 0", i);
    if (nleaf && (nleaf[i] < 1 || nleaf[i] > KDFMM_MAX_LEAF))
      return set_error(KDFMM_ERR_INVALID_ARG, "n_leaf[%d] must lie in [1, %d] (got %d)", i,
                       KDFMM_MAX_LEAF, nleaf[i]);
  }
  if (off[n_sys] > (int64_t(1) << 30))
    return set_error(KDFMM_ERR_INVALID_ARG, "total particle count above 2^30");
  return KDFMM_OK;
}

// Builds the forest whose systems set_systems has just described.
static int build_common(kdfmm_tree_s* t, const double* x, const double* m, const double* h,
                        int64_t n, const kdfmm_params* p, cudaStream_t s) {
  t->built = t->evaluated = t->lists_frozen = false;
  t->n = n;
  t->p = *p;
  const int64_t old_cap = t->cap_n;
  int rc;
  phase_begin(t, KDFMM_PHASE_BUILD, s);
  // After a first build the handle knows how many phase-A levels a tree of
  // this kind needs: build without synchronising (one more level as margin)
  // and read the counters once; a tree that needed more levels is rebuilt
  // with the host following the counters.
  bool done = false;
  if (t->levels_used > 0 && t->cap_n >= n) {
    if ((rc = build_tree(t, x, m, h, s, t->levels_used + 1))) return rc;
    int32_t* hc = t->host_counters;
    cudaMemcpyAsync(hc, t->counters, 32 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&hc[32], t->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if ((rc = check_cuda(cudaStreamSynchronize(s), "build"))) return rc;
    const int32_t st = hc[32];
    if (st & ST_NONFINITE)
      return set_error(KDFMM_ERR_NONFINITE, "non-finite position or non-positive mass / h");
    if (st & ST_INTERNAL) return set_error(KDFMM_ERR_INTERNAL, "pre-order numbering inconsistent");
    if (!(st & (ST_UNFINISHED | ST_CAPACITY))) {
      t->ncells = hc[C_CELLS];
      t->nleaves = hc[C_LEAVES];
      t->depth = hc[C_DEPTH];
      t->nfallback = hc[C_FALLBACK];
      done = true;
    }
  }
  if (!done && (rc = build_tree(t, x, m, h, s, 0))) return rc;
  phase_end(t, KDFMM_PHASE_BUILD, s);
  t->grid_leaves = t->nleaves;
  if (t->cap_n != old_cap || t->L.far_cnt == nullptr)
    if ((rc = grow_eval_buffers(t, t->cap_n))) return rc;
  t->built = true;
  int64_t* hs = t->host_stats;
  hs[KDFMM_STAT_N] = n;
  hs[KDFMM_STAT_NCELLS] = t->ncells;
  hs[KDFMM_STAT_NLEAVES] = t->nleaves;
  hs[KDFMM_STAT_DEPTH] = t->depth;
  hs[KDFMM_STAT_NFAR] = hs[KDFMM_STAT_NNEAR] = hs[KDFMM_STAT_NP2P] = 0;
  hs[KDFMM_STAT_NFALLBACK] = t->nfallback;
  hs[KDFMM_STAT_NEXACT] = hs[KDFMM_STAT_NHEAVY] = 0;
  return KDFMM_OK;
}

// ---------------------------------------------------------------------------
// Captured evaluation.  The first kdfmm_fmm_accel_batched call for a set of
// buffers runs eagerly (the host follows the device counters); its sizes,
// with margins, fix a sequence of launches that needs no host decision
// (phase-A levels, list slots, leaves), which is captured into a CUDA graph
// on a private stream.  Later calls with the same buffers replay the graph
// and read the counters once; a replay whose tree needed more levels, more
// leaves or longer lists than the graph allows is redone eagerly and the
// graph captured again.  KDFMM_GRAPH=0 in the environment turns this off.
// ---------------------------------------------------------------------------
static bool graphs_enabled() {
  const char* v = getenv("KDFMM_GRAPH");
  return !(v != nullptr && strcmp(v, "0") == 0);
}

static void graph_drop(kdfmm_tree_s* t) {
  if (t->graph_exec) cudaGraphExecDestroy(t->graph_exec);
  t->graph_exec = nullptr;
}

static kdfmm_tree_s::GraphKey graph_key_of(const kdfmm_tree_s* t, const double* x, const double* m,
                                           const double* h, double* a, double* phi) {
  kdfmm_tree_s::GraphKey k{};
  k.x = x; k.m = m; k.h = h; k.a = a; k.phi = phi;
  k.n = t->n; k.cap_n = t->cap_n;
  k.cap_far = t->L.cap_far; k.cap_near = t->L.cap_near;
  k.far_cap = t->L.far_cap; k.near_cap = t->L.near_cap; k.seg_cap = t->L.seg_cap;
  k.temp_cap = t->L.temp_cap; k.arena = t->L.arena; k.arena_grid = t->L.arena_grid;
  k.n_sys = t->n_sys; k.cap_sys = t->cap_sys; k.min_nleaf = t->min_nleaf;
  k.soft_kind = t->p.soft_kind; k.precision = t->p.precision; k.r_kern = t->p.r_kern;
  k.expansion = t->p.expansion; k.walk = t->p.walk; k.budget = t->walk_budget;
  return k;
}

// Build (fixed levels), walk (fixed slots), M2L and P2P, with no
// synchronisation and no allocation.
static int enqueue_fixed(kdfmm_tree_s* t, const double* x, const double* m, const double* h,
                         double* a, double* phi, cudaStream_t s) {
  int rc = build_tree(t, x, m, h, s, t->graph_levels);
  if (rc) return rc;
  t->grid_leaves = t->graph_leaves;
  if ((rc = walk_fixed(t, t->graph_leaves, s))) return rc;
  if ((rc = run_m2l(t, s))) return rc;
  return run_p2p(t, a, phi, s);
}

// Captures the fixed sequence sized from the eager evaluation just done.
// A capture that fails leaves the handle without a graph (eager calls).
static void graph_capture(kdfmm_tree_s* t, const double* x, const double* m, const double* h,
                          double* a, double* phi, cudaStream_t s) {
  graph_drop(t);
  if (t->p.walk != KDFMM_WALK_LEAF) return;        // the dual walk's queues follow the host
  if (cudaStreamSynchronize(s) != cudaSuccess) {   // the lists may be copied to larger slots
    cudaGetLastError();
    return;
  }
  if (t->L.exact && !t->L.arena) return;  // lists made by the host between passes
  if (!t->capture_stream &&
      cudaStreamCreateWithFlags(&t->capture_stream, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  t->graph_levels = t->levels_used + 2;
  t->graph_leaves = (int32_t)std::min<int64_t>(t->n, (int64_t)t->nleaves + t->nleaves / 4 + 64);
  if (t->L.arena ? ensure_arena(t, t->graph_leaves, 1.25) : ensure_slots(t, t->graph_leaves)) return;
  if (ensure_segments(t, segments_bound(t) + segments_bound(t) / 4)) return;
  const int32_t grid_eager = t->grid_leaves;
  const int64_t launches0 = t->launches;
  const bool timing = t->timing;
  t->timing = false;
  cudaStream_t cs = t->capture_stream;
  cudaGraph_t g = nullptr;
  int rc = KDFMM_OK;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
    rc = enqueue_fixed(t, x, m, h, a, phi, cs);
    if (cudaStreamEndCapture(cs, &g) != cudaSuccess) rc = KDFMM_ERR_CUDA;
  } else {
    rc = KDFMM_ERR_CUDA;
  }
  if (rc == KDFMM_OK && g != nullptr &&
      cudaGraphInstantiate(&t->graph_exec, g, 0) == cudaSuccess) {
    t->graph_key = graph_key_of(t, x, m, h, a, phi);
    t->graph_launches = t->launches - launches0;
  } else {
    t->graph_exec = nullptr;
  }
  if (g) cudaGraphDestroy(g);
  cudaGetLastError();
  t->launches = launches0;                // captured launches have not run
  t->grid_leaves = grid_eager;
  t->timing = timing;
}

// Replays the graph; 0: done, 1: the tree outgrew the graph (redo eagerly),
// < 0: error.
static int graph_replay(kdfmm_tree_s* t, cudaStream_t s) {
  int rc = check_cuda(cudaGraphLaunch(t->graph_exec, s), "graph launch");
  if (rc) return rc;
  t->launches += t->graph_launches;
  int32_t* hc = t->host_counters;
  cudaMemcpyAsync(hc, t->counters, 32 * sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(&hc[32], t->status, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
  cudaMemcpyAsync(t->host_stats + 16, t->L.near_np, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost, s);
  if ((rc = check_cuda(cudaStreamSynchronize(s), "graph replay"))) return rc;
  const int32_t st = hc[32];
  t->built = t->evaluated = t->lists_frozen = false;
  if (st & ST_NONFINITE)
    return set_error(KDFMM_ERR_NONFINITE, "non-finite position or non-positive mass / h");
  // more leaves than the captured launches cover (M2L and P2P stop at
  // graph_leaves) is redone eagerly too
  if ((st & (ST_UNFINISHED | ST_LISTS | ST_CAPACITY | ST_INTERNAL)) ||
      hc[C_LEAVES] > t->graph_leaves ||
      (!t->L.arena && (hc[C_MAXFAR] > t->L.cap_far || hc[C_MAXNEAR] > t->L.cap_near)))
    return 1;
  t->ncells = hc[C_CELLS];
  t->nleaves = hc[C_LEAVES];
  t->depth = hc[C_DEPTH];
  t->nfallback = hc[C_FALLBACK];
  t->grid_leaves = t->graph_leaves;
  t->built = t->evaluated = true;
  int64_t* hs = t->host_stats;
  hs[KDFMM_STAT_N] = t->n;
  hs[KDFMM_STAT_NCELLS] = t->ncells;
  hs[KDFMM_STAT_NLEAVES] = t->nleaves;
  hs[KDFMM_STAT_DEPTH] = t->depth;
  hs[KDFMM_STAT_NFALLBACK] = t->nfallback;
  hs[KDFMM_STAT_NFAR] = hs[16 + 2];
  hs[KDFMM_STAT_NNEAR] = hs[16 + 3];
  return 0;
}

}  // namespace kdfmm

using namespace kdfmm;

extern "C" {

const char* kdfmm_last_error(void) { return g_err; }

int kdfmm_tree_create(kdfmm_tree* out) {
  if (!out) return set_error(KDFMM_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  kdfmm_tree_s* t = new (std::nothrow) kdfmm_tree_s();
  if (!t) return set_error(KDFMM_ERR_OOM, "handle allocation");
  int rc = check_cuda(cudaGetDevice(&t->device), "cudaGetDevice");
  if (!rc) rc = check_cuda(cudaMalloc(&t->counters, 32 * sizeof(int32_t)), "counters");
  if (!rc) rc = check_cuda(cudaMalloc(&t->status, sizeof(int32_t)), "status");
  if (!rc) rc = check_cuda(cudaMalloc(&t->com_bound, sizeof(float)), "bound");
  if (!rc) rc = check_cuda(cudaMalloc(&t->L.near_np, 4 * sizeof(int64_t)), "stats");
  if (!rc) rc = check_cuda(cudaHostAlloc(&t->host_stats, 64 * sizeof(int64_t), 0), "host stats");
  if (!rc) rc = check_cuda(cudaHostAlloc(&t->host_counters, 64 * sizeof(int32_t), 0), "host counters");
  if (rc) {
    kdfmm_tree_destroy(t);
    return rc;
  }
  memset(t->host_stats, 0, 64 * sizeof(int64_t));
  *out = t;
  return KDFMM_OK;
}

void kdfmm_tree_destroy(kdfmm_tree t) {
  if (!t) return;
  int dev = 0;
  cudaGetDevice(&dev);
  cudaSetDevice(t->device);
  cudaDeviceSynchronize();
  free_build_buffers(t);
  cudaFree(t->counters); cudaFree(t->status); cudaFree(t->com_bound);
  cudaFree(t->L.far_cnt); cudaFree(t->L.near_cnt); cudaFree(t->L.far_off); cudaFree(t->L.near_off);
  cudaFree(t->L.far_idx); cudaFree(t->L.near_idx); cudaFree(t->L.near_np);
  cudaFree(t->L.heavy); cudaFree(t->L.seg_first); cudaFree(t->L.seg_leaf); cudaFree(t->L.seg_part);
  cudaFree(t->L.temp);
  cudaFree(t->mom_partial);
  cudaFree(t->sys_off); cudaFree(t->sys_theta); cudaFree(t->sys_eps); cudaFree(t->sys_nleaf);
  cudaFree(t->sys_root);
  if (t->host_sys_off) cudaFreeHost(t->host_sys_off);
  graph_drop(t);
  if (t->capture_stream) cudaStreamDestroy(t->capture_stream);
  free_dual(t);
  for (cudaEvent_t& e : t->ev)
    if (e) cudaEventDestroy(e);
  if (t->host_stats) cudaFreeHost(t->host_stats);
  if (t->host_counters) cudaFreeHost(t->host_counters);
  cudaGetLastError();
  cudaSetDevice(dev);
  delete t;
}

int kdfmm_tree_build(kdfmm_tree t, const double* x, const double* m, const double* h, int64_t n,
                     const kdfmm_params* p, void* stream) {
  if (!t) return set_error(KDFMM_ERR_INVALID_ARG, "tree is NULL");
  int rc = check_params(p, h);
  if (rc) return rc;
  if (n < 1 || n > (int64_t(1) << 30))
    return set_error(KDFMM_ERR_INVALID_ARG, "n must lie in [1, 2^30] (got %lld)", (long long)n);
  if (!is_device_ptr(x) || !is_device_ptr(m) || (h != nullptr && !is_device_ptr(h)))
    return set_error(KDFMM_ERR_INVALID_ARG, "x, m (and h) must be device pointers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != t->device) return set_error(KDFMM_ERR_INVALID_ARG, "handle belongs to device %d", t->device);
  const int64_t off[2] = {0, n};
  if ((rc = set_systems(t, off, 1, nullptr, nullptr, nullptr, p, s))) return rc;
  return build_common(t, x, m, h, n, p, s);
}

int kdfmm_forest_build(kdfmm_tree t, const double* x, const double* m, const double* h,
                       const int64_t* sys_offset, int32_t n_sys, const double* theta,
                       const double* eps, const int32_t* n_leaf, const kdfmm_params* p,
                       void* stream) {
  // host-side arguments first: they need no device
  int rc = check_params(p, h);
  if (rc) return rc;
  if ((rc = check_systems(sys_offset, n_sys, theta, eps, n_leaf))) return rc;
  if (!t) return set_error(KDFMM_ERR_INVALID_ARG, "tree is NULL");
  if (!is_device_ptr(x) || !is_device_ptr(m) || (h != nullptr && !is_device_ptr(h)))
    return set_error(KDFMM_ERR_INVALID_ARG, "x, m (and h) must be device pointers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != t->device) return set_error(KDFMM_ERR_INVALID_ARG, "handle belongs to device %d", t->device);
  if ((rc = set_systems(t, sys_offset, n_sys, theta, eps, n_leaf, p, s))) return rc;
  return build_common(t, x, m, h, sys_offset[n_sys], p, s);
}

int kdfmm_fmm_accel_batched(kdfmm_tree t, const double* x, const double* m, const double* h,
                            const int64_t* sys_offset, int32_t n_sys, const double* theta,
                            const double* eps, const int32_t* n_leaf, const kdfmm_params* p,
                            double* a, double* phi, void* stream) {
  int rc = check_params(p, h);
  if (rc) return rc;
  if ((rc = check_systems(sys_offset, n_sys, theta, eps, n_leaf))) return rc;
  if (!t) return set_error(KDFMM_ERR_INVALID_ARG, "tree is NULL");
  if (!is_device_ptr(x) || !is_device_ptr(m) || (h != nullptr && !is_device_ptr(h)) ||
      !is_device_ptr(a) || (phi != nullptr && !is_device_ptr(phi)))
    return set_error(KDFMM_ERR_INVALID_ARG, "x, m, a (and h, phi) must be device pointers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev != t->device) return set_error(KDFMM_ERR_INVALID_ARG, "handle belongs to device %d", t->device);
  const bool graphs = graphs_enabled();
  if (graphs && t->graph_exec) {
    if ((rc = set_systems(t, sys_offset, n_sys, theta, eps, n_leaf, p, s))) return rc;
    t->n = sys_offset[n_sys];
    t->p = *p;
    if (graph_key_of(t, x, m, h, a, phi) == t->graph_key) {
      rc = graph_replay(t, s);
      if (rc <= 0) return rc;
    }
    graph_drop(t);                       // outgrown or other buffers: eager, then capture again
  }
  if ((rc = kdfmm_forest_build(t, x, m, h, sys_offset, n_sys, theta, eps, n_leaf, p, stream)))
    return rc;
  if ((rc = kdfmm_fmm_accel(t, a, phi, stream))) return rc;
  if (graphs) graph_capture(t, x, m, h, a, phi, s);
  return KDFMM_OK;
}

int kdfmm_tree_moments(kdfmm_tree t, const double* x, const double* m, const double* h,
                       void* stream) {
  if (!t || !t->built) return set_error(KDFMM_ERR_INVALID_ARG, "tree not built");
  if (!is_device_ptr(x) || !is_device_ptr(m) || (h != nullptr && !is_device_ptr(h)))
    return set_error(KDFMM_ERR_INVALID_ARG, "x, m (and h) must be device pointers");
  if (t->p.soft_kind == KDFMM_SOFT_M4 && h == nullptr)
    return set_error(KDFMM_ERR_INVALID_ARG, "M4 kernel softening needs smoothing lengths h");
  if (!t->evaluated && !t->lists_frozen)
    return set_error(KDFMM_ERR_INVALID_ARG, "evaluate once (kdfmm_fmm_accel) before freezing the lists");
  int rc = recompute_moments(t, x, m, h, static_cast<cudaStream_t>(stream));
  if (rc) return rc;
  t->lists_frozen = true;
  return KDFMM_OK;
}

int kdfmm_fmm_accel(kdfmm_tree t, double* a, double* phi, void* stream) {
  if (!t || !t->built) return set_error(KDFMM_ERR_INVALID_ARG, "tree not built");
  if (!is_device_ptr(a) || (phi != nullptr && !is_device_ptr(phi)))
    return set_error(KDFMM_ERR_INVALID_ARG, "a (and phi) must be device pointers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int rc = KDFMM_OK;
  const bool dual = t->p.walk == KDFMM_WALK_DUAL;
  if (!t->lists_frozen) {              // after kdfmm_tree_moments the lists stay as they were
    phase_begin(t, KDFMM_PHASE_WALK, s);
    if ((rc = dual ? run_dual_walk(t, s) : run_walk(t, s))) return rc;
    phase_end(t, KDFMM_PHASE_WALK, s);
  }
  phase_begin(t, KDFMM_PHASE_M2L, s);
  if ((rc = dual ? run_dual_local(t, s) : run_m2l(t, s))) return rc;
  phase_end(t, KDFMM_PHASE_M2L, s);
  phase_begin(t, KDFMM_PHASE_P2P, s);
  if ((rc = ensure_segments(t, segments_bound(t)))) return rc;
  if ((rc = run_p2p(t, a, phi, s))) return rc;
  phase_end(t, KDFMM_PHASE_P2P, s);
  t->evaluated = true;
  return KDFMM_OK;
}

int kdfmm_total_momentum(const double* m, const double* v, int64_t n, double* out, void* stream) {
  if (n < 1) return set_error(KDFMM_ERR_INVALID_ARG, "n must be >= 1");
  if (!is_device_ptr(m) || !is_device_ptr(v) || !is_device_ptr(out))
    return set_error(KDFMM_ERR_INVALID_ARG, "m, v and out must be device pointers");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t nb = momentum_blocks(n);
  double* scratch = nullptr;
  int rc = check_cuda(cudaMallocAsync(&scratch, (size_t)nb * 6 * sizeof(double), s), "momentum scratch");
  if (rc) return rc;
  rc = momentum(m, v, n, out, scratch, s);
  cudaFreeAsync(scratch, s);
  return rc;
}

int kdfmm_tree_stats(kdfmm_tree t, int64_t* stats) {
  if (!t || !stats) return set_error(KDFMM_ERR_INVALID_ARG, "NULL argument");
  int64_t* hs = t->host_stats;
  if (t->evaluated) {
    int64_t dev[4] = {0, 0, 0, 0};
    int rc = check_cuda(cudaMemcpy(dev, t->L.near_np, 4 * sizeof(int64_t), cudaMemcpyDeviceToHost),
                        "stats copy");
    if (rc) return rc;
    hs[KDFMM_STAT_NP2P] = dev[0];
    hs[KDFMM_STAT_NEXACT] = dev[1];
    int32_t heavy = 0;
    if (t->p.walk == KDFMM_WALK_LEAF &&
        (rc = check_cuda(cudaMemcpy(&heavy, t->counters + C_HEAVY, sizeof(int32_t),
                                    cudaMemcpyDeviceToHost), "stats copy")))
      return rc;
    hs[KDFMM_STAT_NHEAVY] = heavy;
  }
  hs[KDFMM_STAT_LAUNCHES] = t->launches;
  memcpy(stats, hs, KDFMM_NSTATS * sizeof(int64_t));
  return KDFMM_OK;
}

int kdfmm_tree_set_walk_budget(kdfmm_tree t, int32_t budget) {
  if (!t) return set_error(KDFMM_ERR_INVALID_ARG, "tree is NULL");
  if (budget < 0 || budget > (1 << 20))
    return set_error(KDFMM_ERR_INVALID_ARG, "walk budget %d outside [0, 2^20]", (int)budget);
  t->walk_budget = budget;
  return KDFMM_OK;
}

int kdfmm_tree_timing(kdfmm_tree t, int enable, float* ms) {
  if (!t) return set_error(KDFMM_ERR_INVALID_ARG, "tree is NULL");
  if (ms) {
    for (int k = 0; k < KDFMM_NPHASES; ++k) {
      ms[k] = 0.0f;
      if (!t->ev_used[k]) continue;
      int rc = check_cuda(cudaEventSynchronize(t->ev[2 * k + 1]), "timing sync");
      if (rc) return rc;
      rc = check_cuda(cudaEventElapsedTime(&ms[k], t->ev[2 * k], t->ev[2 * k + 1]), "elapsed");
      if (rc) return rc;
    }
  }
  t->timing = enable != 0;
  return KDFMM_OK;
}

int kdfmm_tree_export(kdfmm_tree t, int64_t* perm, int64_t* cell_ints, double* cell_reals,
                      int32_t* leaf_ids, int64_t* far_off, int32_t* far_idx, int64_t* near_off,
                      int32_t* near_idx) {
  if (!t || !t->built) return set_error(KDFMM_ERR_INVALID_ARG, "tree not built");
  int rc = check_cuda(cudaDeviceSynchronize(), "export sync");
  if (rc) return rc;
  const int64_t n = t->n, nc = t->ncells, nl = t->nleaves;
  auto D2H = [&](void* dst, const void* src, size_t bytes) {
    return check_cuda(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost), "export copy");
  };
  if (perm) {
    std::vector<int32_t> v(n);
    if ((rc = D2H(v.data(), t->tp.idx, n * sizeof(int32_t)))) return rc;
    for (int64_t i = 0; i < n; ++i) perm[i] = v[i];
  }
  if (cell_ints) {
    const int32_t* cols[7] = {t->c.first, t->c.count, t->c.left, t->c.right,
                              t->c.parent, t->c.depth, t->c.skip};
    std::vector<int32_t> v(nc);
    for (int k = 0; k < 7; ++k) {
      if ((rc = D2H(v.data(), cols[k], nc * sizeof(int32_t)))) return rc;
      for (int64_t c = 0; c < nc; ++c) cell_ints[7 * c + k] = v[c];
    }
  }
  if (cell_reals) {
    const double* cols[6] = {t->c.M, t->c.cx, t->c.cy, t->c.cz, t->c.s, t->c.hmax};
    std::vector<double> v(6 * nc);
    for (int k = 0; k < 6; ++k) {
      if ((rc = D2H(v.data(), cols[k], nc * sizeof(double)))) return rc;
      for (int64_t c = 0; c < nc; ++c) cell_reals[12 * c + k] = v[c];
    }
    if ((rc = D2H(v.data(), t->c.Q, 6 * nc * sizeof(double)))) return rc;
    for (int64_t c = 0; c < nc; ++c)
      for (int k = 0; k < 6; ++k) cell_reals[12 * c + 6 + k] = v[6 * c + k];
  }
  if (leaf_ids && (rc = D2H(leaf_ids, t->leaf_cells, nl * sizeof(int32_t)))) return rc;
  if (far_off || far_idx || near_off || near_idx) {
    if (!t->evaluated) return set_error(KDFMM_ERR_INVALID_ARG, "no evaluation to export lists from");
    // leaf walk: far and near lists per leaf; dual walk: far lists per cell
    // (nc rows), near lists per leaf.  Entries ascending in every list.
    const bool dual = t->p.walk == KDFMM_WALK_DUAL;
    const int64_t frows = dual ? nc : nl;
    std::vector<int32_t> fc(frows), nc_(nl);
    std::vector<int64_t> fst(frows), nst(nl);
    const int32_t* fcnt = dual ? t->dual.far_cnt : t->L.far_cnt;
    const int64_t* foff = dual ? t->dual.far_off : t->L.far_off;
    const int32_t* fidx = dual ? t->dual.far_idx : t->L.far_idx;
    const int64_t fcap = dual ? t->dual.far_idx_cap : t->L.far_cap;
    if ((rc = D2H(fc.data(), fcnt, frows * sizeof(int32_t)))) return rc;
    if ((rc = D2H(nc_.data(), t->L.near_cnt, nl * sizeof(int32_t)))) return rc;
    if ((rc = D2H(fst.data(), foff, frows * sizeof(int64_t)))) return rc;
    if ((rc = D2H(nst.data(), t->L.near_off, nl * sizeof(int64_t)))) return rc;
    std::vector<int32_t> fs, ns;
    if (far_idx) {
      fs.resize((size_t)fcap);
      if (fcap > 0 && (rc = D2H(fs.data(), fidx, fs.size() * sizeof(int32_t)))) return rc;
    }
    if (near_idx) {
      ns.resize((size_t)t->L.near_cap);
      if ((rc = D2H(ns.data(), t->L.near_idx, ns.size() * sizeof(int32_t)))) return rc;
    }
    int64_t fo = 0, no = 0;
    for (int64_t k = 0; k < frows; ++k) {
      if (far_off) far_off[k] = fo;
      if (far_idx) {
        memcpy(far_idx + fo, fs.data() + fst[k], fc[k] * sizeof(int32_t));
        if (dual) std::sort(far_idx + fo, far_idx + fo + fc[k]);
      }
      fo += fc[k];
    }
    for (int64_t k = 0; k < nl; ++k) {
      if (near_off) near_off[k] = no;
      if (near_idx) {
        memcpy(near_idx + no, ns.data() + nst[k], nc_[k] * sizeof(int32_t));
        if (dual) std::sort(near_idx + no, near_idx + no + nc_[k]);
      }
      no += nc_[k];
    }
    if (far_off) far_off[frows] = fo;
    if (near_off) near_off[nl] = no;
  }
  return KDFMM_OK;
}

int kdfmm_fmm_accel_vjp(kdfmm_tree t, const double* a_bar, double* x_bar, double* m_bar,
                        void* stream) {
  if (!t || !t->evaluated) return set_error(KDFMM_ERR_INVALID_ARG, "no evaluation to differentiate");
  if (t->p.walk != KDFMM_WALK_LEAF)
    return set_error(KDFMM_ERR_INVALID_ARG, "the adjoint covers the leaf-only walk only");
  if (!is_device_ptr(a_bar) || !is_device_ptr(x_bar) || !is_device_ptr(m_bar))
    return set_error(KDFMM_ERR_INVALID_ARG, "a_bar, x_bar and m_bar must be device pointers");
  return run_vjp(t, a_bar, x_bar, m_bar, static_cast<cudaStream_t>(stream));
}

}  // extern "C"
