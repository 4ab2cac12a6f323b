/*
 * kdfmm -- GB300 (sm_103a) kd-tree fast multipole gravity: C ABI.
 *
 * One gravitational force evaluation for N softened particles by the kd-tree
 * FMM analysed in Potashov & Yudin, arXiv 2502.01496 (Sec. 2 and Sec. 4):
 *   tree build     -- centre-of-mass cuts across the longest axis (Sec. 2);
 *   moments        -- M, centre of mass, size s, h_max, quadrupole Q (Eq. 7);
 *   walk           -- for every leaf only, opening criteria Eq. 4 and Eq. 5;
 *   M2L / L2P      -- Eq. 6 and its second-order Taylor expansion Eq. 8;
 *   P2P            -- softened direct sums over opened leaves (Eq. 13);
 *   assembly       -- a = a_short + a_long (Eq. 3), in caller order;
 *   total momentum -- sum_i m_i a_i, the paper's measure of non-conservation
 *                     (Sec. 4, Eq. 30).
 *
 * Conventions shared by every entry point:
 *   - Array arguments are DEVICE pointers to memory the caller owns, unless a
 *     parameter says "host".  Positions are N x 3 row-major float64
 *     (x0 y0 z0 x1 ...); masses, smoothing lengths and potentials are N float64.
 *     Outputs are written in the caller's particle order.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *     Work is enqueued on it; a call returns once its work is enqueued, except
 *     where a parameter says the call synchronises.
 *   - Every call returns a status code (KDFMM_OK or a negative KDFMM_ERR_*);
 *     nothing throws across the ABI.  kdfmm_last_error() returns a message for
 *     the calling thread's last failure.  After KDFMM_ERR_CUDA the handle must
 *     be destroyed.
 *   - G = 1 (Sec. 2, Eq. 1).
 */
#ifndef KDFMM_H
#define KDFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KDFMM_OK 0
#define KDFMM_ERR_INVALID_ARG (-1)  /* bad size, parameter or pointer */
#define KDFMM_ERR_CUDA (-2)         /* a CUDA runtime call failed */
#define KDFMM_ERR_OOM (-3)          /* device allocation failed */
#define KDFMM_ERR_TIMEOUT (-4)      /* a bounded device-side wait gave up */
#define KDFMM_ERR_CAPACITY (-5)     /* an internal list outgrew its capacity */
#define KDFMM_ERR_NONFINITE (-6)    /* NaN/Inf position, non-positive mass or h */
#define KDFMM_ERR_INTERNAL (-7)     /* a device-side consistency check failed */

#define KDFMM_SOFT_PLUMMER 0        /* a = -m d / (d^2 + eps^2)^(3/2); h_i = eps */
#define KDFMM_SOFT_M4 1             /* M4 cubic-spline kernel, per-particle h (Eq. 13) */

#define KDFMM_FP64 0                /* all force arithmetic in float64 */
#define KDFMM_MIXED 1               /* float32 P2P/M2L/L2P with compensated sums */

#define KDFMM_MAX_LEAF 32           /* largest supported n_leaf */

typedef struct kdfmm_tree_s* kdfmm_tree;   /* opaque, library-owned */

/* Far-field expansion.  PHANTOM: Eq. 6 and its first and second derivatives at
 * full order (Eq. 8; the quadrupole reaches the Hessian term, 1/r^6).
 * STANDARD: the standard p = 3 Cartesian series of the multipole section
 * (octupoles dropped; sink and source orders add up to at most p - 1 = 2 in
 * the acceleration), i.e. the quadrupole enters the acceleration at order 0
 * only (highest power of 1/r: 4).  The walk is the same leaf-only walk. */
#define KDFMM_EXPANSION_PHANTOM 0
#define KDFMM_EXPANSION_STANDARD 1

/* Walk.  LEAF: the paper's scheme -- every leaf walks the tree, super-cells
 * never do (Sec. 4), so interactions are one-sided and the total force does
 * not vanish.  DUAL: the symmetric dual-tree walk the paper's conclusions
 * point to (after Dehnen): cells interact in pairs, both ways -- M2L into both
 * cells when theta r > s_A + s_B and the smoothing spheres cannot meet, P2P
 * between the two leaves otherwise, else the larger cell splits -- and every
 * cell's expansion is translated down to the leaves (L2L).  Not the paper's
 * method; a separate mode.  The adjoint and captured graphs cover LEAF only. */
#define KDFMM_WALK_LEAF 0
#define KDFMM_WALK_DUAL 1

typedef struct {
    double theta;        /* opening parameter of Eq. 4, 0 <= theta <= 1 */
    double eps;          /* Plummer softening length (soft_kind 0); also h_i then */
    double r_kern;       /* kernel support radius in units of h in Eq. 5 (2 for M4) */
    int32_t n_leaf;      /* a cell holding more particles is split (Sec. 2); 1..32 */
    int32_t soft_kind;   /* KDFMM_SOFT_PLUMMER or KDFMM_SOFT_M4 */
    int32_t precision;   /* KDFMM_FP64 or KDFMM_MIXED */
    int32_t expansion;   /* KDFMM_EXPANSION_PHANTOM (0) or KDFMM_EXPANSION_STANDARD (1) */
    int32_t walk;        /* KDFMM_WALK_LEAF (0) or KDFMM_WALK_DUAL (1) */
    int32_t reserved;    /* must be 0 */
} kdfmm_params;

/* Statistics of the last build / evaluation (kdfmm_tree_stats indices). */
#define KDFMM_STAT_N 0
#define KDFMM_STAT_NCELLS 1
#define KDFMM_STAT_NLEAVES 2
#define KDFMM_STAT_DEPTH 3        /* deepest cell level (root = 0) */
#define KDFMM_STAT_NFAR 4         /* M2L pairs (sum of far-list lengths) */
#define KDFMM_STAT_NNEAR 5        /* near-list entries (leaf pairs) */
#define KDFMM_STAT_NP2P 6         /* particle-particle interactions, self excluded */
#define KDFMM_STAT_NFALLBACK 7    /* degenerate cuts split by position */
#define KDFMM_STAT_NEXACT 8       /* opening decisions settled in float64 */
#define KDFMM_STAT_LAUNCHES 9     /* kernels launched since the handle was created */
#define KDFMM_STAT_NHEAVY 10      /* leaves whose walk passed the walk budget and was redone
                                     block-wide (leaf walk; 0 for the dual walk) */
#define KDFMM_NSTATS 11

/* Phases timed by kdfmm_tree_timing (milliseconds of the most recent call). */
#define KDFMM_PHASE_BUILD 0       /* kdfmm_tree_build: tree + moments */
#define KDFMM_PHASE_WALK 1        /* interaction lists */
#define KDFMM_PHASE_M2L 2
#define KDFMM_PHASE_P2P 3         /* P2P + L2P + assembly */
#define KDFMM_NPHASES 4

/* Creates an empty handle on the current CUDA device.  Buffers are allocated
 * by the first build and reused by later builds of no more particles.
 * `out` is a host pointer that receives the handle. */
int kdfmm_tree_create(kdfmm_tree* out);

/* Releases the handle and its device memory (synchronises the device). */
void kdfmm_tree_destroy(kdfmm_tree t);

/* kd-tree construction and cell moments (Sec. 2; Eq. 7).
 * x: N x 3 positions, m: N masses (> 0), h: N smoothing lengths (> 0) for
 * KDFMM_SOFT_M4 or NULL for Plummer softening.  The handle keeps its own
 * tree-ordered copies; the caller's arrays may change after the call returns.
 * Cells are cut through their centre of mass across the longest side of their
 * bounding box (ties to the lowest axis); particles with x_axis < com_axis go
 * left, stably; a cut that leaves one side empty splits by position.  Cells
 * are numbered in pre-order.  The sums that decide a cut are pairwise
 * (perfect binary tree over the cell's particles in ascending caller index,
 * zero-padded to a power of two), so the tree is reproducible bit for bit.
 * Synchronises `stream` (the host sizes later launches from device counters).
 * Errors: KDFMM_ERR_INVALID_ARG for n < 1, bad params or NULL pointers,
 * KDFMM_ERR_NONFINITE for NaN/Inf inputs or m <= 0 / h <= 0. */
int kdfmm_tree_build(kdfmm_tree t, const double* x, const double* m, const double* h, int64_t n,
                     const kdfmm_params* p, void* stream);

/* A forest of independent systems in one handle: system k is particles
 * [sys_offset[k], sys_offset[k+1]) of x, m, h, with its own opening parameter
 * theta[k], softening length eps[k] and leaf size n_leaf[k] (Sec. 2 applied
 * to each system alone; the paper evaluates one system at a time).  Each
 * system's tree is exactly the tree kdfmm_tree_build makes for it alone;
 * every phase of the build and of kdfmm_fmm_accel processes all systems in
 * the same launches, and a leaf's walk never leaves its own tree.
 * sys_offset (n_sys + 1 entries, sys_offset[0] = 0, strictly increasing, total
 * <= 2^30), theta, eps and n_leaf (n_sys entries each) are HOST arrays; a
 * NULL theta / eps / n_leaf takes p->theta / p->eps / p->n_leaf for every
 * system.  p->soft_kind, p->precision and p->r_kern apply to all systems.
 * Cells are numbered in pre-order system after system: system k's cells are
 * the contiguous range starting at its root (the cells with parent -1, in
 * system order); kdfmm_tree_export returns the whole forest.  Synchronises
 * `stream`.  Errors as kdfmm_tree_build, and KDFMM_ERR_INVALID_ARG for an
 * empty system, a decreasing offset or a parameter out of range. */
int kdfmm_forest_build(kdfmm_tree t, const double* x, const double* m, const double* h,
                       const int64_t* sys_offset, int32_t n_sys, const double* theta,
                       const double* eps, const int32_t* n_leaf, const kdfmm_params* p,
                       void* stream);

/* kdfmm_forest_build followed by kdfmm_fmm_accel: accelerations a (N x 3) and
 * potentials phi (N or NULL) of every system, in caller order, each system
 * feeling only its own particles. */
int kdfmm_fmm_accel_batched(kdfmm_tree t, const double* x, const double* m, const double* h,
                            const int64_t* sys_offset, int32_t n_sys, const double* theta,
                            const double* eps, const int32_t* n_leaf, const kdfmm_params* p,
                            double* a, double* phi, void* stream);

/* Moments for a frozen tree (Sec. 2; Eq. 7): recomputes M, centre of mass, s,
 * h_max and Q of the existing cells for new positions / masses / smoothing
 * lengths of the same particles (same caller order and n), and freezes the
 * interaction lists of the last kdfmm_fmm_accel: later evaluations reuse them
 * until the next kdfmm_tree_build.  This is the evaluation that
 * kdfmm_fmm_accel_vjp differentiates (topology and lists held fixed), so finite
 * differences of it check the adjoint.  Leaf sums are pairwise over the leaf's
 * particles; a parent's M and sum m x are its left plus its right child's; s is
 * the exact maximum distance; Q the parallel-axis shift of its children's.
 * Needs one evaluation after the build.  Synchronises `stream`.
 * Errors as kdfmm_tree_build. */
int kdfmm_tree_moments(kdfmm_tree t, const double* x, const double* m, const double* h,
                       void* stream);

/* One force evaluation on the built tree: leaf-only walk with Eqs. 4-5,
 * M2L (Eq. 6), L2P (Eq. 8), softened P2P (Eq. 13 / Plummer), a = a_short +
 * a_long (Eq. 3).  a: N x 3 output, phi: N output potential or NULL (the
 * potential is the third-order expansion of -M/R - Q_jk R_j R_k/(2R^5) plus
 * the softened pair potentials).  The handle keeps the interaction lists in
 * fixed slots per leaf or, when a few lists are far longer than the rest (a
 * centrally condensed system), in room reserved per leaf by a one-pass walk
 * whose threads each use a scratch of 4096 int32 entries (at most ~3.2 GB;
 * when that cannot be allocated, in two passes: count, then fill).
 * Synchronises `stream` once (list sizes), again when the lists outgrew their
 * buffers and the walk is repeated. */
int kdfmm_fmm_accel(kdfmm_tree t, double* a, double* phi, void* stream);

/* Vector-Jacobian product of the last evaluation's accelerations with respect
 * to positions and masses, through the same tree and interaction lists (the
 * lists and cell topology are held fixed; smoothing lengths are inputs).
 * The paper has no adjoint; this is the derivative of the evaluation that
 * kdfmm_fmm_accel performs (Eqs. 3, 6, 7, 8, 13): L2P, M2L (r-derivatives by
 * dual numbers, M and Q linear), P2P on the target and on the source side,
 * and the moments (com = sum m x / M, Q of Eq. 7) back to the particles.
 * a_bar: N x 3 cotangent (caller order, device); x_bar: N x 3 and m_bar: N
 * outputs (device, overwritten).  FP64 mode runs every step in float64;
 * mixed mode forms the M2L r-derivatives and the P2P pair terms in float32
 * (as its evaluation does) from float64 differences, with float64 sums.  Cell
 * cotangents and the P2P source-side terms are summed with float64 atomics,
 * so the last bits may vary run to run.  Allocates its scratch (88 bytes per
 * particle, 160 per leaf, 80 per cell) with cudaMallocAsync on `stream`.  Errors:
 * KDFMM_ERR_INVALID_ARG before any evaluation or for non-device pointers,
 * KDFMM_ERR_CUDA on allocation or launch failure. */
int kdfmm_fmm_accel_vjp(kdfmm_tree t, const double* a_bar, double* x_bar, double* m_bar,
                        void* stream);

/* One kick and one drift of a kick-drift-kick leapfrog, in place:
 * v += dt_kick * a, then x += dt_drift * v (no drift when dt_drift is 0).
 * A step of size dt is kick(dt/2) + drift(dt), a force evaluation at the new
 * positions, kick(dt/2); consecutive half kicks may be merged.  The paper
 * follows the centre of mass of leapfrog runs (Sec. 4) but prints no
 * integrator; this is the plain gravity-only one.  x, v, a: N x 3 device
 * arrays (caller order).  Errors: KDFMM_ERR_INVALID_ARG for n outside
 * [1, 2^30], non-finite steps or non-device pointers. */
int kdfmm_kick_drift(double* x, double* v, const double* a, int64_t n, double dt_kick,
                     double dt_drift, void* stream);

/* out[0..2] = sum_i m_i v_i (device pointer to 3 doubles), float64 with a
 * compensated (two-sum) combination of per-block partials in a fixed order,
 * so repeated calls give identical bits.  With v = accelerations this is the
 * total force whose non-zero value the paper demonstrates (Sec. 4, Eq. 30). */
int kdfmm_total_momentum(const double* m, const double* v, int64_t n, double* out, void* stream);

/* The same reduction as kdfmm_total_momentum, for callers that must not
 * allocate device memory while they run: cudaMalloc and cudaFree can
 * synchronise the whole device, can fail or stall when another allocator
 * already holds the memory, and are off limits to code working inside a fixed
 * memory budget.  The paper has no counterpart; it is an interface variant.
 * This call allocates nothing: its scratch is a fixed 48 KiB array (1024
 * partial sums of 6 doubles) that every GPU loading the library keeps until
 * the process exits.  The first call on a device looks up that array's device
 * address (cudaGetSymbolAddress) once; make that first call before any stream
 * capture.  All calls share the array and each overwrites the partials it
 * reads, so nothing needs clearing, but calls whose work overlaps on the GPU
 * (e.g. on two streams at once) race on it.  n must lie in [1, 2^30];
 * larger n, NULL or non-device pointers give KDFMM_ERR_INVALID_ARG.  Results
 * are bit-identical to kdfmm_total_momentum's. */
int kdfmm_total_momentum_noalloc(const double* m, const double* v, int64_t n, double* out,
                                 void* stream);

/* Measurement utility (no counterpart in the paper): the roofline
 * denominators of the ALU-bound kernels on the current device.  Runs two
 * throughput loops on `stream` (independent fused multiply-add chains at full
 * occupancy, best of three timed launches after one warm-up) and writes to
 * out (host, 5 doubles): [0] float32 FMA TFLOP/s measured, [1] float64 FMA
 * TFLOP/s measured, [2] SM count, [3] maximum SM clock in MHz, [4] float32
 * peak derived as SMs x 128 lanes x 2 flop x maximum clock (TFLOP/s).
 * Allocates and frees a small scratch buffer; synchronises the stream.
 * NULL out gives KDFMM_ERR_INVALID_ARG. */
int kdfmm_measure_peaks(double* out, void* stream);

/* Host copies of the handle's statistics (KDFMM_NSTATS int64, host). */
int kdfmm_tree_stats(kdfmm_tree t, int64_t* stats);

/* Copies the tree and the last evaluation's interaction lists to HOST arrays
 * sized from kdfmm_tree_stats: perm (N int64: tree position -> caller index);
 * cell_ints (ncells x 7 int64: first, count, left, right, parent, depth, skip);
 * cell_reals (ncells x 12 double: M, com x y z, s, h_max, Q xx xy xz yy yz zz);
 * leaf_ids (nleaves int32, ascending); far_off / near_off (nleaves + 1 int64);
 * far_idx (NFAR int32) and near_idx (NNEAR int32), ascending within each leaf.
 * With KDFMM_WALK_DUAL the far lists are per cell: far_off has ncells + 1
 * entries.  Any pointer may be NULL to skip that array.  Synchronises the
 * device. */
int kdfmm_tree_export(kdfmm_tree t, int64_t* perm, int64_t* cell_ints, double* cell_reals,
                      int32_t* leaf_ids, int64_t* far_off, int32_t* far_idx, int64_t* near_off,
                      int32_t* near_idx);

/* Tuning (no counterpart in the paper): the number of cells one thread of the
 * leaf walk visits before it hands its leaf to the block-wide walk, which
 * decides every cell of the leaf's system in tiles of 1024 (a leaf in the
 * sparse outskirts of a condensed system can open most of the tree).  budget
 * = 0 restores the default (KDFMM_WALK_BUDGET from the environment, else
 * 4096).  Interaction lists and forces do not depend on it; the arena walk's
 * scratch grows with it (budget x 4 bytes per walk thread).  Takes effect at
 * the next evaluation (a captured batch graph is captured again).  budget
 * outside [0, 2^20] or a NULL handle gives KDFMM_ERR_INVALID_ARG. */
int kdfmm_tree_set_walk_budget(kdfmm_tree t, int32_t budget);

/* Tracing (no counterpart in the paper): with enable = 1 the handle records
 * CUDA events on the caller's stream around each phase of kdfmm_tree_build and
 * kdfmm_fmm_accel.  ms (host, KDFMM_NPHASES floats, may be NULL) receives the
 * durations of the most recent timed call of each phase; the call waits for
 * those events.  enable = 0 stops recording.  Timing changes no result. */
int kdfmm_tree_timing(kdfmm_tree t, int enable, float* ms);

/* Message for the calling thread's most recent failure ("" if none). */
const char* kdfmm_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* KDFMM_H */
