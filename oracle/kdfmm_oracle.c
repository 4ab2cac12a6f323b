/*
 * kd-tree FMM oracle -- TEST INFRASTRUCTURE, NOT PART OF THE PRODUCT PATH.
 *
 * A plain, slow, single-threaded FP64 CPU implementation of one gravitational
 * force evaluation by the kd-tree fast multipole method analysed in Potashov &
 * Yudin, "Non-conservation of linear momentum in widely used hierarchical
 * methods in gravitational gas dynamics" (arXiv 2502.01496), plus the O(N^2)
 * direct sum.  Only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark load this file's library.  The GPU library shares no code,
 * header, table or helper with it.
 *
 * Steps, in the paper's order:
 *   1. kd-tree: cut each cell through its centre of mass, perpendicular to the
 *      longest axis, until a cell holds no more than n_leaf particles (Sec. 2).
 *   2. cell moments: mass M, centre of mass, size s (radius of the smallest
 *      sphere about the centre of mass holding every particle), h_max, and the
 *      traceless quadrupole Q_ij of Eq. 7 (Sec. 2).
 *   3. walk: for every LEAF alpha only, descend from the root; a cell beta is
 *      "opened" when Eq. 4 (theta^2 < (s_beta/r)^2) or Eq. 5 (smoothing spheres
 *      may intersect) holds; an opened leaf is a short-range partner, an opened
 *      super-cell is descended, a cell that is not opened is a long-range
 *      partner (Sec. 2, Sec. 4).
 *   4. M2L: the acceleration field of beta about r = com_alpha - com_beta, Eq. 6,
 *      and its first and second derivatives (a forward-mode Taylor "jet"
 *      evaluation of Eq. 6 exactly as printed).  Optionally the standard p = 3
 *      Cartesian series of the multipole section instead (sink and source
 *      orders add up to at most 2: the quadrupole only at order 0).
 *   5. L2P: second-order Taylor expansion of that field at each particle, Eq. 8.
 *   6. P2P: softened direct summation over the particles of opened leaves,
 *      Plummer softening or the symmetrised M4-kernel Green's function (Eq. 13,
 *      Eq. 15).
 *   7. a = a_short + a_long (Eq. 3).
 *
 * Readings where the paper is silent (listed with reasons in the design notes):
 *   - sums that decide a cut (M and sum m x of a cell) are taken over the cell's
 *     particles in ascending caller index, as the perfect binary (pairwise) tree
 *     over the sequence zero-padded to a power of two;
 *   - longest axis = largest extent of the tight bounding box, ties -> lowest
 *     axis; particles with x_axis < com_axis go left, the rest right, stably;
 *     if one side would be empty the cell is split by position (first floor(n/2)
 *     particles left);
 *   - cells are numbered in pre-order (left subtree before right);
 *   - Eq. 4 is evaluated division-free as theta*theta*r2 < s_beta*s_beta, with
 *     r2 = dx*dx + dy*dy + dz*dz; a cell is also opened when r2 == 0 and, as the
 *     paper states, always when theta == 0;
 *   - Eq. 5 is evaluated as r2 < (s_a + s_b + R_kern*max(h_a, h_b))^2; with
 *     Plummer softening every h_i equals eps;
 *   - r = com_alpha - com_beta (sink minus source), consistent with Eq. 9;
 *   - potential: phi = phi_short + phi_long, phi_long the third-order Taylor
 *     expansion of Phi_beta(R) = -M/R - Q_jk R_j R_k / (2 R^5), whose negative
 *     gradient is Eq. 8 applied to Eq. 6.
 *
 * Compile with -ffp-contract=off and without -ffast-math: every expression is
 * evaluated exactly as written.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#else
static int omp_get_max_threads(void) { return 1; }
#endif

static const double KD_PI = 3.14159265358979323846;

/* ------------------------------------------------------------------------ */
/* Truncated multivariate Taylor polynomials ("jets") in three variables,    */
/* total order <= 3: 20 monomial coefficients c[k] of x1^a x2^b x3^c.        */
/* ------------------------------------------------------------------------ */

#define JN 20
typedef struct { double c[JN]; } jet;

static int g_mono[JN][3];      /* exponents of monomial k */
static int g_mul[JN][JN];      /* index of monomial a*b, or -1 if order > 3 */
static int g_jet_ready = 0;

static int mono_index(int a, int b, int c) {
    for (int k = 0; k < JN; ++k)
        if (g_mono[k][0] == a && g_mono[k][1] == b && g_mono[k][2] == c) return k;
    return -1;
}

static void jet_init(void) {
    if (g_jet_ready) return;
    int k = 0;
    for (int order = 0; order <= 3; ++order)          /* graded, then lexicographic */
        for (int a = order; a >= 0; --a)
            for (int b = order - a; b >= 0; --b) {
                g_mono[k][0] = a; g_mono[k][1] = b; g_mono[k][2] = order - a - b; ++k;
            }
    for (int i = 0; i < JN; ++i)
        for (int j = 0; j < JN; ++j) {
            int a = g_mono[i][0] + g_mono[j][0], b = g_mono[i][1] + g_mono[j][1],
                c = g_mono[i][2] + g_mono[j][2];
            g_mul[i][j] = (a + b + c <= 3) ? mono_index(a, b, c) : -1;
        }
    g_jet_ready = 1;
}

static jet jet_const(double v) { jet r; memset(&r, 0, sizeof r); r.c[0] = v; return r; }
static jet jet_var(double v, int axis) {   /* v + x_axis */
    jet r = jet_const(v); r.c[1 + axis] = 1.0; return r;
}
static jet jet_add(jet a, jet b) { for (int k = 0; k < JN; ++k) a.c[k] += b.c[k]; return a; }
static jet jet_sub(jet a, jet b) { for (int k = 0; k < JN; ++k) a.c[k] -= b.c[k]; return a; }
static jet jet_scale(jet a, double s) { for (int k = 0; k < JN; ++k) a.c[k] *= s; return a; }
static jet jet_mul(jet a, jet b) {
    jet r = jet_const(0.0);
    for (int i = 0; i < JN; ++i) {
        if (a.c[i] == 0.0) continue;
        for (int j = 0; j < JN; ++j) {
            int k = g_mul[i][j];
            if (k >= 0) r.c[k] += a.c[i] * b.c[j];
        }
    }
    return r;
}
/* a0^(-n - 1/2) from correctly rounded operations only (1/sqrt, then n
 * divisions), so that scaling a0 by a power of two scales the result exactly. */
static double half_pow(double a0, int n) {
    double r = 1.0 / sqrt(a0);
    for (int k = 0; k < n; ++k) r = r / a0;
    return r;
}

/* a^p for p = -n - 1/2: with a = a0 + d (d without constant term, d^4 = 0),
 * a^p = sum_{k=0..3} binom(p,k) a0^(p-k) d^k. */
static jet jet_pow_half(jet a, int n) {
    double p = -(double)n - 0.5;
    double a0 = a.c[0];
    jet d = a; d.c[0] = 0.0;
    jet d2 = jet_mul(d, d), d3 = jet_mul(d2, d);
    double b1 = p, b2 = p * (p - 1.0) / 2.0, b3 = p * (p - 1.0) * (p - 2.0) / 6.0;
    jet r = jet_const(half_pow(a0, n));
    r = jet_add(r, jet_scale(d, b1 * half_pow(a0, n + 1)));
    r = jet_add(r, jet_scale(d2, b2 * half_pow(a0, n + 2)));
    r = jet_add(r, jet_scale(d3, b3 * half_pow(a0, n + 3)));
    return r;
}

/* ------------------------------------------------------------------------ */
/* M2L (Eq. 6) and the potential it derives from, as jets in R = r + x.     */
/* ------------------------------------------------------------------------ */

/* Q stored as xx, xy, xz, yy, yz, zz. */
static double qget(const double Q[6], int i, int j) {
    static const int map[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    return Q[map[i][j]];
}

/* Eq. 6 evaluated with jets: a_i(R) = -M Rhat_i / R^2
 *                       + R^-4 (Rhat_k Q_ik - 5/2 Rhat_i Rhat_j Rhat_k Q_jk). */
static void jet_acc_node(const double r[3], double M, const double Q[6], jet acc[3]) {
    jet R[3] = {jet_var(r[0], 0), jet_var(r[1], 1), jet_var(r[2], 2)};
    jet R2 = jet_add(jet_add(jet_mul(R[0], R[0]), jet_mul(R[1], R[1])), jet_mul(R[2], R[2]));
    jet rinv = jet_pow_half(R2, 0);
    jet rinv2 = jet_mul(rinv, rinv);
    jet rinv4 = jet_mul(rinv2, rinv2);
    jet rh[3];
    for (int i = 0; i < 3; ++i) rh[i] = jet_mul(R[i], rinv);
    jet u[3];                                   /* u_i = Rhat_k Q_ik */
    for (int i = 0; i < 3; ++i) {
        u[i] = jet_const(0.0);
        for (int k = 0; k < 3; ++k) u[i] = jet_add(u[i], jet_scale(rh[k], qget(Q, i, k)));
    }
    jet w = jet_const(0.0);                     /* w = Rhat_j Rhat_k Q_jk = Rhat . u */
    for (int j = 0; j < 3; ++j) w = jet_add(w, jet_mul(rh[j], u[j]));
    for (int i = 0; i < 3; ++i) {
        jet mono = jet_scale(jet_mul(rh[i], rinv2), -M);
        jet quad = jet_mul(rinv4, jet_sub(u[i], jet_scale(jet_mul(rh[i], w), 2.5)));
        acc[i] = jet_add(mono, quad);
    }
}

/* Phi_beta(R) = -M/R - Q_jk R_j R_k / (2 R^5): the potential whose negative
 * gradient is Eq. 6 (reading: the paper prints only accelerations). */
static jet jet_pot_node(const double r[3], double M, const double Q[6]) {
    jet R[3] = {jet_var(r[0], 0), jet_var(r[1], 1), jet_var(r[2], 2)};
    jet R2 = jet_add(jet_add(jet_mul(R[0], R[0]), jet_mul(R[1], R[1])), jet_mul(R[2], R[2]));
    jet rinv = jet_pow_half(R2, 0);
    jet rinv5 = jet_pow_half(R2, 2);
    jet qrr = jet_const(0.0);
    for (int j = 0; j < 3; ++j)
        for (int k = 0; k < 3; ++k)
            qrr = jet_add(qrr, jet_scale(jet_mul(R[j], R[k]), qget(Q, j, k)));
    return jet_sub(jet_scale(rinv, -M), jet_scale(jet_mul(qrr, rinv5), 0.5));
}

/* Local expansion of one leaf: Taylor coefficients about its centre of mass. */
typedef struct { double pot[JN]; double acc[3][JN]; } local_exp;

enum { EXP_PHANTOM = 0, EXP_STANDARD = 1 };

static int mono_order(int k) { return g_mono[k][0] + g_mono[k][1] + g_mono[k][2]; }

/* expansion EXP_PHANTOM: Eq. 6 and its potential expanded to full order in
 * the sink displacement x (the quadrupole reaches the Hessian term, 1/r^6).
 * expansion EXP_STANDARD: the standard p = 3 Cartesian series (the multipole
 * section's series with p = 3 and no octupole): sink and source orders add up to
 * at most p - 1 = 2 for the acceleration and p = 3 for the potential, so the
 * monopole enters at every order but the quadrupole (source order 2) only at
 * order 0 of the acceleration and orders <= 1 of the potential (highest power
 * of 1/r: 4).  Both parts are linear in (M, Q), taken separately here. */
static void local_add_m2l(local_exp* L, const double r[3], double M, const double Q[6],
                          int expansion) {
    static const double Q0[6] = {0, 0, 0, 0, 0, 0};
    if (expansion == EXP_PHANTOM) {
        jet acc[3];
        jet_acc_node(r, M, Q, acc);
        jet pot = jet_pot_node(r, M, Q);
        for (int k = 0; k < JN; ++k) {
            L->pot[k] += pot.c[k];
            for (int i = 0; i < 3; ++i) L->acc[i][k] += acc[i].c[k];
        }
        return;
    }
    jet accm[3], accq[3];
    jet_acc_node(r, M, Q0, accm);
    jet_acc_node(r, 0.0, Q, accq);
    jet potm = jet_pot_node(r, M, Q0);
    jet potq = jet_pot_node(r, 0.0, Q);
    for (int k = 0; k < JN; ++k) {
        const int o = mono_order(k);
        L->pot[k] += potm.c[k] + (o <= 1 ? potq.c[k] : 0.0);
        for (int i = 0; i < 3; ++i) L->acc[i][k] += accm[i].c[k] + (o == 0 ? accq[i].c[k] : 0.0);
    }
}

/* Eq. 8: a_i(x) = a_i + x_j d_j a_i + 1/2 x_j x_k d_j d_k a_i -- the jet
 * coefficients of order <= 2 are exactly the Taylor coefficients d^n a / n!.
 * The potential uses the coefficients of order <= 3. */
static void local_eval(const local_exp* L, const double x[3], double a[3], double* phi) {
    double p = 0.0, ai[3] = {0.0, 0.0, 0.0};
    for (int k = 0; k < JN; ++k) {
        const int* e = g_mono[k];
        double xm = 1.0;
        for (int t = 0; t < e[0]; ++t) xm *= x[0];
        for (int t = 0; t < e[1]; ++t) xm *= x[1];
        for (int t = 0; t < e[2]; ++t) xm *= x[2];
        p += L->pot[k] * xm;
        if (e[0] + e[1] + e[2] <= 2)
            for (int i = 0; i < 3; ++i) ai[i] += L->acc[i][k] * xm;
    }
    for (int i = 0; i < 3; ++i) a[i] = ai[i];
    *phi = p;
}

/* ------------------------------------------------------------------------ */
/* Short-range pair interaction (P2P).                                       */
/* ------------------------------------------------------------------------ */

/* M4 cubic spline kernel (Schoenberg B-spline), compact support R_kern = 2,
 * normalised in 3D: W(r,h) = w(q)/h^3, q = r/h, with
 *   w(q) = (1/pi) (1 - 3/2 q^2 + 3/4 q^3)   0 <= q < 1
 *          (1/pi) (2 - q)^3 / 4             1 <= q < 2
 *          0                                q >= 2.
 * F(q) = 4 pi int_0^q w(u) u^2 du is the mass fraction inside r, so the
 * softened force per unit mass is F(q)/r^2, and the softened potential psi
 * (psi -> 1/r for q >= 2, psi' = -F/r^2) is P(q)/h.  F and P below are the
 * closed-form integrals of w. */
static double m4_w(double q) {
    if (q < 1.0) return (1.0 - 1.5 * q * q + 0.75 * q * q * q) / KD_PI;
    if (q < 2.0) { double t = 2.0 - q; return 0.25 * t * t * t / KD_PI; }
    return 0.0;
}
static double m4_F(double q) {
    if (q < 1.0) return (4.0 / 3.0) * q * q * q - 1.2 * pow(q, 5) + 0.5 * pow(q, 6);
    if (q < 2.0)
        return -1.0 / 15.0 + (8.0 / 3.0) * q * q * q - 3.0 * pow(q, 4) + 1.2 * pow(q, 5) - pow(q, 6) / 6.0;
    return 1.0;
}
static double m4_P(double q) {
    if (q < 1.0) return 1.4 - (2.0 / 3.0) * q * q + 0.3 * pow(q, 4) - 0.1 * pow(q, 5);
    if (q < 2.0)
        return 1.6 - (4.0 / 3.0) * q * q + q * q * q - 0.3 * pow(q, 4) + pow(q, 5) / 30.0 - 1.0 / (15.0 * q);
    return 1.0 / q;
}

enum { SOFT_PLUMMER = 0, SOFT_M4 = 1 };

/* Acceleration on particle i and its potential from particle j, d = x_i - x_j.
 * Plummer: a = -m d / (d^2+eps^2)^(3/2), phi = -m / sqrt(d^2+eps^2).
 * M4 (Eq. 13): G = -[phi(r,h_i) + phi(r,h_j)]/2, so a = -m (g_i + g_j)/2 d/r
 * with g = F(q)/r^2, and phi = -m (psi_i + psi_j)/2. */
static void pair_interaction(const double d[3], double mj, double hi, double hj, int kind,
                             double eps, double a[3], double* phi) {
    double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    if (kind == SOFT_PLUMMER) {
        double s2 = r2 + eps * eps;
        double inv = 1.0 / sqrt(s2);
        double f = mj * inv * inv * inv;
        for (int k = 0; k < 3; ++k) a[k] = -f * d[k];
        *phi = -mj * inv;
        return;
    }
    double r = sqrt(r2);
    if (r == 0.0) {                      /* coincident particles: no force */
        a[0] = a[1] = a[2] = 0.0;
        *phi = -mj * 0.5 * (m4_P(0.0) / hi + m4_P(0.0) / hj);
        return;
    }
    double qi = r / hi, qj = r / hj;
    double gi = (qi < 2.0) ? m4_F(qi) / r2 : 1.0 / r2;
    double gj = (qj < 2.0) ? m4_F(qj) / r2 : 1.0 / r2;
    double pi_ = (qi < 2.0) ? m4_P(qi) / hi : 1.0 / r;
    double pj_ = (qj < 2.0) ? m4_P(qj) / hj : 1.0 / r;
    double f = mj * 0.5 * (gi + gj) / r;
    for (int k = 0; k < 3; ++k) a[k] = -f * d[k];
    *phi = -mj * 0.5 * (pi_ + pj_);
}

/* ------------------------------------------------------------------------ */
/* kd-tree (Sec. 2).                                                          */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t first, count;            /* particle range in tree order */
    int32_t left, right, parent, depth, skip;
    double M, com[3], s, hmax, Q[6];
} ocell;

typedef struct {
    int64_t n;
    int32_t n_leaf, soft_kind, expansion;
    double theta, eps, r_kern;
    double *x, *m, *h;               /* copies, caller order */
    int64_t* order;                  /* tree position -> caller index */
    int64_t* scratch;
    double* vbuf;                    /* 4*n scratch for the pairwise sums */
    ocell* cells;
    int32_t ncells, cap, nleaves, maxdepth, nfallback;
    int32_t* leaf_of;                /* tree position -> leaf cell id */
} otree;

/* Perfect binary tree over v[lo, lo+len), len a power of two, entries at or
 * beyond n read as zero. */
static double pairwise_rec(const double* v, int64_t n, int64_t lo, int64_t len) {
    if (lo >= n) return 0.0;
    if (len == 1) return v[lo];
    int64_t half = len / 2;
    return pairwise_rec(v, n, lo, half) + pairwise_rec(v, n, lo + half, half);
}
static double pairwise_sum(const double* v, int64_t n) {
    int64_t p = 1;
    while (p < n) p <<= 1;
    return pairwise_rec(v, n, 0, p);
}

static int32_t new_cell(otree* T) {
    if (T->ncells == T->cap) {
        T->cap = T->cap ? 2 * T->cap : 1024;
        T->cells = (ocell*)realloc(T->cells, sizeof(ocell) * (size_t)T->cap);
    }
    memset(&T->cells[T->ncells], 0, sizeof(ocell));
    return T->ncells++;
}

/* Moments of the particles order[first .. first+n) (ascending caller index
 * when called from the build): M, com by pairwise sums, then s, h_max and Q of
 * Eq. 7 about that centre of mass. */
static void cell_moments(otree* T, int64_t first, int64_t n, ocell* c) {
    double* vm = T->vbuf;
    double* vx = T->vbuf + n;
    double* vy = T->vbuf + 2 * n;
    double* vz = T->vbuf + 3 * n;
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = T->order[first + k];
        double mi = T->m[i];
        vm[k] = mi;
        vx[k] = mi * T->x[3 * i + 0];
        vy[k] = mi * T->x[3 * i + 1];
        vz[k] = mi * T->x[3 * i + 2];
    }
    double M = pairwise_sum(vm, n);
    c->M = M;
    c->com[0] = pairwise_sum(vx, n) / M;
    c->com[1] = pairwise_sum(vy, n) / M;
    c->com[2] = pairwise_sum(vz, n) / M;
    double s2max = 0.0, hmax = 0.0;
    double Q[6] = {0, 0, 0, 0, 0, 0};
    for (int64_t k = 0; k < n; ++k) {
        int64_t i = T->order[first + k];
        double y0 = T->x[3 * i + 0] - c->com[0];
        double y1 = T->x[3 * i + 1] - c->com[1];
        double y2 = T->x[3 * i + 2] - c->com[2];
        double d2 = y0 * y0 + y1 * y1 + y2 * y2;
        if (d2 > s2max) s2max = d2;
        if (T->h[i] > hmax) hmax = T->h[i];
        double mi = T->m[i];
        Q[0] += mi * (3.0 * y0 * y0 - d2);
        Q[1] += mi * (3.0 * y0 * y1);
        Q[2] += mi * (3.0 * y0 * y2);
        Q[3] += mi * (3.0 * y1 * y1 - d2);
        Q[4] += mi * (3.0 * y1 * y2);
        Q[5] += mi * (3.0 * y2 * y2 - d2);
    }
    c->s = sqrt(s2max);
    c->hmax = hmax;
    memcpy(c->Q, Q, sizeof Q);
}

static int32_t build_cell(otree* T, int64_t first, int64_t n, int32_t parent, int32_t depth) {
    int32_t id = new_cell(T);
    ocell c;
    memset(&c, 0, sizeof c);
    c.first = first; c.count = n; c.parent = parent; c.depth = depth;
    c.left = c.right = -1;
    if (depth > T->maxdepth) T->maxdepth = depth;
    cell_moments(T, first, n, &c);
    if (n > T->n_leaf) {
        /* longest axis of the tight bounding box */
        double lo[3], hi[3];
        for (int d = 0; d < 3; ++d) { lo[d] = INFINITY; hi[d] = -INFINITY; }
        for (int64_t k = 0; k < n; ++k) {
            int64_t i = T->order[first + k];
            for (int d = 0; d < 3; ++d) {
                double v = T->x[3 * i + d];
                if (v < lo[d]) lo[d] = v;
                if (v > hi[d]) hi[d] = v;
            }
        }
        int axis = 0;
        double ext0 = hi[0] - lo[0], ext1 = hi[1] - lo[1], ext2 = hi[2] - lo[2];
        double best = ext0;
        if (ext1 > best) { axis = 1; best = ext1; }
        if (ext2 > best) { axis = 2; best = ext2; }
        double cut = c.com[axis];
        /* stable partition: x_axis < cut -> left */
        int64_t nl = 0, nr = 0;
        for (int64_t k = 0; k < n; ++k) {
            int64_t i = T->order[first + k];
            if (T->x[3 * i + axis] < cut) T->order[first + nl++] = i;
            else T->scratch[nr++] = i;
        }
        for (int64_t k = 0; k < nr; ++k) T->order[first + nl + k] = T->scratch[k];
        if (nl == 0 || nl == n) {
            /* degenerate cut: the partition left the order unchanged, so split
             * by position */
            nl = n / 2;
            T->nfallback++;
        }
        c.left = build_cell(T, first, nl, id, depth + 1);
        c.right = build_cell(T, first + nl, n - nl, id, depth + 1);
    } else {
        T->nleaves++;
        for (int64_t k = 0; k < n; ++k) T->leaf_of[first + k] = id;
    }
    c.skip = T->ncells;                 /* pre-order id following this subtree */
    T->cells[id] = c;
    return id;
}

otree* orc_build(int64_t n, const double* x, const double* m, const double* h, double theta,
                 int32_t n_leaf, int32_t soft_kind, double eps, double r_kern, int32_t expansion) {
    if (n <= 0 || n_leaf < 1 || (expansion != EXP_PHANTOM && expansion != EXP_STANDARD)) return NULL;
    jet_init();
    otree* T = (otree*)calloc(1, sizeof(otree));
    T->n = n; T->n_leaf = n_leaf; T->soft_kind = soft_kind;
    T->theta = theta; T->eps = eps; T->r_kern = r_kern; T->expansion = expansion;
    T->x = (double*)malloc(sizeof(double) * 3 * (size_t)n);
    T->m = (double*)malloc(sizeof(double) * (size_t)n);
    T->h = (double*)malloc(sizeof(double) * (size_t)n);
    memcpy(T->x, x, sizeof(double) * 3 * (size_t)n);
    memcpy(T->m, m, sizeof(double) * (size_t)n);
    for (int64_t i = 0; i < n; ++i)
        T->h[i] = (soft_kind == SOFT_PLUMMER || h == NULL) ? eps : h[i];
    T->order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    T->scratch = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    T->vbuf = (double*)malloc(sizeof(double) * 4 * (size_t)n);
    T->leaf_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t i = 0; i < n; ++i) T->order[i] = i;
    build_cell(T, 0, n, -1, 0);
    free(T->scratch); T->scratch = NULL;
    free(T->vbuf); T->vbuf = NULL;
    return T;
}

void orc_free(otree* T) {
    if (!T) return;
    free(T->x); free(T->m); free(T->h); free(T->order); free(T->cells); free(T->leaf_of);
    free(T);
}

int32_t orc_ncells(const otree* T) { return T->ncells; }
int32_t orc_nleaves(const otree* T) { return T->nleaves; }
int32_t orc_maxdepth(const otree* T) { return T->maxdepth; }
int32_t orc_nfallback(const otree* T) { return T->nfallback; }

void orc_get_order(const otree* T, int64_t* order) {
    memcpy(order, T->order, sizeof(int64_t) * (size_t)T->n);
}

/* ints: per cell first, count, left, right, parent, depth, skip (7 x int64);
 * reals: per cell M, com[3], s, hmax, Q[6] (12 doubles). */
void orc_get_cells(const otree* T, int64_t* ints, double* reals) {
    for (int32_t c = 0; c < T->ncells; ++c) {
        const ocell* p = &T->cells[c];
        int64_t* o = ints + 7 * (int64_t)c;
        o[0] = p->first; o[1] = p->count; o[2] = p->left; o[3] = p->right;
        o[4] = p->parent; o[5] = p->depth; o[6] = p->skip;
        double* r = reals + 12 * (int64_t)c;
        r[0] = p->M; r[1] = p->com[0]; r[2] = p->com[1]; r[3] = p->com[2];
        r[4] = p->s; r[5] = p->hmax;
        for (int k = 0; k < 6; ++k) r[6 + k] = p->Q[k];
    }
}

/* ------------------------------------------------------------------------ */
/* Walk (Sec. 2, Sec. 4).                                                     */
/* ------------------------------------------------------------------------ */

/* Eq. 4 and Eq. 5 for the sink alpha and the candidate beta. */
static int open_cell(const otree* T, const ocell* a, const ocell* b) {
    double dx = a->com[0] - b->com[0];
    double dy = a->com[1] - b->com[1];
    double dz = a->com[2] - b->com[2];
    double r2 = dx * dx + dy * dy + dz * dz;
    if (r2 == 0.0) return 1;
    if (T->theta == 0.0) return 1;
    if (T->theta * T->theta * r2 < b->s * b->s) return 1;
    double hm = a->hmax > b->hmax ? a->hmax : b->hmax;
    double rr = a->s + b->s + T->r_kern * hm;
    if (r2 < rr * rr) return 1;
    return 0;
}

typedef struct { int32_t* v; int64_t n, cap; } ivec;
static void ivec_push(ivec* v, int32_t x) {
    if (v->n == v->cap) {
        v->cap = v->cap ? 2 * v->cap : 256;
        v->v = (int32_t*)realloc(v->v, sizeof(int32_t) * (size_t)v->cap);
    }
    v->v[v->n++] = x;
}

static int g_ancestor_far = 0;

static void walk_rec(const otree* T, int32_t alpha, int32_t beta, ivec* far, ivec* near) {
    const ocell* a = &T->cells[alpha];
    const ocell* b = &T->cells[beta];
    if (open_cell(T, a, b)) {
        if (b->left < 0) ivec_push(near, beta);
        else {
            walk_rec(T, alpha, b->left, far, near);
            walk_rec(T, alpha, b->right, far, near);
        }
    } else {
        if (a->first >= b->first && a->first < b->first + b->count) {
#pragma omp atomic
            g_ancestor_far++;
        }
        ivec_push(far, beta);
    }
}

/* Interaction lists of every leaf, leaves in ascending id, entries in
 * ascending id.  Returns the number of leaves. */
typedef struct {
    int32_t nleaves;
    int32_t* leaf_ids;
    int64_t *far_off, *near_off;
    ivec far, near;
} olists;

olists* orc_walk(const otree* T) {
    olists* L = (olists*)calloc(1, sizeof(olists));
    L->nleaves = T->nleaves;
    L->leaf_ids = (int32_t*)malloc(sizeof(int32_t) * (size_t)T->nleaves);
    L->far_off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)T->nleaves + 1));
    L->near_off = (int64_t*)malloc(sizeof(int64_t) * ((size_t)T->nleaves + 1));
    int32_t k = 0;
    g_ancestor_far = 0;
    for (int32_t c = 0; c < T->ncells; ++c) {
        if (T->cells[c].left >= 0) continue;
        L->leaf_ids[k] = c;
        L->far_off[k] = L->far.n;
        L->near_off[k] = L->near.n;
        walk_rec(T, c, 0, &L->far, &L->near);
        ++k;
    }
    L->far_off[k] = L->far.n;
    L->near_off[k] = L->near.n;
    return L;
}
int64_t orc_lists_nfar(const olists* L) { return L->far.n; }
int64_t orc_lists_nnear(const olists* L) { return L->near.n; }
int32_t orc_ancestor_far(void) { return g_ancestor_far; }
void orc_lists_get(const olists* L, int32_t* leaf_ids, int64_t* far_off, int32_t* far_idx,
                   int64_t* near_off, int32_t* near_idx) {
    memcpy(leaf_ids, L->leaf_ids, sizeof(int32_t) * (size_t)L->nleaves);
    memcpy(far_off, L->far_off, sizeof(int64_t) * ((size_t)L->nleaves + 1));
    memcpy(near_off, L->near_off, sizeof(int64_t) * ((size_t)L->nleaves + 1));
    if (L->far.n) memcpy(far_idx, L->far.v, sizeof(int32_t) * (size_t)L->far.n);
    if (L->near.n) memcpy(near_idx, L->near.v, sizeof(int32_t) * (size_t)L->near.n);
}
void orc_lists_free(olists* L) {
    if (!L) return;
    free(L->leaf_ids); free(L->far_off); free(L->near_off); free(L->far.v); free(L->near.v);
    free(L);
}

/* ------------------------------------------------------------------------ */
/* Force evaluation.                                                          */
/* ------------------------------------------------------------------------ */

/* Forces on the particles of leaf alpha from the given far and near lists:
 * M2L of every far cell (Eq. 6) summed into one local expansion, L2P at each
 * particle (Eq. 8), softened pair sums over the near leaves (j != i), and
 * a = a_short + a_long (Eq. 3). */
static void eval_leaf(const otree* T, int32_t alpha, const int32_t* far, int64_t nfar,
                      const int32_t* near, int64_t nnear, double* a, double* phi, double* a_short,
                      double* a_long, double* phi_short, double* phi_long, int64_t* npp) {
    const ocell* ca = &T->cells[alpha];
    local_exp L;
    memset(&L, 0, sizeof L);
    for (int64_t f = 0; f < nfar; ++f) {
        const ocell* cb = &T->cells[far[f]];
        double r[3] = {ca->com[0] - cb->com[0], ca->com[1] - cb->com[1], ca->com[2] - cb->com[2]};
        local_add_m2l(&L, r, cb->M, cb->Q, T->expansion);
    }
    for (int64_t k = 0; k < ca->count; ++k) {
        int64_t i = T->order[ca->first + k];
        const double* xi = &T->x[3 * i];
        double as[3] = {0, 0, 0}, ps = 0.0;
        for (int64_t nb = 0; nb < nnear; ++nb) {
            const ocell* cb = &T->cells[near[nb]];
            for (int64_t q = 0; q < cb->count; ++q) {
                int64_t j = T->order[cb->first + q];
                if (j == i) continue;
                const double* xj = &T->x[3 * j];
                double d[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
                double aij[3], pij;
                pair_interaction(d, T->m[j], T->h[i], T->h[j], T->soft_kind, T->eps, aij, &pij);
                as[0] += aij[0]; as[1] += aij[1]; as[2] += aij[2];
                ps += pij;
                ++*npp;
            }
        }
        double xrel[3] = {xi[0] - ca->com[0], xi[1] - ca->com[1], xi[2] - ca->com[2]};
        double al[3], pl;
        local_eval(&L, xrel, al, &pl);
        for (int d = 0; d < 3; ++d) {
            if (a) a[3 * i + d] = as[d] + al[d];                 /* Eq. 3 */
            if (a_short) a_short[3 * i + d] = as[d];
            if (a_long) a_long[3 * i + d] = al[d];
        }
        if (phi) phi[i] = ps + pl;
        if (phi_short) phi_short[i] = ps;
        if (phi_long) phi_long[i] = pl;
    }
}

/* Evaluates a and phi (caller order) for the particles of the selected leaves
 * (all leaves when nsel < 0), walking the tree for each.  a_short / a_long /
 * phi_short / phi_long may be NULL.  Counts of P2P interactions and M2L pairs
 * go to stats[0], stats[1]. */
int32_t orc_eval(const otree* T, int32_t nsel, const int32_t* sel, double* a, double* phi,
                 double* a_short, double* a_long, double* phi_short, double* phi_long,
                 int64_t* stats) {
    jet_init();
    int64_t npp = 0, nm2l = 0;
    int32_t nl = nsel < 0 ? T->ncells : nsel;
    for (int32_t t = 0; t < nl; ++t) {
        int32_t alpha = nsel < 0 ? t : sel[t];
        if (alpha < 0 || alpha >= T->ncells) return -1;
        if (T->cells[alpha].left >= 0) {
            if (nsel < 0) continue;
            return -2;
        }
        ivec far = {0}, near = {0};
        walk_rec(T, alpha, 0, &far, &near);
        eval_leaf(T, alpha, far.v, far.n, near.v, near.n, a, phi, a_short, a_long, phi_short,
                  phi_long, &npp);
        nm2l += far.n;
        free(far.v);
        free(near.v);
    }
    if (stats) { stats[0] = npp; stats[1] = nm2l; }
    return 0;
}

/* orc_eval for the selected leaves (all when nsel < 0) with the leaves
 * spread over OpenMP threads when compiled with OpenMP (nthreads <= 0: the
 * OpenMP default).  Each leaf's walk and sums are the same steps as in
 * orc_eval and write only that leaf's particles, so a and phi are orc_eval's
 * bit for bit.  Used to time the oracle on every host core. */
int32_t orc_eval_threads(const otree* T, int32_t nsel, const int32_t* sel, double* a, double* phi,
                         int32_t nthreads) {
    jet_init();
    int32_t nl = nsel < 0 ? T->ncells : nsel;
    for (int32_t t = 0; t < nl; ++t) {
        int32_t alpha = nsel < 0 ? t : sel[t];
        if (alpha < 0 || alpha >= T->ncells) return -1;
        if (T->cells[alpha].left >= 0 && nsel >= 0) return -2;
    }
    (void)nthreads;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads > 0 ? nthreads : omp_get_max_threads())
    for (int32_t t = 0; t < nl; ++t) {
        int32_t alpha = nsel < 0 ? t : sel[t];
        if (T->cells[alpha].left >= 0) continue;
        int64_t npp = 0;
        ivec far = {0}, near = {0};
        walk_rec(T, alpha, 0, &far, &near);
        eval_leaf(T, alpha, far.v, far.n, near.v, near.n, a, phi, NULL, NULL, NULL, NULL, &npp);
        free(far.v);
        free(near.v);
    }
    return 0;
}

/* Threads an OpenMP parallel region of orc_eval_threads would use (1 without
 * OpenMP). */
int32_t orc_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Evaluation with given interaction lists (frozen topology): leaf_ids[k] is
 * the k-th leaf, its lists far_idx[far_off[k] .. far_off[k+1]) and near_idx
 * likewise.  All leaves are evaluated. */
int32_t orc_eval_lists(const otree* T, int32_t nleaves, const int32_t* leaf_ids,
                       const int64_t* far_off, const int32_t* far_idx, const int64_t* near_off,
                       const int32_t* near_idx, double* a, double* phi) {
    jet_init();
    int64_t npp = 0;
    for (int32_t k = 0; k < nleaves; ++k) {
        int32_t alpha = leaf_ids[k];
        if (alpha < 0 || alpha >= T->ncells || T->cells[alpha].left >= 0) return -1;
        eval_leaf(T, alpha, far_idx + far_off[k], far_off[k + 1] - far_off[k], near_idx + near_off[k],
                  near_off[k + 1] - near_off[k], a, phi, NULL, NULL, NULL, NULL, &npp);
    }
    return 0;
}

/* Frozen topology: new positions, masses and smoothing lengths for the same
 * particles with the tree's cells kept.  A leaf's M and sum m x are pairwise
 * sums over its particles (tree order); a super-cell's are its left child's
 * plus its right child's; the centre of mass their ratio; s the exact maximum
 * distance; Q by definition (Eq. 7); h_max the maximum.  Cells are visited in
 * reverse pre-order, so children come before their parents. */
int32_t orc_moments_frozen(otree* T, const double* x, const double* m, const double* h) {
    memcpy(T->x, x, sizeof(double) * 3 * (size_t)T->n);
    memcpy(T->m, m, sizeof(double) * (size_t)T->n);
    for (int64_t i = 0; i < T->n; ++i)
        T->h[i] = (T->soft_kind == SOFT_PLUMMER || h == NULL) ? T->eps : h[i];
    double* S = (double*)malloc(sizeof(double) * 3 * (size_t)T->ncells);
    T->vbuf = (double*)malloc(sizeof(double) * 4 * (size_t)T->n);
    for (int32_t c = T->ncells - 1; c >= 0; --c) {
        ocell* p = &T->cells[c];
        if (p->left < 0) {
            double* vm = T->vbuf;
            double* vx = T->vbuf + p->count;
            double* vy = T->vbuf + 2 * p->count;
            double* vz = T->vbuf + 3 * p->count;
            for (int64_t k = 0; k < p->count; ++k) {
                int64_t i = T->order[p->first + k];
                vm[k] = T->m[i];
                vx[k] = T->m[i] * T->x[3 * i];
                vy[k] = T->m[i] * T->x[3 * i + 1];
                vz[k] = T->m[i] * T->x[3 * i + 2];
            }
            p->M = pairwise_sum(vm, p->count);
            S[3 * c] = pairwise_sum(vx, p->count);
            S[3 * c + 1] = pairwise_sum(vy, p->count);
            S[3 * c + 2] = pairwise_sum(vz, p->count);
        } else {
            const ocell* l = &T->cells[p->left];
            const ocell* r = &T->cells[p->right];
            p->M = l->M + r->M;
            for (int d = 0; d < 3; ++d) S[3 * c + d] = S[3 * p->left + d] + S[3 * p->right + d];
        }
        for (int d = 0; d < 3; ++d) p->com[d] = S[3 * c + d] / p->M;
        double s2max = 0.0, hmax = 0.0, Q[6] = {0, 0, 0, 0, 0, 0};
        for (int64_t k = 0; k < p->count; ++k) {
            int64_t i = T->order[p->first + k];
            double y0 = T->x[3 * i] - p->com[0], y1 = T->x[3 * i + 1] - p->com[1];
            double y2 = T->x[3 * i + 2] - p->com[2];
            double d2 = y0 * y0 + y1 * y1 + y2 * y2;
            if (d2 > s2max) s2max = d2;
            if (T->h[i] > hmax) hmax = T->h[i];
            double mi = T->m[i];
            Q[0] += mi * (3.0 * y0 * y0 - d2);
            Q[1] += mi * (3.0 * y0 * y1);
            Q[2] += mi * (3.0 * y0 * y2);
            Q[3] += mi * (3.0 * y1 * y1 - d2);
            Q[4] += mi * (3.0 * y1 * y2);
            Q[5] += mi * (3.0 * y2 * y2 - d2);
        }
        p->s = sqrt(s2max);
        p->hmax = hmax;
        memcpy(p->Q, Q, sizeof Q);
    }
    free(S);
    free(T->vbuf);
    T->vbuf = NULL;
    return 0;
}

/* O(N^2) direct summation with the same pair interaction, j != i, for the
 * selected targets (all when ntarg < 0).  Output rows follow the target list. */
void orc_direct(int64_t n, const double* x, const double* m, const double* h, int32_t soft_kind,
                double eps, int64_t ntarg, const int64_t* targets, double* a, double* phi) {
    int64_t nt = ntarg < 0 ? n : ntarg;
    for (int64_t t = 0; t < nt; ++t) {
        int64_t i = ntarg < 0 ? t : targets[t];
        double hi = (soft_kind == SOFT_PLUMMER || h == NULL) ? eps : h[i];
        double as[3] = {0, 0, 0}, ps = 0.0;
        for (int64_t j = 0; j < n; ++j) {
            if (j == i) continue;
            double hj = (soft_kind == SOFT_PLUMMER || h == NULL) ? eps : h[j];
            double d[3] = {x[3 * i] - x[3 * j], x[3 * i + 1] - x[3 * j + 1], x[3 * i + 2] - x[3 * j + 2]};
            double aij[3], pij;
            pair_interaction(d, m[j], hi, hj, soft_kind, eps, aij, &pij);
            as[0] += aij[0]; as[1] += aij[1]; as[2] += aij[2];
            ps += pij;
        }
        a[3 * t] = as[0]; a[3 * t + 1] = as[1]; a[3 * t + 2] = as[2];
        phi[t] = ps;
    }
}

/* ------------------------------------------------------------------------ */
/* Primitives exposed for the oracle's own pins.                              */
/* ------------------------------------------------------------------------ */

int32_t orc_monomials(int32_t* exps) {
    jet_init();
    for (int k = 0; k < JN; ++k)
        for (int d = 0; d < 3; ++d) exps[3 * k + d] = g_mono[k][d];
    return JN;
}

/* Moments of an arbitrary particle set (all particles, caller order). */
void orc_moments(int64_t n, const double* x, const double* m, double* M, double* com, double* Q,
                 double* s) {
    otree T;
    memset(&T, 0, sizeof T);
    T.n = n;
    T.x = (double*)x; T.m = (double*)m;
    double* hz = (double*)calloc((size_t)n, sizeof(double));
    T.h = hz;
    T.order = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    T.vbuf = (double*)malloc(sizeof(double) * 4 * (size_t)n);
    for (int64_t i = 0; i < n; ++i) T.order[i] = i;
    ocell c;
    cell_moments(&T, 0, n, &c);
    *M = c.M;
    memcpy(com, c.com, sizeof c.com);
    memcpy(Q, c.Q, sizeof c.Q);
    *s = c.s;
    free(hz); free(T.order); free(T.vbuf);
}

/* Local expansion coefficients of one source (M, Q) about r: 20 potential
 * coefficients and 3 x 20 acceleration coefficients (orders <= 3; Eq. 8 uses
 * orders <= 2). */
void orc_m2l(const double* r, double M, const double* Q, int32_t expansion, double* pot,
             double* acc) {
    jet_init();
    local_exp L;
    memset(&L, 0, sizeof L);
    local_add_m2l(&L, r, M, Q, expansion);
    memcpy(pot, L.pot, sizeof L.pot);
    for (int i = 0; i < 3; ++i) memcpy(acc + JN * i, L.acc[i], sizeof(double) * JN);
}

void orc_l2p(const double* pot, const double* acc, const double* x, double* a, double* phi) {
    jet_init();
    local_exp L;
    memcpy(L.pot, pot, sizeof L.pot);
    for (int i = 0; i < 3; ++i) memcpy(L.acc[i], acc + JN * i, sizeof(double) * JN);
    local_eval(&L, x, a, phi);
}

/* Eq. 6 evaluated with plain doubles. */
void orc_acc_node(const double* r, double M, const double* Q, double* a) {
    double R = sqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    double rh[3] = {r[0] / R, r[1] / R, r[2] / R};
    double u[3], w = 0.0;
    for (int i = 0; i < 3; ++i) {
        u[i] = 0.0;
        for (int k = 0; k < 3; ++k) u[i] += rh[k] * qget(Q, i, k);
    }
    for (int j = 0; j < 3; ++j) w += rh[j] * u[j];
    for (int i = 0; i < 3; ++i)
        a[i] = -M * rh[i] / (R * R) + (u[i] - 2.5 * rh[i] * w) / (R * R * R * R);
}

void orc_pair(const double* d, double mj, double hi, double hj, int32_t kind, double eps,
              double* a, double* phi) {
    pair_interaction(d, mj, hi, hj, kind, eps, a, phi);
}

void orc_m4(double q, double* w, double* F, double* P) {
    *w = m4_w(q);
    *F = m4_F(q);
    *P = m4_P(q);
}

/* ------------------------------------------------------------------------ */
/* Symmetric dual-tree walk (the correction the paper's conclusions call for, */
/* after Dehnen 2000/2002): cells interact in pairs, both ways, so that the   */
/* expansions' Newton's third law for mutually interacting cells (Sec. 3)     */
/* carries over to the whole system.  Not the paper's scheme; a separate mode. */
/* ------------------------------------------------------------------------ */

/* Two distinct cells are well separated when theta r > s_A + s_B (Eq. 4 made
 * symmetric: both sizes) and their smoothing spheres cannot intersect
 * (Eq. 5 not satisfied: r >= s_A + s_B + R_kern max(h_A, h_B)).  theta = 0
 * separates nothing. */
static int well_separated(const otree* T, const ocell* a, const ocell* b) {
    if (T->theta == 0.0) return 0;
    double dx = a->com[0] - b->com[0];
    double dy = a->com[1] - b->com[1];
    double dz = a->com[2] - b->com[2];
    double r2 = dx * dx + dy * dy + dz * dz;
    double ss = a->s + b->s;
    if (!(T->theta * T->theta * r2 > ss * ss)) return 0;
    double hm = a->hmax > b->hmax ? a->hmax : b->hmax;
    double rr = ss + T->r_kern * hm;
    return r2 >= rr * rr;
}

typedef struct { ivec a, b; } pairs;
static void pairs_push(pairs* p, int32_t a, int32_t b) { ivec_push(&p->a, a); ivec_push(&p->b, b); }

/* interact(A, B): a cell with itself splits into its children's pairs; a
 * well-separated pair is a far (M2L) pair; two leaves that are not are a near
 * (P2P) pair; otherwise the larger cell (by s; a leaf is never split; ties
 * split A) is split. */
static void dual_rec(const otree* T, int32_t A, int32_t B, pairs* far, pairs* near) {
    const ocell* a = &T->cells[A];
    const ocell* b = &T->cells[B];
    if (A == B) {
        if (a->left < 0) { pairs_push(near, A, A); return; }
        dual_rec(T, a->left, a->left, far, near);
        dual_rec(T, a->right, a->right, far, near);
        dual_rec(T, a->left, a->right, far, near);
        return;
    }
    if (well_separated(T, a, b)) { pairs_push(far, A, B); return; }
    if (a->left < 0 && b->left < 0) { pairs_push(near, A, B); return; }
    int split_a = a->left >= 0 && (b->left < 0 || a->s >= b->s);
    if (split_a) {
        dual_rec(T, a->left, B, far, near);
        dual_rec(T, a->right, B, far, near);
    } else {
        dual_rec(T, A, b->left, far, near);
        dual_rec(T, A, b->right, far, near);
    }
}

/* Lists of the dual walk: far list of every cell (the cells it receives M2L
 * from), near list of every leaf (the leaves it receives P2P from, itself
 * included once); entries in ascending id. */
typedef struct {
    int32_t ncells, nleaves;
    int64_t *far_off, *near_off;     /* ncells + 1, nleaves + 1 */
    int32_t *far_idx, *near_idx;
    int64_t nfar, nnear;
} odual;

static int cmp_i32(const void* x, const void* y) {
    int32_t a = *(const int32_t*)x, b = *(const int32_t*)y;
    return (a > b) - (a < b);
}

static void to_csr(int32_t nrows, const int32_t* rows, const int32_t* cols, int64_t n,
                   int64_t** off_out, int32_t** idx_out) {
    int64_t* off = (int64_t*)calloc((size_t)nrows + 1, sizeof(int64_t));
    for (int64_t e = 0; e < n; ++e) off[rows[e] + 1]++;
    for (int32_t r = 0; r < nrows; ++r) off[r + 1] += off[r];
    int32_t* idx = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t* cur = (int64_t*)malloc(sizeof(int64_t) * ((size_t)nrows + 1));
    memcpy(cur, off, sizeof(int64_t) * ((size_t)nrows + 1));
    for (int64_t e = 0; e < n; ++e) idx[cur[rows[e]]++] = cols[e];
    for (int32_t r = 0; r < nrows; ++r)
        qsort(idx + off[r], (size_t)(off[r + 1] - off[r]), sizeof(int32_t), cmp_i32);
    free(cur);
    *off_out = off;
    *idx_out = idx;
}

odual* orc_dual_walk(const otree* T) {
    pairs far = {{0}, {0}}, near = {{0}, {0}};
    dual_rec(T, 0, 0, &far, &near);
    /* far pairs act both ways; near pairs both ways, a leaf with itself once */
    int64_t nf = 2 * far.a.n, nn = 0;
    int32_t* fr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nf > 0 ? nf : 1));
    int32_t* fc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nf > 0 ? nf : 1));
    for (int64_t e = 0; e < far.a.n; ++e) {
        fr[2 * e] = far.a.v[e]; fc[2 * e] = far.b.v[e];
        fr[2 * e + 1] = far.b.v[e]; fc[2 * e + 1] = far.a.v[e];
    }
    int32_t* rank = (int32_t*)malloc(sizeof(int32_t) * (size_t)T->ncells);
    int32_t nl = 0;
    for (int32_t c = 0; c < T->ncells; ++c) rank[c] = T->cells[c].left < 0 ? nl++ : -1;
    int32_t* nr = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * near.a.n + 1));
    int32_t* nc = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * near.a.n + 1));
    for (int64_t e = 0; e < near.a.n; ++e) {
        int32_t A = near.a.v[e], B = near.b.v[e];
        nr[nn] = rank[A]; nc[nn] = B; ++nn;
        if (A != B) { nr[nn] = rank[B]; nc[nn] = A; ++nn; }
    }
    odual* D = (odual*)calloc(1, sizeof(odual));
    D->ncells = T->ncells;
    D->nleaves = nl;
    D->nfar = nf;
    D->nnear = nn;
    to_csr(T->ncells, fr, fc, nf, &D->far_off, &D->far_idx);
    to_csr(nl, nr, nc, nn, &D->near_off, &D->near_idx);
    free(fr); free(fc); free(nr); free(nc); free(rank);
    free(far.a.v); free(far.b.v); free(near.a.v); free(near.b.v);
    return D;
}
int64_t orc_dual_nfar(const odual* D) { return D->nfar; }
int64_t orc_dual_nnear(const odual* D) { return D->nnear; }
void orc_dual_get(const odual* D, int64_t* far_off, int32_t* far_idx, int64_t* near_off,
                  int32_t* near_idx) {
    memcpy(far_off, D->far_off, sizeof(int64_t) * ((size_t)D->ncells + 1));
    memcpy(near_off, D->near_off, sizeof(int64_t) * ((size_t)D->nleaves + 1));
    if (D->nfar) memcpy(far_idx, D->far_idx, sizeof(int32_t) * (size_t)D->nfar);
    if (D->nnear) memcpy(near_idx, D->near_idx, sizeof(int32_t) * (size_t)D->nnear);
}
void orc_dual_free(odual* D) {
    if (!D) return;
    free(D->far_off); free(D->near_off); free(D->far_idx); free(D->near_idx);
    free(D);
}

/* Forces from the dual walk's lists: every cell's local expansion from its
 * far list (M2L, Eq. 6 or the standard series); at each particle the sum of
 * the expansions of all cells that contain it, each evaluated about its own
 * centre of mass (Eq. 8); plus the softened pair sums over the leaf's near
 * list (j != i). */
int32_t orc_eval_dual(const otree* T, const odual* D, double* a, double* phi) {
    jet_init();
    local_exp* L = (local_exp*)calloc((size_t)T->ncells, sizeof(local_exp));
    if (!L) return -1;
    for (int32_t c = 0; c < T->ncells; ++c) {
        const ocell* ca = &T->cells[c];
        for (int64_t e = D->far_off[c]; e < D->far_off[c + 1]; ++e) {
            const ocell* cb = &T->cells[D->far_idx[e]];
            double r[3] = {ca->com[0] - cb->com[0], ca->com[1] - cb->com[1],
                           ca->com[2] - cb->com[2]};
            local_add_m2l(&L[c], r, cb->M, cb->Q, T->expansion);
        }
    }
    int32_t k = 0;
    for (int32_t alpha = 0; alpha < T->ncells; ++alpha) {
        const ocell* ca = &T->cells[alpha];
        if (ca->left >= 0) continue;
        for (int64_t q = 0; q < ca->count; ++q) {
            int64_t i = T->order[ca->first + q];
            const double* xi = &T->x[3 * i];
            double as[3] = {0, 0, 0}, ps = 0.0;
            for (int64_t e = D->near_off[k]; e < D->near_off[k + 1]; ++e) {
                const ocell* cb = &T->cells[D->near_idx[e]];
                for (int64_t u = 0; u < cb->count; ++u) {
                    int64_t j = T->order[cb->first + u];
                    if (j == i) continue;
                    const double* xj = &T->x[3 * j];
                    double d[3] = {xi[0] - xj[0], xi[1] - xj[1], xi[2] - xj[2]};
                    double aij[3], pij;
                    pair_interaction(d, T->m[j], T->h[i], T->h[j], T->soft_kind, T->eps, aij, &pij);
                    as[0] += aij[0]; as[1] += aij[1]; as[2] += aij[2];
                    ps += pij;
                }
            }
            double al[3] = {0, 0, 0}, pl = 0.0;
            for (int32_t c = alpha; c >= 0; c = T->cells[c].parent) {
                const ocell* cc = &T->cells[c];
                double xrel[3] = {xi[0] - cc->com[0], xi[1] - cc->com[1], xi[2] - cc->com[2]};
                double ac[3], pc;
                local_eval(&L[c], xrel, ac, &pc);
                al[0] += ac[0]; al[1] += ac[1]; al[2] += ac[2];
                pl += pc;
            }
            for (int d = 0; d < 3; ++d) a[3 * i + d] = as[d] + al[d];
            if (phi) phi[i] = ps + pl;
        }
        ++k;
    }
    free(L);
    return 0;
}
