/*
 * fmm_oracle.c -- plain FP64 CPU oracle for the adaptive 2-D fast multipole
 * method of Goude & Engblom, "Adaptive fast multipole methods on the GPU"
 * (arXiv:1205.4611), for the complex-log potential
 *
 *     Phi(y_i) = sum_{j, x_j != y_i} q_j Log(y_i - x_j)        (Eq. 1 / Eq. 2)
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the GPU path is
 * compared against: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark load it.  It shares no code, header, table or helper
 * with the CUDA library and must never be called by the product path.
 *
 * Style: slow, obviously correct.  Every translation operator is its
 * plain closed-form definition (binomial sums written out); the FMM itself
 * follows the paper's order of steps: tree (Sec. 2, Sec. 3.2), connectivity
 * by the theta-criterion (Eq. 3), P2M (Eq. 4), upward M2M, M2L, downward
 * L2L (Sec. 2, Sec. 3.3), L2P (Eq. 5) and the near-field P2P.  Compiled with
 * -ffp-contract=off so no multiply-add is fused behind the reader's back.
 * Every sum runs serially in a fixed order.  Only loops whose iterations are
 * independent (one target box's local expansion in M2L, one evaluation
 * point's L2P + P2P, one target of a direct sum) may be spread over threads
 * (OpenMP, oracle_set_threads); each iteration is still computed by one
 * thread in the same order, so the results do not depend on the thread count.
 *
 * Readings of the paper taken here (the paper is silent or garbled):
 *  - levels: L = min{L : ceil(N / 4^L) <= leaf}; Eq. (Nlevels) is an option.
 *  - split axis: the longer side of the box rectangle, x on a tie (Sec. 2,
 *    "split guided by the eccentricity").
 *  - median: sort the box's sources by (coordinate, original index); the
 *    first floor(n/2) go left (Sec. 2, "split close to the median").
 *  - split line: 0.5*(max_left + min_right); with an empty left side the
 *    line is min(rectangle midpoint, min_right); with no points the midpoint.
 *  - children: (left, right) of the first split, each split once more
 *    along its own longer side; child 4b + 2*h1 + h2.
 *  - within a box, sources are kept in the order of the box's last sort.
 *  - separate evaluation points do not move the splits; a target goes left
 *    iff its coordinate is <= the split line; within a leaf, targets keep
 *    their original index order.
 *  - geometry: centre = rectangle centre, radius = half the diagonal.
 *  - theta-criterion (Eq. 3): well separated iff d > 0 and R + theta*r <= theta*d.
 *  - multipole signs: a_0 = sum q_j, a_k = -sum q_j (x_j - c)^k / k (Eq. 4).
 *  - M2L keeps the branch Log(z_t - z_s) for the a_0 term (the printed
 *    algorithm has two sign slips; the definition below is the exact
 *    Taylor expansion of Eq. 4 about the target centre).
 *  - P2P skips exactly coincident pairs (the j != i / x_j != y_i of Eq. 1-2).
 *  - leaf shortcut (optional, Sec. 2): leaf-level strong pairs passing the
 *    theta-criterion with r and R interchanged become P2L (sources of the
 *    larger box into the smaller box's local) or M2P (multipole of the
 *    smaller box evaluated in the larger box); equal radii never pass.
 *
 * Range: coefficients are unscaled, as in Eq. 4-5, so boxes must satisfy
 * radius^p > 1e-300 (true for every workload this project draws).
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#include "fmm_oracle.h"

/* Threads for the FMM's independent per-target loops; 1 = serial (default). */
static int g_threads = 1;

void oracle_set_threads(int n) { g_threads = n > 0 ? n : 1; }

static double now_s(void)
{
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

typedef double complex cplx;

#define MAXP 64
#define MAXB (2 * MAXP + 2)

static double binom_tab[MAXB][MAXB];
static int binom_ready = 0;

/* C(n, k) by Pascal's rule, in double. */
static double binom(int n, int k)
{
    if (!binom_ready) {
        memset(binom_tab, 0, sizeof(binom_tab));
        for (int i = 0; i < MAXB; ++i) {
            binom_tab[i][0] = 1.0;
            for (int j = 1; j <= i; ++j)
                binom_tab[i][j] = binom_tab[i - 1][j - 1] + (j <= i - 1 ? binom_tab[i - 1][j] : 0.0);
        }
        binom_ready = 1;
    }
    if (k < 0 || k > n) return 0.0;
    return binom_tab[n][k];
}

static int64_t level_base(int l) { return ((INT64_C(1) << (2 * l)) - 1) / 3; }

int64_t oracle_n_boxes(int L) { return level_base(L + 1); }

int oracle_levels_cap(int64_t n, int leaf)
{
    int L = 0;
    int64_t boxes = 1;
    while ((n + boxes - 1) / boxes > leaf) {
        ++L;
        boxes *= 4;
    }
    return L;
}

/* Eq. (Nlevels): N_l = ceil(0.5 * log2(5/8 * N / N_d)), clamped at 0. */
int oracle_levels_eq(int64_t n, int nd)
{
    double v = 0.5 * log2(0.625 * (double)n / (double)nd);
    int L = (int)ceil(v);
    return L < 0 ? 0 : L;
}

/* ------------------------------------------------------------------ */
/* Direct sums (Eq. 1 and Eq. 2).                                      */
/* ------------------------------------------------------------------ */

void oracle_direct(int64_t n_src, const double *src_xy, const double *q,
                   int64_t n_tgt, const double *tgt_xy, double *phi)
{
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n_tgt; ++i) {
        const double yx = tgt_xy[2 * i], yy = tgt_xy[2 * i + 1];
        cplx acc = 0.0;
        for (int64_t j = 0; j < n_src; ++j) {
            double dx = yx - src_xy[2 * j], dy = yy - src_xy[2 * j + 1];
            if (dx == 0.0 && dy == 0.0) continue; /* x_j == y_i */
            acc += CMPLX(q[2 * j], q[2 * j + 1]) * clog(CMPLX(dx, dy));
        }
        phi[2 * i] = creal(acc);
        phi[2 * i + 1] = cimag(acc);
    }
}

/* Direct sum restricted to a list of target indices. */
void oracle_direct_sample(int64_t n_src, const double *src_xy, const double *q,
                          const double *tgt_xy, int64_t n_sample, const int64_t *sample,
                          double *phi)
{
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t s = 0; s < n_sample; ++s) {
        int64_t i = sample[s];
        const double yx = tgt_xy[2 * i], yy = tgt_xy[2 * i + 1];
        cplx acc = 0.0;
        for (int64_t j = 0; j < n_src; ++j) {
            double dx = yx - src_xy[2 * j], dy = yy - src_xy[2 * j + 1];
            if (dx == 0.0 && dy == 0.0) continue;
            acc += CMPLX(q[2 * j], q[2 * j + 1]) * clog(CMPLX(dx, dy));
        }
        phi[2 * s] = creal(acc);
        phi[2 * s + 1] = cimag(acc);
    }
}

/* The harmonic kernel of the paper's experiments (Sec. 5): with
 * G(z_i, z_j) = Gamma_j / (z_j - z_i) and Gamma = q,
 *     u(y_i) = sum_{j, x_j != y_i} q_j / (x_j - y_i)   (= -d/dy of Eq. 1 / Eq. 2).
 * Over all targets (sample NULL) or a list of target indices. */
void oracle_direct_harmonic(int64_t n_src, const double *src_xy, const double *q,
                            int64_t n_tgt, const double *tgt_xy, int64_t n_sample,
                            const int64_t *sample, double *u)
{
    int64_t n_out = sample ? n_sample : n_tgt;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t s = 0; s < n_out; ++s) {
        int64_t i = sample ? sample[s] : s;
        const double yx = tgt_xy[2 * i], yy = tgt_xy[2 * i + 1];
        cplx acc = 0.0;
        for (int64_t j = 0; j < n_src; ++j) {
            double dx = src_xy[2 * j] - yx, dy = src_xy[2 * j + 1] - yy;
            if (dx == 0.0 && dy == 0.0) continue; /* x_j == y_i */
            acc += CMPLX(q[2 * j], q[2 * j + 1]) / CMPLX(dx, dy);
        }
        u[2 * s] = creal(acc);
        u[2 * s + 1] = cimag(acc);
    }
}

/* ------------------------------------------------------------------ */
/* Expansions and their translations (Eq. 4, Eq. 5, Sec. 3.3).          */
/* Arrays of p+1 complex numbers, stored (re, im) interleaved.          */
/* ------------------------------------------------------------------ */

static cplx ld(const double *v, int k) { return CMPLX(v[2 * k], v[2 * k + 1]); }
static void add(double *v, int k, cplx z)
{
    v[2 * k] += creal(z);
    v[2 * k + 1] += cimag(z);
}

/* P2M: multipole of sources about centre c: a_0 = sum q_j,
 * a_k = -sum q_j (x_j - c)^k / k  (expansion of q log(z - x_j), Eq. 4). */
void oracle_p2m(int p, double cx, double cy, int64_t n, const double *xy,
                const double *q, double *a)
{
    cplx c = CMPLX(cx, cy);
    for (int64_t j = 0; j < n; ++j) {
        cplx qj = CMPLX(q[2 * j], q[2 * j + 1]);
        cplx w = CMPLX(xy[2 * j], xy[2 * j + 1]) - c;
        add(a, 0, qj);
        cplx wk = 1.0;
        for (int k = 1; k <= p; ++k) {
            wk = wk * w;
            add(a, k, -qj * wk / (double)k);
        }
    }
}

/* M2P: evaluate the multipole expansion (Eq. 4) at z. */
void oracle_m2p(int p, double cx, double cy, const double *a, double zx, double zy,
                double *out)
{
    cplx w = CMPLX(zx, zy) - CMPLX(cx, cy);
    cplx v = ld(a, 0) * clog(w);
    cplx wk = 1.0;
    for (int k = 1; k <= p; ++k) {
        wk = wk * w;
        v += ld(a, k) / wk;
    }
    out[0] = creal(v);
    out[1] = cimag(v);
}

/* M2M: add to the parent's multipole (centre zp) the child's multipole
 * (centre zc) re-expanded about zp, r = zc - zp:
 *   a'_0 = a_0,
 *   a'_l = sum_{k=1}^{l} C(l-1, k-1) r^{l-k} a_k - a_0 r^l / l.            */
void oracle_m2m(int p, double zcx, double zcy, double zpx, double zpy,
                const double *a, double *out)
{
    cplx r = CMPLX(zcx, zcy) - CMPLX(zpx, zpy);
    cplx rp[MAXP + 1];
    rp[0] = 1.0;
    for (int k = 1; k <= p; ++k) rp[k] = rp[k - 1] * r;
    add(out, 0, ld(a, 0));
    for (int l = 1; l <= p; ++l) {
        cplx s = 0.0;
        for (int k = 1; k <= l; ++k) s += binom(l - 1, k - 1) * rp[l - k] * ld(a, k);
        s -= ld(a, 0) * rp[l] / (double)l;
        add(out, l, s);
    }
}

/* M2L: add to the local expansion about zt (Eq. 5) the Taylor expansion of
 * the multipole about zs (Eq. 4), r = zs - zt, x_k = (-1)^k a_k / r^k:
 *   b_0 += sum_k x_k + a_0 Log(zt - zs),
 *   b_l += ( sum_k C(k+l-1, l) x_k - a_0 / l ) / r^l.                      */
void oracle_m2l(int p, double zsx, double zsy, double ztx, double zty,
                const double *a, double *b)
{
    cplx zs = CMPLX(zsx, zsy), zt = CMPLX(ztx, zty);
    cplx r = zs - zt;
    cplx ir = 1.0 / r;
    cplx ip[MAXP + 1], x[MAXP + 1];
    ip[0] = 1.0;
    for (int k = 1; k <= p; ++k) ip[k] = ip[k - 1] * ir;
    for (int k = 1; k <= p; ++k) x[k] = ((k & 1) ? -1.0 : 1.0) * ld(a, k) * ip[k];
    for (int l = 0; l <= p; ++l) {
        cplx c = 0.0;
        for (int k = 1; k <= p; ++k) c += binom(k + l - 1, l) * x[k];
        if (l == 0)
            add(b, 0, c + ld(a, 0) * clog(zt - zs));
        else
            add(b, l, (c - ld(a, 0) / (double)l) * ip[l]);
    }
}

/* L2L: add to the child's local (centre zc) the parent's local (centre zp)
 * re-expanded about zc, d = zc - zp:  b'_l = sum_{k>=l} C(k, l) b_k d^{k-l}. */
void oracle_l2l(int p, double zpx, double zpy, double zcx, double zcy,
                const double *b, double *out)
{
    cplx d = CMPLX(zcx, zcy) - CMPLX(zpx, zpy);
    cplx dp[MAXP + 1];
    dp[0] = 1.0;
    for (int k = 1; k <= p; ++k) dp[k] = dp[k - 1] * d;
    for (int l = 0; l <= p; ++l) {
        cplx s = 0.0;
        for (int k = l; k <= p; ++k) s += binom(k, l) * ld(b, k) * dp[k - l];
        add(out, l, s);
    }
}

/* L2P: evaluate the local expansion (Eq. 5) at z by Horner's rule. */
void oracle_l2p(int p, double cx, double cy, const double *b, double zx, double zy,
                double *out)
{
    cplx w = CMPLX(zx, zy) - CMPLX(cx, cy);
    cplx v = ld(b, p);
    for (int l = p - 1; l >= 0; --l) v = v * w + ld(b, l);
    out[0] = creal(v);
    out[1] = cimag(v);
}

/* Derivative of the local expansion (Eq. 5) at z: sum_{l>=1} l b_l (z - c)^(l-1). */
void oracle_l2p_deriv(int p, double cx, double cy, const double *b, double zx, double zy,
                      double *out)
{
    cplx w = CMPLX(zx, zy) - CMPLX(cx, cy);
    cplx v = (double)p * ld(b, p);
    for (int l = p - 1; l >= 1; --l) v = v * w + (double)l * ld(b, l);
    out[0] = creal(v);
    out[1] = cimag(v);
}

/* Derivative of the multipole expansion (Eq. 4) at z:
 *   a_0 / (z - c) - sum_{k>=1} k a_k / (z - c)^(k+1). */
void oracle_m2p_deriv(int p, double cx, double cy, const double *a, double zx, double zy,
                      double *out)
{
    cplx w = CMPLX(zx, zy) - CMPLX(cx, cy);
    cplx iw = 1.0 / w;
    cplx v = ld(a, 0) * iw;
    cplx wk = iw;
    for (int k = 1; k <= p; ++k) {
        wk = wk * iw;
        v -= (double)k * ld(a, k) * wk;
    }
    out[0] = creal(v);
    out[1] = cimag(v);
}

/* P2L: add to the local expansion about c (Eq. 5) the Taylor expansion of
 * q log(z - x) for sources x far from c (the leaf shortcut of Sec. 2):
 *   b_0 += q Log(c - x),  b_l += -q / (l (x - c)^l).                        */
void oracle_p2l(int p, double cx, double cy, int64_t n, const double *xy, const double *q,
                double *b)
{
    cplx c = CMPLX(cx, cy);
    for (int64_t j = 0; j < n; ++j) {
        cplx qj = CMPLX(q[2 * j], q[2 * j + 1]);
        cplx x = CMPLX(xy[2 * j], xy[2 * j + 1]);
        add(b, 0, qj * clog(c - x));
        cplx ir = 1.0 / (x - c), pw = 1.0;
        for (int l = 1; l <= p; ++l) {
            pw = pw * ir;
            add(b, l, -qj * pw / (double)l);
        }
    }
}

/* ------------------------------------------------------------------ */
/* Topological phase: median-split pyramid tree (Sec. 2, Sec. 3.2).     */
/* ------------------------------------------------------------------ */

typedef struct {
    double key;
    uint32_t idx;
} keyed;

static int cmp_keyed(const void *pa, const void *pb)
{
    const keyed *a = (const keyed *)pa, *b = (const keyed *)pb;
    if (a->key < b->key) return -1;
    if (a->key > b->key) return 1;
    return (a->idx > b->idx) - (a->idx < b->idx);
}

/* Split perm[lo, lo+n) inside rect (x0, x1, y0, y1): sort by (coordinate,
 * index) along the longer side and cut after floor(n/2) elements.  Writes
 * the axis, the split line and the two child rectangles. */
static void split_box(const double *xy, uint32_t *perm, int64_t lo, int64_t n,
                      const double rect[4], keyed *scratch, int *axis_out,
                      double *line_out, double left[4], double right[4])
{
    double w = rect[1] - rect[0], h = rect[3] - rect[2];
    int axis = (w >= h) ? 0 : 1;
    for (int64_t i = 0; i < n; ++i) {
        uint32_t id = perm[lo + i];
        scratch[i].key = xy[2 * (int64_t)id + axis] + 0.0; /* -0.0 -> +0.0 */
        scratch[i].idx = id;
    }
    qsort(scratch, (size_t)n, sizeof(keyed), cmp_keyed);
    for (int64_t i = 0; i < n; ++i) perm[lo + i] = scratch[i].idx;

    int64_t nl = n / 2;
    double mid = 0.5 * (rect[2 * axis] + rect[2 * axis + 1]);
    double line;
    if (nl > 0)
        line = 0.5 * (scratch[nl - 1].key + scratch[nl].key);
    else if (n > 0)
        line = (mid <= scratch[0].key) ? mid : scratch[0].key;
    else
        line = mid;

    memcpy(left, rect, 4 * sizeof(double));
    memcpy(right, rect, 4 * sizeof(double));
    left[2 * axis + 1] = line;
    right[2 * axis] = line;
    *axis_out = axis;
    *line_out = line;
}

int oracle_build_tree(int64_t n_src, const double *src_xy, int64_t n_tgt,
                      const double *tgt_xy, int L, uint32_t *perm, double *box_rect,
                      int64_t *box_src, int8_t *split_axis, double *split_line,
                      uint32_t *tperm, int64_t *box_tgt)
{
    if (n_src < 1 || L < 0 || L > 12) return -1;
    int64_t nb = oracle_n_boxes(L);

    /* root rectangle: bounding box of sources and targets */
    double x0 = src_xy[0], x1 = src_xy[0], y0 = src_xy[1], y1 = src_xy[1];
    for (int64_t j = 0; j < n_src; ++j) {
        double x = src_xy[2 * j], y = src_xy[2 * j + 1];
        if (x < x0) x0 = x;
        if (x > x1) x1 = x;
        if (y < y0) y0 = y;
        if (y > y1) y1 = y;
    }
    if (tgt_xy) {
        for (int64_t i = 0; i < n_tgt; ++i) {
            double x = tgt_xy[2 * i], y = tgt_xy[2 * i + 1];
            if (x < x0) x0 = x;
            if (x > x1) x1 = x;
            if (y < y0) y0 = y;
            if (y > y1) y1 = y;
        }
    }
    box_rect[0] = x0 + 0.0;
    box_rect[1] = x1 + 0.0;
    box_rect[2] = y0 + 0.0;
    box_rect[3] = y1 + 0.0;
    box_src[0] = 0;
    box_src[1] = n_src;
    for (int64_t j = 0; j < n_src; ++j) perm[j] = (uint32_t)j;

    keyed *scratch = (keyed *)malloc((size_t)n_src * sizeof(keyed));
    if (!scratch) return -2;

    for (int l = 0; l < L; ++l) {
        int64_t nbl = INT64_C(1) << (2 * l);
        for (int64_t b = 0; b < nbl; ++b) {
            int64_t g = level_base(l) + b;
            int64_t lo = box_src[2 * g], n = box_src[2 * g + 1];
            double half[2][4];
            int a1;
            double l1;
            split_box(src_xy, perm, lo, n, &box_rect[4 * g], scratch, &a1, &l1, half[0], half[1]);
            split_axis[3 * g] = (int8_t)a1;
            split_line[3 * g] = l1;
            int64_t nh[2] = {n / 2, n - n / 2};
            int64_t lh[2] = {lo, lo + n / 2};
            for (int h1 = 0; h1 < 2; ++h1) {
                double quad[2][4];
                int a2;
                double l2;
                split_box(src_xy, perm, lh[h1], nh[h1], half[h1], scratch, &a2, &l2, quad[0], quad[1]);
                split_axis[3 * g + 1 + h1] = (int8_t)a2;
                split_line[3 * g + 1 + h1] = l2;
                int64_t nq[2] = {nh[h1] / 2, nh[h1] - nh[h1] / 2};
                int64_t lq[2] = {lh[h1], lh[h1] + nh[h1] / 2};
                for (int h2 = 0; h2 < 2; ++h2) {
                    int64_t c = level_base(l + 1) + 4 * b + 2 * h1 + h2;
                    memcpy(&box_rect[4 * c], quad[h2], 4 * sizeof(double));
                    box_src[2 * c] = lq[h2];
                    box_src[2 * c + 1] = nq[h2];
                }
            }
        }
    }
    free(scratch);

    /* evaluation points */
    if (!tgt_xy) {
        for (int64_t j = 0; j < n_src; ++j) tperm[j] = perm[j];
        memcpy(box_tgt, box_src, (size_t)(2 * nb) * sizeof(int64_t));
        return 0;
    }
    int64_t nleaf = INT64_C(1) << (2 * L);
    int64_t *leaf_of = (int64_t *)malloc((size_t)(n_tgt > 0 ? n_tgt : 1) * sizeof(int64_t));
    int64_t *count = (int64_t *)calloc((size_t)nleaf + 1, sizeof(int64_t));
    if (!leaf_of || !count) {
        free(leaf_of);
        free(count);
        return -2;
    }
    for (int64_t i = 0; i < n_tgt; ++i) {
        double t[2] = {tgt_xy[2 * i], tgt_xy[2 * i + 1]};
        int64_t b = 0;
        for (int l = 0; l < L; ++l) {
            int64_t g = level_base(l) + b;
            int h1 = t[split_axis[3 * g]] <= split_line[3 * g] ? 0 : 1;
            int h2 = t[split_axis[3 * g + 1 + h1]] <= split_line[3 * g + 1 + h1] ? 0 : 1;
            b = 4 * b + 2 * h1 + h2;
        }
        leaf_of[i] = b;
        count[b + 1]++;
    }
    for (int64_t b = 0; b < nleaf; ++b) count[b + 1] += count[b];
    /* stable counting sort by leaf: original index order inside a leaf */
    int64_t *fill = (int64_t *)malloc((size_t)nleaf * sizeof(int64_t));
    if (!fill) {
        free(leaf_of);
        free(count);
        return -2;
    }
    memcpy(fill, count, (size_t)nleaf * sizeof(int64_t));
    for (int64_t i = 0; i < n_tgt; ++i) tperm[fill[leaf_of[i]]++] = (uint32_t)i;
    for (int l = 0; l <= L; ++l) {
        int64_t span = INT64_C(1) << (2 * (L - l));
        int64_t nbl = INT64_C(1) << (2 * l);
        for (int64_t b = 0; b < nbl; ++b) {
            int64_t g = level_base(l) + b;
            box_tgt[2 * g] = count[b * span];
            box_tgt[2 * g + 1] = count[(b + 1) * span] - count[b * span];
        }
    }
    free(fill);
    free(leaf_of);
    free(count);
    return 0;
}

/* ------------------------------------------------------------------ */
/* Connectivity (Sec. 2, theta-criterion Eq. 3; directed lists).         */
/* ------------------------------------------------------------------ */

static void centre_radius(const double *rc, double *cx, double *cy, double *rad)
{
    *cx = 0.5 * (rc[0] + rc[1]);
    *cy = 0.5 * (rc[2] + rc[3]);
    double w = rc[1] - rc[0], h = rc[3] - rc[2];
    *rad = 0.5 * sqrt(w * w + h * h);
}

int oracle_well_separated(const double *rect_b, const double *rect_c, double theta)
{
    double bx, by, rb, cx, cy, rc;
    centre_radius(rect_b, &bx, &by, &rb);
    centre_radius(rect_c, &cx, &cy, &rc);
    double dx = bx - cx, dy = by - cy;
    double d = sqrt(dx * dx + dy * dy);
    double R = rb > rc ? rb : rc, r = rb > rc ? rc : rb;
    return d > 0.0 && (R + theta * r) <= theta * d;
}

/* Directed weak (M2L) and strong lists for every box, global box ids.
 * strong(root) = {root}; for a box b at level l >= 1 the candidates are the
 * children of strong(parent(b)), taken in list order, children 0..3; each
 * is weak if well separated from b, else strong.  Offsets are CSR over all
 * boxes.  Lists are written only when the capacity suffices; the needed
 * sizes are returned either way. */
int oracle_connect(int L, const double *box_rect, double theta, int64_t *weak_off,
                   int32_t *weak, int64_t cap_w, int64_t *strong_off, int32_t *strong,
                   int64_t cap_s, int64_t *n_weak, int64_t *n_strong)
{
    int64_t nb = oracle_n_boxes(L);
    /* lists are built level by level; keep them in a growing buffer */
    int64_t sw = 0, ss = 0;
    int64_t capw_int = 1024, caps_int = 1024;
    int32_t *W = (int32_t *)malloc((size_t)capw_int * sizeof(int32_t));
    int32_t *S = (int32_t *)malloc((size_t)caps_int * sizeof(int32_t));
    int64_t *wo = (int64_t *)malloc((size_t)(nb + 1) * sizeof(int64_t));
    int64_t *so = (int64_t *)malloc((size_t)(nb + 1) * sizeof(int64_t));
    if (!W || !S || !wo || !so) return -2;
    wo[0] = 0;
    so[0] = 0;
    /* root */
    S[ss++] = 0;
    wo[1] = sw;
    so[1] = ss;
    for (int l = 1; l <= L; ++l) {
        int64_t nbl = INT64_C(1) << (2 * l);
        for (int64_t b = 0; b < nbl; ++b) {
            int64_t g = level_base(l) + b;
            int64_t par = level_base(l - 1) + b / 4;
            for (int64_t e = so[par]; e < so[par + 1]; ++e) {
                int64_t s_local = S[e] - level_base(l - 1);
                for (int ch = 0; ch < 4; ++ch) {
                    int64_t c = level_base(l) + 4 * s_local + ch;
                    if (oracle_well_separated(&box_rect[4 * g], &box_rect[4 * c], theta)) {
                        if (sw == capw_int) {
                            capw_int *= 2;
                            W = (int32_t *)realloc(W, (size_t)capw_int * sizeof(int32_t));
                        }
                        W[sw++] = (int32_t)c;
                    } else {
                        if (ss == caps_int) {
                            caps_int *= 2;
                            S = (int32_t *)realloc(S, (size_t)caps_int * sizeof(int32_t));
                        }
                        S[ss++] = (int32_t)c;
                    }
                }
            }
            wo[g + 1] = sw;
            so[g + 1] = ss;
        }
    }
    *n_weak = sw;
    *n_strong = ss;
    memcpy(weak_off, wo, (size_t)(nb + 1) * sizeof(int64_t));
    memcpy(strong_off, so, (size_t)(nb + 1) * sizeof(int64_t));
    if (weak && cap_w >= sw) memcpy(weak, W, (size_t)sw * sizeof(int32_t));
    if (strong && cap_s >= ss) memcpy(strong, S, (size_t)ss * sizeof(int32_t));
    free(W);
    free(S);
    free(wo);
    free(so);
    return 0;
}

/* Shrink-wrapped boxes: the geometry of a box (centre and radius for the
 * theta-criterion and for the expansions) taken from the bounding rectangle
 * of the points it holds (its sources, and its evaluation points when they
 * are separate), coordinates read with -0.0 as +0.0; a box without points
 * keeps its split rectangle.  The splits themselves do not change. */
void oracle_tight_rects(int L, const double *box_rect, const int64_t *box_src,
                        const uint32_t *perm, const double *src_xy, const int64_t *box_tgt,
                        const uint32_t *tperm, const double *tgt_xy, double *out)
{
    int64_t nb = oracle_n_boxes(L);
    for (int64_t g = 0; g < nb; ++g) {
        int any = 0;
        double x0 = 0, x1 = 0, y0 = 0, y1 = 0;
        for (int pass = 0; pass < (tgt_xy ? 2 : 1); ++pass) {
            const int64_t *range = pass ? box_tgt : box_src;
            const uint32_t *pm = pass ? tperm : perm;
            const double *xy = pass ? tgt_xy : src_xy;
            for (int64_t t = 0; t < range[2 * g + 1]; ++t) {
                uint32_t j = pm[range[2 * g] + t];
                double x = xy[2 * j] + 0.0, y = xy[2 * j + 1] + 0.0;
                if (!any) {
                    x0 = x1 = x;
                    y0 = y1 = y;
                    any = 1;
                    continue;
                }
                if (x < x0) x0 = x;
                if (x > x1) x1 = x;
                if (y < y0) y0 = y;
                if (y > y1) y1 = y;
            }
        }
        if (any) {
            out[4 * g] = x0;
            out[4 * g + 1] = x1;
            out[4 * g + 2] = y0;
            out[4 * g + 3] = y1;
        } else {
            for (int k = 0; k < 4; ++k) out[4 * g + k] = box_rect[4 * g + k];
        }
    }
}

/* Leaf shortcut (Sec. 2): at the finest level every strongly coupled pair
 * (t, s), s != t, is tested again with the roles of r and R interchanged,
 * r + theta R <= theta d (r = min radius, R = max radius).  A pair that
 * passes is not summed directly: if s is the larger box its sources go into
 * t's local expansion (P2L list of t), otherwise s's multipole is evaluated
 * at t's points (M2P list of t).  The rest stays in the near (P2P) list.
 * Offsets are over the leaves (4^L + 1 entries), entries are global box ids,
 * each list keeps the order of strong(t).  Capacities are the number of
 * leaf-level strong entries.  A pair also needs r > 0: the test then gives
 * |y - x| >= d - R - r >= r (1/theta - 1) > 0 for every point pair of the two
 * boxes, while a box of radius 0 (all its points equal) can touch a corner of
 * the larger box, where a point of that box may coincide with it. */
int oracle_leaf_shortcut(int L, const double *box_rect, double theta, const int64_t *strong_off,
                         const int32_t *strong, int64_t *near_off, int32_t *near,
                         int64_t *p2l_off, int32_t *p2l, int64_t *m2p_off, int32_t *m2p)
{
    int64_t base = level_base(L), nleaf = INT64_C(1) << (2 * L);
    int64_t nn = 0, np = 0, nm = 0;
    near_off[0] = p2l_off[0] = m2p_off[0] = 0;
    for (int64_t b = 0; b < nleaf; ++b) {
        int64_t g = base + b;
        double tx, ty, rt, sx, sy, rs;
        centre_radius(&box_rect[4 * g], &tx, &ty, &rt);
        for (int64_t e = strong_off[g]; e < strong_off[g + 1]; ++e) {
            int32_t sb = strong[e];
            centre_radius(&box_rect[4 * (int64_t)sb], &sx, &sy, &rs);
            double dx = tx - sx, dy = ty - sy;
            double d = sqrt(dx * dx + dy * dy);
            double R = rt > rs ? rt : rs, r = rt > rs ? rs : rt;
            int pass = sb != g && r > 0.0 && (r + theta * R) <= theta * d;
            if (!pass)
                near[nn++] = sb;
            else if (rs > rt)
                p2l[np++] = sb;
            else
                m2p[nm++] = sb;
        }
        near_off[b + 1] = nn;
        p2l_off[b + 1] = np;
        m2p_off[b + 1] = nm;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* The FMM evaluation (Sec. 2 upward/downward phases, Sec. 3.3).        */
/* ------------------------------------------------------------------ */

typedef struct {
    int L, p;
    const double *rect;
    const int64_t *box_src, *box_tgt;
    const uint32_t *perm, *tperm;
    const int64_t *weak_off, *strong_off;
    const int32_t *weak, *strong;
    const double *src_xy, *q, *tgt_xy;
} fmm_view;

static void centre_of(const fmm_view *v, int64_t g, double *cx, double *cy)
{
    const double *rc = &v->rect[4 * g];
    *cx = 0.5 * (rc[0] + rc[1]);
    *cy = 0.5 * (rc[2] + rc[3]);
}

/* Leaf of each target (by original index). */
static int64_t *target_leaf(const fmm_view *v, int64_t n_tgt)
{
    int64_t *leaf = (int64_t *)malloc((size_t)(n_tgt > 0 ? n_tgt : 1) * sizeof(int64_t));
    if (!leaf) return NULL;
    int64_t base = level_base(v->L), nleaf = INT64_C(1) << (2 * v->L);
    for (int64_t b = 0; b < nleaf; ++b) {
        int64_t g = base + b;
        for (int64_t t = 0; t < v->box_tgt[2 * g + 1]; ++t)
            leaf[v->tperm[v->box_tgt[2 * g] + t]] = g;
    }
    return leaf;
}

/* M2L into the local expansion of box g from every box of its weak list,
 * in list order. */
static void m2l_box(const fmm_view *v, int64_t g, const double *A, double *B)
{
    const int64_t P1 = v->p + 1;
    double tx, ty;
    centre_of(v, g, &tx, &ty);
    for (int64_t e = v->weak_off[g]; e < v->weak_off[g + 1]; ++e) {
        int64_t s = v->weak[e];
        double sx, sy;
        centre_of(v, s, &sx, &sy);
        oracle_m2l(v->p, sx, sy, tx, ty, &A[s * P1 * 2], &B[g * P1 * 2]);
    }
}

/* What the evaluation at one point reads (see eval_point). */
typedef struct {
    const fmm_view *v;
    const double *A, *B;
    const int64_t *leaf;
    int64_t lb;
    const int64_t *sample;
    double *phi;
    const int64_t *near_off;
    const int32_t *near;
    const int64_t *m2p_off;
    const int32_t *m2p;
    int kernel;
} point_ctx;

/* L2P (+ M2P with the leaf shortcut) and the near-field P2P at evaluation
 * point s (or sample[s]); the sources are summed in list order. */
static void eval_point(const point_ctx *c, int64_t s)
{
    const fmm_view *v = c->v;
    const int p = v->p, kernel = c->kernel;
    const int64_t P1 = p + 1, lb = c->lb;
    const int64_t *box_src = v->box_src, *strong_off = v->strong_off;
    const int32_t *strong = v->strong;
    const uint32_t *perm = v->perm;
    const double *src_xy = v->src_xy, *q = v->q, *tgt_xy = v->tgt_xy;
    const int64_t *near_off = c->near_off, *m2p_off = c->m2p_off;
    const int32_t *near = c->near, *m2p = c->m2p;
    const int64_t *sample = c->sample;
    double *phi = c->phi;
    int64_t i = sample ? sample[s] : s;
    int64_t g = c->leaf[i];
    double cx, cy, val[2];
    centre_of(v, g, &cx, &cy);
    const double yx = tgt_xy[2 * i], yy = tgt_xy[2 * i + 1];
    /* kernel 1 (harmonic): u = -d/dy of the log potential */
    if (kernel)
        oracle_l2p_deriv(p, cx, cy, &c->B[g * P1 * 2], yx, yy, val);
    else
        oracle_l2p(p, cx, cy, &c->B[g * P1 * 2], yx, yy, val);
    cplx acc = kernel ? -CMPLX(val[0], val[1]) : CMPLX(val[0], val[1]);
    /* leaf shortcut, M2P: multipoles of the smaller boxes at the point */
    if (m2p_off) {
        int64_t bl = g - lb;
        for (int64_t e = m2p_off[bl]; e < m2p_off[bl + 1]; ++e) {
            int64_t sb = m2p[e];
            double sx, sy, mv[2];
            centre_of(v, sb, &sx, &sy);
            if (kernel) {
                oracle_m2p_deriv(p, sx, sy, &c->A[sb * P1 * 2], yx, yy, mv);
                acc -= CMPLX(mv[0], mv[1]);
            } else {
                oracle_m2p(p, sx, sy, &c->A[sb * P1 * 2], yx, yy, mv);
                acc += CMPLX(mv[0], mv[1]);
            }
        }
    }
    const int64_t e_lo = near_off ? near_off[g - lb] : strong_off[g];
    const int64_t e_hi = near_off ? near_off[g - lb + 1] : strong_off[g + 1];
    const int32_t *nl = near_off ? near : strong;
    for (int64_t e = e_lo; e < e_hi; ++e) {
        int64_t sb = nl[e];
        for (int64_t t = 0; t < box_src[2 * sb + 1]; ++t) {
            uint32_t j = perm[box_src[2 * sb] + t];
            double dx = yx - src_xy[2 * j], dy = yy - src_xy[2 * j + 1];
            if (dx == 0.0 && dy == 0.0) continue;
            if (kernel)
                acc += CMPLX(q[2 * j], q[2 * j + 1]) /
                       CMPLX(src_xy[2 * j] - yx, src_xy[2 * j + 1] - yy);
            else
                acc += CMPLX(q[2 * j], q[2 * j + 1]) * clog(CMPLX(dx, dy));
        }
    }
    phi[2 * s] = creal(acc);
    phi[2 * s + 1] = cimag(acc);
}

int oracle_fmm_evaluate(int L, int p, const double *box_rect, const int64_t *box_src,
                        const int64_t *box_tgt, const uint32_t *perm, const uint32_t *tperm,
                        const int64_t *weak_off, const int32_t *weak, const int64_t *strong_off,
                        const int32_t *strong, int64_t n_src, const double *src_xy,
                        const double *q, int64_t n_tgt, const double *tgt_xy,
                        int64_t n_sample, const int64_t *sample, double *phi,
                        double *seconds, const int64_t *near_off, const int32_t *near,
                        const int64_t *p2l_off, const int32_t *p2l, const int64_t *m2p_off,
                        const int32_t *m2p, int kernel)
{
    (void)n_src;
    double t_start = now_s();
    if (p < 1 || p > MAXP) return -1;
    (void)binom(0, 0); /* fill the binomial table before any threads start */
    fmm_view v = {L, p, box_rect, box_src, box_tgt, perm, tperm, weak_off, strong_off,
                  weak, strong, src_xy, q, tgt_xy};
    int64_t nb = oracle_n_boxes(L);
    int64_t P1 = p + 1;
    double *A = (double *)calloc((size_t)(nb * P1 * 2), sizeof(double)); /* multipoles */
    double *B = (double *)calloc((size_t)(nb * P1 * 2), sizeof(double)); /* locals */
    double *tmp_xy = (double *)malloc((size_t)(2 * (n_src > 0 ? n_src : 1)) * sizeof(double));
    double *tmp_q = (double *)malloc((size_t)(2 * (n_src > 0 ? n_src : 1)) * sizeof(double));
    int64_t *leaf = target_leaf(&v, n_tgt);
    if (!A || !B || !tmp_xy || !tmp_q || !leaf) return -2;

    /* P2M at the leaves */
    int64_t lb = level_base(L), nleaf = INT64_C(1) << (2 * L);
    for (int64_t b = 0; b < nleaf; ++b) {
        int64_t g = lb + b, lo = box_src[2 * g], n = box_src[2 * g + 1];
        for (int64_t t = 0; t < n; ++t) {
            uint32_t j = perm[lo + t];
            tmp_xy[2 * t] = src_xy[2 * j];
            tmp_xy[2 * t + 1] = src_xy[2 * j + 1];
            tmp_q[2 * t] = q[2 * j];
            tmp_q[2 * t + 1] = q[2 * j + 1];
        }
        double cx, cy;
        centre_of(&v, g, &cx, &cy);
        oracle_p2m(p, cx, cy, n, tmp_xy, tmp_q, &A[g * P1 * 2]);
    }
    /* upward pass: M2M, finest level first */
    for (int l = L - 1; l >= 0; --l) {
        int64_t nbl = INT64_C(1) << (2 * l);
        for (int64_t b = 0; b < nbl; ++b) {
            int64_t g = level_base(l) + b;
            double px, py;
            centre_of(&v, g, &px, &py);
            for (int ch = 0; ch < 4; ++ch) {
                int64_t c = level_base(l + 1) + 4 * b + ch;
                double cx, cy;
                centre_of(&v, c, &cx, &cy);
                oracle_m2m(p, cx, cy, px, py, &A[c * P1 * 2], &A[g * P1 * 2]);
            }
        }
    }
    /* downward pass: M2L on every weak pair, then L2L root to leaves; the
     * local expansion of box g gets its weak list's terms in list order */
    if (g_threads > 1) {
#pragma omp parallel for schedule(dynamic, 64) num_threads(g_threads)
        for (int64_t g = 0; g < nb; ++g) m2l_box(&v, g, A, B);
    } else {
        for (int64_t g = 0; g < nb; ++g) m2l_box(&v, g, A, B);
    }
    for (int l = 1; l <= L; ++l) {
        int64_t nbl = INT64_C(1) << (2 * l);
        for (int64_t b = 0; b < nbl; ++b) {
            int64_t g = level_base(l) + b, par = level_base(l - 1) + b / 4;
            double px, py, cx, cy;
            centre_of(&v, par, &px, &py);
            centre_of(&v, g, &cx, &cy);
            oracle_l2l(p, px, py, cx, cy, &B[par * P1 * 2], &B[g * P1 * 2]);
        }
    }
    /* leaf shortcut, P2L: sources of the larger boxes into the leaf's local */
    if (p2l_off) {
        for (int64_t b = 0; b < nleaf; ++b) {
            int64_t g = lb + b;
            double cx, cy;
            centre_of(&v, g, &cx, &cy);
            for (int64_t e = p2l_off[b]; e < p2l_off[b + 1]; ++e) {
                int64_t sb = p2l[e], lo = box_src[2 * sb], n = box_src[2 * sb + 1];
                for (int64_t t = 0; t < n; ++t) {
                    uint32_t j = perm[lo + t];
                    tmp_xy[2 * t] = src_xy[2 * j];
                    tmp_xy[2 * t + 1] = src_xy[2 * j + 1];
                    tmp_q[2 * t] = q[2 * j];
                    tmp_q[2 * t + 1] = q[2 * j + 1];
                }
                oracle_p2l(p, cx, cy, n, tmp_xy, tmp_q, &B[g * P1 * 2]);
            }
        }
    }
    /* L2P and P2P at the evaluation points */
    double t_mid = now_s();
    int64_t n_out = sample ? n_sample : n_tgt;
    const point_ctx pc = {&v, A, B, leaf, lb, sample, phi, near_off, near, m2p_off, m2p,
                          kernel};
    if (g_threads > 1) {
#pragma omp parallel for schedule(dynamic, 16) num_threads(g_threads)
        for (int64_t s = 0; s < n_out; ++s) eval_point(&pc, s);
    } else {
        for (int64_t s = 0; s < n_out; ++s) eval_point(&pc, s);
    }
    if (seconds) {
        seconds[0] = t_mid - t_start; /* P2M, M2M, M2L, L2L */
        seconds[1] = now_s() - t_mid; /* L2P + P2P at the evaluation points */
    }
    free(A);
    free(B);
    free(tmp_xy);
    free(tmp_q);
    free(leaf);
    return 0;
}

/* Branch-consistent direct sum.  Each far pair (i, j) handled through the
 * weak pair (t, s) at some level contributes q_j [Log(c_t - c_s) + Log(1+u)],
 * u = ((y_i - c_t) - (x_j - c_s)) / (c_t - c_s), which is the branch of
 * Log(y_i - x_j) that the expansions converge to; near pairs contribute
 * q_j Log(y_i - x_j).  Without truncation this is what the FMM computes. */
int oracle_direct_branch(int L, const double *box_rect, const int64_t *box_src,
                         const int64_t *box_tgt, const uint32_t *perm, const uint32_t *tperm,
                         const int64_t *weak_off, const int32_t *weak,
                         const int64_t *strong_off, const int32_t *strong,
                         const double *src_xy, const double *q, int64_t n_tgt,
                         const double *tgt_xy, int64_t n_sample, const int64_t *sample,
                         double *phi, const int64_t *near_off, const int32_t *near,
                         const int64_t *p2l_off, const int32_t *p2l, const int64_t *m2p_off,
                         const int32_t *m2p)
{
    fmm_view v = {L, 0, box_rect, box_src, box_tgt, perm, tperm, weak_off, strong_off,
                  weak, strong, src_xy, q, tgt_xy};
    int64_t *leaf = target_leaf(&v, n_tgt);
    if (!leaf) return -2;
    int64_t n_out = sample ? n_sample : n_tgt;
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t s = 0; s < n_out; ++s) {
        int64_t i = sample ? sample[s] : s;
        cplx y = CMPLX(tgt_xy[2 * i], tgt_xy[2 * i + 1]);
        cplx acc = 0.0;
        int64_t leaf_local = leaf[i] - level_base(L);
        for (int l = 1; l <= L; ++l) {
            int64_t g = level_base(l) + (leaf_local >> (2 * (L - l)));
            double tx, ty;
            centre_of(&v, g, &tx, &ty);
            cplx ct = CMPLX(tx, ty);
            for (int64_t e = weak_off[g]; e < weak_off[g + 1]; ++e) {
                int64_t sb = weak[e];
                double sx, sy;
                centre_of(&v, sb, &sx, &sy);
                cplx cs = CMPLX(sx, sy), D = ct - cs;
                cplx logD = clog(D);
                for (int64_t t = 0; t < box_src[2 * sb + 1]; ++t) {
                    uint32_t j = perm[box_src[2 * sb] + t];
                    cplx x = CMPLX(src_xy[2 * j], src_xy[2 * j + 1]);
                    cplx u = ((y - ct) - (x - cs)) / D;
                    acc += CMPLX(q[2 * j], q[2 * j + 1]) * (logD + clog(1.0 + u));
                }
            }
        }
        int64_t g = leaf[i];
        const int64_t bl = g - level_base(L);
        double tx, ty;
        centre_of(&v, g, &tx, &ty);
        const cplx ct = CMPLX(tx, ty);
        if (p2l_off) { /* P2L pairs: Log(c_t - x) + Log(1 + (y - c_t)/(c_t - x)) */
            for (int64_t e = p2l_off[bl]; e < p2l_off[bl + 1]; ++e) {
                int64_t sb = p2l[e];
                for (int64_t t = 0; t < box_src[2 * sb + 1]; ++t) {
                    uint32_t j = perm[box_src[2 * sb] + t];
                    cplx x = CMPLX(src_xy[2 * j], src_xy[2 * j + 1]);
                    acc += CMPLX(q[2 * j], q[2 * j + 1]) *
                           (clog(ct - x) + clog(1.0 + (y - ct) / (ct - x)));
                }
            }
        }
        if (m2p_off) { /* M2P pairs: Log(y - c_s) + Log(1 - (x - c_s)/(y - c_s)) */
            for (int64_t e = m2p_off[bl]; e < m2p_off[bl + 1]; ++e) {
                int64_t sb = m2p[e];
                double sx, sy;
                centre_of(&v, sb, &sx, &sy);
                cplx cs = CMPLX(sx, sy);
                for (int64_t t = 0; t < box_src[2 * sb + 1]; ++t) {
                    uint32_t j = perm[box_src[2 * sb] + t];
                    cplx x = CMPLX(src_xy[2 * j], src_xy[2 * j + 1]);
                    acc += CMPLX(q[2 * j], q[2 * j + 1]) *
                           (clog(y - cs) + clog(1.0 - (x - cs) / (y - cs)));
                }
            }
        }
        const int64_t e_lo = near_off ? near_off[bl] : strong_off[g];
        const int64_t e_hi = near_off ? near_off[bl + 1] : strong_off[g + 1];
        const int32_t *nl = near_off ? near : strong;
        for (int64_t e = e_lo; e < e_hi; ++e) {
            int64_t sb = nl[e];
            for (int64_t t = 0; t < box_src[2 * sb + 1]; ++t) {
                uint32_t j = perm[box_src[2 * sb] + t];
                double dx = creal(y) - src_xy[2 * j], dy = cimag(y) - src_xy[2 * j + 1];
                if (dx == 0.0 && dy == 0.0) continue;
                acc += CMPLX(q[2 * j], q[2 * j + 1]) * clog(CMPLX(dx, dy));
            }
        }
        phi[2 * s] = creal(acc);
        phi[2 * s + 1] = cimag(acc);
    }
    free(leaf);
    return 0;
}
