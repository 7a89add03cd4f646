/*
 * fmm_oracle.h -- declarations of the FP64 CPU oracle (test infrastructure
 * only; see fmm_oracle.c).  Shares nothing with the CUDA library's headers.
 *
 * Box numbering: level-major, box b of level l has global id (4^l - 1)/3 + b;
 * its children are boxes 4b .. 4b+3 of level l+1.
 * Complex numbers are stored as (re, im) pairs of doubles.
 */
#ifndef FMM_ORACLE_H
#define FMM_ORACLE_H
#include <stdint.h>

int64_t oracle_n_boxes(int L);
/* Threads for the FMM's independent per-target loops (M2L per target box,
 * L2P + P2P per evaluation point); 1 = serial, the default.  Results do not
 * depend on it. */
void oracle_set_threads(int n);
int oracle_levels_cap(int64_t n, int leaf);
int oracle_levels_eq(int64_t n, int nd);

void oracle_direct(int64_t n_src, const double *src_xy, const double *q, int64_t n_tgt,
                   const double *tgt_xy, double *phi);
void oracle_direct_sample(int64_t n_src, const double *src_xy, const double *q,
                          const double *tgt_xy, int64_t n_sample, const int64_t *sample,
                          double *phi);

void oracle_p2m(int p, double cx, double cy, int64_t n, const double *xy, const double *q,
                double *a);
void oracle_m2p(int p, double cx, double cy, const double *a, double zx, double zy,
                double *out);
void oracle_m2m(int p, double zcx, double zcy, double zpx, double zpy, const double *a,
                double *out);
void oracle_m2l(int p, double zsx, double zsy, double ztx, double zty, const double *a,
                double *b);
void oracle_l2l(int p, double zpx, double zpy, double zcx, double zcy, const double *b,
                double *out);
void oracle_l2p(int p, double cx, double cy, const double *b, double zx, double zy,
                double *out);

void oracle_p2l(int p, double cx, double cy, int64_t n, const double *xy, const double *q,
                double *b);
void oracle_tight_rects(int L, const double *box_rect, const int64_t *box_src,
                        const uint32_t *perm, const double *src_xy, const int64_t *box_tgt,
                        const uint32_t *tperm, const double *tgt_xy, double *out);
int oracle_leaf_shortcut(int L, const double *box_rect, double theta, const int64_t *strong_off,
                         const int32_t *strong, int64_t *near_off, int32_t *near,
                         int64_t *p2l_off, int32_t *p2l, int64_t *m2p_off, int32_t *m2p);

int oracle_build_tree(int64_t n_src, const double *src_xy, int64_t n_tgt, const double *tgt_xy,
                      int L, uint32_t *perm, double *box_rect, int64_t *box_src,
                      int8_t *split_axis, double *split_line, uint32_t *tperm,
                      int64_t *box_tgt);
int oracle_well_separated(const double *rect_b, const double *rect_c, double theta);
int oracle_connect(int L, const double *box_rect, double theta, int64_t *weak_off,
                   int32_t *weak, int64_t cap_w, int64_t *strong_off, int32_t *strong,
                   int64_t cap_s, int64_t *n_weak, int64_t *n_strong);
int oracle_fmm_evaluate(int L, int p, const double *box_rect, const int64_t *box_src,
                        const int64_t *box_tgt, const uint32_t *perm, const uint32_t *tperm,
                        const int64_t *weak_off, const int32_t *weak, const int64_t *strong_off,
                        const int32_t *strong, int64_t n_src, const double *src_xy,
                        const double *q, int64_t n_tgt, const double *tgt_xy,
                        int64_t n_sample, const int64_t *sample, double *phi,
                        double *seconds /* optional [2]: expansions, evaluation points */,
                        const int64_t *near_off, const int32_t *near, const int64_t *p2l_off,
                        const int32_t *p2l, const int64_t *m2p_off, const int32_t *m2p,
                        int kernel /* 0: Eq. 1 / Eq. 2; 1: harmonic, -d/dy of it */);
void oracle_direct_harmonic(int64_t n_src, const double *src_xy, const double *q,
                            int64_t n_tgt, const double *tgt_xy, int64_t n_sample,
                            const int64_t *sample, double *u);
void oracle_l2p_deriv(int p, double cx, double cy, const double *b, double zx, double zy,
                      double *out);
void oracle_m2p_deriv(int p, double cx, double cy, const double *a, double zx, double zy,
                      double *out);
int oracle_direct_branch(int L, const double *box_rect, const int64_t *box_src,
                         const int64_t *box_tgt, const uint32_t *perm, const uint32_t *tperm,
                         const int64_t *weak_off, const int32_t *weak,
                         const int64_t *strong_off, const int32_t *strong,
                         const double *src_xy, const double *q, int64_t n_tgt,
                         const double *tgt_xy, int64_t n_sample, const int64_t *sample,
                         double *phi, const int64_t *near_off, const int32_t *near,
                         const int64_t *p2l_off, const int32_t *p2l, const int64_t *m2p_off,
                         const int32_t *m2p);
#endif
