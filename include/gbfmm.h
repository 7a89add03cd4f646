/*
 * gbfmm.h -- C ABI of the GB300 (sm_103a) adaptive 2-D fast multipole method
 * for the complex-log potential (Goude & Engblom, "Adaptive fast multipole
 * methods on the GPU", arXiv:1205.4611):
 *
 *     Phi(y_i) = sum_{j, x_j != y_i} q_j Log(y_i - x_j)      (Eq. 1, Eq. 2)
 *
 * Conventions for every entry point:
 *  - Complex numbers are two doubles (re, im), interleaved.  Points are
 *    (x, y) pairs of doubles, interleaved (x0, y0, x1, y1, ...).
 *  - Pointers named *_dev are CUDA device pointers; *_host are host pointers
 *    (pageable or pinned).  The caller owns every buffer it passes; the
 *    library never frees or keeps a caller pointer after the call returns.
 *  - `stream` is a cudaStream_t passed as void* (NULL = the legacy default
 *    stream).  Device work is enqueued on it, in stream order.
 *  - Every call returns an fmm_status; on error fmm_last_error() gives a
 *    message (thread-local, valid until the next call on the same thread).
 *    Nothing aborts, traps or prints.
 *  - The branch of the complex log: far-field pairs use the branch the
 *    expansions converge to, Log(c_t - c_s) + Log(1 + u) with
 *    u = ((y - c_t) - (x - c_s)) / (c_t - c_s) for the interacting boxes
 *    (t, s); near pairs use the principal Log.  Re(Phi) is branch-free.
 */
#ifndef GBFMM_H
#define GBFMM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fmm_tree fmm_tree; /* opaque; owned by the library */

typedef enum {
    FMM_OK = 0,
    FMM_ERR_ARG = -1,       /* invalid argument (sizes, p, theta, NULL pointer) */
    FMM_ERR_NOMEM = -2,     /* device allocation failed */
    FMM_ERR_CUDA = -3,      /* a CUDA runtime call or kernel launch failed */
    FMM_ERR_TIMEOUT = -4,   /* a bounded device-side wait gave up */
    FMM_ERR_NONFINITE = -5  /* a coordinate is NaN or infinite */
} fmm_status;

/* Precision modes. */
enum {
    FMM_PREC_FP64 = 0,  /* every step in FP64 */
    FMM_PREC_MIXED = 1  /* P2P, P2M, M2M, L2L, P2L, M2P and L2P in double-float
                           (pairs of FP32, ~48 bits; p <= 32, FP64 kernels above;
                           P2L and M2P terms c W^k with |W|^k <= 2^-25 in FP32, an
                           absolute error below 2^-49 |c|), M2L in split precision
                           on the tensor cores (p <= 31);
                           tree geometry, stored expansions and the final sums in
                           FP64.  Every leaf pair is evaluated in its own units (a
                           power of two of its radii), so any finite coordinate scale
                           is handled.  Two points closer than 2^-42 of their leaf
                           pair's scale count as coincident and are skipped (FP64:
                           exactly equal points only). */
};

/* Kernels. */
enum {
    FMM_KERNEL_LOG = 0,      /* Phi(y) = sum q_j Log(y - x_j)   (Eq. 1, Eq. 2) */
    FMM_KERNEL_HARMONIC = 1  /* u(y) = sum q_j / (x_j - y): the harmonic kernel
                                Gamma_j / (z_j - z_i) of the paper's experiments (Sec. 5),
                                = -d/dy of the log potential; no branch */
};

/* Level rules. */
enum {
    FMM_LEVELS_CAP = 0, /* L = min{L : ceil(N / 4^L) <= leaf_size} (+ level_shift) */
    FMM_LEVELS_EQ = 1   /* Eq. (Nlevels): L = ceil(0.5 log2(5/8 N / leaf_size)) */
};

typedef struct {
    int p;            /* expansion order, 1 <= p <= 64 (Eq. 4, Eq. 5) */
    double theta;     /* theta-criterion parameter, 0 < theta < 1 (Eq. 3); paper: 0.5 */
    int leaf_size;    /* N_d: particles per finest box, >= 1 */
    int level_rule;   /* FMM_LEVELS_CAP or FMM_LEVELS_EQ */
    int level_shift;  /* extra levels added to the rule's L (>= 0; autotuning) */
    int precision;    /* FMM_PREC_FP64 or FMM_PREC_MIXED */
    int m2l_slices;   /* M2L in FMM_PREC_MIXED with p <= 31: 1..5 = tcgen05 GEMM, one row
                         per weak pair, with that many fp16 digit slices (8 + 9 (s - 1)
                         bits), 0 = default (5 slices, the precision of the double-float
                         path), -1 = double-float summation sweeps (Alg. "Multipole to
                         local translation") */
    int p2p_mode;     /* 0 = default: in self-evaluation with <= 64 points per leaf (either
                         precision), each near pair of points (of distinct leaves, or of one
                         leaf) is evaluated once for both directions (Log(x - y) =
                         Log(y - x) +- i pi); 1 = one pass per evaluation point */
    int p2l_m2p;      /* 1 = leaf shortcut (Sec. 2): at the finest level, strong pairs
                         that pass the theta-criterion with r and R interchanged
                         (r + theta R <= theta d, r > 0) use P2L (source box larger)
                         or M2P (source box smaller) instead of the direct sum;
                         0 = off (default) */
    int box_fit;      /* 1 = shrink-wrapped geometry: every box's centre and radius (theta-
                         criterion, expansions) come from the bounding rectangle of the
                         points it holds (sources, and evaluation points when separate);
                         the splits do not change; 0 = the split rectangles (default) */
    int kernel;       /* FMM_KERNEL_LOG (default) or FMM_KERNEL_HARMONIC: the same tree,
                         lists and expansions; the harmonic kernel differentiates them at
                         the points (L2P, M2P) and sums q / (x - y) in the near field */
    int p2p_item_sources; /* near-field work-item size: a leaf's near list is cut into runs
                             of at most this many sources, one work item (thread block)
                             each (a single leaf may exceed it); 0 = default (2048), else
                             64 .. 65536.  Changes only the summation order */
} fmm_options;

/* Fill *opt with defaults: p = 20, theta = 0.5, leaf_size = 64,
 * FMM_LEVELS_CAP, no level shift, FMM_PREC_FP64. */
void fmm_default_options(fmm_options *opt);

/*
 * Topological phase (Sec. 3.2): build the median-split pyramid tree over the
 * sources and the directed theta-criterion interaction lists.
 *
 *  src_xy_dev : n_src points (device), n_src >= 1.
 *  tgt_xy_dev : n_tgt evaluation points (device), or NULL to evaluate at the
 *               sources (Eq. 1; n_tgt is then ignored).  Evaluation points do
 *               not move the splits; they descend the split lines (Eq. 2).
 *  opt        : options (copied).
 *  out        : receives a new tree; free it with fmm_tree_free.
 *
 * The tree keeps its own copies of the permuted points, so the caller's
 * buffers may be reused once the call returns.  The call synchronises the
 * stream while it sizes the interaction lists (and reports device errors
 * found up to then); the last steps (work-item tables) stay queued on the
 * stream, and fmm_evaluate on any stream waits for them.  Errors:
 * FMM_ERR_ARG, FMM_ERR_NONFINITE, FMM_ERR_NOMEM, FMM_ERR_CUDA.
 */
fmm_status fmm_build_tree(const double *src_xy_dev, int64_t n_src, const double *tgt_xy_dev,
                          int64_t n_tgt, const fmm_options *opt, void *stream, fmm_tree **out);

/*
 * Computational phase (Sec. 3.3): P2M, M2M, M2L, L2L, L2P and P2P on a built
 * tree.
 *
 *  q_dev   : n_src complex strengths (device), in the caller's source order.
 *  phi_dev : n_tgt (or n_src) complex potentials (device), caller's target
 *            order; overwritten.
 *
 * Asynchronous on `stream`: returns once the work is enqueued.  Device-side
 * errors are latched in the tree and returned by fmm_tree_sync.  A tree may
 * be evaluated any number of times with new strengths.  It holds the
 * expansion buffers, so evaluations of one tree run one after the other: an
 * evaluation queued on another stream than the previous one waits (on the
 * device) for that one.  Unless phase timing is on, the far field (P2M .. M2L,
 * L2L, P2L) runs on a second stream of the library's own beside the near field
 * on `stream`, which waits for it (on the device) before the final
 * combination: work the caller queues on `stream` afterwards sees the
 * complete result.
 */
fmm_status fmm_evaluate(fmm_tree *tree, const double *q_dev, double *phi_dev, void *stream);

/* Wait for the tree's work on `stream` and return any latched device error. */
fmm_status fmm_tree_sync(fmm_tree *tree, void *stream);

/*
 * One FMM end to end from HOST buffers: copy points and strengths to the
 * device, build, evaluate, copy the potentials back; synchronous.
 *  src_xy_host : n_src points; tgt_xy_host : n_tgt points or NULL;
 *  q_host : n_src complex; phi_host : n_tgt (or n_src) complex, overwritten.
 */
fmm_status fmm_solve_host(const double *src_xy_host, int64_t n_src, const double *tgt_xy_host,
                          int64_t n_tgt, const double *q_host, double *phi_host,
                          const fmm_options *opt, void *stream);

/*
 * Batched form: many independent problems (Eq. 1 for each, or Eq. 2 with
 * evaluation points of its own).  Instance i owns sources
 * [src_off[i], src_off[i+1]) of the concatenated src_xy_dev; src_off is a
 * host array of n_inst+1 entries with src_off[0] = 0 and every instance
 * non-empty.  With tgt_xy_dev != NULL, instance i is evaluated at the points
 * [tgt_off[i], tgt_off[i+1]) of tgt_xy_dev (host offsets, tgt_off[0] = 0,
 * non-decreasing, at least one point in all); with tgt_xy_dev == NULL
 * (tgt_off ignored) at its sources.  Each instance gets its own tree by the
 * options' level rule; instances with the same number of levels are built
 * together as one tree of several roots (one pass of launches for all of
 * them), and the trees are merged into one forest whose evaluation runs
 * every phase for all instances in a single pass (one launch per phase and
 * level).  The returned tree is used with fmm_evaluate (q and phi are the
 * concatenated arrays in caller order: q over all sources, phi over all
 * evaluation points) and freed with fmm_tree_free.  Synchronises the stream
 * at the end.  Errors: as fmm_build_tree.
 */
fmm_status fmm_build_batched(int n_inst, const int64_t *src_off_host, const double *src_xy_dev,
                             const int64_t *tgt_off_host, const double *tgt_xy_dev,
                             const fmm_options *opt, void *stream, fmm_tree **out);

/*
 * Leaf-size autotuner: for each candidate leaf size, one untimed pass and then
 * `repeats` timed passes of a build followed by `evaluations` evaluations
 * (host clock around the synchronised work); writes the fastest candidate to
 * *best_leaf and, if ms is not NULL, the best time of every candidate to
 * ms[0 .. n_cand-1].  The other options are taken from *opt.
 *  Single problem: n_inst = 0, src_xy_dev / n_src (and optionally separate
 *  evaluation points tgt_xy_dev / n_tgt).  Batched problem: n_inst > 0 with
 *  src_off_host as in fmm_build_batched (tgt_xy_dev must be NULL).
 *  q_dev : strengths for all sources (device).
 * Synchronous.  Allocates a temporary output buffer; every tree it builds is
 * freed before it returns.
 */
fmm_status fmm_autotune_leaf(const double *src_xy_dev, int64_t n_src, const double *tgt_xy_dev,
                             int64_t n_tgt, int n_inst, const int64_t *src_off_host,
                             const double *q_dev, const fmm_options *opt, const int *candidates,
                             int n_cand, int repeats, int evaluations, void *stream,
                             int *best_leaf, float *ms);

/*
 * Autotuner of the work decomposition: times every combination of a leaf
 * size from leaf_cand[0 .. n_leaf-1] and a near-field work-item size
 * (p2p_item_sources) from item_cand[0 .. n_item-1], each as in
 * fmm_autotune_leaf (one untimed pass, the fastest of `repeats` timed passes
 * of a build and `evaluations` evaluations), and writes the fastest pair into
 * opt->leaf_size and opt->p2p_item_sources (the other options are read from
 * *opt).  ms, if not NULL, receives n_leaf * n_item best times, leaf-major.
 * Problem arguments as for fmm_autotune_leaf.  Synchronous; allocates a
 * temporary output buffer.
 */
fmm_status fmm_autotune(const double *src_xy_dev, int64_t n_src, const double *tgt_xy_dev,
                        int64_t n_tgt, int n_inst, const int64_t *src_off_host,
                        const double *q_dev, fmm_options *opt, const int *leaf_cand, int n_leaf,
                        const int *item_cand, int n_item, int repeats, int evaluations,
                        void *stream, float *ms);

/* One-shot batched evaluation: fmm_build_batched + fmm_evaluate + fmm_tree_sync
 * + fmm_tree_free (synchronous); arguments as there (tgt_xy_dev may be NULL). */
fmm_status fmm_evaluate_batched(int n_inst, const int64_t *src_off_host,
                                const int64_t *tgt_off_host, const double *src_xy_dev,
                                const double *tgt_xy_dev, const double *q_dev, double *phi_dev,
                                const fmm_options *opt, void *stream);

/* Replay evaluations of this tree as one CUDA graph (enable = 1): the first
 * fmm_evaluate after enabling, or after q, phi or the stream change, captures
 * the whole computational phase into a graph; later calls launch the graph.
 * Per-phase timings are not collected while the graph is used. */
fmm_status fmm_set_graph(fmm_tree *tree, int enable);

/* Sizes of a built tree (any output pointer may be NULL). */
fmm_status fmm_tree_info(const fmm_tree *tree, int *levels, int64_t *n_boxes, int64_t *n_weak,
                         int64_t *n_strong);

/*
 * Host copies of the topology, for checking (synchronous).  Box ids are
 * level-major: box b of level l is (4^l - 1)/3 + b, children 4b..4b+3.
 *  perm        : n_src uint32, tree position -> source index
 *  tperm       : n_tgt uint32, tree position -> target index (== perm for Eq. 1)
 *  box_rect    : n_boxes * 4 doubles (x0, x1, y0, y1)
 *  box_src     : n_boxes * 2 int64 (start, count) into perm
 *  box_tgt     : n_boxes * 2 int64 (start, count) into tperm
 *  weak_off, strong_off : n_boxes + 1 int64 each (CSR offsets)
 *  weak, strong : n_weak / n_strong int32 box ids
 * Any pointer may be NULL to skip that array.
 */
fmm_status fmm_tree_export(const fmm_tree *tree, uint32_t *perm, uint32_t *tperm, double *box_rect,
                           int64_t *box_src, int64_t *box_tgt, int64_t *weak_off, int32_t *weak,
                           int64_t *strong_off, int32_t *strong);

/* Host copy of the rectangles the box geometry comes from (the split
 * rectangles, or with box_fit = 1 the points' bounding rectangles; a box
 * without points keeps its split rectangle): n_boxes * 4 doubles (x0, x1, y0,
 * y1).  Synchronous. */
fmm_status fmm_tree_export_geometry(const fmm_tree *tree, double *box_rect);

/*
 * The leaf shortcut lists of a tree built with p2l_m2p = 1 (Sec. 2), for
 * checking (synchronous).  At each leaf the strong list (which drives the
 * direct sum without the shortcut) is split, in its own order, into
 *  near  : boxes summed directly (always holds the leaf itself),
 *  p2l   : larger boxes whose sources enter the leaf's local expansion,
 *  m2p   : smaller boxes whose multipoles are evaluated at the leaf's points.
 *  *_off : n_boxes + 1 int64 each (CSR offsets; non-leaf boxes are empty)
 *  near, p2l, m2p : n_near / n_p2l / n_m2p int32 box ids
 * fmm_tree_shortcut_info gives the three sizes.  Any pointer may be NULL.
 * A tree built without the shortcut returns FMM_ERR_ARG.
 */
fmm_status fmm_tree_shortcut_info(const fmm_tree *tree, int64_t *n_near, int64_t *n_p2l,
                                  int64_t *n_m2p);
fmm_status fmm_tree_export_shortcut(const fmm_tree *tree, int64_t *near_off, int32_t *near,
                                    int64_t *p2l_off, int32_t *p2l, int64_t *m2p_off,
                                    int32_t *m2p);

/* Per-phase device times (ms) of the last build / evaluate, when timing is
 * enabled with fmm_set_timing(tree, 1): [0] tree build, [1] connectivity,
 * [2] P2M, [3] M2M, [4] M2L, [5] L2L, [6] everything at the evaluation points
 * ([9] + [10]), [7] permutations, [8] P2L (leaf shortcut), [9] the P2P
 * kernel, [10] M2P (leaf shortcut) and L2P with the final combination.
 * Writes min(n, 11) values.  With timing on, an evaluation runs its phases
 * one after another on the caller's stream (no far-field overlap), so that
 * each span times its own kernels. */
fmm_status fmm_get_timings(const fmm_tree *tree, float *ms, int n);
fmm_status fmm_set_timing(fmm_tree *tree, int enable);

/* Release a tree (NULL is a no-op).  Waits for the tree's last evaluation,
 * on whatever stream it was queued, and for the build stream; the tree's
 * device buffers go to the library's block cache for later builds. */
void fmm_tree_free(fmm_tree *tree);

/*
 * Direct sum of Eq. (1) / Eq. (2) that allocates no device memory.  The paper
 * has no counterpart: this entry point exists for callers that cannot
 * allocate when they need a potential (code holding an allocator or pool
 * lock, real-time loops with a fixed memory budget, hosts that only lend the
 * library buffers they own).  It runs a variant of the FP64 near-field
 * kernel whose partial sums live in a static 4 MiB device array that every
 * GPU loading the library holds until the process exits.
 *
 *  src_xy_dev : n_src points (device), q_dev : n_src complex strengths (device)
 *  tgt_xy_dev : n_tgt evaluation points (device), or NULL to evaluate at the
 *               sources (exactly coincident pairs are skipped)
 *  phi_dev    : n_tgt (or n_src) complex potentials (device), overwritten,
 *               principal branch of Log.
 *
 * Sizes are limited by the static array: ceil(n_tgt/64) * ceil(n_src/2048)
 * must not exceed 4096; larger calls return FMM_ERR_ARG with a message.
 * The call makes no cudaMalloc or cudaFree (nor any allocating routine) and
 * is asynchronous on `stream`.  The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current;
 * make that first call before any stream capture.  All calls share the
 * array: calls that overlap on the GPU race and must be ordered by the
 * caller; nothing in it needs to start at zero.
 */
fmm_status fmm_direct_noalloc(const double *src_xy_dev, int64_t n_src, const double *q_dev,
                              const double *tgt_xy_dev, int64_t n_tgt, double *phi_dev,
                              void *stream);

/* Number of CUDA kernel launches this library has issued in this process
 * (all threads, all devices); for accounting work in benchmarks. */
int64_t fmm_launch_count(void);

/*
 * Device memory taken through the library's block cache, in bytes, summed
 * over all devices of the process (the paper has no counterpart; it reports
 * a tree's HBM footprint):
 *  in_use : blocks held by live trees and running calls,
 *  peak   : the largest in_use since the process started or the last reset,
 *  cached : freed blocks kept for reuse (not returned to the driver).
 * Any pointer may be NULL; reset_peak != 0 sets peak to the current in_use
 * after reading it.  Host-side bookkeeping only; never fails.
 */
fmm_status fmm_memory_info(int64_t *in_use, int64_t *peak, int64_t *cached, int reset_peak);

/*
 * Host-side fault injection for testing the error paths (the paper has no
 * counterpart).  Nothing is done on the GPU:
 *  FMM_INJECT_ALLOC_FAILURE, arg = k >= 0: the device allocation after k
 *    more successful ones fails as if the device were out of memory (the call
 *    then returns FMM_ERR_NOMEM and releases what it holds); arg < 0 disarms.
 *  FMM_INJECT_STATUS, arg = bits: the next fmm_tree_sync (any thread) ORs the
 *    bits into the device status word it read, e.g. 4 (a bounded device wait
 *    gave up) maps to FMM_ERR_TIMEOUT, 1 (non-finite input) to
 *    FMM_ERR_NONFINITE.
 * Returns FMM_ERR_ARG for an unknown `what`.
 */
enum { FMM_INJECT_ALLOC_FAILURE = 1, FMM_INJECT_STATUS = 2 };
fmm_status fmm_debug_inject(int what, int64_t arg);

/* Message of the last error on this thread ("" if none). */
const char *fmm_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GBFMM_H */
