// Internal host-side declarations of the GB300 FMM library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <string>
#include <vector>

#include "../../include/gbfmm.h"

namespace gbfmm {

// Device blocks from the library's cache (api.cu): a block freed on stream s
// is reused by later allocations on s; dev_cache_stream_idle(s, mark), called
// after a synchronisation of s that followed dev_cache_mark(), opens the
// blocks freed on s up to the mark to every stream; dev_cache_trim drains the
// device and returns every cached block to the driver.
cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);
uint64_t dev_cache_mark();
void dev_cache_stream_idle(cudaStream_t s, uint64_t mark);
void dev_cache_trim();

// Stream-ordered device buffer list owned by a tree or a call.
struct DevArena {
    cudaStream_t stream = nullptr;
    std::vector<void *> ptrs;
    cudaError_t alloc(void **p, size_t bytes);
    void release();
};

template <class T>
inline cudaError_t arena_alloc(DevArena &a, T **p, size_t count) {
    return a.alloc(reinterpret_cast<void **>(p), count * sizeof(T) + 16);
}

// Page-locked host words for small device-to-host reads (counts, totals,
// status), taken from a process-wide pool for the lifetime of the object:
// copies into them are truly asynchronous, so several reads share one
// stream synchronisation.
constexpr int HOST_STAGE_WORDS = 64;
struct HostStage {
    uint32_t *w = nullptr;
    HostStage();
    ~HostStage();
    HostStage(const HostStage &) = delete;
    HostStage &operator=(const HostStage &) = delete;
};

// Evaluation events: 0 start, 1 after the permutations, 2..6 after P2M, M2M,
// M2L, L2L, P2L, 9 / 7 around the P2P kernel, 10 / 11 around M2P, 12 / 8
// around the final combination.
constexpr int N_EVAL_EVENTS = 13;
struct Timing {
    bool enabled = false;
    cudaEvent_t ev[N_EVAL_EVENTS] = {};
    float ms[11] = {};
};
constexpr int N_TIMINGS = 11;

// A built tree (single instance or a forest of batched instances).
struct Tree {
    // options
    int p = 20;
    double theta = 0.5;
    int leaf = 64;
    int precision = 0;
    int m2l_slices = 0;
    int p2l_m2p = 0;          // leaf P2L / M2P shortcut on (Sec. 2)
    int box_fit = 0;          // geometry from the points' bounding rectangles
    int kernel = 0;           // 0: q Log(y - x); 1: harmonic, q / (x - y)
    int p2p_cap = 2048;       // near-field sources per P2P work item (a leaf may exceed it)
    // sizes
    int L = 0;                // levels of a single instance (max over instances)
    int64_t n_src = 0, n_tgt = 0;
    bool separate = false;
    int64_t n_boxes = 0;
    int n_inst = 1;
    // roots built together (instances with the same L; build_topology): box
    // ids are level-major over the roots; root r owns sources
    // [root_off[r], root_off[r+1]) and evaluation points [root_toff[r],
    // root_toff[r+1]) (host offsets; unused when n_roots == 1)
    int n_roots = 1;
    std::vector<int64_t> root_off, root_toff;
    // topology (device)
    uint32_t *perm = nullptr;   // [n_src] tree pos -> source index
    double2 *xs = nullptr;      // [n_src] permuted sources
    uint32_t *tperm = nullptr;  // [n_tgt]
    double2 *xt = nullptr;      // [n_tgt]
    double4 *rect = nullptr;    // [n_boxes] x0 x1 y0 y1 (split rectangles)
    double4 *rect_geo = nullptr;  // [n_boxes] rectangles the geometry comes from (rect, or tight)
    int2 *box_src = nullptr;    // [n_boxes] start, count
    int2 *box_tgt = nullptr;    // [n_boxes]
    double4 *geom = nullptr;    // [n_boxes] cx, cy, sigma, 1/sigma
    int8_t *split_axis = nullptr;  // [n_internal*3]
    double *split_line = nullptr;  // [n_internal*3]
    int *weak_off = nullptr, *weak = nullptr;
    int *weak_tgt = nullptr;    // [n_weak] target box of every weak entry (tensor M2L)
    int *strong_off = nullptr, *strong = nullptr;
    int64_t n_weak = 0, n_strong = 0;
    // leaf shortcut (Sec. 2): the leaf strong lists split into near (P2P),
    // P2L (source box larger) and M2P (source box smaller); CSR over all
    // boxes, empty except at leaves; allocated only with p2l_m2p
    int *near_off = nullptr, *near = nullptr;
    int *p2l_off = nullptr, *p2l = nullptr;
    int *m2p_off = nullptr, *m2p = nullptr;
    int64_t n_near = 0, n_p2l = 0, n_m2p = 0;
    const int *p2p_list = nullptr;  // list the P2P items index: strong, or near
    const int *p2p_off = nullptr;   // its CSR offsets
    // symmetric near field (p2p_sym.cu): self-evaluation, mixed, leaves <= 64 points
    bool sym = false;
    int4 *sym_items = nullptr;      // (leaf, e0, e1, row slot) over p2p_list
    int *sym_order = nullptr;
    int n_sym_items = 0;
    int4 *sym_m2p_items = nullptr;  // M2P items (leaf, 0, ~e0, ~e1)
    int *sym_m2p_order = nullptr;
    int n_sym_m2p = 0;
    int64_t sym_p2p_slots = 0;      // partial slots of the P2P items (M2P slots follow)
    int *sym_coff = nullptr;        // [n_leaves + 1] slots of each leaf, in slot order
    int *sym_cslot = nullptr;
    double2 *sym_partial = nullptr; // [slots * 64]
    // built by the connectivity step unless the symmetric near field is used
    bool p2p_items_needed = true;
    // work items per chunk of <= 64 evaluation points: P2P items (target leaf,
    // first target, run [e0, e1) of p2p_list), then, with the leaf shortcut,
    // M2P items (target leaf, first target, ~e0, ~e1) over the M2P list
    int4 *p2p_items = nullptr;
    int *p2p_order = nullptr;   // launch order: P2P items, then M2P items, each by
                                // decreasing cost
    int n_items = 0;
    int n_p2p_items = 0;        // order[0, n_p2p_items) are the P2P items
    int2 *p2p_chunks = nullptr; // (target leaf, first target) per chunk of <= 64 targets
    int *p2p_item0 = nullptr;   // [n_chunks+1] first item of each chunk
    int n_chunks = 0;
    double2 *p2p_partial = nullptr;  // [n_items * 64] partial near-field sums
    // box relations (explicit, so that a forest of trees uses the same kernels)
    int *parent = nullptr;      // [n_boxes] parent id, -1 for roots
    int *child0 = nullptr;      // [n_boxes] first child id, -1 for leaves
    int *lvl_boxes = nullptr;   // box ids grouped by level; level l is
                                // [level_start[l], level_start[l+1])
    int *leaves = nullptr;      // ids of the leaf boxes
    int n_leaves = 0;
    // evaluation buffers
    double2 *qs = nullptr;      // [n_src] permuted strengths
    // mixed precision (df32 near field)
    float4 *xs_loc = nullptr;   // [n_src] df32 offsets from the leaf centre
    float4 *xt_loc = nullptr;   // [n_tgt]
    float4 *qs_df = nullptr;    // [n_src] df32 permuted strengths
    float4 *mpole_df = nullptr; // [n_boxes*(p+1)] df32 multipoles
    int2 *m2l_items = nullptr;  // (target box, first weak entry) runs of <= 64 pairs
    uint4 *m2l_bslices = nullptr;  // tensor M2L: digit slices of the operator
    int *m2l_fexp = nullptr;       // tensor M2L: per-row exponents of the operator
    // tensor M2L pair table (tree geometry only, built once): per weak entry
    // ir = 2^e0 / r and Log(z_t - z_s) (double-float complex), exponent offsets
    float4 *m2l_pir = nullptr;
    float4 *m2l_plog = nullptr;
    int2 *m2l_pa = nullptr;
    int n_m2l_items = 0;
    uint32_t *m2l_cnt = nullptr;   // [n_boxes + 1] M2L items per box, scanned (build time)
    uint32_t *sym_cnt = nullptr;   // [3 (n_leaves + 1)] symmetric item / slot / M2P counts
    int *sym_leaf_of_box = nullptr;  // [n_boxes + 1]
    double2 *mpole = nullptr;   // [n_boxes*(p+1)]
    double2 *local = nullptr;   // [n_boxes*(p+1)]
    int *status = nullptr;      // device status word
    // CUDA graph of one evaluation (optional)
    bool use_graph = false;
    cudaGraphExec_t graph_exec = nullptr;
    const void *g_q = nullptr, *g_phi = nullptr;
    cudaStream_t g_stream = nullptr;
    cudaStream_t cap_stream = nullptr;  // private stream used only for capture
    int64_t graph_kernels = 0;
    // per-level offsets into lvl_boxes
    int64_t level_start[20] = {};
    DevArena mem;
    Timing timing;
    // recorded on the build stream after the last build work; evaluations on
    // any stream wait for it
    cudaEvent_t build_done = nullptr;
    // recorded after every evaluation on a stream other than mem.stream;
    // the tree's buffers are released only after it
    cudaEvent_t eval_done = nullptr;
    cudaStream_t last_eval_stream = nullptr;
    // fork / join of the far field's stream within one evaluation, and the
    // point where the multipoles are complete (M2P in the near field reads them)
    cudaEvent_t far_fork = nullptr, far_join = nullptr, far_mpole = nullptr;
};

// record timing event i of an evaluation (when timing is enabled)
void mark_event(Tree &t, int i, cudaStream_t s);

// kernel launches issued by this library (process-wide count)
void note_launch();

// Launch of a library kernel with programmatic stream serialisation (the
// kernel must begin with pdl_wait(), common.cuh); counted by note_launch.
template <class... P, class... A>
inline cudaError_t launch_k(void (*k)(P...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                            A &&...args) {
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    note_launch();
    return cudaLaunchKernelEx(&cfg, k, static_cast<A &&>(args)...);
}
int64_t launch_count();

// error reporting
void set_error(const std::string &msg);
std::string last_error_message();  // this thread's last message
fmm_status cuda_fail(cudaError_t e, const char *what);

// primitives (prims.cu)
// Exclusive scan of n uint32 values: out[i] = base + sum_{k<i} in[k];
// out[n] = base + total.  `base_dev` may be NULL (base 0).  in == out allowed.
cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n,
                               const uint32_t *base_dev, DevArena &scratch, cudaStream_t s);
// k <= 3 exclusive scans of arrays of the same length n in one pair of
// launches (out[i][n] receives the total of in[i]; in-place allowed).
cudaError_t exclusive_scan_u32_sets(int k, const uint32_t *const *in, uint32_t *const *out,
                                    int64_t n, DevArena &scratch, cudaStream_t s);
// Stable LSD radix sort of (keys, vals) over the 8-bit key digits selected by
// digit_mask (bit j = bits [8j, 8j+8)); digits left out must be constant.
// Buffers are ping-ponged; the result ends in *keys / *vals (pointers may swap).
cudaError_t radix_sort_pairs(uint64_t **keys, uint32_t **vals, uint64_t *keys_alt,
                             uint32_t *vals_alt, int64_t n, uint32_t digit_mask,
                             DevArena &scratch, cudaStream_t s);
// Two independent sorts of equal length in the same launches (keys[0..1] etc.).
cudaError_t radix_sort_pairs2(uint64_t **keys, uint32_t **vals, uint64_t **keys_alt,
                              uint32_t **vals_alt, int64_t n, uint32_t digit_mask,
                              DevArena &scratch, cudaStream_t s);
inline uint32_t digits_for_bits(int bits) { return bits <= 0 ? 0u : (1u << ((bits + 7) / 8)) - 1u; }

// phases
fmm_status build_topology(Tree &t, const double *src_xy, const double *tgt_xy,
                          const int64_t *inst_off, cudaStream_t s);
// `stage` holds >= 16 page-locked words (HostStage); `pre_sync`, when given,
// enqueues further work and reads (into stage + 16 ...) before the final
// synchronisation of the connectivity build, which serves them too.
fmm_status build_connectivity(Tree &t, cudaStream_t s, uint32_t *stage,
                              const std::function<fmm_status()> &pre_sync = nullptr);
fmm_status compute_geom(Tree &t, cudaStream_t s);
// Forest of n_inst instances (sources src_off[i] .. src_off[i+1]; with
// tgt_xy, evaluation points tgt_off[i] .. tgt_off[i+1], host offsets):
// instances with the same number of levels are built as one tree of R roots.
fmm_status build_forest(Tree &F, int n_inst, const int64_t *src_off, const double *src_xy,
                        const int64_t *tgt_off, const double *tgt_xy, const fmm_options &opt,
                        int (*levels_for)(int64_t, const fmm_options &), bool p2p_items_needed,
                        cudaStream_t s);
fmm_status run_evaluate(Tree &t, const double *q, double *phi, cudaStream_t s);
// a second stream of the calling host thread on the current device (null if
// it cannot be made), and the tree's fork / join events for it (made once)
cudaStream_t side_stream();
bool side_events(Tree &t);
// parts of the work at the evaluation points (launch_eval / launch_eval_sym)
enum { EVAL_P2P = 0, EVAL_M2P = 1, EVAL_COMBINE = 2 };
fmm_status launch_eval(Tree &t, double *phi, cudaStream_t s, int part);
// mixed precision (p2p_mixed.cu)
cudaError_t upload_df_tables();
cudaError_t upload_df_tables_m2l();
fmm_status prepare_mixed_points(Tree &t, cudaStream_t s);
fmm_status permute_q_mixed(Tree &t, const double *q, cudaStream_t s);
fmm_status launch_p2p_mixed(Tree &t, cudaStream_t s);
// the combination at separate evaluation points with a double-float L2P
// (mixed precision, p <= 32)
bool combine_mixed_ok(const Tree &t);
fmm_status launch_combine_mixed(Tree &t, double *phi, cudaStream_t s);
int m2l_mixed_max_p();
// M2L work items: counts (enqueued; the total lands in *total_host after the
// next synchronisation), then the fill
fmm_status m2l_items_count(Tree &t, cudaStream_t s, uint32_t *total_host);
fmm_status m2l_items_fill(Tree &t, uint32_t total, cudaStream_t s);
fmm_status launch_m2l_mixed(Tree &t, cudaStream_t s);
// mixed M2L set-up: zeroed locals and the df32 multipoles (read by M2L and M2P)
fmm_status m2l_prepare_mixed(Tree &t, cudaStream_t s);
// mixed-precision P2M (expand_mixed.cu)
int p2m_mixed_max_p();
fmm_status launch_p2m_mixed(Tree &t, cudaStream_t s);
cudaError_t upload_binom_df();
int translate_mixed_max_p();
// M2M into the parents of `level`; L2L from the parents of `level`
fmm_status launch_m2m_mixed(Tree &t, int level, cudaStream_t s);
fmm_status launch_l2l_mixed(Tree &t, int level, cudaStream_t s);
// leaf shortcut kernels (shortcut.cu)
cudaError_t upload_df_tables_sc();
fmm_status launch_p2l(Tree &t, cudaStream_t s);
fmm_status launch_m2p(Tree &t, cudaStream_t s);
// M2P items (leaf, first target, ~e0, ~e1); item order[k] writes partial[order[k] * 64 + i]
fmm_status launch_m2p_items(Tree &t, const int4 *items, const int *order, int n,
                            double2 *partial, cudaStream_t s);
// symmetric near field (p2p_sym.cu)
cudaError_t upload_df_tables_sym();
// symmetric items: counts (enqueued; three totals land in tot_host[0..2]
// after the next synchronisation), then the fill
fmm_status sym_items_count(Tree &t, cudaStream_t s, uint32_t *tot_host);
fmm_status sym_items_fill(Tree &t, const uint32_t *tot, cudaStream_t s);
fmm_status launch_eval_sym(Tree &t, double *phi, cudaStream_t s, int part);
// tensor-core M2L (m2l_tc.cu)
cudaError_t upload_df_tables_tc();
int m2l_tc_max_p();
// M2L runs on the tensor cores (k_m2l_tc, over runs of the weak list; the
// per-box M2L item table of the df32 sweeps is then not built)
inline bool m2l_on_tensor_cores(const Tree &t) {
    return t.precision == FMM_PREC_MIXED && t.m2l_slices > 0 && t.p <= m2l_tc_max_p();
}
int m2l_tc_max_slices();
fmm_status build_m2l_tc_operator(Tree &t, int slices, cudaStream_t s);
// the pair table of the weak list (after the geometry and weak_tgt exist)
fmm_status build_m2l_pairs(Tree &t, cudaStream_t s);
fmm_status launch_m2l_tc(Tree &t, cudaStream_t s);

}  // namespace gbfmm
