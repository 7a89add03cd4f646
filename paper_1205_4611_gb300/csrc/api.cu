// C ABI entry points (include/gbfmm.h): argument checking, tree ownership,
// orchestration of the topological and computational phases, host-buffer
// convenience path and topology export.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <tuple>
#include <unordered_map>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace gbfmm {

cudaError_t ensure_tables();

static thread_local std::string g_err;
static std::atomic<int64_t> g_launches{0};

void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
static void g_launches_add(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
static void g_launches_sub(int64_t n) { g_launches.fetch_sub(n, std::memory_order_relaxed); }
int64_t launch_count() { return g_launches.load(std::memory_order_relaxed); }

void set_error(const std::string &msg) { g_err = msg; }
std::string last_error_message() { return g_err; }

fmm_status cuda_fail(cudaError_t e, const char *what) {
    g_err = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return FMM_ERR_NOMEM;
    return FMM_ERR_CUDA;
}

// ------------------------------------------------------------ device block cache
//
// A build allocates about a hundred buffers, and a stream-ordered
// cudaMallocAsync / cudaFreeAsync pair costs ~13 us of host time on the
// Grace host; after each of the build's synchronisations the GPU waits for
// exactly that host work.  Freed blocks are therefore kept, by size class,
// for later work on the stream that freed them (stream order makes that
// reuse safe), or in an idle pool once a synchronisation of their stream has
// completed their last use (usable by any stream).  At most CACHE_LIMIT bytes
// are kept; the rest goes back to the driver.
namespace {
constexpr size_t CACHE_LIMIT = size_t(16) << 30;
// a sentinel "stream" for blocks no pending work uses (a real handle is a
// pointer, never all ones)
const cudaStream_t IDLE_STREAM = reinterpret_cast<cudaStream_t>(~uintptr_t(0));
struct Cached {
    void *p;
    uint64_t seq;  // release order
};
std::mutex g_cache_mu;
std::map<std::tuple<int, cudaStream_t, size_t>, std::vector<Cached>> g_cache;
std::unordered_map<void *, std::pair<int, size_t>> g_block;  // block -> (device, class bytes)
size_t g_cached = 0;
uint64_t g_seq = 0;
// bytes of the blocks handed out and not yet freed, and their high-water mark
size_t g_in_use = 0, g_in_use_peak = 0;
// host-side fault injection (fmm_debug_inject): the allocation after this
// many more successful ones fails (-1: off)
std::atomic<int64_t> g_fail_alloc_after{-1};
std::atomic<int> g_inject_status{0};

void note_in_use(size_t cb) {  // caller holds g_cache_mu
    g_in_use += cb;
    g_in_use_peak = std::max(g_in_use_peak, g_in_use);
}

// class sizes m 2^e with m in 4..8 (<= 25 % rounding), at least 256 B
size_t class_bytes(size_t bytes) {
    bytes = std::max<size_t>(bytes, 256);
    int e = 0;
    while ((bytes - 1) >> (e + 3)) ++e;
    const size_t m = (bytes + (size_t(1) << e) - 1) >> e;
    return m << e;
}
}  // namespace

cudaError_t dev_alloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const size_t cb = class_bytes(bytes);
    {
        // an injected failure (testing hook) behaves like an exhausted device
        int64_t left = g_fail_alloc_after.load();
        while (left >= 0 && !g_fail_alloc_after.compare_exchange_weak(left, left - 1)) {
        }
        if (left == 0) return cudaErrorMemoryAllocation;
    }
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        for (cudaStream_t k : {s, IDLE_STREAM}) {
            auto it = g_cache.find(std::make_tuple(dev, k, cb));
            if (it != g_cache.end() && !it->second.empty()) {
                *p = it->second.back().p;
                it->second.pop_back();
                g_cached -= cb;
                note_in_use(cb);
                return cudaSuccess;
            }
        }
    }
    e = cudaMallocAsync(p, cb, s);
    if (e != cudaSuccess) {
        // the cache may hold the memory: give it back and try once more
        cudaGetLastError();
        dev_cache_trim();
        e = cudaMallocAsync(p, cb, s);
        if (e != cudaSuccess) return e;
    }
    std::lock_guard<std::mutex> lk(g_cache_mu);
    g_block[*p] = std::make_pair(dev, cb);
    note_in_use(cb);
    return cudaSuccess;
}

void dev_free(void *p, cudaStream_t s) {
    if (!p) return;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        auto it = g_block.find(p);
        if (it != g_block.end()) {
            const size_t cb = it->second.second;
            g_in_use -= cb;
            if (g_cached + cb <= CACHE_LIMIT) {
                g_cache[std::make_tuple(it->second.first, s, cb)].push_back(Cached{p, ++g_seq});
                g_cached += cb;
                return;
            }
            g_block.erase(it);
        }
    }
    cudaFreeAsync(p, s);
}

uint64_t dev_cache_mark() {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    return g_seq;
}

void dev_cache_stream_idle(cudaStream_t s, uint64_t mark) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    std::vector<std::pair<std::tuple<int, cudaStream_t, size_t>, Cached>> moved;
    for (auto &kv : g_cache) {
        if (std::get<1>(kv.first) != s) continue;
        auto &v = kv.second;
        size_t w = 0;
        for (const Cached &c : v) {
            if (c.seq <= mark)
                moved.emplace_back(kv.first, c);
            else
                v[w++] = c;
        }
        v.resize(w);
    }
    for (auto &m : moved)
        g_cache[std::make_tuple(std::get<0>(m.first), IDLE_STREAM, std::get<2>(m.first))]
            .push_back(m.second);
}

void dev_cache_trim() {
    // every cached block is idle once the device has drained
    cudaDeviceSynchronize();
    std::vector<void *> all;
    {
        std::lock_guard<std::mutex> lk(g_cache_mu);
        for (auto &kv : g_cache)
            for (const Cached &c : kv.second) {
                g_block.erase(c.p);
                all.push_back(c.p);
            }
        g_cache.clear();
        g_cached = 0;
    }
    for (void *p : all) cudaFree(p);
}

cudaError_t DevArena::alloc(void **p, size_t bytes) {
    cudaError_t e = dev_alloc(p, bytes, stream);
    if (e == cudaSuccess) ptrs.push_back(*p);
    return e;
}

void DevArena::release() {
    for (void *p : ptrs) dev_free(p, stream);
    ptrs.clear();
}

// Pool of page-locked stage blocks (never returned to the system: a block is
// allocated once and reused by later builds, on any thread).
static std::mutex g_stage_mu;
static std::vector<uint32_t *> g_stage_pool;

HostStage::HostStage() {
    {
        std::lock_guard<std::mutex> lk(g_stage_mu);
        if (!g_stage_pool.empty()) {
            w = g_stage_pool.back();
            g_stage_pool.pop_back();
        }
    }
    if (!w && cudaMallocHost(reinterpret_cast<void **>(&w), HOST_STAGE_WORDS * sizeof(uint32_t)) !=
                  cudaSuccess)
        w = nullptr;
}

HostStage::~HostStage() {
    if (!w) return;
    std::lock_guard<std::mutex> lk(g_stage_mu);
    g_stage_pool.push_back(w);
}

// Counts, one synchronisation, then the fill (used where no earlier
// synchronisation can carry the counts).
static fmm_status m2l_items_sync(Tree &t, cudaStream_t s) {
    HostStage hs;
    if (!hs.w) return set_error("page-locked stage allocation failed"), FMM_ERR_NOMEM;
    if (m2l_on_tensor_cores(t)) return m2l_items_fill(t, 0, s);  // no item table
    fmm_status st = m2l_items_count(t, s, hs.w);
    cudaError_t e;
    if (st == FMM_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = cuda_fail(e, "m2l items");
    if (st == FMM_OK) st = m2l_items_fill(t, hs.w[0], s);
    return st;
}

static fmm_status sym_items_sync(Tree &t, cudaStream_t s) {
    HostStage hs;
    if (!hs.w) return set_error("page-locked stage allocation failed"), FMM_ERR_NOMEM;
    fmm_status st = sym_items_count(t, s, hs.w);
    cudaError_t e;
    if (st == FMM_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = cuda_fail(e, "sym items");
    if (st == FMM_OK) st = sym_items_fill(t, hs.w, s);
    return st;
}

static int levels_for(int64_t n, const fmm_options &o) {
    int L = 0;
    if (o.level_rule == FMM_LEVELS_EQ) {
        double v = 0.5 * std::log2(0.625 * (double)n / (double)o.leaf_size);
        L = (int)std::ceil(v);
        if (L < 0) L = 0;
    } else {
        int64_t boxes = 1;
        while ((n + boxes - 1) / boxes > o.leaf_size) {
            ++L;
            boxes *= 4;
        }
    }
    return L + o.level_shift;
}

static fmm_status check_options(const fmm_options *opt) {
    if (!opt) return set_error("options pointer is NULL"), FMM_ERR_ARG;
    if (opt->p < 1 || opt->p > MAXP) return set_error("p must be in [1, 64]"), FMM_ERR_ARG;
    if (!(opt->theta > 0.0 && opt->theta < 1.0))
        return set_error("theta must be in (0, 1)"), FMM_ERR_ARG;
    if (opt->leaf_size < 1) return set_error("leaf_size must be >= 1"), FMM_ERR_ARG;
    if (opt->level_rule != FMM_LEVELS_CAP && opt->level_rule != FMM_LEVELS_EQ)
        return set_error("unknown level_rule"), FMM_ERR_ARG;
    if (opt->level_shift < 0 || opt->level_shift > 8)
        return set_error("level_shift must be in [0, 8]"), FMM_ERR_ARG;
    if (opt->precision != FMM_PREC_FP64 && opt->precision != FMM_PREC_MIXED)
        return set_error("unknown precision"), FMM_ERR_ARG;
    if (opt->m2l_slices < -1 || opt->m2l_slices > m2l_tc_max_slices())
        return set_error("m2l_slices must be in [-1, 5]"), FMM_ERR_ARG;
    if (opt->p2l_m2p != 0 && opt->p2l_m2p != 1) return set_error("p2l_m2p must be 0 or 1"), FMM_ERR_ARG;
    if (opt->p2p_mode != 0 && opt->p2p_mode != 1) return set_error("p2p_mode must be 0 or 1"), FMM_ERR_ARG;
    if (opt->box_fit != 0 && opt->box_fit != 1) return set_error("box_fit must be 0 or 1"), FMM_ERR_ARG;
    if (opt->kernel != FMM_KERNEL_LOG && opt->kernel != FMM_KERNEL_HARMONIC)
        return set_error("unknown kernel"), FMM_ERR_ARG;
    if (opt->p2p_item_sources != 0 &&
        (opt->p2p_item_sources < 64 || opt->p2p_item_sources > 65536))
        return set_error("p2p_item_sources must be 0 or in [64, 65536]"), FMM_ERR_ARG;
    return FMM_OK;
}

// The symmetric near field (p2p_sym.cu) serves self-evaluation in both
// precisions when every leaf holds at most 64 points: with the median splits a leaf of
// an instance of n points at level L holds at most ceil(n / 4^L).
static bool sym_eligible(const fmm_options &o, bool separate, const int64_t *n, int n_inst,
                         const int *L) {
    if (o.p2p_mode != 0 || separate) return false;
    for (int i = 0; i < n_inst; ++i) {
        const int64_t cells = int64_t(1) << (2 * L[i]);
        if ((n[i] + cells - 1) / cells > 64) return false;
    }
    return true;
}

}  // namespace gbfmm

using namespace gbfmm;

struct fmm_tree {
    Tree t;
};

extern "C" {

void fmm_default_options(fmm_options *opt) {
    if (!opt) return;
    std::memset(opt, 0, sizeof(*opt));
    opt->p = 20;
    opt->theta = 0.5;
    opt->leaf_size = 64;
    opt->level_rule = FMM_LEVELS_CAP;
    opt->level_shift = 0;
    opt->precision = FMM_PREC_FP64;
}

const char *fmm_last_error(void) { return g_err.c_str(); }

int64_t fmm_launch_count(void) { return launch_count(); }

fmm_status fmm_memory_info(int64_t *in_use, int64_t *peak, int64_t *cached, int reset_peak) {
    std::lock_guard<std::mutex> lk(g_cache_mu);
    if (in_use) *in_use = (int64_t)g_in_use;
    if (peak) *peak = (int64_t)g_in_use_peak;
    if (cached) *cached = (int64_t)g_cached;
    if (reset_peak) g_in_use_peak = g_in_use;
    return FMM_OK;
}

fmm_status fmm_debug_inject(int what, int64_t arg) {
    g_err.clear();
    if (what == FMM_INJECT_ALLOC_FAILURE) {
        g_fail_alloc_after = arg < 0 ? -1 : arg;
        return FMM_OK;
    }
    if (what == FMM_INJECT_STATUS) {
        g_inject_status = (int)arg;
        return FMM_OK;
    }
    return set_error("unknown injection"), FMM_ERR_ARG;
}

fmm_status fmm_build_tree(const double *src_xy_dev, int64_t n_src, const double *tgt_xy_dev,
                          int64_t n_tgt, const fmm_options *opt, void *stream, fmm_tree **out) {
    g_err.clear();
    if (!out) return set_error("out is NULL"), FMM_ERR_ARG;
    *out = nullptr;
    fmm_status st = check_options(opt);
    if (st != FMM_OK) return st;
    if (!src_xy_dev) return set_error("src_xy_dev is NULL"), FMM_ERR_ARG;
    if (n_src < 1 || n_src > (int64_t)INT32_MAX / 2)
        return set_error("n_src must be in [1, 2^30]"), FMM_ERR_ARG;
    if (tgt_xy_dev && (n_tgt < 1 || n_tgt > (int64_t)INT32_MAX / 2))
        return set_error("n_tgt must be in [1, 2^30]"), FMM_ERR_ARG;
    int L = levels_for(n_src, *opt);
    if (L > 12) return set_error("tree deeper than 12 levels"), FMM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = ensure_tables();
    if (e != cudaSuccess) return cuda_fail(e, "tables");
    fmm_tree *h = new (std::nothrow) fmm_tree;
    if (!h) return set_error("host allocation failed"), FMM_ERR_NOMEM;
    Tree &t = h->t;
    t.p = opt->p;
    t.theta = opt->theta;
    t.leaf = opt->leaf_size;
    t.precision = opt->precision;
    t.m2l_slices = opt->m2l_slices == 0 ? m2l_tc_max_slices() : opt->m2l_slices;  // 0: 5 slices
    t.p2l_m2p = opt->p2l_m2p;
    t.box_fit = opt->box_fit;
    t.kernel = opt->kernel;
    t.p2p_cap = opt->p2p_item_sources ? opt->p2p_item_sources : 2048;
    t.L = L;
    t.n_src = n_src;
    t.separate = tgt_xy_dev != nullptr;
    t.n_tgt = t.separate ? n_tgt : n_src;
    t.mem.stream = s;
    HostStage hs;
    if (!hs.w) {
        fmm_tree_free(h);
        return set_error("page-locked stage allocation failed"), FMM_ERR_NOMEM;
    }
    // device-side spans of the tree and connectivity builds
    cudaEvent_t bev[3] = {};
    for (auto &ev : bev)
        if ((e = cudaEventCreate(&ev)) != cudaSuccess) st = cuda_fail(e, "event");
    if (st == FMM_OK) cudaEventRecord(bev[0], s);
    if (st == FMM_OK) st = build_topology(t, src_xy_dev, tgt_xy_dev, nullptr, s);
    if (st == FMM_OK) cudaEventRecord(bev[1], s);
    // the M2L and symmetric item counts ride on the connectivity build's
    // final synchronisation (stage words 16 and 20..22)
    const bool want_m2l = t.precision == FMM_PREC_MIXED && t.p <= m2l_mixed_max_p();
    const bool want_sym = sym_eligible(*opt, t.separate, &n_src, 1, &L);
    t.p2p_items_needed = !want_sym;  // the symmetric near field has items of its own
    auto pre_sync = [&]() -> fmm_status {
        cudaEventRecord(bev[2], s);
        fmm_status r = FMM_OK;
        if (want_m2l && !m2l_on_tensor_cores(t)) r = m2l_items_count(t, s, hs.w + 16);
        if (r == FMM_OK && want_sym) r = sym_items_count(t, s, hs.w + 20);
        return r;
    };
    if (st == FMM_OK) st = build_connectivity(t, s, hs.w, pre_sync);
    if (st == FMM_OK) {
        cudaEventElapsedTime(&t.timing.ms[0], bev[0], bev[1]);
        cudaEventElapsedTime(&t.timing.ms[1], bev[1], bev[2]);
    }
    for (auto &ev : bev)
        if (ev) cudaEventDestroy(ev);
    if (st == FMM_OK && want_m2l)
        st = m2l_items_fill(t, m2l_on_tensor_cores(t) ? 0u : hs.w[16], s);
    // the mixed path's point offsets and the tensor M2L's pair table need
    // nothing that the remaining item tables produce: they run on the second
    // stream meanwhile, joined before the end of the build
    cudaStream_t g = s;
    if (st == FMM_OK) {
        cudaStream_t side = side_stream();
        if (side && side_events(t) && cudaEventRecord(t.far_fork, s) == cudaSuccess &&
            cudaStreamWaitEvent(side, t.far_fork, 0) == cudaSuccess)
            g = side;
    }
    if (st == FMM_OK && t.precision == FMM_PREC_MIXED) st = prepare_mixed_points(t, g);
    if (st == FMM_OK && t.precision == FMM_PREC_MIXED && t.m2l_slices > 0 &&
        t.p <= m2l_tc_max_p())
        st = build_m2l_tc_operator(t, t.m2l_slices, g);
    if (st == FMM_OK && m2l_on_tensor_cores(t)) st = build_m2l_pairs(t, g);
    const cudaError_t ej = g != s ? cudaEventRecord(t.far_join, g) : cudaSuccess;
    if (st == FMM_OK && want_sym) st = sym_items_fill(t, hs.w + 20, s);
    if (g != s) {  // joined on every path
        if (ej == cudaSuccess) {
            cudaStreamWaitEvent(s, t.far_join, 0);
        } else {
            cudaStreamSynchronize(g);
            if (st == FMM_OK) st = cuda_fail(ej, "build join");
        }
    }
    if (st == FMM_OK) {
        const size_t nc = (size_t)t.n_boxes * (t.p + 1);
        if ((e = arena_alloc(t.mem, &t.qs, t.n_src)) != cudaSuccess ||
            (e = arena_alloc(t.mem, &t.mpole, nc)) != cudaSuccess ||
            (e = arena_alloc(t.mem, &t.local, nc)) != cudaSuccess)
            st = cuda_fail(e, "expansion buffers");
    }
    // the work after the connectivity build's synchronisation (work-item
    // tables) stays stream-ordered: evaluations wait for this event
    if (st == FMM_OK &&
        ((e = cudaEventCreateWithFlags(&t.build_done, cudaEventDisableTiming)) != cudaSuccess ||
         (e = cudaEventRecord(t.build_done, s)) != cudaSuccess || (e = cudaGetLastError()) != cudaSuccess))
        st = cuda_fail(e, "build");
    if (st != FMM_OK) {
        fmm_tree_free(h);
        return st;
    }
    *out = h;
    return FMM_OK;
}

static fmm_status run_evaluate_or_replay(Tree &t, const double *q_dev, double *phi_dev,
                                         cudaStream_t s);

fmm_status fmm_evaluate(fmm_tree *tree, const double *q_dev, double *phi_dev, void *stream) {
    g_err.clear();
    if (!tree || !q_dev || !phi_dev) return set_error("NULL argument"), FMM_ERR_ARG;
    Tree &t = tree->t;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (t.build_done && (e = cudaStreamWaitEvent(s, t.build_done, 0)) != cudaSuccess)
        return cuda_fail(e, "wait for the build");
    // evaluations of one tree share its expansion buffers: one on another
    // stream than the previous one waits for it
    if (t.eval_done && s != t.last_eval_stream &&
        (e = cudaStreamWaitEvent(s, t.eval_done, 0)) != cudaSuccess)
        return cuda_fail(e, "wait for the previous evaluation");
    if (!t.eval_done &&
        (e = cudaEventCreateWithFlags(&t.eval_done, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "event");
    fmm_status st = run_evaluate_or_replay(t, q_dev, phi_dev, s);
    if (st == FMM_OK) {
        if ((e = cudaEventRecord(t.eval_done, s)) != cudaSuccess) return cuda_fail(e, "event");
        t.last_eval_stream = s;
    }
    return st;
}

static fmm_status run_evaluate_or_replay(Tree &t, const double *q_dev, double *phi_dev,
                                         cudaStream_t s) {
    cudaError_t e;
    if (!t.use_graph) return run_evaluate(t, q_dev, phi_dev, s);
    if (!t.graph_exec || t.g_q != q_dev || t.g_phi != phi_dev || t.g_stream != s) {
        if (t.graph_exec) {
            cudaGraphExecDestroy(t.graph_exec);
            t.graph_exec = nullptr;
        }
        // capture on a private stream (the legacy default stream cannot be
        // captured); the graph is then launched on the caller's stream
        if (!t.cap_stream &&
            (e = cudaStreamCreateWithFlags(&t.cap_stream, cudaStreamNonBlocking)) != cudaSuccess)
            return cuda_fail(e, "capture stream");
        const bool timing = t.timing.enabled;
        t.timing.enabled = false;
        const int64_t before = launch_count();
        if ((e = cudaStreamBeginCapture(t.cap_stream, cudaStreamCaptureModeThreadLocal)) !=
            cudaSuccess)
            return cuda_fail(e, "graph capture");
        fmm_status st = run_evaluate(t, q_dev, phi_dev, t.cap_stream);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(t.cap_stream, &g);
        t.timing.enabled = timing;
        if (st != FMM_OK) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) return cuda_fail(e, "graph capture");
        e = cudaGraphInstantiate(&t.graph_exec, g, 0);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(e, "graph instantiate");
        t.graph_kernels = launch_count() - before;
        g_launches_sub(t.graph_kernels);  // captured, not launched
        t.g_q = q_dev;
        t.g_phi = phi_dev;
        t.g_stream = s;
    }
    if ((e = cudaGraphLaunch(t.graph_exec, s)) != cudaSuccess) return cuda_fail(e, "graph launch");
    g_launches_add(t.graph_kernels);
    return FMM_OK;
}

fmm_status fmm_tree_sync(fmm_tree *tree, void *stream) {
    g_err.clear();
    if (!tree) return set_error("NULL tree"), FMM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int st = 0;
    cudaError_t e = cudaMemcpyAsync(&st, tree->t.status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(e, "sync");
    Tree &t = tree->t;
    if (t.timing.enabled) {
        // (slot, first event, last event)
        // (slot, first event, last event)
        static const int span[8][3] = {{7, 0, 1}, {2, 1, 2}, {3, 2, 3}, {4, 3, 4},
                                       {5, 4, 5}, {8, 5, 6}, {9, 9, 7}, {10, 10, 11}};
        for (int i = 0; i < 8; ++i)
            cudaEventElapsedTime(&t.timing.ms[span[i][0]], t.timing.ev[span[i][1]],
                                 t.timing.ev[span[i][2]]);
        float comb = 0.f;
        cudaEventElapsedTime(&comb, t.timing.ev[12], t.timing.ev[8]);
        t.timing.ms[10] += comb;
        t.timing.ms[6] = t.timing.ms[9] + t.timing.ms[10];
    }
    st |= g_inject_status.exchange(0);  // testing hook (fmm_debug_inject), 0 otherwise
    if (st & ST_TIMEOUT) return set_error("device wait timed out"), FMM_ERR_TIMEOUT;
    if (st & ST_NONFINITE) return set_error("non-finite input"), FMM_ERR_NONFINITE;
    if (st) return set_error("device status " + std::to_string(st)), FMM_ERR_CUDA;
    return FMM_OK;
}

fmm_status fmm_solve_host(const double *src_xy_host, int64_t n_src, const double *tgt_xy_host,
                          int64_t n_tgt, const double *q_host, double *phi_host,
                          const fmm_options *opt, void *stream) {
    g_err.clear();
    if (!src_xy_host || !q_host || !phi_host) return set_error("NULL argument"), FMM_ERR_ARG;
    if (n_src < 1) return set_error("n_src must be >= 1"), FMM_ERR_ARG;
    if (tgt_xy_host && n_tgt < 1) return set_error("n_tgt must be >= 1"), FMM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int64_t m = tgt_xy_host ? n_tgt : n_src;
    DevArena io;
    io.stream = s;
    double *src = nullptr, *tgt = nullptr, *q = nullptr, *phi = nullptr;
    cudaError_t e;
    fmm_status st = FMM_OK;
    if ((e = io.alloc((void **)&src, 16 * (size_t)n_src)) != cudaSuccess ||
        (e = io.alloc((void **)&q, 16 * (size_t)n_src)) != cudaSuccess ||
        (e = io.alloc((void **)&phi, 16 * (size_t)m)) != cudaSuccess ||
        (tgt_xy_host && (e = io.alloc((void **)&tgt, 16 * (size_t)n_tgt)) != cudaSuccess)) {
        io.release();
        return cuda_fail(e, "solve buffers");
    }
    // the strengths are needed only by the evaluation: their copy runs on a
    // side stream while the tree is built
    // (one stream and two events per thread and device)
    static thread_local cudaStream_t side_of[64] = {};
    static thread_local cudaEvent_t side_ev_of[64][2] = {};
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess || dev >= 64) {
        io.release();
        return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidDevice, "device");
    }
    cudaStream_t &side = side_of[dev];
    cudaEvent_t *side_ev = side_ev_of[dev];
    if (!side && (e = cudaStreamCreateWithFlags(&side, cudaStreamNonBlocking)) != cudaSuccess) {
        side = nullptr;
        io.release();
        return cuda_fail(e, "copy stream");
    }
    for (int k = 0; k < 2; ++k)
        if (!side_ev[k] &&
            (e = cudaEventCreateWithFlags(&side_ev[k], cudaEventDisableTiming)) != cudaSuccess) {
            side_ev[k] = nullptr;
            io.release();
            return cuda_fail(e, "copy event");
        }
    e = cudaMemcpyAsync(src, src_xy_host, 16 * (size_t)n_src, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess && tgt)
        e = cudaMemcpyAsync(tgt, tgt_xy_host, 16 * (size_t)n_tgt, cudaMemcpyHostToDevice, s);
    // the side stream starts after the buffers' earlier users on s
    if (e == cudaSuccess) e = cudaEventRecord(side_ev[0], s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(side, side_ev[0], 0);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(q, q_host, 16 * (size_t)n_src, cudaMemcpyHostToDevice, side);
    if (e == cudaSuccess) e = cudaEventRecord(side_ev[1], side);
    if (e != cudaSuccess) {
        cudaStreamSynchronize(side);
        io.release();
        return cuda_fail(e, "copy in");
    }
    fmm_tree *tree = nullptr;
    st = fmm_build_tree(src, n_src, tgt, n_tgt, opt, stream, &tree);
    if (st == FMM_OK && (e = cudaStreamWaitEvent(s, side_ev[1], 0)) != cudaSuccess)
        st = cuda_fail(e, "wait for the strengths");
    if (st == FMM_OK) st = fmm_evaluate(tree, q, phi, stream);
    if (st == FMM_OK) {
        e = cudaMemcpyAsync(phi_host, phi, 16 * (size_t)m, cudaMemcpyDeviceToHost, s);
        if (e != cudaSuccess) st = cuda_fail(e, "copy out");
    }
    if (st == FMM_OK) st = fmm_tree_sync(tree, stream);
    fmm_tree_free(tree);
    // q's copy is complete before its buffer returns to the cache under s
    cudaStreamWaitEvent(s, side_ev[1], 0);
    io.release();
    if (st == FMM_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = cuda_fail(e, "solve");
    return st;
}

fmm_status fmm_tree_info(const fmm_tree *tree, int *levels, int64_t *n_boxes, int64_t *n_weak,
                         int64_t *n_strong) {
    g_err.clear();
    if (!tree) return set_error("NULL tree"), FMM_ERR_ARG;
    const Tree &t = tree->t;
    if (levels) *levels = t.L;
    if (n_boxes) *n_boxes = t.n_boxes;
    if (n_weak) *n_weak = t.n_weak;
    if (n_strong) *n_strong = t.n_strong;
    return FMM_OK;
}

fmm_status fmm_tree_export(const fmm_tree *tree, uint32_t *perm, uint32_t *tperm, double *box_rect,
                           int64_t *box_src, int64_t *box_tgt, int64_t *weak_off, int32_t *weak,
                           int64_t *strong_off, int32_t *strong) {
    g_err.clear();
    if (!tree) return set_error("NULL tree"), FMM_ERR_ARG;
    const Tree &t = tree->t;
    cudaStream_t s = t.mem.stream;
    cudaError_t e = cudaStreamSynchronize(s);
    const int64_t nb = t.n_boxes;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        if (e == cudaSuccess && dst && bytes) e = cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost);
    };
    cp(perm, t.perm, 4 * (size_t)t.n_src);
    cp(tperm, t.tperm, 4 * (size_t)t.n_tgt);
    cp(box_rect, t.rect, 32 * (size_t)nb);
    std::vector<int2> tmp2;
    auto pairs = [&](int64_t *dst, const int2 *src) {
        if (!dst || e != cudaSuccess) return;
        tmp2.resize(nb);
        cp(tmp2.data(), src, 8 * (size_t)nb);
        for (int64_t i = 0; i < nb; ++i) {
            dst[2 * i] = tmp2[i].x;
            dst[2 * i + 1] = tmp2[i].y;
        }
    };
    pairs(box_src, t.box_src);
    pairs(box_tgt, t.box_tgt);
    std::vector<int> tmp1;
    auto offs = [&](int64_t *dst, const int *src) {
        if (!dst || e != cudaSuccess) return;
        tmp1.resize(nb + 1);
        cp(tmp1.data(), src, 4 * (size_t)(nb + 1));
        for (int64_t i = 0; i <= nb; ++i) dst[i] = tmp1[i];
    };
    offs(weak_off, t.weak_off);
    offs(strong_off, t.strong_off);
    cp(weak, t.weak, 4 * (size_t)t.n_weak);
    cp(strong, t.strong, 4 * (size_t)t.n_strong);
    if (e != cudaSuccess) return cuda_fail(e, "export");
    return FMM_OK;
}

fmm_status fmm_tree_export_geometry(const fmm_tree *tree, double *box_rect) {
    g_err.clear();
    if (!tree || !box_rect) return set_error("NULL argument"), FMM_ERR_ARG;
    const Tree &t = tree->t;
    cudaError_t e = cudaStreamSynchronize(t.mem.stream);
    if (e == cudaSuccess)
        e = cudaMemcpy(box_rect, t.rect_geo, 32 * (size_t)t.n_boxes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "export geometry");
    return FMM_OK;
}

fmm_status fmm_tree_shortcut_info(const fmm_tree *tree, int64_t *n_near, int64_t *n_p2l,
                                  int64_t *n_m2p) {
    g_err.clear();
    if (!tree) return set_error("NULL tree"), FMM_ERR_ARG;
    const Tree &t = tree->t;
    if (!t.p2l_m2p) return set_error("tree built without the leaf shortcut"), FMM_ERR_ARG;
    if (n_near) *n_near = t.n_near;
    if (n_p2l) *n_p2l = t.n_p2l;
    if (n_m2p) *n_m2p = t.n_m2p;
    return FMM_OK;
}

fmm_status fmm_tree_export_shortcut(const fmm_tree *tree, int64_t *near_off, int32_t *near,
                                    int64_t *p2l_off, int32_t *p2l, int64_t *m2p_off,
                                    int32_t *m2p) {
    g_err.clear();
    if (!tree) return set_error("NULL tree"), FMM_ERR_ARG;
    const Tree &t = tree->t;
    if (!t.p2l_m2p) return set_error("tree built without the leaf shortcut"), FMM_ERR_ARG;
    cudaError_t e = cudaStreamSynchronize(t.mem.stream);
    const int64_t nb = t.n_boxes;
    std::vector<int> tmp;
    auto offs = [&](int64_t *dst, const int *src) {
        if (!dst || e != cudaSuccess) return;
        tmp.resize(nb + 1);
        e = cudaMemcpy(tmp.data(), src, 4 * (size_t)(nb + 1), cudaMemcpyDeviceToHost);
        for (int64_t i = 0; i <= nb && e == cudaSuccess; ++i) dst[i] = tmp[i];
    };
    auto ents = [&](int32_t *dst, const int *src, int64_t n) {
        if (dst && n && e == cudaSuccess)
            e = cudaMemcpy(dst, src, 4 * (size_t)n, cudaMemcpyDeviceToHost);
    };
    offs(near_off, t.near_off);
    offs(p2l_off, t.p2l_off);
    offs(m2p_off, t.m2p_off);
    ents(near, t.near, t.n_near);
    ents(p2l, t.p2l, t.n_p2l);
    ents(m2p, t.m2p, t.n_m2p);
    if (e != cudaSuccess) return cuda_fail(e, "export shortcut");
    return FMM_OK;
}

fmm_status fmm_set_timing(fmm_tree *tree, int enable) {
    if (!tree) return set_error("NULL tree"), FMM_ERR_ARG;
    Tree &t = tree->t;
    if (enable && !t.timing.ev[0]) {
        for (int i = 0; i < N_EVAL_EVENTS; ++i) {
            cudaError_t e = cudaEventCreate(&t.timing.ev[i]);
            if (e != cudaSuccess) return cuda_fail(e, "event");
        }
    }
    t.timing.enabled = enable != 0;
    return FMM_OK;
}

fmm_status fmm_get_timings(const fmm_tree *tree, float *ms, int n) {
    if (!tree || (!ms && n > 0)) return set_error("NULL argument"), FMM_ERR_ARG;
    for (int i = 0; i < std::min(n, N_TIMINGS); ++i) ms[i] = tree->t.timing.ms[i];
    return FMM_OK;
}

void fmm_tree_free(fmm_tree *tree) {
    if (!tree) return;
    Tree *t = &tree->t;
    if (t->graph_exec) cudaGraphExecDestroy(t->graph_exec);
    if (t->cap_stream) cudaStreamDestroy(t->cap_stream);
    for (int i = 0; i < N_EVAL_EVENTS; ++i)
        if (t->timing.ev[i]) cudaEventDestroy(t->timing.ev[i]);
    if (t->build_done) cudaEventDestroy(t->build_done);
    if (t->far_fork) cudaEventDestroy(t->far_fork);
    if (t->far_join) cudaEventDestroy(t->far_join);
    if (t->far_mpole) cudaEventDestroy(t->far_mpole);
    if (t->eval_done) {
        // an evaluation on another stream may still read the tree's buffers
        cudaStreamWaitEvent(t->mem.stream, t->eval_done, 0);
        cudaEventDestroy(t->eval_done);
    }
    t->mem.release();
    const uint64_t mark = dev_cache_mark();
    if (cudaStreamSynchronize(t->mem.stream) == cudaSuccess)
        dev_cache_stream_idle(t->mem.stream, mark);
    delete tree;
}

fmm_status fmm_build_batched(int n_inst, const int64_t *src_off_host, const double *src_xy_dev,
                             const int64_t *tgt_off_host, const double *tgt_xy_dev,
                             const fmm_options *opt, void *stream, fmm_tree **out) {
    g_err.clear();
    if (!out) return set_error("out is NULL"), FMM_ERR_ARG;
    *out = nullptr;
    fmm_status st = check_options(opt);
    if (st != FMM_OK) return st;
    if (n_inst < 1 || !src_off_host || !src_xy_dev)
        return set_error("need n_inst >= 1, offsets and points"), FMM_ERR_ARG;
    if (src_off_host[0] != 0) return set_error("src_off[0] must be 0"), FMM_ERR_ARG;
    for (int i = 0; i < n_inst; ++i)
        if (src_off_host[i + 1] <= src_off_host[i])
            return set_error("every instance needs at least one source"), FMM_ERR_ARG;
    if (src_off_host[n_inst] > (int64_t)INT32_MAX / 2)
        return set_error("too many sources"), FMM_ERR_ARG;
    const bool separate = tgt_xy_dev != nullptr;
    if (separate) {
        if (!tgt_off_host) return set_error("evaluation points need tgt_off"), FMM_ERR_ARG;
        if (tgt_off_host[0] != 0) return set_error("tgt_off[0] must be 0"), FMM_ERR_ARG;
        for (int i = 0; i < n_inst; ++i)
            if (tgt_off_host[i + 1] < tgt_off_host[i])
                return set_error("tgt_off must be non-decreasing"), FMM_ERR_ARG;
        if (tgt_off_host[n_inst] < 1 || tgt_off_host[n_inst] > (int64_t)INT32_MAX / 2)
            return set_error("need 1 .. 2^30 evaluation points"), FMM_ERR_ARG;
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e = ensure_tables();
    if (e != cudaSuccess) return cuda_fail(e, "tables");
    fmm_tree *h = new (std::nothrow) fmm_tree;
    if (!h) return set_error("host allocation failed"), FMM_ERR_NOMEM;
    Tree &t = h->t;
    t.p = opt->p;
    t.theta = opt->theta;
    t.leaf = opt->leaf_size;
    t.precision = opt->precision;
    t.m2l_slices = opt->m2l_slices == 0 ? m2l_tc_max_slices() : opt->m2l_slices;  // 0: 5 slices
    t.p2l_m2p = opt->p2l_m2p;
    t.box_fit = opt->box_fit;
    t.kernel = opt->kernel;
    t.p2p_cap = opt->p2p_item_sources ? opt->p2p_item_sources : 2048;
    t.mem.stream = s;
    bool want_sym;
    {
        std::vector<int64_t> sizes(n_inst);
        std::vector<int> levels(n_inst);
        for (int i = 0; i < n_inst; ++i) {
            sizes[i] = src_off_host[i + 1] - src_off_host[i];
            levels[i] = levels_for(sizes[i], *opt);
        }
        want_sym = sym_eligible(*opt, separate, sizes.data(), n_inst, levels.data());
    }
    // the per-point P2P items are only built for forests without the
    // symmetric near field (it has items of its own)
    st = build_forest(t, n_inst, src_off_host, src_xy_dev, separate ? tgt_off_host : nullptr,
                      tgt_xy_dev, *opt, levels_for, !want_sym, s);
    if (st == FMM_OK && t.precision == FMM_PREC_MIXED) st = prepare_mixed_points(t, s);
    if (st == FMM_OK && t.precision == FMM_PREC_MIXED && t.p <= m2l_mixed_max_p())
        st = m2l_items_sync(t, s);
    if (st == FMM_OK && want_sym) st = sym_items_sync(t, s);
    if (st == FMM_OK && t.precision == FMM_PREC_MIXED && t.m2l_slices > 0 &&
        t.p <= m2l_tc_max_p())
        st = build_m2l_tc_operator(t, t.m2l_slices, s);
    if (st == FMM_OK && m2l_on_tensor_cores(t)) st = build_m2l_pairs(t, s);
    if (st == FMM_OK) {
        const size_t nc = (size_t)t.n_boxes * (t.p + 1);
        if ((e = arena_alloc(t.mem, &t.qs, t.n_src)) != cudaSuccess ||
            (e = arena_alloc(t.mem, &t.mpole, nc)) != cudaSuccess ||
            (e = arena_alloc(t.mem, &t.local, nc)) != cudaSuccess)
            st = cuda_fail(e, "expansion buffers");
    }
    if (st == FMM_OK && (e = cudaStreamSynchronize(s)) != cudaSuccess) st = cuda_fail(e, "build");
    if (st != FMM_OK) {
        fmm_tree_free(h);
        return st;
    }
    *out = h;
    return FMM_OK;
}

fmm_status fmm_evaluate_batched(int n_inst, const int64_t *src_off_host,
                                const int64_t *tgt_off_host, const double *src_xy_dev,
                                const double *tgt_xy_dev, const double *q_dev, double *phi_dev,
                                const fmm_options *opt, void *stream) {
    fmm_tree *tree = nullptr;
    fmm_status st = fmm_build_batched(n_inst, src_off_host, src_xy_dev, tgt_off_host, tgt_xy_dev,
                                      opt, stream, &tree);
    if (st != FMM_OK) return st;
    st = fmm_evaluate(tree, q_dev, phi_dev, stream);
    if (st == FMM_OK) st = fmm_tree_sync(tree, stream);
    fmm_tree_free(tree);
    return st;
}

// Times every (leaf size, near-field item size) combination: one untimed
// pass, then the fastest of `repeats` timed passes of a build followed by
// `evaluations` evaluations (host clock around the synchronised work).
static fmm_status autotune(const double *src_xy_dev, int64_t n_src, const double *tgt_xy_dev,
                           int64_t n_tgt, int n_inst, const int64_t *src_off_host,
                           const double *q_dev, const fmm_options *opt, const int *leaf_cand,
                           int n_leaf, const int *item_cand, int n_item, int repeats,
                           int evaluations, void *stream, int *best_leaf, int *best_item,
                           float *ms) {
    g_err.clear();
    if (!src_xy_dev || !q_dev || !opt || !leaf_cand || n_leaf < 1 || !best_leaf ||
        (n_item > 0 && !item_cand))
        return set_error("autotune: missing argument"), FMM_ERR_ARG;
    if (repeats < 1 || evaluations < 1) return set_error("autotune: repeats, evaluations >= 1"), FMM_ERR_ARG;
    const bool batched = n_inst > 0;
    if (batched && (!src_off_host || tgt_xy_dev))
        return set_error("autotune: batched problems need offsets and no separate points"),
               FMM_ERR_ARG;
    const int64_t n_all = batched ? src_off_host[n_inst] : n_src;
    const int64_t m = (!batched && tgt_xy_dev) ? n_tgt : n_all;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    double2 *phi = nullptr;
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&phi), 16 * (size_t)std::max<int64_t>(m, 1), s);
    if (e != cudaSuccess) return cuda_fail(e, "autotune buffer");
    fmm_status st = FMM_OK;
    double best = 0.0;
    const int ni = std::max(n_item, 1);
    *best_leaf = leaf_cand[0];
    if (best_item) *best_item = n_item > 0 ? item_cand[0] : opt->p2p_item_sources;
    for (int c = 0; c < n_leaf * ni && st == FMM_OK; ++c) {
        fmm_options o = *opt;
        o.leaf_size = leaf_cand[c / ni];
        if (n_item > 0) o.p2p_item_sources = item_cand[c % ni];
        double tmin = 0.0;
        // one untimed pass, then the fastest of `repeats` timed passes (build + evaluations)
        for (int r = 0; r <= repeats && st == FMM_OK; ++r) {
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) {
                st = cuda_fail(e, "autotune");
                break;
            }
            auto t0 = std::chrono::steady_clock::now();
            fmm_tree *tree = nullptr;
            st = batched ? fmm_build_batched(n_inst, src_off_host, src_xy_dev, nullptr, nullptr,
                                             &o, stream, &tree)
                         : fmm_build_tree(src_xy_dev, n_src, tgt_xy_dev, n_tgt, &o, stream, &tree);
            for (int k = 0; k < evaluations && st == FMM_OK; ++k)
                st = fmm_evaluate(tree, q_dev, reinterpret_cast<double *>(phi), stream);
            if (st == FMM_OK) st = fmm_tree_sync(tree, stream);
            fmm_tree_free(tree);
            const double dt = std::chrono::duration<double, std::milli>(
                                  std::chrono::steady_clock::now() - t0).count();
            if (r > 0 && (r == 1 || dt < tmin)) tmin = dt;
        }
        if (st != FMM_OK) break;
        if (ms) ms[c] = (float)tmin;
        if (c == 0 || tmin < best) {
            best = tmin;
            *best_leaf = o.leaf_size;
            if (best_item) *best_item = o.p2p_item_sources;
        }
    }
    dev_free(phi, s);
    cudaStreamSynchronize(s);
    return st;
}

fmm_status fmm_autotune_leaf(const double *src_xy_dev, int64_t n_src, const double *tgt_xy_dev,
                             int64_t n_tgt, int n_inst, const int64_t *src_off_host,
                             const double *q_dev, const fmm_options *opt, const int *candidates,
                             int n_cand, int repeats, int evaluations, void *stream,
                             int *best_leaf, float *ms) {
    return autotune(src_xy_dev, n_src, tgt_xy_dev, n_tgt, n_inst, src_off_host, q_dev, opt,
                    candidates, n_cand, nullptr, 0, repeats, evaluations, stream, best_leaf,
                    nullptr, ms);
}

fmm_status fmm_autotune(const double *src_xy_dev, int64_t n_src, const double *tgt_xy_dev,
                        int64_t n_tgt, int n_inst, const int64_t *src_off_host,
                        const double *q_dev, fmm_options *opt, const int *leaf_cand, int n_leaf,
                        const int *item_cand, int n_item, int repeats, int evaluations,
                        void *stream, float *ms) {
    if (!opt || n_item < 1) return set_error("autotune: missing argument"), FMM_ERR_ARG;
    int bl = 0, bi = 0;
    fmm_status st = autotune(src_xy_dev, n_src, tgt_xy_dev, n_tgt, n_inst, src_off_host, q_dev,
                             opt, leaf_cand, n_leaf, item_cand, n_item, repeats, evaluations,
                             stream, &bl, &bi, ms);
    if (st == FMM_OK) {
        opt->leaf_size = bl;
        opt->p2p_item_sources = bi;
    }
    return st;
}

fmm_status fmm_set_graph(fmm_tree *tree, int enable) {
    if (!tree) return set_error("NULL tree"), FMM_ERR_ARG;
    tree->t.use_graph = enable != 0;
    return FMM_OK;
}

}  // extern "C"
