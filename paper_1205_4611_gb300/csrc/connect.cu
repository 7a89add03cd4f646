// Topological phase, part 2 (Sec. 3.2, "connecting"): directed interaction
// lists by the theta-criterion (Eq. 3).  A box is strongly coupled to itself;
// at level l >= 1 the candidates of box b are the children of the strong set
// of b's parent, taken in list order, children 0..3; a candidate that is well
// separated from b becomes weak (an M2L source), the others stay strong
// (Sec. 2).  Leaf strong lists drive the near-field P2P.  One thread per box
// and one launch per level, as in the paper (Sec. 3.2); lists are CSR over
// all boxes, counted, scanned and filled on the device with no host round
// trip; a capacity overflow is latched and the build is retried larger.
//
// The P2P work list is built here too: items are (target leaf, chunk of at
// most 64 targets, run of the leaf's strong list with at most 2048 sources);
// they are launched in order of decreasing pair count and their partial sums
// are combined per target, in item order, by the evaluation's last kernel.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace gbfmm {

int64_t tree_level_base(int l);

namespace {

constexpr int P2P_CHUNK = 64;     // targets per work item
constexpr int P2P_SRC_CAP = 2048; // near-field sources per work item (one leaf may exceed)

__host__ __device__ inline int64_t lb(int l) { return ((int64_t(1) << (2 * l)) - 1) / 3; }

__global__ void k_conn_init(int *weak_off, int *strong_off, int *strong) {
    weak_off[0] = 0;
    weak_off[1] = 0;
    strong_off[0] = 0;
    strong_off[1] = 1;
    strong[0] = 0;
}

GBI Rect to_rect(double4 v) { return Rect{v.x, v.y, v.z, v.w}; }

template <bool FILL>
__global__ void k_conn_level(int l, const double4 *__restrict__ rect, double theta,
                             const int *__restrict__ strong_prev_off, const int *__restrict__ strong_in,
                             int64_t cap_s, int *__restrict__ weak_off, int *__restrict__ weak,
                             int64_t cap_w, int *__restrict__ strong_off, int *__restrict__ strong,
                             uint32_t *wcnt, uint32_t *scnt, int *status) {
    int64_t nbl = int64_t(1) << (2 * l);
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbl) return;
    int64_t g = lb(l) + b, par = lb(l - 1) + b / 4;
    int e0 = strong_prev_off[par], e1 = strong_prev_off[par + 1];
    if ((int64_t)e1 > cap_s) {
        atomicOr(status, ST_LIST_OVERFLOW);
        e1 = e0;
    }
    Rect rb = to_rect(rect[g]);
    int nw = 0, ns = 0;
    int wo = 0, so = 0;
    if (FILL) {
        wo = weak_off[g];
        so = strong_off[g];
    }
    for (int e = e0; e < e1; ++e) {
        int64_t sl = strong_in[e] - lb(l - 1);
        for (int ch = 0; ch < 4; ++ch) {
            int64_t c = lb(l) + 4 * sl + ch;
            bool ws = well_separated(rb, to_rect(rect[c]), theta);
            if (ws) {
                if (FILL) {
                    if ((int64_t)wo + nw < cap_w)
                        weak[wo + nw] = (int)c;
                    else
                        atomicOr(status, ST_LIST_OVERFLOW);
                }
                ++nw;
            } else {
                if (FILL) {
                    if ((int64_t)so + ns < cap_s)
                        strong[so + ns] = (int)c;
                    else
                        atomicOr(status, ST_LIST_OVERFLOW);
                }
                ++ns;
            }
        }
    }
    if (!FILL) {
        wcnt[b] = (uint32_t)nw;
        scnt[b] = (uint32_t)ns;
    }
}

// Chunks of <= P2P_CHUNK targets per target leaf.
__global__ void k_leaf_chunks(int64_t nleaf, int64_t leaf0, const int2 *__restrict__ box_tgt,
                              int chunk, uint32_t *cnt) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int nt = box_tgt[leaf0 + b].y;
    cnt[b] = (uint32_t)((nt + chunk - 1) / chunk);
}

// Runs of the leaf's strong list holding <= cap sources (a single leaf may
// exceed it on its own); returns the number of runs, optionally writing them.
GBI int source_runs(const int *__restrict__ strong, int e0, int e1, const int2 *__restrict__ box_src,
                    int cap, int *starts) {
    int nr = 0, acc = 0;
    for (int e = e0; e < e1; ++e) {
        int n = box_src[strong[e]].y;
        if (e == e0 || acc + n > cap) {
            if (starts) starts[nr] = e;
            ++nr;
            acc = 0;
        }
        acc += n;
    }
    return nr;
}

__global__ void k_leaf_runs(int64_t nleaf, int64_t leaf0, const int *__restrict__ strong_off,
                            const int *__restrict__ strong, const int2 *__restrict__ box_src,
                            const uint32_t *__restrict__ chunks, int cap, uint32_t *runs,
                            uint32_t *items) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int64_t g = leaf0 + b;
    int r = source_runs(strong, strong_off[g], strong_off[g + 1], box_src, cap, nullptr);
    runs[b] = (uint32_t)r;
    items[b] = (uint32_t)r * chunks[b];
}

// Items (leaf, first target, strong-list run), ordered by chunk then run;
// chunk c owns items [item0[c], item0[c+1]).  key/val feed the cost sort.
__global__ void k_fill_items(int64_t nleaf, int64_t leaf0, const int2 *__restrict__ box_tgt,
                             const int2 *__restrict__ box_src, const int *__restrict__ strong_off,
                             const int *__restrict__ strong, int chunk, int cap,
                             const uint32_t *__restrict__ chunk_off,
                             const uint32_t *__restrict__ item_off, int2 *chunks, int *item0,
                             int4 *items, uint64_t *key, uint32_t *val) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int64_t g = leaf0 + b;
    int2 tt = box_tgt[g];
    int e0 = strong_off[g], e1 = strong_off[g + 1];
    int nr = source_runs(strong, e0, e1, box_src, cap, nullptr);
    uint32_t c = chunk_off[b], it = item_off[b];
    for (int t0 = 0; t0 < tt.y; t0 += chunk, ++c) {
        int nt = min(chunk, tt.y - t0);
        chunks[c] = make_int2((int)g, t0);
        item0[c] = (int)it;
        // walk the runs again, emitting one item each
        int acc = 0, rs = e0;
        for (int e = e0; e <= e1; ++e) {
            int n = e < e1 ? box_src[strong[e]].y : 0;
            bool cut = (e == e1) || (e > rs && acc + n > cap);
            if (cut && e > rs) {
                uint64_t cost = (uint64_t)nt * (uint64_t)acc;
                if (cost > 0xffffffffull) cost = 0xffffffffull;
                items[it] = make_int4((int)g, t0, rs, e);
                key[it] = 0xffffffffull - cost;
                val[it] = it;
                ++it;
                rs = e;
                acc = 0;
            }
            acc += n;
        }
    }
    (void)nr;
}

__global__ void k_set_last(int *item0, int64_t n_chunks, int n_items) {
    item0[n_chunks] = n_items;
}

__global__ void k_copy_u32(int64_t n, const uint32_t *__restrict__ in, int *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int)in[i];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

fmm_status build_connectivity(Tree &t, cudaStream_t s) {
    const int L = t.L;
    const int64_t nb = t.n_boxes;
    int64_t cap_w = 160 * nb + 64, cap_s = 48 * nb + 64;
    cudaError_t e;
    for (int attempt = 0; attempt < 8; ++attempt) {
        DevArena tmp;
        tmp.stream = s;
        DevArena lists;
        lists.stream = s;
#define CK(call)                           \
    do {                                   \
        if ((e = (call)) != cudaSuccess) { \
            tmp.release();                 \
            lists.release();               \
            return cuda_fail(e, #call);    \
        }                                  \
    } while (0)
        int *weak_off, *weak, *strong_off, *strong;
        CK(arena_alloc(lists, &weak_off, nb + 1));
        CK(arena_alloc(lists, &strong_off, nb + 1));
        CK(arena_alloc(lists, &weak, cap_w));
        CK(arena_alloc(lists, &strong, cap_s));
        CK(cudaMemsetAsync(t.status, 0, sizeof(int), s));
        k_conn_init<<<1, 1, 0, s>>>(weak_off, strong_off, strong); note_launch();
        CK(cudaGetLastError());
        uint32_t *wcnt, *scnt;
        int64_t maxl = int64_t(1) << (2 * L);
        CK(arena_alloc(tmp, &wcnt, maxl + 1));
        CK(arena_alloc(tmp, &scnt, maxl + 1));
        for (int l = 1; l <= L; ++l) {
            int64_t nbl = int64_t(1) << (2 * l);
            k_conn_level<false><<<nblk(nbl, 128), 128, 0, s>>>(
                l, t.rect, t.theta, strong_off, strong, cap_s, weak_off, weak, cap_w, strong_off,
                strong, wcnt, scnt, t.status); note_launch();
            CK(cudaGetLastError());
            uint32_t *wo = reinterpret_cast<uint32_t *>(weak_off + lb(l));
            uint32_t *so = reinterpret_cast<uint32_t *>(strong_off + lb(l));
            CK(exclusive_scan_u32(wcnt, wo, nbl, wo, tmp, s));
            CK(exclusive_scan_u32(scnt, so, nbl, so, tmp, s));
            k_conn_level<true><<<nblk(nbl, 128), 128, 0, s>>>(
                l, t.rect, t.theta, strong_off, strong, cap_s, weak_off, weak, cap_w, strong_off,
                strong, wcnt, scnt, t.status); note_launch();
            CK(cudaGetLastError());
        }
        // P2P work items over the target leaves: chunks of <= P2P_CHUNK targets
        // times runs of <= P2P_SRC_CAP near-field sources
        const int64_t nleaf = int64_t(1) << (2 * L), leaf0 = lb(L);
        uint32_t *chunks_cnt, *runs, *items_cnt;
        CK(arena_alloc(tmp, &chunks_cnt, nleaf + 1));
        CK(arena_alloc(tmp, &runs, nleaf + 1));
        CK(arena_alloc(tmp, &items_cnt, nleaf + 1));
        k_leaf_chunks<<<nblk(nleaf, 256), 256, 0, s>>>(nleaf, leaf0, t.box_tgt, P2P_CHUNK, chunks_cnt); note_launch();
        CK(cudaGetLastError());
        k_leaf_runs<<<nblk(nleaf, 128), 128, 0, s>>>(nleaf, leaf0, strong_off, strong, t.box_src,
                                                     chunks_cnt, P2P_SRC_CAP, runs, items_cnt); note_launch();
        CK(cudaGetLastError());
        CK(exclusive_scan_u32(chunks_cnt, chunks_cnt, nleaf, nullptr, tmp, s));
        CK(exclusive_scan_u32(items_cnt, items_cnt, nleaf, nullptr, tmp, s));
        int host[4];
        int hstat = 0;
        CK(cudaMemcpyAsync(&host[0], weak_off + nb, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&host[1], strong_off + nb, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&host[2], chunks_cnt + nleaf, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&host[3], items_cnt + nleaf, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&hstat, t.status, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hstat & ST_LIST_OVERFLOW) {
            cap_w = std::max<int64_t>(2 * cap_w, (int64_t)host[0] + 64);
            cap_s = std::max<int64_t>(2 * cap_s, (int64_t)host[1] + 64);
            tmp.release();
            lists.release();
            continue;
        }
        const int n_chunks = host[2], n_items = host[3];
        int2 *chunks;
        int *item0, *order;
        int4 *items;
        uint64_t *key, *kalt;
        uint32_t *val, *valt;
        double2 *partial;
        CK(arena_alloc(lists, &chunks, (size_t)n_chunks + 1));
        CK(arena_alloc(lists, &item0, (size_t)n_chunks + 1));
        CK(arena_alloc(lists, &items, (size_t)n_items + 1));
        CK(arena_alloc(lists, &order, (size_t)n_items + 1));
        CK(arena_alloc(lists, &partial, (size_t)n_items * P2P_CHUNK + 1));
        CK(arena_alloc(tmp, &key, (size_t)n_items + 1));
        CK(arena_alloc(tmp, &kalt, (size_t)n_items + 1));
        CK(arena_alloc(tmp, &val, (size_t)n_items + 1));
        CK(arena_alloc(tmp, &valt, (size_t)n_items + 1));
        k_fill_items<<<nblk(nleaf, 128), 128, 0, s>>>(nleaf, leaf0, t.box_tgt, t.box_src,
                                                      strong_off, strong, P2P_CHUNK, P2P_SRC_CAP,
                                                      chunks_cnt, items_cnt, chunks, item0, items,
                                                      key, val); note_launch();
        CK(cudaGetLastError());
        k_set_last<<<1, 1, 0, s>>>(item0, n_chunks, n_items); note_launch();
        CK(cudaGetLastError());
        if (n_items > 1) CK(radix_sort_pairs(&key, &val, kalt, valt, n_items, 0xfu, tmp, s));
        k_copy_u32<<<nblk(n_items, 256), 256, 0, s>>>(n_items, val, order); note_launch();
        CK(cudaGetLastError());
        CK(cudaStreamSynchronize(s));
        tmp.release();
        // hand the lists over to the tree
        for (void *p : lists.ptrs) t.mem.ptrs.push_back(p);
        lists.ptrs.clear();
        t.weak_off = weak_off;
        t.weak = weak;
        t.strong_off = strong_off;
        t.strong = strong;
        t.n_weak = host[0];
        t.n_strong = host[1];
        t.p2p_items = items;
        t.n_items = n_items;
        t.p2p_order = order;
        t.p2p_chunks = chunks;
        t.p2p_item0 = item0;
        t.n_chunks = n_chunks;
        t.p2p_partial = partial;
#undef CK
        return FMM_OK;
    }
    set_error("interaction lists did not fit after repeated growth");
    return FMM_ERR_NOMEM;
}

}  // namespace gbfmm
