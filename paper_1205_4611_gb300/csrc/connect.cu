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
// The P2P work list is built here too: one item per (target leaf, chunk of
// at most P2P_CHUNK targets), ordered by decreasing pair count so that the
// longest items start first.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace gbfmm {

int64_t tree_level_base(int l);

namespace {

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

// Chunks per target leaf.
__global__ void k_leaf_chunks(int64_t nleaf, int64_t leaf0, const int2 *__restrict__ box_tgt,
                              int chunk, uint32_t *cnt) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int nt = box_tgt[leaf0 + b].y;
    cnt[b] = (uint32_t)((nt + chunk - 1) / chunk);
}

// One item per chunk; cost = targets * near-field sources, sorted descending.
__global__ void k_fill_items(int64_t nleaf, int64_t leaf0, const int2 *__restrict__ box_tgt,
                             const int2 *__restrict__ box_src, const int *__restrict__ strong_off,
                             const int *__restrict__ strong, int chunk,
                             const uint32_t *__restrict__ off, int2 *items, uint64_t *key,
                             uint32_t *val) {
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int64_t g = leaf0 + b;
    int2 tt = box_tgt[g];
    int64_t nsrc = 0;
    for (int e = strong_off[g]; e < strong_off[g + 1]; ++e) nsrc += box_src[strong[e]].y;
    uint32_t o = off[b];
    for (int t0 = 0, k = 0; t0 < tt.y; t0 += chunk, ++k) {
        int nt = min(chunk, tt.y - t0);
        uint64_t cost = (uint64_t)nt * (uint64_t)nsrc;
        if (cost > 0xffffffffull) cost = 0xffffffffull;
        items[o + k] = make_int2((int)g, t0);
        key[o + k] = 0xffffffffull - cost;
        val[o + k] = o + k;
    }
}

__global__ void k_gather_items(int64_t n, const uint32_t *__restrict__ order,
                               const int2 *__restrict__ in, int2 *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = in[order[i]];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

constexpr int P2P_CHUNK = 64;

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
        // P2P work items over the target leaves
        const int64_t nleaf = int64_t(1) << (2 * L), leaf0 = lb(L);
        const int64_t max_items = nleaf + (t.separate ? t.n_tgt : t.n_src) / P2P_CHUNK + 1;
        uint32_t *cnt;
        int2 *items_raw, *items;
        uint64_t *key, *kalt;
        uint32_t *val, *valt;
        CK(arena_alloc(tmp, &cnt, nleaf + 1));
        CK(arena_alloc(tmp, &items_raw, max_items));
        CK(arena_alloc(tmp, &key, max_items));
        CK(arena_alloc(tmp, &kalt, max_items));
        CK(arena_alloc(tmp, &val, max_items));
        CK(arena_alloc(tmp, &valt, max_items));
        CK(arena_alloc(lists, &items, max_items));
        k_leaf_chunks<<<nblk(nleaf, 256), 256, 0, s>>>(nleaf, leaf0, t.box_tgt, P2P_CHUNK, cnt); note_launch();
        CK(cudaGetLastError());
        CK(exclusive_scan_u32(cnt, cnt, nleaf, nullptr, tmp, s));
        k_fill_items<<<nblk(nleaf, 128), 128, 0, s>>>(nleaf, leaf0, t.box_tgt, t.box_src,
                                                      strong_off, strong, P2P_CHUNK, cnt,
                                                      items_raw, key, val); note_launch();
        CK(cudaGetLastError());
        int host[4];
        int hstat = 0;
        CK(cudaMemcpyAsync(&host[0], weak_off + nb, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&host[1], strong_off + nb, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&host[2], cnt + nleaf, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaMemcpyAsync(&hstat, t.status, sizeof(int), cudaMemcpyDeviceToHost, s));
        CK(cudaStreamSynchronize(s));
        if (hstat & ST_LIST_OVERFLOW) {
            cap_w = std::max<int64_t>(2 * cap_w, (int64_t)host[0] + 64);
            cap_s = std::max<int64_t>(2 * cap_s, (int64_t)host[1] + 64);
            tmp.release();
            lists.release();
            continue;
        }
        const int n_items = host[2];
        if (n_items > 1) {
            CK(radix_sort_pairs(&key, &val, kalt, valt, n_items, 0xfu, tmp, s));
        }
        k_gather_items<<<nblk(n_items, 256), 256, 0, s>>>(n_items, val, items_raw, items); note_launch();
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
#undef CK
        return FMM_OK;
    }
    set_error("interaction lists did not fit after repeated growth");
    return FMM_ERR_NOMEM;
}

}  // namespace gbfmm
