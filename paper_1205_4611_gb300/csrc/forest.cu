// Batched form: many independent FMM instances evaluated in one pass.
//
// Every instance gets its own pyramid tree and interaction lists (built with
// the single-instance code on the same stream); the trees are then merged
// into one forest whose arrays use global box ids, global source positions
// and global list offsets.  The evaluation kernels only use explicit box
// relations (leaf list, boxes per level, parent / first child, CSR lists,
// work items), so a forest is evaluated by exactly the launches of a single
// tree: one P2M over all leaves, one M2M and one L2L launch per level over
// all instances, one M2L over all weak pairs, one P2P over all work items
// and one combine.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <thread>
#include <vector>

#include "common.cuh"
#include "internal.h"

namespace gbfmm {

namespace {

__host__ __device__ inline int64_t lb(int l) { return ((int64_t(1) << (2 * l)) - 1) / 3; }

__global__ void k_copy_add(int64_t n, const int *__restrict__ in, int *out, int add) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i] + add;
}

__global__ void k_copy_int2_add(int64_t n, const int2 *__restrict__ in, int2 *out, int addx,
                                int addy) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        int2 v = in[i];
        out[i] = make_int2(v.x + addx, v.y + addy);
    }
}

// Work items: box id + ax; P2P items (run e0 >= 0) index the near-field list
// (+ az), M2P items (~e0, ~e1) the M2P list (+ am, i.e. ~e - am).
__global__ void k_copy_items_add(int64_t n, const int4 *__restrict__ in, int4 *out, int ax,
                                 int az, int am) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        int4 v = in[i];
        if (v.z >= 0)
            out[i] = make_int4(v.x + ax, v.y, v.z + az, v.w + az);
        else
            out[i] = make_int4(v.x + ax, v.y, v.z - am, v.w - am);
    }
}

__global__ void k_gather_src(int64_t n, const uint32_t *__restrict__ perm,
                             const double2 *__restrict__ in, double2 *out) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[perm[i]];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

cudaError_t ensure_tables();

fmm_status build_forest(Tree &F, int n_inst, const int64_t *src_off, const double *src_xy,
                        const fmm_options &opt, int (*levels_for)(int64_t, const fmm_options &),
                        bool p2p_items_needed, cudaStream_t s) {
    cudaError_t e;
    std::vector<Tree *> T(n_inst, nullptr);
    auto cleanup = [&]() {
        for (Tree *t : T)
            if (t) {
                t->mem.release();
                delete t;
            }
    };
#define CK(call)                        \
    do {                                \
        if ((e = (call)) != cudaSuccess) { \
            cleanup();                  \
            return cuda_fail(e, #call); \
        }                               \
    } while (0)
    // 1. one tree per instance (self-evaluation).  The builds are launch- and
    // synchronisation-bound, so several host threads build instances at once,
    // each on a private stream; the merge below runs on the caller's stream
    // after all of them have finished.
    int Lmax = 0;
    for (int i = 0; i < n_inst; ++i) {
        Tree *t = new Tree;
        T[i] = t;
        t->p = opt.p;
        t->theta = opt.theta;
        t->leaf = opt.leaf_size;
        t->precision = FMM_PREC_FP64;  // mixed-mode data are prepared on the forest
        t->p2p_items_needed = p2p_items_needed;
        t->p2l_m2p = opt.p2l_m2p;
        t->box_fit = opt.box_fit;
        t->L = levels_for(src_off[i + 1] - src_off[i], opt);
        if (t->L > 12) {
            cleanup();
            set_error("an instance needs more than 12 levels");
            return FMM_ERR_ARG;
        }
        t->n_src = t->n_tgt = src_off[i + 1] - src_off[i];
        Lmax = std::max(Lmax, t->L);
    }
    {
        int dev = 0;
        CK(cudaGetDevice(&dev));
        // the caller's stream may hold the points' producer: wait for it first
        CK(cudaStreamSynchronize(s));
        const unsigned hw = std::max(1u, std::thread::hardware_concurrency());
        const int nthr = (int)std::min<int64_t>(std::min<unsigned>(hw, 8u), n_inst);
        std::atomic<int> next{0};
        std::atomic<int> failed{0};
        std::vector<fmm_status> wst(nthr, FMM_OK);
        std::vector<std::string> werr(nthr);
        auto work = [&](int w) {
            cudaStream_t ws = nullptr;
            cudaError_t ce = cudaSetDevice(dev);
            if (ce == cudaSuccess) ce = cudaStreamCreateWithFlags(&ws, cudaStreamNonBlocking);
            if (ce != cudaSuccess) {
                wst[w] = cuda_fail(ce, "forest worker");
                werr[w] = "forest worker stream";
                failed = 1;
                return;
            }
            std::vector<int> mine;
            HostStage hs;
            if (!hs.w) {
                wst[w] = FMM_ERR_NOMEM;
                werr[w] = "page-locked stage allocation failed";
                failed = 1;
            }
            for (int i = next++; i < n_inst && !failed; i = next++) {
                Tree *t = T[i];
                mine.push_back(i);
                t->mem.stream = ws;
                fmm_status st = build_topology(*t, src_xy + 2 * src_off[i], nullptr, nullptr, ws);
                if (st == FMM_OK) st = build_connectivity(*t, ws, hs.w);
                if (st != FMM_OK) {
                    wst[w] = st;
                    werr[w] = last_error_message();
                    failed = 1;
                }
            }
            const uint64_t mark = dev_cache_mark();
            if (cudaStreamSynchronize(ws) == cudaSuccess) dev_cache_stream_idle(ws, mark);
            for (int i : mine) T[i]->mem.stream = s;  // freed after the merge, in its order
            cudaStreamDestroy(ws);
        };
        std::vector<std::thread> pool;
        for (int w = 1; w < nthr; ++w) pool.emplace_back(work, w);
        work(0);
        for (auto &th : pool) th.join();
        for (int w = 0; w < nthr; ++w)
            if (wst[w] != FMM_OK) {
                cleanup();
                set_error(werr[w]);
                return wst[w];
            }
    }
    // 2. offsets
    std::vector<int64_t> box_base(n_inst + 1, 0), weak_base(n_inst + 1, 0),
        strong_base(n_inst + 1, 0), item_base(n_inst + 1, 0), chunk_base(n_inst + 1, 0),
        near_base(n_inst + 1, 0), p2l_base(n_inst + 1, 0), m2p_base(n_inst + 1, 0),
        p2p_item_base(n_inst + 1, 0);
    for (int i = 0; i < n_inst; ++i) {
        box_base[i + 1] = box_base[i] + T[i]->n_boxes;
        weak_base[i + 1] = weak_base[i] + T[i]->n_weak;
        strong_base[i + 1] = strong_base[i] + T[i]->n_strong;
        item_base[i + 1] = item_base[i] + T[i]->n_items;
        chunk_base[i + 1] = chunk_base[i] + T[i]->n_chunks;
        p2p_item_base[i + 1] = p2p_item_base[i] + T[i]->n_p2p_items;
        near_base[i + 1] = near_base[i] + T[i]->n_near;
        p2l_base[i + 1] = p2l_base[i] + T[i]->n_p2l;
        m2p_base[i + 1] = m2p_base[i] + T[i]->n_m2p;
    }
    const bool shortcut = opt.p2l_m2p != 0;
    const int64_t nb = box_base[n_inst], n_src = src_off[n_inst];
    if (nb > INT32_MAX / 2 || weak_base[n_inst] > INT32_MAX / 2) {
        cleanup();
        set_error("forest too large");
        return FMM_ERR_ARG;
    }
    F.n_inst = n_inst;
    F.L = Lmax;
    F.n_src = F.n_tgt = n_src;
    F.separate = false;
    F.n_boxes = nb;
    F.n_weak = weak_base[n_inst];
    F.n_strong = strong_base[n_inst];
    F.n_items = (int)item_base[n_inst];
    F.n_chunks = (int)chunk_base[n_inst];
    F.n_p2p_items = (int)p2p_item_base[n_inst];
    F.n_near = near_base[n_inst];
    F.n_p2l = p2l_base[n_inst];
    F.n_m2p = m2p_base[n_inst];
    // 3. merged device arrays
    CK(arena_alloc(F.mem, &F.perm, n_src));
    CK(arena_alloc(F.mem, &F.xs, n_src));
    CK(arena_alloc(F.mem, &F.rect, nb));
    if (opt.box_fit)
        CK(arena_alloc(F.mem, &F.rect_geo, nb));
    else
        F.rect_geo = F.rect;
    CK(arena_alloc(F.mem, &F.geom, nb));
    CK(arena_alloc(F.mem, &F.box_src, nb));
    CK(arena_alloc(F.mem, &F.weak_off, nb + 1));
    CK(arena_alloc(F.mem, &F.strong_off, nb + 1));
    CK(arena_alloc(F.mem, &F.weak, F.n_weak + 1));
    CK(arena_alloc(F.mem, &F.strong, F.n_strong + 1));
    if (shortcut) {
        CK(arena_alloc(F.mem, &F.near_off, nb + 1));
        CK(arena_alloc(F.mem, &F.p2l_off, nb + 1));
        CK(arena_alloc(F.mem, &F.m2p_off, nb + 1));
        CK(arena_alloc(F.mem, &F.near, F.n_near + 1));
        CK(arena_alloc(F.mem, &F.p2l, F.n_p2l + 1));
        CK(arena_alloc(F.mem, &F.m2p, F.n_m2p + 1));
    }
    F.p2p_list = shortcut ? F.near : F.strong;
    F.p2p_off = shortcut ? F.near_off : F.strong_off;
    CK(arena_alloc(F.mem, &F.p2p_items, (size_t)F.n_items + 1));
    CK(arena_alloc(F.mem, &F.p2p_order, (size_t)F.n_items + 1));
    CK(arena_alloc(F.mem, &F.p2p_chunks, (size_t)F.n_chunks + 1));
    CK(arena_alloc(F.mem, &F.p2p_item0, (size_t)F.n_chunks + 1));
    CK(arena_alloc(F.mem, &F.p2p_partial, (size_t)F.n_items * 64 + 1));
    CK(arena_alloc(F.mem, &F.status, 1));
    CK(cudaMemsetAsync(F.status, 0, sizeof(int), s));
    for (int i = 0; i < n_inst; ++i) {
        Tree &t = *T[i];
        const int bb = (int)box_base[i], sb = (int)src_off[i];
        launch_k(k_copy_add, nblk(t.n_src, 256), 256, 0, s, t.n_src,
                 reinterpret_cast<const int *>(t.perm), reinterpret_cast<int *>(F.perm) + sb, sb);
        CK(cudaMemcpyAsync(F.rect + bb, t.rect, t.n_boxes * sizeof(double4),
                           cudaMemcpyDeviceToDevice, s));
        if (opt.box_fit)
            CK(cudaMemcpyAsync(F.rect_geo + bb, t.rect_geo, t.n_boxes * sizeof(double4),
                               cudaMemcpyDeviceToDevice, s));
        launch_k(k_copy_int2_add, nblk(t.n_boxes, 256), 256, 0, s, t.n_boxes, t.box_src,
                 F.box_src + bb, sb, 0);
        launch_k(k_copy_add, nblk(t.n_boxes, 256), 256, 0, s, t.n_boxes, t.weak_off,
                 F.weak_off + bb, (int)weak_base[i]);
        launch_k(k_copy_add, nblk(t.n_boxes, 256), 256, 0, s, t.n_boxes, t.strong_off,
                 F.strong_off + bb, (int)strong_base[i]);
        if (t.n_weak) {
            launch_k(k_copy_add, nblk(t.n_weak, 256), 256, 0, s, t.n_weak, t.weak,
                     F.weak + weak_base[i], bb);
        }
        launch_k(k_copy_add, nblk(t.n_strong, 256), 256, 0, s, t.n_strong, t.strong,
                 F.strong + strong_base[i], bb);
        if (shortcut) {
            const int *offs[3] = {t.near_off, t.p2l_off, t.m2p_off};
            const int *ents[3] = {t.near, t.p2l, t.m2p};
            int *foffs[3] = {F.near_off, F.p2l_off, F.m2p_off};
            int *fents[3] = {F.near, F.p2l, F.m2p};
            const int64_t bases[3] = {near_base[i], p2l_base[i], m2p_base[i]};
            const int64_t counts[3] = {t.n_near, t.n_p2l, t.n_m2p};
            for (int k = 0; k < 3; ++k) {
                launch_k(k_copy_add, nblk(t.n_boxes, 256), 256, 0, s, t.n_boxes, offs[k],
                         foffs[k] + bb, (int)bases[k]);
                if (counts[k]) {
                    launch_k(k_copy_add, nblk(counts[k], 256), 256, 0, s, counts[k], ents[k],
                             fents[k] + bases[k], bb);
                }
            }
        }
        // the items index the list their instance's P2P used (strong or near)
        const int list_base = (int)(shortcut ? near_base[i] : strong_base[i]);
        if (t.n_items) {
            launch_k(k_copy_items_add, nblk(t.n_items, 256), 256, 0, s, t.n_items, t.p2p_items,
                     F.p2p_items + item_base[i], bb, list_base, (int)m2p_base[i]);
            // launch order: every instance's P2P items, then every instance's M2P items
            const int np = t.n_p2p_items, nm = t.n_items - t.n_p2p_items;
            if (np) {
                launch_k(k_copy_add, nblk(np, 256), 256, 0, s, np, t.p2p_order,
                         F.p2p_order + p2p_item_base[i], (int)item_base[i]);
            }
            if (nm) {
                launch_k(k_copy_add, nblk(nm, 256), 256, 0, s, nm, t.p2p_order + np,
                         F.p2p_order + F.n_p2p_items + (item_base[i] - p2p_item_base[i]),
                         (int)item_base[i]);
            }
        }
        if (t.n_chunks) {
            launch_k(k_copy_int2_add, nblk(t.n_chunks, 256), 256, 0, s, t.n_chunks, t.p2p_chunks,
                     F.p2p_chunks + chunk_base[i], bb, 0);
            launch_k(k_copy_add, nblk(t.n_chunks, 256), 256, 0, s, t.n_chunks, t.p2p_item0,
                     F.p2p_item0 + chunk_base[i], (int)item_base[i]);
        }
        CK(cudaGetLastError());
    }
    // closing entries of the CSR / chunk offsets
    {
        int tail[6] = {(int)F.n_weak, (int)F.n_strong, F.n_items,
                       (int)F.n_near, (int)F.n_p2l, (int)F.n_m2p};
        CK(cudaMemcpyAsync(F.weak_off + nb, &tail[0], 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(F.strong_off + nb, &tail[1], 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(F.p2p_item0 + F.n_chunks, &tail[2], 4, cudaMemcpyHostToDevice, s));
        if (shortcut) {
            CK(cudaMemcpyAsync(F.near_off + nb, &tail[3], 4, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(F.p2l_off + nb, &tail[4], 4, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(F.m2p_off + nb, &tail[5], 4, cudaMemcpyHostToDevice, s));
        }
        CK(cudaStreamSynchronize(s));  // the host tail values must outlive the copies
    }
    launch_k(k_gather_src, nblk(n_src, 256), 256, 0, s, n_src, F.perm,
             reinterpret_cast<const double2 *>(src_xy), F.xs);
    CK(cudaGetLastError());
    F.tperm = F.perm;
    F.xt = F.xs;
    F.box_tgt = F.box_src;
    {
        fmm_status st = compute_geom(F, s);
        if (st != FMM_OK) {
            cleanup();
            return st;
        }
    }
    // 4. relations, boxes by level and leaves (host-built)
    std::vector<int> parent(nb), child0(nb), lvl, leaves;
    lvl.reserve(nb);
    for (int i = 0; i < n_inst; ++i) {
        const int L = T[i]->L;
        for (int l = 0; l <= L; ++l)
            for (int64_t b = 0; b < (int64_t(1) << (2 * l)); ++b) {
                int64_t g = box_base[i] + lb(l) + b;
                parent[g] = l > 0 ? (int)(box_base[i] + lb(l - 1) + b / 4) : -1;
                child0[g] = l < L ? (int)(box_base[i] + lb(l + 1) + 4 * b) : -1;
                if (l == L) leaves.push_back((int)g);
            }
    }
    for (int l = 0; l <= Lmax; ++l) {
        F.level_start[l] = (int64_t)lvl.size();
        for (int i = 0; i < n_inst; ++i)
            if (T[i]->L >= l)
                for (int64_t b = 0; b < (int64_t(1) << (2 * l)); ++b)
                    lvl.push_back((int)(box_base[i] + lb(l) + b));
    }
    F.level_start[Lmax + 1] = (int64_t)lvl.size();
    F.n_leaves = (int)leaves.size();
    CK(arena_alloc(F.mem, &F.parent, nb));
    CK(arena_alloc(F.mem, &F.child0, nb));
    CK(arena_alloc(F.mem, &F.lvl_boxes, nb));
    CK(arena_alloc(F.mem, &F.leaves, leaves.size()));
    CK(cudaMemcpyAsync(F.parent, parent.data(), nb * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(F.child0, child0.data(), nb * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(F.lvl_boxes, lvl.data(), nb * sizeof(int), cudaMemcpyHostToDevice, s));
    CK(cudaMemcpyAsync(F.leaves, leaves.data(), leaves.size() * sizeof(int),
                       cudaMemcpyHostToDevice, s));
    CK(cudaStreamSynchronize(s));  // host vectors are released on return
    cleanup();
#undef CK
    return FMM_OK;
}

}  // namespace gbfmm
