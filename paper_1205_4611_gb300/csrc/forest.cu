// Batched form: many independent FMM instances evaluated in one pass.
//
// Instances with the same number of levels L are built together as one tree
// with R roots (tree.cu, connect.cu: box ids level-major over the roots, root
// r's children 4r .. 4r+3, and so on), so a whole group costs the launches
// and synchronisations of a single build: one bounding-box launch for all
// roots, one presort, the same split rounds and connectivity levels.  The
// group trees (one per distinct L, a handful) are then merged into one forest
// whose arrays use global box ids, global source and target positions and
// global list offsets.  The evaluation kernels only use explicit box
// relations (leaf list, boxes per level, parent / first child, CSR lists,
// work items), so a forest is evaluated by exactly the launches of a single
// tree: one P2M over all leaves, one M2M and one L2L launch per level over
// all instances, one M2L over all weak pairs, one P2P over all work items
// and one combine.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <string>
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

// Group position -> caller index: root r of the group holds the caller's
// points [coff[r], coff[r] + goff[r+1] - goff[r]) at group positions
// [goff[r], goff[r+1]).
__global__ void k_group_map(int64_t n, int R, const int64_t *__restrict__ goff,
                            const int64_t *__restrict__ coff, uint32_t *map) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = R;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (goff[mid] <= i)
            lo = mid;
        else
            hi = mid;
    }
    map[i] = (uint32_t)(coff[lo] + (i - goff[lo]));
}

// out[i] = map[perm[i]]: a group tree's permutation in caller indices.
__global__ void k_compose(int64_t n, const uint32_t *__restrict__ perm,
                          const uint32_t *__restrict__ map, uint32_t *out) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = map[perm[i]];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

cudaError_t ensure_tables();

fmm_status build_forest(Tree &F, int n_inst, const int64_t *src_off, const double *src_xy,
                        const int64_t *tgt_off, const double *tgt_xy, const fmm_options &opt,
                        int (*levels_for)(int64_t, const fmm_options &), bool p2p_items_needed,
                        cudaStream_t s) {
    cudaError_t e;
    const bool separate = tgt_xy != nullptr;
    std::vector<Tree *> T;
    std::vector<uint32_t *> gmap, tgmap;  // per group: position -> caller index
    DevArena maps;
    maps.stream = s;
    auto cleanup = [&]() {
        for (Tree *t : T)
            if (t) {
                t->mem.release();
                delete t;
            }
        maps.release();
    };
#define CK(call)                        \
    do {                                \
        if ((e = (call)) != cudaSuccess) { \
            cleanup();                  \
            return cuda_fail(e, #call); \
        }                               \
    } while (0)
    // 1. instances grouped by their number of levels; each group is one tree
    // with a root per instance (in caller order), built on the caller's stream
    std::map<int, std::vector<int>> by_level;
    int Lmax = 0;
    for (int i = 0; i < n_inst; ++i) {
        const int L = levels_for(src_off[i + 1] - src_off[i], opt);
        if (L > 12) {
            cleanup();
            set_error("an instance needs more than 12 levels");
            return FMM_ERR_ARG;
        }
        by_level[L].push_back(i);
        Lmax = std::max(Lmax, L);
    }
    const int n_groups = (int)by_level.size();
    std::vector<int64_t> group_src(n_groups + 1, 0), group_tgt(n_groups + 1, 0);
    {
        HostStage hs;
        if (!hs.w) {
            cleanup();
            set_error("page-locked stage allocation failed");
            return FMM_ERR_NOMEM;
        }
        int g = 0;
        for (auto &kv : by_level) {
            const std::vector<int> &inst = kv.second;
            const int R = (int)inst.size();
            Tree *t = new Tree;
            T.push_back(t);
            t->p = opt.p;
            t->theta = opt.theta;
            t->leaf = opt.leaf_size;
            t->precision = FMM_PREC_FP64;  // mixed-mode data are prepared on the forest
            t->p2p_items_needed = p2p_items_needed;
            t->p2l_m2p = opt.p2l_m2p;
            t->box_fit = opt.box_fit;
            t->p2p_cap = opt.p2p_item_sources ? opt.p2p_item_sources : 2048;
            t->L = kv.first;
            t->n_roots = R;
            t->separate = separate;
            t->mem.stream = s;
            // group offsets of the roots' points, and where they sit in the caller's arrays
            std::vector<int64_t> coff(R + 1, 0), ctoff(R + 1, 0);
            t->root_off.assign(R + 1, 0);
            t->root_toff.assign(R + 1, 0);
            for (int r = 0; r < R; ++r) {
                const int i = inst[r];
                t->root_off[r + 1] = t->root_off[r] + (src_off[i + 1] - src_off[i]);
                coff[r] = src_off[i];
                if (separate) {
                    t->root_toff[r + 1] = t->root_toff[r] + (tgt_off[i + 1] - tgt_off[i]);
                    ctoff[r] = tgt_off[i];
                }
            }
            t->n_src = t->root_off[R];
            t->n_tgt = separate ? t->root_toff[R] : t->n_src;
            group_src[g + 1] = group_src[g] + t->n_src;
            group_tgt[g + 1] = group_tgt[g] + t->n_tgt;
            // the group's points, contiguous (root by root)
            int64_t *offs_d;
            uint32_t *map, *tmap = nullptr;
            double2 *gsrc, *gtgt = nullptr;
            DevArena tmp;
            tmp.stream = s;
            auto fail = [&](cudaError_t ce, const char *what) {
                tmp.release();
                cleanup();
                return cuda_fail(ce, what);
            };
            if ((e = arena_alloc(tmp, &offs_d, 4 * ((size_t)R + 1))) != cudaSuccess ||
                (e = arena_alloc(maps, &map, (size_t)t->n_src)) != cudaSuccess ||
                (e = arena_alloc(tmp, &gsrc, (size_t)t->n_src)) != cudaSuccess)
                return fail(e, "forest group");
            if ((e = cudaMemcpyAsync(offs_d, t->root_off.data(), (R + 1) * 8,
                                     cudaMemcpyHostToDevice, s)) != cudaSuccess ||
                (e = cudaMemcpyAsync(offs_d + R + 1, coff.data(), (R + 1) * 8,
                                     cudaMemcpyHostToDevice, s)) != cudaSuccess)
                return fail(e, "forest group offsets");
            launch_k(k_group_map, nblk(t->n_src, 256), 256, 0, s, t->n_src, R, offs_d,
                     offs_d + R + 1, map);
            launch_k(k_gather_src, nblk(t->n_src, 256), 256, 0, s, t->n_src, map,
                     reinterpret_cast<const double2 *>(src_xy), gsrc);
            if (separate) {
                if ((e = arena_alloc(maps, &tmap, (size_t)t->n_tgt)) != cudaSuccess ||
                    (e = arena_alloc(tmp, &gtgt, (size_t)t->n_tgt)) != cudaSuccess)
                    return fail(e, "forest group targets");
                if ((e = cudaMemcpyAsync(offs_d + 2 * (R + 1), t->root_toff.data(), (R + 1) * 8,
                                         cudaMemcpyHostToDevice, s)) != cudaSuccess ||
                    (e = cudaMemcpyAsync(offs_d + 3 * (R + 1), ctoff.data(), (R + 1) * 8,
                                         cudaMemcpyHostToDevice, s)) != cudaSuccess)
                    return fail(e, "forest group offsets");
                launch_k(k_group_map, nblk(t->n_tgt, 256), 256, 0, s, t->n_tgt, R,
                         offs_d + 2 * (R + 1), offs_d + 3 * (R + 1), tmap);
                launch_k(k_gather_src, nblk(t->n_tgt, 256), 256, 0, s, t->n_tgt, tmap,
                         reinterpret_cast<const double2 *>(tgt_xy), gtgt);
            }
            if ((e = cudaGetLastError()) != cudaSuccess) return fail(e, "forest group gather");
            fmm_status st = build_topology(*t, reinterpret_cast<const double *>(gsrc),
                                           reinterpret_cast<const double *>(gtgt), nullptr, s);
            if (st == FMM_OK) st = build_connectivity(*t, s, hs.w);
            // the host offsets must outlive their copies; the build synchronised
            tmp.release();
            if (st != FMM_OK) {
                cleanup();
                return st;
            }
            gmap.push_back(map);
            tgmap.push_back(tmap);
            ++g;
        }
    }
    // 2. offsets
    const int NT = n_groups;
    std::vector<int64_t> box_base(NT + 1, 0), weak_base(NT + 1, 0), strong_base(NT + 1, 0),
        item_base(NT + 1, 0), chunk_base(NT + 1, 0), near_base(NT + 1, 0), p2l_base(NT + 1, 0),
        m2p_base(NT + 1, 0), p2p_item_base(NT + 1, 0);
    for (int i = 0; i < NT; ++i) {
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
    const int64_t nb = box_base[NT], n_src = src_off[n_inst];
    const int64_t n_tgt = separate ? tgt_off[n_inst] : n_src;
    if (nb > INT32_MAX / 2 || weak_base[NT] > INT32_MAX / 2) {
        cleanup();
        set_error("forest too large");
        return FMM_ERR_ARG;
    }
    F.n_inst = n_inst;
    F.L = Lmax;
    F.n_src = n_src;
    F.n_tgt = n_tgt;
    F.separate = separate;
    F.n_boxes = nb;
    F.n_weak = weak_base[NT];
    F.n_strong = strong_base[NT];
    F.n_items = (int)item_base[NT];
    F.n_chunks = (int)chunk_base[NT];
    F.n_p2p_items = (int)p2p_item_base[NT];
    F.n_near = near_base[NT];
    F.n_p2l = p2l_base[NT];
    F.n_m2p = m2p_base[NT];
    // 3. merged device arrays
    CK(arena_alloc(F.mem, &F.perm, n_src));
    CK(arena_alloc(F.mem, &F.xs, n_src));
    if (separate) {
        CK(arena_alloc(F.mem, &F.tperm, n_tgt));
        CK(arena_alloc(F.mem, &F.xt, n_tgt));
        CK(arena_alloc(F.mem, &F.box_tgt, nb));
    }
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
    for (int i = 0; i < NT; ++i) {
        Tree &t = *T[i];
        const int bb = (int)box_base[i], sb = (int)group_src[i], tb = (int)group_tgt[i];
        launch_k(k_compose, nblk(t.n_src, 256), 256, 0, s, t.n_src, t.perm, gmap[i], F.perm + sb);
        if (separate) {
            launch_k(k_compose, nblk(t.n_tgt, 256), 256, 0, s, t.n_tgt, t.tperm, tgmap[i],
                     F.tperm + tb);
            launch_k(k_copy_int2_add, nblk(t.n_boxes, 256), 256, 0, s, t.n_boxes, t.box_tgt,
                     F.box_tgt + bb, tb, 0);
        }
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
        // the items index the list their group's P2P used (strong or near)
        const int list_base = (int)(shortcut ? near_base[i] : strong_base[i]);
        if (t.n_items) {
            launch_k(k_copy_items_add, nblk(t.n_items, 256), 256, 0, s, t.n_items, t.p2p_items,
                     F.p2p_items + item_base[i], bb, list_base, (int)m2p_base[i]);
            // launch order: every group's P2P items, then every group's M2P items
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
    // closing entries of the CSR / chunk offsets (the host values live until
    // the synchronisation at the end)
    const int tail[6] = {(int)F.n_weak, (int)F.n_strong, F.n_items,
                         (int)F.n_near, (int)F.n_p2l, (int)F.n_m2p};
    {
        CK(cudaMemcpyAsync(F.weak_off + nb, &tail[0], 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(F.strong_off + nb, &tail[1], 4, cudaMemcpyHostToDevice, s));
        CK(cudaMemcpyAsync(F.p2p_item0 + F.n_chunks, &tail[2], 4, cudaMemcpyHostToDevice, s));
        if (shortcut) {
            CK(cudaMemcpyAsync(F.near_off + nb, &tail[3], 4, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(F.p2l_off + nb, &tail[4], 4, cudaMemcpyHostToDevice, s));
            CK(cudaMemcpyAsync(F.m2p_off + nb, &tail[5], 4, cudaMemcpyHostToDevice, s));
        }
    }
    launch_k(k_gather_src, nblk(n_src, 256), 256, 0, s, n_src, F.perm,
             reinterpret_cast<const double2 *>(src_xy), F.xs);
    CK(cudaGetLastError());
    if (separate) {
        launch_k(k_gather_src, nblk(n_tgt, 256), 256, 0, s, n_tgt, F.tperm,
                 reinterpret_cast<const double2 *>(tgt_xy), F.xt);
        CK(cudaGetLastError());
    } else {
        F.tperm = F.perm;
        F.xt = F.xs;
        F.box_tgt = F.box_src;
    }
    {
        fmm_status st = compute_geom(F, s);
        if (st != FMM_OK) {
            cleanup();
            return st;
        }
    }
    // 4. relations, boxes by level and leaves (host-built): group i has
    // R_i roots and level-major ids, level l from R_i lb(l)
    std::vector<int> parent(nb), child0(nb), lvl, leaves;
    lvl.reserve(nb);
    for (int i = 0; i < NT; ++i) {
        const int L = T[i]->L;
        const int64_t R = T[i]->n_roots;
        for (int l = 0; l <= L; ++l)
            for (int64_t b = 0; b < (R << (2 * l)); ++b) {
                int64_t g = box_base[i] + R * lb(l) + b;
                parent[g] = l > 0 ? (int)(box_base[i] + R * lb(l - 1) + b / 4) : -1;
                child0[g] = l < L ? (int)(box_base[i] + R * lb(l + 1) + 4 * b) : -1;
                if (l == L) leaves.push_back((int)g);
            }
    }
    for (int l = 0; l <= Lmax; ++l) {
        F.level_start[l] = (int64_t)lvl.size();
        for (int i = 0; i < NT; ++i)
            if (T[i]->L >= l) {
                const int64_t R = T[i]->n_roots;
                for (int64_t b = 0; b < (R << (2 * l)); ++b)
                    lvl.push_back((int)(box_base[i] + R * lb(l) + b));
            }
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
