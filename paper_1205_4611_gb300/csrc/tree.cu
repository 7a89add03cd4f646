// Topological phase, part 1 (Sec. 3.2, "sorting"): the median-split pyramid
// tree.  Every box is split twice per level, along the longer side of its
// rectangle, at the median of its sources ordered by (coordinate, index)
// (Sec. 2; Alg. "Partitioning with successive splits" is the paper's GPU
// design, replaced here by an exact deterministic scheme):
//
//   1. both coordinates are presorted once (stable LSD radix sort of
//      order-preserving 64-bit keys, ties by index);
//   2. each split round keeps one x-ordered and one y-ordered index list per
//      box segment; the median is the middle of the segment's list along the
//      split axis, every element is flagged left/right, and both lists are
//      stably partitioned by the flag (a global exclusive scan ranks them);
//   3. within a leaf, sources are left in the order of the leaf's last split
//      axis, which is the order a per-box sort produces.
//
// Evaluation points descend the split lines (<= line goes left) and are
// grouped by leaf with a stable radix sort (original order inside a leaf).
#include <cuda_runtime.h>

#include <algorithm>
#include <utility>

#include "common.cuh"
#include "internal.h"

namespace gbfmm {

namespace {

GBI double canon(double x) { return __dadd_rn(x, 0.0); }

__host__ __device__ inline int64_t level_base(int l) { return ((int64_t(1) << (2 * l)) - 1) / 3; }

GBI void warp_minmax(uint64_t &mn, uint64_t &mx, uint64_t &o) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        uint64_t a = __shfl_xor_sync(0xffffffffu, mn, d);
        uint64_t b = __shfl_xor_sync(0xffffffffu, mx, d);
        uint64_t c = __shfl_xor_sync(0xffffffffu, o, d);
        mn = a < mn ? a : mn;
        mx = b > mx ? b : mx;
        o |= c;
    }
}

// acc[0..3] = min x, max x, min y, max y (order keys); acc[4], acc[5] = OR over
// sources of (key ^ key of source 0) for x and y: the key bits that vary.
__global__ void k_bbox(const double2 *__restrict__ src, int64_t n, const double2 *__restrict__ tgt,
                       int64_t m, unsigned long long *acc, int *status) {
    uint64_t rx = order_key(src[0].x), ry = order_key(src[0].y);
    uint64_t mnx = ~0ull, mxx = 0, mny = ~0ull, mxy = 0, ox = 0, oy = 0;
    bool bad = false;
    int64_t tot = n + m;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        double2 p = i < n ? src[i] : tgt[i - n];
        if (!isfinite(p.x) || !isfinite(p.y)) {
            bad = true;
            continue;
        }
        uint64_t kx = order_key(p.x), ky = order_key(p.y);
        mnx = kx < mnx ? kx : mnx;
        mxx = kx > mxx ? kx : mxx;
        mny = ky < mny ? ky : mny;
        mxy = ky > mxy ? ky : mxy;
        if (i < n) {
            ox |= kx ^ rx;
            oy |= ky ^ ry;
        }
    }
    warp_minmax(mnx, mxx, ox);
    warp_minmax(mny, mxy, oy);
    if (bad) atomicOr(status, ST_NONFINITE);
    if ((threadIdx.x & 31) == 0) {
        atomicMin(&acc[0], (unsigned long long)mnx);
        atomicMax(&acc[1], (unsigned long long)mxx);
        atomicMin(&acc[2], (unsigned long long)mny);
        atomicMax(&acc[3], (unsigned long long)mxy);
        atomicOr(&acc[4], (unsigned long long)ox);
        atomicOr(&acc[5], (unsigned long long)oy);
    }
}

__global__ void k_root(const unsigned long long *acc, int64_t n, double4 *rect, int2 *box_src,
                       int *seg_start, int *seg_cnt, double4 *seg_rect) {
    double4 r = make_double4(canon(key_to_double(acc[0])), canon(key_to_double(acc[1])),
                             canon(key_to_double(acc[2])), canon(key_to_double(acc[3])));
    rect[0] = r;
    box_src[0] = make_int2(0, (int)n);
    seg_start[0] = 0;
    seg_cnt[0] = (int)n;
    seg_rect[0] = r;
}

__global__ void k_init_keys(const double2 *__restrict__ src, int64_t n, uint64_t *kx,
                            uint64_t *ky, uint32_t *ix, uint32_t *iy) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 p = src[i];
    kx[i] = order_key(p.x);
    ky[i] = order_key(p.y);
    ix[i] = (uint32_t)i;
    iy[i] = (uint32_t)i;
}

GBI double coord(const double2 *src, uint32_t idx, int axis) {
    double2 p = src[idx];
    return canon(axis ? p.y : p.x);
}

// One thread per segment of round r: axis, median split, child rectangles.
__global__ void k_seg_split(int r, int nseg, const int *__restrict__ s_start,
                            const int *__restrict__ s_cnt, const double4 *__restrict__ s_rect,
                            int *n_start, int *n_cnt, double4 *n_rect, int *s_nl, int8_t *s_axis,
                            const uint32_t *__restrict__ listX, const uint32_t *__restrict__ listY,
                            const double2 *__restrict__ src, double4 *rect, int2 *box_src,
                            int8_t *split_axis, double *split_line) {
    int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= nseg) return;
    int start = s_start[s], n = s_cnt[s];
    double4 rc = s_rect[s];
    double w = __dsub_rn(rc.y, rc.x), h = __dsub_rn(rc.w, rc.z);
    int axis = (w >= h) ? 0 : 1;
    int nl = n / 2;
    const uint32_t *list = axis ? listY : listX;
    double lo = axis ? rc.z : rc.x, hi = axis ? rc.w : rc.y;
    double mid = __dmul_rn(0.5, __dadd_rn(lo, hi));
    double line;
    if (nl > 0) {
        double a = coord(src, list[start + nl - 1], axis);
        double b = coord(src, list[start + nl], axis);
        line = __dmul_rn(0.5, __dadd_rn(a, b));
    } else if (n > 0) {
        double c0 = coord(src, list[start], axis);
        line = (mid <= c0) ? mid : c0;
    } else {
        line = mid;
    }
    double4 left = rc, right = rc;
    if (axis == 0) {
        left.y = line;
        right.x = line;
    } else {
        left.w = line;
        right.z = line;
    }
    n_start[2 * s] = start;
    n_cnt[2 * s] = nl;
    n_rect[2 * s] = left;
    n_start[2 * s + 1] = start + nl;
    n_cnt[2 * s + 1] = n - nl;
    n_rect[2 * s + 1] = right;
    s_nl[s] = nl;
    s_axis[s] = (int8_t)axis;
    int l = r >> 1;
    if ((r & 1) == 0) {
        int64_t g = level_base(l) + s;
        split_axis[3 * g] = (int8_t)axis;
        split_line[3 * g] = line;
    } else {
        int64_t g = level_base(l) + (s >> 1);
        int h1 = s & 1;
        split_axis[3 * g + 1 + h1] = (int8_t)axis;
        split_line[3 * g + 1 + h1] = line;
        int64_t c0 = level_base(l + 1) + 2 * (int64_t)s;
        rect[c0] = left;
        box_src[c0] = make_int2(start, nl);
        rect[c0 + 1] = right;
        box_src[c0 + 1] = make_int2(start + nl, n - nl);
    }
}

// Flag every element left (0) / right (1) from its position in the segment's
// list along the split axis; positions move to segment 2s + side.
__global__ void k_flag(int64_t n, const int *__restrict__ pos_seg, const int *__restrict__ s_start,
                       const int *__restrict__ s_nl, const int8_t *__restrict__ s_axis,
                       const uint32_t *__restrict__ listX, const uint32_t *__restrict__ listY,
                       uint8_t *flag, int *pos_seg_next) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int s = pos_seg[i];
    int side = (int)(i - s_start[s]) >= s_nl[s] ? 1 : 0;
    uint32_t e = s_axis[s] ? listY[i] : listX[i];
    flag[e] = (uint8_t)side;
    pos_seg_next[i] = 2 * s + side;
}

// Stable partition of both lists inside every segment by the flag.
__global__ void k_partition(int64_t n, const int *__restrict__ pos_seg,
                            const int *__restrict__ s_start, const int *__restrict__ s_nl,
                            const uint32_t *__restrict__ listX, const uint32_t *__restrict__ listY,
                            const uint8_t *__restrict__ flag, const uint32_t *__restrict__ GX,
                            const uint32_t *__restrict__ GY, uint32_t *outX, uint32_t *outY) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const uint32_t *list = blockIdx.y ? listY : listX;
    const uint32_t *G = blockIdx.y ? GY : GX;
    uint32_t *out = blockIdx.y ? outY : outX;
    int s = pos_seg[i];
    int start = s_start[s], nl = s_nl[s];
    uint32_t e = list[i];
    int left_before = (int)(G[i] - G[start]);
    int pos;
    if (flag[e] == 0)
        pos = start + left_before;
    else
        pos = start + nl + ((int)(i - start) - left_before);
    out[pos] = e;
}

__global__ void k_final_perm(int64_t n, int L, const int *__restrict__ pos_seg,
                             const int8_t *__restrict__ last_axis, const uint32_t *__restrict__ listX,
                             const uint32_t *__restrict__ listY, uint32_t *perm) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (L == 0) {
        perm[i] = (uint32_t)i;
        return;
    }
    int leaf = pos_seg[i];
    perm[i] = last_axis[leaf >> 1] ? listY[i] : listX[i];
}

__global__ void k_gather2(int64_t n, const uint32_t *__restrict__ perm,
                          const double2 *__restrict__ in, double2 *out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = in[perm[i]];
}

__global__ void k_descend(int64_t m, const double2 *__restrict__ tgt, int L,
                          const int8_t *__restrict__ split_axis, const double *__restrict__ split_line,
                          uint64_t *key, uint32_t *idx) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double2 p = tgt[i];
    double t[2] = {p.x, p.y};
    int64_t b = 0;
    for (int l = 0; l < L; ++l) {
        int64_t g = level_base(l) + b;
        int h1 = t[split_axis[3 * g]] <= split_line[3 * g] ? 0 : 1;
        int h2 = t[split_axis[3 * g + 1 + h1]] <= split_line[3 * g + 1 + h1] ? 0 : 1;
        b = 4 * b + 2 * h1 + h2;
    }
    key[i] = (uint64_t)b;
    idx[i] = (uint32_t)i;
}

GBI int64_t lower_bound_u64(const uint64_t *a, int64_t n, uint64_t v) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < v)
            lo = mid + 1;
        else
            hi = mid;
    }
    return lo;
}

__global__ void k_tgt_ranges(int64_t n_boxes, int L, const uint64_t *__restrict__ keys, int64_t m,
                             int2 *box_tgt) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_boxes) return;
    int l = 0;
    while (level_base(l + 1) <= g) ++l;
    int64_t b = g - level_base(l);
    uint64_t first = (uint64_t)b << (2 * (L - l)), last = (uint64_t)(b + 1) << (2 * (L - l));
    int64_t s = lower_bound_u64(keys, m, first), e = lower_bound_u64(keys, m, last);
    box_tgt[g] = make_int2((int)s, (int)(e - s));
}

// Parent / first-child relations, boxes by level (identity here: the single
// tree is level-major) and the leaf list.
__global__ void k_relations(int64_t n_boxes, int L, int *parent, int *child0, int *lvl_boxes,
                            int *leaves) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_boxes) return;
    int l = 0;
    while (level_base(l + 1) <= g) ++l;
    int64_t b = g - level_base(l);
    parent[g] = l > 0 ? (int)(level_base(l - 1) + b / 4) : -1;
    child0[g] = l < L ? (int)(level_base(l + 1) + 4 * b) : -1;
    lvl_boxes[g] = (int)g;
    if (l == L) leaves[b] = (int)g;
}

__global__ void k_geom(int64_t n_boxes, const double4 *__restrict__ rect, double4 *geom) {
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_boxes) return;
    double4 r4 = rect[g];
    Rect r{r4.x, r4.y, r4.z, r4.w};
    double cx, cy, rad;
    centre_radius(r, cx, cy, rad);
    int e = scale_exponent(rad);
    geom[g] = make_double4(cx, cy, ldexp(1.0, e), ldexp(1.0, -e));
}

// Shrink-wrapped geometry: the bounding rectangle of a leaf's points (its
// sources, and its evaluation points when separate), -0.0 read as +0.0; a leaf
// without points keeps its split rectangle.  One warp per leaf.
__global__ void k_tight_leaf(int64_t nleaf, const int *__restrict__ leaves,
                             const int2 *__restrict__ box_src, const double2 *__restrict__ xs,
                             const int2 *__restrict__ box_tgt, const double2 *__restrict__ xt,
                             int separate, const double4 *__restrict__ rect, double4 *geo) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nleaf) return;
    const int64_t g = leaves[w];
    double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (int pass = 0; pass < (separate ? 2 : 1); ++pass) {
        const int2 r = pass ? box_tgt[g] : box_src[g];
        const double2 *pts = pass ? xt : xs;
        for (int i = lane; i < r.y; i += 32) {
            const double2 p = pts[r.x + i];
            const double x = canon(p.x), y = canon(p.y);
            x0 = fmin(x0, x);
            x1 = fmax(x1, x);
            y0 = fmin(y0, y);
            y1 = fmax(y1, y);
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        x0 = fmin(x0, __shfl_xor_sync(0xffffffffu, x0, d));
        x1 = fmax(x1, __shfl_xor_sync(0xffffffffu, x1, d));
        y0 = fmin(y0, __shfl_xor_sync(0xffffffffu, y0, d));
        y1 = fmax(y1, __shfl_xor_sync(0xffffffffu, y1, d));
    }
    if (lane == 0) geo[g] = (x0 <= x1) ? make_double4(x0, x1, y0, y1) : rect[g];
}

// A parent's bounding rectangle: the union of those of its children that
// hold points (entries of `boxes` without children are skipped).
__global__ void k_tight_union(int64_t n, const int *__restrict__ boxes,
                              const int *__restrict__ child0, const int2 *__restrict__ box_src,
                              const int2 *__restrict__ box_tgt, int separate,
                              const double4 *__restrict__ rect, double4 *geo) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t g = boxes[i], c0 = child0[g];
    if (c0 < 0) return;
    double x0 = INFINITY, x1 = -INFINITY, y0 = INFINITY, y1 = -INFINITY;
    for (int c = 0; c < 4; ++c) {
        const int64_t k = c0 + c;
        if (box_src[k].y + (separate ? box_tgt[k].y : 0) == 0) continue;
        const double4 r = geo[k];
        x0 = fmin(x0, r.x);
        x1 = fmax(x1, r.y);
        y0 = fmin(y0, r.z);
        y1 = fmax(y1, r.w);
    }
    geo[g] = (x0 <= x1) ? make_double4(x0, x1, y0, y1) : rect[g];
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

int64_t tree_level_base(int l) { return level_base(l); }

fmm_status compute_geom(Tree &t, cudaStream_t s) {
    k_geom<<<blocks_for(t.n_boxes, 256), 256, 0, s>>>(t.n_boxes, t.rect_geo, t.geom); note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "geometry");
}

fmm_status build_topology(Tree &t, const double *src_xy, const double *tgt_xy,
                          const int64_t * /*inst_off*/, cudaStream_t s) {
    const double2 *src = reinterpret_cast<const double2 *>(src_xy);
    const double2 *tgt = reinterpret_cast<const double2 *>(tgt_xy);
    const int64_t n = t.n_src, m = t.separate ? t.n_tgt : 0;
    const int L = t.L;
    DevArena tmp;
    tmp.stream = s;
    cudaError_t e;
#define CK(call)                                   \
    do {                                           \
        if ((e = (call)) != cudaSuccess) {         \
            tmp.release();                         \
            return cuda_fail(e, #call);            \
        }                                          \
    } while (0)

    const int64_t nb = level_base(L + 1);
    const int64_t nint = L > 0 ? level_base(L) : 1;
    t.n_boxes = nb;
    for (int l = 0; l <= L + 1; ++l) t.level_start[l] = level_base(l);
    CK(arena_alloc(t.mem, &t.rect, nb));
    CK(arena_alloc(t.mem, &t.box_src, nb));
    CK(arena_alloc(t.mem, &t.geom, nb));
    CK(arena_alloc(t.mem, &t.split_axis, 3 * nint));
    CK(arena_alloc(t.mem, &t.split_line, 3 * nint));
    CK(arena_alloc(t.mem, &t.perm, n));
    CK(arena_alloc(t.mem, &t.xs, n));
    CK(arena_alloc(t.mem, &t.status, 1));
    CK(cudaMemsetAsync(t.status, 0, sizeof(int), s));

    // bounding box of sources and targets, validity, varying key bits
    unsigned long long *acc;
    CK(arena_alloc(tmp, &acc, 6));
    unsigned long long init[6] = {~0ull, 0ull, ~0ull, 0ull, 0ull, 0ull};
    CK(cudaMemcpyAsync(acc, init, sizeof(init), cudaMemcpyHostToDevice, s));
    {
        int64_t tot = n + m;
        unsigned g = (unsigned)std::min<int64_t>(blocks_for(tot, 256), 152 * 8);
        k_bbox<<<g, 256, 0, s>>>(src, n, tgt, m, acc, t.status); note_launch();
        CK(cudaGetLastError());
    }
    unsigned long long hacc[6];
    int hstat = 0;
    CK(cudaMemcpyAsync(hacc, acc, sizeof(hacc), cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(&hstat, t.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    if (hstat & ST_NONFINITE) {
        tmp.release();
        set_error("a coordinate is NaN or infinite");
        return FMM_ERR_NONFINITE;
    }
    uint32_t mask_x = 0, mask_y = 0;
    for (int d = 0; d < 8; ++d) {
        if ((hacc[4] >> (8 * d)) & 0xffull) mask_x |= 1u << d;
        if ((hacc[5] >> (8 * d)) & 0xffull) mask_y |= 1u << d;
    }

    // segment state (double-buffered) sized for the finest level
    const int64_t max_seg = int64_t(1) << (2 * L);
    int *seg_start[2], *seg_cnt[2], *seg_nl;
    double4 *seg_rect[2];
    int8_t *seg_axis;
    for (int k = 0; k < 2; ++k) {
        CK(arena_alloc(tmp, &seg_start[k], max_seg));
        CK(arena_alloc(tmp, &seg_cnt[k], max_seg));
        CK(arena_alloc(tmp, &seg_rect[k], max_seg));
    }
    CK(arena_alloc(tmp, &seg_nl, max_seg));
    CK(arena_alloc(tmp, &seg_axis, max_seg));
    k_root<<<1, 1, 0, s>>>(acc, n, t.rect, t.box_src, seg_start[0], seg_cnt[0], seg_rect[0]); note_launch();
    CK(cudaGetLastError());

    const unsigned gb = blocks_for(n, 256);
    if (L == 0) {
        k_final_perm<<<gb, 256, 0, s>>>(n, 0, nullptr, nullptr, nullptr, nullptr, t.perm); note_launch();
        CK(cudaGetLastError());
    } else {
        uint64_t *kx, *ky, *kalt;
        uint32_t *lx, *ly, *lalt, *lx2, *ly2, *G;
        int *pseg[2];
        uint8_t *flag;
        CK(arena_alloc(tmp, &kx, n));
        CK(arena_alloc(tmp, &ky, n));
        CK(arena_alloc(tmp, &kalt, n));
        CK(arena_alloc(tmp, &lx, n));
        CK(arena_alloc(tmp, &ly, n));
        CK(arena_alloc(tmp, &lalt, n));
        CK(arena_alloc(tmp, &lx2, n));
        CK(arena_alloc(tmp, &ly2, n));
        CK(arena_alloc(tmp, &G, 2 * (n + 1)));
        CK(arena_alloc(tmp, &pseg[0], n));
        CK(arena_alloc(tmp, &pseg[1], n));
        CK(arena_alloc(tmp, &flag, n));
        k_init_keys<<<gb, 256, 0, s>>>(src, n, kx, ky, lx, ly); note_launch();
        CK(cudaGetLastError());
        {
            uint64_t *kx0 = kx;
            uint32_t *lx0 = lx;
            CK(radix_sort_pairs(&kx, &lx, kalt, lalt, n, mask_x, tmp, s));
            // the buffers the x result does not occupy serve the y sort
            uint64_t *kfree = (kx == kx0) ? kalt : kx0;
            uint32_t *lfree = (lx == lx0) ? lalt : lx0;
            CK(radix_sort_pairs(&ky, &ly, kfree, lfree, n, mask_y, tmp, s));
        }
        CK(cudaMemsetAsync(pseg[0], 0, n * sizeof(int), s));
        int cur = 0;
        uint32_t *GX = G, *GY = G + (n + 1);
        for (int r = 0; r < 2 * L; ++r) {
            int nseg = 1 << r;
            k_seg_split<<<blocks_for(nseg, 128), 128, 0, s>>>(
                r, nseg, seg_start[cur], seg_cnt[cur], seg_rect[cur], seg_start[cur ^ 1],
                seg_cnt[cur ^ 1], seg_rect[cur ^ 1], seg_nl, seg_axis, lx, ly, src, t.rect,
                t.box_src, t.split_axis, t.split_line); note_launch();
            CK(cudaGetLastError());
            k_flag<<<gb, 256, 0, s>>>(n, pseg[cur], seg_start[cur], seg_nl, seg_axis, lx, ly,
                                      flag, pseg[cur ^ 1]); note_launch();
            CK(cudaGetLastError());
            CK(dual_left_scan(lx, ly, flag, n, GX, GY, tmp, s));
            k_partition<<<dim3(gb, 2), 256, 0, s>>>(n, pseg[cur], seg_start[cur], seg_nl, lx, ly,
                                                    flag, GX, GY, lx2, ly2); note_launch();
            CK(cudaGetLastError());
            std::swap(lx, lx2);
            std::swap(ly, ly2);
            cur ^= 1;
        }
        // pseg[cur] holds the leaf of every position; seg_axis the last round's axes
        k_final_perm<<<gb, 256, 0, s>>>(n, L, pseg[cur], seg_axis, lx, ly, t.perm); note_launch();
        CK(cudaGetLastError());
    }
    k_gather2<<<gb, 256, 0, s>>>(n, t.perm, src, t.xs); note_launch();
    CK(cudaGetLastError());

    if (t.separate) {
        CK(arena_alloc(t.mem, &t.tperm, m));
        CK(arena_alloc(t.mem, &t.xt, m));
        CK(arena_alloc(t.mem, &t.box_tgt, nb));
        uint64_t *key, *kalt;
        uint32_t *idx, *ialt;
        CK(arena_alloc(tmp, &key, m));
        CK(arena_alloc(tmp, &kalt, m));
        CK(arena_alloc(tmp, &idx, m));
        CK(arena_alloc(tmp, &ialt, m));
        if (m > 0) {
            k_descend<<<blocks_for(m, 256), 256, 0, s>>>(m, tgt, L, t.split_axis, t.split_line,
                                                         key, idx); note_launch();
            CK(cudaGetLastError());
            CK(radix_sort_pairs(&key, &idx, kalt, ialt, m, digits_for_bits(2 * L), tmp, s));
            CK(cudaMemcpyAsync(t.tperm, idx, m * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
            k_gather2<<<blocks_for(m, 256), 256, 0, s>>>(m, t.tperm, tgt, t.xt); note_launch();
            CK(cudaGetLastError());
        }
        k_tgt_ranges<<<blocks_for(nb, 256), 256, 0, s>>>(nb, L, key, m, t.box_tgt); note_launch();
        CK(cudaGetLastError());
    } else {
        t.tperm = t.perm;
        t.xt = t.xs;
        t.box_tgt = t.box_src;
    }
    t.n_leaves = (int)(int64_t(1) << (2 * L));
    CK(arena_alloc(t.mem, &t.parent, nb));
    CK(arena_alloc(t.mem, &t.child0, nb));
    CK(arena_alloc(t.mem, &t.lvl_boxes, nb));
    CK(arena_alloc(t.mem, &t.leaves, t.n_leaves));
    k_relations<<<blocks_for(nb, 256), 256, 0, s>>>(nb, L, t.parent, t.child0, t.lvl_boxes,
                                                    t.leaves); note_launch();
    CK(cudaGetLastError());
    // box geometry: the split rectangles, or the points' bounding rectangles
    if (t.box_fit) {
        CK(arena_alloc(t.mem, &t.rect_geo, nb));
        k_tight_leaf<<<blocks_for((int64_t)t.n_leaves * 32, 128), 128, 0, s>>>(
            t.n_leaves, t.leaves, t.box_src, t.xs, t.box_tgt, t.xt, t.separate ? 1 : 0, t.rect,
            t.rect_geo); note_launch();
        CK(cudaGetLastError());
        for (int l = L - 1; l >= 0; --l) {
            const int64_t nl = level_base(l + 1) - level_base(l);
            k_tight_union<<<blocks_for(nl, 128), 128, 0, s>>>(
                nl, t.lvl_boxes + level_base(l), t.child0, t.box_src, t.box_tgt,
                t.separate ? 1 : 0, t.rect, t.rect_geo); note_launch();
            CK(cudaGetLastError());
        }
    } else {
        t.rect_geo = t.rect;
    }
    k_geom<<<blocks_for(nb, 256), 256, 0, s>>>(nb, t.rect_geo, t.geom); note_launch();
    CK(cudaGetLastError());
    // temporaries are stream-ordered: freeing them here is safe
    tmp.release();
#undef CK
    return FMM_OK;
}

}  // namespace gbfmm
