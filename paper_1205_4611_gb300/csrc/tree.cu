// Topological phase, part 1 (Sec. 3.2, "sorting"): the median-split pyramid
// tree.  Every box is split twice per level, along the longer side of its
// rectangle, at the median of its sources ordered by (coordinate, index)
// (Sec. 2; Alg. "Partitioning with successive splits" is the paper's GPU
// design, replaced here by an exact deterministic scheme):
//
//   1. both coordinates are presorted once (stable LSD radix sort of
//      order-preserving 64-bit keys, ties by index);
//   2. every source becomes an entry (x rank, y rank); each split round
//      keeps one x-ordered and one y-ordered entry list per box segment; the
//      median is the middle of the segment's list along the split axis, and
//      both lists are stably partitioned by comparing each entry's rank on
//      that axis with the median's (rounds over long segments run over the
//      whole array, the last rounds of every short segment in shared memory);
//   3. within a leaf, sources are left in the order of the leaf's last split
//      axis, which is the order a per-box sort produces.
//
// Evaluation points descend the split lines (<= line goes left) and are
// grouped by leaf with a stable radix sort (original order inside a leaf).
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <utility>

#include "common.cuh"
#include "internal.h"

namespace gbfmm {

namespace {

GBI double canon(double x) { return __dadd_rn(x, 0.0); }

// Box ids are level-major over R roots (R trees with the same number of
// levels, built together): level l holds boxes [R lb(l), R lb(l+1)) with
// lb(l) = (4^l - 1)/3, and box B of level l (counted from R lb(l)) has
// children 4B .. 4B+3; root r owns boxes r 4^l .. (r+1) 4^l - 1 of level l.
// R = 1 is a single tree.
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

constexpr int BB_THREADS = 256;

// acc[0..3] = min x, max x, min y, max y (order keys); acc[4], acc[5] = OR over
// sources of (key ^ key of source 0) for x and y: the key bits that vary.
// Reduced per warp, then per block in shared memory, then one set of atomics
// per block.
__global__ void __launch_bounds__(BB_THREADS)
    k_bbox(const double2 *__restrict__ src, int64_t n, const double2 *__restrict__ tgt, int64_t m,
           unsigned long long *acc, int *status) {
    pdl_wait();
    __shared__ uint64_t red[6][BB_THREADS / 32];
    __shared__ int sbad;
    if (threadIdx.x == 0) sbad = 0;
    uint64_t rx = order_key(src[0].x), ry = order_key(src[0].y);
    uint64_t mnx = ~0ull, mxx = 0, mny = ~0ull, mxy = 0, ox = 0, oy = 0;
    bool bad = false;
    int64_t tot = n + m;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < tot;
         i += (int64_t)gridDim.x * blockDim.x) {
        double2 p = i < n ? src[i] : tgt[i - n];
        uint64_t kx = order_key(p.x), ky = order_key(p.y);
        // NaN or infinity: exponent bits all ones
        if (((__double_as_longlong(p.x) >> 52) & 0x7ff) == 0x7ff ||
            ((__double_as_longlong(p.y) >> 52) & 0x7ff) == 0x7ff) {
            bad = true;
            continue;
        }
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
    __syncthreads();
    if (bad) sbad = 1;
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = mnx;
        red[1][w] = mxx;
        red[2][w] = mny;
        red[3][w] = mxy;
        red[4][w] = ox;
        red[5][w] = oy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < BB_THREADS / 32; ++k) {
            mnx = red[0][k] < mnx ? red[0][k] : mnx;
            mxx = red[1][k] > mxx ? red[1][k] : mxx;
            mny = red[2][k] < mny ? red[2][k] : mny;
            mxy = red[3][k] > mxy ? red[3][k] : mxy;
            ox |= red[4][k];
            oy |= red[5][k];
        }
        atomicMin(&acc[0], (unsigned long long)mnx);
        atomicMax(&acc[1], (unsigned long long)mxx);
        atomicMin(&acc[2], (unsigned long long)mny);
        atomicMax(&acc[3], (unsigned long long)mxy);
        atomicOr(&acc[4], (unsigned long long)ox);
        atomicOr(&acc[5], (unsigned long long)oy);
        if (sbad) atomicOr(status, ST_NONFINITE);
    }
}

// R > 1 roots: block r reduces root r's sources [soff[r], soff[r+1]) and
// evaluation points [toff[r], toff[r+1]) (toff NULL: none) into acc[6 r ..
// 6 r + 3] (min x, max x, min y, max y as order keys); the key bits that vary
// inside any root (each root's keys against its first source) are OR-ed into
// acc[6 R], acc[6 R + 1].
__global__ void __launch_bounds__(BB_THREADS)
    k_bbox_roots(int R, const double2 *__restrict__ src, const int64_t *__restrict__ soff,
                 const double2 *__restrict__ tgt, const int64_t *__restrict__ toff,
                 unsigned long long *acc, int *status) {
    pdl_wait();
    __shared__ uint64_t red[6][BB_THREADS / 32];
    __shared__ int sbad;
    const int r = blockIdx.x;
    if (threadIdx.x == 0) sbad = 0;
    const int64_t s0 = soff[r], s1 = soff[r + 1];
    const int64_t t0 = toff ? toff[r] : 0, t1 = toff ? toff[r + 1] : 0;
    const int64_t ns = s1 - s0, tot = ns + (t1 - t0);
    const uint64_t rx = order_key(src[s0].x), ry = order_key(src[s0].y);
    uint64_t mnx = ~0ull, mxx = 0, mny = ~0ull, mxy = 0, ox = 0, oy = 0;
    bool bad = false;
    for (int64_t i = threadIdx.x; i < tot; i += BB_THREADS) {
        double2 p = i < ns ? src[s0 + i] : tgt[t0 + i - ns];
        if (((__double_as_longlong(p.x) >> 52) & 0x7ff) == 0x7ff ||
            ((__double_as_longlong(p.y) >> 52) & 0x7ff) == 0x7ff) {
            bad = true;
            continue;
        }
        uint64_t kx = order_key(p.x), ky = order_key(p.y);
        mnx = kx < mnx ? kx : mnx;
        mxx = kx > mxx ? kx : mxx;
        mny = ky < mny ? ky : mny;
        mxy = ky > mxy ? ky : mxy;
        if (i < ns) {
            ox |= kx ^ rx;
            oy |= ky ^ ry;
        }
    }
    warp_minmax(mnx, mxx, ox);
    warp_minmax(mny, mxy, oy);
    __syncthreads();
    if (bad) sbad = 1;
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        red[0][w] = mnx;
        red[1][w] = mxx;
        red[2][w] = mny;
        red[3][w] = mxy;
        red[4][w] = ox;
        red[5][w] = oy;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < BB_THREADS / 32; ++k) {
            mnx = red[0][k] < mnx ? red[0][k] : mnx;
            mxx = red[1][k] > mxx ? red[1][k] : mxx;
            mny = red[2][k] < mny ? red[2][k] : mny;
            mxy = red[3][k] > mxy ? red[3][k] : mxy;
            ox |= red[4][k];
            oy |= red[5][k];
        }
        acc[6 * r + 0] = mnx;
        acc[6 * r + 1] = mxx;
        acc[6 * r + 2] = mny;
        acc[6 * r + 3] = mxy;
        atomicOr(&acc[6 * R], (unsigned long long)ox);
        atomicOr(&acc[6 * R + 1], (unsigned long long)oy);
        if (sbad) atomicOr(status, ST_NONFINITE);
    }
}

// The R roots: rectangle (the bounding box of its points), sources, and the
// round-0 segment of each.
__global__ void k_roots(int R, const unsigned long long *acc, const int64_t *__restrict__ soff,
                        double4 *rect, int2 *box_src, int *seg_start, int *seg_cnt,
                        double4 *seg_rect) {
    pdl_wait();
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= R) return;
    const unsigned long long *a = acc + 6 * r;
    double4 rc = make_double4(canon(key_to_double(a[0])), canon(key_to_double(a[1])),
                              canon(key_to_double(a[2])), canon(key_to_double(a[3])));
    const int st = (int)soff[r], n = (int)(soff[r + 1] - soff[r]);
    rect[r] = rc;
    box_src[r] = make_int2(st, n);
    seg_start[r] = st;
    seg_cnt[r] = n;
    seg_rect[r] = rc;
}

// The root of every position (positions of root r: [off[r], off[r+1])).
__global__ void k_root_of(int64_t n, int R, const int64_t *__restrict__ off, int *out) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int lo = 0, hi = R;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (off[mid] <= i)
            lo = mid;
        else
            hi = mid;
    }
    out[i] = lo;
}

// Keys of a second, stable sort that groups the presorted lists by root:
// key = root of the source at each position.
__global__ void k_root_keys(int64_t n, const int *__restrict__ root, const uint32_t *__restrict__ lx,
                            const uint32_t *__restrict__ ly, uint64_t *kx, uint64_t *ky) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    kx[i] = (uint64_t)root[lx[i]];
    ky[i] = (uint64_t)root[ly[i]];
}

__global__ void k_bbox_init(unsigned long long *acc) {
    pdl_wait();
    if (threadIdx.x < 6) acc[threadIdx.x] = (threadIdx.x == 0 || threadIdx.x == 2) ? ~0ull : 0ull;
}

__global__ void k_root(const unsigned long long *acc, int64_t n, double4 *rect, int2 *box_src,
                       int *seg_start, int *seg_cnt, double4 *seg_rect) {
    pdl_wait();
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
    pdl_wait();
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

// ------------------------------------------------------------ split rounds
//
// Every source is carried as an entry (rank in the x order, rank in the y
// order); ranks are unique, so they compare like (coordinate, index).  A box
// segment keeps its entries in two lists, one sorted by each rank.  Splitting
// along an axis at the median sends an entry left iff its rank along that axis
// is below the median entry's rank: the list along the split axis is already
// partitioned, the other one is partitioned stably, and both by the same test,
// with no per-source flag array.  Early rounds (segments longer than
// LOC_CAP) run over the whole array (count, then scan + scatter); the
// remaining rounds of each segment run in one block in shared memory.

constexpr int PT_THREADS = 256;
constexpr int PT_ITEMS = 8;
constexpr int PT_TILE = PT_THREADS * PT_ITEMS;
constexpr int PT_DIRECT_TILES = 1024;  // up to this many tiles a block sums its prefix itself
constexpr int LOC_CAP = 2048;          // entries of a segment split in shared memory
constexpr int LOC_THREADS = 256;
constexpr int LOC_ITEMS = LOC_CAP / LOC_THREADS;
constexpr int SEG_THREADS = 1024;
constexpr int LOC_MAX_ROUNDS = 12;     // sub-segments per block at most 2^(LOC_MAX_ROUNDS - 1)
constexpr size_t LOC_SMEM = 4 * LOC_CAP * sizeof(uint2) + 2 * LOC_CAP * sizeof(int) +
                            2 * (LOC_CAP + 8) * sizeof(uint16_t);

GBI uint32_t rank_on(uint2 e, int axis) { return axis ? e.y : e.x; }


// The split of one segment (Sec. 2: longer side, median of the sources in
// (coordinate, index) order, line halfway between the two middle sources).
// ex/ey hold the segment's entries at [start, start + n) (global or shared).
struct SegOut {
    int axis, nl;
    uint32_t rmed;
    double line;
    double4 left, right;
};

GBI SegOut split_segment(int start, int n, double4 rc, const uint2 *ex, const uint2 *ey,
                         const uint32_t *__restrict__ lx, const uint32_t *__restrict__ ly,
                         const double2 *__restrict__ src) {
    SegOut o;
    const double w = __dsub_rn(rc.y, rc.x), h = __dsub_rn(rc.w, rc.z);
    o.axis = (w >= h) ? 0 : 1;
    o.nl = n / 2;
    const uint2 *el = o.axis ? ey : ex;
    const uint32_t *sorted = o.axis ? ly : lx;
    const double lo = o.axis ? rc.z : rc.x, hi = o.axis ? rc.w : rc.y;
    const double mid = __dmul_rn(0.5, __dadd_rn(lo, hi));
    o.rmed = n > 0 ? rank_on(el[start + o.nl], o.axis) : 0u;
    if (o.nl > 0) {
        const double a = coord(src, sorted[rank_on(el[start + o.nl - 1], o.axis)], o.axis);
        const double b = coord(src, sorted[o.rmed], o.axis);
        o.line = __dmul_rn(0.5, __dadd_rn(a, b));
    } else if (n > 0) {
        const double c0 = coord(src, sorted[o.rmed], o.axis);
        o.line = (mid <= c0) ? mid : c0;
    } else {
        o.line = mid;
    }
    o.left = rc;
    o.right = rc;
    if (o.axis == 0) {
        o.left.y = o.line;
        o.right.x = o.line;
    } else {
        o.left.w = o.line;
        o.right.z = o.line;
    }
    return o;
}

// The tree arrays of one split: round r splits segment s (global id over the
// R roots: segment s of round r belongs to root s >> r).
GBI void record_split(int r, int R, int64_t s, int start, int n, const SegOut &o, double4 *rect,
                      int2 *box_src, int8_t *split_axis, double *split_line) {
    const int l = r >> 1;
    if ((r & 1) == 0) {
        const int64_t g = R * level_base(l) + s;
        split_axis[3 * g] = (int8_t)o.axis;
        split_line[3 * g] = o.line;
    } else {
        const int64_t g = R * level_base(l) + (s >> 1);
        const int h1 = (int)(s & 1);
        split_axis[3 * g + 1 + h1] = (int8_t)o.axis;
        split_line[3 * g + 1 + h1] = o.line;
        const int64_t c0 = R * level_base(l + 1) + 2 * s;
        rect[c0] = o.left;
        box_src[c0] = make_int2(start, o.nl);
        rect[c0 + 1] = o.right;
        box_src[c0 + 1] = make_int2(start + o.nl, n - o.nl);
    }
}

// info of a segment in a global round: start, left count, left entries of all
// earlier segments, median rank | axis << 31
GBI int4 pack_info(int start, int nl, uint32_t G, uint32_t rmed, int axis) {
    return make_int4(start, nl, (int)G, (int)(rmed | ((uint32_t)axis << 31)));
}
GBI int info_axis(int4 f) { return (int)((uint32_t)f.w >> 31); }
GBI uint32_t info_rmed(int4 f) { return (uint32_t)f.w & 0x7fffffffu; }

// Global round r: one block splits every segment (in chunks of SEG_THREADS,
// carrying the running count of left entries).
__global__ void __launch_bounds__(SEG_THREADS)
    k_seg_split(int r, int R, int nseg, const int *__restrict__ s_start, const int *__restrict__ s_cnt,
                const double4 *__restrict__ s_rect, int *n_start, int *n_cnt, double4 *n_rect,
                int4 *info, const uint2 *__restrict__ ex, const uint2 *__restrict__ ey,
                const uint32_t *__restrict__ lx, const uint32_t *__restrict__ ly,
                const double2 *__restrict__ src, double4 *rect, int2 *box_src,
                int8_t *split_axis, double *split_line) {
    pdl_wait();
    __shared__ uint32_t wt[SEG_THREADS / 32];
    uint32_t carry = 0;
    for (int base = 0; base < nseg; base += SEG_THREADS) {
        const int s = base + threadIdx.x;
        SegOut o{};
        int start = 0, n = 0;
        if (s < nseg) {
            start = s_start[s];
            n = s_cnt[s];
            o = split_segment(start, n, s_rect[s], ex, ey, lx, ly, src);
        }
        uint32_t excl;
        const uint32_t tot = block_scan_excl<SEG_THREADS>(s < nseg ? (uint32_t)o.nl : 0u, excl, wt);
        if (s < nseg) {
            info[s] = pack_info(start, o.nl, carry + excl, o.rmed, o.axis);
            n_start[2 * s] = start;
            n_cnt[2 * s] = o.nl;
            n_rect[2 * s] = o.left;
            n_start[2 * s + 1] = start + o.nl;
            n_cnt[2 * s + 1] = n - o.nl;
            n_rect[2 * s + 1] = o.right;
            record_split(r, R, s, start, n, o, rect, box_src, split_axis, split_line);
        }
        carry += tot;
    }
}

// Left entries per tile of both lists (blockIdx.y selects the list).
__global__ void __launch_bounds__(PT_THREADS)
    k_pcount(int64_t n, const int *__restrict__ pos_seg, const int4 *__restrict__ info,
             const uint2 *__restrict__ ex, const uint2 *__restrict__ ey, uint32_t *sums,
             int ntiles) {
    pdl_wait();
    __shared__ uint32_t wt[PT_THREADS / 32];
    const uint2 *el = blockIdx.y ? ey : ex;
    const int64_t base = (int64_t)blockIdx.x * PT_TILE;
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < PT_ITEMS; ++j) {
        const int64_t i = base + j * PT_THREADS + threadIdx.x;
        if (i < n) {
            const int4 f = info[pos_seg[i]];
            c += rank_on(el[i], info_axis(f)) < info_rmed(f) ? 1u : 0u;
        }
    }
    uint32_t excl;
    const uint32_t tot = block_scan_excl<PT_THREADS>(c, excl, wt);
    if (threadIdx.x == 0) sums[(int64_t)blockIdx.y * ntiles + blockIdx.x] = tot;
}

// Exclusive prefix of the tile counts of both lists, in place (one block).
__global__ void __launch_bounds__(SEG_THREADS) k_tile_scan(uint32_t *sums, int ntiles) {
    pdl_wait();
    __shared__ uint32_t wt[SEG_THREADS / 32];
    for (int list = 0; list < 2; ++list) {
        uint32_t *a = sums + (int64_t)list * ntiles;
        uint32_t carry = 0;
        for (int base = 0; base < ntiles; base += SEG_THREADS) {
            const int k = base + threadIdx.x;
            const uint32_t v = k < ntiles ? a[k] : 0u;
            uint32_t excl;
            const uint32_t tot = block_scan_excl<SEG_THREADS>(v, excl, wt);
            if (k < ntiles) a[k] = carry + excl;
            carry += tot;
        }
    }
}

// Stable partition of both lists inside every segment; list 0's blocks also
// write the segment of every position for the next round.  The tile's entries
// are staged in shared memory in (left ones, right ones) order with their
// destinations, so that consecutive threads store consecutive positions.
__global__ void __launch_bounds__(PT_THREADS)
    k_part(int64_t n, const int *__restrict__ pos_seg, const int4 *__restrict__ info,
           const uint2 *__restrict__ ex, const uint2 *__restrict__ ey, uint2 *ox, uint2 *oy,
           const uint32_t *__restrict__ sums, int ntiles, int *pos_seg_next) {
    pdl_wait();
    __shared__ uint32_t wt[PT_THREADS / 32];
    __shared__ uint2 sE[PT_TILE];
    __shared__ int sP[PT_TILE];
    const uint2 *el = blockIdx.y ? ey : ex;
    uint2 *out = blockIdx.y ? oy : ox;
    const uint32_t *ts = sums + (int64_t)blockIdx.y * ntiles;
    const int64_t tile0 = (int64_t)blockIdx.x * PT_TILE;
    const int64_t i0 = tile0 + threadIdx.x * PT_ITEMS;
    // the tile's entries and segments first (independent loads in flight)
    uint2 e[PT_ITEMS];
    int sg[PT_ITEMS];
#pragma unroll
    for (int j = 0; j < PT_ITEMS; ++j) {
        const int64_t i = i0 + j;
        e[j] = i < n ? el[i] : make_uint2(0u, 0u);
        sg[j] = i < n ? pos_seg[i] : 0;
    }
    uint32_t part = 0;
    if (ntiles <= PT_DIRECT_TILES)
        for (int k = threadIdx.x; k < (int)blockIdx.x; k += PT_THREADS) part += ts[k];
    bool left[PT_ITEMS];
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < PT_ITEMS; ++j) {
        const int4 f = info[sg[j]];
        left[j] = i0 + j < n && rank_on(e[j], info_axis(f)) < info_rmed(f);
        c += left[j] ? 1u : 0u;
    }
    uint32_t prefix;
    if (ntiles <= PT_DIRECT_TILES) {
        uint32_t dummy;
        prefix = block_scan_excl<PT_THREADS>(part, dummy, wt);
    } else {
        prefix = ts[blockIdx.x];  // already scanned by k_tile_scan
    }
    uint32_t excl;
    const uint32_t nleft = block_scan_excl<PT_THREADS>(c, excl, wt);
    uint32_t run = excl;  // left entries of the tile before i0
#pragma unroll
    for (int j = 0; j < PT_ITEMS; ++j) {
        const int64_t i = i0 + j;
        if (i < n) {
            const int4 f = info[sg[j]];
            const int st = f.x, nl = f.y;
            const int lb = (int)(prefix + run - (uint32_t)f.z);  // left entries in [st, i)
            const int pos = left[j] ? st + lb : st + nl + ((int)(i - st) - lb);
            const int tl = (int)(i - tile0);
            const int lp = left[j] ? (int)run : (int)nleft + (tl - (int)run);
            sE[lp] = e[j];
            sP[lp] = pos;
            if (blockIdx.y == 0) pos_seg_next[i] = 2 * sg[j] + ((int)(i - st) >= nl ? 1 : 0);
            run += left[j] ? 1u : 0u;
        }
    }
    __syncthreads();
    const int nt = (n - tile0 < PT_TILE) ? (int)(n - tile0) : PT_TILE;
    for (int lp = threadIdx.x; lp < nt; lp += PT_THREADS) out[sP[lp]] = sE[lp];
}

// The remaining rounds r0 .. 2L-1 of one segment of round r0 (<= LOC_CAP
// entries) in shared memory.  Block b reads its segment from the round-r0
// arrays (id b) and keeps its sub-segments' starts, counts, rectangles and
// split info in its own region [b 2^(2L-r0), (b+1) 2^(2L-r0)) of two other
// segment-array buffers (alternating by round), so blocks at different rounds
// never touch each other's entries.  Ends by writing the leaf order: within a
// leaf, sources follow the list of its last split axis.
__global__ void __launch_bounds__(LOC_THREADS)
    k_tree_local(int r0, int L, int R, const int *__restrict__ in_start, const int *__restrict__ in_cnt,
                 const double4 *__restrict__ in_rect, int *a_start, int *a_cnt, double4 *a_rect,
                 int *b_start, int *b_cnt, double4 *b_rect, int4 *info,
                 const uint2 *__restrict__ ex, const uint2 *__restrict__ ey,
                 const uint32_t *__restrict__ lx, const uint32_t *__restrict__ ly,
                 const double2 *__restrict__ src, double4 *rect, int2 *box_src,
                 int8_t *split_axis, double *split_line, uint32_t *perm) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char lsm[];
    uint2 *const Ebase = reinterpret_cast<uint2 *>(lsm);  // [buffer][list][LOC_CAP]
    int *const pbase = reinterpret_cast<int *>(Ebase + 4 * LOC_CAP);  // [buffer][LOC_CAP]
    uint16_t *const scan0 = reinterpret_cast<uint16_t *>(pbase + 2 * LOC_CAP);  // [list][LOC_CAP + 8]
    __shared__ uint32_t wt[LOC_THREADS / 32];
#define LOC_E(buf, list) (Ebase + ((buf) * 2 + (list)) * LOC_CAP)
#define LOC_P(buf) (pbase + (buf) * LOC_CAP)
#define LOC_S(list) (scan0 + (list) * (LOC_CAP + 8))

    const int64_t b = blockIdx.x;
    const int64_t rb = b << (2 * L - r0);  // this block's region of the segment arrays
    const int gstart = in_start[b], nb = min(in_cnt[b], LOC_CAP);
    for (int j = threadIdx.x; j < nb; j += LOC_THREADS) {
        LOC_E(0, 0)[j] = ex[gstart + j];
        LOC_E(0, 1)[j] = ey[gstart + j];
        LOC_P(0)[j] = 0;
    }
    __syncthreads();
    int cb = 0;  // entry buffer of the current round
    for (int r = r0; r < 2 * L; ++r) {
        const int nsub = 1 << (r - r0);
        const int64_t g0 = b * nsub;  // tree id of the first sub-segment of this round
        const bool odd = ((r - r0) & 1) != 0;
        // this round's table: the input (first round), then a, b, a, ...
        const int *cs = r == r0 ? in_start + b : (odd ? a_start : b_start) + rb;
        const int *cc = r == r0 ? in_cnt + b : (odd ? a_cnt : b_cnt) + rb;
        const double4 *cr = r == r0 ? in_rect + b : (odd ? a_rect : b_rect) + rb;
        int *ns = (odd ? b_start : a_start) + rb;
        int *nc = (odd ? b_cnt : a_cnt) + rb;
        double4 *nr = (odd ? b_rect : a_rect) + rb;
        int4 *inf = info + rb;
        const uint2 *Ex = LOC_E(cb, 0), *Ey = LOC_E(cb, 1);
        const int *ps = LOC_P(cb);
        for (int t = threadIdx.x; t < nsub; t += LOC_THREADS) {
            const int start = cs[t], n = cc[t];
            const SegOut o = split_segment(start - gstart, n, cr[t], Ex, Ey, lx, ly, src);
            inf[t] = pack_info(start - gstart, o.nl, 0u, o.rmed, o.axis);
            ns[2 * t] = start;
            nc[2 * t] = o.nl;
            nr[2 * t] = o.left;
            ns[2 * t + 1] = start + o.nl;
            nc[2 * t + 1] = n - o.nl;
            nr[2 * t + 1] = o.right;
            record_split(r, R, g0 + t, start, n, o, rect, box_src, split_axis, split_line);
        }
        __syncthreads();
        // left flags and their block-wide exclusive scan, both lists
        const int j0 = threadIdx.x * LOC_ITEMS;
        for (int list = 0; list < 2; ++list) {
            const uint2 *El = list ? Ey : Ex;
            uint16_t *sl = LOC_S(list);
            uint32_t c = 0;
#pragma unroll
            for (int k = 0; k < LOC_ITEMS; ++k) {
                const int j = j0 + k;
                if (j < nb) {
                    const int4 f = inf[ps[j]];
                    c += rank_on(El[j], info_axis(f)) < info_rmed(f) ? 1u : 0u;
                }
            }
            uint32_t excl;
            block_scan_excl<LOC_THREADS>(c, excl, wt);
#pragma unroll
            for (int k = 0; k < LOC_ITEMS; ++k) {
                const int j = j0 + k;
                if (j < nb) {
                    sl[j] = (uint16_t)excl;
                    const int4 f = inf[ps[j]];
                    excl += rank_on(El[j], info_axis(f)) < info_rmed(f) ? 1u : 0u;
                }
            }
        }
        __syncthreads();
        // stable partition of every sub-segment, both lists
        for (int list = 0; list < 2; ++list) {
            const uint2 *El = list ? Ey : Ex;
            uint2 *On = LOC_E(cb ^ 1, list);
            const uint16_t *sl = LOC_S(list);
            for (int j = threadIdx.x; j < nb; j += LOC_THREADS) {
                const int sub = ps[j];
                const int4 f = inf[sub];
                const int st = f.x, nl = f.y;
                const uint2 e = El[j];
                const bool lft = rank_on(e, info_axis(f)) < info_rmed(f);
                const int lb = (int)sl[j] - (int)sl[st];
                const int pos = lft ? st + lb : st + nl + (j - st - lb);
                On[pos] = e;
                if (list == 0) LOC_P(cb ^ 1)[j] = 2 * sub + (j - st >= nl ? 1 : 0);
            }
        }
        __syncthreads();
        if (r == 2 * L - 1) {
            // leaf order: the list of the last split axis of each leaf
            for (int j = threadIdx.x; j < nb; j += LOC_THREADS) {
                const int ax = info_axis(inf[ps[j]]);
                const uint2 e = LOC_E(cb ^ 1, ax)[j];
                perm[gstart + j] = ax ? ly[e.y] : lx[e.x];
            }
        }
        cb ^= 1;
    }
#undef LOC_E
#undef LOC_P
#undef LOC_S
}

// Rank of every source in each presorted order, then the entry lists.
__global__ void k_ranks(int64_t n, const uint32_t *__restrict__ lx, const uint32_t *__restrict__ ly,
                        uint32_t *rx, uint32_t *ry) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    rx[lx[i]] = (uint32_t)i;
    ry[ly[i]] = (uint32_t)i;
}

__global__ void k_entries(int64_t n, const uint32_t *__restrict__ lx,
                          const uint32_t *__restrict__ ly, const uint32_t *__restrict__ rx,
                          const uint32_t *__restrict__ ry, uint2 *ex, uint2 *ey) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    ex[i] = make_uint2((uint32_t)i, ry[lx[i]]);
    ey[i] = make_uint2(rx[ly[i]], (uint32_t)i);
}

// Leaf order when the leaves are longer than LOC_CAP (all rounds global).
__global__ void k_final_perm(int64_t n, int L, const int *__restrict__ pos_seg,
                             const int4 *__restrict__ info, const uint2 *__restrict__ ex,
                             const uint2 *__restrict__ ey, const uint32_t *__restrict__ lx,
                             const uint32_t *__restrict__ ly, uint32_t *perm) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (L == 0) {
        perm[i] = (uint32_t)i;
        return;
    }
    const int ax = info_axis(info[pos_seg[i] >> 1]);
    perm[i] = ax ? ly[ey[i].y] : lx[ex[i].x];
}

__global__ void k_gather2(int64_t n, const uint32_t *__restrict__ perm,
                          const double2 *__restrict__ in, double2 *out) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = in[perm[i]];
}

// The leaf of every evaluation point: down its root's split lines (<= line
// goes left); the key is the leaf's index over all roots' leaves.
__global__ void k_descend(int64_t m, const double2 *__restrict__ tgt, int L, int R,
                          const int64_t *__restrict__ toff,
                          const int8_t *__restrict__ split_axis, const double *__restrict__ split_line,
                          uint64_t *key, uint32_t *idx) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    double2 p = tgt[i];
    double t[2] = {p.x, p.y};
    int64_t b = 0;
    if (R > 1) {  // the root of point i: the last r with toff[r] <= i
        int lo = 0, hi = R;
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (toff[mid] <= i)
                lo = mid;
            else
                hi = mid;
        }
        b = lo;
    }
    for (int l = 0; l < L; ++l) {
        int64_t g = R * level_base(l) + b;
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

__global__ void k_tgt_ranges(int64_t n_boxes, int L, int R, const uint64_t *__restrict__ keys,
                             int64_t m, int2 *box_tgt) {
    pdl_wait();
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_boxes) return;
    int l = 0;
    while (R * level_base(l + 1) <= g) ++l;
    int64_t b = g - R * level_base(l);
    uint64_t first = (uint64_t)b << (2 * (L - l)), last = (uint64_t)(b + 1) << (2 * (L - l));
    int64_t s = lower_bound_u64(keys, m, first), e = lower_bound_u64(keys, m, last);
    box_tgt[g] = make_int2((int)s, (int)(e - s));
}

// Parent / first-child relations, boxes by level (identity here: the boxes
// are level-major) and the leaf list.
__global__ void k_relations(int64_t n_boxes, int L, int R, int *parent, int *child0,
                            int *lvl_boxes, int *leaves) {
    pdl_wait();
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= n_boxes) return;
    int l = 0;
    while (R * level_base(l + 1) <= g) ++l;
    int64_t b = g - R * level_base(l);
    parent[g] = l > 0 ? (int)(R * level_base(l - 1) + b / 4) : -1;
    child0[g] = l < L ? (int)(R * level_base(l + 1) + 4 * b) : -1;
    lvl_boxes[g] = (int)g;
    if (l == L) leaves[b] = (int)g;
}

__global__ void k_geom(int64_t n_boxes, const double4 *__restrict__ rect, double4 *geom) {
    pdl_wait();
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
// without points keeps its split rectangle.  One warp per leaf; minima and
// maxima are taken on the order keys (integer operations).
__global__ void k_tight_leaf(int64_t nleaf, const int *__restrict__ leaves,
                             const int2 *__restrict__ box_src, const double2 *__restrict__ xs,
                             const int2 *__restrict__ box_tgt, const double2 *__restrict__ xt,
                             int separate, const double4 *__restrict__ rect, double4 *geo) {
    pdl_wait();
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nleaf) return;
    const int64_t g = leaves[w];
    uint64_t x0 = ~0ull, x1 = 0, y0 = ~0ull, y1 = 0;
    for (int pass = 0; pass < (separate ? 2 : 1); ++pass) {
        const int2 r = pass ? box_tgt[g] : box_src[g];
        const double2 *pts = pass ? xt : xs;
        for (int i = lane; i < r.y; i += 32) {
            const double2 p = pts[r.x + i];
            const uint64_t kx = order_key(p.x), ky = order_key(p.y);
            x0 = kx < x0 ? kx : x0;
            x1 = kx > x1 ? kx : x1;
            y0 = ky < y0 ? ky : y0;
            y1 = ky > y1 ? ky : y1;
        }
    }
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        const uint64_t a = __shfl_xor_sync(0xffffffffu, x0, d);
        const uint64_t b = __shfl_xor_sync(0xffffffffu, x1, d);
        const uint64_t c = __shfl_xor_sync(0xffffffffu, y0, d);
        const uint64_t e = __shfl_xor_sync(0xffffffffu, y1, d);
        x0 = a < x0 ? a : x0;
        x1 = b > x1 ? b : x1;
        y0 = c < y0 ? c : y0;
        y1 = e > y1 ? e : y1;
    }
    if (lane == 0)
        geo[g] = (x0 <= x1) ? make_double4(key_to_double(x0), key_to_double(x1),
                                           key_to_double(y0), key_to_double(y1))
                            : rect[g];
}

// A parent's bounding rectangle: the union of those of its children that
// hold points (entries of `boxes` without children are skipped).
GBI void tight_union_box(int64_t g, const int *__restrict__ child0,
                         const int2 *__restrict__ box_src, const int2 *__restrict__ box_tgt,
                         int separate, const double4 *__restrict__ rect, double4 *geo) {
    const int64_t c0 = child0[g];
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

__global__ void k_tight_union(int64_t n, const int *__restrict__ boxes,
                              const int *__restrict__ child0, const int2 *__restrict__ box_src,
                              const int2 *__restrict__ box_tgt, int separate,
                              const double4 *__restrict__ rect, double4 *geo) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    tight_union_box(boxes[i], child0, box_src, box_tgt, separate, rect, geo);
}

// Levels l1 .. 0 (at most TU_THREADS boxes each) in one block, level after
// level: a level's rectangles are complete before its parents read them.
constexpr int TU_THREADS = 1024;
__global__ void __launch_bounds__(TU_THREADS)
    k_tight_union_top(int l1, int R, const int *__restrict__ child0,
                      const int2 *__restrict__ box_src, const int2 *__restrict__ box_tgt,
                      int separate, const double4 *__restrict__ rect, double4 *geo) {
    pdl_wait();
    for (int l = l1; l >= 0; --l) {
        const int64_t g0 = R * level_base(l), nl = R * (level_base(l + 1) - level_base(l));
        for (int64_t i = threadIdx.x; i < nl; i += TU_THREADS)
            tight_union_box(g0 + i, child0, box_src, box_tgt, separate, rect, geo);
        __syncthreads();
    }
}

inline unsigned blocks_for(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace


fmm_status compute_geom(Tree &t, cudaStream_t s) {
    launch_k(k_geom, blocks_for(t.n_boxes, 256), 256, 0, s, t.n_boxes, t.rect_geo, t.geom);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "geometry");
}

fmm_status build_topology(Tree &t, const double *src_xy, const double *tgt_xy,
                          const int64_t * /*inst_off*/, cudaStream_t s) {
    const double2 *src = reinterpret_cast<const double2 *>(src_xy);
    const double2 *tgt = reinterpret_cast<const double2 *>(tgt_xy);
    const int64_t n = t.n_src, m = t.separate ? t.n_tgt : 0;
    const int L = t.L;
    // R > 1: the trees of R instances with the same L at once; root r owns the
    // sources [root_off[r], root_off[r+1]) (and the evaluation points
    // [root_toff[r], root_toff[r+1]) when separate)
    const int R = t.n_roots;
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

    if (R > 1 && ((int64_t)t.root_off.size() != R + 1 ||
                  (t.separate && (int64_t)t.root_toff.size() != R + 1))) {
        set_error("root offsets missing");
        return FMM_ERR_ARG;
    }
    const int64_t nb = R * level_base(L + 1);
    const int64_t nint = L > 0 ? R * level_base(L) : 1;
    t.n_boxes = nb;
    for (int l = 0; l <= L + 1; ++l) t.level_start[l] = R * level_base(l);
    int64_t n_max = n;  // the most sources of one root
    if (R > 1) {
        n_max = 0;
        for (int r = 0; r < R; ++r) n_max = std::max(n_max, t.root_off[r + 1] - t.root_off[r]);
    }
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
    int64_t *soff_d = nullptr, *toff_d = nullptr;
    HostStage hs;
    if (!hs.w) {
        tmp.release();
        set_error("page-locked stage allocation failed");
        return FMM_ERR_NOMEM;
    }
    unsigned long long hacc[6];
    if (R == 1) {
        CK(arena_alloc(tmp, &acc, 6));
        launch_k(k_bbox_init, 1, 32, 0, s, acc);
        CK(cudaGetLastError());
        int64_t tot = n + m;
        unsigned g = (unsigned)std::min<int64_t>(blocks_for(tot, 256), 152 * 8);
        launch_k(k_bbox, g, 256, 0, s, src, n, tgt, m, acc, t.status);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(hs.w, acc, 6 * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
    } else {
        CK(arena_alloc(tmp, &acc, 6 * (size_t)R + 2));
        CK(arena_alloc(tmp, &soff_d, (size_t)R + 1));
        CK(cudaMemcpyAsync(soff_d, t.root_off.data(), (R + 1) * sizeof(int64_t),
                           cudaMemcpyHostToDevice, s));
        if (t.separate) {
            CK(arena_alloc(tmp, &toff_d, (size_t)R + 1));
            CK(cudaMemcpyAsync(toff_d, t.root_toff.data(), (R + 1) * sizeof(int64_t),
                               cudaMemcpyHostToDevice, s));
        }
        CK(cudaMemsetAsync(acc, 0, (6 * (size_t)R + 2) * sizeof(unsigned long long), s));
        launch_k(k_bbox_roots, (unsigned)R, BB_THREADS, 0, s, R, src, soff_d, tgt, toff_d, acc,
                 t.status);
        CK(cudaGetLastError());
        CK(cudaMemcpyAsync(hs.w + 8, acc + 6 * R, 2 * sizeof(unsigned long long),
                           cudaMemcpyDeviceToHost, s));
    }
    CK(cudaMemcpyAsync(hs.w + 12, t.status, sizeof(int), cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::memcpy(hacc, hs.w, sizeof(hacc));
    const int hstat = (int)hs.w[12];
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
    const int64_t max_seg = (int64_t)R << (2 * L);
    int *seg_start[2], *seg_cnt[2];
    double4 *seg_rect[2];
    int4 *info;
    for (int k = 0; k < 2; ++k) {
        CK(arena_alloc(tmp, &seg_start[k], max_seg));
        CK(arena_alloc(tmp, &seg_cnt[k], max_seg));
        CK(arena_alloc(tmp, &seg_rect[k], max_seg));
    }
    CK(arena_alloc(tmp, &info, max_seg));
    if (R == 1)
        launch_k(k_root, 1, 1, 0, s, acc, n, t.rect, t.box_src, seg_start[0], seg_cnt[0],
                 seg_rect[0]);
    else
        launch_k(k_roots, blocks_for(R, 128), 128, 0, s, R, acc, soff_d, t.rect, t.box_src,
                 seg_start[0], seg_cnt[0], seg_rect[0]);
    CK(cudaGetLastError());

    const unsigned gb = blocks_for(n, 256);
    if (L == 0) {
        launch_k(k_final_perm, gb, 256, 0, s, n, 0, nullptr, nullptr, nullptr, nullptr, nullptr,
                 nullptr, t.perm);
        CK(cudaGetLastError());
    } else {
        uint64_t *kx, *ky, *kalt, *kalt2;
        uint32_t *lx, *ly, *lalt, *lalt2;
        CK(arena_alloc(tmp, &kx, n));
        CK(arena_alloc(tmp, &ky, n));
        CK(arena_alloc(tmp, &kalt, n));
        CK(arena_alloc(tmp, &kalt2, n));
        CK(arena_alloc(tmp, &lx, n));
        CK(arena_alloc(tmp, &ly, n));
        CK(arena_alloc(tmp, &lalt, n));
        CK(arena_alloc(tmp, &lalt2, n));
        launch_k(k_init_keys, gb, 256, 0, s, src, n, kx, ky, lx, ly);
        CK(cudaGetLastError());
        uint64_t *kfree0, *kfree1;  // key buffers free after the two sorts
        {
            // both coordinates in the same launches (a digit constant in one of
            // them is a stable no-op pass there)
            uint64_t *const kbuf[2][2] = {{kx, kalt}, {ky, kalt2}};
            uint32_t *const vbuf[2][2] = {{lx, lalt}, {ly, lalt2}};
            uint64_t *K[2] = {kx, ky}, *KA[2] = {kalt, kalt2};
            uint32_t *V[2] = {lx, ly}, *VA[2] = {lalt, lalt2};
            CK(radix_sort_pairs2(K, V, KA, VA, n, mask_x | mask_y, tmp, s));
            kx = K[0];
            ky = K[1];
            lx = V[0];
            ly = V[1];
            if (R > 1) {
                // then stably by root: each root's sources form one block of
                // both orders, sorted by (coordinate, index) inside it
                int *root;
                CK(arena_alloc(tmp, &root, n));
                launch_k(k_root_of, gb, 256, 0, s, n, R, soff_d, root);
                launch_k(k_root_keys, gb, 256, 0, s, n, root, lx, ly, kx, ky);
                CK(cudaGetLastError());
                int bits = 1;
                while ((int64_t(1) << bits) < R) ++bits;
                // the coordinate keys are spent; the ping-pong partners are
                // the other buffer of each pair (the first sort may have
                // ended in either)
                uint64_t *K2[2] = {kx, ky}, *KA2[2];
                uint32_t *V2[2] = {lx, ly}, *VA2[2];
                for (int y = 0; y < 2; ++y) {
                    KA2[y] = K2[y] == kbuf[y][0] ? kbuf[y][1] : kbuf[y][0];
                    VA2[y] = V2[y] == vbuf[y][0] ? vbuf[y][1] : vbuf[y][0];
                }
                CK(radix_sort_pairs2(K2, V2, KA2, VA2, n, digits_for_bits(bits), tmp, s));
                kx = K2[0];
                ky = K2[1];
                lx = V2[0];
                ly = V2[1];
            }
            kfree0 = kx;  // the sorted keys are not needed any more
            kfree1 = ky;
        }
        // entry lists: (x rank, y rank) in x order and in y order
        uint2 *ex = reinterpret_cast<uint2 *>(kfree0), *ey = reinterpret_cast<uint2 *>(kfree1);
        uint2 *ex2, *ey2;
        CK(arena_alloc(tmp, &ex2, n));
        CK(arena_alloc(tmp, &ey2, n));
        {
            uint32_t *rx = reinterpret_cast<uint32_t *>(ex2), *ry = reinterpret_cast<uint32_t *>(ey2);
            launch_k(k_ranks, gb, 256, 0, s, n, lx, ly, rx, ry);
            CK(cudaGetLastError());
            launch_k(k_entries, gb, 256, 0, s, n, lx, ly, rx, ry, ex, ey);
            CK(cudaGetLastError());
        }
        // rounds r < r0 over the whole array; r0 .. 2L-1 per segment in shared memory
        int r0 = 0;
        while (r0 < 2 * L && ((n_max + (int64_t(1) << r0) - 1) >> r0) > LOC_CAP) ++r0;
        const bool local = r0 < 2 * L;
        if (local) r0 = std::max(r0, 2 * L - LOC_MAX_ROUNDS);
        int cur = 0;
        if (r0 > 0) {
            const int ntiles = (int)((n + PT_TILE - 1) / PT_TILE);
            int *pseg[2];
            uint32_t *sums;
            CK(arena_alloc(tmp, &pseg[0], n));
            CK(arena_alloc(tmp, &pseg[1], n));
            CK(arena_alloc(tmp, &sums, 2 * (size_t)ntiles));
            if (R == 1)
                CK(cudaMemsetAsync(pseg[0], 0, n * sizeof(int), s));
            else
                launch_k(k_root_of, gb, 256, 0, s, n, R, soff_d, pseg[0]);
            for (int r = 0; r < r0; ++r) {
                const int nseg = R << r;
                launch_k(k_seg_split, 1, SEG_THREADS, 0, s, r, R, nseg, seg_start[cur], seg_cnt[cur],
                         seg_rect[cur], seg_start[cur ^ 1], seg_cnt[cur ^ 1], seg_rect[cur ^ 1],
                         info, ex, ey, lx, ly, src, t.rect, t.box_src, t.split_axis, t.split_line);
                CK(cudaGetLastError());
                launch_k(k_pcount, dim3(ntiles, 2), PT_THREADS, 0, s, n, pseg[cur], info, ex, ey,
                         sums, ntiles);
                CK(cudaGetLastError());
                if (ntiles > PT_DIRECT_TILES) {
                    launch_k(k_tile_scan, 1, SEG_THREADS, 0, s, sums, ntiles);
                    CK(cudaGetLastError());
                }
                launch_k(k_part, dim3(ntiles, 2), PT_THREADS, 0, s, n, pseg[cur], info, ex, ey, ex2,
                         ey2, sums, ntiles, pseg[cur ^ 1]);
                CK(cudaGetLastError());
                std::swap(ex, ex2);
                std::swap(ey, ey2);
                cur ^= 1;
            }
            if (!local) {
                // pseg[cur] holds the leaf of every position; info the last round's axes
                launch_k(k_final_perm, gb, 256, 0, s, n, L, pseg[cur], info, ex, ey, lx, ly,
                         t.perm);
                CK(cudaGetLastError());
            }
        }
        if (local) {
            static const cudaError_t attr = cudaFuncSetAttribute(
                k_tree_local, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)LOC_SMEM);
            CK(attr);
            int *st3, *cn3;
            double4 *rc3;
            CK(arena_alloc(tmp, &st3, max_seg));
            CK(arena_alloc(tmp, &cn3, max_seg));
            CK(arena_alloc(tmp, &rc3, max_seg));
            launch_k(k_tree_local, (unsigned)((int64_t)R << r0), LOC_THREADS, LOC_SMEM, s, r0, L, R,
                     seg_start[cur], seg_cnt[cur], seg_rect[cur], seg_start[cur ^ 1],
                     seg_cnt[cur ^ 1], seg_rect[cur ^ 1], st3, cn3, rc3, info, ex, ey, lx, ly, src,
                     t.rect, t.box_src, t.split_axis, t.split_line, t.perm);
            CK(cudaGetLastError());
        }
    }
    launch_k(k_gather2, gb, 256, 0, s, n, t.perm, src, t.xs);
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
            launch_k(k_descend, blocks_for(m, 256), 256, 0, s, m, tgt, L, R, toff_d, t.split_axis,
                     t.split_line, key, idx);
            CK(cudaGetLastError());
            int rbits = 0;
            while ((int64_t(1) << rbits) < R) ++rbits;
            CK(radix_sort_pairs(&key, &idx, kalt, ialt, m, digits_for_bits(2 * L + rbits), tmp, s));
            CK(cudaMemcpyAsync(t.tperm, idx, m * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s));
            launch_k(k_gather2, blocks_for(m, 256), 256, 0, s, m, t.tperm, tgt, t.xt);
            CK(cudaGetLastError());
        }
        launch_k(k_tgt_ranges, blocks_for(nb, 256), 256, 0, s, nb, L, R, key, m, t.box_tgt);
        CK(cudaGetLastError());
    } else {
        t.tperm = t.perm;
        t.xt = t.xs;
        t.box_tgt = t.box_src;
    }
    t.n_leaves = (int)((int64_t)R << (2 * L));
    CK(arena_alloc(t.mem, &t.parent, nb));
    CK(arena_alloc(t.mem, &t.child0, nb));
    CK(arena_alloc(t.mem, &t.lvl_boxes, nb));
    CK(arena_alloc(t.mem, &t.leaves, t.n_leaves));
    launch_k(k_relations, blocks_for(nb, 256), 256, 0, s, nb, L, R, t.parent, t.child0,
             t.lvl_boxes, t.leaves);
    CK(cudaGetLastError());
    // box geometry: the split rectangles, or the points' bounding rectangles
    if (t.box_fit) {
        CK(arena_alloc(t.mem, &t.rect_geo, nb));
        launch_k(k_tight_leaf, blocks_for((int64_t)t.n_leaves * 32, 128), 128, 0, s, t.n_leaves,
                 t.leaves, t.box_src, t.xs, t.box_tgt, t.xt, t.separate ? 1 : 0, t.rect,
                 t.rect_geo);
        CK(cudaGetLastError());
        // the levels with at most TU_THREADS boxes run in one block, the
        // deeper ones one launch per level
        int l_top = L - 1;
        while (l_top >= 0 && R * (level_base(l_top + 1) - level_base(l_top)) > TU_THREADS) --l_top;
        for (int l = L - 1; l > l_top; --l) {
            const int64_t nl = R * (level_base(l + 1) - level_base(l));
            launch_k(k_tight_union, blocks_for(nl, 128), 128, 0, s, nl, t.lvl_boxes + R * level_base(l),
                     t.child0, t.box_src, t.box_tgt, t.separate ? 1 : 0, t.rect, t.rect_geo);
            CK(cudaGetLastError());
        }
        if (l_top >= 0) {
            launch_k(k_tight_union_top, 1, TU_THREADS, 0, s, l_top, R, t.child0, t.box_src,
                     t.box_tgt, t.separate ? 1 : 0, t.rect, t.rect_geo);
            CK(cudaGetLastError());
        }
    } else {
        t.rect_geo = t.rect;
    }
    launch_k(k_geom, blocks_for(nb, 256), 256, 0, s, nb, t.rect_geo, t.geom);
    CK(cudaGetLastError());
    // temporaries are stream-ordered: freeing them here is safe
    tmp.release();
#undef CK
    return FMM_OK;
}

}  // namespace gbfmm
