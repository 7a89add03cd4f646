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
// With the leaf shortcut on (Sec. 2), every leaf strong pair other than the
// box itself is tested again with r and R interchanged, r + theta R <=
// theta d; a pair that passes leaves the near list for the P2L list (source
// box larger) or the M2P list (source box smaller).  The P2P items then run
// over the near lists.
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

namespace {

constexpr int P2P_CHUNK = 64;     // targets per work item
constexpr int M2P_RUN = 16;       // leaf shortcut: M2P list entries per work item

// Box ids are level-major over R roots (a forest of R trees with the same
// number of levels): level l holds boxes [R lb(l), R lb(l+1)), box B of level
// l (counted from R lb(l)) has children 4B .. 4B+3 of level l+1.  R = 1 is a
// single tree.
__host__ __device__ inline int64_t lb(int l) { return ((int64_t(1) << (2 * l)) - 1) / 3; }

// Every root is its own strong list and has an empty weak list.
__global__ void k_conn_init(int R, int *weak_off, int *strong_off, int *strong) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > R) return;
    weak_off[i] = 0;
    strong_off[i] = i;
    if (i < R) strong[i] = i;
}

// Theta-criterion (Eq. 3) from precomputed centres and radii, bit-identical to
// the reference rounding sequence d = sqrt(dx^2 + dy^2), R + theta r <= theta d:
// a comparison of squares decides every pair that is clear by a relative
// margin of 1e-12, the exact expression decides the rest.
// `swapped` tests r + theta R <= theta d instead (the leaf shortcut).
GBI bool weak_pair(double bx, double by, double rb, double cx, double cy, double rc,
                   double theta, bool swapped = false) {
    double dx = __dsub_rn(bx, cx), dy = __dsub_rn(by, cy);
    double d2 = __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy));
    if (!(d2 > 0.0)) return false;
    double R = rb > rc ? rb : rc, r = rb > rc ? rc : rb;
    double a = swapped ? __dadd_rn(r, __dmul_rn(theta, R)) : __dadd_rn(R, __dmul_rn(theta, r));
    double lhs = a * a, rhs = theta * theta * d2;
    if (lhs < rhs * (1.0 - 1e-12)) return true;
    if (lhs > rhs * (1.0 + 1e-12)) return false;
    return a <= __dmul_rn(theta, __dsqrt_rn(d2));
}

// Float pre-test of the same criterion from df32 centres (x hi, x lo, y hi,
// y lo) and float radii: every float quantity is within ~20 units of 2^-24
// of its FP64 value, so a pair clear by a relative margin of 1e-5 gets the
// FP64 test's answer (1 weak, 0 not weak); -1: decide in FP64.
GBI int weak_pair_f(float4 b, float rb, float4 c, float rc, float theta, bool swapped) {
    const float dx = __fadd_rn(__fsub_rn(b.x, c.x), __fsub_rn(b.y, c.y));
    const float dy = __fadd_rn(__fsub_rn(b.z, c.z), __fsub_rn(b.w, c.w));
    const float d2 = __fmaf_rn(dx, dx, __fmul_rn(dy, dy));
    const float R = fmaxf(rb, rc), r = fminf(rb, rc);
    const float a = swapped ? __fmaf_rn(theta, R, r) : __fmaf_rn(theta, r, R);
    const float lhs = __fmul_rn(a, a), rhs = __fmul_rn(__fmul_rn(theta, theta), d2);
    if (lhs < __fmul_rn(rhs, 1.0f - 1e-5f)) return 1;
    if (lhs > __fmul_rn(rhs, 1.0f + 1e-5f)) return 0;
    return -1;
}

// candidates of box b of level l: the 4 children of each entry of strong(parent)
__global__ void k_cand_count(int l, int R, const int *__restrict__ strong_off, uint32_t *ncand) {
    pdl_wait();
    int64_t nbl = (int64_t)R << (2 * l);
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nbl) return;
    int64_t par = R * lb(l - 1) + b / 4;
    ncand[b] = 4u * (uint32_t)(strong_off[par + 1] - strong_off[par]);
}

GBI int64_t owner_of(const uint32_t *off, int64_t n, uint32_t i) {
    // largest b in [0, n) with off[b] <= i
    int64_t lo = 0, hi = n;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) >> 1;
        if (off[mid] <= i)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__global__ void k_cand_test(int l, int R, const uint32_t *__restrict__ cand_off,
                            const int *__restrict__ strong_off, const int *__restrict__ strong,
                            const double4 *__restrict__ geom, const double *__restrict__ rad,
                            const float4 *__restrict__ gfl, const float *__restrict__ radf,
                            double theta, uint32_t *wflag, int *cand_box) {
    pdl_wait();
    const int64_t nbl = (int64_t)R << (2 * l);
    const uint32_t total = cand_off[nbl];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += gridDim.x * blockDim.x) {
        int64_t b = owner_of(cand_off, nbl, i);
        uint32_t k = i - cand_off[b];
        int64_t par = R * lb(l - 1) + b / 4;
        int s = strong[strong_off[par] + (int)(k >> 2)];
        int64_t c = R * lb(l) + 4 * (s - R * lb(l - 1)) + (k & 3);
        int64_t g = R * lb(l) + b;
        int wf = weak_pair_f(gfl[g], radf[g], gfl[c], radf[c], (float)theta, false);
        if (wf < 0) {
            const double4 gb = geom[g], gc = geom[c];
            wf = weak_pair(gb.x, gb.y, rad[g], gc.x, gc.y, rad[c], theta) ? 1 : 0;
        }
        const bool w = wf == 1;
        wflag[i] = w ? 1u : 0u;
        cand_box[i] = (int)c;
    }
}

// Every candidate is weak or strong: with wpos = wbase + #weak before i, the
// strong position is sbase + i - #weak before i.
__global__ void k_cand_scatter(int l, int R, const uint32_t *__restrict__ cand_off,
                               const uint32_t *__restrict__ wflag,
                               const uint32_t *__restrict__ wpos, const int *__restrict__ wbase,
                               const int *__restrict__ sbase, const int *__restrict__ cand_box,
                               int *weak, int64_t cap_w, int *strong, int64_t cap_s, int *status) {
    pdl_wait();
    const uint32_t total = cand_off[(int64_t)R << (2 * l)];
    const uint32_t wb = (uint32_t)*wbase, sb = (uint32_t)*sbase;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += gridDim.x * blockDim.x) {
        if (wflag[i]) {
            uint32_t o = wpos[i];
            if ((int64_t)o < cap_w)
                weak[o] = cand_box[i];
            else
                atomicOr(status, ST_LIST_OVERFLOW);
        } else {
            uint32_t o = sb + i - (wpos[i] - wb);
            if ((int64_t)o < cap_s)
                strong[o] = cand_box[i];
            else
                atomicOr(status, ST_LIST_OVERFLOW);
        }
    }
}

// weak_off / strong_off of level l; the level's bases are read before any
// thread overwrites them (thread b = 0 writes the same values back).
__global__ void k_cand_offsets(int l, int R, const uint32_t *__restrict__ cand_off,
                               const uint32_t *__restrict__ wpos, int *weak_off, int *strong_off) {
    pdl_wait();
    int64_t nbl = (int64_t)R << (2 * l);
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b > nbl) return;
    const int64_t g0 = R * lb(l);
    const uint32_t wb = (uint32_t)weak_off[g0], sb = (uint32_t)strong_off[g0];
    uint32_t ci = cand_off[b];
    weak_off[g0 + b] = (int)wpos[ci];
    strong_off[g0 + b] = (int)(sb + ci - (wpos[ci] - wb));
}

// Levels 1 .. l1 in one block, level after level, while a level has at most
// SH_CAND candidates (R 16^l bounds them: a box has at most 4^l, the children
// of its parent's strong boxes, all in its own tree): the counts, the theta
// tests, the scans, the lists and their offsets as the per-level kernels
// make them, with the candidates in shared memory and without their launches.
constexpr int SH_THREADS = 1024;
constexpr int SH_CAND = 4096;         // candidates of a level
constexpr int SH_BOX = SH_THREADS;    // boxes of a level: R 4^l <= R 16^l / 4 for l >= 1
constexpr int SH_ITEMS = SH_CAND / SH_THREADS;
__global__ void __launch_bounds__(SH_THREADS)
    k_conn_shallow(int l1, int R, const double4 *__restrict__ geom, const double *__restrict__ rad,
                   const float4 *__restrict__ gfl, const float *__restrict__ radf, double theta,
                   int *weak_off, int *strong_off, int *weak, int64_t cap_w, int *strong,
                   int64_t cap_s, int *status) {
    pdl_wait();
    __shared__ uint32_t s_off[SH_BOX + 1];
    __shared__ uint32_t s_wpos[SH_CAND];  // weak candidates before i
    __shared__ int s_box[SH_CAND];
    __shared__ uint8_t s_w[SH_CAND];
    __shared__ uint32_t wt[SH_THREADS / 32];
    __shared__ uint32_t s_base[2];
    for (int l = 1; l <= l1; ++l) {
        const int nbl = R << (2 * l);
        const int64_t g0 = R * lb(l), p0 = R * lb(l - 1);
        // the level's list bases, written by the previous level (or the roots)
        if (threadIdx.x == 0) {
            s_base[0] = (uint32_t)weak_off[g0];
            s_base[1] = (uint32_t)strong_off[g0];
        }
        const int b = threadIdx.x;
        uint32_t cnt = 0;
        if (b < nbl) {
            const int64_t par = p0 + b / 4;
            cnt = 4u * (uint32_t)(strong_off[par + 1] - strong_off[par]);
        }
        uint32_t excl;
        const uint32_t total = block_scan_excl<SH_THREADS>(cnt, excl, wt);
        if (b < nbl) s_off[b] = excl;
        if (b == 0) s_off[nbl] = total;
        __syncthreads();
        // theta tests of SH_ITEMS consecutive candidates per thread
        const int i0 = threadIdx.x * SH_ITEMS;
        uint32_t wsum = 0;
#pragma unroll
        for (int k = 0; k < SH_ITEMS; ++k) {
            const int i = i0 + k;
            if (i >= (int)total) break;
            int lo = 0, hi = nbl;  // the largest box bb with s_off[bb] <= i
            while (hi - lo > 1) {
                const int mid = (lo + hi) >> 1;
                if (s_off[mid] <= (uint32_t)i)
                    lo = mid;
                else
                    hi = mid;
            }
            const uint32_t kk = (uint32_t)i - s_off[lo];
            const int64_t par = p0 + lo / 4;
            const int sb = strong[strong_off[par] + (int)(kk >> 2)];
            const int64_t c = g0 + 4 * (sb - p0) + (kk & 3);
            const int64_t g = g0 + lo;
            int wf = weak_pair_f(gfl[g], radf[g], gfl[c], radf[c], (float)theta, false);
            if (wf < 0) {
                const double4 gb = geom[g], gc = geom[c];
                wf = weak_pair(gb.x, gb.y, rad[g], gc.x, gc.y, rad[c], theta) ? 1 : 0;
            }
            s_w[i] = wf == 1 ? 1 : 0;
            s_box[i] = (int)c;
            wsum += wf == 1 ? 1u : 0u;
        }
        uint32_t wex;
        const uint32_t nweak = block_scan_excl<SH_THREADS>(wsum, wex, wt);
#pragma unroll
        for (int k = 0; k < SH_ITEMS; ++k) {
            const int i = i0 + k;
            if (i >= (int)total) break;
            s_wpos[i] = wex;
            wex += s_w[i];
        }
        __syncthreads();
        const uint32_t wb = s_base[0], sbase = s_base[1];
        for (int i = threadIdx.x; i < (int)total; i += SH_THREADS) {
            if (s_w[i]) {
                const uint32_t o = wb + s_wpos[i];
                if ((int64_t)o < cap_w)
                    weak[o] = s_box[i];
                else
                    atomicOr(status, ST_LIST_OVERFLOW);
            } else {
                const uint32_t o = sbase + (uint32_t)i - s_wpos[i];
                if ((int64_t)o < cap_s)
                    strong[o] = s_box[i];
                else
                    atomicOr(status, ST_LIST_OVERFLOW);
            }
        }
        for (int bb = threadIdx.x; bb <= nbl; bb += SH_THREADS) {
            const uint32_t ci = s_off[bb];
            const uint32_t wp = ci < total ? s_wpos[ci] : nweak;
            weak_off[g0 + bb] = (int)(wb + wp);
            strong_off[g0 + bb] = (int)(sbase + ci - wp);
        }
        __syncthreads();  // this level's lists and offsets before the next level reads them
    }
}

__global__ void k_radius(int64_t nb, const double4 *__restrict__ rect, double *rad,
                         float4 *gfl, float *radf) {
    pdl_wait();
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nb) return;
    double4 r4 = rect[g];
    Rect r{r4.x, r4.y, r4.z, r4.w};
    double cx, cy, rr;
    centre_radius(r, cx, cy, rr);
    rad[g] = rr;
    // df32 centre and float radius for the float pre-test
    const float xh = __double2float_rn(cx), yh = __double2float_rn(cy);
    gfl[g] = make_float4(xh, __double2float_rn(cx - (double)xh), yh,
                         __double2float_rn(cy - (double)yh));
    radf[g] = __double2float_rn(rr);
}

// Chunks of <= P2P_CHUNK targets per target leaf.
__global__ void k_leaf_chunks(int64_t nleaf, int64_t leaf0, const int2 *__restrict__ box_tgt,
                              int chunk, uint32_t *cnt) {
    pdl_wait();
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

// Per leaf: work items of its chunks (P2P runs, plus M2P runs of at most
// M2P_RUN entries of the leaf's M2P list when the shortcut is on), and how
// many of them are P2P items.
__global__ void k_leaf_runs(int64_t nleaf, int64_t leaf0, const int *__restrict__ p2p_off,
                            const int *__restrict__ p2p_list, const int2 *__restrict__ box_src,
                            const uint32_t *__restrict__ chunks, int cap,
                            const int *__restrict__ m2p_off, uint32_t *items,
                            uint32_t *items_p2p) {
    pdl_wait();
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int64_t g = leaf0 + b;
    int r = source_runs(p2p_list, p2p_off[g], p2p_off[g + 1], box_src, cap, nullptr);
    int rm = m2p_off ? (m2p_off[g + 1] - m2p_off[g] + M2P_RUN - 1) / M2P_RUN : 0;
    items[b] = (uint32_t)(r + rm) * chunks[b];
    items_p2p[b] = (uint32_t)r * chunks[b];
}

// Items of each chunk: its P2P items (leaf, first target, run [e0, e1) of the
// near-field list), then its M2P items (leaf, first target, ~e0, ~e1) over the
// M2P list; chunk c owns items [item0[c], item0[c+1]).  Sort keys put all P2P
// items before all M2P items, each kind in order of decreasing cost.
__global__ void k_fill_items(int64_t nleaf, int64_t leaf0, const int2 *__restrict__ box_tgt,
                             const int2 *__restrict__ box_src, const int *__restrict__ p2p_off,
                             const int *__restrict__ p2p_list, const int *__restrict__ m2p_off,
                             int chunk, int cap, const uint32_t *__restrict__ chunk_off,
                             const uint32_t *__restrict__ item_off, int2 *chunks, int *item0,
                             int4 *items, uint64_t *key, uint32_t *val) {
    pdl_wait();
    int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    int64_t g = leaf0 + b;
    int2 tt = box_tgt[g];
    int e0 = p2p_off[g], e1 = p2p_off[g + 1];
    uint32_t c = chunk_off[b], it = item_off[b];
    for (int t0 = 0; t0 < tt.y; t0 += chunk, ++c) {
        int nt = min(chunk, tt.y - t0);
        chunks[c] = make_int2((int)g, t0);
        item0[c] = (int)it;
        // walk the runs again, emitting one item each
        int acc = 0, rs = e0;
        for (int e = e0; e <= e1; ++e) {
            int n = e < e1 ? box_src[p2p_list[e]].y : 0;
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
        if (m2p_off) {
            const int m1 = m2p_off[g + 1];
            for (int e = m2p_off[g]; e < m1; e += M2P_RUN) {
                const int ee = min(e + M2P_RUN, m1);
                uint64_t cost = (uint64_t)nt * (uint64_t)(ee - e);
                items[it] = make_int4((int)g, t0, ~e, ~ee);
                key[it] = (1ull << 32) | (0xffffffffull - cost);
                val[it] = it;
                ++it;
            }
        }
    }
}

__global__ void k_set_last(int *item0, int64_t n_chunks, int n_items) {
    pdl_wait();
    item0[n_chunks] = n_items;
}

__global__ void k_copy_u32(int64_t n, const uint32_t *__restrict__ in, int *out) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int)in[i];
}

// Leaf shortcut class of the strong pair (b, c): 0 near, 1 P2L, 2 M2P.
// Besides the swapped criterion the smaller radius must be positive: the
// test then keeps every point pair of the two boxes at least r (1/theta - 1)
// apart, while a box of radius 0 (all its points equal) can sit on a corner
// of the larger box, where that box may hold a copy of the same point.
GBI int shortcut_class(int64_t b, int64_t c, const double4 *__restrict__ geom,
                       const double *__restrict__ rad, const float4 *__restrict__ gfl,
                       const float *__restrict__ radf, double theta) {
    if (b == c) return 0;
    // radii are >= 0: their bit patterns order like their values
    const long long ib = __double_as_longlong(rad[b]), ic = __double_as_longlong(rad[c]);
    if ((ib < ic ? ib : ic) == 0) return 0;
    int w = weak_pair_f(gfl[b], radf[b], gfl[c], radf[c], (float)theta, true);
    if (w < 0) {
        const double4 gb = geom[b], gc = geom[c];
        w = weak_pair(gb.x, gb.y, rad[b], gc.x, gc.y, rad[c], theta, true) ? 1 : 0;
    }
    if (!w) return 0;
    return ic > ib ? 1 : 2;
}

// Leaf shortcut at the finest level, flattened over its candidates: class
// flags of the strong candidates (weak candidates get none).
__global__ void k_cand_short(int l, int R, const uint32_t *__restrict__ cand_off,
                             const uint32_t *__restrict__ wflag, const int *__restrict__ cand_box,
                             const double4 *__restrict__ geom, const double *__restrict__ rad,
                             const float4 *__restrict__ gfl, const float *__restrict__ radf,
                             double theta, uint32_t *nflag, uint32_t *pflag, uint32_t *mflag) {
    pdl_wait();
    const int64_t nbl = (int64_t)R << (2 * l);
    const uint32_t total = cand_off[nbl];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += gridDim.x * blockDim.x) {
        int k = -1;
        if (!wflag[i]) {
            int64_t b = owner_of(cand_off, nbl, i);
            k = shortcut_class(R * lb(l) + b, cand_box[i], geom, rad, gfl, radf, theta);
        }
        nflag[i] = k == 0;
        pflag[i] = k == 1;
        mflag[i] = k == 2;
    }
}

__global__ void k_short_scatter(int l, int R, const uint32_t *__restrict__ cand_off,
                                const uint32_t *__restrict__ nflag,
                                const uint32_t *__restrict__ pflag,
                                const uint32_t *__restrict__ mflag,
                                const uint32_t *__restrict__ npos, const uint32_t *__restrict__ ppos,
                                const uint32_t *__restrict__ mpos, const int *__restrict__ cand_box,
                                int *near, int *p2l, int *m2p) {
    pdl_wait();
    const uint32_t total = cand_off[(int64_t)R << (2 * l)];
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += gridDim.x * blockDim.x) {
        const int c = cand_box[i];
        if (nflag[i])
            near[npos[i]] = c;
        else if (pflag[i])
            p2l[ppos[i]] = c;
        else if (mflag[i])
            m2p[mpos[i]] = c;
    }
}

// Offsets of the leaves (level l = L); boxes above the leaves have empty lists.
__global__ void k_short_offsets(int l, int R, const uint32_t *__restrict__ cand_off,
                                const uint32_t *__restrict__ npos,
                                const uint32_t *__restrict__ ppos,
                                const uint32_t *__restrict__ mpos, int *near_off, int *p2l_off,
                                int *m2p_off) {
    pdl_wait();
    int64_t nbl = (int64_t)R << (2 * l);
    const int64_t g0 = R * lb(l);
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int64_t j = i; j < g0; j += (int64_t)gridDim.x * blockDim.x) {
        near_off[j] = 0;
        p2l_off[j] = 0;
        m2p_off[j] = 0;
    }
    if (i > nbl) return;
    uint32_t ci = cand_off[i];
    near_off[g0 + i] = (int)npos[ci];
    p2l_off[g0 + i] = (int)ppos[ci];
    m2p_off[g0 + i] = (int)mpos[ci];
}

// Trees of one box (L = 0): every root is its own near list.
__global__ void k_short_root(int R, int *near_off, int *near, int *p2l_off, int *m2p_off) {
    pdl_wait();
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > R) return;
    near_off[i] = i;
    if (i < R) near[i] = i;
    p2l_off[i] = 0;
    m2p_off[i] = 0;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

// Grow a device int buffer to hold at least `need` entries, keeping `keep`.
static cudaError_t grow(int **buf, int64_t *cap, int64_t need, int64_t keep, cudaStream_t s) {
    if (need <= *cap) return cudaSuccess;
    int64_t nc = std::max<int64_t>(need, 2 * *cap);
    int *nbuf = nullptr;
    cudaError_t e = dev_alloc(reinterpret_cast<void **>(&nbuf), nc * sizeof(int), s);
    if (e != cudaSuccess) return e;
    if (*buf && keep > 0) {
        e = cudaMemcpyAsync(nbuf, *buf, std::min(keep, *cap) * sizeof(int),
                            cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) return e;
    }
    if (*buf) dev_free(*buf, s);
    *buf = nbuf;
    *cap = nc;
    return cudaSuccess;
}

fmm_status build_connectivity(Tree &t, cudaStream_t s, uint32_t *stage,
                              const std::function<fmm_status()> &pre_sync) {
    const int L = t.L;
    const int R = t.n_roots;
    const int64_t nb = t.n_boxes;
    cudaError_t e;
    DevArena tmp;
    tmp.stream = s;
    DevArena lists;
    lists.stream = s;
    DevArena cand;  // candidate buffers, regrown per level
    cand.stream = s;
    int *weak = nullptr, *strong = nullptr;
    int64_t cap_w = 0, cap_s = 0;
#define CK(call)                           \
    do {                                   \
        if ((e = (call)) != cudaSuccess) { \
            tmp.release();                 \
            cand.release();                \
            lists.release();               \
            if (weak) dev_free(weak, s); \
            if (strong) dev_free(strong, s); \
            return cuda_fail(e, #call);    \
        }                                  \
    } while (0)
    int *weak_off, *strong_off;
    CK(arena_alloc(lists, &weak_off, nb + 1));
    CK(arena_alloc(lists, &strong_off, nb + 1));
    // every candidate lands in exactly one list, so 1 + the running candidate
    // count bounds both lists; they grow before a level is scattered
    int64_t bound = R;
    CK(grow(&weak, &cap_w, 40 * nb + 64, 0, s));
    CK(grow(&strong, &cap_s, 16 * nb + 64 + R, 0, s));
    CK(cudaMemsetAsync(t.status, 0, sizeof(int), s));
    launch_k(k_conn_init, nblk(R + 1, 256), 256, 0, s, R, weak_off, strong_off, strong);
    CK(cudaGetLastError());
    // per-box radius (same rounding sequence as the theta-test reference)
    double *rad;
    float4 *gfl;
    float *radf;
    CK(arena_alloc(tmp, &rad, nb));
    CK(arena_alloc(tmp, &gfl, nb));
    CK(arena_alloc(tmp, &radf, nb));
    launch_k(k_radius, nblk(nb, 256), 256, 0, s, nb, t.rect_geo, rad, gfl, radf);
    CK(cudaGetLastError());
    // leaf shortcut lists (built at the finest level, below)
    const bool shortcut = t.p2l_m2p != 0;
    int *near_off = nullptr, *p2l_off = nullptr, *m2p_off = nullptr;
    int *near = nullptr, *p2l = nullptr, *m2p = nullptr;
    uint32_t hshort[3] = {0, 0, 0};
    if (shortcut) {
        CK(arena_alloc(lists, &near_off, nb + 1));
        CK(arena_alloc(lists, &p2l_off, nb + 1));
        CK(arena_alloc(lists, &m2p_off, nb + 1));
    }
    if (shortcut && L == 0) {
        CK(arena_alloc(lists, &near, R));
        CK(arena_alloc(lists, &p2l, 1));
        CK(arena_alloc(lists, &m2p, 1));
        launch_k(k_short_root, nblk(R + 1, 256), 256, 0, s, R, near_off, near, p2l_off, m2p_off);
        CK(cudaGetLastError());
        hshort[0] = (uint32_t)R;
    }
    int64_t maxl = (int64_t)R << (2 * L);
    uint32_t *cand_off;
    CK(arena_alloc(tmp, &cand_off, maxl + 1));
    int64_t cand_cap = 0;
    uint32_t *wflag = nullptr, *wpos = nullptr;
    int *cand_box = nullptr;
    // the shallow levels in one block (not the leaf level of the shortcut split:
    // its classification needs the candidate arrays)
    int l_sh = 0;
    while (l_sh < L && ((int64_t)R << (4 * (l_sh + 1))) <= SH_CAND && !(shortcut && l_sh + 1 == L))
        ++l_sh;
    if (l_sh > 0) {
        const int64_t keep = bound;
        for (int l = 1; l <= l_sh; ++l) bound += (int64_t)R << (4 * l);
        CK(grow(&weak, &cap_w, bound, keep, s));
        CK(grow(&strong, &cap_s, bound, keep, s));
        launch_k(k_conn_shallow, 1, SH_THREADS, 0, s, l_sh, R, t.geom, rad, gfl, radf, t.theta,
                 weak_off, strong_off, weak, cap_w, strong, cap_s, t.status);
        CK(cudaGetLastError());
    }
    for (int l = l_sh + 1; l <= L; ++l) {
        int64_t nbl = (int64_t)R << (2 * l);
        launch_k(k_cand_count, nblk(nbl, 256), 256, 0, s, l, R, strong_off, cand_off);
        CK(cudaGetLastError());
        CK(exclusive_scan_u32(cand_off, cand_off, nbl, nullptr, tmp, s));
        // a box of level l has at most 4^l candidates (the children of the
        // parent's strong boxes, all in its own tree): while the level's
        // R 16^l bound stays below 2^20 it sizes the buffers and no
        // synchronisation is needed (the kernels read the actual count on the
        // device); deeper levels, and the leaf level of the shortcut split
        // (its scans need the count), read it
        uint32_t total;
        if (((int64_t)R << (4 * l)) <= (int64_t(1) << 20) && !(shortcut && l == L)) {
            total = (uint32_t)((int64_t)R << (4 * l));
        } else {
            CK(cudaMemcpyAsync(stage, cand_off + nbl, 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            total = stage[0];
        }
        if ((int64_t)total + 1 > cand_cap) {
            cand.release();
            cand_cap = std::max<int64_t>((int64_t)total + 1, 2 * cand_cap);
            CK(arena_alloc(cand, &wflag, cand_cap));
            CK(arena_alloc(cand, &wpos, cand_cap + 1));
            CK(arena_alloc(cand, &cand_box, cand_cap));
        }
        const int64_t keep = bound;
        bound += total;
        CK(grow(&weak, &cap_w, bound, keep, s));
        CK(grow(&strong, &cap_s, bound, keep, s));
        unsigned grid = (unsigned)std::min<int64_t>(nblk(total, 256), 152 * 16);
        launch_k(k_cand_test, grid, 256, 0, s, l, R, cand_off, strong_off, strong, t.geom, rad,
                 gfl, radf, t.theta, wflag, cand_box);
        CK(cudaGetLastError());
        uint32_t *wbase = reinterpret_cast<uint32_t *>(weak_off + R * lb(l));
        CK(exclusive_scan_u32(wflag, wpos, total, wbase, tmp, s));
        launch_k(k_cand_scatter, grid, 256, 0, s, l, R, cand_off, wflag, wpos, weak_off + R * lb(l),
                 strong_off + R * lb(l), cand_box, weak, cap_w, strong, cap_s, t.status);
        CK(cudaGetLastError());
        launch_k(k_cand_offsets, nblk(nbl + 1, 256), 256, 0, s, l, R, cand_off, wpos, weak_off,
                 strong_off);
        CK(cudaGetLastError());
        if (shortcut && l == L) {
            // near / P2L / M2P split of the leaf strong lists, in their order
            uint32_t *fl[3], *pos[3];
            for (int k = 0; k < 3; ++k) {
                CK(arena_alloc(tmp, &fl[k], (size_t)total + 1));
                CK(arena_alloc(tmp, &pos[k], (size_t)total + 1));
            }
            launch_k(k_cand_short, grid, 256, 0, s, l, R, cand_off, wflag, cand_box, t.geom, rad,
                     gfl, radf, t.theta, fl[0], fl[1], fl[2]);
            CK(cudaGetLastError());
            {
                const uint32_t *in3[3] = {fl[0], fl[1], fl[2]};
                CK(exclusive_scan_u32_sets(3, in3, pos, total, tmp, s));
            }
            for (int k = 0; k < 3; ++k)
                CK(cudaMemcpyAsync(stage + 1 + k, pos[k] + total, 4, cudaMemcpyDeviceToHost, s));
            CK(cudaStreamSynchronize(s));
            for (int k = 0; k < 3; ++k) hshort[k] = stage[1 + k];
            CK(arena_alloc(lists, &near, (size_t)hshort[0] + 1));
            CK(arena_alloc(lists, &p2l, (size_t)hshort[1] + 1));
            CK(arena_alloc(lists, &m2p, (size_t)hshort[2] + 1));
            launch_k(k_short_scatter, grid, 256, 0, s, l, R, cand_off, fl[0], fl[1], fl[2], pos[0],
                     pos[1], pos[2], cand_box, near, p2l, m2p);
            CK(cudaGetLastError());
            launch_k(k_short_offsets, nblk(nbl + 1, 256), 256, 0, s, l, R, cand_off, pos[0], pos[1],
                     pos[2], near_off, p2l_off, m2p_off);
            CK(cudaGetLastError());
        }
    }
    cand.release();
    const int *p2p_off = shortcut ? near_off : strong_off;
    const int *p2p_list = shortcut ? near : strong;
    // work items over the target leaves: chunks of <= P2P_CHUNK targets times
    // runs of <= t.p2p_cap near-field sources (and of <= M2P_RUN M2P boxes)
    const int64_t nleaf = (int64_t)R << (2 * L), leaf0 = R * lb(L);
    // (skipped when the caller evaluates the near field with its own items)
    uint32_t *chunks_cnt, *items_p2p, *items_cnt;
    CK(arena_alloc(tmp, &chunks_cnt, nleaf + 1));
    CK(arena_alloc(tmp, &items_p2p, nleaf + 1));
    CK(arena_alloc(tmp, &items_cnt, nleaf + 1));
    if (t.p2p_items_needed) {
        launch_k(k_leaf_chunks, nblk(nleaf, 256), 256, 0, s, nleaf, leaf0, t.box_tgt, P2P_CHUNK,
                 chunks_cnt);
        CK(cudaGetLastError());
        launch_k(k_leaf_runs, nblk(nleaf, 128), 128, 0, s, nleaf, leaf0, p2p_off, p2p_list,
                 t.box_src, chunks_cnt, t.p2p_cap, m2p_off, items_cnt, items_p2p);
        CK(cudaGetLastError());
        uint32_t *arr3[3] = {chunks_cnt, items_cnt, items_p2p};
        const uint32_t *in3[3] = {chunks_cnt, items_cnt, items_p2p};
        CK(exclusive_scan_u32_sets(3, in3, arr3, nleaf, tmp, s));
    } else {
        CK(cudaMemsetAsync(chunks_cnt + nleaf, 0, 4, s));
        CK(cudaMemsetAsync(items_cnt + nleaf, 0, 4, s));
        CK(cudaMemsetAsync(items_p2p + nleaf, 0, 4, s));
    }
    // stage words 4..9: items, weak, strong, chunks, all items, status
    CK(cudaMemcpyAsync(stage + 4, items_p2p + nleaf, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(stage + 5, weak_off + nb, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(stage + 6, strong_off + nb, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(stage + 7, chunks_cnt + nleaf, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(stage + 8, items_cnt + nleaf, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(stage + 9, t.status, 4, cudaMemcpyDeviceToHost, s));
    if (pre_sync) {
        // the caller's work on the finished lists shares this synchronisation
        t.near_off = near_off;
        t.near = near;
        t.m2p_off = m2p_off;
        t.p2p_list = shortcut ? near : strong;
        t.p2p_off = shortcut ? near_off : strong_off;
        t.weak_off = weak_off;
        t.strong_off = strong_off;
        fmm_status pst = pre_sync();
        if (pst != FMM_OK) {
            tmp.release();
            lists.release();
            dev_free(weak, s);
            dev_free(strong, s);
            return pst;
        }
    }
    CK(cudaStreamSynchronize(s));
    const int host[5] = {(int)stage[5], (int)stage[6], (int)stage[7], (int)stage[8], (int)stage[4]};
    const int hstat = (int)stage[9];
    if (hstat & ST_LIST_OVERFLOW) {
        tmp.release();
        lists.release();
        dev_free(weak, s);
        dev_free(strong, s);
        set_error("interaction list capacity exceeded");
        return FMM_ERR_CUDA;
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
    if (t.p2p_items_needed) {
        launch_k(k_fill_items, nblk(nleaf, 128), 128, 0, s, nleaf, leaf0, t.box_tgt, t.box_src,
                 p2p_off, p2p_list, m2p_off, P2P_CHUNK, t.p2p_cap, chunks_cnt, items_cnt, chunks,
                 item0, items, key, val);
        CK(cudaGetLastError());
        launch_k(k_set_last, 1, 1, 0, s, item0, n_chunks, n_items);
        CK(cudaGetLastError());
        if (n_items > 1)
            CK(radix_sort_pairs(&key, &val, kalt, valt, n_items, shortcut ? 0x1fu : 0xfu, tmp, s));
        launch_k(k_copy_u32, nblk(n_items, 256), 256, 0, s, n_items, val, order);
        CK(cudaGetLastError());
    }
    tmp.release();
    // hand the lists over to the tree
    for (void *p : lists.ptrs) t.mem.ptrs.push_back(p);
    lists.ptrs.clear();
    t.mem.ptrs.push_back(weak);
    t.mem.ptrs.push_back(strong);
    t.weak_off = weak_off;
    t.weak = weak;
    t.strong_off = strong_off;
    t.strong = strong;
    t.n_weak = host[0];
    t.n_strong = host[1];
    t.near_off = near_off;
    t.near = near;
    t.p2l_off = p2l_off;
    t.p2l = p2l;
    t.m2p_off = m2p_off;
    t.m2p = m2p;
    t.n_near = hshort[0];
    t.n_p2l = hshort[1];
    t.n_m2p = hshort[2];
    t.p2p_list = p2p_list;
    t.p2p_off = p2p_off;
    t.p2p_items = items;
    t.n_items = n_items;
    t.n_p2p_items = host[4];
    t.p2p_order = order;
    t.p2p_chunks = chunks;
    t.p2p_item0 = item0;
    t.n_chunks = n_chunks;
    t.p2p_partial = partial;
#undef CK
    return FMM_OK;
}

}  // namespace gbfmm
