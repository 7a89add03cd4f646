// Leaf shortcut (Sec. 2): at the finest level, a strongly coupled pair of
// leaves (t, s) that meets the theta-criterion with r and R interchanged is
// handled through one expansion instead of the direct sum:
//
//   P2L  (s larger than t)  the sources of s go straight into t's local
//        expansion:  b_0 += q Log(c_t - x),  b_l += -q / (l (x - c_t)^l);
//   M2P  (s smaller than t) s's multipole is evaluated at t's points:
//        a_0 Log(y - c_s) + sum_k a_k / (y - c_s)^k.
//
// Radius-normalised (sigma = 2^e >= radius, as in expand.cu):
//   P2L  W = sigma_t / (x - c_t),  B_0 += q Log(c_t - x),  B_l += -q W^l / l
//   M2P  W = sigma_s / (y - c_s),  value = A_0 Log(y - c_s) + sum_k A_k W^k
// The swapped test gives |W| <= sigma / (2 r) < 1 in both cases.
//
// P2L runs after L2L and adds into the leaf's local (one warp per target
// leaf, one source per lane, a warp reduction per coefficient).  M2P runs
// over work items (leaf, chunk of <= 64 evaluation points, run of <= 16 M2P
// boxes; one thread per point, Horner's rule) whose partial sums the combine
// kernel adds with the P2P items' partial sums, in item order, so that long
// M2P lists (a large leaf next to a dense cluster) do not form a tail.  FP64
// kernels serve FMM_PREC_FP64; FMM_PREC_MIXED uses double-float versions
// (positions as df32 offsets re-based between the two leaf centres, as in
// the mixed P2P) for p <= 32, and the FP64 kernels above that.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "df32.cuh"
#include "internal.h"

namespace gbfmm {

namespace {

// This translation unit's copy of the df32 tables.
__device__ __align__(16) float d_dftab_sc[DF_TAB_FLOATS];

constexpr int SC_THREADS = 64;   // M2P: evaluation points per work item
constexpr int SC_MIXED_MAXP = 32;
constexpr int M2P_RUN_MAX = 16;  // M2P list entries per work item (connect.cu)

GBI cd warp_sum_cd(cd v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.re += shfl_xor_d(v.re, o);
        v.im += shfl_xor_d(v.im, o);
    }
    return v;
}

// ------------------------------------------------------------------ FP64

// P2L, FP64: one warp per target leaf (entries of `leaves`).
__global__ void k_p2l64(int64_t nleaf, const int *__restrict__ leaves, int p,
                        const int *__restrict__ p2l_off, const int *__restrict__ p2l,
                        const int2 *__restrict__ box_src, const double4 *__restrict__ geom,
                        const double2 *__restrict__ xs, const double2 *__restrict__ qs,
                        double2 *__restrict__ local) {
    pdl_wait();
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nleaf) return;
    const int64_t g = leaves[w];
    const int e0 = p2l_off[g], e1 = p2l_off[g + 1];
    if (e0 == e1) return;
    const double4 gt = geom[g];
    cd acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int e = e0; e < e1; ++e) {
        const int2 bs = box_src[p2l[e]];
        for (int c0 = 0; c0 < bs.y; c0 += 32) {
            const int j = c0 + lane;
            cd W{0, 0}, q{0, 0}, lg{0, 0};
            if (j < bs.y) {
                const double2 x = xs[bs.x + j], qq = qs[bs.x + j];
                q = cd{qq.x, qq.y};
                W = cscale(cinv(cd{x.x - gt.x, x.y - gt.y}), gt.z);
                // Log(c_t - x) from the coordinates (an exactly shared ordinate gives +0)
                lg = cmul(q, clog_principal(cd{gt.x - x.x, gt.y - x.y}));
            }
            lg = warp_sum_cd(lg);
            if (lane == 0) acc[0] = cadd(acc[0], lg);
            cd pw = q;
            for (int k = 1; k <= p; ++k) {
                pw = cmul(pw, W);
                cd t = warp_sum_cd(pw);
                if (lane == (k & 31)) acc[k >> 5] = cadd(acc[k >> 5], cscale(t, -1.0 / k));
            }
        }
    }
    double2 *out = local + g * (p + 1);
    for (int j = 0; j < 3; ++j) {
        const int k = lane + 32 * j;
        if (k <= p) {
            double2 o = out[k];
            out[k] = make_double2(o.x + acc[j].re, o.y + acc[j].im);
        }
    }
}

// M2P, FP64: one CTA per M2P work item (leaf, chunk of <= 64 evaluation
// points, run of <= M2P_RUN entries of the leaf's M2P list), one thread per
// point; writes the item's partial sums.
// KERN 1 (harmonic kernel): -d/dy of the M2P value, (sum_k k A_k W^k - A_0) / (y - c_s).
template <int KERN>
__global__ void __launch_bounds__(SC_THREADS)
    k_m2p64(const int4 *__restrict__ items, const int *__restrict__ order, int p,
            const int2 *__restrict__ box_tgt, const double4 *__restrict__ geom,
            const int *__restrict__ m2p, const double2 *__restrict__ xt,
            const double2 *__restrict__ mpole, double2 *__restrict__ partial) {
    pdl_wait();
    __shared__ double2 sa[M2P_RUN_MAX][MAXP + 1];
    const int idx = order[blockIdx.x];
    const int4 it = items[idx];
    const int64_t g = it.x;
    const int e0 = ~it.z, ne = ~it.w - e0;
    for (int i = threadIdx.x; i < ne * (p + 1); i += SC_THREADS) {
        const int j = i / (p + 1), k = i - j * (p + 1);
        sa[j][k] = mpole[(int64_t)m2p[e0 + j] * (p + 1) + k];
    }
    __syncthreads();
    const int2 bt = box_tgt[g];
    const int nt = min(SC_THREADS, bt.y - it.y);
    if ((int)threadIdx.x >= nt) return;
    const double2 y = xt[(int64_t)bt.x + it.y + threadIdx.x];
    cd acc{0, 0};
    for (int j = 0; j < ne; ++j) {
        const double4 gs = geom[m2p[e0 + j]];
        const cd z{y.x - gs.x, y.y - gs.y};
        const cd iz = cinv(z);
        const cd W = cscale(iz, gs.z);
        if (KERN == 1) {
            cd h = cscale(cd{sa[j][p].x, sa[j][p].y}, (double)p);
            for (int k = p - 1; k >= 1; --k)
                h = cadd(cmul(h, W), cscale(cd{sa[j][k].x, sa[j][k].y}, (double)k));
            h = cmul(h, W);
            acc = cadd(acc, cmul(csub(h, cd{sa[j][0].x, sa[j][0].y}), iz));
        } else {
            cd h{sa[j][p].x, sa[j][p].y};
            for (int k = p - 1; k >= 1; --k) h = cadd(cmul(h, W), cd{sa[j][k].x, sa[j][k].y});
            h = cmul(h, W);
            acc = cadd(acc, cadd(h, cmul(cd{sa[j][0].x, sa[j][0].y}, clog_principal(z))));
        }
    }
    partial[(int64_t)idx * SC_THREADS + threadIdx.x] = make_double2(acc.re, acc.im);
}

// ------------------------------------------------------------------ df32

GBI df split_d(double v) {
    float hi = __double2float_rn(v);
    float lo = __double2float_rn(v - (double)hi);
    return df{hi, lo};
}

struct dc {
    df re, im;
};

GBI dc dc_add(const dc &a, const dc &b) { return dc{df_add(a.re, b.re), df_add(a.im, b.im)}; }

GBI dc dc_mul(const dc &a, const dc &b) {
    return dc{df_dot2(a.re, b.re, df_neg(a.im), b.im), df_dot2(a.re, b.im, a.im, b.re)};
}

// a b with the low parts left unnormalised (powers chains)
GBI dc dc_mul_lz(const dc &a, const dc &b) {
    return dc{df_dot2_lz(a.re, b.re, df_neg(a.im), b.im), df_dot2_lz(a.re, b.im, a.im, b.re)};
}

// h W + a (a Horner step), low parts left unnormalised
GBI dc dc_fma(const dc &h, const dc &W, const dc &a) {
    return dc{df_dot2_add_lz(h.re, W.re, df_neg(h.im), W.im, a.re),
              df_dot2_add_lz(h.re, W.im, h.im, W.re, a.im)};
}

GBI dc dc_scalef(const dc &a, float s) {  // s a power of two: exact
    return dc{df{a.re.hi * s, a.re.lo * s}, df{a.im.hi * s, a.im.lo * s}};
}

// The first power k at which |W|^k <= 2^-25, from w2 = |W|^2 (W a P2L / M2P
// ratio, |W| < 1): a term c W^k from there on carries at most 2^-24 of
// relative error in float, i.e. at most 2^-49 |c|, below the double-float
// rounding of the leading terms, so those powers (and Horner steps) run in
// float.  The fast log2 is an upper bound after the 2^-10 margin (its error
// is below 2^-21 absolute near 1 and 2 ulps elsewhere); p + 1 (no float
// part) when |W|^2 >= 2^-0.5 or when no k <= p qualifies; at least 1.
GBI int float_tail_start(float w2, int p) {
    const float l = __log2f(w2) + 0x1p-10f;
    if (!(l < -0.5f)) return p + 1;
    return max(1, min((int)ceilf(-50.0f / l), p + 1));
}

// 1/z = conj(z) / |z|^2 with one Newton step on 1/|z|^2.
GBI dc dc_inv(const dc &z) {
    const df inv = df_recip(df_dot2(z.re, z.re, z.im, z.im));
    return dc{df_mul(z.re, inv), df_neg(df_mul(z.im, inv))};
}

// Principal Log(z 2^ep) of a df32 complex z != 0 in pair units (z.im snapped
// by the caller), ecst = log_ecst(2 ep):
// 0.5 ln |z_hi|^2 + ep ln 2 + i atan2(z_hi) + z_lo / z_hi to first order.
GBI dc dc_log(const dc &z, const float *tab, const float *atab, float ecst) {
    const df Ex = z.re, Ey = z.im;
    df p1 = two_prod(Ex.hi, Ex.hi), p2 = two_prod(Ey.hi, Ey.hi);
    df S = two_sum(p1.hi, p2.hi);
    float slo = F_ADD(S.lo, F_ADD(p1.lo, p2.lo));
    float inv = F_RCP(S.hi);
    df ln = df_log_f(S.hi, tab, ecst);
    df an = df_atan2_f(Ey.hi, Ex.hi, atab);
    float cr = F_MUL(F_FMA(Ex.lo, Ex.hi, F_MUL(Ey.lo, Ey.hi)), inv);
    float ci = F_MUL(F_FMA(Ey.lo, Ex.hi, -F_MUL(Ex.lo, Ey.hi)), inv);
    df Lr = fast_sum(F_MUL(0.5f, ln.hi), F_FMA(0.5f, F_FMA(slo, inv, ln.lo), cr));
    df Li = fast_sum(an.hi, F_ADD(an.lo, ci));
    return dc{Lr, Li};
}

GBI double df_to_d(df v) { return (double)v.hi + (double)v.lo; }

// Rounding level of the re-based offsets of a leaf pair in pair units (as in
// the mixed P2P; f_a, f_b the two radii in those units): differences at or
// below it are the same coordinate.
GBI float pair_tau(df Dx, df Dy, float f_a, float f_b) {
    return (fabsf(Dx.hi) + fabsf(Dy.hi) + 2.0f * (f_a + f_b)) * 0x1p-42f;
}

GBI df shfl_lane_df(df v, int lane) {
    return df{__shfl_sync(0xffffffffu, v.hi, lane), __shfl_sync(0xffffffffu, v.lo, lane)};
}

// lazily normalised df32 accumulation (normalise before combining sums)
GBI df df_acc(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    return df{s.hi, F_ADD(s.lo, F_ADD(a.lo, b.lo))};
}

// P2L, df32: one warp per target leaf.  The sources of the leaf's P2L boxes
// are dealt to the lanes round-robin across box boundaries; every lane keeps
// its own sums of q Log(c_t - x) and q W^k (k = 1..p): coefficients below
// P2L_KREG in registers, the others in shared memory (rows of 33 float4 per
// coefficient: lane-private slots, conflict-free both ways), so the rest of
// the coefficient loop stays a short runtime loop.  At the end the register
// sums are added over the 32 lanes by a butterfly (the same total in every
// lane), lane k adds up a shared-memory coefficient k over the lanes in lane
// order, and each sum, scaled by -1/k in FP64, goes to the leaf's local
// expansion.
constexpr int P2L_WARPS = 4;
constexpr int P2L_ROW = 33;  // float4 per coefficient row (32 lanes + 1 pad)
constexpr int P2L_KREG = 8;  // coefficients 0 .. 7 summed in registers

GBI df shfl_xor_df(df v, int m) {
    return df{__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

__global__ void __launch_bounds__(32 * P2L_WARPS)
    k_p2l_mixed(int64_t nleaf, const int *__restrict__ leaves, int p,
                const int *__restrict__ p2l_off, const int *__restrict__ p2l,
                const int2 *__restrict__ box_src, const double4 *__restrict__ geom,
                const float4 *__restrict__ xs_loc, const float4 *__restrict__ qs,
                double2 *__restrict__ local) {
    pdl_wait();
    // the log / arctangent tables are read from global memory (L1-resident):
    // one lookup per source, and the shared memory goes to the sums
    extern __shared__ float4 p2l_acc[];  // [warp][k - P2L_KREG][P2L_ROW]
    const float *tab = d_dftab_sc;
    const float *atab = tab + ATAN_OFF;
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * P2L_WARPS + wib;
    if (w >= nleaf) return;
    const int64_t g = leaves[w];
    const int e0 = p2l_off[g], e1 = p2l_off[g + 1];
    if (e0 == e1) return;
    const int nrow = max(p + 1 - P2L_KREG, 0);
    float4 *acc = p2l_acc + (size_t)wib * nrow * P2L_ROW;
    for (int k = 0; k < nrow; ++k) acc[k * P2L_ROW + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    df sr[P2L_KREG], si[P2L_KREG];
#pragma unroll
    for (int k = 0; k < P2L_KREG; ++k) sr[k] = si[k] = df{0.f, 0.f};
    const double4 gt = geom[g];
    int done = 0;  // sources of the list before the current box
    for (int c0 = e0; c0 < e1; c0 += 32) {
        // the geometry of 32 boxes of the list, one per lane (the FP64 pipe is
        // narrow: each box's offsets are formed once, then broadcast), in the
        // units of the leaf pair (PairUnits)
        int2 bs_l = make_int2(0, 0);
        df Dx_l{0.f, 0.f}, Dy_l{0.f, 0.f};
        float tau_l = 0.f;
        PairUnits u_l{1.f, 1.f, LOG_ECST0, 0};
        if (c0 + lane < e1) {
            const int sb = p2l[c0 + lane];
            bs_l = box_src[sb];
            const double4 gs = geom[sb];
            u_l = pair_units(gt.z, gs.z);
            const double inv = pow2d(-u_l.ep);
            Dx_l = split_d((gs.x - gt.x) * inv);  // c_s - c_t
            Dy_l = split_d((gs.y - gt.y) * inv);
            tau_l = pair_tau(Dx_l, Dy_l, u_l.fs, u_l.ft);
        }
        const int nbx = min(32, e1 - c0);
        for (int bi = 0; bi < nbx; ++bi) {
            const int2 bs = make_int2(__shfl_sync(0xffffffffu, bs_l.x, bi),
                                      __shfl_sync(0xffffffffu, bs_l.y, bi));
            const df Dx = shfl_lane_df(Dx_l, bi), Dy = shfl_lane_df(Dy_l, bi);
            const float tau = __shfl_sync(0xffffffffu, tau_l, bi);
            const float ft = __shfl_sync(0xffffffffu, u_l.ft, bi);
            const float fs = __shfl_sync(0xffffffffu, u_l.fs, bi);
            const float ecst = __shfl_sync(0xffffffffu, u_l.ecst, bi);
            for (int j = (lane - done % 32 + 32) % 32; j < bs.y; j += 32) {
                const float4 xl = xs_loc[bs.x + j], qq = qs[bs.x + j];
                const dc q{df{qq.x, qq.y}, df{qq.z, qq.w}};
                // d = x - c_t = (c_s - c_t) + (x - c_s), in pair units
                const dc d{df_add(Dx, df{F_MUL(xl.x, fs), F_MUL(xl.y, fs)}),
                           df_add(Dy, df{F_MUL(xl.z, fs), F_MUL(xl.w, fs)})};
                const dc W = dc_scalef(dc_inv(d), ft);  // sigma_t / (x - c_t)
                dc m{df_neg(d.re), df_neg(d.im)};  // c_t - x
                if (fabsf(m.im.hi) <= tau) m.im = df{0.0f, 0.0f};
                const dc lg = dc_mul(q, dc_log(m, tab, atab, ecst));
                sr[0] = df_acc(sr[0], lg.re);
                si[0] = df_acc(si[0], lg.im);
                dc pw = q;
#pragma unroll
                for (int k = 1; k < P2L_KREG; ++k) {
                    if (k <= p) {  // uniform
                        pw = dc_mul_lz(pw, W);
                        sr[k] = df_acc(sr[k], pw.re);
                        si[k] = df_acc(si[k], pw.im);
                    }
                }
                const int kf = max(P2L_KREG, float_tail_start(
                                                  F_FMA(W.re.hi, W.re.hi, F_MUL(W.im.hi, W.im.hi)), p));
                int k = P2L_KREG;
#pragma unroll 2
                for (; k < kf; ++k) {
                    pw = dc_mul_lz(pw, W);
                    float4 *ak = acc + (k - P2L_KREG) * P2L_ROW + lane;
                    const float4 a = *ak;
                    const df r = df_acc(df{a.x, a.y}, pw.re), i = df_acc(df{a.z, a.w}, pw.im);
                    *ak = make_float4(r.hi, r.lo, i.hi, i.lo);
                }
                if (k <= p) {
                    // |W|^k <= 2^-25 from here on: q W^k in float (float_tail_start)
                    float pr = F_ADD(pw.re.hi, pw.re.lo), pi = F_ADD(pw.im.hi, pw.im.lo);
                    const float wr = W.re.hi, wi = W.im.hi;
                    for (; k <= p; ++k) {
                        const float nr = F_FMA(pr, wr, -F_MUL(pi, wi));
                        pi = F_FMA(pr, wi, F_MUL(pi, wr));
                        pr = nr;
                        float4 *ak = acc + (k - P2L_KREG) * P2L_ROW + lane;
                        const float4 a = *ak;
                        const df r = two_sum(a.x, pr), i = two_sum(a.z, pi);
                        *ak = make_float4(r.hi, F_ADD(r.lo, a.y), i.hi, F_ADD(i.lo, a.w));
                    }
                }
            }
            done += bs.y;
        }
    }
    __syncwarp();
    double2 *out = local + g * (p + 1);
#pragma unroll
    for (int k = 0; k < P2L_KREG; ++k) {
        df r = fast_sum(sr[k].hi, sr[k].lo), i = fast_sum(si[k].hi, si[k].lo);
#pragma unroll
        for (int m = 16; m >= 1; m >>= 1) {
            r = df_add(r, shfl_xor_df(r, m));
            i = df_add(i, shfl_xor_df(i, m));
        }
        if (lane == k && k <= p) {
            const double f = k == 0 ? 1.0 : -1.0 / k;
            const double2 o = out[k];
            out[k] = make_double2(o.x + f * df_to_d(r), o.y + f * df_to_d(i));
        }
    }
    for (int k = lane + P2L_KREG; k <= p; k += 32) {
        df r{0.f, 0.f}, i{0.f, 0.f};
        for (int j = 0; j < 32; ++j) {
            const float4 a = acc[(k - P2L_KREG) * P2L_ROW + j];
            r = df_add(r, fast_sum(a.x, a.y));
            i = df_add(i, fast_sum(a.z, a.w));
        }
        const double f = -1.0 / k;
        const double2 o = out[k];
        out[k] = make_double2(o.x + f * df_to_d(r), o.y + f * df_to_d(i));
    }
}

// M2P, df32: as k_m2p64; the Horner steps from the first k with |W|^k <= 2^-25
// on run in float (float_tail_start), the rest in double-float.
template <int KERN>
__global__ void __launch_bounds__(SC_THREADS)
    k_m2p_mixed(const int4 *__restrict__ items, const int *__restrict__ order, int p,
                const int2 *__restrict__ box_tgt, const double4 *__restrict__ geom,
                const int *__restrict__ m2p, const float4 *__restrict__ xt_loc,
                const float4 *__restrict__ mp, double2 *__restrict__ partial) {
    pdl_wait();
    __shared__ __align__(16) float tab[DF_TAB_FLOATS];
    __shared__ float4 sa[M2P_RUN_MAX][SC_MIXED_MAXP + 1];
    __shared__ float4 sD[M2P_RUN_MAX];      // c_t - c_s of every box as df32 (x, y), pair units
    __shared__ float4 stau[M2P_RUN_MAX];    // (rounding level, sigma_s, sigma_t, log constant)
    __shared__ double sinv[M2P_RUN_MAX];    // 2^-ep of every box (pair units -> absolute)
    for (int i = threadIdx.x; i < DF_TAB_FLOATS; i += SC_THREADS) tab[i] = d_dftab_sc[i];
    const float *atab = tab + ATAN_OFF;
    const int idx = order[blockIdx.x];
    const int4 it = items[idx];
    const int64_t g = it.x;
    const int e0 = ~it.z, ne = ~it.w - e0;
    const double4 gt = geom[g];
    for (int i = threadIdx.x; i < ne * (p + 1); i += SC_THREADS) {
        const int j = i / (p + 1), k = i - j * (p + 1);
        sa[j][k] = mp[(int64_t)m2p[e0 + j] * (p + 1) + k];
    }
    if ((int)threadIdx.x < ne) {
        // box geometry once per block (the FP64 pipe is narrow)
        const double4 gs = geom[m2p[e0 + threadIdx.x]];
        const PairUnits u = pair_units(gt.z, gs.z);
        const double inv = pow2d(-u.ep);
        const df Dx = split_d((gt.x - gs.x) * inv), Dy = split_d((gt.y - gs.y) * inv);  // c_t - c_s
        sD[threadIdx.x] = make_float4(Dx.hi, Dx.lo, Dy.hi, Dy.lo);
        stau[threadIdx.x] = make_float4(pair_tau(Dx, Dy, u.fs, u.ft), u.fs, u.ft, u.ecst);
        sinv[threadIdx.x] = inv;
    }
    __syncthreads();
    const int2 bt = box_tgt[g];
    const int nt = min(SC_THREADS, bt.y - it.y);
    if ((int)threadIdx.x >= nt) return;
    // this point's offset, in units of the target leaf's sigma
    const float4 yl = xt_loc[(int64_t)bt.x + it.y + threadIdx.x];
    dc acc{{0.f, 0.f}, {0.f, 0.f}};
    double hr = 0.0, hi_ = 0.0;  // harmonic kernel: terms in absolute units
    for (int j = 0; j < ne; ++j) {
        const float4 d4 = sD[j];
        const float4 ts = stau[j];
        const df Dx{d4.x, d4.y}, Dy{d4.z, d4.w};
        // z = y - c_s = (c_t - c_s) + (y - c_t), in pair units
        dc z{df_add(Dx, df{F_MUL(yl.x, ts.z), F_MUL(yl.y, ts.z)}),
             df_add(Dy, df{F_MUL(yl.z, ts.z), F_MUL(yl.w, ts.z)})};
        if (fabsf(z.im.hi) <= ts.x) z.im = df{0.0f, 0.0f};
        const dc iz = dc_inv(z);
        const dc W = dc_scalef(iz, ts.y);  // sigma_s / (y - c_s)
        const dc a0{df{sa[j][0].x, sa[j][0].y}, df{sa[j][0].z, sa[j][0].w}};
        // Horner from k = p down; the steps k >= kf (|W|^kf <= 2^-25) in float
        const int kf = float_tail_start(F_FMA(W.re.hi, W.re.hi, F_MUL(W.im.hi, W.im.hi)), p);
        const float wr = W.re.hi, wi = W.im.hi;
        if (KERN == 1) {
            dc h;
            int k = p - 1;
            if (kf <= p) {
                float hr = F_MUL(sa[j][p].x, (float)p), hi = F_MUL(sa[j][p].z, (float)p);
                for (; k >= kf; --k) {
                    const float nr = F_FMA(hr, wr, F_FMA(-hi, wi, F_MUL(sa[j][k].x, (float)k)));
                    hi = F_FMA(hr, wi, F_FMA(hi, wr, F_MUL(sa[j][k].z, (float)k)));
                    hr = nr;
                }
                h = dc{df{hr, 0.f}, df{hi, 0.f}};
            } else {
                h = dc{df_mulf(df{sa[j][p].x, sa[j][p].y}, (float)p),
                       df_mulf(df{sa[j][p].z, sa[j][p].w}, (float)p)};
            }
            for (; k >= 1; --k) {
                const dc ak{df_mulf(df{sa[j][k].x, sa[j][k].y}, (float)k),
                            df_mulf(df{sa[j][k].z, sa[j][k].w}, (float)k)};
                h = dc_fma(h, W, ak);
            }
            h = dc_mul(h, W);
            // 1/(y - c_s) = 2^-ep / z: this box's term added in FP64
            const dc tm = dc_mul(dc_add(h, dc{df_neg(a0.re), df_neg(a0.im)}), iz);
            hr += df_to_d(tm.re) * sinv[j];
            hi_ += df_to_d(tm.im) * sinv[j];
        } else {
            dc h;
            int k = p - 1;
            if (kf <= p) {
                float hr = sa[j][p].x, hi = sa[j][p].z;
                for (; k >= kf; --k) {
                    const float nr = F_FMA(hr, wr, F_FMA(-hi, wi, sa[j][k].x));
                    hi = F_FMA(hr, wi, F_FMA(hi, wr, sa[j][k].z));
                    hr = nr;
                }
                h = dc{df{hr, 0.f}, df{hi, 0.f}};
            } else {
                h = dc{df{sa[j][p].x, sa[j][p].y}, df{sa[j][p].z, sa[j][p].w}};
            }
            for (; k >= 1; --k)
                h = dc_fma(h, W, dc{df{sa[j][k].x, sa[j][k].y}, df{sa[j][k].z, sa[j][k].w}});
            h = dc_mul(h, W);
            acc = dc_add(acc, dc_add(h, dc_mul(a0, dc_log(z, tab, atab, ts.w))));
        }
    }
    partial[(int64_t)idx * SC_THREADS + threadIdx.x] =
        KERN == 1 ? make_double2(hr, hi_) : make_double2(df_to_d(acc.re), df_to_d(acc.im));
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

cudaError_t upload_df_tables_sc() {
    alignas(16) static float tab[DF_TAB_FLOATS];
    df32_fill_tables(tab);
    return cudaMemcpyToSymbol(d_dftab_sc, tab, sizeof(tab));
}

static bool mixed_ok(const Tree &t) {
    return t.precision == FMM_PREC_MIXED && t.p <= SC_MIXED_MAXP && t.mpole_df && t.xs_loc &&
           t.qs_df;
}

fmm_status launch_p2l(Tree &t, cudaStream_t s) {
    if (!t.p2l_m2p || t.n_p2l == 0) return FMM_OK;
    const int64_t nleaf = t.n_leaves;
    if (mixed_ok(t)) {
        const int smem =
            P2L_WARPS * std::max(t.p + 1 - P2L_KREG, 0) * P2L_ROW * (int)sizeof(float4);
        static const cudaError_t attr = cudaFuncSetAttribute(
            k_p2l_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
            P2L_WARPS * (SC_MIXED_MAXP + 1 - P2L_KREG) * P2L_ROW * (int)sizeof(float4));
        if (attr != cudaSuccess) return cuda_fail(attr, "p2l smem");
        launch_k(k_p2l_mixed, nblk(nleaf, P2L_WARPS), 32 * P2L_WARPS, smem, s, nleaf, t.leaves, t.p,
                 t.p2l_off, t.p2l, t.box_src, t.geom, t.xs_loc, t.qs_df, t.local);
    } else {
        launch_k(k_p2l64, nblk(nleaf * 32, 128), 128, 0, s, nleaf, t.leaves, t.p, t.p2l_off, t.p2l,
                 t.box_src, t.geom, t.xs, t.qs, t.local);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "p2l");
}

fmm_status launch_m2p_items(Tree &t, const int4 *items, const int *order, int n,
                            double2 *partial, cudaStream_t s) {
    if (n <= 0) return FMM_OK;
    if (mixed_ok(t)) {
        launch_k((t.kernel ? k_m2p_mixed<1> : k_m2p_mixed<0>), n, SC_THREADS, 0, s, items, order,
                 t.p, t.box_tgt, t.geom, t.m2p, t.xt_loc, t.mpole_df, partial);
    } else {
        launch_k((t.kernel ? k_m2p64<1> : k_m2p64<0>), n, SC_THREADS, 0, s, items, order, t.p,
                 t.box_tgt, t.geom, t.m2p, t.xt, t.mpole, partial);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "m2p");
}

fmm_status launch_m2p(Tree &t, cudaStream_t s) {
    const int n = t.n_items - t.n_p2p_items;
    if (!t.p2l_m2p || n <= 0) return FMM_OK;
    const int *order = t.p2p_order + t.n_p2p_items;
    if (mixed_ok(t)) {
        launch_k((t.kernel ? k_m2p_mixed<1> : k_m2p_mixed<0>), n, SC_THREADS, 0, s, t.p2p_items,
                 order, t.p, t.box_tgt, t.geom, t.m2p, t.xt_loc, t.mpole_df, t.p2p_partial);
    } else {
        launch_k((t.kernel ? k_m2p64<1> : k_m2p64<0>), n, SC_THREADS, 0, s, t.p2p_items, order, t.p,
                 t.box_tgt, t.geom, t.m2p, t.xt, t.mpole, t.p2p_partial);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "m2p");
}

}  // namespace gbfmm
