// Symmetric near field for self-evaluation (Eq. 1) in double-float.
//
// When the evaluation points are the sources, every near pair of distinct
// leaves (t, s) appears in both near lists (the theta-criterion and the
// swapped test are symmetric in the two boxes), and each point pair is
// needed in both directions.  With z = y_i - x_j the reverse term is
//   Log(x_j - y_i) = Log(-z) = Log(z) + i pi sgn,
//   sgn = +1 if Im z < 0, or Im z = 0 and Re z > 0;  -1 otherwise,
// which is exactly what a direct evaluation of x_j - y_i returns on the
// principal branch (an exactly shared ordinate gives +0 both ways).  So one
// logarithm serves both directions.
//
// Work items are (leaf t, run [e0, e1) of t's near list holding at most
// p2p_cap sources; a single leaf may exceed it); only entries s >= t are
// taken.  For s = t the item takes each unordered pair of the leaf once,
// in nt/2 steps of a cyclic schedule (thread i with point i + k mod nt),
// the reverse term passed through shared memory.  For s > t it evaluates the 64 x 64 tile once,
// 16 sources at a time: phase 1 (thread = target i of t) forms Log(z), adds
// q_j Log(z) to the row sum of i and stores Log(z) + i pi sgn in shared
// memory; phase 2 (thread = (source j of s, quarter of t's points)) forms
// sum_i q_i (Log(z) + i pi sgn) for the column.  Row sums (one per item)
// and column sums (one per item and s) land in separate slots of the
// partial buffer; every leaf's slots are listed in slot order, and the
// combine kernel adds them to the L2P value in that order (deterministic).
//
// Eligible: evaluation at the sources, at most 64 points per leaf (the leaf
// is one 64-point chunk).  The same items serve the FP64 path
// (k_p2p_sym64, FP64 differences and the CUDA math library's log).
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>

#include "common.cuh"
#include "df32.cuh"
#include "internal.h"

namespace gbfmm {

// This translation unit's copy of the df32 tables.
__device__ float d_dftab_sym[DF_TAB_FLOATS];

namespace {

constexpr int SY_THREADS = 64;
constexpr int SY_SUB = 16;        // sources per sub-tile
constexpr int SY_LSTRIDE = SY_SUB + 1;  // float4 per target row of the Log buffer (padded)
constexpr int SY_M2P_RUN = 16;    // M2P list entries per M2P item

GBI df split_d(double v) {
    float hi = __double2float_rn(v);
    float lo = __double2float_rn(v - (double)hi);
    return df{hi, lo};
}

// a - b for df32 a, b.  The closing Fast2Sum is exact when the low sum does
// not outgrow the high difference; otherwise (a high difference within a
// few ulps) its error is of the order of the rounding of al - bl, which the
// TwoSum form makes as well.
GBI df df_diff(float ah, float al, float bh, float bl) {
    df s = two_sum(ah, -bh);
    float lo = F_ADD(s.lo, F_SUB(al, bl));
    return fast_sum(s.hi, lo);
}

// Log(E 2^ep) of a df32 difference E in pair units (not coincident), as in
// the mixed P2P; ecst = log_ecst(2 ep).
GBI void df_clog(df Ex, df Ey, const float *tab, const float *atab, float ecst, df &Lr,
                 df &Li) {
    df p1 = two_prod(Ex.hi, Ex.hi), p2 = two_prod(Ey.hi, Ey.hi);
    df S = two_sum(p1.hi, p2.hi);
    float slo = F_ADD(S.lo, F_ADD(p1.lo, p2.lo));
    float inv = F_RCP(S.hi);
    df ln = df_log_f(S.hi, tab, ecst);
    df an = df_atan2_f(Ey.hi, Ex.hi, atab);
    float cr = F_MUL(F_FMA(Ex.lo, Ex.hi, F_MUL(Ey.lo, Ey.hi)), inv);
    float ci = F_MUL(F_FMA(Ey.lo, Ex.hi, -F_MUL(Ex.lo, Ey.hi)), inv);
    Lr = fast_sum(F_MUL(0.5f, ln.hi), F_FMA(0.5f, F_FMA(slo, inv, ln.lo), cr));
    Li = fast_sum(an.hi, F_ADD(an.lo, ci));
}

// Im Log(-z) = Im Log(z) + pi sgn for the reverse direction (sgn = +1 if
// Im z < 0, or Im z = 0 and Re z > 0; -1 otherwise).  |Im Log z| <= pi, so
// the high parts add by an exact Fast2Sum; the low part is left
// unnormalised (the multiply-accumulate takes it through an FMA).
GBI df rev_im(df Ex, df Ey, df Li) {
    const bool up = (Ey.hi < 0.0f) || (Ey.hi == 0.0f && Ex.hi > 0.0f);
    const float ph = up ? PI_HI : -PI_HI, pl = up ? PI_LO : -PI_LO;
    const df s = fast_sum(ph, Li.hi);
    return df{s.hi, F_ADD(s.lo, F_ADD(Li.lo, pl))};
}

// acc += q * L for df32 complex q = (q.x + q.y, q.z + q.w), L = (Lr, Li)
GBI void cmac(df &ar, df &ai, const float4 q, df Lr, df Li) {
    df a1 = two_prod(q.x, Lr.hi), a2 = two_prod(q.z, Li.hi);
    df b1 = two_prod(q.x, Li.hi), b2 = two_prod(q.z, Lr.hi);
    float rlo = F_FMA(q.x, Lr.lo, F_FMA(q.y, Lr.hi, F_SUB(a1.lo, a2.lo)));
    rlo = F_FMA(-q.z, Li.lo, F_FMA(-q.w, Li.hi, rlo));
    float ilo = F_FMA(q.x, Li.lo, F_FMA(q.y, Li.hi, F_ADD(b1.lo, b2.lo)));
    ilo = F_FMA(q.z, Lr.lo, F_FMA(q.w, Lr.hi, ilo));
    df s1 = two_sum(ar.hi, a1.hi);
    df s2 = two_sum(s1.hi, -a2.hi);
    ar = df{s2.hi, F_ADD(ar.lo, F_ADD(F_ADD(s1.lo, s2.lo), rlo))};
    df t1 = two_sum(ai.hi, b1.hi);
    df t2 = two_sum(t1.hi, b2.hi);
    ai = df{t2.hi, F_ADD(ai.lo, F_ADD(F_ADD(t1.lo, t2.lo), ilo))};
}

GBI df shfl_df(df v, int m) {
    return df{__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

// 1/E for a df32 complex E != 0: conj(E) / |E|^2 with one Newton step on 1/|E|^2.
GBI void df_cinv(df Ex, df Ey, df &Rr, df &Ri) {
    const df inv = df_recip(df_dot2(Ex, Ex, Ey, Ey));
    Rr = df_mul(Ex, inv);
    Ri = df_neg(df_mul(Ey, inv));
}

// Item = (leaf t, e0, e1, row slot); column slots follow the row slot, one
// per entry s > t of the run, in run order.  KERN 0: the log kernel (row term
// q_j Log(z), reverse Log(z) + i pi sgn); KERN 1: the harmonic kernel (row
// term q_j / (x_j - y_i) = -q_j / z, reverse q_i / z).
template <int KERN>
__global__ void __launch_bounds__(SY_THREADS)
    k_p2p_sym(const int4 *__restrict__ items, const int *__restrict__ order,
              const int2 *__restrict__ box_src, const double4 *__restrict__ geom,
              const int *__restrict__ list, const float4 *__restrict__ xs_loc,
              const float4 *__restrict__ qs, double2 *__restrict__ partial) {
    pdl_wait();
    __shared__ __align__(16) float tab[DF_TAB_FLOATS];
    __shared__ float4 sd[SY_SUB], sq[SY_SUB];
    __shared__ float4 sqi[SY_THREADS];
    __shared__ float4 lbuf[SY_THREADS * SY_LSTRIDE];
    __shared__ float4 red[SY_SUB][2];
    for (int i = threadIdx.x; i < DF_TAB_FLOATS; i += SY_THREADS) tab[i] = d_dftab_sym[i];
    const float *atab = tab + ATAN_OFF;
    const int tid = threadIdx.x;
    const int4 it = items[order[blockIdx.x]];
    const int64_t g = it.x;
    const int2 bt = box_src[g];
    const int nt = min(bt.y, SY_THREADS);  // <= 64 by eligibility; the clamp keeps accesses in bounds
    const bool valid = tid < nt;
    const double4 gt = geom[g];
    // this thread's point, in units of the leaf's sigma (rescaled per source leaf)
    const float4 et = valid ? xs_loc[bt.x + tid] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float4 qi = valid ? qs[bt.x + tid] : make_float4(0.f, 0.f, 0.f, 0.f);
    sqi[tid] = qi;
    // row sums: df32 within one source box (<= 64 terms), then added into FP64,
    // so the rounding of a run does not grow with its length
    df ar{0.f, 0.f}, ai{0.f, 0.f};
    double sr = 0.0, si = 0.0;
    int col = it.w + 1;
    // phase-2 mapping: source jl of the sub-tile, quarter part of the targets
    const int jl = tid & 15, part = tid >> 4;
    const int lane = tid & 31;
    for (int c0 = it.y; c0 < it.z; c0 += 32) {
      // the geometry of 32 entries of the run, one per lane of each warp (the
      // FP64 pipe is narrow: each box's offsets are formed once per warp), in
      // the units of the leaf pair (PairUnits)
      int sbox_l = -1;
      int2 bs_l = make_int2(0, 0);
      float4 D_l = make_float4(0.f, 0.f, 0.f, 0.f);
      float tau_l = 0.f;
      PairUnits u_l{1.f, 1.f, LOG_ECST0, 0};
      if (c0 + lane < it.z) {
          sbox_l = list[c0 + lane];
          bs_l = box_src[sbox_l];
          const double4 gs = geom[sbox_l];
          u_l = pair_units(gt.z, gs.z);
          const double inv = pow2d(-u_l.ep);
          const df Dx = split_d((gs.x - gt.x) * inv), Dy = split_d((gs.y - gt.y) * inv);
          D_l = make_float4(Dx.hi, Dx.lo, Dy.hi, Dy.lo);
          tau_l = (fabsf(Dx.hi) + fabsf(Dy.hi) + 2.0f * (u_l.fs + u_l.ft)) * 0x1p-42f;
      }
      const int nbx = min(32, it.z - c0);
      for (int bi = 0; bi < nbx; ++bi) {
        const int sbox = __shfl_sync(0xffffffffu, sbox_l, bi);
        if (sbox < g) continue;  // uniform over the CTA
        const int2 bs = make_int2(__shfl_sync(0xffffffffu, bs_l.x, bi),
                                  min(__shfl_sync(0xffffffffu, bs_l.y, bi), SY_THREADS));
        const df Dx{__shfl_sync(0xffffffffu, D_l.x, bi), __shfl_sync(0xffffffffu, D_l.y, bi)};
        const df Dy{__shfl_sync(0xffffffffu, D_l.z, bi), __shfl_sync(0xffffffffu, D_l.w, bi)};
        const float tau = __shfl_sync(0xffffffffu, tau_l, bi);
        const float tau2 = fmaxf(tau * tau, 1e-36f);
        const float ft = __shfl_sync(0xffffffffu, u_l.ft, bi);
        const float fs = __shfl_sync(0xffffffffu, u_l.fs, bi);
        const float ecst = __shfl_sync(0xffffffffu, u_l.ecst, bi);
        // 1/D = 2^-ep / D' for the harmonic kernel
        const double hs = KERN == 1 ? pow2d(-__shfl_sync(0xffffffffu, u_l.ep, bi)) : 1.0;
        const float4 e = make_float4(F_MUL(et.x, ft), F_MUL(et.y, ft), F_MUL(et.z, ft),
                                     F_MUL(et.w, ft));
        const bool self = sbox == g;
        if (self) {
            // The leaf with itself: every unordered pair once.  In step k
            // (1 .. nt/2) thread t takes the pair (t, u = t + k mod nt) (at
            // k = nt/2 with nt even only t < k), adds its row term to its own
            // sums and hands the reverse term (log kernel: q_t (Log(z) +
            // i pi sgn); harmonic: q_t / z) to point u through a shared slot;
            // t -> u is one-to-one, so every slot is written once per step.
            // (Here ft = fs = 1 and D = 0: the offsets are the points'.)
            float4 *spos = lbuf;               // the leaf's offsets
            float4 *srev = lbuf + SY_THREADS;  // the reverse terms of one step
            __syncthreads();  // the previous box's buffers fully consumed
            spos[tid] = e;
            __syncthreads();
            for (int k = 1; k <= nt / 2; ++k) {
                int u = tid + k;
                if (u >= nt) u -= nt;
                df rr{0.f, 0.f}, ri{0.f, 0.f};
                if (valid && (2 * k < nt || tid < k)) {
                    const float4 d = spos[u];
                    df Ex = df_diff(e.x, e.y, d.x, d.y);
                    df Ey = df_diff(e.z, e.w, d.z, d.w);
                    if (fabsf(Ey.hi) <= tau) Ey = df{0.0f, 0.0f};
                    const float S = F_FMA(Ex.hi, Ex.hi, F_MUL(Ey.hi, Ey.hi));
                    if (S > tau2 && KERN == 1) {  // else coincident: skipped both ways
                        df Rr, Ri;
                        df_cinv(Ex, Ey, Rr, Ri);
                        cmac(ar, ai, sqi[u], df_neg(Rr), df_neg(Ri));
                        cmac(rr, ri, qi, Rr, Ri);
                    } else if (S > tau2) {
                        df Lr, Li;
                        df_clog(Ex, Ey, tab, atab, ecst, Lr, Li);
                        cmac(ar, ai, sqi[u], Lr, Li);
                        cmac(rr, ri, qi, Lr, rev_im(Ex, Ey, Li));
                    }
                }
                if (valid) srev[u] = make_float4(rr.hi, rr.lo, ri.hi, ri.lo);
                __syncthreads();
                if (valid) {
                    const float4 v = srev[tid];
                    const df s1 = two_sum(ar.hi, v.x), s2 = two_sum(ai.hi, v.z);
                    ar = df{s1.hi, F_ADD(ar.lo, F_ADD(s1.lo, v.y))};
                    ai = df{s2.hi, F_ADD(ai.lo, F_ADD(s2.lo, v.w))};
                }
                __syncthreads();
            }
        }
        for (int j0 = 0; j0 < (self ? 0 : bs.y); j0 += SY_SUB) {
            const int nn = min(SY_SUB, bs.y - j0);
            __syncthreads();  // previous sub-tile fully consumed
            if (tid < nn) {
                const float4 xl = xs_loc[bs.x + j0 + tid];
                df dx = df_add(Dx, df{F_MUL(xl.x, fs), F_MUL(xl.y, fs)}),
                   dy = df_add(Dy, df{F_MUL(xl.z, fs), F_MUL(xl.w, fs)});
                sd[tid] = make_float4(dx.hi, dx.lo, dy.hi, dy.lo);
                sq[tid] = qs[bs.x + j0 + tid];
            }
            __syncthreads();
            // ---- phase 1: thread = target i
            for (int j = 0; j < nn; ++j) {
                float4 Lp = make_float4(0.f, 0.f, 0.f, 0.f);
                if (valid) {
                    const float4 d = sd[j];
                    df Ex = df_diff(e.x, e.y, d.x, d.y);
                    df Ey = df_diff(e.z, e.w, d.z, d.w);
                    if (fabsf(Ey.hi) <= tau) Ey = df{0.0f, 0.0f};
                    const float S = F_FMA(Ex.hi, Ex.hi, F_MUL(Ey.hi, Ey.hi));
                    if (S > tau2 && KERN == 1) {  // else coincident: skipped both ways
                        df Rr, Ri;
                        df_cinv(Ex, Ey, Rr, Ri);
                        cmac(ar, ai, sq[j], df_neg(Rr), df_neg(Ri));
                        Lp = make_float4(Rr.hi, Rr.lo, Ri.hi, Ri.lo);
                    } else if (S > tau2) {
                        df Lr, Li;
                        df_clog(Ex, Ey, tab, atab, ecst, Lr, Li);
                        cmac(ar, ai, sq[j], Lr, Li);
                        const df Lj = rev_im(Ex, Ey, Li);  // reverse direction
                        Lp = make_float4(Lr.hi, Lr.lo, Lj.hi, Lj.lo);
                    }
                }
                lbuf[tid * SY_LSTRIDE + j] = Lp;
            }
            __syncthreads();
            // ---- phase 2: thread = (source jl, targets [16 part, 16 part + 16))
            df cr{0.f, 0.f}, ci{0.f, 0.f};
            if (jl < nn) {
                const int i0 = 16 * part, i1 = min(i0 + 16, nt);
                for (int i = i0; i < i1; ++i) {
                    const float4 L = lbuf[i * SY_LSTRIDE + jl];
                    cmac(cr, ci, sqi[i], df{L.x, L.y}, df{L.z, L.w});
                }
            }
            cr = fast_sum(cr.hi, cr.lo);
            ci = fast_sum(ci.hi, ci.lo);
            cr = df_add(cr, shfl_df(cr, 16));  // parts 0 + 1 (warp 0), 2 + 3 (warp 1)
            ci = df_add(ci, shfl_df(ci, 16));
            if (tid >= 32 && part == 2) red[jl][0] = make_float4(cr.hi, cr.lo, ci.hi, ci.lo);
            __syncthreads();
            if (tid < 16 && jl < nn) {
                const float4 o = red[jl][0];
                const df rr = df_add(cr, df{o.x, o.y}), ii = df_add(ci, df{o.z, o.w});
                partial[(int64_t)col * SY_THREADS + j0 + jl] =
                    make_double2(((double)rr.hi + (double)rr.lo) * hs,
                                 ((double)ii.hi + (double)ii.lo) * hs);
            }
        }
        sr += ((double)ar.hi + (double)ar.lo) * hs;
        si += ((double)ai.hi + (double)ai.lo) * hs;
        ar = df{0.f, 0.f};
        ai = df{0.f, 0.f};
        if (!self) ++col;
      }
    }
    if (valid) partial[(int64_t)it.w * SY_THREADS + tid] = make_double2(sr, si);
}

// The same items in FP64 (the FP64 path): z = y_i - x_j in FP64, the log by
// the CUDA math library as in the per-point FP64 kernel; the reverse term of
// the log kernel is Log(z) + i pi sgn, of the harmonic kernel +q_i / z.
template <int KERN>
__global__ void __launch_bounds__(SY_THREADS)
    k_p2p_sym64(const int4 *__restrict__ items, const int *__restrict__ order,
                const int2 *__restrict__ box_src, const int *__restrict__ list,
                const double2 *__restrict__ xs, const double2 *__restrict__ qs,
                double2 *__restrict__ partial) {
    pdl_wait();
    __shared__ double2 sx[SY_SUB], sq[SY_SUB];
    __shared__ double2 sqi[SY_THREADS];
    __shared__ double2 lbuf[SY_THREADS * SY_LSTRIDE];
    __shared__ double2 red[SY_SUB];
    const int tid = threadIdx.x;
    const int4 it = items[order[blockIdx.x]];
    const int64_t g = it.x;
    const int2 bt = box_src[g];
    const int nt = min(bt.y, SY_THREADS);  // <= 64 by eligibility; the clamp keeps accesses in bounds
    const bool valid = tid < nt;
    const double2 y = valid ? xs[bt.x + tid] : make_double2(0.0, 0.0);
    sqi[tid] = valid ? qs[bt.x + tid] : make_double2(0.0, 0.0);
    double ar = 0.0, ai = 0.0;
    int col = it.w + 1;
    const int jl = tid & 15, part = tid >> 4;
    for (int e = it.y; e < it.z; ++e) {
        const int sbox = list[e];
        if (sbox < g) continue;  // uniform over the CTA
        const int2 bs = make_int2(box_src[sbox].x, min(box_src[sbox].y, SY_THREADS));
        const bool self = sbox == g;
        if (self) {
            // the leaf with itself, every unordered pair once (the cyclic
            // schedule of the mixed kernel above)
            double2 *srev = lbuf;
            __syncthreads();  // the previous box's buffers fully consumed
            lbuf[SY_THREADS + tid] = y;
            __syncthreads();
            for (int k = 1; k <= nt / 2; ++k) {
                int u = tid + k;
                if (u >= nt) u -= nt;
                double2 rv = make_double2(0.0, 0.0);
                if (valid && (2 * k < nt || tid < k)) {
                    const double2 xu = lbuf[SY_THREADS + u];
                    const double dx = y.x - xu.x, dy = y.y - xu.y;
                    if (!(dx == 0.0 && dy == 0.0)) {  // x_j == y_i: skipped both ways
                        const double2 qu = sqi[u], qt = sqi[tid];
                        double vr, vi, wr, wi;
                        if (KERN == 1) {
                            const double r = -1.0 / fma(dx, dx, dy * dy);
                            vr = dx * r;
                            vi = -dy * r;
                            wr = -vr;
                            wi = -vi;
                        } else {
                            vr = 0.5 * log(fma(dx, dx, dy * dy));
                            vi = atan2(dy, dx);
                            const bool up = dy < 0.0 || (dy == 0.0 && dx > 0.0);
                            wr = vr;
                            wi = vi + (up ? CUDART_PI : -CUDART_PI);
                        }
                        ar += qu.x * vr - qu.y * vi;
                        ai += qu.x * vi + qu.y * vr;
                        rv = make_double2(qt.x * wr - qt.y * wi, qt.x * wi + qt.y * wr);
                    }
                }
                if (valid) srev[u] = rv;
                __syncthreads();
                if (valid) {
                    ar += srev[tid].x;
                    ai += srev[tid].y;
                }
                __syncthreads();
            }
            continue;  // uniform
        }
        for (int j0 = 0; j0 < bs.y; j0 += SY_SUB) {
            const int nn = min(SY_SUB, bs.y - j0);
            __syncthreads();  // previous sub-tile fully consumed
            if (tid < nn) {
                sx[tid] = xs[bs.x + j0 + tid];
                sq[tid] = qs[bs.x + j0 + tid];
            }
            __syncthreads();
            // ---- phase 1: thread = target i
            for (int j = 0; j < nn; ++j) {
                double2 Lp = make_double2(0.0, 0.0);
                if (valid) {
                    const double dx = y.x - sx[j].x, dy = y.y - sx[j].y;
                    if (!(dx == 0.0 && dy == 0.0)) {  // x_j == y_i: skipped both ways
                        const double2 qj = sq[j];
                        double vr, vi;
                        if (KERN == 1) {
                            // q / (x - y) = -q conj(z) / |z|^2
                            const double r = -1.0 / fma(dx, dx, dy * dy);
                            vr = dx * r;
                            vi = -dy * r;
                        } else {
                            vr = 0.5 * log(fma(dx, dx, dy * dy));
                            vi = atan2(dy, dx);
                        }
                        ar += qj.x * vr - qj.y * vi;
                        ai += qj.x * vi + qj.y * vr;
                        if (KERN == 1) {
                            Lp = make_double2(-vr, -vi);  // 1 / (y - x) = -1 / (x - y)
                        } else {
                            // reverse direction: Log(-z) = Log(z) + i pi sgn
                            const bool up = dy < 0.0 || (dy == 0.0 && dx > 0.0);
                            Lp = make_double2(vr, vi + (up ? CUDART_PI : -CUDART_PI));
                        }
                    }
                }
                lbuf[tid * SY_LSTRIDE + j] = Lp;
            }
            __syncthreads();
            // ---- phase 2: thread = (source jl, targets [16 part, 16 part + 16))
            double cr = 0.0, ci = 0.0;
            if (jl < nn) {
                const int i0 = 16 * part, i1 = min(i0 + 16, nt);
                for (int i = i0; i < i1; ++i) {
                    const double2 L = lbuf[i * SY_LSTRIDE + jl];
                    const double2 qi = sqi[i];
                    cr += qi.x * L.x - qi.y * L.y;
                    ci += qi.x * L.y + qi.y * L.x;
                }
            }
            cr += shfl_xor_d(cr, 16);  // parts 0 + 1 (warp 0), 2 + 3 (warp 1)
            ci += shfl_xor_d(ci, 16);
            if (tid >= 32 && part == 2) red[jl] = make_double2(cr, ci);
            __syncthreads();
            if (tid < 16 && jl < nn) {
                const double2 o = red[jl];
                partial[(int64_t)col * SY_THREADS + j0 + jl] = make_double2(cr + o.x, ci + o.y);
            }
        }
        ++col;
    }
    if (valid) partial[(int64_t)it.w * SY_THREADS + tid] = make_double2(ar, ai);
}

// FP64 L2P (Horner's rule, as the per-point combine) plus the leaf's partial
// sums in slot order.
__global__ void __launch_bounds__(SY_THREADS)
    k_combine_sym64(const int *__restrict__ leaves, const int *__restrict__ coff,
                    const int *__restrict__ cslot, int p, const int2 *__restrict__ box_tgt,
                    const double4 *__restrict__ geom, const double2 *__restrict__ xt,
                    const uint32_t *__restrict__ tperm, const double2 *__restrict__ local,
                    const double2 *__restrict__ partial, double2 *__restrict__ phi, int kern) {
    pdl_wait();
    __shared__ double2 sb[MAXP + 1];
    const int b = blockIdx.x;
    const int64_t g = leaves[b];
    for (int i = threadIdx.x; i <= p; i += SY_THREADS) sb[i] = local[g * (p + 1) + i];
    __syncthreads();
    const int2 bt = box_tgt[g];
    if ((int)threadIdx.x >= bt.y) return;
    const int pos = bt.x + threadIdx.x;
    const double2 y = xt[pos];
    const double4 ge = geom[g];
    const cd w{(y.x - ge.x) * ge.w, (y.y - ge.y) * ge.w};
    cd acc;
    if (kern) {
        // -d/dy sum B_l w^l = -(1/sigma) sum l B_l w^(l-1)
        acc = cscale(cd{sb[p].x, sb[p].y}, (double)p);
        for (int l = p - 1; l >= 1; --l)
            acc = cadd(cmul(acc, w), cscale(cd{sb[l].x, sb[l].y}, (double)l));
        acc = cscale(acc, -ge.w);
    } else {
        acc = cd{sb[p].x, sb[p].y};
        for (int l = p - 1; l >= 0; --l) acc = cadd(cmul(acc, w), cd{sb[l].x, sb[l].y});
    }
    for (int k = coff[b]; k < coff[b + 1]; ++k) {
        const double2 v = partial[(int64_t)cslot[k] * SY_THREADS + threadIdx.x];
        acc.re += v.x;
        acc.im += v.y;
    }
    phi[tperm[pos]] = make_double2(acc.re, acc.im);
}

// L2P (Horner's rule in double-float on the local expansion, converted once
// per leaf) plus the leaf's partial sums in slot order (FP64).
__global__ void __launch_bounds__(SY_THREADS)
    k_combine_sym(const int *__restrict__ leaves, const int *__restrict__ coff,
                  const int *__restrict__ cslot, int p, const int2 *__restrict__ box_tgt,
                  const double4 *__restrict__ geom, const float4 *__restrict__ xt_loc,
                  const uint32_t *__restrict__ tperm, const double2 *__restrict__ local,
                  const double2 *__restrict__ partial, double2 *__restrict__ phi, int kern) {
    pdl_wait();
    __shared__ float4 sb[MAXP + 1];
    const int b = blockIdx.x;
    const int64_t g = leaves[b];
    for (int i = threadIdx.x; i <= p; i += SY_THREADS) {
        const double2 v = local[g * (p + 1) + i];
        const df re = split_d(v.x), im = split_d(v.y);
        sb[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    __syncthreads();
    const int2 bt = box_tgt[g];
    if ((int)threadIdx.x >= bt.y) return;
    const int pos = bt.x + threadIdx.x;
    const float4 yl = xt_loc[pos];  // w = (y - c) / sigma as df32
    const double isig = geom[g].w;  // power of two: exact scaling in FP64
    const df wr{yl.x, yl.y}, wi{yl.z, yl.w};
    // kern 0: sum B_l w^l;  kern 1: -d/dy of it, -(1/sigma) sum l B_l w^(l-1)
    const float fp = kern ? (float)p : 1.0f;
    df hr = df_mulf(df{sb[p].x, sb[p].y}, fp), hi = df_mulf(df{sb[p].z, sb[p].w}, fp);
    // h = h * w + (l) B_l
    if (kern) {
        for (int l = p - 1; l >= 1; --l)
            df_horner_step(hr, hi, wr, wi, df_mulf(df{sb[l].x, sb[l].y}, (float)l),
                           df_mulf(df{sb[l].z, sb[l].w}, (float)l));
    } else {
        for (int l = p - 1; l >= 0; --l)
            df_horner_step(hr, hi, wr, wi, df{sb[l].x, sb[l].y}, df{sb[l].z, sb[l].w});
    }
    const double sc = kern ? -isig : 1.0;  // a power of two: exact
    double ar = sc * ((double)hr.hi + (double)hr.lo), ai = sc * ((double)hi.hi + (double)hi.lo);
    for (int k = coff[b]; k < coff[b + 1]; ++k) {
        const double2 v = partial[(int64_t)cslot[k] * SY_THREADS + threadIdx.x];
        ar += v.x;
        ai += v.y;
    }
    phi[tperm[pos]] = make_double2(ar, ai);
}

// ---------------------------------------------------------------- items

// Runs of the entries s >= g of list [e0, e1) holding <= cap sources; the
// number of runs and of entries s > g.
GBI void upper_runs(const int *__restrict__ list, int e0, int e1, int64_t g,
                    const int2 *__restrict__ box_src, int cap, int &nruns, int &ncols) {
    nruns = 0;
    ncols = 0;
    int acc = 0;
    bool open = false;
    for (int e = e0; e < e1; ++e) {
        const int s = list[e];
        if (s < g) continue;
        const int n = box_src[s].y;
        if (!open || acc + n > cap) {
            ++nruns;
            acc = 0;
            open = true;
        }
        acc += n;
        if (s > g) ++ncols;
    }
}

__global__ void k_sym_count(int nleaf, int cap, const int *__restrict__ leaves,
                            const int *__restrict__ off, const int *__restrict__ list,
                            const int2 *__restrict__ box_src, const int *__restrict__ m2p_off,
                            uint32_t *n_items, uint32_t *n_slots, uint32_t *n_m2p,
                            int *leaf_of_box) {
    pdl_wait();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    const int64_t g = leaves[b];
    leaf_of_box[g] = b;
    int nr, nc;
    upper_runs(list, off[g], off[g + 1], g, box_src, cap, nr, nc);
    n_items[b] = (uint32_t)nr;
    n_slots[b] = (uint32_t)(nr + nc);
    n_m2p[b] = m2p_off ? (uint32_t)((m2p_off[g + 1] - m2p_off[g] + SY_M2P_RUN - 1) / SY_M2P_RUN)
                       : 0u;
}

// Items, their sort keys (decreasing cost), and for every slot the leaf
// that receives it.  M2P slots follow all P2P slots.
__global__ void k_sym_fill(int nleaf, int cap, const int *__restrict__ leaves,
                           const int *__restrict__ off,
                           const int *__restrict__ list, const int2 *__restrict__ box_src,
                           const int *__restrict__ m2p_off, const int *__restrict__ leaf_of_box,
                           const uint32_t *__restrict__ item_off,
                           const uint32_t *__restrict__ slot_off,
                           const uint32_t *__restrict__ m2p_item_off, uint32_t n_p2p_slots,
                           int4 *items, uint64_t *key, uint32_t *val, int4 *m2p_items,
                           uint32_t *recv) {
    pdl_wait();
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nleaf) return;
    const int64_t g = leaves[b];
    const int e0 = off[g], e1 = off[g + 1];
    const int nt = box_src[g].y;
    uint32_t it = item_off[b], slot = slot_off[b];
    int acc = 0, rs = -1, cols = 0;
    auto emit = [&](int re) {
        uint64_t cost = (uint64_t)nt * (uint64_t)acc;
        if (cost > 0xffffffffull) cost = 0xffffffffull;
        items[it] = make_int4((int)g, rs, re, (int)slot);
        key[it] = 0xffffffffull - cost;
        val[it] = it;
        recv[slot] = (uint32_t)b;  // row slot; its column slots are filled below
        ++it;
        slot += 1 + cols;
    };
    for (int e = e0; e < e1; ++e) {
        const int s = list[e];
        if (s < g) continue;
        const int n = box_src[s].y;
        if (rs >= 0 && acc + n > cap) {
            emit(e);
            rs = -1;
        }
        if (rs < 0) {
            rs = e;
            acc = 0;
            cols = 0;
        }
        acc += n;
        if (s > g) ++cols;
    }
    if (rs >= 0) emit(e1);
    // column slots: the m-th entry s > g of an item goes to slot row + 1 + m
    it = item_off[b];
    slot = slot_off[b];
    {
        int4 cur = items[it];
        int m = 0;
        for (int e = e0; e < e1; ++e) {
            const int s = list[e];
            if (s < g) continue;
            if (e >= cur.z) {  // next item
                slot += 1 + m;
                ++it;
                cur = items[it];
                m = 0;
            }
            if (s > g) {
                recv[slot + 1 + m] = (uint32_t)leaf_of_box[s];
                ++m;
            }
        }
    }
    if (m2p_off) {
        uint32_t k = m2p_item_off[b];
        const int m1 = m2p_off[g + 1];
        for (int e = m2p_off[g]; e < m1; e += SY_M2P_RUN, ++k) {
            m2p_items[k] = make_int4((int)g, 0, ~e, ~min(e + SY_M2P_RUN, m1));
            recv[n_p2p_slots + k] = (uint32_t)b;
        }
    }
}

// Launch order of the P2P items: classes of decreasing cost (key = 2^32 - 1
// - cost), eight per power of two (the three bits after the leading one),
// in any order within a class; cost 0 last.
constexpr int COST_CLASSES = 32 * 8 + 1;
GBI int cost_class(uint64_t key) {
    const uint32_t cost = (uint32_t)(0xffffffffull - key);
    if (!cost) return COST_CLASSES - 1;
    const int lz = __clz(cost);
    const uint32_t next3 = lz < 31 ? ((cost << (lz + 1)) >> 29) : 0u;
    return lz * 8 + 7 - (int)next3;
}

__global__ void k_cost_count(int64_t n, const uint64_t *__restrict__ key, uint32_t *cnt) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicAdd(&cnt[cost_class(key[i])], 1u);
}

__global__ void k_cost_place(int64_t n, const uint64_t *__restrict__ key,
                             const uint32_t *__restrict__ cnt, uint32_t *cursor, int *order) {
    pdl_wait();
    __shared__ uint32_t base[COST_CLASSES];
    if (threadIdx.x < 32) {
        // exclusive prefix of the class counts, one warp
        uint32_t carry = 0;
        for (int c0 = 0; c0 < COST_CLASSES; c0 += 32) {
            const int c = c0 + (int)threadIdx.x;
            const uint32_t v = c < COST_CLASSES ? cnt[c] : 0u;
            uint32_t x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, x, o);
                if ((int)threadIdx.x >= o) x += t;
            }
            if (c < COST_CLASSES) base[c] = carry + x - v;
            carry += __shfl_sync(0xffffffffu, x, 31);
        }
    }
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cost_class(key[i]);
    order[base[c] + atomicAdd(&cursor[c], 1u)] = (int)i;
}

__global__ void k_iota(int64_t n, uint32_t *v) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) v[i] = (uint32_t)i;
}

__global__ void k_to_u64(int64_t n, const uint32_t *__restrict__ in, uint64_t *out) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = in[i];
}

__global__ void k_hist_recv(int64_t n, const uint32_t *__restrict__ recv, uint32_t nleaf,
                            uint32_t *cnt) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && recv[i] < nleaf) atomicAdd(&cnt[recv[i]], 1u);
}

__global__ void k_copy_i32(int64_t n, const uint32_t *__restrict__ in, int *out) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int)in[i];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

cudaError_t upload_df_tables_sym() {
    alignas(16) static float tab[DF_TAB_FLOATS];
    df32_fill_tables(tab);
    return cudaMemcpyToSymbol(d_dftab_sym, tab, sizeof(tab));
}

fmm_status sym_items_count(Tree &t, cudaStream_t s, uint32_t *tot_host) {
    cudaError_t e;
    DevArena tmp;
    tmp.stream = s;
#define CK(call)                           \
    do {                                   \
        if ((e = (call)) != cudaSuccess) { \
            tmp.release();                 \
            return cuda_fail(e, #call);    \
        }                                  \
    } while (0)
    const int nleaf = t.n_leaves;
    const int *off = t.p2p_off, *list = t.p2p_list;
    const int *m2p_off = t.p2l_m2p ? t.m2p_off : nullptr;
    CK(arena_alloc(t.mem, &t.sym_cnt, 3 * ((size_t)nleaf + 1)));
    CK(arena_alloc(t.mem, &t.sym_leaf_of_box, (size_t)t.n_boxes + 1));
    uint32_t *n_items = t.sym_cnt, *n_slots = n_items + nleaf + 1, *n_m2p = n_slots + nleaf + 1;
    launch_k(k_sym_count, nblk(nleaf, 128), 128, 0, s, nleaf, t.p2p_cap, t.leaves, off, list,
             t.box_src,
             m2p_off, n_items, n_slots, n_m2p, t.sym_leaf_of_box);
    CK(cudaGetLastError());
    {
        const uint32_t *in3[3] = {n_items, n_slots, n_m2p};
        uint32_t *out3[3] = {n_items, n_slots, n_m2p};
        CK(exclusive_scan_u32_sets(3, in3, out3, nleaf, tmp, s));
    }
    CK(cudaMemcpyAsync(tot_host + 0, n_items + nleaf, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(tot_host + 1, n_slots + nleaf, 4, cudaMemcpyDeviceToHost, s));
    CK(cudaMemcpyAsync(tot_host + 2, n_m2p + nleaf, 4, cudaMemcpyDeviceToHost, s));
    tmp.release();
#undef CK
    return FMM_OK;
}

fmm_status sym_items_fill(Tree &t, const uint32_t *tot, cudaStream_t s) {
    cudaError_t e;
    DevArena tmp;
    tmp.stream = s;
    DevArena keep;
    keep.stream = s;
#define CK(call)                           \
    do {                                   \
        if ((e = (call)) != cudaSuccess) { \
            tmp.release();                 \
            keep.release();                \
            return cuda_fail(e, #call);    \
        }                                  \
    } while (0)
    const int nleaf = t.n_leaves;
    const int *off = t.p2p_off, *list = t.p2p_list;
    const int *m2p_off = t.p2l_m2p ? t.m2p_off : nullptr;
    uint32_t *n_items = t.sym_cnt, *n_slots = n_items + nleaf + 1, *n_m2p = n_slots + nleaf + 1;
    int *leaf_of_box = t.sym_leaf_of_box;
    const int64_t ni = tot[0], np2p_slots = tot[1], nm = tot[2], nslots = np2p_slots + nm;
    int4 *items, *m2p_items;
    int *order, *m2p_order, *coff, *cslot;
    double2 *partial;
    uint64_t *key, *kalt, *rkey, *rkalt;
    uint32_t *val, *valt, *recv, *rval, *rvalt, *ccnt;
    CK(arena_alloc(keep, &items, (size_t)ni + 1));
    CK(arena_alloc(keep, &order, (size_t)ni + 1));
    CK(arena_alloc(keep, &m2p_items, (size_t)nm + 1));
    CK(arena_alloc(keep, &m2p_order, (size_t)nm + 1));
    CK(arena_alloc(keep, &coff, (size_t)nleaf + 1));
    CK(arena_alloc(keep, &cslot, (size_t)nslots + 1));
    CK(arena_alloc(keep, &partial, (size_t)nslots * SY_THREADS + 1));
    CK(arena_alloc(tmp, &key, (size_t)ni + 1));
    CK(arena_alloc(tmp, &kalt, (size_t)ni + 1));
    CK(arena_alloc(tmp, &val, (size_t)ni + 1));
    CK(arena_alloc(tmp, &valt, (size_t)ni + 1));
    CK(arena_alloc(tmp, &recv, (size_t)nslots + 1));
    CK(arena_alloc(tmp, &rkey, (size_t)nslots + 1));
    CK(arena_alloc(tmp, &rkalt, (size_t)nslots + 1));
    CK(arena_alloc(tmp, &rval, (size_t)nslots + 1));
    CK(arena_alloc(tmp, &rvalt, (size_t)nslots + 1));
    CK(arena_alloc(tmp, &ccnt, (size_t)nleaf + 1));
    launch_k(k_sym_fill, nblk(nleaf, 128), 128, 0, s, nleaf, t.p2p_cap, t.leaves, off, list,
             t.box_src,
             m2p_off, leaf_of_box, n_items, n_slots, n_m2p, (uint32_t)np2p_slots, items, key, val,
             m2p_items, recv);
    CK(cudaGetLastError());
    // P2P items by decreasing cost class (powers of two; the launch order only
    // balances the load, every item writes its own slots); M2P items in list order
    if (ni > 0) {
        uint32_t *bcnt;
        CK(arena_alloc(tmp, &bcnt, 2 * COST_CLASSES));
        CK(cudaMemsetAsync(bcnt, 0, 2 * COST_CLASSES * sizeof(uint32_t), s));
        const unsigned gi = nblk(ni, 256);
        launch_k(k_cost_count, gi, 256, 0, s, ni, key, bcnt);
        launch_k(k_cost_place, gi, 256, 0, s, ni, key, bcnt, bcnt + COST_CLASSES, order);
        CK(cudaGetLastError());
    }
    if (nm > 0) {
        launch_k(k_iota, nblk(nm, 256), 256, 0, s, nm, reinterpret_cast<uint32_t *>(m2p_order));
        CK(cudaGetLastError());
    }
    // every leaf's slots in slot order: stable sort of the slots by receiving leaf
    if (nslots > 0) {
        launch_k(k_to_u64, nblk(nslots, 256), 256, 0, s, nslots, recv, rkey);
        launch_k(k_iota, nblk(nslots, 256), 256, 0, s, nslots, rval);
        CK(cudaGetLastError());
        int bits = 1;
        while ((int64_t(1) << bits) < nleaf) ++bits;
        if (nslots > 1)
            CK(radix_sort_pairs(&rkey, &rval, rkalt, rvalt, nslots, digits_for_bits(bits), tmp, s));
        launch_k(k_copy_i32, nblk(nslots, 256), 256, 0, s, nslots, rval, cslot);
        CK(cudaGetLastError());
    }
    CK(cudaMemsetAsync(ccnt, 0, ((size_t)nleaf + 1) * 4, s));
    if (nslots > 0) {
        launch_k(k_hist_recv, nblk(nslots, 256), 256, 0, s, nslots, recv, (uint32_t)nleaf, ccnt);
        CK(cudaGetLastError());
    }
    CK(exclusive_scan_u32(ccnt, ccnt, nleaf, nullptr, tmp, s));
    launch_k(k_copy_i32, nblk(nleaf + 1, 256), 256, 0, s, nleaf + 1, ccnt, coff);
    CK(cudaGetLastError());
    tmp.release();
    for (void *p : keep.ptrs) t.mem.ptrs.push_back(p);
    keep.ptrs.clear();
    t.sym = true;
    t.sym_items = items;
    t.sym_order = order;
    t.n_sym_items = (int)ni;
    t.sym_m2p_items = m2p_items;
    t.sym_m2p_order = m2p_order;
    t.n_sym_m2p = (int)nm;
    t.sym_p2p_slots = np2p_slots;
    t.sym_coff = coff;
    t.sym_cslot = cslot;
    t.sym_partial = partial;
#undef CK
    return FMM_OK;
}

fmm_status launch_eval_sym(Tree &t, double *phi, cudaStream_t s, int part) {
    cudaError_t e;
    const bool fp64 = t.precision == FMM_PREC_FP64;
    if (part == EVAL_P2P && t.n_sym_items > 0) {
        if (fp64)
            launch_k((t.kernel ? k_p2p_sym64<1> : k_p2p_sym64<0>), t.n_sym_items, SY_THREADS, 0, s,
                     t.sym_items, t.sym_order, t.box_src, t.p2p_list, t.xs, t.qs, t.sym_partial);
        else
            launch_k((t.kernel ? k_p2p_sym<1> : k_p2p_sym<0>), t.n_sym_items, SY_THREADS, 0, s,
                     t.sym_items, t.sym_order, t.box_src, t.geom, t.p2p_list, t.xs_loc, t.qs_df,
                     t.sym_partial);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "p2p sym");
    }
    if (part == EVAL_M2P && t.n_sym_m2p > 0) {
        fmm_status st = launch_m2p_items(t, t.sym_m2p_items, t.sym_m2p_order, t.n_sym_m2p,
                                         t.sym_partial + (size_t)t.sym_p2p_slots * SY_THREADS, s);
        if (st != FMM_OK) return st;
    }
    if (part == EVAL_COMBINE && t.n_leaves > 0) {
        if (fp64)
            launch_k(k_combine_sym64, t.n_leaves, SY_THREADS, 0, s, t.leaves, t.sym_coff,
                     t.sym_cslot, t.p, t.box_tgt, t.geom, t.xt, t.tperm, t.local, t.sym_partial,
                     reinterpret_cast<double2 *>(phi), t.kernel);
        else
            launch_k(k_combine_sym, t.n_leaves, SY_THREADS, 0, s, t.leaves, t.sym_coff,
                     t.sym_cslot, t.p, t.box_tgt, t.geom, t.xt_loc, t.tperm, t.local,
                     t.sym_partial, reinterpret_cast<double2 *>(phi), t.kernel);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "combine sym");
    }
    return FMM_OK;
}

}  // namespace gbfmm
