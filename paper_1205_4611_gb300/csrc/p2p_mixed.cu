// Mixed-precision near field: P2P (Alg. "Direct evaluation between boxes")
// with every pair evaluated in double-float arithmetic on the FP32 pipes
// (L2P and the combination of partial sums stay in FP64, see p2p.cu).
//
// Positions enter as df32 offsets from their own leaf centre in units of the
// leaf's sigma (split once from FP64; the scaling is an exact power of two).
// A (target leaf t, source leaf s) pair works in the pair's units 2^ep
// (PairUnits, df32.cuh), so its float quantities are O(1) at any absolute
// scale of the coordinates: the source offsets are re-based to the target
// centre, d = (c_s - c_t) 2^-ep + (x - c_s) 2^-ep, while the tile is staged in
// shared memory, the target offsets are rescaled once per source leaf, the
// logarithm takes ep ln 2 through its exponent term and a harmonic term 1/D
// the factor 2^-ep when the tile's sum is added in FP64; a pair then needs
//   D = e - d                       (two TwoSums per coordinate)
//   S = |D_hi|^2 as df32            (two exact products, one TwoSum)
//   ln S, atan2(D_hi)               (df32 log and arctangent, df32.cuh)
//   + (D_lo / D_hi)                 (first-order correction, |D_lo| < 2^-23 |D_hi|)
//   Phi += q Log(D)                 (df32 complex multiply-accumulate)
// Pairs whose difference is below the rounding level of the re-based
// offsets (2^-42 of the pair's scale) are treated as coincident and skipped,
// which is exact for duplicated points (Eq. 1, j != i); a y-difference at
// that level is snapped to +0 so exactly shared ordinates fall on the
// principal branch the way FP64 subtraction puts them (+0, arg = +pi).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "df32.cuh"
#include "internal.h"

namespace gbfmm {

__device__ float d_dftab[DF_TAB_FLOATS];

namespace {

constexpr int MX_THREADS = 64;
constexpr int MX_TILE = 64;

GBI df split_d(double v) {
    float hi = __double2float_rn(v);
    float lo = __double2float_rn(v - (double)hi);
    return df{hi, lo};
}

// df32 offset of every point from the centre of its leaf, in units of the
// leaf's sigma (one block per leaf).
__global__ void k_split_local(const int *__restrict__ leaves, const int2 *__restrict__ range,
                              const double4 *__restrict__ geom, const double2 *__restrict__ pts,
                              float4 *__restrict__ out) {
    pdl_wait();
    int64_t g = leaves[blockIdx.x];
    int2 r = range[g];
    double4 ge = geom[g];
    for (int i = threadIdx.x; i < r.y; i += blockDim.x) {
        double2 p = pts[r.x + i];
        df x = split_d((p.x - ge.x) * ge.w), y = split_d((p.y - ge.y) * ge.w);
        out[r.x + i] = make_float4(x.hi, x.lo, y.hi, y.lo);
    }
}

__global__ void k_permute_q_df(int64_t n, const uint32_t *__restrict__ perm,
                               const double2 *__restrict__ q, float4 *__restrict__ qs) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 v = q[perm[i]];
    df r = split_d(v.x), m = split_d(v.y);
    qs[i] = make_float4(r.hi, r.lo, m.hi, m.lo);
}

// D = a - b for df32 a, b; normalised.
// a - b for df32 a, b.  The closing Fast2Sum is exact when the low sum does
// not outgrow the high difference; otherwise (a high difference within a
// few ulps) its error is of the order of the rounding of al - bl, which the
// TwoSum form makes as well.
GBI df df_diff(float ah, float al, float bh, float bl) {
    df s = two_sum(ah, -bh);
    float lo = F_ADD(s.lo, F_SUB(al, bl));
    return fast_sum(s.hi, lo);
}

GBI int threads_per_target(int nt) { return nt <= 16 ? 4 : (nt <= 32 ? 2 : 1); }

// 1/E for a df32 complex E != 0: conj(E) / |E|^2 with one Newton step on 1/|E|^2.
GBI void df_cinv(df Ex, df Ey, df &Rr, df &Ri) {
    const df inv = df_recip(df_dot2(Ex, Ex, Ey, Ey));
    Rr = df_mul(Ex, inv);
    Ri = df_neg(df_mul(Ey, inv));
}

// One work item (target leaf, chunk of <= 64 points, run of the strong list):
// partial near-field sums in df32, written as FP64 (hi + lo is exact).
// KERN 0: q Log(y - x) (Eq. 1, Eq. 2); KERN 1: q / (x - y) (harmonic kernel).
template <int KERN>
__global__ void __launch_bounds__(MX_THREADS)
    k_p2p_mixed(const int4 *__restrict__ items, const int *__restrict__ order,
                const int2 *__restrict__ box_tgt, const int2 *__restrict__ box_src,
                const double4 *__restrict__ geom, const int *__restrict__ strong,
                const float4 *__restrict__ xt_loc, const float4 *__restrict__ xs_loc,
                const float4 *__restrict__ qs, double2 *__restrict__ partial) {
    pdl_wait();
    __shared__ __align__(16) float tab[DF_TAB_FLOATS];
    __shared__ float4 sd[MX_TILE], sq[MX_TILE];
    for (int i = threadIdx.x; i < DF_TAB_FLOATS; i += MX_THREADS) tab[i] = d_dftab[i];
    const float *atab = tab + ATAN_OFF;
    const int idx = order[blockIdx.x];
    const int4 it = items[idx];
    const int64_t g = it.x;
    const int2 bt = box_tgt[g];
    const int nt = min(MX_THREADS, bt.y - it.y);
    const int tpt = threads_per_target(nt);
    const int my = threadIdx.x / tpt, sub = threadIdx.x % tpt;
    const bool valid = my < nt;
    const double4 gt = geom[g];
    const float4 et = valid ? xt_loc[bt.x + it.y + my] : make_float4(0.f, 0.f, 0.f, 0.f);
    // df32 sums within one tile of sources, added into FP64 after each tile
    df ar{0.f, 0.f}, ai{0.f, 0.f};
    double rr = 0.0, ri = 0.0;
    for (int ei = it.z; ei < it.w; ++ei) {
        const int sbox = strong[ei];
        const int2 bs = box_src[sbox];
        const double4 gs = geom[sbox];
        const PairUnits u = pair_units(gt.z, gs.z);
        const double inv = pow2d(-u.ep);
        const df Dx = split_d((gs.x - gt.x) * inv), Dy = split_d((gs.y - gt.y) * inv);
        // rounding level of the re-based offsets for this leaf pair
        const float scale = fabsf(Dx.hi) + fabsf(Dy.hi) + 2.0f * (u.fs + u.ft);
        const float tau = scale * 0x1p-42f;
        const float tau2 = fmaxf(tau * tau, 1e-36f);
        const float4 e = make_float4(F_MUL(et.x, u.ft), F_MUL(et.y, u.ft), F_MUL(et.z, u.ft),
                                     F_MUL(et.w, u.ft));
        const double hs = KERN == 1 ? inv : 1.0;  // 1/D = 2^-ep / D'
        for (int c0 = 0; c0 < bs.y; c0 += MX_TILE) {
            const int nn = min(MX_TILE, bs.y - c0);
            __syncthreads();
            if (threadIdx.x < nn) {
                float4 xl = xs_loc[bs.x + c0 + threadIdx.x];
                df dx = df_add(Dx, df{F_MUL(xl.x, u.fs), F_MUL(xl.y, u.fs)}),
                   dy = df_add(Dy, df{F_MUL(xl.z, u.fs), F_MUL(xl.w, u.fs)});
                sd[threadIdx.x] = make_float4(dx.hi, dx.lo, dy.hi, dy.lo);
                sq[threadIdx.x] = qs[bs.x + c0 + threadIdx.x];
            }
            __syncthreads();
            if (!valid) continue;
            for (int j = sub; j < nn; j += tpt) {
                const float4 d = sd[j];
                df Ex = df_diff(e.x, e.y, d.x, d.y);
                df Ey = df_diff(e.z, e.w, d.z, d.w);
                if (fabsf(Ey.hi) <= tau) Ey = df{0.0f, 0.0f};
                df p1 = two_prod(Ex.hi, Ex.hi), p2 = two_prod(Ey.hi, Ey.hi);
                df S = two_sum(p1.hi, p2.hi);
                if (!(S.hi > tau2)) continue;  // coincident pair
                df Lr, Li;
                if (KERN == 1) {
                    // q / (x - y) = -q / D
                    df_cinv(Ex, Ey, Lr, Li);
                    Lr = df_neg(Lr);
                    Li = df_neg(Li);
                } else {
                    float slo = F_ADD(S.lo, F_ADD(p1.lo, p2.lo));
                    float inv = F_RCP(S.hi);
                    df ln = df_log_f(S.hi, tab, u.ecst);
                    df an = df_atan2_f(Ey.hi, Ex.hi, atab);
                    // Log(D) = 0.5 ln S + i atan2 + D_lo / D_hi (first order)
                    float cr = F_MUL(F_FMA(Ex.lo, Ex.hi, F_MUL(Ey.lo, Ey.hi)), inv);
                    float ci = F_MUL(F_FMA(Ey.lo, Ex.hi, -F_MUL(Ex.lo, Ey.hi)), inv);
                    Lr = fast_sum(F_MUL(0.5f, ln.hi), F_FMA(0.5f, F_FMA(slo, inv, ln.lo), cr));
                    Li = fast_sum(an.hi, F_ADD(an.lo, ci));
                }
                // Phi += q * Log(D), q = (qr, qi) in df32
                const float4 q = sq[j];
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
            rr += ((double)ar.hi + (double)ar.lo) * hs;
            ri += ((double)ai.hi + (double)ai.lo) * hs;
            ar = df{0.f, 0.f};
            ai = df{0.f, 0.f};
        }
    }
    // combine the threads of one evaluation point (adjacent lanes), in FP64
    for (int m = 1; m < tpt; m <<= 1) {
        rr += __shfl_xor_sync(0xffffffffu, rr, m);
        ri += __shfl_xor_sync(0xffffffffu, ri, m);
    }
    if (valid && sub == 0) partial[(int64_t)idx * MX_THREADS + my] = make_double2(rr, ri);
}

// L2P in double-float (Horner's rule on the local expansion, converted once
// per chunk; w = (y - c) / sigma is the stored df32 offset of the point) plus
// the chunk's partial sums in item order (FP64): the mixed path's combination
// at separate evaluation points.  kern 0: sum B_l w^l; kern 1: -d/dy of it,
// -(1/sigma) sum l B_l w^(l-1).
constexpr int CB_MAXP = 32;
__global__ void __launch_bounds__(MX_THREADS)
    k_combine_mixed(const int2 *__restrict__ chunks, const int *__restrict__ item0, int p,
                    const int2 *__restrict__ box_tgt, const double4 *__restrict__ geom,
                    const float4 *__restrict__ xt_loc, const uint32_t *__restrict__ tperm,
                    const double2 *__restrict__ local, const double2 *__restrict__ partial,
                    double2 *__restrict__ phi, int kern) {
    pdl_wait();
    __shared__ float4 sb[CB_MAXP + 1];
    const int c = blockIdx.x;
    const int2 ch = chunks[c];
    const int64_t g = ch.x;
    for (int i = threadIdx.x; i <= p; i += MX_THREADS) {
        const double2 v = local[g * (p + 1) + i];
        const df re = split_d(v.x), im = split_d(v.y);
        sb[i] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    __syncthreads();
    const int2 bt = box_tgt[g];
    const int nt = min(MX_THREADS, bt.y - ch.y);
    if ((int)threadIdx.x >= nt) return;
    const int pos = bt.x + ch.y + threadIdx.x;
    const float4 yl = xt_loc[pos];
    const df wr{yl.x, yl.y}, wi{yl.z, yl.w};
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
    const double sc = kern ? -geom[g].w : 1.0;  // a power of two: exact
    double ar = sc * ((double)hr.hi + (double)hr.lo), ai = sc * ((double)hi.hi + (double)hi.lo);
    for (int it = item0[c]; it < item0[c + 1]; ++it) {
        const double2 v = partial[(int64_t)it * MX_THREADS + threadIdx.x];
        ar += v.x;
        ai += v.y;
    }
    phi[tperm[pos]] = make_double2(ar, ai);
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

cudaError_t upload_df_tables() {
    alignas(16) static float tab[DF_TAB_FLOATS];
    df32_fill_tables(tab);
    return cudaMemcpyToSymbol(d_dftab, tab, sizeof(tab));
}

// Per-point df32 offsets from the leaf centres (tree build, mixed mode).
fmm_status prepare_mixed_points(Tree &t, cudaStream_t s) {
    cudaError_t e;
    const int64_t nleaf = t.n_leaves;
    if ((e = arena_alloc(t.mem, &t.xs_loc, t.n_src)) != cudaSuccess)
        return cuda_fail(e, "mixed points");
    launch_k(k_split_local, (unsigned)nleaf, 128, 0, s, t.leaves, t.box_src, t.geom, t.xs,
             t.xs_loc);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "split sources");
    if (t.separate) {
        if ((e = arena_alloc(t.mem, &t.xt_loc, t.n_tgt)) != cudaSuccess)
            return cuda_fail(e, "mixed targets");
        launch_k(k_split_local, (unsigned)nleaf, 128, 0, s, t.leaves, t.box_tgt, t.geom, t.xt,
                 t.xt_loc);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "split targets");
    } else {
        t.xt_loc = t.xs_loc;
    }
    if ((e = arena_alloc(t.mem, &t.qs_df, t.n_src)) != cudaSuccess)
        return cuda_fail(e, "mixed strengths");
    return FMM_OK;
}

fmm_status permute_q_mixed(Tree &t, const double *q, cudaStream_t s) {
    launch_k(k_permute_q_df, nblk(t.n_src, 256), 256, 0, s, t.n_src, t.perm,
             reinterpret_cast<const double2 *>(q), t.qs_df);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "permute q (mixed)");
}

fmm_status launch_p2p_mixed(Tree &t, cudaStream_t s) {
    auto k = t.kernel ? k_p2p_mixed<1> : k_p2p_mixed<0>;
    launch_k(k, t.n_p2p_items, MX_THREADS, 0, s, t.p2p_items, t.p2p_order, t.box_tgt, t.box_src,
             t.geom, t.p2p_list, t.xt_loc, t.xs_loc, t.qs_df, t.p2p_partial);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "p2p mixed");
}

bool combine_mixed_ok(const Tree &t) {
    return t.precision == FMM_PREC_MIXED && t.p <= CB_MAXP && t.xt_loc != nullptr;
}

fmm_status launch_combine_mixed(Tree &t, double *phi, cudaStream_t s) {
    launch_k(k_combine_mixed, t.n_chunks, MX_THREADS, 0, s, t.p2p_chunks, t.p2p_item0, t.p,
             t.box_tgt, t.geom, t.xt_loc, t.tperm, t.local, t.p2p_partial,
             reinterpret_cast<double2 *>(phi), t.kernel);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "combine mixed");
}

}  // namespace gbfmm
