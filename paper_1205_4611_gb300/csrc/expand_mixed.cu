// Mixed-precision upward and downward translations in double-float
// arithmetic (expansions stay stored in FP64; every operation below runs on
// the FP32 pipes, which GB300 has 64 times as many of as FP64 units).
//
// P2M (Eq. 4 at the leaves).
// In the radius-normalised variables of expand.cu, A_0 = sum q_j and
// A_k = -(1/k) sum q_j w_j^k with w_j = (x_j - c) / sigma.  The mixed path
// already holds x_j - c as a df32 pair (the per-point offsets from the leaf
// centre, p2p_mixed.cu), and sigma is a power of two, so w_j is exact in
// df32 (formed by one FP64 scaling per source).  One warp per leaf; the
// leaf's sources are dealt to the lanes, every lane keeps its sums of
// q w^k in registers (PM >= p slots, static indices), and one warp
// reduction per coefficient at the end writes the multipole in FP64
// (hi + lo is exact in FP64), scaled by -1/k.
//
// M2M and L2L: the closed forms of expand.cu (radius-normalised), evaluated
// by Horner's rule in the shift d (rho for M2M) with df32 binomials:
//   M2M  A'_l += -A_0 rho^l / l + sum_{k=1}^{l} C(l-1, k-1) s^k A_k rho^{l-k}
//   L2L  B'_l += s^l sum_{k=l}^{p} C(k, l) B_k d^{k-l}
// One CTA per parent box, one warp per child, lane l = coefficient l; M2M
// sums the four children's contributions in shared memory.
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "df32.cuh"
#include "internal.h"

namespace gbfmm {

namespace {

struct dc {
    df re, im;
};

// a b with the low parts left unnormalised (power chains)
GBI dc dc_mul_lz(const dc &a, const dc &b) {
    return dc{df_dot2_lz(a.re, b.re, df_neg(a.im), b.im), df_dot2_lz(a.re, b.im, a.im, b.re)};
}

GBI df split_d(double v) {
    float hi = __double2float_rn(v);
    float lo = __double2float_rn(v - (double)hi);
    return df{hi, lo};
}

// lazily normalised df32 accumulation (normalise before combining sums)
GBI df df_acc(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    return df{s.hi, F_ADD(s.lo, F_ADD(a.lo, b.lo))};
}

// P2M, df32: one warp per leaf, its sources dealt to the lanes; every lane
// keeps its own sums of q w^k (k = 0..p), w = (x - c) / sigma (the stored
// df32 offset: offsets are kept in units of their leaf's sigma), in shared
// memory (rows of 33 float4 per coefficient, lane-private slots), and at the
// end lane k adds up coefficient k over the 32 lanes in lane order and
// writes it scaled by -1/k (k >= 1).
constexpr int P2M_WARPS = 4;
constexpr int P2M_ROW = 33;

__global__ void __launch_bounds__(32 * P2M_WARPS)
    k_p2m_mixed(int64_t nleaf, const int *__restrict__ leaves, int p,
                const int2 *__restrict__ box_src, const double4 *__restrict__ geom,
                const float4 *__restrict__ xs_loc, const float4 *__restrict__ qs,
                double2 *__restrict__ mpole) {
    pdl_wait();
    extern __shared__ float4 p2m_acc[];  // [warp][k][P2M_ROW]
    const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t w = (int64_t)blockIdx.x * P2M_WARPS + wib;
    if (w >= nleaf) return;
    const int64_t g = leaves[w];
    const int2 bs = box_src[g];
    float4 *acc = p2m_acc + (size_t)wib * (p + 1) * P2M_ROW;
    for (int k = 0; k <= p; ++k) acc[k * P2M_ROW + lane] = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j = lane; j < bs.y; j += 32) {
        const float4 xl = xs_loc[bs.x + j], qq = qs[bs.x + j];
        const dc W{df{xl.x, xl.y}, df{xl.z, xl.w}};
        dc pw{df{qq.x, qq.y}, df{qq.z, qq.w}};
        {
            const float4 a = acc[lane];
            const df r = df_acc(df{a.x, a.y}, pw.re), i = df_acc(df{a.z, a.w}, pw.im);
            acc[lane] = make_float4(r.hi, r.lo, i.hi, i.lo);
        }
#pragma unroll 2
        for (int k = 1; k <= p; ++k) {
            pw = dc_mul_lz(pw, W);
            const float4 a = acc[k * P2M_ROW + lane];
            const df r = df_acc(df{a.x, a.y}, pw.re), i = df_acc(df{a.z, a.w}, pw.im);
            acc[k * P2M_ROW + lane] = make_float4(r.hi, r.lo, i.hi, i.lo);
        }
    }
    __syncwarp();
    double2 *out = mpole + g * (p + 1);
    for (int k = lane; k <= p; k += 32) {
        df r{0.f, 0.f}, i{0.f, 0.f};
        for (int j = 0; j < 32; ++j) {
            const float4 a = acc[k * P2M_ROW + j];
            r = df_add(r, fast_sum(a.x, a.y));
            i = df_add(i, fast_sum(a.z, a.w));
        }
        const double f = k == 0 ? 1.0 : -1.0 / k;
        out[k] = make_double2(f * ((double)r.hi + (double)r.lo), f * ((double)i.hi + (double)i.lo));
    }
}

constexpr int TR_MAXP = 32;
constexpr int BINOM_DF_N = TR_MAXP + 1;  // C(n, k) for n <= 32, as df32 (exact)
__device__ float2 d_binom_df[BINOM_DF_N * (BINOM_DF_N + 1) / 2];

// Rows 0 .. p of the table, staged in shared memory by every block of the
// translation kernels (a Horner step must not wait on a global load).
constexpr int BINOM_ENTRIES = BINOM_DF_N * (BINOM_DF_N + 1) / 2;
GBI void stage_binom(float2 *sbin, int p) {
    const int nb = (p + 1) * (p + 2) / 2;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) sbin[i] = d_binom_df[i];
}
GBI df binom_s(const float2 *sbin, int n, int k) {
    const float2 v = sbin[n * (n + 1) / 2 + k];
    return df{v.x, v.y};
}

GBI dc dc_add(const dc &a, const dc &b) { return dc{df_add(a.re, b.re), df_add(a.im, b.im)}; }

GBI dc dc_scale(const dc &a, df s) { return dc{df_mul(a.re, s), df_mul(a.im, s)}; }

// M2M for the parents listed in `boxes` (entries without children skipped).
__global__ void __launch_bounds__(128)
    k_m2m_mixed(const int *__restrict__ boxes, const int *__restrict__ child0, int p,
                const double4 *__restrict__ geom, const int2 *__restrict__ box_src,
                double2 *mpole) {
    pdl_wait();
    __shared__ float4 sa[4][TR_MAXP + 1];
    __shared__ float4 red[4][TR_MAXP + 1];
    __shared__ float2 sbin[BINOM_ENTRIES];
    const int64_t g = boxes[blockIdx.x];
    const int64_t c0 = child0[g];
    if (c0 < 0) return;
    const int c = threadIdx.x >> 5, l = threadIdx.x & 31;
    stage_binom(sbin, p);
    for (int i = threadIdx.x; i < 4 * (p + 1); i += blockDim.x) {
        const int cc = i / (p + 1), k = i - cc * (p + 1);
        const double2 v = mpole[(c0 + cc) * (p + 1) + k];
        const df re = split_d(v.x), im = split_d(v.y);
        sa[cc][k] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    __syncthreads();
    const double4 gp = geom[g], gc = geom[c0 + c];
    const dc rho{split_d((gc.x - gp.x) * gp.w), split_d((gc.y - gp.y) * gp.w)};
    const float s = (float)(gc.z * gp.w);  // sigma_c / sigma_p, a power of two <= 1
    // a child without sources has a zero multipole; with shrink-wrapped
    // geometry its centre may lie outside a parent of radius 0 (1/sigma beyond
    // the range), so it contributes zero instead of being translated
    const bool empty = box_src[c0 + c].y == 0;
    if (l <= p && empty) red[c][l] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (l <= p && !empty) {
        const float4 a0 = sa[c][0];
        dc acc{df{a0.x, a0.y}, df{a0.z, a0.w}};
        if (l > 0) {
            // acc = -A_0 / l, then acc = acc * rho + C(l-1, k-1) s^k A_k, k = 1..l
            const df il = split_d(-1.0 / l);
            acc = dc_scale(acc, il);
            float sk = 1.0f;
            for (int k = 1; k <= l; ++k) {
                sk *= s;
                const float4 ak = sa[c][k];
                df b = binom_s(sbin, l - 1, k - 1);
                b = df{b.hi * sk, b.lo * sk};  // exact (power of two)
                const dc t = dc_scale(dc{df{ak.x, ak.y}, df{ak.z, ak.w}}, b);
                df_horner_step(acc.re, acc.im, rho.re, rho.im, t.re, t.im);
            }
            acc = dc{fast_sum(acc.re.hi, acc.re.lo), fast_sum(acc.im.hi, acc.im.lo)};
        }
        red[c][l] = make_float4(acc.re.hi, acc.re.lo, acc.im.hi, acc.im.lo);
    }
    __syncthreads();
    if (c == 0 && l <= p) {
        dc sum{df{red[0][l].x, red[0][l].y}, df{red[0][l].z, red[0][l].w}};
        for (int cc = 1; cc < 4; ++cc)
            sum = dc_add(sum, dc{df{red[cc][l].x, red[cc][l].y}, df{red[cc][l].z, red[cc][l].w}});
        mpole[g * (p + 1) + l] = make_double2((double)sum.re.hi + (double)sum.re.lo,
                                              (double)sum.im.hi + (double)sum.im.lo);
    }
}

// L2L from the parents listed in `boxes` into their four children (added).
__global__ void __launch_bounds__(128)
    k_l2l_mixed(const int *__restrict__ boxes, const int *__restrict__ child0, int p,
                const double4 *__restrict__ geom, const int2 *__restrict__ box_tgt,
                double2 *local) {
    pdl_wait();
    __shared__ float4 sb[TR_MAXP + 1];
    __shared__ float2 sbin[BINOM_ENTRIES];
    const int64_t g = boxes[blockIdx.x];
    const int64_t c0 = child0[g];
    if (c0 < 0) return;
    const int c = threadIdx.x >> 5, l = threadIdx.x & 31;
    stage_binom(sbin, p);
    for (int k = threadIdx.x; k <= p; k += blockDim.x) {
        const double2 v = local[g * (p + 1) + k];
        const df re = split_d(v.x), im = split_d(v.y);
        sb[k] = make_float4(re.hi, re.lo, im.hi, im.lo);
    }
    __syncthreads();
    // a child without evaluation points never uses its local expansion (nor do
    // its children); skipped, as its centre may lie outside a parent of radius 0
    if (l > p || box_tgt[c0 + c].y == 0) return;
    const double4 gp = geom[g], gc = geom[c0 + c];
    const dc d{split_d((gc.x - gp.x) * gp.w), split_d((gc.y - gp.y) * gp.w)};
    const float s = (float)(gc.z * gp.w);
    double2 *out = local + (c0 + c) * (p + 1) + l;
    const double2 o = *out;  // in flight during the Horner chain
    // acc = sum_{k=l}^{p} C(k, l) B_k d^{k-l} by Horner from k = p down
    dc acc{df{0.f, 0.f}, df{0.f, 0.f}};
    for (int k = p; k >= l; --k) {
        const float4 bk = sb[k];
        const dc t = dc_scale(dc{df{bk.x, bk.y}, df{bk.z, bk.w}}, binom_s(sbin, k, l));
        df_horner_step(acc.re, acc.im, d.re, d.im, t.re, t.im);
    }
    float sl = 1.0f;
    for (int i = 0; i < l; ++i) sl *= s;
    *out = make_double2(o.x + sl * ((double)acc.re.hi + (double)acc.re.lo),
                        o.y + sl * ((double)acc.im.hi + (double)acc.im.lo));
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

cudaError_t upload_binom_df() {
    static float2 tab[BINOM_DF_N * (BINOM_DF_N + 1) / 2];
    static double row[BINOM_DF_N + 1];
    for (int n = 0; n < BINOM_DF_N; ++n) {
        // Pascal's rule in FP64 (exact: C(32, 16) < 2^53)
        for (int k = n; k >= 0; --k) row[k] = (k == 0 || k == n) ? 1.0 : row[k] + row[k - 1];
        for (int k = 0; k <= n; ++k) {
            float hi = (float)row[k];
            tab[n * (n + 1) / 2 + k] = make_float2(hi, (float)(row[k] - (double)hi));
        }
    }
    return cudaMemcpyToSymbol(d_binom_df, tab, sizeof(tab));
}

int translate_mixed_max_p() { return TR_MAXP; }

fmm_status launch_m2m_mixed(Tree &t, int level, cudaStream_t s) {
    const int64_t n = t.level_start[level + 1] - t.level_start[level];
    if (n <= 0) return FMM_OK;
    launch_k(k_m2m_mixed, (unsigned)n, 128, 0, s, t.lvl_boxes + t.level_start[level], t.child0, t.p,
             t.geom, t.box_src, t.mpole);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "m2m mixed");
}

fmm_status launch_l2l_mixed(Tree &t, int level, cudaStream_t s) {
    const int64_t n = t.level_start[level + 1] - t.level_start[level];
    if (n <= 0) return FMM_OK;
    launch_k(k_l2l_mixed, (unsigned)n, 128, 0, s, t.lvl_boxes + t.level_start[level], t.child0, t.p,
             t.geom, t.box_tgt, t.local);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "l2l mixed");
}

int p2m_mixed_max_p() { return 32; }

fmm_status launch_p2m_mixed(Tree &t, cudaStream_t s) {
    const int64_t nleaf = t.n_leaves;
    const int smem = P2M_WARPS * (t.p + 1) * P2M_ROW * (int)sizeof(float4);
    static const cudaError_t attr =
        cudaFuncSetAttribute(k_p2m_mixed, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             P2M_WARPS * (TR_MAXP + 1) * P2M_ROW * (int)sizeof(float4));
    if (attr != cudaSuccess) return cuda_fail(attr, "p2m smem");
    launch_k(k_p2m_mixed, nblk(nleaf, P2M_WARPS), 32 * P2M_WARPS, smem, s, nleaf, t.leaves, t.p,
             t.box_src, t.geom, t.xs_loc, t.qs_df, t.mpole);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "p2m mixed");
}

}  // namespace gbfmm
