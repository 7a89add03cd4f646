// Mixed-precision P2M (Eq. 4 at the leaves) in double-float arithmetic.
//
// In the radius-normalised variables of expand.cu, A_0 = sum q_j and
// A_k = -(1/k) sum q_j w_j^k with w_j = (x_j - c) / sigma.  The mixed path
// already holds x_j - c as a df32 pair (the per-point offsets from the leaf
// centre, p2p_mixed.cu), and sigma is a power of two, so w_j is exact in
// df32 (formed by one FP64 scaling per source).  One warp per leaf; the
// leaf's sources are dealt to the lanes, every lane keeps its sums of
// q w^k in registers (PM >= p slots, static indices), and one warp
// reduction per coefficient at the end writes the multipole in FP64
// (hi + lo is exact in FP64), scaled by -1/k.
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

GBI dc dc_mul(const dc &a, const dc &b) {
    df rr = df_mul(a.re, b.re), ii = df_mul(a.im, b.im);
    df ri = df_mul(a.re, b.im), ir = df_mul(a.im, b.re);
    return dc{df_add(rr, df_neg(ii)), df_add(ri, ir)};
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

GBI df shfl_df(df v, int m) {
    return df{__shfl_xor_sync(0xffffffffu, v.hi, m), __shfl_xor_sync(0xffffffffu, v.lo, m)};
}

template <int PM>
__global__ void __launch_bounds__(128)
    k_p2m_mixed(int64_t nleaf, const int *__restrict__ leaves, int p,
                const int2 *__restrict__ box_src, const double4 *__restrict__ geom,
                const float4 *__restrict__ xs_loc, const float4 *__restrict__ qs,
                double2 *__restrict__ mpole) {
    const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (w >= nleaf) return;
    const int64_t g = leaves[w];
    const int2 bs = box_src[g];
    // 1/sigma, a power of two; applied in FP64 (exact) because it overflows a
    // float for boxes of radius below 2^-126 (and 2^1000 for radius 0)
    const double isig = geom[g].w;
    df ar[PM + 1], ai[PM + 1];
#pragma unroll
    for (int k = 0; k <= PM; ++k) ar[k] = ai[k] = df{0.f, 0.f};
    for (int j = lane; j < bs.y; j += 32) {
        const float4 xl = xs_loc[bs.x + j], qq = qs[bs.x + j];
        const dc W{split_d(((double)xl.x + (double)xl.y) * isig),
                   split_d(((double)xl.z + (double)xl.w) * isig)};
        dc pw{df{qq.x, qq.y}, df{qq.z, qq.w}};
        ar[0] = df_acc(ar[0], pw.re);
        ai[0] = df_acc(ai[0], pw.im);
#pragma unroll
        for (int k = 1; k <= PM; ++k) {
            if (k <= p) {
                pw = dc_mul(pw, W);
                ar[k] = df_acc(ar[k], pw.re);
                ai[k] = df_acc(ai[k], pw.im);
            }
        }
    }
    double2 *out = mpole + g * (p + 1);
#pragma unroll
    for (int k = 0; k <= PM; ++k) {
        if (k <= p) {
            df r = fast_sum(ar[k].hi, ar[k].lo), i = fast_sum(ai[k].hi, ai[k].lo);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                r = df_add(r, shfl_df(r, o));
                i = df_add(i, shfl_df(i, o));
            }
            if (lane == (k & 31)) {
                const double f = k == 0 ? 1.0 : -1.0 / k;
                out[k] = make_double2(f * ((double)r.hi + (double)r.lo),
                                      f * ((double)i.hi + (double)i.lo));
            }
        }
    }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

int p2m_mixed_max_p() { return 32; }

fmm_status launch_p2m_mixed(Tree &t, cudaStream_t s) {
    const int64_t nleaf = t.n_leaves;
    auto k = t.p <= 8 ? k_p2m_mixed<8> : t.p <= 16 ? k_p2m_mixed<16>
             : t.p <= 24 ? k_p2m_mixed<24> : k_p2m_mixed<32>;
    k<<<nblk(nleaf * 32, 128), 128, 0, s>>>(nleaf, t.leaves, t.p, t.box_src, t.geom, t.xs_loc,
                                            t.qs_df, t.mpole); note_launch();
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "p2m mixed");
}

}  // namespace gbfmm
