// M2L on the tensor cores (tcgen05): the binomial contraction of every weak
// pair as an exact split-precision bf16 GEMM with FP32 accumulation in TMEM.
//
// For a weak pair (s -> t), r = z_s - z_t, u = sigma_s / r, v = sigma_t / r
// (radius-normalised expansions, expand.cu), the M2L of Alg. "Multipole to
// local translation" (its two summation sweeps) applies the fixed operator
//     c_l = sum_{k=1}^{p} C(k+l-1, l) x_k,      x_k = (-1)^k A_k u^k.
// Scaled so that every entry is <= 1/2,
//     Ahat_{lk} = C(k+l-1, l) 2^-(k+l),  xhat_k = 2^k x_k,  chat_l = sum_k Ahat_lk xhat_k,
//     B_0 += chat_0 + A_0 Log(z_t - z_s),  B_l += (chat_l - A_0 2^-l / l) (2v)^l.
// One GEMM row is one component (real or imaginary) of one pair's xhat; the
// operator rows are the output index l.  Rows and operator rows are split
// into s signed 8-bit digits (integers in [-128, 128], exact in bf16) under a
// per-row power-of-two scale; the digit products of one "level" d = i + j sum
// exactly in FP32 (|product| <= 2^14, at most 6*32 terms), so every level is
// an exact integer, and the levels are recombined in double-float.  With
// s = 6 the split carries 47 bits, the same as the double-float sweeps.
//
// Per CTA (128 threads, persistent over work items of <= 64 pairs of one
// target): slices of the 128 rows -> shared memory (UMMA canonical K-major
// layout, no swizzle) -> one thread issues s(s+1)/2 * 2 MMAs (M=128, N=32,
// K=16) into s TMEM accumulators -> tcgen05.commit on an mbarrier -> each
// thread reads its row back with tcgen05.ld, recombines, rescales, and the
// per-target sum over the item's pairs is added to the local expansion with
// FP64 atomics.  Every wait is bounded; a wait that gives up sets the tree's
// status word and the item is skipped.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "df32.cuh"
#include "internal.h"

namespace gbfmm {

namespace {

constexpr int TC_ROWS = 128;   // GEMM rows per tile = 64 pairs x (re, im)
constexpr int TC_NK = 32;      // K (k = 1..p) and N (l = 0..p) padded to 32
constexpr int TC_MAXS = 6;     // digit slices
constexpr int A_SLICE_BYTES = TC_ROWS * TC_NK * 2;  // 8 KB
constexpr int B_SLICE_BYTES = TC_NK * TC_NK * 2;    // 2 KB
constexpr int TC_SBO = (TC_NK / 8) * 128;           // 8-row group stride
constexpr int TC_LBO = 128;                         // core-matrix stride along K
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;

__device__ float d_tctab[DF_TAB_FLOATS];

__host__ __device__ inline int kmaj_off(int row, int k) {
    return (row >> 3) * TC_SBO + (k >> 3) * TC_LBO + (row & 7) * 16 + (k & 7) * 2;
}

GBI uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

GBI uint64_t umma_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3FFF);
    d |= (uint64_t)((TC_LBO >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((TC_SBO >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;  // descriptor version; base offset 0; no swizzle
    return d;
}

// kind::f16 instruction descriptor: D = F32, A = B = BF16, both K-major,
// N = 32, M = 128.
constexpr uint32_t TC_IDESC = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_NK >> 3) << 17) |
                              ((uint32_t)(TC_ROWS >> 4) << 24);

GBI float pow2f(int e) { return __int_as_float((e + 127) << 23); }  // e in [-126, 127]

GBI df split_d(double v) {
    float hi = __double2float_rn(v);
    float lo = __double2float_rn(v - (double)hi);
    return df{hi, lo};
}

struct dc {
    df re, im;
};
GBI dc dc_mul(const dc &a, const dc &b) {
    df rr = df_mul(a.re, b.re), ii = df_mul(a.im, b.im);
    df ri = df_mul(a.re, b.im), ir = df_mul(a.im, b.re);
    return dc{df_add(rr, df_neg(ii)), df_add(ri, ir)};
}
GBI df df_acc(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    return df{s.hi, F_ADD(s.lo, F_ADD(a.lo, b.lo))};
}
GBI df shfl_df(df v, int m, unsigned mask = 0xffffffffu) {
    return df{__shfl_xor_sync(mask, v.hi, m), __shfl_xor_sync(mask, v.lo, m)};
}
GBI df df_divf(df a, float b) {
    float q1 = F_MUL(a.hi, F_RCP(b));
    float r = F_ADD(F_FMA(-q1, b, a.hi), a.lo);
    float q2 = F_MUL(r, F_RCP(b));
    return fast_sum(q1, q2);
}
GBI float rint_magic(float t) {  // round to nearest integer, |t| < 2^22
    return F_SUB(F_ADD(t, 12582912.0f), 12582912.0f);
}

GBI void tmem_ld32(uint32_t addr, float *v) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
          "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__global__ void __launch_bounds__(TC_ROWS)
    k_m2l_tc(const int2 *__restrict__ items, int n_items, int p, int S,
             const double4 *__restrict__ geom, const int *__restrict__ weak_off,
             const int *__restrict__ weak, const float4 *__restrict__ mp,
             const uint4 *__restrict__ bslices, const int *__restrict__ fexp,
             double2 *__restrict__ local, int *status) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sA = smem_raw;                            // S x 8 KB
    unsigned char *sB = smem_raw + TC_MAXS * A_SLICE_BYTES;  // S x 2 KB
    __shared__ float tab[DF_TAB_FLOATS];
    __shared__ float2 red[4][TC_NK][2];
    __shared__ int sf[TC_NK];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int comp = tid & 1, q = tid >> 1;  // GEMM row tid = component comp of pair q
    // one-time set-up: tables, operator slices, mbarrier, TMEM
    for (int i = tid; i < DF_TAB_FLOATS; i += TC_ROWS) tab[i] = d_tctab[i];
    for (int i = tid; i < S * B_SLICE_BYTES / 16; i += TC_ROWS)
        reinterpret_cast<uint4 *>(sB)[i] = bslices[i];
    if (tid < TC_NK) sf[tid] = fexp[tid];
    if (tid == 0) {
        abort_flag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(
            smem_u32(&tmem_base)));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tmem_base;
    uint32_t phase = 0;

    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int2 it = items[item];
        const int64_t g = it.x;
        const int e0 = it.y, n_pairs = min(64, weak_off[g + 1] - e0);
        const bool active = q < n_pairs;
        const double4 gt = geom[g];
        // ---------------- prescale: xhat_k (this row's component) in df32
        df xk[TC_NK];
#pragma unroll
        for (int k = 0; k < TC_NK; ++k) xk[k] = df{0.f, 0.f};
        dc v{df{0.f, 0.f}, df{0.f, 0.f}};
        dc A0{df{0.f, 0.f}, df{0.f, 0.f}};
        df Dx{0.f, 0.f}, Dy{0.f, 0.f};
        int emax = 0;
        if (active) {
            const int64_t s = weak[e0 + q];
            const double4 gs = geom[s];
            Dx = split_d(gt.x - gs.x);  // z_t - z_s
            Dy = split_d(gt.y - gs.y);
            df n2 = df_add(df_mul(Dx, Dx), df_mul(Dy, Dy));
            float i0 = F_RCP(n2.hi);
            df corr = df_add(df{1.0f, 0.f}, df_neg(df_mulf(n2, i0)));
            df inv = df_add(df{i0, 0.f}, df_mulf(corr, i0));
            dc ir{df_neg(df_mul(Dx, inv)), df_mul(Dy, inv)};  // 1/r, r = -D
            const float su = 2.0f * (float)gs.z, sv = 2.0f * (float)gt.z;
            dc u2{df{ir.re.hi * su, ir.re.lo * su}, df{ir.im.hi * su, ir.im.lo * su}};  // 2u
            v = dc{df{ir.re.hi * sv, ir.re.lo * sv}, df{ir.im.hi * sv, ir.im.lo * sv}};  // 2v
            const float4 *A = mp + s * (p + 1);
            const float4 a0 = A[0];
            A0 = dc{df{a0.x, a0.y}, df{a0.z, a0.w}};
            dc pw = u2;
            float amax = 0.f;
#pragma unroll
            for (int k = 1; k <= TC_NK; ++k) {
                if (k <= p) {
                    const float4 a4 = A[k];
                    dc x = dc_mul(dc{df{a4.x, a4.y}, df{a4.z, a4.w}}, pw);
                    df val = comp ? x.im : x.re;
                    xk[k - 1] = (k & 1) ? df_neg(val) : val;
                    amax = fmaxf(amax, fabsf(xk[k - 1].hi));
                    pw = dc_mul(pw, u2);
                }
            }
            // row scale 2^emax > max |xhat|
            emax = amax > 0.f ? ((__float_as_int(amax) >> 23) & 0xff) - 126 : 0;
            emax = max(min(emax, 100), -100);
        }
        // ---------------- digit slices of this row into shared memory, 8 columns at a time
        {
            const float sc = pow2f(-emax);
#pragma unroll
            for (int kg = 0; kg < TC_NK / 8; ++kg) {
                uint32_t packed[TC_MAXS][4];
#pragma unroll
                for (int h = 0; h < 8; h += 2) {
                    float dg[2][TC_MAXS];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const df xv = xk[8 * kg + h + e];
                        float x = F_MUL(xv.hi, sc), lo = F_MUL(xv.lo, sc);
                        float t = F_MUL(x, 128.0f);
                        dg[e][0] = rint_magic(t);
                        x = F_SUB(t, dg[e][0]);
#pragma unroll
                        for (int j = 1; j < 3; ++j) {
                            t = F_MUL(x, 256.0f);
                            dg[e][j] = rint_magic(t);
                            x = F_SUB(t, dg[e][j]);
                        }
                        x = F_ADD(x, F_MUL(lo, 8388608.0f));  // lo at the scale of digit 3
#pragma unroll
                        for (int j = 3; j < TC_MAXS; ++j) {
                            t = F_MUL(x, 256.0f);
                            dg[e][j] = rint_magic(t);
                            x = F_SUB(t, dg[e][j]);
                        }
                    }
#pragma unroll
                    for (int j = 0; j < TC_MAXS; ++j) {
                        __nv_bfloat162 b2 = __floats2bfloat162_rn(dg[0][j], dg[1][j]);
                        packed[j][h / 2] = *reinterpret_cast<uint32_t *>(&b2);
                    }
                }
#pragma unroll
                for (int j = 0; j < TC_MAXS; ++j) {
                    if (j < S)
                        *reinterpret_cast<uint4 *>(sA + j * A_SLICE_BYTES + kmaj_off(tid, 8 * kg)) =
                            make_uint4(packed[j][0], packed[j][1], packed[j][2], packed[j][3]);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---------------- MMAs: level d accumulates sum_{i+j=d} A_j B_i^T
        if (tid == 0) {
            for (int d = 0; d < S; ++d) {
                for (int i = 0; i <= d; ++i) {
                    const int j = d - i;
                    for (int kk = 0; kk < TC_NK / 16; ++kk) {
                        uint64_t da = umma_desc(smem_u32(sA + j * A_SLICE_BYTES) + kk * 256);
                        uint64_t db = umma_desc(smem_u32(sB + i * B_SLICE_BYTES) + kk * 256);
                        uint32_t dt = tbase + (uint32_t)(d * TC_NK);
                        uint32_t en = (i > 0 || kk > 0) ? 1u : 0u;
                        asm volatile(
                            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(
                                dt),
                            "l"(da), "l"(db), "r"(TC_IDESC), "r"(en));
                    }
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&mbar)));
        }
        uint32_t done = 0;
        for (uint32_t itw = 0; itw < TC_WAIT_LIMIT && !done; ++itw) {
            asm volatile(
                "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                "selp.u32 %0, 1, 0, p;\n\t}\n"
                : "=r"(done)
                : "r"(smem_u32(&mbar)), "r"(phase));
        }
        phase ^= 1u;
        if (!done) {
            atomicOr(status, ST_TIMEOUT);
            abort_flag = 1;
        }
        asm volatile("tcgen05.fence::after_thread_sync;");
        __syncthreads();
        if (abort_flag) break;
        // ---------------- read back this row, recombine the levels in df32
        df ch[TC_NK];
        {
            float Dv[TC_NK];
            tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)((S - 1) * TC_NK), Dv);
#pragma unroll
            for (int l = 0; l < TC_NK; ++l) ch[l] = df{Dv[l], 0.f};
            for (int d = S - 2; d >= 0; --d) {
                tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(d * TC_NK), Dv);
#pragma unroll
                for (int l = 0; l < TC_NK; ++l) {
                    // ch = ch * 2^-8 + D_d (D_d exact integers)
                    df t = df{F_MUL(ch[l].hi, 0.00390625f), F_MUL(ch[l].lo, 0.00390625f)};
                    df s2 = two_sum(Dv[l], t.hi);
                    ch[l] = fast_sum(s2.hi, F_ADD(s2.lo, t.lo));
                }
            }
        }
        // ---------------- rescale, postscale, reduce over the item's pairs
        dc vp = v;
#pragma unroll
        for (int l = 0; l < TC_NK; ++l) {
            if (l > p) continue;  // uniform over the CTA
            // chat_l = 2^(emax + f_l - 14) * sum_d 2^-8d D_d
            const float sl = pow2f(emax + sf[l] - 14);
            df c{F_MUL(ch[l].hi, sl), F_MUL(ch[l].lo, sl)};
            df other = shfl_df(c, 1);
            dc cc{comp ? other : c, comp ? c : other};
            df contrib{0.f, 0.f};
            if (active) {
                dc term;
                if (l == 0) {
                    df S2 = df_add(df_mul(Dx, Dx), df_mul(Dy, Dy));
                    df ln = df_log_f(S2.hi, tab);
                    df lr = fast_sum(F_MUL(0.5f, ln.hi),
                                     F_MUL(0.5f, F_FMA(S2.lo, F_RCP(S2.hi), ln.lo)));
                    df an = df_atan2_f(Dy.hi, Dx.hi, tab + 5 * LOG_TAB);
                    float ci = F_MUL(F_FMA(Dy.lo, Dx.hi, -F_MUL(Dx.lo, Dy.hi)), F_RCP(S2.hi));
                    df li = fast_sum(an.hi, F_ADD(an.lo, ci));
                    dc t0 = dc_mul(A0, dc{lr, li});
                    term = dc{df_add(cc.re, t0.re), df_add(cc.im, t0.im)};
                } else {
                    const float il = pow2f(-l);
                    dc a0l{df_divf(df{A0.re.hi * il, A0.re.lo * il}, (float)l),
                           df_divf(df{A0.im.hi * il, A0.im.lo * il}, (float)l)};
                    dc dd{df_add(cc.re, df_neg(a0l.re)), df_add(cc.im, df_neg(a0l.im))};
                    term = dc_mul(dd, vp);
                    vp = dc_mul(vp, v);
                }
                contrib = comp ? term.im : term.re;
            }
#pragma unroll
            for (int m = 2; m < 32; m <<= 1) contrib = df_acc(contrib, shfl_df(contrib, m));
            if (lane < 2) red[warp][l][comp] = make_float2(contrib.hi, contrib.lo);
        }
        __syncthreads();
        if (tid < 2 * (p + 1)) {
            const int l = tid >> 1, c = tid & 1;
            df sum{0.f, 0.f};
#pragma unroll
            for (int w = 0; w < 4; ++w) sum = df_acc(sum, df{red[w][l][c].x, red[w][l][c].y});
            double *out = reinterpret_cast<double *>(local + g * (p + 1));
            atomicAdd(out + 2 * l + c, (double)sum.hi + (double)sum.lo);
        }
        // the next item overwrites sA, red and TMEM only after everybody is done here
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tbase));
}

__global__ void k_mpole_df_tc(int64_t n, const double2 *__restrict__ in, float4 *__restrict__ out) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 v = in[i];
    df r = split_d(v.x), m = split_d(v.y);
    out[i] = make_float4(r.hi, r.lo, m.hi, m.lo);
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

}  // namespace

cudaError_t upload_df_tables_tc() {
    static float tab[DF_TAB_FLOATS];
    df32_fill_tables(tab);
    return cudaMemcpyToSymbol(d_tctab, tab, sizeof(tab));
}

int m2l_tc_max_p() { return TC_NK - 1; }

// Digit slices of the scaled operator Ahat_{lk} = C(k+l-1, l) 2^-(k+l)
// (row l, column k-1), per-row exponents f_l with |row| < 2^f_l, in the
// canonical K-major layout; exact from long-double binomials.
fmm_status build_m2l_tc_operator(Tree &t, int slices, cudaStream_t s) {
    const int p = t.p;
    std::vector<unsigned char> bytes((size_t)TC_MAXS * B_SLICE_BYTES, 0);
    std::vector<int> fexp(TC_NK, 0);
    for (int l = 0; l <= p; ++l) {
        long double row[TC_NK] = {};
        long double mx = 0;
        for (int k = 1; k <= p; ++k) {
            long double c = 1;  // C(k+l-1, l)
            for (int i = 1; i <= l; ++i) c = c * (long double)(k - 1 + i) / (long double)i;
            c = roundl(c);
            row[k - 1] = ldexpl(c, -(k + l));
            if (row[k - 1] > mx) mx = row[k - 1];
        }
        int f = 0;
        if (mx > 0) {
            frexpl(mx, &f);  // mx = m 2^f, m in [0.5, 1)
        }
        fexp[l] = f;
        for (int k = 0; k < TC_NK; ++k) {
            long double x = ldexpl(row[k], -f);  // in [0, 1)
            long double t0 = x * 128.0L;
            for (int j = 0; j < TC_MAXS; ++j) {
                long double dgt = roundl(t0);
                x = t0 - dgt;
                t0 = x * 256.0L;
                __nv_bfloat16 b = __float2bfloat16_rn((float)dgt);
                std::memcpy(&bytes[(size_t)j * B_SLICE_BYTES + kmaj_off(l, k)], &b, 2);
            }
        }
    }
    cudaError_t e;
    if ((e = arena_alloc(t.mem, &t.m2l_bslices, bytes.size() / 16)) != cudaSuccess ||
        (e = arena_alloc(t.mem, &t.m2l_fexp, TC_NK)) != cudaSuccess)
        return cuda_fail(e, "m2l operator");
    if ((e = cudaMemcpyAsync(t.m2l_bslices, bytes.data(), bytes.size(), cudaMemcpyHostToDevice, s)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(t.m2l_fexp, fexp.data(), TC_NK * sizeof(int), cudaMemcpyHostToDevice,
                             s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
        return cuda_fail(e, "m2l operator upload");
    t.m2l_slices = slices;
    return FMM_OK;
}

fmm_status launch_m2l_tc(Tree &t, cudaStream_t s) {
    cudaError_t e;
    const int64_t nc = t.n_boxes * (int64_t)(t.p + 1);
    if ((e = cudaMemsetAsync(t.local, 0, nc * sizeof(double2), s)) != cudaSuccess)
        return cuda_fail(e, "zero locals");
    k_mpole_df_tc<<<nblk(nc, 256), 256, 0, s>>>(nc, t.mpole, t.mpole_df); note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "mpole df32");
    if (t.n_m2l_items == 0) return FMM_OK;
    // pad so that at most two CTAs share an SM (2 x 256 TMEM columns)
    const int smem = std::max(TC_MAXS * (A_SLICE_BYTES + B_SLICE_BYTES), 100 * 1024);
    static bool attr_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev]) {
        if ((e = cudaFuncSetAttribute(k_m2l_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      smem)) != cudaSuccess)
            return cuda_fail(e, "m2l tc smem");
        attr_set[dev] = true;
    }
    const int grid = (int)std::min<int64_t>(t.n_m2l_items, 2 * 152);
    k_m2l_tc<<<grid, TC_ROWS, smem, s>>>(t.m2l_items, t.n_m2l_items, t.p, t.m2l_slices, t.geom,
                                         t.weak_off, t.weak, t.mpole_df,
                                         reinterpret_cast<const uint4 *>(t.m2l_bslices),
                                         t.m2l_fexp, t.local, t.status); note_launch();
    e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "m2l tc");
}

}  // namespace gbfmm
