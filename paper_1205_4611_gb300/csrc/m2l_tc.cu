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
#include <map>
#include <mutex>
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
// M = 128, N = n.
GBI uint32_t tc_idesc(int n) {  // n a multiple of 16, <= 256
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
           ((uint32_t)(TC_ROWS >> 4) << 24);
}

GBI float pow2f(int e) { return __int_as_float((e + 127) << 23); }  // e in [-126, 127]

GBI df split_d(double v) {
    float hi = __double2float_rn(v);
    float lo = __double2float_rn(v - (double)hi);
    return df{hi, lo};
}

GBI df df_acc(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    return df{s.hi, F_ADD(s.lo, F_ADD(a.lo, b.lo))};
}
GBI df shfl_df(df v, int m, unsigned mask = 0xffffffffu) {
    return df{__shfl_xor_sync(mask, v.hi, m), __shfl_xor_sync(mask, v.lo, m)};
}
// c - a b in one pass
GBI df df_sub_mul(df c, df a, df b) {
    const df p = two_prod(a.hi, b.hi);
    const df s = two_sum(c.hi, -p.hi);
    const float t = F_FMA(a.hi, b.lo, F_FMA(a.lo, b.hi, p.lo));
    return fast_sum(s.hi, F_ADD(s.lo, F_SUB(c.lo, t)));
}
GBI float rint_magic(float t) {  // round to nearest integer, |t| < 2^22
    return F_SUB(F_ADD(t, 12582912.0f), 12582912.0f);
}

GBI void tmem_ld16(uint32_t addr, float *v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
        "%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15])
        : "r"(addr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 16-byte asynchronous global -> shared copy (completes at cp_async_wait)
GBI void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src));
}
GBI void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src));
}
GBI void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
GBI void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

constexpr int TC_THREADS = 2 * TC_ROWS;  // two threads per GEMM row
// dynamic shared memory: slices of A (S x 8 KB), of the operator (S x 2 KB),
// then the staged multipoles of the next item (64 pairs x 32 float4)
constexpr int TC_SMP_OFF = TC_MAXS * (A_SLICE_BYTES + B_SLICE_BYTES);
constexpr int TC_SMP_BYTES = 64 * TC_NK * 16;
constexpr int RED_STRIDE = TC_ROWS + 1;  // float2 per row of the reduction buffer (padded)

// 2^e for e >= -126 (smaller: 0); e <= 127
GBI float pow2f_or0(int e) { return e < -126 ? 0.0f : pow2f(e); }

// binary exponent of a normal double (floor(log2 x); exact for sigma = 2^e)
GBI int exp_of(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) - 1023; }


// One CTA of 256 threads per item (<= 64 weak pairs of one target box).  GEMM
// row r = 2q + c is component c (0 = re, 1 = im) of pair q; threads r and
// r + 128 share the row (warps w and w + 4 read the same TMEM lanes): half
// h = 0 takes k = 1..16 of the prescale and l = 0..15 of the postscale, half
// h = 1 takes k = 17..31 and l = 16..31.  The two rows of a pair split every
// complex product between them (each forms its own component and takes the
// partner's through a shuffle).
//
// Scaled variables: with 2^e0 = max(sigma_s, sigma_t) and ir = 2^e0 / r,
//   xhat_k = (-1)^k A_k (2u)^k = (-1)^k 2^{k a_s} A_k ir^k,   a_s = e_s - e0 + 1,
//   (2v)^l = 2^{l a_t} ir^l,                                  a_t = e_t - e0 + 1,
// so one chain of powers of ir (|ir| <= 1/2 under the theta-criterion) serves
// the prescale and the postscale, and every other factor is an exact power
// of two (underflowing to 0 where the term is negligible).
template <int PM>
__global__ void __launch_bounds__(TC_THREADS)
    k_m2l_tc(int n_weak, int p, int S, const double4 *__restrict__ geom,
             const int *__restrict__ weak, const int *__restrict__ weak_tgt,
             const float4 *__restrict__ mp, const uint4 *__restrict__ bslices,
             const int *__restrict__ fexp, double2 *__restrict__ local, int *status) {
    pdl_wait();
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sA = smem_raw;                            // S x 8 KB
    unsigned char *sB = smem_raw + TC_MAXS * A_SLICE_BYTES;  // S x 2 KB
    float2 *red = reinterpret_cast<float2 *>(smem_raw);      // [l][row], aliases sA after the MMAs
    __shared__ __align__(16) float tab[DF_TAB_FLOATS];
    __shared__ int sf[TC_NK];
    __shared__ float2 sinv[TC_NK];  // 2^-l / l as df32
    __shared__ float samax[2][TC_ROWS];
    __shared__ __align__(16) double4 sgeo[64];  // next item: geometry of its source boxes
    __shared__ __align__(16) double4 sgt[64];   // next item: geometry of its target boxes
    __shared__ int stgt[64];                    // next item: target box of every pair
    __shared__ int snp;                         // next item: number of pairs
    // this item, per pair: ir = 2^e0 / r and D = z_t - z_s as df32, the
    // exponent offsets (a_s, a_t) and the target box (formed once per pair)
    __shared__ __align__(16) float4 pir[64], pD[64];
    __shared__ int4 pe[64];
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5;
    const int row = tid & (TC_ROWS - 1), h = tid >> 7;
    const int comp = row & 1, q = row >> 1;
    const int kb = 16 * h;  // this half's first column (k - 1, and l)
    // one-time set-up: tables, operator slices, mbarrier, TMEM
    for (int i = tid; i < DF_TAB_FLOATS; i += TC_THREADS) tab[i] = d_tctab[i];
    for (int i = tid; i < S * B_SLICE_BYTES / 16; i += TC_THREADS)
        reinterpret_cast<uint4 *>(sB)[i] = bslices[i];
    if (tid < TC_NK) {
        sf[tid] = fexp[tid];
        const df v = tid ? split_d(ldexp(1.0, -tid) / tid) : df{0.f, 0.f};
        sinv[tid] = make_float2(v.hi, v.lo);
    }
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
    const uint32_t tlane = (uint32_t)((warp & 3) * 32) << 16;
    uint32_t phase = 0;
    float4 *smp = reinterpret_cast<float4 *>(smem_raw + TC_SMP_OFF);  // [pair][k]

    // Stage item `nx` (its multipoles, box geometry and sizes) into shared memory
    // with asynchronous copies; they complete at the next cp_async_wait.
    const int n_items = (n_weak + 63) / 64;  // item k: weak entries [64 k, 64 k + 64)
    auto prefetch = [&](int nx) {
        if (nx >= n_items) return;
        const int e0 = nx * 64;
        const int npn = min(64, n_weak - e0);
        // warp w copies pairs w, w + 8, ..., lane k coefficient k (p < 32)
        for (int pq = warp; pq < npn; pq += TC_THREADS / 32) {
            const int lane = tid & 31;
            if (lane <= p)
                cp_async16(smp + pq * (p + 1) + lane,
                           mp + (int64_t)weak[e0 + pq] * (p + 1) + lane);
        }
        if (tid < npn) {
            const double4 *src = geom + weak[e0 + tid];
            cp_async16(&sgeo[tid], src);
            cp_async16(reinterpret_cast<char *>(&sgeo[tid]) + 16,
                       reinterpret_cast<const char *>(src) + 16);
        } else if (tid >= 128 && tid - 128 < npn) {
            const int qn = tid - 128;
            const double4 *tg = geom + weak_tgt[e0 + qn];
            cp_async16(&sgt[qn], tg);
            cp_async16(reinterpret_cast<char *>(&sgt[qn]) + 16,
                       reinterpret_cast<const char *>(tg) + 16);
            cp_async4(&stgt[qn], weak_tgt + e0 + qn);
        }
        if (tid == TC_THREADS - 1) snp = npn;
        cp_async_commit();
    };
    prefetch(blockIdx.x);
    cp_async_wait();
    __syncthreads();

    for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
        const int n_pairs = snp;
        // ---------------- per-pair geometry, once per pair (the FP64 pipe is narrow)
        if (tid < 64) {
            float4 ir4 = make_float4(0.f, 0.f, 0.f, 0.f), D4 = make_float4(1.f, 0.f, 0.f, 0.f);
            int4 e4 = make_int4(0, 0, 0, 0);
            if (tid < n_pairs) {
                const double4 gs = sgeo[tid], gt = sgt[tid];
                const int e_s = exp_of(gs.z), e_t = exp_of(gt.z);
                // 2^e0 >= the larger sigma, and not below 2^-100 |D| (boxes of radius ~0
                // far apart: their powers underflow to 0, which is their true size)
                const int e_d = max(exp_of(fabs(gt.x - gs.x)), exp_of(fabs(gt.y - gs.y)));
                const int e0 = max(max(e_s, e_t), e_d - 100);
                // D = z_t - z_s (FP64 difference: an exactly shared ordinate gives +0)
                const df Dx = split_d(gt.x - gs.x), Dy = split_d(gt.y - gs.y);
                // Ds = D / 2^e0: both float parts scaled by a power of two (exact);
                // through FP64 when 2^-e0 lies outside the float range
                df Dsx, Dsy;
                if (e0 > -127 && e0 < 127) {
                    const float f = __int_as_float((127 - e0) << 23);
                    Dsx = df{F_MUL(Dx.hi, f), F_MUL(Dx.lo, f)};
                    Dsy = df{F_MUL(Dy.hi, f), F_MUL(Dy.lo, f)};
                } else {
                    const double sc0 = __hiloint2double((1023 - e0) << 20, 0);  // 2^-e0
                    Dsx = split_d((gt.x - gs.x) * sc0);
                    Dsy = split_d((gt.y - gs.y) * sc0);
                }
                // ir = 2^e0 / r with r = -D:  -conj(Ds) / |Ds|^2
                const df n2 = df_dot2(Dsx, Dsx, Dsy, Dsy);
                const float i0 = F_RCP(n2.hi);
                const df corr = df_add(df{1.0f, 0.f}, df_neg(df_mulf(n2, i0)));
                const df inv = df_add(df{i0, 0.f}, df_mulf(corr, i0));
                const df ir_re = df_neg(df_mul(Dsx, inv)), ir_im = df_mul(Dsy, inv);
                ir4 = make_float4(ir_re.hi, ir_re.lo, ir_im.hi, ir_im.lo);
                D4 = make_float4(Dx.hi, Dx.lo, Dy.hi, Dy.lo);
                e4 = make_int4(e_s - e0 + 1, e_t - e0 + 1, stgt[tid], 0);
            }
            pir[tid] = ir4;
            pD[tid] = D4;
            pe[tid] = e4;
        }
        __syncthreads();
        const bool active = q < n_pairs;
        const float4 ir4 = pir[q], D4 = pD[q];
        const int a_s = pe[q].x, a_t = pe[q].y;
        const df Dx{D4.x, D4.y}, Dy{D4.z, D4.w};
        const df ir_re{ir4.x, ir4.y}, ir_im{ir4.z, ir4.w};
        const df ir_own = comp ? ir_im : ir_re, ir_oth = comp ? ir_re : ir_im;
        const df ir_oth_s = comp ? ir_oth : df_neg(ir_oth);
        const float4 *Ap = smp + q * (p + 1);  // this row's pair
        const float4 a0v = active ? Ap[0] : make_float4(0.f, 0.f, 0.f, 0.f);
        const df A0re{a0v.x, a0v.y}, A0im{a0v.z, a0v.w};
        // ---------------- powers ir^(kb+1) to start this half's chain
        df P_own = ir_own, P_oth = ir_oth;
        df pbase = df{0.f, 0.f};  // own component of ir^kb (half 1: ir^16)
        if (h) {
            // ir^16 by four squarings:  re = Pre^2 - Pim^2,  im = 2 Pre Pim
#pragma unroll
            for (int sq = 0; sq < 4; ++sq) {
                const df nxt = df_dot2(P_own, comp ? P_oth : P_own, comp ? P_oth : df_neg(P_oth),
                                       comp ? P_own : P_oth);
                P_own = nxt;
                P_oth = shfl_df(nxt, 1);
            }
            pbase = P_own;
            const df nxt = df_dot2(ir_own, comp ? P_oth : P_own, ir_oth_s, comp ? P_own : P_oth);
            P_own = nxt;
            P_oth = shfl_df(nxt, 1);
        }
        // ---------------- prescale: xhat_k (own component), k = kb+1 .. kb+16
        df xk[16], pk[16];
        float amax = 0.f;
        // 2^{k a_s} as a running product of powers of two (0 past the float range)
        float sk = pow2f_or0((kb + 1) * a_s);
        const float fs = pow2f_or0(a_s);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
            const int k = kb + kk + 1;
            xk[kk] = df{0.f, 0.f};
            pk[kk] = df{0.f, 0.f};
            if (k <= p && k <= PM) {
                const float4 a4 = active ? Ap[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                const df Are{a4.x, a4.y}, Aim{a4.z, a4.w};
                // own component of A_k ir^k:  re = Are Pre - Aim Pim,  im = Are Pim + Aim Pre
                df x = df_dot2(Are, P_own, Aim, comp ? P_oth : df_neg(P_oth));
                x = df{F_MUL(x.hi, sk), F_MUL(x.lo, sk)};
                sk = F_MUL(sk, fs);
                xk[kk] = (k & 1) ? df_neg(x) : x;
                amax = fmaxf(amax, fabsf(x.hi));
                pk[kk] = P_own;
                const df nxt = df_dot2(ir_own, comp ? P_oth : P_own, ir_oth_s,
                                       comp ? P_own : P_oth);
                P_own = nxt;
                P_oth = shfl_df(nxt, 1);
            }
        }
        samax[h][row] = amax;
        __syncthreads();  // staged multipoles are overwritten below; row maxima complete
        amax = fmaxf(samax[0][row], samax[1][row]);
        int emax = amax > 0.f ? ((__float_as_int(amax) >> 23) & 0xff) - 126 : 0;
        emax = max(min(emax, 100), -100);
        // ---------------- digit slices of this half-row into shared memory
        {
            const float scl = pow2f(-emax);
#pragma unroll
            for (int kg2 = 0; kg2 < 2; ++kg2) {
                uint32_t packed[TC_MAXS][4];
#pragma unroll
                for (int hh = 0; hh < 8; hh += 2) {
                    float dg[2][TC_MAXS];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const df xv = xk[8 * kg2 + hh + e];
                        float x = F_MUL(xv.hi, scl), lo = F_MUL(xv.lo, scl);
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
                        packed[j][hh / 2] = *reinterpret_cast<uint32_t *>(&b2);
                    }
                }
#pragma unroll
                for (int j = 0; j < TC_MAXS; ++j) {
                    if (j < S)
                        *reinterpret_cast<uint4 *>(sA + j * A_SLICE_BYTES +
                                                   kmaj_off(row, kb + 8 * kg2)) =
                            make_uint4(packed[j][0], packed[j][1], packed[j][2], packed[j][3]);
                }
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        // ---------------- MMAs: level d accumulates sum_{i+j=d} A_j B_i^T.  One
        // MMA chain per A slice j covers its levels d = j .. S-1 at once: the
        // operator slices B_0 .. B_{S-1-j} are consecutive in shared memory, so
        // they form one N = 32 (S - j) operand written to TMEM columns from 32 j.
        if (tid == 0) {
            for (int j = 0; j < S; ++j) {
                const uint32_t idesc = tc_idesc(TC_NK * (S - j));
                for (int kk = 0; kk < TC_NK / 16; ++kk) {
                    uint64_t da = umma_desc(smem_u32(sA + j * A_SLICE_BYTES) + kk * 256);
                    uint64_t db = umma_desc(smem_u32(sB) + kk * 256);
                    uint32_t dt = tbase + (uint32_t)(j * TC_NK);
                    uint32_t en = (j > 0 || kk > 0) ? 1u : 0u;
                    asm volatile(
                        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
                        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(dt),
                        "l"(da), "l"(db), "r"(idesc), "r"(en));
                }
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                    smem_u32(&mbar)));
        }
        // the next item's data, copied while the tensor cores and the rest of
        // this item run (the staged multipoles of this item are consumed)
        prefetch(item + gridDim.x);
        // Log(z_t - z_s) for the l = 0 term (half 0) while the tensor cores run
        df lr{0.f, 0.f}, li{0.f, 0.f};
        if (h == 0) {
            const df S2 = df_add(df_mul(Dx, Dx), df_mul(Dy, Dy));
            const df ln = df_log_f(S2.hi, tab);
            lr = fast_sum(F_MUL(0.5f, ln.hi), F_MUL(0.5f, F_FMA(S2.lo, F_RCP(S2.hi), ln.lo)));
            const df an = df_atan2_f(Dy.hi, Dx.hi, tab + ATAN_OFF);
            const float ci = F_MUL(F_FMA(Dy.lo, Dx.hi, -F_MUL(Dx.lo, Dy.hi)), F_RCP(S2.hi));
            li = fast_sum(an.hi, F_ADD(an.lo, ci));
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
        asm volatile("fence.proxy.async.shared::cta;");  // sA is rewritten (red) below
        __syncthreads();
        if (abort_flag) break;
        // ---------------- read back this half-row, recombine the levels in df32
        df ch[16];
        {
            float Dv[16];
            tmem_ld16(tbase + tlane + (uint32_t)((S - 1) * TC_NK + kb), Dv);
#pragma unroll
            for (int l = 0; l < 16; ++l) ch[l] = df{Dv[l], 0.f};
            int d = S - 2;
            if (d >= 0) {
                // the two lowest levels in one float: |D| < 2^22, so the rounding
                // of D_{S-2} + 2^-8 D_{S-1} is below 2^-2 units of level S-2, i.e.
                // 2^-(8 (S-2) + 2) units of level 0: below both the truncation of
                // the S digit slices (2^(22 - 8 S) units) and, for S = 6, the df32
                // rounding of level-0 values up to 2^22 (2^-26 units)
                tmem_ld16(tbase + tlane + (uint32_t)(d * TC_NK + kb), Dv);
#pragma unroll
                for (int l = 0; l < 16; ++l) ch[l] = df{F_FMA(ch[l].hi, 0.00390625f, Dv[l]), 0.f};
                --d;
            }
            for (; d >= 0; --d) {
                tmem_ld16(tbase + tlane + (uint32_t)(d * TC_NK + kb), Dv);
#pragma unroll
                for (int l = 0; l < 16; ++l) {
                    // ch = ch * 2^-8 + D_d (D_d exact integers)
                    df t = df{F_MUL(ch[l].hi, 0.00390625f), F_MUL(ch[l].lo, 0.00390625f)};
                    df s2 = two_sum(Dv[l], t.hi);
                    ch[l] = fast_sum(s2.hi, F_ADD(s2.lo, t.lo));
                }
            }
        }
        // ---------------- rescale, postscale; one term per (l, row) into shared memory
        const df A0own = comp ? A0im : A0re;
        float vs = pow2f_or0(kb * a_t);  // 2^{l a_t}, a running product
        const float ft = pow2f_or0(a_t);
#pragma unroll
        for (int ll = 0; ll < 16; ++ll) {
            const int l = kb + ll;
            if (l > p || l > PM) continue;  // uniform over the warp
            // chat_l = 2^(emax + f_l - 14) * sum_d 2^-8d D_d (own component)
            const float sl = pow2f(emax + sf[l] - 14);
            const df c{F_MUL(ch[ll].hi, sl), F_MUL(ch[ll].lo, sl)};
            df term;
            if (l == 0) {
                // + A_0 Log(z_t - z_s):  re = A0re lr - A0im li,  im = A0re li + A0im lr
                const df t0 = df_dot2(A0re, comp ? li : lr, comp ? A0im : df_neg(A0im),
                                      comp ? lr : li);
                term = df_add(c, t0);
            } else {
                // (chat_l - A_0 2^-l / l) (2v)^l;  (2v)^l = 2^{l a_t} ir^l, ir^l = pk of k = l
                const df il{sinv[l].x, sinv[l].y};
                const df dd_own = df_sub_mul(c, A0own, il);
                const df dd_oth = shfl_df(dd_own, 1);
                // ir^l: pk[ll - 1] holds ir^(kb + ll), and ir^kb is pbase
                const df pw = ll == 0 ? pbase : pk[ll > 0 ? ll - 1 : 0];
                const df V_own{F_MUL(pw.hi, vs), F_MUL(pw.lo, vs)};
                const df V_oth = shfl_df(V_own, 1);
                // re = dre Vre - dim Vim ;  im = dre Vim + dim Vre
                const df dre = comp ? dd_oth : dd_own, dim = comp ? dd_own : dd_oth;
                term = df_dot2(dre, V_own, dim, comp ? V_oth : df_neg(V_oth));
            }
            red[l * RED_STRIDE + row] = active ? make_float2(term.hi, term.lo) : make_float2(0.f, 0.f);
            vs = F_MUL(vs, ft);
        }
        __syncthreads();
        // ---------------- sum over the item's pairs: output (l, c) by four threads
        {
            const int o = tid >> 2, qq = tid & 3;  // o = 2 l + c
            const int l = o >> 1, c = o & 1;
            const int g_first = pe[0].z, g_last = pe[n_pairs - 1].z;
            if (g_first == g_last) {  // one target box (uniform over the CTA)
                df sum{0.f, 0.f};
                if (l <= p) {
                    for (int pq = qq; pq < n_pairs; pq += 4) {
                        const float2 v = red[l * RED_STRIDE + 2 * pq + c];
                        sum = df_acc(sum, df{v.x, v.y});
                    }
                }
                sum = fast_sum(sum.hi, sum.lo);
                sum = df_add(sum, shfl_df(sum, 1));
                sum = df_add(sum, shfl_df(sum, 2));
                if (qq == 0 && l <= p) {
                    double *out = reinterpret_cast<double *>(local + (int64_t)g_first * (p + 1));
                    atomicAdd(out + 2 * l + c, (double)sum.hi + (double)sum.lo);
                }
            } else if (l <= p) {
                // pairs of several target boxes (consecutive in entry order): each
                // thread sums a contiguous quarter and adds at every change of box
                const int q0 = 16 * qq, q1 = min(q0 + 16, n_pairs);
                df sum{0.f, 0.f};
                int gcur = -1;
                for (int pq = q0; pq < q1; ++pq) {
                    const int gq = pe[pq].z;
                    if (gq != gcur) {
                        if (gcur >= 0) {
                            double *out = reinterpret_cast<double *>(local + (int64_t)gcur * (p + 1));
                            atomicAdd(out + 2 * l + c, (double)sum.hi + (double)sum.lo);
                        }
                        gcur = gq;
                        sum = df{0.f, 0.f};
                    }
                    const float2 v = red[l * RED_STRIDE + 2 * pq + c];
                    sum = df_acc(sum, df{v.x, v.y});
                }
                if (gcur >= 0) {
                    double *out = reinterpret_cast<double *>(local + (int64_t)gcur * (p + 1));
                    atomicAdd(out + 2 * l + c, (double)sum.hi + (double)sum.lo);
                }
            }
        }
        // the next item overwrites sA / red and TMEM only after everybody is done
        // here, and reads the data prefetched above
        cp_async_wait();
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tbase));
}



}  // namespace

cudaError_t upload_df_tables_tc() {
    alignas(16) static float tab[DF_TAB_FLOATS];
    df32_fill_tables(tab);
    return cudaMemcpyToSymbol(d_tctab, tab, sizeof(tab));
}

int m2l_tc_max_p() { return TC_NK - 1; }

// Digit slices of the scaled operator Ahat_{lk} = C(k+l-1, l) 2^-(k+l)
// (row l, column k-1), per-row exponents f_l with |row| < 2^f_l, in the
// canonical K-major layout; exact from long-double binomials.  The operator
// depends only on p: it is built once per (device, p) and kept for the life
// of the process (a few KB).
static std::mutex g_op_mu;
static std::map<std::pair<int, int>, std::pair<uint4 *, int *>> g_op_cache;

fmm_status build_m2l_tc_operator(Tree &t, int slices, cudaStream_t /*s*/) {
    const int p = t.p;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "m2l operator");
    std::lock_guard<std::mutex> lk(g_op_mu);
    auto it = g_op_cache.find({dev, p});
    if (it == g_op_cache.end()) {
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
        uint4 *bs = nullptr;
        int *fx = nullptr;
        if ((e = cudaMalloc(reinterpret_cast<void **>(&bs), bytes.size())) != cudaSuccess ||
            (e = cudaMalloc(reinterpret_cast<void **>(&fx), TC_NK * sizeof(int))) != cudaSuccess ||
            (e = cudaMemcpy(bs, bytes.data(), bytes.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(fx, fexp.data(), TC_NK * sizeof(int), cudaMemcpyHostToDevice)) !=
                cudaSuccess) {
            if (bs) cudaFree(bs);
            if (fx) cudaFree(fx);
            return cuda_fail(e, "m2l operator upload");
        }
        it = g_op_cache.emplace(std::make_pair(dev, p), std::make_pair(bs, fx)).first;
    }
    t.m2l_bslices = it->second.first;
    t.m2l_fexp = it->second.second;
    t.m2l_slices = slices;
    return FMM_OK;
}

fmm_status launch_m2l_tc(Tree &t, cudaStream_t s) {
    cudaError_t e;
    if (t.n_weak == 0) return FMM_OK;
    // at most two CTAs share an SM (2 x 256 TMEM columns): 128 registers x 256
    // threads fill half the register file, and a third CTA's shared memory
    // would not fit either
    const int smem = TC_SMP_OFF + TC_SMP_BYTES;
    auto k = t.p <= 16 ? k_m2l_tc<16> : t.p <= 24 ? k_m2l_tc<24> : k_m2l_tc<31>;
    const int ki = t.p <= 16 ? 0 : t.p <= 24 ? 1 : 2;
    static bool attr_set[64][3] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && !attr_set[dev][ki]) {
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem)) !=
            cudaSuccess)
            return cuda_fail(e, "m2l tc smem");
        attr_set[dev][ki] = true;
    }
    const int64_t n_items = (t.n_weak + 63) / 64;
    const int grid = (int)std::min<int64_t>(n_items, 2 * 152);
    launch_k(k, grid, TC_THREADS, smem, s, (int)t.n_weak, t.p, t.m2l_slices, t.geom, t.weak,
             t.weak_tgt, t.mpole_df, reinterpret_cast<const uint4 *>(t.m2l_bslices), t.m2l_fexp,
             t.local, t.status);
    e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "m2l tc");
}

}  // namespace gbfmm
