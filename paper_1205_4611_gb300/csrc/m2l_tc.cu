// M2L on the tensor cores (tcgen05): the binomial contraction of every weak
// pair as an exact split-precision fp16 GEMM with FP32 accumulation in TMEM,
// one GEMM row per pair.
//
// For a weak pair (s -> t), r = z_s - z_t, u = sigma_s / r, v = sigma_t / r
// (radius-normalised expansions, expand.cu), the M2L of Alg. "Multipole to
// local translation" (its two summation sweeps) applies the fixed operator
//     c_l = sum_{k=1}^{p} C(k+l-1, l) x_k,      x_k = (-1)^k A_k u^k,
// and B_l += (c_l - A_0 / l) v^l (l >= 1), B_0 += c_0 + A_0 Log(z_t - z_s).
// Scaled so that every operator entry is at most 1/2,
//     Ahat_{l0} = -2^-l / l (l >= 1),  Ahat_{lk} = C(k+l-1, l) 2^-(k+l) (k >= 1),
//     xhat_0 = A_0,  xhat_k = (-1)^k A_k (2u)^k,   chat_l = sum_{k=0}^{p} Ahat_lk xhat_k,
//     B_0 += chat_0 + A_0 Log(z_t - z_s),          B_l += chat_l (2v)^l,
// so the a_0 term of the local expansion is one more column of the fixed
// operator.  With 2^e0 = max(sigma_s, sigma_t) and ir = 2^e0 / r,
// (2u)^k = 2^{k a_s} ir^k and (2v)^l = 2^{l a_t} ir^l (a_s, a_t exact
// exponent offsets): one chain of powers of ir serves both scalings.
//
// Exact split precision.  Row q of the GEMM is pair q; its real and imaginary
// parts are two A operands that share the operator.  Every row is scaled by a
// power of two to |xhat| < 1 and cut into S signed digits (the first of 8
// bits, the others of 9: integers of magnitude <= 260, exact in fp16); the
// operator rows likewise (per-row exponent f_l).  A digit product is an
// integer below 2^16.1, so the sum of "level" d = i + j (at most 5 slice
// pairs of K = 32) stays below 2^24 and is exact in its FP32 accumulator.
// Slice A_j times the consecutive operator slices B_0 .. B_{5-j} is one MMA
// of N = 32 (6 - j) into the accumulators of levels j .. 5 (a zero sixth
// operator slice lets the A_0 product initialise all six).  Levels 0-2
// recombine exactly in double-float, levels 3-5 (below 2^-24 of level 0) as
// one float tail.  With S = 5 the digits carry 44 bits of each row; the
// levels left out (d >= 6) are below 2^-50 of level 0.
//
// Per CTA (persistent, one per SM, 512 threads): an item is 128 consecutive
// weak entries (across target boxes).  Four threads share a pair: quarter Q
// takes a group of consecutive expansion indices (the same k for the prescale
// and l for the postscale; quarter 0 one more, as index 0 costs almost
// nothing), which sit in GEMM positions [8Q, 8Q + 8) of K and N, so each
// thread writes one 16-byte chunk per digit slice and reads 8 TMEM columns
// per accumulator.  Per item: prescale -> component 0's digits in shared
// memory (canonical K-major layout, no swizzle) -> one thread issues its MMAs
// and commits them to the component's mbarrier -> component 1's digits while
// the tensor cores run component 0 -> its MMAs -> the next item's data is
// copied in (cp.async) while the tensor cores run -> each thread reads its
// row back with tcgen05.ld (component 0 while component 1 runs), recombines,
// postscales, and the per-target sums over the item's pairs go to the local expansions with FP64
// atomics.  The pair geometry (ir, Log(z_t - z_s), exponent offsets) depends
// on the tree only and is computed once per build (k_m2l_pairs).
//
// Every wait is bounded; a wait that gives up sets the tree's status word
// (ST_TIMEOUT), the CTA stops taking items, waits once more (with a longer
// bound) for its last commits and only then releases its tensor memory.
#include <cuda_fp16.h>
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

constexpr int R_ROWS = 128;                        // pairs per item = GEMM rows (M)
constexpr int R_NK = 32;                           // K and N positions
constexpr int R_S = 5;                             // most digit slices
constexpr int R_THREADS = 512;                     // four threads per pair
constexpr int X_SLICE = R_ROWS * R_NK * 2;         // 8 KB: one slice of one component
constexpr int B_SLICE = R_NK * R_NK * 2;           // 2 KB
constexpr int R_SBO = (R_NK / 8) * 128;            // 8-row group stride
constexpr int R_LBO = 128;                         // core-matrix stride along K
constexpr int RED_STRIDE = R_ROWS + R_ROWS / 16;   // float2 per (component, l) row, padded
constexpr int R_LEV = 6;                           // digit levels kept = accumulators per component
constexpr int R_CCOLS = R_LEV * R_NK;              // TMEM columns per component (192)
constexpr int R_TCOLS = 512;                       // TMEM columns allocated (2 x 192 used)
constexpr uint32_t R_WAIT_LIMIT = 1u << 22;
constexpr uint32_t R_DRAIN_LIMIT = 1u << 26;
constexpr float MAGIC = 12582912.0f;               // 1.5 * 2^23: round to an integer
constexpr int X_BYTES = R_S * 2 * X_SLICE;         // 80 KB
constexpr int B_BYTES = R_LEV * B_SLICE;           // 12 KB: S operator slices, zeros above

__host__ __device__ constexpr int pm_of(int p) { return p <= 16 ? 16 : p <= 24 ? 24 : 31; }
// First expansion index of quarter Q for the compiled order PM (indices
// 0 .. PM): quarter 0 takes one index more than the others, as index 0 costs
// almost nothing (xhat_0 = A_0, and the l = 0 term needs no power of ir).
__host__ __device__ constexpr int qstart(int pm, int Q) {
    return pm == 31 ? 8 * Q : (Q == 0 ? 0 : 1 + Q * (pm / 4));
}
__host__ __device__ constexpr int qcount(int pm, int Q) {
    return (Q == 3 ? pm + 1 : qstart(pm, Q + 1)) - qstart(pm, Q);
}
// GEMM position (K index of xhat_k, N index of chat_l) of expansion index k:
// quarter Q's indices sit in positions [8 Q, 8 Q + 8)
__host__ __device__ inline int gemm_pos(int k, int pm) {
    int Q = 3;
    while (Q > 0 && k < qstart(pm, Q)) --Q;
    return 8 * Q + (k - qstart(pm, Q));
}

__device__ float d_pairtab[DF_TAB_FLOATS];

__host__ __device__ inline int kmaj_off(int row, int k) {
    return (row >> 3) * R_SBO + (k >> 3) * R_LBO + (row & 7) * 16 + (k & 7) * 2;
}

GBI uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// kind::f16 instruction descriptor: D = F32, A = B = F16 (formats 0), both
// K-major, M = 128, N = n.
GBI uint32_t f16_idesc(int n) {  // n a multiple of 16, <= 256
    return (1u << 4) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(R_ROWS >> 4) << 24);
}

// Shared-memory matrix descriptor (canonical K-major layout, no swizzle):
// bits 0-13 start address / 16, 16-29 leading-byte offset / 16 (next core
// matrix along K), 32-45 stride-byte offset / 16 (next 8-row group), bit 46
// the descriptor version, base offset 0.  Low word: the start address
// (shared addresses are below 2^18, so the field never carries into the
// offsets) and the leading-byte offset; the high word is constant.
GBI uint32_t umma_desc_lo(uint32_t saddr) {
    return ((saddr >> 4) & 0x3FFFu) | ((uint32_t)(R_LBO >> 4) << 16);
}
constexpr uint32_t UMMA_DESC_HI = (uint32_t)(R_SBO >> 4) | (1u << 14);  // version bit 46

// D[col ..] (+)= A B^T over K = 32 (two MMAs of K = 16): A (128 x 32) and B
// (n x 32) in the canonical K-major layout, given by the low words of their
// descriptors (+16 per K = 16 step of 256 B); acc = false overwrites the
// accumulator.
GBI void mma_k32(uint32_t d, uint32_t da_lo, uint32_t db_lo, int n, bool acc) {
    const uint32_t idesc = f16_idesc(n);
#pragma unroll
    for (int kk = 0; kk < R_NK / 16; ++kk) {
        const uint32_t en = (acc || kk > 0) ? 1u : 0u;
        asm volatile(
            "{\n\t.reg .pred p;\n\t.reg .b64 da, db;\n\t"
            "mov.b64 da, {%1, %5};\n\tmov.b64 db, {%2, %5};\n\t"
            "setp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], da, db, %3, p;\n\t}\n" ::"r"(d),
            "r"(da_lo + 16u * kk), "r"(db_lo + 16u * kk), "r"(idesc), "r"(en),
            "n"(UMMA_DESC_HI));
    }
}

GBI float pow2f(int e) { return __int_as_float((e + 127) << 23); }  // e in [-126, 127]
GBI float pow2f_or0(int e) { return e < -126 ? 0.0f : pow2f(e); }    // e <= 127
// binary exponent of a normal double (floor(log2 x); exact for sigma = 2^e)
GBI int exp_of(double x) { return ((__double2hiint(x) >> 20) & 0x7ff) - 1023; }

GBI df split_d(double v) {
    float hi = __double2float_rn(v);
    float lo = __double2float_rn(v - (double)hi);
    return df{hi, lo};
}
GBI df df_acc(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    return df{s.hi, F_ADD(s.lo, F_ADD(a.lo, b.lo))};
}

struct cdf {
    df re, im;
};
GBI cdf cmul(const cdf &a, const cdf &b) {
    return cdf{df_dot2(a.re, b.re, df_neg(a.im), b.im), df_dot2(a.re, b.im, a.im, b.re)};
}
// a b with the low parts left unnormalised (power chains, the postscale)
GBI cdf cmul_lz(const cdf &a, const cdf &b) {
    return cdf{df_dot2_lz(a.re, b.re, df_neg(a.im), b.im), df_dot2_lz(a.re, b.im, a.im, b.re)};
}
GBI cdf csq(const cdf &a) {
    const df m = df_mul(a.re, a.im);
    return cdf{df_dot2(a.re, a.re, df_neg(a.im), a.im), df{F_ADD(m.hi, m.hi), F_ADD(m.lo, m.lo)}};
}
// a^n by squaring (n >= 0, warp-uniform)
GBI cdf cpow(const cdf &a, int n) {
    cdf r{df{1.f, 0.f}, df{0.f, 0.f}}, b = a;
    bool first = true;
    while (n) {
        if (n & 1) {
            r = first ? b : cmul(r, b);
            first = false;
        }
        n >>= 1;
        if (n) b = csq(b);
    }
    return r;
}

// Three accumulators (8 columns each, at a + 32 i) for this warp's 32
// lanes, and the wait for them, in one statement (the registers are defined
// only after the wait).
GBI void tmem_ld8x3(uint32_t a, float (*v)[8]) {
    uint32_t r[24];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%24];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%8,%9,%10,%11,%12,%13,%14,%15}, [%25];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%16,%17,%18,%19,%20,%21,%22,%23}, [%26];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
          "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
          "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23])
        : "r"(a), "r"(a + 32), "r"(a + 64)
        : "memory");
#pragma unroll
    for (int k = 0; k < 3; ++k)
#pragma unroll
        for (int i = 0; i < 8; ++i) v[k][i] = __uint_as_float(r[8 * k + i]);
}
// One accumulator (8 columns at a) and the wait for it.
GBI void tmem_ld8(uint32_t a, float *v) {
    uint32_t r[8];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7])
        : "r"(a)
        : "memory");
#pragma unroll
    for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

GBI void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst)), "l"(src));
}
GBI void cp_async8(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src));
}
GBI void cp_async4(void *dst, const void *src) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src));
}
GBI void cp_async_commit() { asm volatile("cp.async.commit_group;"); }
GBI void cp_async_wait() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Bounded wait for the completion of phase `parity` of an mbarrier.
GBI bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit) {
    uint32_t done = 0;
    for (uint32_t it = 0; it < limit && !done; ++it) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}\n"
            : "=r"(done)
            : "r"(smem_u32(bar)), "r"(parity));
    }
    return done != 0;
}

// The S digits of one component: v = (hi, lo) with |hi + lo| < 2^emax;
// s256 = 2^(8 - emax), s17 = 2^(17 - emax).  Digit 0 has 8 bits, the others
// 9; every step is exact (the remainder after each digit is formed by an
// FMA), the low part enters through an exact TwoSum at the scale of digit 2.
GBI void slice5(df v, float s256, float s17, float *d) {
    float t = F_FMA(v.hi, s256, MAGIC);
    d[0] = F_SUB(t, MAGIC);
    float r = F_FMA(v.hi, s256, -d[0]);
    t = F_FMA(r, 512.0f, MAGIC);
    d[1] = F_SUB(t, MAGIC);
    r = F_FMA(r, 512.0f, -d[1]);
    const df s = two_sum(r, F_MUL(v.lo, s17));
    t = F_FMA(s.hi, 512.0f, MAGIC);
    d[2] = F_SUB(t, MAGIC);
    r = F_FMA(s.hi, 512.0f, -d[2]);
    r = F_FMA(s.lo, 512.0f, r);
    t = F_FMA(r, 512.0f, MAGIC);
    d[3] = F_SUB(t, MAGIC);
    r = F_FMA(r, 512.0f, -d[3]);
    t = F_FMA(r, 512.0f, MAGIC);
    d[4] = F_SUB(t, MAGIC);
}

GBI uint32_t pack_h2(float a, float b) {
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}

// Level values of one output -> chat in units of level 0 (double-float):
// D0 + 2^-9 D1 + 2^-18 D2 exactly (two TwoSums), plus the tail of levels
// 3-5, 2^-27 D3 + 2^-36 D4 + 2^-45 D5, formed in float (lowest level first).
GBI df recombine(float D0, float D1, float D2, float tail) {
    const df a = two_sum(D0, F_MUL(D1, 0x1p-9f));
    const df b = two_sum(a.hi, F_MUL(D2, 0x1p-18f));
    return fast_sum(b.hi, F_ADD(tail, F_ADD(a.lo, b.lo)));
}

// Pair geometry of every weak entry (depends on the tree only): ir = 2^e0 / r
// and Log(z_t - z_s) as double-float complex numbers, and the exponent
// offsets (a_s, a_t) = (e_s - e0 + 1, e_t - e0 + 1).
__global__ void k_m2l_pairs(int64_t n_weak, const double4 *__restrict__ geom,
                            const int *__restrict__ weak, const int *__restrict__ weak_tgt,
                            float4 *__restrict__ pir, float4 *__restrict__ plog,
                            int2 *__restrict__ pa) {
    pdl_wait();
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_weak) return;
    const double4 gs = geom[weak[e]], gt = geom[weak_tgt[e]];
    const int e_s = exp_of(gs.z), e_t = exp_of(gt.z);
    // D = z_t - z_s (FP64 difference: an exactly shared ordinate gives +0)
    const double dx = gt.x - gs.x, dy = gt.y - gs.y;
    const int e_d = max(exp_of(fabs(dx)), exp_of(fabs(dy)));
    // 2^e0 >= the larger sigma, and not below 2^-60 |D| (boxes of radius ~0
    // far apart: their powers underflow to 0, which is their true size), so
    // that |D / 2^e0|^2 < 2^124 stays in the float range
    const int e0 = max(max(e_s, e_t), e_d - 60);
    // Dm = D / 2^e_d as df32 (|Dm| in [1, 2^1.5)): the one FP64 split (the FP64
    // pipe is narrow); the other scaling of D follows in float, exactly
    const double scd = __hiloint2double((1023 - e_d) << 20, 0);  // 2^-e_d (|e_d| < 1000)
    const df Dmx = split_d(dx * scd), Dmy = split_d(dy * scd);
    // ir = 2^e0 / r with r = -D:  -conj(Ds) / |Ds|^2,  Ds = D / 2^e0 = Dm 2^(e_d - e0);
    // e_d - e0 <= 60 by the choice of e0, and >= -3 for a well-separated pair
    const float fsd = __int_as_float((min(max(e_d - e0, -126), 127) + 127) << 23);
    const df Dsx{F_MUL(Dmx.hi, fsd), F_MUL(Dmx.lo, fsd)};
    const df Dsy{F_MUL(Dmy.hi, fsd), F_MUL(Dmy.lo, fsd)};
    const df n2 = df_dot2(Dsx, Dsx, Dsy, Dsy);
    const float i0 = F_RCP(n2.hi);
    const df corr = df_add(df{1.0f, 0.f}, df_neg(df_mulf(n2, i0)));
    const df inv = df_add(df{i0, 0.f}, df_mulf(corr, i0));
    const df ir_re = df_neg(df_mul(Dsx, inv)), ir_im = df_mul(Dsy, inv);
    // Log(D): ln |D|^2 = ln |Dm|^2 + 2 e_d ln 2, the shift through the log's
    // exponent term
    const df S2 = df_dot2(Dmx, Dmx, Dmy, Dmy);
    const df ln = df_log_f(S2.hi, d_pairtab, log_ecst(2 * e_d));
    const df lr = fast_sum(F_MUL(0.5f, ln.hi), F_MUL(0.5f, F_FMA(S2.lo, F_RCP(S2.hi), ln.lo)));
    const df an = df_atan2_f(Dmy.hi, Dmx.hi, d_pairtab + ATAN_OFF);
    const float ci = F_MUL(F_FMA(Dmy.lo, Dmx.hi, -F_MUL(Dmx.lo, Dmy.hi)), F_RCP(S2.hi));
    const df li = fast_sum(an.hi, F_ADD(an.lo, ci));
    pir[e] = make_float4(ir_re.hi, ir_re.lo, ir_im.hi, ir_im.lo);
    plog[e] = make_float4(lr.hi, lr.lo, li.hi, li.lo);
    pa[e] = make_int2(e_s - e0 + 1, e_t - e0 + 1);
}

template <int PM>
__global__ void __launch_bounds__(R_THREADS, 1)
    k_m2l_tc(int n_weak, int p, int S, const float4 *__restrict__ pir,
             const float4 *__restrict__ plog, const int2 *__restrict__ pa,
             const int *__restrict__ weak, const int *__restrict__ weak_tgt,
             const float4 *__restrict__ mp, const uint4 *__restrict__ bops,
             const int *__restrict__ fexp, double2 *__restrict__ local, int *status) {
    pdl_wait();
    constexpr int NK = qcount(PM, 0) > qcount(PM, 3) ? qcount(PM, 0) : qcount(PM, 3);
    static_assert(NK <= 8 && qcount(PM, 1) <= NK && qcount(PM, 2) <= NK, "quarter layout");
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *sX = smem_raw;            // [slice][component] x 8 KB
    unsigned char *sB = smem_raw + X_BYTES;  // [scale][slice] x 2 KB
    float4 *smp = reinterpret_cast<float4 *>(smem_raw + X_BYTES + B_BYTES);  // [pair][MS]
    float2 *red = reinterpret_cast<float2 *>(smem_raw);  // [c][l][RED_STRIDE], after the MMAs
    __shared__ __align__(16) float4 s_ir[2][R_ROWS];
    __shared__ __align__(16) float4 s_log[2][R_ROWS];
    __shared__ __align__(8) int2 s_a[2][R_ROWS];
    __shared__ int s_tgt[2][R_ROWS];
    __shared__ int s_np[2];
    __shared__ float s_amax[4][R_ROWS];
    __shared__ __align__(16) float4 s_t0[R_ROWS];  // A_0 Log(z_t - z_s) per pair
    __shared__ uint32_t s_bnd[R_ROWS / 32];  // pairs that start a new target box
    __shared__ int s_f[R_NK];
    __shared__ __align__(8) uint64_t mbar[2];
    __shared__ uint32_t tmem_base;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int q = tid & (R_ROWS - 1), Q = tid >> 7;
    const int QG = Q == 0 ? 0 : Q == 1 ? qstart(PM, 1) : Q == 2 ? qstart(PM, 2) : qstart(PM, 3);
    const int MS = (p + 1) | 1;  // staged multipole stride (odd: no bank conflicts)
    // positions this thread holds: expansion indices QG .. QG + cnt - 1
    const int qc = Q == 0 ? qcount(PM, 0) : Q == 1 ? qcount(PM, 1) : Q == 2 ? qcount(PM, 2)
                                                                          : qcount(PM, 3);
    const int cnt = min(qc, p - QG + 1);

    // one-time set-up: zero digits (positions never written stay 0), operator
    for (int i = tid; i < X_BYTES / 16; i += R_THREADS)
        reinterpret_cast<uint4 *>(sX)[i] = make_uint4(0u, 0u, 0u, 0u);
    for (int i = tid; i < B_BYTES / 16; i += R_THREADS)
        reinterpret_cast<uint4 *>(sB)[i] =
            i < S * (B_SLICE / 16) ? bops[i] : make_uint4(0u, 0u, 0u, 0u);
    if (tid < R_NK) s_f[tid] = fexp[tid];
    if (tid == 0) {
        abort_flag = 0;
        // the issuing thread commits once to each component's barrier
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&tmem_base)),
                     "n"(R_TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tbase = tmem_base;
    const uint32_t tlane = (uint32_t)((warp & 3) * 32) << 16;

    const int n_items = (n_weak + R_ROWS - 1) / R_ROWS;  // item k: entries [128 k, 128 k + 128)
    // Stage item nx (multipoles of its source boxes, pair data, target boxes)
    // into shared memory; the copies complete at the next cp_async_wait.
    auto prefetch = [&](int nx, int b) {
        if (nx >= n_items) return;
        const int e0 = nx * R_ROWS;
        const int npn = min(R_ROWS, n_weak - e0);
        // warp w copies pairs w + 16 j (j < 8), lane k coefficient k (p < 32);
        // lane j first loads the source box of pair w + 16 j (all at once)
        constexpr int NW = R_THREADS / 32;
        const int mine = warp + NW * (lane & 7);
        const int box_l = mine < npn ? weak[e0 + mine] : 0;
#pragma unroll
        for (int j = 0; j < R_ROWS / NW; ++j) {
            const int pq = warp + NW * j;
            const int box = __shfl_sync(0xffffffffu, box_l, j);
            if (pq < npn && lane <= p)
                cp_async16(smp + pq * MS + lane, mp + (int64_t)box * (p + 1) + lane);
        }
        if (tid < npn) {
            cp_async16(&s_ir[b][tid], pir + e0 + tid);
            cp_async16(&s_log[b][tid], plog + e0 + tid);
            cp_async8(&s_a[b][tid], pa + e0 + tid);
            cp_async4(&s_tgt[b][tid], weak_tgt + e0 + tid);
        }
        if (tid == 0) s_np[b] = npn;
        cp_async_commit();
    };
    prefetch(blockIdx.x, 0);
    cp_async_wait();
    __syncthreads();

    int buf = 0;
    uint32_t phase = 0;
    for (int item = blockIdx.x; item < n_items; item += gridDim.x, buf ^= 1, phase ^= 1u) {
        const int n_pairs = s_np[buf];
        const bool active = q < n_pairs;
        const float4 ir4 = active ? s_ir[buf][q] : make_float4(0.f, 0.f, 0.f, 0.f);
        const int2 aa = active ? s_a[buf][q] : make_int2(0, 0);
        const cdf ir{df{ir4.x, ir4.y}, df{ir4.z, ir4.w}};
        const float4 *Ap = smp + q * MS;
        if (tid < R_ROWS) {  // warps 0-3: the segments of equal target box
            const bool start = active && (q == 0 || s_tgt[buf][q] != s_tgt[buf][q - 1]);
            const uint32_t bits = __ballot_sync(0xffffffffu, start);
            if (lane == 0) s_bnd[warp] = bits;
        }
        // ---------------- powers ir^(QG + kk) and the prescale
        cdf pw[NK], xk[NK];
        float amax = 0.f;
        {
            cdf P = cpow(ir, QG);
            float sk = pow2f_or0(QG * aa.x);
            const float fs = pow2f_or0(aa.x);
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) {
                pw[kk] = P;
                xk[kk] = cdf{df{0.f, 0.f}, df{0.f, 0.f}};
                if (kk < cnt) {  // uniform over the warp
                    const int k = QG + kk;
                    const float4 a4 = active ? Ap[k] : make_float4(0.f, 0.f, 0.f, 0.f);
                    const cdf a{df{a4.x, a4.y}, df{a4.z, a4.w}};
                    const cdf x = k == 0 ? a : cmul(a, P);  // xhat_0 = A_0
                    if (k == 0) {
                        // A_0 Log(z_t - z_s), added to B_0 in the postscale
                        const float4 lg = active ? s_log[buf][q] : make_float4(0.f, 0.f, 0.f, 0.f);
                        const cdf t0 = cmul(a, cdf{df{lg.x, lg.y}, df{lg.z, lg.w}});
                        s_t0[q] = make_float4(t0.re.hi, t0.re.lo, t0.im.hi, t0.im.lo);
                    }
                    const float sg = (k & 1) ? -sk : sk;
                    xk[kk] = cdf{df{F_MUL(x.re.hi, sg), F_MUL(x.re.lo, sg)},
                                 df{F_MUL(x.im.hi, sg), F_MUL(x.im.lo, sg)}};
                    amax = fmaxf(amax, fmaxf(fabsf(xk[kk].re.hi), fabsf(xk[kk].im.hi)));
                    sk = F_MUL(sk, fs);
                    if (kk + 1 < cnt) P = cmul_lz(P, ir);
                }
            }
        }
        s_amax[Q][q] = amax;
        __syncthreads();
        amax = fmaxf(fmaxf(s_amax[0][q], s_amax[1][q]), fmaxf(s_amax[2][q], s_amax[3][q]));
        int emax = amax > 0.f ? ((__float_as_int(amax) >> 23) & 0xff) - 126 : 0;  // 2^emax > amax
        emax = max(min(emax, 100), -100);
        // ---------------- digit slices of this thread's 8 positions and the
        // MMAs, one component at a time: the tensor cores run component 0 while
        // component 1 is sliced.  Component c: accumulator of level d at TMEM
        // columns 192 c + 32 d (d = 0 .. 5).  Slice A_j times the operator
        // slices B_0 .. B_{5-j} (consecutive in shared memory; B_i = 0 for
        // i >= S) is one MMA chain of N = 32 (6 - j) from column 32 j: levels
        // j .. 5 at once; the A_0 chain overwrites (it covers every level).
        {
            const float s256 = pow2f(8 - emax), s17 = pow2f(17 - emax);
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                uint32_t pk[R_S][4];
#pragma unroll
                for (int e2 = 0; e2 < 4; ++e2) {
                    float dg[2][R_S];
#pragma unroll
                    for (int e = 0; e < 2; ++e) {
                        const int kk = 2 * e2 + e;
                        if (kk < NK) {  // positions >= NK hold no index (digits 0)
                            const df v = c ? xk[kk < NK ? kk : 0].im : xk[kk < NK ? kk : 0].re;
                            slice5(v, s256, s17, dg[e]);
                        } else {
#pragma unroll
                            for (int j = 0; j < R_S; ++j) dg[e][j] = 0.f;
                        }
                    }
#pragma unroll
                    for (int j = 0; j < R_S; ++j) pk[j][e2] = pack_h2(dg[0][j], dg[1][j]);
                }
#pragma unroll
                for (int j = 0; j < R_S; ++j)
                    if (j < S)
                        *reinterpret_cast<uint4 *>(sX + (j * 2 + c) * X_SLICE + kmaj_off(q, 8 * Q)) =
                            make_uint4(pk[j][0], pk[j][1], pk[j][2], pk[j][3]);
                asm volatile("fence.proxy.async.shared::cta;");
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncthreads();
                asm volatile("tcgen05.fence::after_thread_sync;");
                if (tid == 0) {
                    const uint32_t db = umma_desc_lo(smem_u32(sB));
                    const uint32_t da = umma_desc_lo(smem_u32(sX) + c * X_SLICE);
                    const uint32_t td = tbase + R_CCOLS * c;
#pragma unroll 1
                    for (int j = 0; j < S; ++j)
                        mma_k32(td + R_NK * j, da + (uint32_t)((2 * j * X_SLICE) >> 4), db,
                                R_NK * (R_LEV - j), j > 0);
                    asm volatile(
                        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 "
                        "[%0];" ::"r"(smem_u32(&mbar[c])));
                }
            }
        }
        // the next item's data, copied while the tensor cores run (this item's
        // staged multipoles are consumed; its pair data sit in the other buffer)
        prefetch(item + gridDim.x, buf ^ 1);
        // ---------------- read back this thread's 8 positions, both components
        df ch[2][NK];
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            if (!mbar_wait(&mbar[c], phase, R_WAIT_LIMIT)) {
                atomicOr(status, ST_TIMEOUT);
                abort_flag = 1;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t ta = tbase + tlane + (uint32_t)(R_CCOLS * c + 8 * Q);
            float v[3][8], tl[NK];
            tmem_ld8(ta + 5 * R_NK, v[0]);  // the tail, levels 5, 4, 3
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) tl[kk] = F_MUL(v[0][kk], 0x1p-45f);
            tmem_ld8(ta + 4 * R_NK, v[0]);
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) tl[kk] = F_FMA(v[0][kk], 0x1p-36f, tl[kk]);
            tmem_ld8(ta + 3 * R_NK, v[0]);
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) tl[kk] = F_FMA(v[0][kk], 0x1p-27f, tl[kk]);
            tmem_ld8x3(ta, v);  // levels 0 .. 2
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) {
                if (kk >= cnt) continue;  // uniform over the warp
                ch[c][kk] = recombine(v[0][kk], v[1][kk], v[2][kk], tl[kk]);
            }
        }
        asm volatile("fence.proxy.async.shared::cta;");  // the digits area becomes `red`
        // ---------------- postscale: B_l += chat_l (2v)^l, (2v)^l = 2^{l a_t} ir^l
        {
            float vs = pow2f_or0(QG * aa.y);
            const float ft = pow2f_or0(aa.y);
            float2 *rr = red + q + (q >> 4);
#pragma unroll
            for (int kk = 0; kk < NK; ++kk) {
                if (kk < cnt) {
                    const int l = QG + kk;
                    const float sl = pow2f_or0(emax + s_f[l] - 16);
                    const cdf c{df{F_MUL(ch[0][kk].hi, sl), F_MUL(ch[0][kk].lo, sl)},
                                df{F_MUL(ch[1][kk].hi, sl), F_MUL(ch[1][kk].lo, sl)}};
                    cdf term;
                    if (l == 0) {
                        // + A_0 Log(z_t - z_s), formed in the prescale
                        const float4 t0 = s_t0[q];
                        term = cdf{df_add(c.re, df{t0.x, t0.y}), df_add(c.im, df{t0.z, t0.w})};
                    } else {
                        const cdf V{df{F_MUL(pw[kk].re.hi, vs), F_MUL(pw[kk].re.lo, vs)},
                                    df{F_MUL(pw[kk].im.hi, vs), F_MUL(pw[kk].im.lo, vs)}};
                        term = cmul_lz(c, V);
                    }
                    if (!active) term = cdf{df{0.f, 0.f}, df{0.f, 0.f}};
                    rr[(0 * R_NK + l) * RED_STRIDE] = make_float2(term.re.hi, term.re.lo);
                    rr[(1 * R_NK + l) * RED_STRIDE] = make_float2(term.im.hi, term.im.lo);
                    vs = F_MUL(vs, ft);
                }
            }
        }
        __syncthreads();
        if (abort_flag) break;
        // ---------------- sums over the item's pairs per target box: output
        // (component c, index l) by eight consecutive lanes
        {
            const int o = tid >> 3, part = tid & 7;
            const int c = o & 1, l = o >> 1;
            if (l <= p) {
                const float2 *row = red + (c * R_NK + l) * RED_STRIDE;
                const int g_first = s_tgt[buf][0], g_last = s_tgt[buf][n_pairs - 1];
                const int q0 = 16 * part, q1 = min(q0 + 16, n_pairs);
                if (g_first == g_last) {  // one target box (uniform over the CTA)
                    df sum{0.f, 0.f};
                    for (int j = q0; j < q1; ++j) {
                        const float2 v = row[j + (j >> 4)];
                        sum = df_acc(sum, df{v.x, v.y});
                    }
                    sum = fast_sum(sum.hi, sum.lo);
                    const unsigned gm = 0xffu << (lane & 24);
#pragma unroll
                    for (int m = 1; m < 8; m <<= 1)
                        sum = df_add(sum, df{__shfl_xor_sync(gm, sum.hi, m),
                                             __shfl_xor_sync(gm, sum.lo, m)});
                    if (part == 0) {
                        double *out = reinterpret_cast<double *>(local + (int64_t)g_first * (p + 1));
                        atomicAdd(out + 2 * l + c, (double)sum.hi + (double)sum.lo);
                    }
                } else if (q0 < q1) {
                    // a contiguous run of 16 pairs; add at every start of a box
                    const uint32_t bw = s_bnd[part >> 1] >> (16 * (part & 1));
                    df sum{0.f, 0.f};
                    int gcur = s_tgt[buf][q0];
#pragma unroll 4
                    for (int j = q0; j < q1; ++j) {
                        if (j > q0 && ((bw >> (j - q0)) & 1u)) {
                            double *out = reinterpret_cast<double *>(local + (int64_t)gcur * (p + 1));
                            atomicAdd(out + 2 * l + c, (double)sum.hi + (double)sum.lo);
                            gcur = s_tgt[buf][j];
                            sum = df{0.f, 0.f};
                        }
                        const float2 v = row[j + (j >> 4)];
                        sum = df_acc(sum, df{v.x, v.y});
                    }
                    double *out = reinterpret_cast<double *>(local + (int64_t)gcur * (p + 1));
                    atomicAdd(out + 2 * l + c, (double)sum.hi + (double)sum.lo);
                }
            }
        }
        // the next item overwrites the digits (`red`) and TMEM only after
        // everybody is done here, and reads the data prefetched above
        cp_async_wait();
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
    }
    cp_async_wait();
    if (abort_flag) {
        // a wait gave up: let the last item's MMAs drain (a longer bound)
        // before the tensor memory they write is released
        const bool d0 = mbar_wait(&mbar[0], phase, R_DRAIN_LIMIT);
        const bool d1 = mbar_wait(&mbar[1], phase, R_DRAIN_LIMIT);
        (void)d0;
        (void)d1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tbase), "n"(R_TCOLS));
}

}  // namespace

cudaError_t upload_df_tables_tc() {
    alignas(16) static float tab[DF_TAB_FLOATS];
    df32_fill_tables(tab);
    return cudaMemcpyToSymbol(d_pairtab, tab, sizeof(tab));
}

int m2l_tc_max_p() { return R_NK - 1; }
int m2l_tc_max_slices() { return R_S; }

// Digit slices of the scaled operator (row l, column k; Ahat_{l0} = -2^-l / l,
// Ahat_{lk} = C(k+l-1, l) 2^-(k+l)) with per-row exponents f_l (|row| < 2^f_l),
// in the canonical K-major layout at the GEMM positions of (l, k), followed
// by one zero slice.  Exact from long-double binomials (C(61, 30) < 2^64).
// The operator depends only on p: it is built once per (device, p) and kept
// for the life of the process (12 KB).
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
        const int pm = pm_of(p);
        std::vector<unsigned char> bytes((size_t)B_BYTES, 0);
        std::vector<int> fexp(R_NK, 0);
        for (int l = 0; l <= p; ++l) {
            long double row[R_NK] = {};
            long double mx = 0;
            for (int k = 0; k <= p; ++k) {
                long double v;
                if (k == 0) {
                    v = l == 0 ? 0.0L : -ldexpl(1.0L, -l) / (long double)l;
                } else {
                    long double c = 1;  // C(k+l-1, l)
                    for (int i = 1; i <= l; ++i) c = c * (long double)(k - 1 + i) / (long double)i;
                    c = roundl(c);
                    v = ldexpl(c, -(k + l));
                }
                row[k] = v;
                if (fabsl(v) > mx) mx = fabsl(v);
            }
            int f = 0;
            if (mx > 0) frexpl(mx, &f);  // mx = m 2^f, m in [0.5, 1)
            fexp[l] = f;
            const int n = gemm_pos(l, pm);
            for (int k = 0; k <= p; ++k) {
                long double x = ldexpl(row[k], -f);  // in (-1, 1)
                long double t0 = x * 256.0L;
                for (int j = 0; j < R_S; ++j) {
                    const long double dgt = roundl(t0);
                    x = t0 - dgt;
                    t0 = x * 512.0L;
                    const __half h = __float2half_rn((float)dgt);
                    std::memcpy(&bytes[(size_t)j * B_SLICE + kmaj_off(n, gemm_pos(k, pm))], &h, 2);
                }
            }
        }
        uint4 *bs = nullptr;
        int *fx = nullptr;
        if ((e = cudaMalloc(reinterpret_cast<void **>(&bs), bytes.size())) != cudaSuccess ||
            (e = cudaMalloc(reinterpret_cast<void **>(&fx), R_NK * sizeof(int))) != cudaSuccess ||
            (e = cudaMemcpy(bs, bytes.data(), bytes.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
            (e = cudaMemcpy(fx, fexp.data(), R_NK * sizeof(int), cudaMemcpyHostToDevice)) !=
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

fmm_status build_m2l_pairs(Tree &t, cudaStream_t s) {
    cudaError_t e;
    const int64_t nw = t.n_weak;
    if ((e = arena_alloc(t.mem, &t.m2l_pir, (size_t)nw + 1)) != cudaSuccess ||
        (e = arena_alloc(t.mem, &t.m2l_plog, (size_t)nw + 1)) != cudaSuccess ||
        (e = arena_alloc(t.mem, &t.m2l_pa, (size_t)nw + 1)) != cudaSuccess)
        return cuda_fail(e, "m2l pair table");
    if (nw == 0) return FMM_OK;
    launch_k(k_m2l_pairs, (unsigned)((nw + 255) / 256), 256, 0, s, nw, t.geom, t.weak, t.weak_tgt,
             t.m2l_pir, t.m2l_plog, t.m2l_pa);
    e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "m2l pair table");
}

fmm_status launch_m2l_tc(Tree &t, cudaStream_t s) {
    cudaError_t e;
    if (t.n_weak == 0) return FMM_OK;
    const int MS = (t.p + 1) | 1;
    const int smem = X_BYTES + B_BYTES + R_ROWS * MS * 16;
    const int pm = pm_of(t.p);
    auto k = pm == 16 ? k_m2l_tc<16> : pm == 24 ? k_m2l_tc<24> : k_m2l_tc<31>;
    const int ki = pm == 16 ? 0 : pm == 24 ? 1 : 2;
    static bool attr_set[64][3] = {};
    static int n_sm[64] = {};
    int dev = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return cuda_fail(e, "m2l tc device");
    if (dev >= 64) return set_error("device ordinal out of range"), FMM_ERR_ARG;
    if (!attr_set[dev][ki]) {
        const int most = X_BYTES + B_BYTES + R_ROWS * 33 * 16;  // p = 31
        if ((e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, most)) !=
            cudaSuccess)
            return cuda_fail(e, "m2l tc smem");
        attr_set[dev][ki] = true;
    }
    if (!n_sm[dev] &&
        (e = cudaDeviceGetAttribute(&n_sm[dev], cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess)
        return cuda_fail(e, "m2l tc SM count");
    const int64_t n_items = (t.n_weak + R_ROWS - 1) / R_ROWS;
    const int grid = (int)std::min<int64_t>(n_items, n_sm[dev]);  // one CTA per SM
    launch_k(k, grid, R_THREADS, smem, s, (int)t.n_weak, t.p, t.m2l_slices, t.m2l_pir, t.m2l_plog,
             t.m2l_pa, t.weak, t.weak_tgt, t.mpole_df, reinterpret_cast<const uint4 *>(t.m2l_bslices),
             t.m2l_fexp, t.local, t.status);
    e = cudaGetLastError();
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "m2l tc");
}

}  // namespace gbfmm
