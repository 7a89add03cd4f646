// Double-float ("df32") arithmetic and a double-float complex logarithm for
// the mixed-precision near field.  A df32 value is an unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2 (about 48 significant bits).
//
// Building blocks (error-free transformations):
//   two_sum   Knuth's TwoSum: s + e == a + b exactly, no ordering needed.
//   fast_sum  Dekker's Fast2Sum: exact when |a| >= |b| (or a == 0).
//   two_prod  FMA-based product: p + e == a * b exactly.
// All are written with explicitly rounded intrinsics so the compiler cannot
// contract or reassociate them.
//
// Logarithm: table-driven method of P. T. P. Tang ("Table-driven
// implementation of the logarithm function in IEEE floating-point
// arithmetic", ACM TOMS 16(4), 1990): s = 2^E m, m in [1, 2); with the table
// point c_k = 1 + (k + 1/2)/64 nearest to m, ln s = E ln 2 + ln c_k + ln(1 + f),
// f = (m - c_k)/c_k, |f| < 2^-7, and ln(1 + f) by its Taylor series to f^6.
//
// Arctangent: octant reduction to t = v/u in [0, 1], a table point c_k = k/64
// near t, and atan(t) = atan(c_k) + atan(d), d = (t - c_k)/(1 + t c_k),
// |d| < 1.004 * 2^-7, by its Taylor series to d^5 (the classical argument reduction, e.g. J.-M. Muller,
// "Elementary Functions", ch. 6).  Undoing the octant reduction adds a
// quadrant offset and signs to atan(t); the table holds, for each of the eight
// (swap, x < 0, sign of y) cases, the signed offset + sign * atan(c_k), so one
// double-float addition of the signed atan(d) finishes the argument.
//
// Tables are filled on the host from long-double libm values (df32_tables()).
// Accuracy target: absolute error below 2^-42 for ln|z| and arg z when z is
// given as a df32 pair with |lo| < 2^-20 |hi|.
#pragma once
#include <math.h>
#include <stdint.h>

#if defined(__CUDACC__)
#define DF_HD __host__ __device__ __forceinline__
#else
#define DF_HD inline
#endif

#if defined(__CUDA_ARCH__)
#define F_ADD(a, b) __fadd_rn((a), (b))
#define F_SUB(a, b) __fsub_rn((a), (b))
#define F_MUL(a, b) __fmul_rn((a), (b))
#define F_FMA(a, b, c) __fmaf_rn((a), (b), (c))
#define F_RCP(a) df_rcp_approx(a)
// MUFU reciprocal (about 1 ulp); every use below corrects it with a residual
__device__ __forceinline__ float df_rcp_approx(float a) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(a));
    return r;
}
#else
#include <cmath>
#include <cstring>

using std::signbit;
static inline float df_host_add(float a, float b) {
    volatile float r = a + b;
    return r;
}
static inline float df_host_sub(float a, float b) {
    volatile float r = a - b;
    return r;
}
static inline float df_host_mul(float a, float b) {
    volatile float r = a * b;
    return r;
}
#define F_ADD(a, b) df_host_add((a), (b))
#define F_SUB(a, b) df_host_sub((a), (b))
#define F_MUL(a, b) df_host_mul((a), (b))
#define F_FMA(a, b, c) std::fmaf((a), (b), (c))
#define F_RCP(a) (1.0f / (a))
#endif

namespace gbfmm {

struct df {
    float hi, lo;
};

DF_HD df two_sum(float a, float b) {
    float s = F_ADD(a, b);
    float bb = F_SUB(s, a);
    float e = F_ADD(F_SUB(a, F_SUB(s, bb)), F_SUB(b, bb));
    return df{s, e};
}

DF_HD df fast_sum(float a, float b) {
    float s = F_ADD(a, b);
    float e = F_SUB(b, F_SUB(s, a));
    return df{s, e};
}

DF_HD df two_prod(float a, float b) {
    float p = F_MUL(a, b);
    float e = F_FMA(a, b, -p);
    return df{p, e};
}

// df + df (normalised result)
DF_HD df df_add(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    float lo = F_ADD(s.lo, F_ADD(a.lo, b.lo));
    return fast_sum(s.hi, lo);
}

DF_HD df df_neg(df a) { return df{-a.hi, -a.lo}; }

// df * df
DF_HD df df_mul(df a, df b) {
    df p = two_prod(a.hi, b.hi);
    float lo = F_FMA(a.hi, b.lo, F_FMA(a.lo, b.hi, p.lo));
    return fast_sum(p.hi, lo);
}

// df * float
DF_HD df df_mulf(df a, float b) {
    df p = two_prod(a.hi, b);
    float lo = F_FMA(a.lo, b, p.lo);
    return fast_sum(p.hi, lo);
}

// a * b + c * d in one pass: the two exact high products are added with
// TwoSum and every low-order term (product errors, cross terms, the sum's
// error) is gathered into one float before the final Fast2Sum.  The error
// is the same order as df_add(df_mul(a, b), df_mul(c, d)), with 19
// operations instead of 25.
DF_HD df df_dot2(df a, df b, df c, df d) {
    df p = two_prod(a.hi, b.hi), r = two_prod(c.hi, d.hi);
    df s = two_sum(p.hi, r.hi);
    float t = F_FMA(a.hi, b.lo, p.lo);
    t = F_FMA(a.lo, b.hi, t);
    t = F_FMA(c.hi, d.lo, t);
    t = F_FMA(c.lo, d.hi, t);
    t = F_ADD(t, r.lo);
    return fast_sum(s.hi, F_ADD(s.lo, t));
}

// a * b + c * d + e in one pass (a Horner step of a complex product plus a
// coefficient): one more TwoSum for e, 26 operations instead of 30.
DF_HD df df_dot2_add(df a, df b, df c, df d, df e) {
    df p = two_prod(a.hi, b.hi), r = two_prod(c.hi, d.hi);
    df s = two_sum(p.hi, r.hi);
    df u = two_sum(s.hi, e.hi);
    float t = F_FMA(a.hi, b.lo, p.lo);
    t = F_FMA(a.lo, b.hi, t);
    t = F_FMA(c.hi, d.lo, t);
    t = F_FMA(c.lo, d.hi, t);
    t = F_ADD(t, F_ADD(r.lo, e.lo));
    return fast_sum(u.hi, F_ADD(F_ADD(s.lo, u.lo), t));
}

// df_dot2 and df_dot2_add without the closing Fast2Sum: hi + lo is the same
// value, the low part is not renormalised.  For chains (powers, Horner steps)
// whose results feed further products or error-free sums: a product takes
// the low part through an FMA, so the error stays relative to the magnitudes
// of the products, as with renormalised operands.
DF_HD df df_dot2_lz(df a, df b, df c, df d) {
    df p = two_prod(a.hi, b.hi), r = two_prod(c.hi, d.hi);
    df s = two_sum(p.hi, r.hi);
    float t = F_FMA(a.hi, b.lo, p.lo);
    t = F_FMA(a.lo, b.hi, t);
    t = F_FMA(c.hi, d.lo, t);
    t = F_FMA(c.lo, d.hi, t);
    t = F_ADD(t, r.lo);
    return df{s.hi, F_ADD(s.lo, t)};
}
DF_HD df df_dot2_add_lz(df a, df b, df c, df d, df e) {
    df p = two_prod(a.hi, b.hi), r = two_prod(c.hi, d.hi);
    df s = two_sum(p.hi, r.hi);
    df u = two_sum(s.hi, e.hi);
    float t = F_FMA(a.hi, b.lo, p.lo);
    t = F_FMA(a.lo, b.hi, t);
    t = F_FMA(c.hi, d.lo, t);
    t = F_FMA(c.lo, d.hi, t);
    t = F_ADD(t, F_ADD(r.lo, e.lo));
    return df{u.hi, F_ADD(F_ADD(s.lo, u.lo), t)};
}

// 1/n for a positive df32 n (hi + lo, |lo| <= 2^-24 |hi|) as an unnormalised
// df32 pair: the reciprocal approximation i0 of hi and one Newton step,
// 1/n = i0 (1 + e + O(e^2)), e = 1 - n i0 = (1 - hi i0) - lo i0 formed by two
// FMAs (|e| <= ~2^-22; the first residual is exact for a reciprocal within
// an ulp, so e carries one rounding).
DF_HD df df_recip(df n) {
    const float i0 = F_RCP(n.hi);
    const float e = F_FMA(-n.lo, i0, F_FMA(-n.hi, i0, 1.0f));
    return df{i0, F_MUL(i0, e)};
}

// One Horner step h = h w + b on df32 complex numbers given as (re, im)
// pairs, the low parts left unnormalised.
DF_HD void df_horner_step(df &hr, df &hi, df wr, df wi, df br, df bi) {
    const df nr = df_dot2_add_lz(hr, wr, df_neg(hi), wi, br);
    const df ni = df_dot2_add_lz(hr, wi, hi, wr, bi);
    hr = nr;
    hi = ni;
}

// Table layout (floats, 16-byte aligned), filled by df32_fill_tables():
//   log: 64 entries of {r_hi, r_lo, L_hi, L_lo}, r = 1/c_k, L = ln c_k (one
//        16-byte load; c_k itself is formed from the mantissa bits)
//   atan: 8 cases x 65 entries of {T_hi, T_lo}, T = s (offset_c + sign_c atan(k/64))
//         with (offset, sign) = (0, +1), (pi/2, -1), (pi, -1), (pi/2, +1) for
//         c = swap + 2 (x < 0), and s = -1 for the cases 4..7 (y negative)
constexpr int LOG_TAB = 64;
constexpr int ATAN_TAB = 65;
constexpr int ATAN_OFF = 4 * LOG_TAB;  // first float of the arctangent tables
constexpr int DF_TAB_FLOATS = ATAN_OFF + 8 * 2 * ATAN_TAB;

// hi = ln 2, pi, pi/2 rounded to float; lo = the float nearest the remainder
constexpr float LN2_HI = 0x1.62e430p-1f;
constexpr float LN2_LO = -0x1.05c610p-29f;
constexpr float PI_HI = 0x1.921fb6p+1f;
constexpr float PI_LO = -0x1.777a5cp-24f;
constexpr float PI2_HI = 0x1.921fb6p+0f;
constexpr float PI2_LO = -0x1.777a5cp-25f;

// Fill the lookup tables (host side, long-double libm).
inline void df32_fill_tables(float *tab) {
    for (int k = 0; k < LOG_TAB; ++k) {
        long double c = 1.0L + (k + 0.5L) / 64.0L;
        long double r = 1.0L / c, L = logl(c);
        float rh = (float)r, Lh = (float)L;
        float *t = tab + 4 * k;
        t[0] = rh;
        t[1] = (float)(r - (long double)rh);
        t[2] = Lh;
        t[3] = (float)(L - (long double)Lh);
    }
    float *a = tab + ATAN_OFF;
    const long double pi = 3.141592653589793238462643383279502884L;
    const long double off[4] = {0.0L, pi / 2, pi, pi / 2};
    const long double sgn[4] = {1.0L, -1.0L, -1.0L, 1.0L};
    for (int c = 0; c < 8; ++c)
        for (int k = 0; k < ATAN_TAB; ++k) {
            const long double sy = (c & 4) ? -1.0L : 1.0L;
            long double T = sy * (off[c & 3] + sgn[c & 3] * atanl((long double)k / 64.0L));
            float Th = (float)T;
            a[2 * (c * ATAN_TAB + k)] = Th;
            a[2 * (c * ATAN_TAB + k) + 1] = (float)(T - (long double)Th);
        }
}

// Exponent constant of df_log_f: with ecst = 2^23 + 127 - b the result is
// ln(s 2^b) (b an integer, |b| < 2^22): the exponent term of the reduction
// takes the shift at no cost.  Kernels that form their differences in units
// of 2^e (offsets scaled by an exact power of two) pass b = 2e for ln |D|^2.
constexpr float LOG_ECST0 = 8388608.0f + 127.0f;
DF_HD float log_ecst(int b) { return LOG_ECST0 - (float)b; }

// ln(s 2^b) for a float s > 0 (normal), as a df32 pair (hi, lo) whose low part
// is not renormalised (callers add it into their own Fast2Sum); ecst = log_ecst(b).
DF_HD df df_log_f(float s, const float *tab, float ecst = LOG_ECST0) {
#if defined(__CUDA_ARCH__)
    int bits = __float_as_int(s);
#else
    int bits;
    std::memcpy(&bits, &s, 4);
#endif
    int k = (bits >> 17) & 63;
    int mb = (bits & 0x007fffff) | 0x3f800000;
#if defined(__CUDA_ARCH__)
    float m = __int_as_float(mb);
#else
    float m;
    std::memcpy(&m, &mb, 4);
#endif
    // c_k = 1 + (k + 1/2)/64: the top six mantissa bits of m, then a one
#if defined(__CUDA_ARCH__)
    const float c = __int_as_float(0x3f800000 | (bits & 0x007e0000) | 0x00010000);
    const float4 t4 = *reinterpret_cast<const float4 *>(tab + 4 * k);
    const float rh = t4.x, rl = t4.y, Lh = t4.z, Ll = t4.w;
#else
    int cb = 0x3f800000 | (bits & 0x007e0000) | 0x00010000;
    float c;
    std::memcpy(&c, &cb, 4);
    const float *t = tab + 4 * k;
    const float rh = t[0], rl = t[1], Lh = t[2], Ll = t[3];
#endif
    // E as a float without an int->float conversion: 2^23 + e - 2^23
#if defined(__CUDA_ARCH__)
    float Ef = F_SUB(__int_as_float(0x4B000000 | ((bits >> 23) & 0xff)), ecst);
#else
    float Ef = (float)(((bits >> 23) & 0xff) - 127) + (LOG_ECST0 - ecst);
#endif
    float u = F_SUB(m, c);  // exact (Sterbenz)
    // f = u / c as df32
    float fh = F_MUL(u, rh);
    float fl = F_FMA(u, rl, F_FMA(u, rh, -fh));
    // ln(1+f) = f - f^2/2 + f^3 (1/3 - f/4 + f^2/5 - f^3/6)
    df q = two_prod(fh, fh);
    float tail = F_MUL(F_MUL(q.hi, fh),
                       F_FMA(fh, F_FMA(fh, F_FMA(fh, -1.0f / 6.0f, 0.2f), -0.25f), 1.0f / 3.0f));
    // |f^2 / 2| < |f| (|f| < 2^-6): Fast2Sum is exact
    df a = fast_sum(fh, F_MUL(-0.5f, q.hi));
    float plo = F_ADD(a.lo, F_FMA(-0.5f, q.lo, F_FMA(-fh, fl, F_ADD(fl, tail))));
    // E ln 2 (exact product + correction) + ln c_k
    df e2 = two_prod(Ef, LN2_HI);
    float elo = F_FMA(Ef, LN2_LO, e2.lo);
    // |E ln 2| >= 0.693 > ln c_k for E != 0 (and E = 0 gives 0): Fast2Sum is exact
    // (E here includes the shift b)
    df b = fast_sum(e2.hi, Lh);
    df r = two_sum(b.hi, a.hi);
    float lo = F_ADD(F_ADD(r.lo, b.lo), F_ADD(F_ADD(elo, Ll), plo));
    return df{r.hi, lo};  // not renormalised: every caller folds lo into its own Fast2Sum
}

#if defined(__CUDACC__)
// Units of a leaf pair in the double-float kernels.  Point offsets are kept
// in units of their own leaf's sigma = 2^e (geometry radii are powers of two,
// so the scaling is exact); a pair of leaves (t, s) works in units of 2^ep,
// ep = max(e_t, e_s): offsets are rescaled by ft = 2^(e_t - ep) and
// fs = 2^(e_s - ep) (exact; 0 below the float range, where a leaf has radius
// ~0 and all its offsets are 0), and centre differences by inv = 2^-ep in
// FP64, so every float quantity of the pair is O(1) whatever the absolute
// scale of the coordinates.  In absolute units ln |D|^2 is
// df_log_f(|D'|^2, tab, ecst) and a harmonic term 1/D is inv / D'.
struct PairUnits {
    float ft, fs, ecst;
    int ep;
};
__device__ __forceinline__ int pow2_exponent(double sigma) {
    return ((__double2hiint(sigma) >> 20) & 0x7ff) - 1023;
}
__device__ __forceinline__ float pow2f_le0(int e) {  // 2^e (e <= 0); 0 below the float range
    return e < -126 ? 0.0f : __int_as_float((e + 127) << 23);
}
__device__ __forceinline__ double pow2d(int e) {  // 2^e, |e| <= 1022
    return __hiloint2double((1023 + e) << 20, 0);
}
__device__ __forceinline__ PairUnits pair_units(double sig_t, double sig_s) {
    const int et = pow2_exponent(sig_t), es = pow2_exponent(sig_s);
    const int ep = et > es ? et : es;
    return PairUnits{pow2f_le0(et - ep), pow2f_le0(es - ep), log_ecst(2 * ep), ep};
}
#endif

// atan2(y, x) for floats (not both zero), principal value in (-pi, pi], as a
// df32 pair whose low part is not renormalised (as df_log_f).
DF_HD df df_atan2_f(float y, float x, const float *atab) {
    float ax = fabsf(x), ay = fabsf(y);
    bool swap = ay > ax;
    float u = swap ? ay : ax, v = swap ? ax : ay;  // 0 <= v <= u
    // c_k = k/64 with k = round(63.75 v/u): the scale just under 64 keeps
    // v/(c_k u) >= 1/2 for k >= 1 even when v/u is rounded, so v - c_k u below
    // is exact (Sterbenz), while |d| stays below 1.004 * 2^-7.
    float t0 = F_MUL(v, F_RCP(u));
    float kf = F_FMA(t0, 63.75f, 12582912.0f);  // 1.5 * 2^23 rounding trick
#if defined(__CUDA_ARCH__)
    int k = __float_as_int(kf) - 0x4B400000;
#else
    int k;
    std::memcpy(&k, &kf, 4);
    k -= 0x4B400000;
#endif
    // in range for any input; a NaN (z == 0, never used) must not index out
    k = (unsigned)k > 64u ? 64 : k;
    float ck = F_MUL(F_SUB(kf, 12582912.0f), 1.0f / 64.0f);
    // d = (t - c_k) / (1 + t c_k) = (v - c_k u) / (u + c_k v), one division
    df cu = two_prod(ck, u);
    float nh = F_SUB(v, cu.hi);  // exact
    df cv = two_prod(ck, v);
    df den = fast_sum(u, cv.hi);  // u >= c_k v
    float denlo = F_ADD(den.lo, cv.lo);
    float rd = F_RCP(den.hi);
    float d0 = F_MUL(nh, rd);
    float rem = F_FMA(-d0, den.hi, nh);
    rem = F_ADD(rem, F_FMA(-d0, denlo, -cu.lo));
    float d1 = F_MUL(rem, rd);
    // normalised: the cubic term below is formed from d.hi alone
    df d = fast_sum(d0, d1);
    // atan(d) = d - d^3/3 + d^5/5
    float d2 = F_MUL(d.hi, d.hi);
    float corr = F_MUL(F_MUL(d2, d.hi), F_FMA(d2, 0.2f, -1.0f / 3.0f));
    // undo the reduction: T_c(k) + s sign_c atan(d), c = swap + 2 (x < 0) +
    // 4 (sign bit of y); the overall sign of atan(d) is that of swap ^ (x < 0) ^ y
#if defined(__CUDA_ARCH__)
    const uint32_t ny = (uint32_t)__float_as_int(y) >> 31;
#else
    uint32_t ny;
    std::memcpy(&ny, &y, 4);
    ny >>= 31;
#endif
    const uint32_t sw = swap ? 1u : 0u, nx = x < 0.0f ? 1u : 0u;
    const int c = (int)(sw | (nx << 1) | (ny << 2));
    const uint32_t sgb = (sw ^ nx ^ ny) << 31;
#if defined(__CUDA_ARCH__)
    const float sg = __int_as_float((int)(0x3f800000u | sgb));
#else
    const uint32_t sgi = 0x3f800000u | sgb;
    float sg;
    std::memcpy(&sg, &sgi, 4);
#endif
    const float *T = atab + 2 * (c * ATAN_TAB + k);
    df s = two_sum(T[0], F_MUL(sg, d.hi));
    float lo = F_ADD(s.lo, F_ADD(T[1], F_MUL(sg, F_ADD(d.lo, corr))));
    return df{s.hi, lo};  // not renormalised: every caller folds lo into its own Fast2Sum
}

}  // namespace gbfmm
