// Shared device helpers of the GB300 FMM library (internal).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#define GBI __device__ __forceinline__

// Programmatic dependent launch: every kernel of the library is launched with
// programmatic stream serialisation (launch_k, internal.h) and begins with
// pdl_wait(), which returns once the kernels before it in the stream have
// completed and their writes are visible.  The launch of a kernel then
// overlaps the end of the one before it instead of following its completion.
GBI void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

namespace gbfmm {

// Device status bits (latched with atomicOr into the tree's status word).
enum : int {
    ST_NONFINITE = 1,
    ST_LIST_OVERFLOW = 2,
    ST_TIMEOUT = 4,
    ST_BAD_INDEX = 8,
};

constexpr int MAXP = 64;

// ---------------------------------------------------------------- geometry
// Order-preserving 64-bit key of a double (after -0.0 -> +0.0), integer
// operations only (the FP64 pipe is narrow on this part).
GBI uint64_t order_key(double x) {
    uint64_t b = (uint64_t)__double_as_longlong(x);
    b = (b == 0x8000000000000000ull) ? 0ull : b;
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
GBI double key_to_double(uint64_t k) {
    uint64_t b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

struct Rect {
    double x0, x1, y0, y1;
};

// Centre = rectangle centre, radius = half the diagonal; explicit rounding
// (no contraction) so that host and device agree bit for bit.
GBI void centre_radius(const Rect &r, double &cx, double &cy, double &rad) {
    cx = __dmul_rn(0.5, __dadd_rn(r.x0, r.x1));
    cy = __dmul_rn(0.5, __dadd_rn(r.y0, r.y1));
    double w = __dsub_rn(r.x1, r.x0), h = __dsub_rn(r.y1, r.y0);
    rad = __dmul_rn(0.5, __dsqrt_rn(__dadd_rn(__dmul_rn(w, w), __dmul_rn(h, h))));
}

// Theta-criterion (Eq. 3): R + theta r <= theta d, with d > 0.
GBI bool well_separated(const Rect &b, const Rect &c, double theta) {
    double bx, by, rb, cx, cy, rc;
    centre_radius(b, bx, by, rb);
    centre_radius(c, cx, cy, rc);
    double dx = __dsub_rn(bx, cx), dy = __dsub_rn(by, cy);
    double d = __dsqrt_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    double R = rb > rc ? rb : rc, r = rb > rc ? rc : rb;
    return d > 0.0 && __dadd_rn(R, __dmul_rn(theta, r)) <= __dmul_rn(theta, d);
}

// ---------------------------------------------------------------- complex FP64
struct cd {
    double re, im;
};
GBI cd cmk(double a, double b) { return cd{a, b}; }
GBI cd cadd(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
GBI cd csub(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
GBI cd cmul(cd a, cd b) { return cd{fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)}; }
GBI cd cscale(cd a, double s) { return cd{a.re * s, a.im * s}; }
GBI cd cinv(cd a) {
    double s = 1.0 / fma(a.re, a.re, a.im * a.im);
    return cd{a.re * s, -a.im * s};
}
GBI cd clog_principal(cd a) {
    return cd{0.5 * log(fma(a.re, a.re, a.im * a.im)), atan2(a.im, a.re)};
}

// Power-of-two box scale sigma >= radius (sigma = 2^e); exact to apply.
GBI int scale_exponent(double rad) {
    if (!(rad >= 0x1p-1000)) return -1000;
    int e;
    frexp(rad, &e);
    return e;
}

// Block-wide exclusive scan (blockDim.x == NT); returns the block total.
template <int NT>
__device__ __forceinline__ uint32_t block_scan_excl(uint32_t v, uint32_t &excl,
                                                    uint32_t *warp_tot) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_tot[warp] = x;
    __syncthreads();
    uint32_t wp = 0, tot = 0;
#pragma unroll
    for (int w = 0; w < NT / 32; ++w) {
        const uint32_t t = warp_tot[w];
        wp += (w < warp) ? t : 0u;
        tot += t;
    }
    excl = wp + x - v;
    __syncthreads();
    return tot;
}

// ---------------------------------------------------------------- warp helpers
GBI double shfl_xor_d(double v, int m) { return __shfl_xor_sync(0xffffffffu, v, m); }

}  // namespace gbfmm
