// Host build of the double-float primitives of the mixed path (df32.cuh),
// measured against long double on seeded random inputs.  Prints one JSON
// object of maximum errors; tests/test_df32_host.py holds the bounds.
//
//   log      ln s, s in [2^-8, 2^8]: absolute error; over [2^-100, 2^100] and
//            with the exponent shift of pair units: error / max(1, |ln|)
//   atan2    angles over (-pi, pi], radii over [2^-20, 2^20]: absolute error
//   recip    1/n for df32 n over [2^-30, 2^30]: relative error
//   horner   sum_k b_k w^k (p = 24, |w| <= 1, complex df32 b_k) by
//            df_horner_step: error / sum_k |b_k| |w|^k
//   dot2     a b + c d by df_dot2 and df_dot2_lz: error / (|a b| + |c d|)
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>

#include "df32.cuh"

using namespace gbfmm;

static uint64_t state = 0x2545F4914F6CDD1Dull;
static double urand() {  // 53-bit uniform in [0, 1) from a 64-bit LCG
    state = state * 6364136223846793005ull + 1442695040888963407ull;
    return (double)(state >> 11) * 0x1p-53;
}
static df split(long double v) {
    const float hi = (float)v;
    return df{hi, (float)(v - (long double)hi)};
}
static long double val(df a) { return (long double)a.hi + (long double)a.lo; }

int main(int argc, char **argv) {
    static float tab[DF_TAB_FLOATS];
    df32_fill_tables(tab);
    const int n = argc > 1 ? std::atoi(argv[1]) : 200000;
    const long double LN2 = 0.693147180559945309417232121458176568L;
    long double log_small = 0, log_rel = 0, log_shift = 0, atan_abs = 0, recip_rel = 0;
    long double horner_rel = 0, dot_rel = 0, dot_lz_rel = 0;
    for (int i = 0; i < n; ++i) {
        const float s = (float)std::exp2(-8.0 + 16.0 * urand());
        log_small = fmaxl(log_small, fabsl(val(df_log_f(s, tab)) - logl((long double)s)));
        const float s2 = (float)std::exp2(-100.0 + 200.0 * urand());
        const long double r2 = logl((long double)s2);
        log_rel = fmaxl(log_rel, fabsl(val(df_log_f(s2, tab)) - r2) / fmaxl(1.0L, fabsl(r2)));
        const int b = 2 * (int)(urand() * 200.0) - 200;
        const long double r3 = logl((long double)s) + b * LN2;
        log_shift =
            fmaxl(log_shift, fabsl(val(df_log_f(s, tab, log_ecst(b))) - r3) / fmaxl(1.0L, fabsl(r3)));

        const double ang = 2.0 * M_PI * urand() - M_PI, rad = std::exp2(-20.0 + 40.0 * urand());
        const float x = (float)(rad * std::cos(ang)), y = (float)(rad * std::sin(ang));
        if (x != 0.0f || y != 0.0f)
            atan_abs = fmaxl(atan_abs, fabsl(val(df_atan2_f(y, x, tab + ATAN_OFF)) -
                                             atan2l((long double)y, (long double)x)));

        const df nd = split(std::exp2(-30.0 + 60.0 * urand()));
        recip_rel = fmaxl(recip_rel, fabsl(val(df_recip(nd)) * val(nd) - 1.0L));

        if (i % 16 == 0) {
            const int p = 24;
            const long double wm = urand(), wa = 2.0 * M_PI * urand();
            const df wr = split(wm * cosl(wa)), wi = split(wm * sinl(wa));
            df hr{0.f, 0.f}, hi{0.f, 0.f};
            long double er = 0, ei = 0, scale = 0, wpow = 1;
            const long double Wr = val(wr), Wi = val(wi);
            df br[25], bi[25];
            for (int k = 0; k <= p; ++k) {
                br[k] = split(2.0 * urand() - 1.0);
                bi[k] = split(2.0 * urand() - 1.0);
            }
            for (int k = p; k >= 0; --k) {
                df_horner_step(hr, hi, wr, wi, br[k], bi[k]);
                const long double tr = er * Wr - ei * Wi + val(br[k]);
                ei = er * Wi + ei * Wr + val(bi[k]);
                er = tr;
            }
            for (int k = 0; k <= p; ++k) {
                scale += hypotl(val(br[k]), val(bi[k])) * wpow;
                wpow *= hypotl(Wr, Wi);
            }
            horner_rel = fmaxl(horner_rel, hypotl(val(hr) - er, val(hi) - ei) / scale);
        }

        const df a = split(2.0 * urand() - 1.0), bb = split(2.0 * urand() - 1.0);
        const df c = split(2.0 * urand() - 1.0), d = split(2.0 * urand() - 1.0);
        const long double ex = val(a) * val(bb) + val(c) * val(d);
        const long double sc = fabsl(val(a) * val(bb)) + fabsl(val(c) * val(d));
        dot_rel = fmaxl(dot_rel, fabsl(val(df_dot2(a, bb, c, d)) - ex) / sc);
        dot_lz_rel = fmaxl(dot_lz_rel, fabsl(val(df_dot2_lz(a, bb, c, d)) - ex) / sc);
    }
    std::printf(
        "{\"log_small_abs\": %.6Le, \"log_rel\": %.6Le, \"log_shift_rel\": %.6Le, "
        "\"atan_abs\": %.6Le, \"recip_rel\": %.6Le, \"horner_rel\": %.6Le, \"dot2_rel\": %.6Le, "
        "\"dot2_lz_rel\": %.6Le}\n",
        log_small, log_rel, log_shift, atan_abs, recip_rel, horner_rel, dot_rel, dot_lz_rel);
    return 0;
}
