// Mixed-precision M2L: the paper's scaled M2L shift (Alg. "Multipole to local
// translation": prescaling by r^-k, two summation sweeps, postscaling) run
// in double-float arithmetic on the FP32 pipes, two lanes per shift (real and
// imaginary part are independent during the sweeps, Sec. 3.3).
//
// In the radius-normalised variables of expand.cu (r = z_s - z_t,
// u = sigma_s / r, v = sigma_t / r):
//   prescale   b_{k-1} = (-1)^k A_k u^k            k = 1..p,  b_p = 0
//   sweep 1    for k = 2..p:  for j = p-k..p-1:  b_j += b_{j+1}
//   sweep 2    for k = p..1:  for j = k..p:      b_j += b_{j-1}
//   postscale  B_0 += b_0 + A_0 Log(z_t - z_s),  B_l += (b_l - A_0 / l) v^l
// (the printed listing's first sweep subtracts and its log term is
// -a_0 log r; this is the reading that reproduces the exact expansion).
//
// Work items are (target box, run of <= 64 weak pairs); one warp per item,
// 16 shifts in flight, a shuffle reduction per coefficient at the end and one
// FP64 atomic add per coefficient into the target's local expansion.
// Register arrays are right-aligned in a compile-time width PM >= p so that
// every index is static: entry j of the listing lives in slot j + (PM - p).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "df32.cuh"
#include "internal.h"

namespace gbfmm {

namespace {

// This translation unit's copy of the df32 tables (device symbols are not
// shared across translation units without relocatable device code).
__device__ float d_dftab[DF_TAB_FLOATS];

constexpr int M2L_CHUNK = 64;

GBI df split_d(double v) {
    float hi = __double2float_rn(v);
    float lo = __double2float_rn(v - (double)hi);
    return df{hi, lo};
}

struct dc {
    df re, im;
};

GBI dc dc_mul(const dc &a, const dc &b) {
    return dc{df_dot2(a.re, b.re, df_neg(a.im), b.im), df_dot2(a.re, b.im, a.im, b.re)};
}

// lazily normalised df32 accumulation
GBI df df_acc(df a, df b) {
    df s = two_sum(a.hi, b.hi);
    return df{s.hi, F_ADD(s.lo, F_ADD(a.lo, b.lo))};
}

GBI df shfl_df(df v, int m, unsigned mask = 0xffffffffu) {
    return df{__shfl_xor_sync(mask, v.hi, m), __shfl_xor_sync(mask, v.lo, m)};
}

// a / b for a df32 a and a float b (one correction step)
GBI df df_divf(df a, float b) {
    float q1 = F_MUL(a.hi, F_RCP(b));
    float r = F_ADD(F_FMA(-q1, b, a.hi), a.lo);
    float q2 = F_MUL(r, F_RCP(b));
    return fast_sum(q1, q2);
}

// multipoles FP64 -> df32 (re_hi, re_lo, im_hi, im_lo)
__global__ void k_mpole_df(int64_t n, const double2 *__restrict__ in, float4 *__restrict__ out) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double2 v = in[i];
    df r = split_d(v.x), m = split_d(v.y);
    out[i] = make_float4(r.hi, r.lo, m.hi, m.lo);
}

template <int PM>
__global__ void __launch_bounds__(128)
    k_m2l_mixed(const int2 *__restrict__ items, int n_items, int p,
                const double4 *__restrict__ geom, const int *__restrict__ weak_off,
                const int *__restrict__ weak, const float4 *__restrict__ mp,
                double2 *__restrict__ local) {
    pdl_wait();
    __shared__ __align__(16) float tab[DF_TAB_FLOATS];
    // per-lane accumulators live in shared memory (keeps registers, and so
    // occupancy, for the sweeps): sacc[warp][coefficient slot][lane]
    __shared__ float2 sacc[4][PM + 1][32];
    for (int i = threadIdx.x; i < DF_TAB_FLOATS; i += blockDim.x) tab[i] = d_dftab[i];
    const int lane = threadIdx.x & 31, comp = lane & 1, slot = lane >> 1;
    const int wib = threadIdx.x >> 5;
#pragma unroll
    for (int i = 0; i <= PM; ++i) sacc[wib][i][lane] = make_float2(0.f, 0.f);
    __syncthreads();
    const int item = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (item >= n_items) return;
    // the two lanes of one shift run the same iterations; shuffle within the pair
    const unsigned pmask = 3u << (lane & ~1);
    const int2 it = items[item];
    const int64_t g = it.x;
    const int e1 = min(it.y + M2L_CHUNK, weak_off[g + 1]);
    const int q = PM - p;  // right-alignment shift
    const double4 gt = geom[g];
    for (int e = it.y + slot; e < e1; e += 16) {
        const int64_t s = weak[e];
        const double4 gs = geom[s];
        // D = z_t - z_s in the units of the pair, 2^ep (PairUnits; an exactly
        // shared ordinate gives +0)
        const PairUnits pu = pair_units(gt.z, gs.z);
        const double pinv = pow2d(-pu.ep);
        const df Dx = split_d((gt.x - gs.x) * pinv), Dy = split_d((gt.y - gs.y) * pinv);
        // 1/r with r = -D:  1/r = -conj(D) / |D|^2
        df n2 = df_add(df_mul(Dx, Dx), df_mul(Dy, Dy));
        float rc = F_RCP(n2.hi);
        float i0 = rc;
        df corr = df_add(df{1.0f, 0.f}, df_neg(df_mulf(n2, i0)));  // 1 - n2 * i0
        df inv = df_add(df{i0, 0.f}, df_mulf(corr, i0));              // Newton step
        dc ir{df_neg(df_mul(Dx, inv)), df_mul(Dy, inv)};
        // u = sigma_s / r, v = sigma_t / r: the radii in pair units are fs, ft
        const float sig_s = pu.fs, sig_t = pu.ft;
        dc u{df{ir.re.hi * sig_s, ir.re.lo * sig_s}, df{ir.im.hi * sig_s, ir.im.lo * sig_s}};
        dc v{df{ir.re.hi * sig_t, ir.re.lo * sig_t}, df{ir.im.hi * sig_t, ir.im.lo * sig_t}};
        const float4 *A = mp + s * (p + 1);
        // prescale: slot k'-1 holds b_{k-1} = (-1)^k A_k u^k, k = k' - q
        df b[PM + 1];
#pragma unroll
        for (int i = 0; i <= PM; ++i) b[i] = df{0.f, 0.f};
        dc pw = u;
#pragma unroll
        for (int kk = 1; kk <= PM; ++kk) {
            if (kk > q) {
                const int k = kk - q;
                const float4 a4 = A[k];
                dc ak{df{a4.x, a4.y}, df{a4.z, a4.w}};
                dc x = dc_mul(ak, pw);
                df val = comp ? x.im : x.re;
                b[kk - 1] = (k & 1) ? df_neg(val) : val;
                pw = dc_mul(pw, u);
            }
        }
        // sweep 1 (entries j + q, j = p-k .. p-1)
#pragma unroll
        for (int k = 2; k <= PM; ++k) {
            if (k <= p) {
#pragma unroll
                for (int jj = PM - k; jj < PM; ++jj) b[jj] = df_acc(b[jj], b[jj + 1]);
            }
        }
        // sweep 2 (k = p .. 1, entries j + q, j = k .. p)
#pragma unroll
        for (int kk = PM; kk >= 1; --kk) {
            if (kk > q) {
#pragma unroll
                for (int jj = kk; jj <= PM; ++jj) b[jj] = df_acc(b[jj], b[jj - 1]);
            }
        }
        // postscale and accumulate
        const float4 a0 = A[0];
        const dc A0{df{a0.x, a0.y}, df{a0.z, a0.w}};
        {
            // l = 0: b_0 + A_0 Log(z_t - z_s)
            df S = df_add(df_mul(Dx, Dx), df_mul(Dy, Dy));
            df ln = df_log_f(S.hi, tab, pu.ecst);
            float ln_lo = F_FMA(0.5f, F_FMA(S.lo, F_RCP(S.hi), ln.lo), 0.f);
            df lr = fast_sum(F_MUL(0.5f, ln.hi), ln_lo);
            // arg of the df32 D: atan2 of the high parts plus first-order correction
            df an = df_atan2_f(Dy.hi, Dx.hi, tab + ATAN_OFF);
            float ci = F_MUL(F_FMA(Dy.lo, Dx.hi, -F_MUL(Dx.lo, Dy.hi)), F_RCP(S.hi));
            df li = fast_sum(an.hi, F_ADD(an.lo, ci));
            dc lg{lr, li};
            dc t = dc_mul(A0, lg);
            const df t0 = comp ? t.im : t.re;
#pragma unroll
            for (int jj = 0; jj <= PM; ++jj)
                if (jj == q) {
                    float2 a = sacc[wib][jj][lane];
                    df r = df_acc(df{a.x, a.y}, df_add(b[jj], t0));
                    sacc[wib][jj][lane] = make_float2(r.hi, r.lo);
                }
        }
        dc vp = v;
#pragma unroll
        for (int jj = 1; jj <= PM; ++jj) {
            if (jj > q) {
                const int l = jj - q;
                // c_l - A_0 / l (complex; the partner lane holds the other part)
                df mine = b[jj];
                df other = shfl_df(mine, 1, pmask);
                dc c{comp ? other : mine, comp ? mine : other};
                dc a0l{df_divf(A0.re, (float)l), df_divf(A0.im, (float)l)};
                dc d{df_add(c.re, df_neg(a0l.re)), df_add(c.im, df_neg(a0l.im))};
                dc t = dc_mul(d, vp);
                float2 a = sacc[wib][jj][lane];
                df r = df_acc(df{a.x, a.y}, comp ? t.im : t.re);
                sacc[wib][jj][lane] = make_float2(r.hi, r.lo);
                vp = dc_mul(vp, v);
            }
        }
    }
    // reduce over the 16 slots of the same component
    double *out = reinterpret_cast<double *>(local + g * (p + 1));
#pragma unroll
    for (int jj = 0; jj <= PM; ++jj) {
        float2 a2 = sacc[wib][jj][lane];
        df a{a2.x, a2.y};
#pragma unroll
        for (int m = 2; m < 32; m <<= 1) a = df_acc(a, shfl_df(a, m));
        if (slot == 0 && jj >= q)
            atomicAdd(out + 2 * (jj - q) + comp, (double)a.hi + (double)a.lo);
    }
}

__global__ void k_m2l_items_count(int64_t nb, const int *__restrict__ weak_off, uint32_t *cnt) {
    pdl_wait();
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nb) return;
    int n = weak_off[g + 1] - weak_off[g];
    cnt[g] = (uint32_t)((n + M2L_CHUNK - 1) / M2L_CHUNK);
}

__global__ void k_m2l_items_fill(int64_t nb, const int *__restrict__ weak_off,
                                 const uint32_t *__restrict__ off, int2 *items) {
    pdl_wait();
    int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= nb) return;
    int e0 = weak_off[g], e1 = weak_off[g + 1];
    uint32_t o = off[g];
    for (int e = e0; e < e1; e += M2L_CHUNK) items[o++] = make_int2((int)g, e);
}

// target box of every weak entry: one warp per box
__global__ void k_weak_tgt(int64_t nb, const int *__restrict__ weak_off, int *weak_tgt) {
    pdl_wait();
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (g >= nb) return;
    const int e1 = weak_off[g + 1];
    for (int e = weak_off[g] + (threadIdx.x & 31); e < e1; e += 32) weak_tgt[e] = (int)g;
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

template <int PM>
cudaError_t launch_pm(Tree &t, cudaStream_t s) {
    unsigned grid = nblk((int64_t)t.n_m2l_items * 32, 128);
    launch_k(k_m2l_mixed<PM>, grid, 128, 0, s, t.m2l_items, t.n_m2l_items, t.p, t.geom, t.weak_off,
             t.weak, t.mpole_df, t.local);
    return cudaGetLastError();
}

}  // namespace

cudaError_t upload_df_tables_m2l() {
    alignas(16) static float tab[DF_TAB_FLOATS];
    df32_fill_tables(tab);
    return cudaMemcpyToSymbol(d_dftab, tab, sizeof(tab));
}

// Largest order served by the df32 sweeps (register budget); above it the
// mixed mode runs M2L in FP64.
int m2l_mixed_max_p() { return 32; }

fmm_status m2l_items_count(Tree &t, cudaStream_t s, uint32_t *total_host) {
    cudaError_t e;
    const int64_t nb = t.n_boxes;
    DevArena tmp;
    tmp.stream = s;
    if ((e = arena_alloc(t.mem, &t.m2l_cnt, nb + 1)) != cudaSuccess) return cuda_fail(e, "m2l items");
    launch_k(k_m2l_items_count, nblk(nb, 256), 256, 0, s, nb, t.weak_off, t.m2l_cnt);
    if ((e = exclusive_scan_u32(t.m2l_cnt, t.m2l_cnt, nb, nullptr, tmp, s)) != cudaSuccess ||
        (e = cudaMemcpyAsync(total_host, t.m2l_cnt + nb, 4, cudaMemcpyDeviceToHost, s)) !=
            cudaSuccess) {
        tmp.release();
        return cuda_fail(e, "m2l items scan");
    }
    tmp.release();
    return FMM_OK;
}

fmm_status m2l_items_fill(Tree &t, uint32_t total, cudaStream_t s) {
    cudaError_t e;
    const int64_t nb = t.n_boxes;
    const bool tc = m2l_on_tensor_cores(t);
    t.n_m2l_items = tc ? 0 : (int)total;
    if (!tc) {
        if ((e = arena_alloc(t.mem, &t.m2l_items, (size_t)total + 1)) != cudaSuccess)
            return cuda_fail(e, "m2l items");
        launch_k(k_m2l_items_fill, nblk(nb, 256), 256, 0, s, nb, t.weak_off, t.m2l_cnt,
                 t.m2l_items);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "m2l items fill");
    }
    if ((e = arena_alloc(t.mem, &t.mpole_df, (size_t)nb * (t.p + 1))) != cudaSuccess)
        return cuda_fail(e, "df32 multipoles");
    if (tc) {
        // the tensor M2L takes the weak list in runs of 128 entries across boxes
        if ((e = arena_alloc(t.mem, &t.weak_tgt, (size_t)t.n_weak + 1)) != cudaSuccess)
            return cuda_fail(e, "weak targets");
        launch_k(k_weak_tgt, nblk(nb * 32, 256), 256, 0, s, nb, t.weak_off, t.weak_tgt);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "weak targets");
    }
    return FMM_OK;
}

fmm_status m2l_prepare_mixed(Tree &t, cudaStream_t s) {
    cudaError_t e;
    const int64_t nc = t.n_boxes * (int64_t)(t.p + 1);
    if ((e = cudaMemsetAsync(t.local, 0, nc * sizeof(double2), s)) != cudaSuccess)
        return cuda_fail(e, "zero locals");
    launch_k(k_mpole_df, nblk(nc, 256), 256, 0, s, nc, t.mpole, t.mpole_df);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "mpole df32");
    return FMM_OK;
}

fmm_status launch_m2l_mixed(Tree &t, cudaStream_t s) {
    cudaError_t e;
    if (t.n_m2l_items == 0) return FMM_OK;
    const int p = t.p;
    if (p <= 8)
        e = launch_pm<8>(t, s);
    else if (p <= 12)
        e = launch_pm<12>(t, s);
    else if (p <= 16)
        e = launch_pm<16>(t, s);
    else if (p <= 20)
        e = launch_pm<20>(t, s);
    else if (p <= 24)
        e = launch_pm<24>(t, s);
    else if (p <= 28)
        e = launch_pm<28>(t, s);
    else
        e = launch_pm<32>(t, s);
    return e == cudaSuccess ? FMM_OK : cuda_fail(e, "m2l mixed");
}

}  // namespace gbfmm
