// Computational phase (Sec. 3.3), FP64: P2M, M2M, M2L, L2L.
//
// Expansions are stored radius-normalised: with sigma_b = 2^e_b >= the box
// radius (a power of two, so scaling is exact), the multipole of Eq. (4) is
// kept as  A_k = a_k / sigma^k  and the local of Eq. (5) as  B_l = b_l sigma^l.
// Every translation below is the closed form of the paper's shift written in
// those variables:
//
//   P2M  A_0 = sum q_j,  A_k = -sum q_j w_j^k / k,   w_j = (x_j - c) / sigma
//   M2M  (child c -> parent p, rho = (z_c - z_p)/sigma_p, s = sigma_c/sigma_p)
//        A'_0 += A_0,  A'_l += sum_{k=1}^{l} C(l-1,k-1) rho^{l-k} s^k A_k - A_0 rho^l / l
//   M2L  (source s -> target t, r = z_s - z_t, u = sigma_s / r, v = sigma_t / r)
//        x_k = (-1)^k A_k u^k,  c_l = sum_{k=1}^{p} C(k+l-1, l) x_k
//        B_0 += c_0 + A_0 Log(z_t - z_s),  B_l += (c_l - A_0 / l) v^l
//   L2L  (parent p -> child c, d = (z_c - z_p)/sigma_p, s = sigma_c/sigma_p)
//        B'_l += s^l sum_{k=l}^{p} C(k,l) d^{k-l} B_k
//
// (Alg. "Multipole to multipole translation", "Local to local translation",
// "Multipole to local translation" compute the same operators by scaled
// summation sweeps; the M2L a_0 term uses the branch Log(z_t - z_s).)
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace gbfmm {

namespace {

constexpr int BINOM_N = 130;  // C(n, k) for n < 130
__device__ double d_binom[BINOM_N * (BINOM_N + 1) / 2];
__device__ double d_inv[MAXP + 2];

GBI double binom(int n, int k) { return d_binom[n * (n + 1) / 2 + k]; }

GBI cd warp_sum(cd v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        v.re += shfl_xor_d(v.re, o);
        v.im += shfl_xor_d(v.im, o);
    }
    return v;
}

// Inclusive multiplicative scan over the 32 lanes: lane j gets prod_{i<=j} v_i.
GBI cd warp_prod_scan(cd v) {
    int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        double re = __shfl_up_sync(0xffffffffu, v.re, o);
        double im = __shfl_up_sync(0xffffffffu, v.im, o);
        if (lane >= o) v = cmul(v, cd{re, im});
    }
    return v;
}

// P2M at the leaves: one warp per leaf, one source per lane, powers by
// recurrence, butterfly reductions per coefficient.
__global__ void k_p2m(int64_t nleaf, const int *__restrict__ leaves, int p,
                      const int2 *__restrict__ box_src,
                      const double4 *__restrict__ geom, const double2 *__restrict__ xs,
                      const double2 *__restrict__ qs, double2 *__restrict__ mpole) {
    pdl_wait();
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (w >= nleaf) return;
    int64_t g = leaves[w];
    int2 bs = box_src[g];
    double4 ge = geom[g];
    cd acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int c0 = 0; c0 < bs.y; c0 += 32) {
        int j = c0 + lane;
        cd wv{0, 0}, q{0, 0};
        if (j < bs.y) {
            double2 x = xs[bs.x + j], qq = qs[bs.x + j];
            wv = cd{(x.x - ge.x) * ge.w, (x.y - ge.y) * ge.w};
            q = cd{qq.x, qq.y};
        }
        cd s0 = warp_sum(q);
        if (lane == 0) acc[0] = cadd(acc[0], s0);
        cd pw{1.0, 0.0};
        for (int k = 1; k <= p; ++k) {
            pw = cmul(pw, wv);
            cd t = cscale(cmul(q, pw), -d_inv[k]);
            t = warp_sum(t);
            if (lane == (k & 31)) acc[k >> 5] = cadd(acc[k >> 5], t);
        }
    }
    double2 *out = mpole + g * (p + 1);
    for (int j = 0; j < 3; ++j) {
        int k = lane + 32 * j;
        if (k <= p) out[k] = make_double2(acc[j].re, acc[j].im);
    }
}

// M2M for the boxes of one level (entries of `boxes`; leaves, child0 < 0,
// are skipped): one block per box, one thread per coefficient.
__global__ void k_m2m(const int *__restrict__ boxes, const int *__restrict__ child0, int p,
                      const double4 *__restrict__ geom, const int2 *__restrict__ box_src,
                      double2 *mpole) {
    pdl_wait();
    __shared__ double2 ch[4][MAXP + 1];
    const int64_t g = boxes[blockIdx.x];
    const int64_t c0 = child0[g];
    if (c0 < 0) return;
    int l = threadIdx.x;
    for (int i = threadIdx.x; i < 4 * (p + 1); i += blockDim.x) {
        int c = i / (p + 1), k = i % (p + 1);
        ch[c][k] = mpole[(c0 + c) * (p + 1) + k];
    }
    __syncthreads();
    if (l > p) return;
    double4 gp = geom[g];
    cd acc{0, 0};
    for (int c = 0; c < 4; ++c) {
        // a child without sources has a zero multipole; with shrink-wrapped
        // geometry its centre may lie outside a parent of radius 0 (1/sigma
        // beyond the range), so it is skipped rather than translated
        if (box_src[c0 + c].y == 0) continue;
        double4 gc = geom[c0 + c];
        cd rho{(gc.x - gp.x) * gp.w, (gc.y - gp.y) * gp.w};
        // s = sigma_c / sigma_p and 1/s: powers of two, exact
        double sc = gc.z * gp.w, isc = gp.z * gc.w;
        cd a0{ch[c][0].x, ch[c][0].y};
        if (l == 0) {
            acc = cadd(acc, a0);
            continue;
        }
        // k from l down to 1: rho^{l-k} grows, s^k shrinks
        cd pw{1.0, 0.0};
        double sk = 1.0;
        for (int i = 0; i < l; ++i) sk *= sc;  // s^l (exact, power of two)
        cd sum{0, 0};
        for (int k = l; k >= 1; --k) {
            cd ak{ch[c][k].x, ch[c][k].y};
            sum = cadd(sum, cscale(cmul(pw, ak), binom(l - 1, k - 1) * sk));
            pw = cmul(pw, rho);
            sk *= isc;
        }
        // pw = rho^l now
        sum = csub(sum, cscale(cmul(a0, pw), d_inv[l]));
        acc = cadd(acc, sum);
    }
    mpole[g * (p + 1) + l] = make_double2(acc.re, acc.im);
}

// M2L over all weak pairs, one warp per target box; writes (not adds) the
// local expansion of every box.  Lane j holds u^(j+1) and v^(j+1) after a
// multiplicative warp scan; lane l owns output coefficients l, l+32, l+64.
__global__ void k_m2l(int64_t n_boxes, int p, const double4 *__restrict__ geom,
                      const int *__restrict__ weak_off, const int *__restrict__ weak,
                      const double2 *__restrict__ mpole, double2 *__restrict__ local) {
    pdl_wait();
    __shared__ double2 xbuf[4][MAXP + 2];
    int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (w >= n_boxes) return;
    int64_t g = w;
    double4 gt = geom[g];
    cd acc[3] = {{0, 0}, {0, 0}, {0, 0}};
    for (int e = weak_off[g]; e < weak_off[g + 1]; ++e) {
        int64_t s = weak[e];
        double4 gs = geom[s];
        cd r{gs.x - gt.x, gs.y - gt.y};
        cd ir = cinv(r);
        cd u = cscale(ir, gs.z), v = cscale(ir, gt.z);
        cd up = warp_prod_scan(u), vp = warp_prod_scan(v);
        cd u32{__shfl_sync(0xffffffffu, up.re, 31), __shfl_sync(0xffffffffu, up.im, 31)};
        cd v32{__shfl_sync(0xffffffffu, vp.re, 31), __shfl_sync(0xffffffffu, vp.im, 31)};
        cd vl0{__shfl_up_sync(0xffffffffu, vp.re, 1), __shfl_up_sync(0xffffffffu, vp.im, 1)};
        if (lane == 0) vl0 = cd{1.0, 0.0};
        cd vl[3];
        vl[0] = vl0;
        vl[1] = cmul(vl0, v32);
        vl[2] = cmul(vl[1], v32);
        const double2 *a = mpole + s * (p + 1);
        for (int j = 0; j < 2; ++j) {
            int k = lane + 1 + 32 * j;
            if (k <= p) {
                cd pk = j ? cmul(up, u32) : up;
                double2 ak = a[k];
                cd x = cmul(cd{ak.x, ak.y}, pk);
                if (k & 1) x = cd{-x.re, -x.im};
                xbuf[wib][k] = make_double2(x.re, x.im);
            }
        }
        __syncwarp();
        double2 a0d = a[0];
        cd a0{a0d.x, a0d.y};
        for (int j = 0; j < 3; ++j) {
            int l = lane + 32 * j;
            if (l > p) break;
            cd c{0, 0};
            for (int k = 1; k <= p; ++k) {
                double2 xk = xbuf[wib][k];
                double bn = binom(k + l - 1, l);
                c.re = fma(bn, xk.x, c.re);
                c.im = fma(bn, xk.y, c.im);
            }
            cd term;
            if (l == 0)
                // Log(z_t - z_s) from the centres directly: an exactly shared
                // coordinate gives +0.0 (not -0.0), which fixes the side of the
                // branch cut the same way as the complex subtraction does
                term = cadd(c, cmul(a0, clog_principal(cd{gt.x - gs.x, gt.y - gs.y})));
            else
                term = cmul(csub(c, cscale(a0, d_inv[l])), vl[j]);
            acc[j] = cadd(acc[j], term);
        }
        __syncwarp();
    }
    double2 *out = local + g * (p + 1);
    for (int j = 0; j < 3; ++j) {
        int l = lane + 32 * j;
        if (l <= p) out[l] = make_double2(acc[j].re, acc[j].im);
    }
}

// L2L for the boxes of one level (entries of `boxes`, each with a parent):
// one block per box, one thread per coefficient; adds to the box's local.
__global__ void k_l2l(const int *__restrict__ boxes, const int *__restrict__ parent, int p,
                      const double4 *__restrict__ geom, const int2 *__restrict__ box_tgt,
                      double2 *local) {
    pdl_wait();
    __shared__ double2 par[MAXP + 1];
    const int64_t g = boxes[blockIdx.x], gpar = parent[g];
    // a box without evaluation points never uses its local expansion (nor do
    // its children); skipped, as its centre may lie outside a parent of radius 0
    if (box_tgt[g].y == 0) return;
    for (int i = threadIdx.x; i <= p; i += blockDim.x) par[i] = local[gpar * (p + 1) + i];
    __syncthreads();
    int l = threadIdx.x;
    if (l > p) return;
    double4 gp = geom[gpar], gc = geom[g];
    cd d{(gc.x - gp.x) * gp.w, (gc.y - gp.y) * gp.w};
    double sc = gc.z * gp.w;
    double sl = 1.0;
    for (int i = 0; i < l; ++i) sl *= sc;
    cd sum{0, 0}, pw{1.0, 0.0};
    for (int k = l; k <= p; ++k) {
        cd bk{par[k].x, par[k].y};
        sum = cadd(sum, cscale(cmul(pw, bk), binom(k, l)));
        pw = cmul(pw, d);
    }
    sum = cscale(sum, sl);
    double2 old = local[g * (p + 1) + l];
    local[g * (p + 1) + l] = make_double2(old.x + sum.re, old.y + sum.im);
}

__global__ void k_permute_q(int64_t n, const uint32_t *__restrict__ perm,
                            const double2 *__restrict__ q, double2 *qs) {
    pdl_wait();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) qs[i] = q[perm[i]];
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)std::max<int64_t>(1, (n + t - 1) / t); }

std::mutex g_tab_mu;
bool g_tab_ready[64] = {};

}  // namespace

cudaError_t ensure_tables() {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    std::lock_guard<std::mutex> lk(g_tab_mu);
    if (dev < 64 && g_tab_ready[dev]) return cudaSuccess;
    static double tab[BINOM_N * (BINOM_N + 1) / 2];
    static double inv[MAXP + 2];
    for (int n = 0; n < BINOM_N; ++n) {
        tab[n * (n + 1) / 2] = 1.0;
        tab[n * (n + 1) / 2 + n] = 1.0;
        for (int k = 1; k < n; ++k)
            tab[n * (n + 1) / 2 + k] = tab[(n - 1) * n / 2 + k - 1] + tab[(n - 1) * n / 2 + k];
    }
    inv[0] = 0.0;
    for (int k = 1; k < MAXP + 2; ++k) inv[k] = 1.0 / k;
    if ((e = cudaMemcpyToSymbol(d_binom, tab, sizeof(tab))) != cudaSuccess) return e;
    if ((e = cudaMemcpyToSymbol(d_inv, inv, sizeof(inv))) != cudaSuccess) return e;
    if ((e = upload_df_tables()) != cudaSuccess) return e;
    if ((e = upload_df_tables_m2l()) != cudaSuccess) return e;
    if ((e = upload_df_tables_tc()) != cudaSuccess) return e;
    if ((e = upload_df_tables_sc()) != cudaSuccess) return e;
    if ((e = upload_binom_df()) != cudaSuccess) return e;
    if ((e = upload_df_tables_sym()) != cudaSuccess) return e;
    // Keep freed stream-ordered memory in this process's default pool instead
    // of returning it to the driver at every synchronisation: tree builds
    // allocate and free their scratch each call (a pool attribute of this
    // process, not a device setting).
    {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t keep = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    if (dev < 64) g_tab_ready[dev] = true;
    return cudaSuccess;
}


void mark_event(Tree &t, int i, cudaStream_t s) {
    if (t.timing.enabled) cudaEventRecord(t.timing.ev[i], s);
}

static inline void mark(Tree &t, int i, cudaStream_t s) { mark_event(t, i, s); }

// The second stream (the far field of an evaluation, the build's last
// independent steps): one per host thread and device, of the default
// priority.  (With the highest priority the step measured 1 % slower: the
// M2L kernel's blocks, which each take a whole SM, then hold SMs idle while
// the near field's blocks on them drain.)
cudaStream_t side_stream() {
    static thread_local cudaStream_t of[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
    if (!of[dev] && cudaStreamCreateWithFlags(&of[dev], cudaStreamNonBlocking) != cudaSuccess)
        of[dev] = nullptr;
    return of[dev];
}

bool side_events(Tree &t) {
    if (t.far_mpole) return true;
    cudaEvent_t *evs[3] = {&t.far_fork, &t.far_join, &t.far_mpole};
    for (cudaEvent_t *ev : evs)
        if (!*ev && cudaEventCreateWithFlags(ev, cudaEventDisableTiming) != cudaSuccess) {
            *ev = nullptr;
            return false;
        }
    return true;
}

fmm_status run_evaluate(Tree &t, const double *q, double *phi, cudaStream_t s) {
    cudaError_t e;
    const int p = t.p, L = t.L;
    fmm_status st = FMM_OK;
    mark(t, 0, s);
    launch_k(k_permute_q, nblk(t.n_src, 256), 256, 0, s, t.n_src, t.perm,
             reinterpret_cast<const double2 *>(q), t.qs);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "permute");
    if (t.precision == FMM_PREC_MIXED) {
        st = permute_q_mixed(t, q, s);
        if (st != FMM_OK) return st;
    }
    mark(t, 1, s);
    // ---- far field: the upward pass (P2M, M2M), M2L, the downward pass with
    // the leaf shortcut's P2L.  The near field shares only the multipoles with
    // it (M2P reads them, after the upward pass) until the final combination,
    // so unless phase timing is on (the phases then run one after another on
    // s, each span timing its own kernels) it runs on a second stream f,
    // joined before M2P (multipoles) and before the combination (locals): its
    // latency-bound levels and the kernels' tails fill in beside the P2P
    // blocks.  (Pinning M2L between two parts of the P2P items instead, so
    // that P2P blocks never hold the SMs it waits for, measured slower.)
    cudaStream_t f = s;
    if (!t.timing.enabled) {
        cudaStream_t fs = side_stream();
        if (fs && side_events(t) && cudaEventRecord(t.far_fork, s) == cudaSuccess &&
            cudaStreamWaitEvent(fs, t.far_fork, 0) == cudaSuccess)
            f = fs;
    }
    auto upward = [&](cudaStream_t x) -> fmm_status {
        cudaError_t e;
        fmm_status st = FMM_OK;
        const int64_t nleaf = t.n_leaves;
        if (t.precision == FMM_PREC_MIXED && p <= p2m_mixed_max_p()) {
            st = launch_p2m_mixed(t, x);
            if (st != FMM_OK) return st;
        } else {
            launch_k(k_p2m, nblk(nleaf * 32, 128), 128, 0, x, nleaf, t.leaves, p, t.box_src,
                     t.geom, t.xs, t.qs, t.mpole);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "p2m");
        }
        mark(t, 2, x);
        const bool mixed_tr = t.precision == FMM_PREC_MIXED && p <= translate_mixed_max_p();
        for (int l = L - 1; l >= 0; --l) {
            if (mixed_tr) {
                st = launch_m2m_mixed(t, l, x);
                if (st != FMM_OK) return st;
                continue;
            }
            launch_k(k_m2m, (unsigned)(t.level_start[l + 1] - t.level_start[l]),
                     64 + 32 * (p >= 64), 0, x, t.lvl_boxes + t.level_start[l], t.child0, p,
                     t.geom, t.box_src, t.mpole);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "m2m");
        }
        mark(t, 3, x);
        return FMM_OK;
    };
    auto m2l = [&](cudaStream_t x) -> fmm_status {
        cudaError_t e;
        fmm_status st = FMM_OK;
        const bool m2l_df = t.precision == FMM_PREC_MIXED && t.p <= m2l_mixed_max_p();
        if (t.precision == FMM_PREC_MIXED && t.m2l_slices > 0 && t.p <= m2l_tc_max_p()) {
            st = launch_m2l_tc(t, x);
            if (st != FMM_OK) return st;
        } else if (m2l_df) {
            st = launch_m2l_mixed(t, x);
            if (st != FMM_OK) return st;
        } else {
            launch_k(k_m2l, nblk(t.n_boxes * 32, 128), 128, 0, x, t.n_boxes, p, t.geom,
                     t.weak_off, t.weak, t.mpole, t.local);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "m2l");
        }
        mark(t, 4, x);
        return FMM_OK;
    };
    auto downward = [&](cudaStream_t x) -> fmm_status {
        cudaError_t e;
        fmm_status st = FMM_OK;
        const bool mixed_tr = t.precision == FMM_PREC_MIXED && p <= translate_mixed_max_p();
        for (int l = 1; l <= L; ++l) {
            if (mixed_tr) {  // parents at level l - 1 into their children
                st = launch_l2l_mixed(t, l - 1, x);
                if (st != FMM_OK) return st;
                continue;
            }
            launch_k(k_l2l, (unsigned)(t.level_start[l + 1] - t.level_start[l]),
                     64 + 32 * (p >= 64), 0, x, t.lvl_boxes + t.level_start[l], t.parent, p,
                     t.geom, t.box_tgt, t.local);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "l2l");
        }
        mark(t, 5, x);
        st = launch_p2l(t, x);  // leaf shortcut (no-op unless enabled)
        if (st != FMM_OK) return st;
        mark(t, 6, x);
        return FMM_OK;
    };
    st = upward(f);
    // the df32 multipoles (M2L, M2P) and zeroed locals; then the multipoles
    // are complete for the near field's M2P
    if (st == FMM_OK && t.precision == FMM_PREC_MIXED && t.p <= m2l_mixed_max_p())
        st = m2l_prepare_mixed(t, f);
    if (st == FMM_OK && f != s && (e = cudaEventRecord(t.far_mpole, f)) != cudaSuccess)
        st = cuda_fail(e, "far-field stage");
    if (st == FMM_OK) st = m2l(f);
    if (st == FMM_OK) st = downward(f);
    // joined on every path, so that nothing the caller frees is still in use on f
    if (f != s && (e = cudaEventRecord(t.far_join, f)) == cudaSuccess && st != FMM_OK)
        cudaStreamWaitEvent(s, t.far_join, 0);
    if (st != FMM_OK) return st;
    if (f != s && e != cudaSuccess) return cuda_fail(e, "far-field join");
    // ---- near field, M2P, then the combination with L2P
    auto part = [&](int k, cudaStream_t ps) {
        return t.sym ? launch_eval_sym(t, phi, ps, k) : launch_eval(t, phi, ps, k);
    };
    mark(t, 9, s);
    if ((st = part(EVAL_P2P, s)) != FMM_OK) return st;
    mark(t, 7, s);
    if (f != s && (e = cudaStreamWaitEvent(s, t.far_mpole, 0)) != cudaSuccess)
        return cuda_fail(e, "far-field stage");
    mark(t, 10, s);
    if ((st = part(EVAL_M2P, s)) != FMM_OK) return st;
    mark(t, 11, s);
    if (f != s && (e = cudaStreamWaitEvent(s, t.far_join, 0)) != cudaSuccess)
        return cuda_fail(e, "far-field join");
    mark(t, 12, s);
    if ((st = part(EVAL_COMBINE, s)) != FMM_OK) return st;
    mark(t, 8, s);
    return FMM_OK;
}

}  // namespace gbfmm
