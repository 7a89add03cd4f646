// Near-field direct evaluation (P2P, Alg. "Direct evaluation between boxes")
// and local evaluation (L2P, Eq. 5), FP64.
//
// Work items are (target leaf, chunk of <= 64 evaluation points, run of the
// leaf's near-field list: the strong list, or with the leaf shortcut its near
// part); one CTA of 64 threads per item, one to four threads
// per evaluation point depending on how many points the chunk holds (the
// paper's "one to four threads per evaluation point"), source tiles staged
// in shared memory.  Items (and the shortcut's M2P items) write partial sums;
// k_combine then adds, per evaluation point and in item order, the L2P value
// and the partial sums and
// writes the potential in the caller's order (un-permute fused).
// Exactly coincident pairs are skipped (j != i in Eq. 1, x_j != y_i in Eq. 2).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace gbfmm {

namespace {

constexpr int EV_THREADS = 64;

GBI int threads_per_target(int nt) { return nt <= 16 ? 4 : (nt <= 32 ? 2 : 1); }

// KERN 0: q Log(y - x) (Eq. 1, Eq. 2); KERN 1: q / (x - y) (harmonic kernel).
template <int KERN>
__global__ void __launch_bounds__(EV_THREADS)
    k_p2p64(const int4 *__restrict__ items, const int *__restrict__ order,
            const int2 *__restrict__ box_tgt, const int2 *__restrict__ box_src,
            const int *__restrict__ strong, const double2 *__restrict__ xt,
            const double2 *__restrict__ xs, const double2 *__restrict__ qs,
            double2 *__restrict__ partial) {
    pdl_wait();
    __shared__ double2 sx[EV_THREADS], sq[EV_THREADS];
    const int idx = order[blockIdx.x];
    const int4 it = items[idx];
    const int2 bt = box_tgt[it.x];
    const int nt = min(EV_THREADS, bt.y - it.y);
    const int tpt = threads_per_target(nt);
    const int my = threadIdx.x / tpt, sub = threadIdx.x % tpt;
    const bool valid = my < nt;
    double2 y = valid ? xt[bt.x + it.y + my] : make_double2(0.0, 0.0);
    double ar = 0.0, ai = 0.0;
    for (int e = it.z; e < it.w; ++e) {
        const int2 bs = box_src[strong[e]];
        for (int c0 = 0; c0 < bs.y; c0 += EV_THREADS) {
            const int nn = min(EV_THREADS, bs.y - c0);
            __syncthreads();
            if (threadIdx.x < nn) {
                sx[threadIdx.x] = xs[bs.x + c0 + threadIdx.x];
                sq[threadIdx.x] = qs[bs.x + c0 + threadIdx.x];
            }
            __syncthreads();
            if (!valid) continue;
            for (int j = sub; j < nn; j += tpt) {
                double dx = y.x - sx[j].x, dy = y.y - sx[j].y;
                if (dx == 0.0 && dy == 0.0) continue;
                double2 q = sq[j];
                if (KERN == 1) {
                    // q / (x - y) = -q conj(D) / |D|^2
                    const double r = -1.0 / fma(dx, dx, dy * dy);
                    const double vr = dx * r, vi = -dy * r;
                    ar += q.x * vr - q.y * vi;
                    ai += q.x * vi + q.y * vr;
                } else {
                    double lr = 0.5 * log(fma(dx, dx, dy * dy));
                    double th = atan2(dy, dx);
                    ar += q.x * lr - q.y * th;
                    ai += q.x * th + q.y * lr;
                }
            }
        }
    }
    // combine the threads of one evaluation point (adjacent lanes)
    for (int m = 1; m < tpt; m <<= 1) {
        ar += __shfl_xor_sync(0xffffffffu, ar, m);
        ai += __shfl_xor_sync(0xffffffffu, ai, m);
    }
    if (valid && sub == 0) partial[(int64_t)idx * EV_THREADS + my] = make_double2(ar, ai);
}

// L2P by Horner's rule plus the partial near-field sums, in item order.
__global__ void __launch_bounds__(EV_THREADS)
    k_combine(const int2 *__restrict__ chunks, const int *__restrict__ item0, int p,
              const int2 *__restrict__ box_tgt, const double4 *__restrict__ geom,
              const double2 *__restrict__ xt, const uint32_t *__restrict__ tperm,
              const double2 *__restrict__ local, const double2 *__restrict__ partial,
              double2 *__restrict__ phi, int kern) {
    pdl_wait();
    __shared__ double2 sb[MAXP + 1];
    const int c = blockIdx.x;
    const int2 ch = chunks[c];
    const int64_t g = ch.x;
    for (int i = threadIdx.x; i <= p; i += EV_THREADS) sb[i] = local[g * (p + 1) + i];
    __syncthreads();
    const int2 bt = box_tgt[g];
    const int nt = min(EV_THREADS, bt.y - ch.y);
    if (threadIdx.x >= nt) return;
    const int pos = bt.x + ch.y + threadIdx.x;
    const double2 y = xt[pos];
    const double4 ge = geom[g];
    cd w{(y.x - ge.x) * ge.w, (y.y - ge.y) * ge.w};
    cd acc;
    if (kern) {
        // -d/dy sum B_l w^l = -(1/sigma) sum l B_l w^(l-1)
        acc = cscale(cd{sb[p].x, sb[p].y}, (double)p);
        for (int l = p - 1; l >= 1; --l)
            acc = cadd(cmul(acc, w), cscale(cd{sb[l].x, sb[l].y}, (double)l));
        acc = cscale(acc, -ge.w);
    } else {
        acc = cd{sb[p].x, sb[p].y};
        for (int l = p - 1; l >= 0; --l) acc = cadd(cmul(acc, w), cd{sb[l].x, sb[l].y});
    }
    for (int it = item0[c]; it < item0[c + 1]; ++it) {
        double2 v = partial[(int64_t)it * EV_THREADS + threadIdx.x];
        acc.re += v.x;
        acc.im += v.y;
    }
    phi[tperm[pos]] = make_double2(acc.re, acc.im);
}

}  // namespace

fmm_status launch_eval(Tree &t, double *phi, cudaStream_t s, int part) {
    cudaError_t e;
    if (part == EVAL_P2P && t.n_p2p_items > 0) {
        if (t.precision == FMM_PREC_MIXED) {
            fmm_status st = launch_p2p_mixed(t, s);
            if (st != FMM_OK) return st;
        } else {
            auto k = t.kernel ? k_p2p64<1> : k_p2p64<0>;
            launch_k(k, t.n_p2p_items, EV_THREADS, 0, s, t.p2p_items, t.p2p_order, t.box_tgt,
                     t.box_src, t.p2p_list, t.xt, t.xs, t.qs, t.p2p_partial);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "p2p64");
        }
    }
    if (part == EVAL_M2P && t.n_items > t.n_p2p_items) {  // M2P items of the leaf shortcut
        fmm_status st = launch_m2p(t, s);
        if (st != FMM_OK) return st;
    }
    if (part == EVAL_COMBINE && t.n_chunks > 0 && combine_mixed_ok(t))
        return launch_combine_mixed(t, phi, s);
    if (part == EVAL_COMBINE && t.n_chunks > 0) {
        launch_k(k_combine, t.n_chunks, EV_THREADS, 0, s, t.p2p_chunks, t.p2p_item0, t.p, t.box_tgt,
                 t.geom, t.xt, t.tperm, t.local, t.p2p_partial, reinterpret_cast<double2 *>(phi),
                 t.kernel);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "combine");
    }
    return FMM_OK;
}

}  // namespace gbfmm
