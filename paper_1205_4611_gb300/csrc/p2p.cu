// Local evaluation (L2P, Eq. 5) and near-field direct evaluation (P2P,
// Alg. "Direct evaluation between boxes"), fused: one CTA per work item
// (a target leaf chunk of <= 64 evaluation points, one point per thread),
// source tiles of the strongly coupled leaves staged in shared memory; the
// result is written straight to the caller's order (un-permute fused).
// Exactly coincident pairs are skipped (the j != i of Eq. 1, x_j != y_i of
// Eq. 2).
#include <cuda_runtime.h>

#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace gbfmm {

namespace {

constexpr int EV_THREADS = 64;

__global__ void __launch_bounds__(EV_THREADS)
    k_eval64(const int2 *__restrict__ items, int p, const int2 *__restrict__ box_tgt,
             const int2 *__restrict__ box_src, const double4 *__restrict__ geom,
             const int *__restrict__ strong_off, const int *__restrict__ strong,
             const double2 *__restrict__ xt, const uint32_t *__restrict__ tperm,
             const double2 *__restrict__ xs, const double2 *__restrict__ qs,
             const double2 *__restrict__ local, double2 *__restrict__ phi) {
    __shared__ double2 sx[EV_THREADS], sq[EV_THREADS];
    __shared__ double2 sb[MAXP + 1];
    int2 it = items[blockIdx.x];
    const int64_t g = it.x;
    const int2 bt = box_tgt[g];
    const int nt = min(EV_THREADS, bt.y - it.y);
    for (int i = threadIdx.x; i <= p; i += EV_THREADS) sb[i] = local[g * (p + 1) + i];
    __syncthreads();
    const bool valid = threadIdx.x < nt;
    const int pos = bt.x + it.y + threadIdx.x;
    double2 y = valid ? xt[pos] : make_double2(0.0, 0.0);
    // L2P by Horner's rule in w = (y - c) / sigma
    const double4 ge = geom[g];
    cd w{(y.x - ge.x) * ge.w, (y.y - ge.y) * ge.w};
    cd acc{sb[p].x, sb[p].y};
    for (int l = p - 1; l >= 0; --l) acc = cadd(cmul(acc, w), cd{sb[l].x, sb[l].y});
    // P2P over the strong leaves, in list order
    const int e0 = strong_off[g], e1 = strong_off[g + 1];
    for (int e = e0; e < e1; ++e) {
        const int2 bs = box_src[strong[e]];
        for (int c0 = 0; c0 < bs.y; c0 += EV_THREADS) {
            const int nn = min(EV_THREADS, bs.y - c0);
            __syncthreads();
            if (threadIdx.x < nn) {
                sx[threadIdx.x] = xs[bs.x + c0 + threadIdx.x];
                sq[threadIdx.x] = qs[bs.x + c0 + threadIdx.x];
            }
            __syncthreads();
            if (valid) {
                for (int j = 0; j < nn; ++j) {
                    double dx = y.x - sx[j].x, dy = y.y - sx[j].y;
                    if (dx == 0.0 && dy == 0.0) continue;
                    double lr = 0.5 * log(fma(dx, dx, dy * dy));
                    double th = atan2(dy, dx);
                    double2 q = sq[j];
                    acc.re += q.x * lr - q.y * th;
                    acc.im += q.x * th + q.y * lr;
                }
            }
        }
    }
    if (valid) phi[tperm[pos]] = make_double2(acc.re, acc.im);
}

}  // namespace

fmm_status launch_eval(Tree &t, double *phi, cudaStream_t s) {
    if (t.n_items == 0) return FMM_OK;
    if (t.precision == FMM_PREC_MIXED) return launch_eval_mixed(t, phi, s);
    k_eval64<<<t.n_items, EV_THREADS, 0, s>>>(t.p2p_items, t.p, t.box_tgt, t.box_src, t.geom,
                                              t.strong_off, t.strong, t.xt, t.tperm, t.xs, t.qs,
                                              t.local, reinterpret_cast<double2 *>(phi)); note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "eval64");
    return FMM_OK;
}

}  // namespace gbfmm
