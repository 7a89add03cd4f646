// Direct near-field sum with no device allocation (fmm_direct_noalloc).
//
// Some callers cannot allocate device memory at the moment they need a
// potential: code running under a memory-pool or allocator lock, real-time
// loops whose memory budget is fixed up front, or hosts that only lend this
// library buffers they own.  This entry point evaluates the direct sum of
// Eq. (1) / Eq. (2) with a variant of the FP64 P2P kernel whose partial sums
// (one per (64-point chunk, 2048-source run) work item) live in a file-scope
// static device array instead of a buffer allocated per tree.
//
// The array is 4 MiB (262144 partial sums); a call needs
// ceil(n_tgt / 64) * ceil(n_src / 2048) * 64 of them and is rejected with
// FMM_ERR_ARG beyond that.  Every GPU that loads the library holds the array
// until the process exits.  All calls share it and it keeps the last call's
// contents: nothing in it needs to start at zero (every slot the combine
// kernel reads is written earlier in the same call), but calls that overlap
// on the GPU (two streams, or two host threads) race on it and must be
// ordered by the caller.
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "internal.h"

namespace gbfmm {

namespace {

constexpr int NA_THREADS = 64;        // evaluation points per work item
constexpr int NA_RUN = 2048;          // sources per work item
constexpr int64_t NA_SLOTS = 262144;  // partial sums held by the static array

static __device__ __align__(256) double2 na_partial[NA_SLOTS];

// Device address of na_partial per device (host code cannot use the symbol
// itself as a device pointer).
std::mutex na_mu;
double2 *na_ptr[64] = {};

__global__ void __launch_bounds__(NA_THREADS)
    k_p2p64_direct(const double2 *__restrict__ src, int64_t n_src, const double2 *__restrict__ q,
                   const double2 *__restrict__ tgt, int64_t n_tgt, int runs,
                   double2 *__restrict__ partial) {
    pdl_wait();
    __shared__ double2 sx[NA_THREADS], sq[NA_THREADS];
    const int item = blockIdx.x;
    const int chunk = item / runs, run = item % runs;
    const int64_t t0 = (int64_t)chunk * NA_THREADS;
    const int64_t s0 = (int64_t)run * NA_RUN;
    const int64_t s1 = min(s0 + (int64_t)NA_RUN, n_src);
    const bool valid = t0 + threadIdx.x < n_tgt;
    const double2 y = valid ? tgt[t0 + threadIdx.x] : make_double2(0.0, 0.0);
    double ar = 0.0, ai = 0.0;
    for (int64_t c0 = s0; c0 < s1; c0 += NA_THREADS) {
        const int nn = (int)min((int64_t)NA_THREADS, s1 - c0);
        __syncthreads();
        if (threadIdx.x < nn) {
            sx[threadIdx.x] = src[c0 + threadIdx.x];
            sq[threadIdx.x] = q[c0 + threadIdx.x];
        }
        __syncthreads();
        if (!valid) continue;
        for (int j = 0; j < nn; ++j) {
            double dx = y.x - sx[j].x, dy = y.y - sx[j].y;
            if (dx == 0.0 && dy == 0.0) continue;  // x_j == y_i
            double lr = 0.5 * log(fma(dx, dx, dy * dy));
            double th = atan2(dy, dx);
            double2 qq = sq[j];
            ar += qq.x * lr - qq.y * th;
            ai += qq.x * th + qq.y * lr;
        }
    }
    if (valid) partial[(int64_t)item * NA_THREADS + threadIdx.x] = make_double2(ar, ai);
}

__global__ void k_combine_direct(int64_t n_tgt, int runs, const double2 *__restrict__ partial,
                                 double2 *__restrict__ phi) {
    pdl_wait();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_tgt) return;
    const int64_t chunk = i / NA_THREADS, lane = i % NA_THREADS;
    double re = 0.0, im = 0.0;
    for (int r = 0; r < runs; ++r) {
        double2 v = partial[(chunk * runs + r) * NA_THREADS + lane];
        re += v.x;
        im += v.y;
    }
    phi[i] = make_double2(re, im);
}

}  // namespace

}  // namespace gbfmm

using namespace gbfmm;

extern "C" fmm_status fmm_direct_noalloc(const double *src_xy_dev, int64_t n_src,
                                         const double *q_dev, const double *tgt_xy_dev,
                                         int64_t n_tgt, double *phi_dev, void *stream) {
    set_error("");
    if (!src_xy_dev || !q_dev || !phi_dev || n_src < 1)
        return set_error("need sources, strengths and an output"), FMM_ERR_ARG;
    const double2 *tgt = reinterpret_cast<const double2 *>(tgt_xy_dev ? tgt_xy_dev : src_xy_dev);
    const int64_t m = tgt_xy_dev ? n_tgt : n_src;
    if (m < 1) return set_error("need at least one evaluation point"), FMM_ERR_ARG;
    const int64_t chunks = (m + NA_THREADS - 1) / NA_THREADS;
    const int64_t runs = (n_src + NA_RUN - 1) / NA_RUN;
    // compared without forming the product, which could overflow for huge sizes
    if (runs > NA_SLOTS / NA_THREADS || chunks > NA_SLOTS / NA_THREADS / runs)
        return set_error("fmm_direct_noalloc: ceil(n_tgt/64) * ceil(n_src/2048) * 64 exceeds the "
                         "262144 partial sums of its static scratch"),
               FMM_ERR_ARG;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "fmm_direct_noalloc: device");
    if (dev < 0 || dev >= 64) return set_error("device ordinal out of range"), FMM_ERR_ARG;
    double2 *scratch;
    {
        std::lock_guard<std::mutex> lk(na_mu);
        if (!na_ptr[dev]) {
            // once per device, with that device current
            void *p = nullptr;
            e = cudaGetSymbolAddress(&p, na_partial);
            if (e != cudaSuccess) return cuda_fail(e, "fmm_direct_noalloc: scratch address");
            na_ptr[dev] = static_cast<double2 *>(p);
        }
        scratch = na_ptr[dev];
    }
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    launch_k(k_p2p64_direct, (unsigned)(chunks * runs), NA_THREADS, 0, s,
             reinterpret_cast<const double2 *>(src_xy_dev), n_src,
             reinterpret_cast<const double2 *>(q_dev), tgt, m, (int)runs, scratch);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fmm_direct_noalloc");
    launch_k(k_combine_direct, (unsigned)((m + 255) / 256), 256, 0, s, m, (int)runs, scratch,
             reinterpret_cast<double2 *>(phi_dev));
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "fmm_direct_noalloc");
    return FMM_OK;
}
