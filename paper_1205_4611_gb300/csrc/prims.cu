// Device primitives of the tree build: exclusive scan and a stable LSD radix
// sort of (64-bit key, 32-bit value) pairs.  Deterministic: no atomics decide
// any order.
#include <cuda_runtime.h>

#include <utility>

#include "common.cuh"
#include "internal.h"

namespace gbfmm {

namespace {

constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// Block-wide exclusive scan of one value per thread; returns the block total.
__device__ uint32_t block_exclusive_scan(uint32_t v, uint32_t &excl) {
    __shared__ uint32_t warp_tot[SCAN_THREADS / 32];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    for (int w = 0; w < SCAN_THREADS / 32; ++w) {
        uint32_t t = warp_tot[w];
        if (w < warp) wp += t;
        tot += t;
    }
    excl = wp + x - v;
    __syncthreads();
    return tot;
}

__global__ void k_scan_reduce(const uint32_t *__restrict__ in, int64_t n,
                              uint32_t *__restrict__ sums) {
    pdl_wait();
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint32_t s = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t k = base + i;
        if (k < n) s += in[k];
    }
    uint32_t excl;
    uint32_t tot = block_exclusive_scan(s, excl);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// Scans one tile per block; block b adds prefix[b] (or base for a single block).
__global__ void k_scan_apply(const uint32_t *in, uint32_t *out, int64_t n,
                             const uint32_t *__restrict__ prefix,
                             const uint32_t *__restrict__ base_dev) {
    pdl_wait();
    __shared__ uint32_t tile[SCAN_TILE];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t k = base + i;
        tile[i] = (k < n) ? in[k] : 0u;
    }
    __syncthreads();
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        v[j] = tile[threadIdx.x * SCAN_ITEMS + j];
        s += v[j];
    }
    uint32_t excl;
    uint32_t tot = block_exclusive_scan(s, excl);
    uint32_t off = prefix ? prefix[blockIdx.x] : (base_dev ? *base_dev : 0u);
    uint32_t run = off + excl;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        tile[threadIdx.x * SCAN_ITEMS + j] = run;
        run += v[j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t k = base + i;
        if (k < n) out[k] = tile[i];
    }
    if (threadIdx.x == 0 && base + SCAN_TILE >= n) out[n] = off + tot;
}

// ------------------------------------------------ two-pass scans (<= SCAN_MAX_TILES tiles)
//
// Pass 1 reduces every tile; pass 2 scans each tile, every block adding the
// sum of all earlier tiles, which it reads itself (at most SCAN_MAX_TILES).
// Values come through a loader, so a scan can read a transformed input.
// blockIdx.y selects one of up to three independent scans of the same length.
constexpr int SCAN_MAX_TILES = 4096;
constexpr int SCAN_MAX_SETS = 3;

struct LoadArr {
    const uint32_t *in;
    GBI uint32_t operator()(int64_t i) const { return in[i]; }
};

template <class Ld>
struct ScanSets {
    Ld ld[SCAN_MAX_SETS];
    uint32_t *out[SCAN_MAX_SETS];
    const uint32_t *base[SCAN_MAX_SETS];  // device word added to every output, or NULL
};

template <class Ld>
__global__ void k_scan2_reduce(ScanSets<Ld> S, int64_t n, uint32_t *__restrict__ sums, int nb) {
    pdl_wait();
    const Ld ld = S.ld[blockIdx.y];
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    uint32_t s = 0;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t k = base + i;
        if (k < n) s += ld(k);
    }
    uint32_t excl;
    uint32_t tot = block_exclusive_scan(s, excl);
    if (threadIdx.x == 0) sums[(int64_t)blockIdx.y * nb + blockIdx.x] = tot;
}

template <class Ld>
__global__ void k_scan2_apply(ScanSets<Ld> S, int64_t n, const uint32_t *__restrict__ sums,
                              int nb) {
    pdl_wait();
    __shared__ uint32_t tile[SCAN_TILE];
    const Ld ld = S.ld[blockIdx.y];
    uint32_t *out = S.out[blockIdx.y];
    const uint32_t *bp = S.base[blockIdx.y];
    const uint32_t *ts = sums + (int64_t)blockIdx.y * nb;
    // prefix of the earlier tiles
    uint32_t part = 0;
    for (int k = threadIdx.x; k < (int)blockIdx.x; k += SCAN_THREADS) part += ts[k];
    uint32_t dummy;
    const uint32_t prefix = block_exclusive_scan(part, dummy);
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE;
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t k = base + i;
        tile[i] = (k < n) ? ld(k) : 0u;
    }
    __syncthreads();
    uint32_t v[SCAN_ITEMS];
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        v[j] = tile[threadIdx.x * SCAN_ITEMS + j];
        s += v[j];
    }
    uint32_t excl;
    uint32_t tot = block_exclusive_scan(s, excl);
    const uint32_t off = (bp ? *bp : 0u) + prefix;
    uint32_t run = off + excl;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        tile[threadIdx.x * SCAN_ITEMS + j] = run;
        run += v[j];
    }
    __syncthreads();
    for (int i = threadIdx.x; i < SCAN_TILE; i += SCAN_THREADS) {
        int64_t k = base + i;
        if (k < n) out[k] = tile[i];
    }
    if (threadIdx.x == 0 && base + SCAN_TILE >= n) out[n] = off + tot;
}

template <class Ld>
cudaError_t scan2(const ScanSets<Ld> &S, int nscan, int64_t n, DevArena &scratch,
                  cudaStream_t s) {
    const int nb = (int)((n + SCAN_TILE - 1) / SCAN_TILE);
    uint32_t *sums = nullptr;
    cudaError_t e = arena_alloc(scratch, &sums, (size_t)nscan * nb + 1);
    if (e != cudaSuccess) return e;
    launch_k(k_scan2_reduce<Ld>, dim3(nb, nscan), SCAN_THREADS, 0, s, S, n, sums, nb);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    launch_k(k_scan2_apply<Ld>, dim3(nb, nscan), SCAN_THREADS, 0, s, S, n, sums, nb);
    return cudaGetLastError();
}

}  // namespace

cudaError_t exclusive_scan_u32_sets(int k, const uint32_t *const *in, uint32_t *const *out,
                                    int64_t n, DevArena &scratch, cudaStream_t s) {
    if (k == 1 || n <= 0 || (n + SCAN_TILE - 1) / SCAN_TILE > SCAN_MAX_TILES) {
        for (int i = 0; i < k; ++i) {
            cudaError_t e = exclusive_scan_u32(in[i], out[i], n, nullptr, scratch, s);
            if (e != cudaSuccess) return e;
        }
        return cudaSuccess;
    }
    if (k < 1 || k > SCAN_MAX_SETS) return cudaErrorInvalidValue;
    ScanSets<LoadArr> S{};
    for (int i = 0; i < k; ++i) {
        S.ld[i] = LoadArr{in[i]};
        S.out[i] = out[i];
        S.base[i] = nullptr;
    }
    return scan2(S, k, n, scratch, s);
}

cudaError_t exclusive_scan_u32(const uint32_t *in, uint32_t *out, int64_t n,
                               const uint32_t *base_dev, DevArena &scratch, cudaStream_t s) {
    if (n > 0 && (n + SCAN_TILE - 1) / SCAN_TILE <= SCAN_MAX_TILES &&
        (n + SCAN_TILE - 1) / SCAN_TILE > 1) {
        ScanSets<LoadArr> S{};
        S.ld[0] = LoadArr{in};
        S.out[0] = out;
        S.base[0] = base_dev;
        return scan2(S, 1, n, scratch, s);
    }
    if (n <= 0) {
        // out[0] = base
        if (base_dev)
            return cudaMemcpyAsync(out, base_dev, sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
        return cudaMemsetAsync(out, 0, sizeof(uint32_t), s);
    }
    int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (nb == 1) {
        launch_k(k_scan_apply, 1, SCAN_THREADS, 0, s, in, out, n, nullptr, base_dev);
        return cudaGetLastError();
    }
    uint32_t *sums = nullptr;
    cudaError_t e = arena_alloc(scratch, &sums, (size_t)nb + 1);
    if (e != cudaSuccess) return e;
    launch_k(k_scan_reduce, (unsigned)nb, SCAN_THREADS, 0, s, in, n, sums);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    e = exclusive_scan_u32(sums, sums, nb, base_dev, scratch, s);
    if (e != cudaSuccess) return e;
    launch_k(k_scan_apply, (unsigned)nb, SCAN_THREADS, 0, s, in, out, n, sums, nullptr);
    return cudaGetLastError();
}

// ---------------------------------------------------------------- radix sort
//
// Stable LSD radix sort, 8-bit digits, one or two independent arrays of the
// same length per launch (blockIdx.y).  Per digit: a tile histogram (also
// summed per digit), one block per digit scanning that digit's tile counts
// (tile-major order gives the stable global offsets), and a scatter that
// ranks the tile stably, reorders it by digit in shared memory and writes
// each digit's run of the tile contiguously.

namespace {

constexpr int RS_THREADS = 256;
constexpr int RS_WARPS = RS_THREADS / 32;
constexpr int RS_CHUNKS = 8;  // 32-element chunks per warp
constexpr int RS_TILE = RS_THREADS * RS_CHUNKS;
constexpr int RS_SMEM = RS_TILE * 12 + RS_WARPS * 257 * 4 + 3 * 256 * 4;

struct RsArrays {
    const uint64_t *kin[2];
    const uint32_t *vin[2];
    uint64_t *kout[2];
    uint32_t *vout[2];
};

// counts[(y * 256 + d) * nblocks + b]; totals[y * 256 + d]
__global__ void __launch_bounds__(RS_THREADS)
    k_rs_hist(RsArrays A, int64_t n, int shift, uint32_t *__restrict__ counts,
              uint32_t *__restrict__ totals, int nblocks) {
    pdl_wait();
    __shared__ uint32_t h[256];
    const int y = blockIdx.y;
    const uint64_t *keys = A.kin[y];
    h[threadIdx.x] = 0;
    __syncthreads();
    const int64_t base = (int64_t)blockIdx.x * RS_TILE;
    for (int i = threadIdx.x; i < RS_TILE; i += RS_THREADS) {
        const int64_t k = base + i;
        if (k < n) atomicAdd(&h[(keys[k] >> shift) & 255u], 1u);
    }
    __syncthreads();
    const uint32_t c = h[threadIdx.x];
    counts[((int64_t)y * 256 + threadIdx.x) * nblocks + blockIdx.x] = c;
    if (c) atomicAdd(&totals[y * 256 + threadIdx.x], c);
}

// Block (d, y): offsets of digit d in every tile = (all smaller digits) +
// (digit d in earlier tiles); in place over counts.
__global__ void __launch_bounds__(RS_THREADS)
    k_rs_scan(uint32_t *__restrict__ counts, const uint32_t *__restrict__ totals, int nblocks) {
    pdl_wait();
    const int d = blockIdx.x, y = blockIdx.y;
    uint32_t part = 0;
    if ((int)threadIdx.x < d) part = totals[y * 256 + threadIdx.x];
    uint32_t dummy;
    uint32_t carry = block_exclusive_scan(part, dummy);  // sum of the smaller digits
    uint32_t *c = counts + ((int64_t)y * 256 + d) * nblocks;
    for (int b0 = 0; b0 < nblocks; b0 += RS_THREADS) {
        const int b = b0 + threadIdx.x;
        const uint32_t v = b < nblocks ? c[b] : 0u;
        uint32_t excl;
        const uint32_t tot = block_exclusive_scan(v, excl);
        if (b < nblocks) c[b] = carry + excl;
        carry += tot;
    }
}

// Stable scatter: warp w of a block owns elements [tile + 256 w, tile + 256
// (w+1)), walked in 32-element chunks in order; lanes rank equal digits by
// lane order.  The tile is reordered by digit in shared memory, then written
// out so that consecutive threads write consecutive positions of a digit's run.
__global__ void __launch_bounds__(RS_THREADS)
    k_rs_scatter(RsArrays A, int64_t n, int shift, const uint32_t *__restrict__ offs,
                 int nblocks) {
    pdl_wait();
    extern __shared__ __align__(16) unsigned char rs_sm[];
    uint64_t *skey = reinterpret_cast<uint64_t *>(rs_sm);
    uint32_t *sval = reinterpret_cast<uint32_t *>(skey + RS_TILE);
    uint32_t(*wh)[257] = reinterpret_cast<uint32_t(*)[257]>(sval + RS_TILE);
    uint32_t *lbase = reinterpret_cast<uint32_t *>(wh + RS_WARPS);  // [256] tile-local start
    uint32_t *gbase = lbase + 256;                                 // [256] global start
    uint32_t *cnt = gbase + 256;                                   // [256] tile counts
    const int y = blockIdx.y;
    const uint64_t *kin = A.kin[y];
    const uint32_t *vin = A.vin[y];
    uint64_t *kout = A.kout[y];
    uint32_t *vout = A.vout[y];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < RS_WARPS * 257; i += RS_THREADS) (&wh[0][0])[i] = 0;
    __syncthreads();
    const int64_t tile0 = (int64_t)blockIdx.x * RS_TILE;
    const int64_t w0 = tile0 + warp * (32 * RS_CHUNKS);
    uint64_t k[RS_CHUNKS];
    uint32_t v[RS_CHUNKS];
    int dg[RS_CHUNKS];
#pragma unroll
    for (int c = 0; c < RS_CHUNKS; ++c) {
        const int64_t idx = w0 + c * 32 + lane;
        if (idx < n) {
            k[c] = kin[idx];
            v[c] = vin[idx];
            dg[c] = (int)((k[c] >> shift) & 255u);
        } else {
            k[c] = 0;
            v[c] = 0;
            dg[c] = 256;  // past every digit
        }
    }
    const unsigned lt = (1u << lane) - 1u;
    // lanes holding the same digit (an element past the end holds 256): nine
    // ballots, kept for the placement pass below
    unsigned peers[RS_CHUNKS];
#pragma unroll
    for (int c = 0; c < RS_CHUNKS; ++c) {
        unsigned m = 0xffffffffu;
#pragma unroll
        for (int b = 0; b < 9; ++b) {
            const bool bit = (dg[c] >> b) & 1;
            const unsigned bal = __ballot_sync(0xffffffffu, bit);
            m &= bit ? bal : ~bal;
        }
        peers[c] = m;
        if ((m & lt) == 0) wh[warp][dg[c]] += __popc(m);
        __syncwarp();
    }
    __syncthreads();
    {
        // per digit: the tile count, then each warp's start inside the digit's run
        const int d = threadIdx.x;
        uint32_t run = 0;
        for (int w = 0; w < RS_WARPS; ++w) {
            const uint32_t c = wh[w][d];
            wh[w][d] = run;
            run += c;
        }
        cnt[d] = run;
        gbase[d] = offs[((int64_t)y * 256 + d) * nblocks + blockIdx.x];
    }
    __syncthreads();
    {
        uint32_t excl;
        block_exclusive_scan(cnt[threadIdx.x], excl);
        lbase[threadIdx.x] = excl;
    }
    __syncthreads();
#pragma unroll
    for (int c = 0; c < RS_CHUNKS; ++c) {
        const unsigned m = peers[c];
        if (dg[c] < 256) {
            const uint32_t lp = lbase[dg[c]] + wh[warp][dg[c]] + __popc(m & lt);
            skey[lp] = k[c];
            sval[lp] = v[c];
        }
        __syncwarp();
        if ((m & lt) == 0 && dg[c] < 256) wh[warp][dg[c]] += __popc(m);
        __syncwarp();
    }
    __syncthreads();
    const int nt = (n - tile0 < RS_TILE) ? (int)(n - tile0) : RS_TILE;
    for (int lp = threadIdx.x; lp < nt; lp += RS_THREADS) {
        const uint64_t kk = skey[lp];
        const int d = (int)((kk >> shift) & 255u);
        const uint32_t g = gbase[d] + (uint32_t)lp - lbase[d];
        kout[g] = kk;
        vout[g] = sval[lp];
    }
}

cudaError_t radix_sort_multi(int nsort, uint64_t **keys, uint32_t **vals, uint64_t **keys_alt,
                             uint32_t **vals_alt, int64_t n, uint32_t digit_mask,
                             DevArena &scratch, cudaStream_t s) {
    if (n <= 1 || digit_mask == 0) return cudaSuccess;
    const int nblocks = (int)((n + RS_TILE - 1) / RS_TILE);
    int ndig = 0;
    for (int d = 0; d < 8; ++d) ndig += (digit_mask >> d) & 1u;
    uint32_t *counts = nullptr, *totals = nullptr;
    cudaError_t e = arena_alloc(scratch, &counts, (size_t)nsort * 256 * nblocks + 1);
    if (e == cudaSuccess) e = arena_alloc(scratch, &totals, (size_t)ndig * nsort * 256);
    if (e == cudaSuccess) e = cudaMemsetAsync(totals, 0, (size_t)ndig * nsort * 256 * 4, s);
    if (e != cudaSuccess) return e;
    static const cudaError_t attr = cudaFuncSetAttribute(
        k_rs_scatter, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM);
    if (attr != cudaSuccess) return attr;
    RsArrays A{};
    uint64_t *ka[2], *kb[2];
    uint32_t *va[2], *vb[2];
    for (int y = 0; y < nsort; ++y) {
        ka[y] = keys[y];
        kb[y] = keys_alt[y];
        va[y] = vals[y];
        vb[y] = vals_alt[y];
    }
    const dim3 grid(nblocks, nsort);
    int di = 0;
    for (int shift = 0; shift < 64; shift += 8) {
        if (!((digit_mask >> (shift / 8)) & 1u)) continue;
        for (int y = 0; y < nsort; ++y) {
            A.kin[y] = ka[y];
            A.vin[y] = va[y];
            A.kout[y] = kb[y];
            A.vout[y] = vb[y];
        }
        uint32_t *tot = totals + (size_t)di * nsort * 256;
        launch_k(k_rs_hist, grid, RS_THREADS, 0, s, A, n, shift, counts, tot, nblocks);
        launch_k(k_rs_scan, dim3(256, nsort), RS_THREADS, 0, s, counts, tot, nblocks);
        launch_k(k_rs_scatter, grid, RS_THREADS, RS_SMEM, s, A, n, shift, counts, nblocks);
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        for (int y = 0; y < nsort; ++y) {
            std::swap(ka[y], kb[y]);
            std::swap(va[y], vb[y]);
        }
        ++di;
    }
    for (int y = 0; y < nsort; ++y) {
        keys[y] = ka[y];
        vals[y] = va[y];
    }
    return cudaSuccess;
}

}  // namespace

cudaError_t radix_sort_pairs(uint64_t **keys, uint32_t **vals, uint64_t *keys_alt,
                             uint32_t *vals_alt, int64_t n, uint32_t digit_mask,
                             DevArena &scratch, cudaStream_t s) {
    uint64_t *kalt[1] = {keys_alt};
    uint32_t *valt[1] = {vals_alt};
    return radix_sort_multi(1, keys, vals, kalt, valt, n, digit_mask, scratch, s);
}

cudaError_t radix_sort_pairs2(uint64_t **keys, uint32_t **vals, uint64_t **keys_alt,
                              uint32_t **vals_alt, int64_t n, uint32_t digit_mask,
                              DevArena &scratch, cudaStream_t s) {
    return radix_sort_multi(2, keys, vals, keys_alt, vals_alt, n, digit_mask, scratch, s);
}

}  // namespace gbfmm
