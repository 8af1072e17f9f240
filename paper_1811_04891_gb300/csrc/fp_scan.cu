// fp_scan.cu -- device-wide exclusive prefix sum of int32 counts (offsets of
// the pair stream, the hash-cell lists and the per-element pair buckets).
// Three phases per level: block-local scans with per-block totals, a
// recursive scan of the totals, and a uniform add.
#include <cuda_runtime.h>
#include <stdint.h>

#include "fp_internal.h"

namespace fpg {

constexpr int SCAN_THREADS = 512;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

// exclusive scan of one tile; writes out[i] for i < n and the tile total
__global__ void __launch_bounds__(SCAN_THREADS) k_scan_tile(const int32_t* __restrict__ in, int32_t* __restrict__ out,
                                                           int32_t* __restrict__ totals, int64_t n)
{
    __shared__ int32_t warp_sums[SCAN_THREADS / 32];
    const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int32_t v[SCAN_ITEMS];
    int32_t sum = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        sum += v[i];
    }
    // inclusive warp scan of per-thread sums
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int32_t x = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int32_t w = (lane < SCAN_THREADS / 32) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int32_t y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < SCAN_THREADS / 32) warp_sums[lane] = w;
    }
    __syncthreads();
    int32_t run = x - sum + (warp > 0 ? warp_sums[warp - 1] : 0);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < n) out[base + i] = run;
        run += v[i];
    }
    if (threadIdx.x == SCAN_THREADS - 1) totals[blockIdx.x] = run;
}

__global__ void k_scan_add(int32_t* __restrict__ out, const int32_t* __restrict__ prefix, int64_t n)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += prefix[i / SCAN_TILE];
}

__global__ void k_scan_total(int32_t* __restrict__ out, const int32_t* __restrict__ in, int64_t n)
{
    // out[n] = out[n-1] + in[n-1]  (n >= 1), or 0
    out[n] = n > 0 ? out[n - 1] + in[n - 1] : 0;
}

int64_t scan_tmp_elems(int64_t n)
{
    int64_t t = 0;
    int64_t m = n;
    while (m > SCAN_TILE) {
        m = (m + SCAN_TILE - 1) / SCAN_TILE;
        t += 2 * (m + 1);
    }
    return t + 2 * (SCAN_TILE + 1);
}

// out[0..n) exclusive prefix, out[n] total; tmp per scan_tmp_elems
static cudaError_t scan_rec(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, cudaStream_t s)
{
    if (n <= 0) return cudaSuccess;
    const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
    int32_t* totals = tmp;
    int32_t* prefix = tmp + (nb + 1);
    k_scan_tile<<<(unsigned)nb, SCAN_THREADS, 0, s>>>(in, out, totals, n);
    count_launch();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || nb == 1) return err;
    err = scan_rec(totals, prefix, nb, tmp + 2 * (nb + 1), s);
    if (err != cudaSuccess) return err;
    k_scan_add<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(out, prefix, n);
    count_launch();
    return cudaGetLastError();
}

cudaError_t scan_exclusive(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, cudaStream_t s)
{
    cudaError_t err = scan_rec(in, out, n, tmp, s);
    if (err != cudaSuccess) return err;
    k_scan_total<<<1, 1, 0, s>>>(out, in, n);
    count_launch();
    return cudaGetLastError();
}

}  // namespace fpg
