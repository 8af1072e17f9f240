// fp_probe.cu -- arithmetic peak probes for the roofline of the Newton and
// eval kernels.
//
// The location stage is bound by arithmetic, not by HBM: its roofline needs
// the FP64 and FP32 multiply-add rates of this GPU, and the rate of the
// double-float multiply-add (df_fma_acc) that the mixed form uses for its
// FP64-accuracy work on the FP32 pipes.  Each probe launches a full,
// persistent grid (blocks_per_sm blocks of 256 threads on every SM); every
// thread runs kChains independent dependency chains of `iters` steps, so
// the pipes see enough independent work to hide their latency.  A step is
//   FP64:  x = fma(x, a, b)                     (2 flops)
//   FP32:  x = fmaf(x, a, b)                    (2 flops)
//   DF:    x = c + x * a in double-float        (counted as 2 FP64-class flops)
//   FP32x2: packed pair fma on a float2          (4 flops)
//   DFx2:  two DF steps in packed pairs (df2_fma_acc, 4 FP64-class flops)
// The multiplier a is just below 1 and the addend small, so no chain
// overflows or underflows.  Each thread stores the sum of its chains, so no
// step can be optimised away.  Each probe uses the operand form that
// measured fastest: the FP64 probe takes a and the addend as per-thread
// register values (perturbed by the thread index below their last bit) --
// straight from the kernel parameters, as operands common to the warp, it
// measured 16 % slower (1.06 against 1.26 TFLOP/s); the FP32 and
// double-float probes take them from the parameters (with register operands
// they measured 3-13 % slower).
#include "fp_common.cuh"
#include "fp_internal.h"

namespace fpg {

constexpr int kChains = 8;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads) k_probe_f64(int64_t iters, double a0, double b0, double* sink)
{
    const double a = a0 + (double)(threadIdx.x & 7) * 1e-17, b = b0 + (double)(threadIdx.x & 3) * 1e-19;
    double x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (double)(threadIdx.x + c);
#pragma unroll 4
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fma(x[c], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_f32(int64_t iters, float a, float b, double* sink)
{
    float x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = (float)(threadIdx.x + c);
#pragma unroll 4
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = fmaf(x[c], a, b);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c];
    sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = (double)s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_df(int64_t iters, float ah, float al, float ch, float cl,
                                                           double* sink)
{
    df x[kChains];
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = {(float)(threadIdx.x + c), 0.0f};
#pragma unroll 2
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) {
            df acc = {ch, cl};
            df_fma_acc(acc, x[c], ah, al);
            x[c] = acc;
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += (double)x[c].hi + (double)x[c].lo;
    sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_f32x2(int64_t iters, float a, float b, double* sink)
{
    float2 x[kChains];
    const float2 a2 = make_float2(a, a), b2 = make_float2(b, b);
#pragma unroll
    for (int c = 0; c < kChains; ++c) x[c] = make_float2((float)(threadIdx.x + c), (float)(threadIdx.x + c + 1));
#pragma unroll 4
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kChains; ++c) x[c] = __ffma2_rn(x[c], a2, b2);
    }
    float s = 0.0f;
#pragma unroll
    for (int c = 0; c < kChains; ++c) s += x[c].x + x[c].y;
    sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = (double)s;
}

__global__ void __launch_bounds__(kProbeThreads) k_probe_df2(int64_t iters, float ah, float al, float ch, float cl,
                                                            double* sink)
{
    constexpr int kPairs = kChains / 2;
    df2 x[kPairs];
    const float2 ah2 = make_float2(ah, ah), al2 = make_float2(al, al);
#pragma unroll
    for (int c = 0; c < kPairs; ++c)
        x[c] = {make_float2((float)(threadIdx.x + 2 * c), (float)(threadIdx.x + 2 * c + 1)), make_float2(0.0f, 0.0f)};
#pragma unroll 2
    for (int64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < kPairs; ++c) {
            df2 acc = {make_float2(ch, ch), make_float2(cl, cl)};
            df2_fma_acc(acc, x[c].hi, x[c].lo, ah2, al2);
            x[c] = acc;
        }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < kPairs; ++c)
        s += (double)x[c].hi.x + (double)x[c].lo.x + (double)x[c].hi.y + (double)x[c].lo.y;
    sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = s;
}

}  // namespace fpg

extern "C" fp_status fp_fma_probe(int kind, int64_t iters, int blocks_per_sm, double* sink, double* flops,
                                  void* stream)
{
    using namespace fpg;
    if (kind < 0 || kind > 4 || iters < 1 || blocks_per_sm < 1 || blocks_per_sm > 8 || !sink)
        return FP_ERR_INVALID_ARG;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return FP_ERR_CUDA;
    const unsigned grid = (unsigned)(sms * blocks_per_sm);
    cudaStream_t s = (cudaStream_t)stream;
    if (kind == 0)
        k_probe_f64<<<grid, kProbeThreads, 0, s>>>(iters, 0.9999999, 1e-7, sink);
    else if (kind == 1)
        k_probe_f32<<<grid, kProbeThreads, 0, s>>>(iters, 0.9999f, 1e-4f, sink);
    else if (kind == 3)
        k_probe_f32x2<<<grid, kProbeThreads, 0, s>>>(iters, 0.9999f, 1e-4f, sink);
    else {
        const double a = 0.99999999, c = 1e-8;
        const float ah = (float)a, ch = (float)c;
        const float al = (float)(a - (double)ah), cl = (float)(c - (double)ch);
        if (kind == 2) k_probe_df<<<grid, kProbeThreads, 0, s>>>(iters, ah, al, ch, cl, sink);
        else k_probe_df2<<<grid, kProbeThreads, 0, s>>>(iters, ah, al, ch, cl, sink);
    }
    count_launch();
    if (cudaGetLastError() != cudaSuccess) return FP_ERR_CUDA;
    if (flops) *flops = (kind == 3 ? 4.0 : 2.0) * kChains * (double)iters * grid * kProbeThreads;
    return FP_OK;
}

extern "C" int64_t fp_probe_threads(int blocks_per_sm)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return -1;
    return (int64_t)sms * blocks_per_sm * fpg::kProbeThreads;
}
