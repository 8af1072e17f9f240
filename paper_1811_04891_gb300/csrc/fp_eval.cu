// fp_eval.cu -- findpts_eval (Sec. 2.1): interpolate F nodal fields at located
// points by sum factorisation, out[f][p] = sum_ijk F_ijk h_i(r) h_j(s) h_k(t),
// in FP64; quiet NaN for points that were not found.
#include <algorithm>
#include <climits>

#include "fp_common.cuh"
#include "fp_internal.h"

namespace fpg {

struct EvalArgs {
    int64_t E;
    int64_t P;
    const int32_t* code;
    const int32_t* elem;
    const double* rst;
    int F;
    const double* fields;
    double* out;
};

// One thread per point, or (SPLIT) one thread per (point, field): small
// calls (an interface sub-iteration evaluates a few 10^4 points) are
// latency-bound, and splitting the fields gives F times the threads; each
// field's operations are the same either way.
template <int n, bool SPLIT>
__global__ void __launch_bounds__(128) k_eval(EvalArgs A, BasisTab tab)
{
    constexpr int n3 = n * n * n;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t p = SPLIT ? t / A.F : t;
    if (p >= A.P) return;
    const int f0 = SPLIT ? (int)(t % A.F) : 0, f1 = SPLIT ? f0 + 1 : A.F;
    const int e = A.elem[p];
    if (A.code[p] == FP_CODE_NOT_FOUND || e < 0 || e >= A.E) {
        for (int f = f0; f < f1; ++f) A.out[(int64_t)f * A.P + p] = __longlong_as_double(0x7ff8000000000000ULL);
        return;
    }
    double hr[n], hs[n], ht[n];
    lagrange_h<n, double>(tab.xi, tab.ci, A.rst[p], hr);
    lagrange_h<n, double>(tab.xi, tab.ci, A.rst[A.P + p], hs);
    lagrange_h<n, double>(tab.xi, tab.ci, A.rst[2 * A.P + p], ht);
    for (int f = f0; f < f1; ++f)
        A.out[(int64_t)f * A.P + p] = contract<n, double>(A.fields + ((int64_t)f * A.E + e) * n3, hr, hs, ht);
}

// calls with at most this many (point, field) values take one thread each
constexpr int64_t kSplitEval = int64_t(1) << 21;

cudaError_t launch_eval(int n, int64_t E, int64_t P, const int32_t* code, const int32_t* elem, const double* rst,
                        int F, const double* fields, double* out, const BasisTab& tab, cudaStream_t s)
{
    if (P == 0) return cudaSuccess;
    EvalArgs a{E, P, code, elem, rst, F, fields, out};
    const bool split = P * F <= kSplitEval;
    const unsigned grid = (unsigned)(((split ? P * F : P) + 127) / 128);
    switch (n) {
#define FP_CASE(NN)                                                  \
    case NN:                                                         \
        if (split) k_eval<NN, true><<<grid, 128, 0, s>>>(a, tab);    \
        else k_eval<NN, false><<<grid, 128, 0, s>>>(a, tab);         \
        break;
        FP_CASE(2) FP_CASE(3) FP_CASE(4) FP_CASE(5) FP_CASE(6) FP_CASE(7) FP_CASE(8) FP_CASE(9)
        FP_CASE(10) FP_CASE(11) FP_CASE(12) FP_CASE(13) FP_CASE(14) FP_CASE(15) FP_CASE(16)
#undef FP_CASE
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace fpg

// ---------------------------------------------------------------------------
// Double-float evaluation for the mixed form.
//
// Every nodal value f is posted once as an unevaluated sum of two floats,
// f = f_hi + f_lo (f_hi = fl(f), f_lo = fl(f - f_hi), 48 significant bits),
// and each basis value h(r), computed in FP64, is split the same way.  The
// contraction then runs on the FP32 pipes: each product f*h is formed exactly
// in its leading part (p = f_hi*h_hi, e = fma(f_hi, h_hi, -p)) plus the
// first-order cross terms, and the sum is carried as a (hi, lo) pair with an
// error-free two-sum.  The result is rounded to FP64 at the end.  Relative
// error is a few units of 2^-48 times the sum of |terms|.
// ---------------------------------------------------------------------------
namespace fpg {

struct Eval2Args {
    int64_t E;
    int64_t P;
    const int32_t* code;
    const int32_t* elem;
    const double* rst;
    int F;
    const float2* fields;     // [F][E][n3] posted: per row n high parts, then n low parts
    double* out;
};

template <int n, bool SPLIT>
__global__ void __launch_bounds__(128) k_eval_df(Eval2Args A, BasisTab tab)
{
    constexpr int n3 = n * n * n;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t p = SPLIT ? t / A.F : t;
    if (p >= A.P) return;
    const int f0 = SPLIT ? (int)(t % A.F) : 0, f1 = SPLIT ? f0 + 1 : A.F;
    const int e = A.elem[p];
    if (A.code[p] == FP_CODE_NOT_FOUND || A.code[p] == FP_CODE_RETRY || e < 0 || e >= A.E) {
        for (int f = f0; f < f1; ++f) A.out[(int64_t)f * A.P + p] = __longlong_as_double(0x7ff8000000000000ULL);
        return;
    }
    double hr[n], hs[n], ht[n];
    lagrange_h<n, double>(tab.xi, tab.ci, A.rst[p], hr);
    lagrange_h<n, double>(tab.xi, tab.ci, A.rst[A.P + p], hs);
    lagrange_h<n, double>(tab.xi, tab.ci, A.rst[2 * A.P + p], ht);
    float rh[n], rl[n], sh[n], sl[n], th[n], tl[n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
        df a = df_split(hr[i]), b = df_split(hs[i]), c = df_split(ht[i]);
        rh[i] = a.hi; rl[i] = a.lo; sh[i] = b.hi; sl[i] = b.lo; th[i] = c.hi; tl[i] = c.lo;
    }
    for (int f = f0; f < f1; ++f)
        A.out[(int64_t)f * A.P + p] = contract_df<n>(A.fields + ((int64_t)f * A.E + e) * n3, rh, rl, sh, sl, th, tl);
}

// ---- posted points: the split basis values of located points, computed once
// and reused by every evaluation at the same (e, r) (the interface points of
// a Schwarz step are evaluated once per sub-iteration).  Layout [6n][P]:
// rh, rl, sh, sl, th, tl, each n rows, so consecutive threads load
// consecutive words; elem = -1 marks points without a value.
template <int n>
__global__ void k_points_basis(int64_t P, const int32_t* __restrict__ code, const int32_t* __restrict__ elem,
                               const double* __restrict__ rst, float* __restrict__ basis, int32_t* __restrict__ pe,
                               BasisTab tab)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= P) return;
    const bool ok = !(code[p] == FP_CODE_NOT_FOUND || code[p] == FP_CODE_RETRY || elem[p] < 0);
    pe[p] = ok ? elem[p] : -1;
    if (!ok) return;
    double h[n];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
        lagrange_h<n, double>(tab.xi, tab.ci, rst[d * P + p], h);
#pragma unroll
        for (int i = 0; i < n; ++i) {
            const df v = df_split(h[i]);
            basis[((int64_t)(2 * d) * n + i) * P + p] = v.hi;
            basis[((int64_t)(2 * d + 1) * n + i) * P + p] = v.lo;
        }
    }
}

template <int n>
__global__ void __launch_bounds__(128) k_eval_points_df(int64_t E, int64_t P, int F, const int32_t* __restrict__ pe,
                                                        const float* __restrict__ basis,
                                                        const float2* __restrict__ fields, double* __restrict__ out)
{
    constexpr int n3 = n * n * n;
    const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t p = t / F;
    if (p >= P) return;
    const int f = (int)(t % F);
    const int e = pe[p];
    if (e < 0 || e >= E) {
        out[(int64_t)f * P + p] = __longlong_as_double(0x7ff8000000000000ULL);
        return;
    }
    float rh[n], rl[n], sh[n], sl[n], th[n], tl[n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
        rh[i] = __ldg(basis + (int64_t)(0 * n + i) * P + p);
        rl[i] = __ldg(basis + (int64_t)(1 * n + i) * P + p);
        sh[i] = __ldg(basis + (int64_t)(2 * n + i) * P + p);
        sl[i] = __ldg(basis + (int64_t)(3 * n + i) * P + p);
        th[i] = __ldg(basis + (int64_t)(4 * n + i) * P + p);
        tl[i] = __ldg(basis + (int64_t)(5 * n + i) * P + p);
    }
    out[(int64_t)f * P + p] = contract_df<n>(fields + ((int64_t)f * E + e) * n3, rh, rl, sh, sl, th, tl);
}

// posted fields: value v -> (hi, lo) = (fl32(v), fl32(v - hi)), each row of
// n nodes stored as its n high parts then its n low parts (see row_df)
__global__ void k_split_df(int64_t count, int n, const double* __restrict__ src, float2* __restrict__ dst)
{
    float* d = reinterpret_cast<float*>(dst);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < count; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t row = i / n, c = i - row * n;
        const double v = src[i];
        const float h = (float)v;
        d[2 * n * row + c] = h;
        d[2 * n * row + n + c] = (float)(v - (double)h);
    }
}

cudaError_t launch_split_df(int64_t count, int n, const double* src, float2* dst, cudaStream_t s)
{
    const int64_t blocks = std::min<int64_t>((count + 255) / 256, 152 * 32);
    k_split_df<<<(unsigned)std::max<int64_t>(blocks, 1), 256, 0, s>>>(count, n, src, dst);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_points_basis(int n, int64_t P, const int32_t* code, const int32_t* elem, const double* rst,
                                float* basis, int32_t* pe, const BasisTab& tab, cudaStream_t s)
{
    if (P == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((P + 127) / 128);
    switch (n) {
#define FP_CASE(NN) \
    case NN: k_points_basis<NN><<<grid, 128, 0, s>>>(P, code, elem, rst, basis, pe, tab); break;
        FP_CASE(2) FP_CASE(3) FP_CASE(4) FP_CASE(5) FP_CASE(6) FP_CASE(7) FP_CASE(8) FP_CASE(9)
        FP_CASE(10) FP_CASE(11) FP_CASE(12) FP_CASE(13) FP_CASE(14) FP_CASE(15) FP_CASE(16)
#undef FP_CASE
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_eval_points_df(int n, int64_t E, int64_t P, int F, const int32_t* pe, const float* basis,
                                  const float2* fields, double* out, cudaStream_t s)
{
    if (P == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((P * F + 127) / 128);
    switch (n) {
#define FP_CASE(NN) \
    case NN: k_eval_points_df<NN><<<grid, 128, 0, s>>>(E, P, F, pe, basis, fields, out); break;
        FP_CASE(2) FP_CASE(3) FP_CASE(4) FP_CASE(5) FP_CASE(6) FP_CASE(7) FP_CASE(8) FP_CASE(9)
        FP_CASE(10) FP_CASE(11) FP_CASE(12) FP_CASE(13) FP_CASE(14) FP_CASE(15) FP_CASE(16)
#undef FP_CASE
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_eval_df(int n, int64_t E, int64_t P, const int32_t* code, const int32_t* elem, const double* rst,
                           int F, const float2* fields, double* out, const BasisTab& tab, cudaStream_t s)
{
    if (P == 0) return cudaSuccess;
    Eval2Args a{E, P, code, elem, rst, F, fields, out};
    const bool split = P * F <= kSplitEval;
    const unsigned grid = (unsigned)(((split ? P * F : P) + 127) / 128);
    switch (n) {
#define FP_CASE(NN)                                                     \
    case NN:                                                            \
        if (split) k_eval_df<NN, true><<<grid, 128, 0, s>>>(a, tab);    \
        else k_eval_df<NN, false><<<grid, 128, 0, s>>>(a, tab);         \
        break;
        FP_CASE(2) FP_CASE(3) FP_CASE(4) FP_CASE(5) FP_CASE(6) FP_CASE(7) FP_CASE(8) FP_CASE(9)
        FP_CASE(10) FP_CASE(11) FP_CASE(12) FP_CASE(13) FP_CASE(14) FP_CASE(15) FP_CASE(16)
#undef FP_CASE
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace fpg

// ---------------------------------------------------------------------------
// Fused evaluation in the element-sorted pair order of the find (one thread
// per winning pair; neighbouring threads work on the same element, so its
// field rows are served from L1 instead of being re-read from DRAM).
// ---------------------------------------------------------------------------
namespace fpg {

template <int n>
__device__ __forceinline__ void eval_point_f64(const double* __restrict__ F64, int64_t E, int F, int e, double r0,
                                               double r1, double r2, const BasisTab& tab, double* __restrict__ out,
                                               int64_t P, int64_t p)
{
    constexpr int n3 = n * n * n;
    double hr[n], hs[n], ht[n];
    lagrange_h<n, double>(tab.xi, tab.ci, r0, hr);
    lagrange_h<n, double>(tab.xi, tab.ci, r1, hs);
    lagrange_h<n, double>(tab.xi, tab.ci, r2, ht);
    for (int f = 0; f < F; ++f)
        out[(int64_t)f * P + p] = contract<n, double>(F64 + ((int64_t)f * E + e) * n3, hr, hs, ht);
}

template <int n>
__device__ __forceinline__ void eval_point_df(const float2* __restrict__ Fdf, int64_t E, int F, int e, double r0,
                                              double r1, double r2, const BasisTab& tab, double* __restrict__ out,
                                              int64_t P, int64_t p)
{
    constexpr int n3 = n * n * n;
    double hr[n], hs[n], ht[n];
    lagrange_h<n, double>(tab.xi, tab.ci, r0, hr);
    lagrange_h<n, double>(tab.xi, tab.ci, r1, hs);
    lagrange_h<n, double>(tab.xi, tab.ci, r2, ht);
    float rh[n], rl[n], sh[n], sl[n], th[n], tl[n];
#pragma unroll
    for (int i = 0; i < n; ++i) {
        df a = df_split(hr[i]), b = df_split(hs[i]), c = df_split(ht[i]);
        rh[i] = a.hi; rl[i] = a.lo; sh[i] = b.hi; sl[i] = b.lo; th[i] = c.hi; tl[i] = c.lo;
    }
    for (int f = 0; f < F; ++f)
        out[(int64_t)f * P + p] = contract_df<n>(Fdf + ((int64_t)f * E + e) * n3, rh, rl, sh, sl, th, tl);
}

struct EvalPairsArgs {
    int64_t E, P, cap;
    const int32_t* dcount;
    const int32_t* order;
    const int32_t* pair_elem;
    const int32_t* pair_pt;
    const double* prst;
    EvalSpec ev;
    const int32_t* s_lo;      // batch groups: the group's sorted positions [*s_lo, *s_hi)
    const int32_t* s_hi;
    int32_t ebase;            // batch groups: subtracted from pair_elem
    int walk;                 // pair results at sorted positions (else at pair slots)
};

template <int n, bool DF>
__global__ void __launch_bounds__(128) k_eval_pairs(EvalPairsArgs A, BasisTab tab)
{
    int64_t s0 = 0, s1;
    if (A.s_lo) {
        s0 = *A.s_lo;
        s1 = *A.s_hi;
    } else {
        const int64_t t = *A.dcount;
        s1 = t < A.cap ? t : A.cap;
    }
    for (int64_t s = s0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < s1; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = A.order[s];
        const int32_t p = A.pair_pt[q];
        if (p < 0) continue;                              // not the point's winning pair
        const int e = A.pair_elem[q] - A.ebase;
        const int64_t w = A.walk ? s : q;
        const double r0 = A.prst[w], r1 = A.prst[A.cap + w], r2 = A.prst[2 * A.cap + w];
        if (DF)
            eval_point_df<n>(A.ev.fdf, A.E, A.ev.F, e, r0, r1, r2, tab, A.ev.out, A.P, p);
        else
            eval_point_f64<n>(A.ev.f64, A.E, A.ev.F, e, r0, r1, r2, tab, A.ev.out, A.P, p);
    }
}

// Fused double-float evaluation with each element's posted fields staged in
// shared memory: a block takes kStageTile consecutive sorted pairs (the pairs
// of one element are consecutive), copies the fields of each element the
// tile touches into shared memory once, in ascending element order, and the
// threads whose pairs lie in that element read their rows from there.
constexpr int kStageTile = 128;

template <int n>
__global__ void __launch_bounds__(kStageTile) k_eval_pairs_staged(EvalPairsArgs A, BasisTab tab)
{
    constexpr int n3 = n * n * n;
    extern __shared__ float4 stage4[];               // F * n3 float2: the current element's fields
    float2* stage = reinterpret_cast<float2*>(stage4);
    __shared__ int ecur;
    int64_t s0 = 0, s1;
    if (A.s_lo) {
        s0 = *A.s_lo;
        s1 = *A.s_hi;
    } else {
        const int64_t t = *A.dcount;
        s1 = t < A.cap ? t : A.cap;
    }
    const int F = A.ev.F;
    for (int64_t base = s0 + (int64_t)blockIdx.x * kStageTile; base < s1;
         base += (int64_t)gridDim.x * kStageTile) {
        const int64_t s = base + threadIdx.x;
        int32_t p = -1;
        int e = -1;
        float rh[n], rl[n], sh[n], sl[n], th[n], tl[n];
        if (s < s1) {
            const int32_t q = A.order[s];
            p = A.pair_pt[q];
            e = A.pair_elem[q] - A.ebase;
            if (p >= 0) {
                const int64_t w = A.walk ? s : q;
                double hr[n], hs[n], ht[n];
                lagrange_h<n, double>(tab.xi, tab.ci, A.prst[w], hr);
                lagrange_h<n, double>(tab.xi, tab.ci, A.prst[A.cap + w], hs);
                lagrange_h<n, double>(tab.xi, tab.ci, A.prst[2 * A.cap + w], ht);
#pragma unroll
                for (int i = 0; i < n; ++i) {
                    const df a = df_split(hr[i]), b = df_split(hs[i]), c = df_split(ht[i]);
                    rh[i] = a.hi; rl[i] = a.lo; sh[i] = b.hi; sl[i] = b.lo; th[i] = c.hi; tl[i] = c.lo;
                }
            }
        }
        bool done = p < 0;                           // losers and threads past the end have nothing to do
        for (;;) {
            if (threadIdx.x == 0) ecur = INT_MAX;
            __syncthreads();
            if (!done) atomicMin(&ecur, e);
            __syncthreads();
            const int ec = ecur;
            if (ec == INT_MAX) break;                // uniform: every thread read the same value
            for (int f = 0; f < F; ++f) {
                const float2* src = A.ev.fdf + ((int64_t)f * A.E + ec) * n3;
                if constexpr (n3 % 2 == 0) {
                    const float4* s4 = reinterpret_cast<const float4*>(src);
                    float4* d4 = stage4 + f * (n3 / 2);
                    for (int v = threadIdx.x; v < n3 / 2; v += kStageTile) d4[v] = __ldg(s4 + v);
                } else {
                    for (int v = threadIdx.x; v < n3; v += kStageTile) stage[f * n3 + v] = __ldg(src + v);
                }
            }
            __syncthreads();
            if (!done && e == ec) {
                for (int f = 0; f < F; ++f)
                    A.ev.out[(int64_t)f * A.P + p] = contract_df<n, true>(stage + f * n3, rh, rl, sh, sl, th, tl);
                done = true;
            }
            __syncthreads();                         // the next element overwrites the stage
        }
    }
}

// staging is used when one element's posted fields fit in this much shared
// memory (larger ones are evaluated from L1 / L2 as without staging)
constexpr int64_t kStageMaxBytes = 48 * 1024;

cudaError_t launch_eval_pairs(int n, int64_t E, int64_t P, const int32_t* dcount, int64_t cap, const int32_t* order,
                              const int32_t* pair_elem, const int32_t* pair_pt, const double* prst,
                              const EvalSpec& ev, const BasisTab& tab, unsigned grid, cudaStream_t s,
                              const int32_t* s_lo, const int32_t* s_hi, int32_t ebase, bool walk)
{
    EvalPairsArgs a{E, P, cap, dcount, order, pair_elem, pair_pt, prst, ev, s_lo, s_hi, ebase, walk ? 1 : 0};
    const bool df = ev.fdf != nullptr;
    const int64_t stage_bytes = (int64_t)ev.F * n * n * n * (int64_t)sizeof(float2);
    const bool staged = df && ev.staged && stage_bytes <= kStageMaxBytes;
    switch (n) {
#define FP_CASE(NN)                                                                       \
    case NN:                                                                              \
        if (staged) k_eval_pairs_staged<NN><<<grid, kStageTile, stage_bytes, s>>>(a, tab); \
        else if (df) k_eval_pairs<NN, true><<<grid, 128, 0, s>>>(a, tab);                 \
        else k_eval_pairs<NN, false><<<grid, 128, 0, s>>>(a, tab);                        \
        break;
        FP_CASE(2) FP_CASE(3) FP_CASE(4) FP_CASE(5) FP_CASE(6) FP_CASE(7) FP_CASE(8) FP_CASE(9)
        FP_CASE(10) FP_CASE(11) FP_CASE(12) FP_CASE(13) FP_CASE(14) FP_CASE(15) FP_CASE(16)
#undef FP_CASE
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace fpg
