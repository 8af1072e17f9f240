// fp_eval.cu -- findpts_eval (Sec. 2.1): interpolate F nodal fields at located
// points by sum factorisation, out[f][p] = sum_ijk F_ijk h_i(r) h_j(s) h_k(t),
// in FP64; quiet NaN for points that were not found.
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

template <int n>
__global__ void __launch_bounds__(128) k_eval(EvalArgs A, BasisTab tab)
{
    constexpr int n3 = n * n * n;
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= A.P) return;
    const int e = A.elem[p];
    if (A.code[p] == FP_CODE_NOT_FOUND || e < 0 || e >= A.E) {
        for (int f = 0; f < A.F; ++f) A.out[(int64_t)f * A.P + p] = __longlong_as_double(0x7ff8000000000000ULL);
        return;
    }
    double hr[n], hs[n], ht[n];
    lagrange_h<n, double>(tab.xi, tab.ci, A.rst[p], hr);
    lagrange_h<n, double>(tab.xi, tab.ci, A.rst[A.P + p], hs);
    lagrange_h<n, double>(tab.xi, tab.ci, A.rst[2 * A.P + p], ht);
    for (int f = 0; f < A.F; ++f)
        A.out[(int64_t)f * A.P + p] = contract<n, double>(A.fields + ((int64_t)f * A.E + e) * n3, hr, hs, ht);
}

cudaError_t launch_eval(int n, int64_t E, int64_t P, const int32_t* code, const int32_t* elem, const double* rst,
                        int F, const double* fields, double* out, const BasisTab& tab, cudaStream_t s)
{
    if (P == 0) return cudaSuccess;
    EvalArgs a{E, P, code, elem, rst, F, fields, out};
    const unsigned grid = (unsigned)((P + 127) / 128);
    switch (n) {
#define FP_CASE(NN) \
    case NN: k_eval<NN><<<grid, 128, 0, s>>>(a, tab); break;
        FP_CASE(2) FP_CASE(3) FP_CASE(4) FP_CASE(5) FP_CASE(6) FP_CASE(7) FP_CASE(8) FP_CASE(9)
        FP_CASE(10) FP_CASE(11) FP_CASE(12) FP_CASE(13) FP_CASE(14) FP_CASE(15) FP_CASE(16)
#undef FP_CASE
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

}  // namespace fpg
