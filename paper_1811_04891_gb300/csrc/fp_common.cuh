// fp_common.cuh -- internal types and device building blocks shared by the
// library's translation units (never by the CPU oracle).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/findpts_gb.h"

namespace fpg {

constexpr int NMAX = 16;   // GLL points per direction, N <= 15

// Lagrange data on the GLL points of one order: abscissae xi and the
// normalisers ci = 1 / prod_{m != i} (xi_i - xi_m).  Passed by value as a
// kernel argument, so every read is a uniform constant-bank load.
struct BasisTab {
    double xi[NMAX];
    double ci[NMAX];
    float xif[NMAX];
    float cif[NMAX];
    float xil[NMAX];    // low parts: xi = xif + xil, ci = cif + cil to about 48 bits
    float cil[NMAX];
};

// Per-element search data (FP64), built once by the hull kernel.
struct ElemBox {
    double c[3];        // frame origin (mean of the 8 vertices)
    double Ai[9];       // y = Ai (x - c): inverse of the vertex-averaged affine frame
    double olo[3];      // bounds of y over the element (Bernstein hull) minus pad
    double ohi[3];      //   ... plus pad
    double blo[3];      // axis-aligned Bernstein-hull bounds minus pad
    double bhi[3];      //   ... plus pad
    double he;          // diagonal of the axis box spanned by the element's nodes
    double spare;
};

// FP32 copy of ElemBox for the mixed form's screen, rounded outward with
// margins that cover the FP32 evaluation of the tests (never tighter than
// the FP64 boxes).
struct ElemBox32 {
    float c[3];
    float Ai[9];
    float olo[3], ohi[3];
    float blo[3], bhi[3];
};

struct HashGrid {
    double org[3];
    double inv[3];      // 1 / cell size
    int dim[3];
    int pad_;
    int64_t ncell;
};

// Batches: one instance's search structures, as the batch screen reads them.
struct BInst {
    HashGrid g;
    const int32_t* cell_start;
    const int32_t* cell_elems;
    const int32_t* sub;
    const ElemBox* boxes;
    const ElemBox32* boxes32;
    int64_t p0;          // first point of the instance (caller's order)
    int32_t ebase;       // batch element id of the instance's element 0
    int32_t pad_;
};

struct BScreenArgs {
    int ninst;
    const BInst* inst;   // [ninst]
    const int64_t* p0;   // [ninst + 1] first point of each instance
    int64_t P;           // points of the batch (row stride of pts)
    const double* pts;   // [3][P]
    int32_t* cnt;
    const int32_t* off;
    int32_t* pair_elem;
    int32_t* pair_pt;
    int64_t cap;
    uint32_t* mask;      // [P] count-pass candidate masks (see ScreenArgs::mask)
};

// A pair that lost its point's classification is marked by storing ~p
// (negative) in pair_pt: the fused eval skips it, and the point index stays
// recoverable (the batch tuner reruns the Newton stage on the same pairs).
__device__ __forceinline__ int64_t pair_point(int32_t v) { return v < 0 ? (int64_t)(~v) : (int64_t)v; }

struct FindParams {
    double tol_accept;  // relative to h_e
    double tol_border;  // relative to h_e
    double band;        // absolute tie band = tie_band * L
    int max_newton;
    int mixed;
    int refine;         // mixed form: compensated residuals per pair before the FP64 fallback
};

// ---------------------------------------------------------------------------
// Lagrange basis on the GLL points by prefix / suffix products:
//   h_i(r) = ci_i * prod_{m<i} (r - xi_m) * prod_{m>i} (r - xi_m)
// and its derivative by the product rule applied to the running products.
// ---------------------------------------------------------------------------
template <int n, typename T>
__device__ __forceinline__ void lagrange_hd(const T* __restrict__ xi, const T* __restrict__ ci,
                                            T r, T (&h)[n], T (&d)[n])
{
    T dm[n];
#pragma unroll
    for (int m = 0; m < n; ++m) dm[m] = r - xi[m];
    T pre[n], dpre[n];
    pre[0] = T(1);
    dpre[0] = T(0);
#pragma unroll
    for (int i = 1; i < n; ++i) {
        dpre[i] = dpre[i - 1] * dm[i - 1] + pre[i - 1];
        pre[i] = pre[i - 1] * dm[i - 1];
    }
    T suf = T(1), dsuf = T(0);
#pragma unroll
    for (int i = n - 1; i >= 0; --i) {
        h[i] = ci[i] * (pre[i] * suf);
        d[i] = ci[i] * (dpre[i] * suf + pre[i] * dsuf);
        dsuf = dsuf * dm[i] + suf;
        suf = suf * dm[i];
    }
}

template <int n, typename T>
__device__ __forceinline__ void lagrange_h(const T* __restrict__ xi, const T* __restrict__ ci,
                                           T r, T (&h)[n])
{
    T dm[n];
#pragma unroll
    for (int m = 0; m < n; ++m) dm[m] = r - xi[m];
    T pre[n];
    pre[0] = T(1);
#pragma unroll
    for (int i = 1; i < n; ++i) pre[i] = pre[i - 1] * dm[i - 1];
    T suf = T(1);
#pragma unroll
    for (int i = n - 1; i >= 0; --i) {
        h[i] = ci[i] * (pre[i] * suf);
        suf = suf * dm[i];
    }
}

template <typename T> struct Tab;
template <> struct Tab<double> {
    static __device__ __forceinline__ const double* xi(const BasisTab& b) { return b.xi; }
    static __device__ __forceinline__ const double* ci(const BasisTab& b) { return b.ci; }
};
template <> struct Tab<float> {
    static __device__ __forceinline__ const float* xi(const BasisTab& b) { return b.xif; }
    static __device__ __forceinline__ const float* ci(const BasisTab& b) { return b.cif; }
};

// Load one row of n contiguous values (vectorised when n is even and the row
// is 16-byte aligned, which holds for every row when n is even).
template <int n>
__device__ __forceinline__ void load_row(const double* __restrict__ p, double (&v)[n])
{
    if constexpr (n % 2 == 0) {
        const double2* q = reinterpret_cast<const double2*>(p);
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            double2 t = __ldg(q + i);
            v[2 * i] = t.x;
            v[2 * i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < n; ++i) v[i] = __ldg(p + i);
    }
}

template <int n>
__device__ __forceinline__ void load_row(const float* __restrict__ p, float (&v)[n])
{
    if constexpr (n % 4 == 0) {
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int i = 0; i < n / 4; ++i) {
            float4 t = __ldg(q + i);
            v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
    } else if constexpr (n % 2 == 0) {
        const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            float2 t = __ldg(q + i);
            v[2 * i] = t.x; v[2 * i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < n; ++i) v[i] = __ldg(p + i);
    }
}

// ---------------------------------------------------------------------------
// Element map x(r) and Jacobian by sum factorisation (Sec. 2: O(N^{d+1})
// tensor-product work).  X[a] points at coordinate a's n^3 nodes of one
// element.  Contract i (contiguous rows) with h_r and h_r', then j with h_s
// and h_s', then k with h_t and h_t'.
// ---------------------------------------------------------------------------
template <int n, typename T>
__device__ __forceinline__ void map_jac(const T* __restrict__ X0, const T* __restrict__ X1,
                                        const T* __restrict__ X2, const T (&hr)[n],
                                        const T (&dr)[n], const T (&hs)[n], const T (&ds)[n],
                                        const T* ht, const T* dt, T (&x)[3], T (&J)[9])
{
    // The j and k loops stay rolled: unrolled, the contraction is inlined
    // eight times over in the Newton kernels and runs ~1.8x slower (measured).
    // (Packed FP32 pairs for the i sums, as the double-float rows use them,
    // measured slower here: 26.4 against 25.8 ms for the mixed Newton stage.)
    T xa[3] = {0, 0, 0}, xr[3] = {0, 0, 0}, xs[3] = {0, 0, 0}, xt[3] = {0, 0, 0};
#pragma unroll 1
    for (int k = 0; k < n; ++k) {
        T c[3] = {0, 0, 0}, cs[3] = {0, 0, 0}, cr[3] = {0, 0, 0};
#pragma unroll 1
        for (int j = 0; j < n; ++j) {
            const int off = n * (j + n * k);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const T* row = (a == 0 ? X0 : (a == 1 ? X1 : X2)) + off;
                T v[n];
                load_row<n>(row, v);
                T u = 0, w = 0;
#pragma unroll
                for (int i = 0; i < n; ++i) {
                    u = fma(hr[i], v[i], u);
                    w = fma(dr[i], v[i], w);
                }
                c[a] = fma(hs[j], u, c[a]);
                cs[a] = fma(ds[j], u, cs[a]);
                cr[a] = fma(hs[j], w, cr[a]);
            }
        }
        const T tk = ht[k], dk = dt[k];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            xa[a] = fma(tk, c[a], xa[a]);
            xt[a] = fma(dk, c[a], xt[a]);
            xs[a] = fma(tk, cs[a], xs[a]);
            xr[a] = fma(tk, cr[a], xr[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        x[a] = xa[a];
        J[3 * a + 0] = xr[a];
        J[3 * a + 1] = xs[a];
        J[3 * a + 2] = xt[a];
    }
}

// Value-only contraction of one nodal array F (n^3) at a point.
template <int n, typename T>
__device__ __forceinline__ T contract(const T* __restrict__ F, const T (&hr)[n], const T (&hs)[n],
                                      const T* ht)
{
    T acc = 0;
#pragma unroll 1
    for (int k = 0; k < n; ++k) {
        T c = 0;
#pragma unroll 1
        for (int j = 0; j < n; ++j) {
            T v[n];
            load_row<n>(F + n * (j + n * k), v);
            T u = 0;
#pragma unroll
            for (int i = 0; i < n; ++i) u = fma(hr[i], v[i], u);
            c = fma(hs[j], u, c);
        }
        acc = fma(ht[k], c, acc);
    }
    return acc;
}

// ---------------------------------------------------------------------------
// Double-float arithmetic on the FP32 pipes (Dekker / Knuth error-free
// transformations).  A value is carried as an unevaluated sum hi + lo of two
// floats (about 48 significant bits).  df_fma_acc adds the product of two
// double-floats to an accumulator: the leading product is formed exactly
// (p = ah*bh, its rounding error by one fma), the cross terms ah*bl + al*bh
// are added to that error, and the sum acc.hi + p is an error-free two-sum
// whose error goes to the low part.  Used by the mixed form's residuals and
// evaluation, and by the peak probe that measures its throughput.
// ---------------------------------------------------------------------------
struct df {
    float hi, lo;
};

__device__ __forceinline__ df df_split(double v)
{
    const float h = (float)v;
    return {h, (float)(v - (double)h)};
}

// The error-free transformations below need every sum and product rounded
// on its own: the _rn intrinsics are never contracted into an fma by the
// compiler.

// acc += (ah + al) * (bh + bl)
__device__ __forceinline__ void df_fma_acc(df& acc, float ah, float al, float bh, float bl)
{
    const float p = __fmul_rn(ah, bh);
    const float pe = fmaf(ah, bh, -p);
    const float t = fmaf(ah, bl, fmaf(al, bh, pe));
    const float s = __fadd_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    acc.hi = s;
    acc.lo = __fadd_rn(acc.lo, __fadd_rn(err, t));
}

__device__ __forceinline__ void df_fma_acc(df& acc, const df& a, float bh, float bl)
{
    df_fma_acc(acc, a.hi, a.lo, bh, bl);
}

// the first term of a sum: df_fma_acc into a zero accumulator without the
// two-sum (the same value, up to the sign of a zero)
__device__ __forceinline__ df df_prod(float ah, float al, float bh, float bl)
{
    const float p = __fmul_rn(ah, bh);
    const float pe = fmaf(ah, bh, -p);
    return {p, fmaf(ah, bl, fmaf(al, bh, pe))};
}

// Two double-floats side by side in packed FP32 pairs (x and y lanes of a
// float2): every packed operation is the scalar one on each lane, rounded
// the same way, so df2_fma_acc gives exactly two df_fma_acc results.
struct df2 {
    float2 hi, lo;
};

__device__ __forceinline__ float2 f2_neg(float2 a) { return make_float2(-a.x, -a.y); }

__device__ __forceinline__ void df2_fma_acc(df2& acc, float2 ah, float2 al, float2 bh, float2 bl)
{
    const float2 p = __fmul2_rn(ah, bh);
    const float2 pe = __ffma2_rn(ah, bh, f2_neg(p));
    const float2 t = __ffma2_rn(ah, bl, __ffma2_rn(al, bh, pe));
    const float2 s = __fadd2_rn(acc.hi, p);
    const float2 bb = __fadd2_rn(s, f2_neg(acc.hi));
    const float2 err = __fadd2_rn(__fadd2_rn(acc.hi, f2_neg(__fadd2_rn(s, f2_neg(bb)))), __fadd2_rn(p, f2_neg(bb)));
    acc.hi = s;
    acc.lo = __fadd2_rn(acc.lo, __fadd2_rn(err, t));
}

// the first term of a packed pair of sums (df_prod on both lanes)
__device__ __forceinline__ df2 df2_prod(float2 ah, float2 al, float2 bh, float2 bl)
{
    const float2 p = __fmul2_rn(ah, bh);
    const float2 pe = __ffma2_rn(ah, bh, f2_neg(p));
    return {p, __ffma2_rn(ah, bl, __ffma2_rn(al, bh, pe))};
}

// the sum of a packed pair's two lanes: error-free two-sum of the leading
// parts, the low parts and the error added to the low part
__device__ __forceinline__ df df2_join(const df2& a)
{
    const float s = __fadd_rn(a.hi.x, a.hi.y);
    const float bb = __fsub_rn(s, a.hi.x);
    const float err = __fadd_rn(__fsub_rn(a.hi.x, __fsub_rn(s, bb)), __fsub_rn(a.hi.y, bb));
    return {s, __fadd_rn(__fadd_rn(a.lo.x, a.lo.y), err)};
}

// renormalise (fast two-sum): |lo| below one unit in the last place of hi
__device__ __forceinline__ void df_norm(df& a)
{
    const float t = __fadd_rn(a.hi, a.lo);
    a.lo = __fsub_rn(a.lo, __fsub_rn(t, a.hi));
    a.hi = t;
}

// a * b: exact leading product plus the cross terms, renormalised
__device__ __forceinline__ df df_mul(df a, df b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, fmaf(a.lo, b.hi, e));
    const float s = __fadd_rn(p, e);
    return {s, __fsub_rn(e, __fsub_rn(s, p))};
}

// a - b: error-free two-sum of the leading parts, then the low parts
__device__ __forceinline__ df df_sub(df a, df b)
{
    const float s = __fsub_rn(a.hi, b.hi);
    const float bb = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(-b.hi, bb));
    const float lo = __fadd_rn(err, __fsub_rn(a.lo, b.lo));
    const float t = __fadd_rn(s, lo);
    return {t, __fsub_rn(lo, __fsub_rn(t, s))};
}

// One row of a double-float contraction: sum_i (vh_i + vl_i)(rh_i + rl_i),
// even i in the x lanes and odd i in the y lanes of packed FP32 pairs (one
// instruction does both), the lanes joined by an error-free two-sum and the
// result renormalised.  Every double-float contraction (Newton residuals and
// field evaluation) goes through this routine, so all of them round alike.
template <int n>
__device__ __forceinline__ df row_df(const float (&vh)[n], const float (&vl)[n], const float (&rh)[n],
                                     const float (&rl)[n])
{
    df2 u = df2_prod(make_float2(vh[0], vh[1]), make_float2(vl[0], vl[1]), make_float2(rh[0], rh[1]),
                     make_float2(rl[0], rl[1]));
#pragma unroll
    for (int m = 1; m < n / 2; ++m)
        df2_fma_acc(u, make_float2(vh[2 * m], vh[2 * m + 1]), make_float2(vl[2 * m], vl[2 * m + 1]),
                    make_float2(rh[2 * m], rh[2 * m + 1]), make_float2(rl[2 * m], rl[2 * m + 1]));
    df r = df2_join(u);
    if constexpr (n % 2 == 1) df_fma_acc(r, vh[n - 1], vl[n - 1], rh[n - 1], rl[n - 1]);
    df_norm(r);
    return r;
}

// n floats of a row held in shared memory (plain loads, vectors for even n)
template <int n>
__device__ __forceinline__ void load_row_sm(const float* p, float (&v)[n])
{
    if constexpr (n % 4 == 0) {
        const float4* q = reinterpret_cast<const float4*>(p);
#pragma unroll
        for (int i = 0; i < n / 4; ++i) {
            const float4 t = q[i];
            v[4 * i] = t.x; v[4 * i + 1] = t.y; v[4 * i + 2] = t.z; v[4 * i + 3] = t.w;
        }
    } else if constexpr (n % 2 == 0) {
        const float2* q = reinterpret_cast<const float2*>(p);
#pragma unroll
        for (int i = 0; i < n / 2; ++i) {
            const float2 t = q[i];
            v[2 * i] = t.x; v[2 * i + 1] = t.y;
        }
    } else {
#pragma unroll
        for (int i = 0; i < n; ++i) v[i] = p[i];
    }
}

// Posted (double-float) fields keep each row of n nodes as its n high parts
// followed by its n low parts (n float2 slots), so both halves load as
// aligned vectors for even n.  SM: the row is in shared memory.
template <int n, bool SM = false>
__device__ __forceinline__ df row_df(const float2* __restrict__ rowp, const float (&rh)[n], const float (&rl)[n])
{
    const float* row = reinterpret_cast<const float*>(rowp);
    float vh[n], vl[n];
    if constexpr (SM) {
        load_row_sm<n>(row, vh);
        load_row_sm<n>(row + n, vl);
    } else {
        load_row<n>(row, vh);
        load_row<n>(row + n, vl);
    }
    return row_df<n>(vh, vl, rh, rl);
}

// sum_ijk F_ijk h_i h_j h_k for one element's double-float values Fe (n^3,
// i fastest) and split basis values; rounded to FP64.  SM: Fe is in shared
// memory.
template <int n, bool SM = false>
__device__ __forceinline__ double contract_df(const float2* __restrict__ Fe, const float (&rh)[n],
                                              const float (&rl)[n], const float (&sh)[n], const float (&sl)[n],
                                              const float (&th)[n], const float (&tl)[n])
{
    df acc = {0.0f, 0.0f};
#pragma unroll 1
    for (int k = 0; k < n; ++k) {
        df ck = {0.0f, 0.0f};
        // two rows in flight: their loads and two-sums overlap
#pragma unroll 2
        for (int j = 0; j < n; ++j) {
            const df u = row_df<n, SM>(Fe + n * (j + n * k), rh, rl);
            df_fma_acc(ck, u, sh[j], sl[j]);
        }
        df_norm(ck);
        df_fma_acc(acc, ck, th[k], tl[k]);
    }
    return (double)acc.hi + (double)acc.lo;
}

}  // namespace fpg
