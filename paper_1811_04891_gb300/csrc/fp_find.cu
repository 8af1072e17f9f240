// fp_find.cu -- point location (Sec. 2.1, findpts) as a pair stream.
//
//  1. k_screen<false>  per point: hash cell -> candidate list, session
//                      filter (sub != tag), axis box, box in the element's
//                      affine frame; count the survivors.
//  2. scan             per-point pair offsets.
//  3. k_screen<true>   write the (point, element) pairs in point order.
//  4. k_ehist / scan / k_escatter   counting sort of the pairs by element, so
//                      neighbouring threads work on the same element and its
//                      geometry is served by broadcast loads from L1.
//  5. Newton         per pair: seed at the nearest mapped GLL node (or the
//                      point's previous (e, r) on a moving mesh), then
//                      box-constrained trust-region Newton on
//                      ||x^e(r) - x*||^2.  FP64 form: k_newton<n>.  Mixed
//                      form: k_newton_mixed<n,CAP> runs the seed and the early
//                      iterations in FP32 on element-local coordinates, a
//                      compensated refinement and one FP64 step;
//                      k_newton64_full<n> finishes the pairs that step did
//                      not confirm in full FP64.
//  6. k_rank<n,3>      per point: classify its pairs (INSIDE / BORDER), lowest
//                      element id within a subdomain, owner = argmax of the
//                      interpolated distance field D^k with lower-id tie band.
#include <algorithm>

#include "fp_common.cuh"
#include "fp_internal.h"
#include "fp_rank.cuh"

namespace fpg {

// ---------------------------------------------------------------------------
// screening
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool inside_boxes(const ElemBox* __restrict__ bp, double x, double y, double z)
{
    const double* b = reinterpret_cast<const double*>(bp);
    // ElemBox layout: c[0..2], Ai[3..11], olo[12..14], ohi[15..17], blo[18..20], bhi[21..23]
    if (x < __ldg(b + 18) || x > __ldg(b + 21) || y < __ldg(b + 19) || y > __ldg(b + 22) ||
        z < __ldg(b + 20) || z > __ldg(b + 23))
        return false;
    const double dx = x - __ldg(b + 0), dy = y - __ldg(b + 1), dz = z - __ldg(b + 2);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        double v = __ldg(b + 3 + 3 * a) * dx + __ldg(b + 4 + 3 * a) * dy + __ldg(b + 5 + 3 * a) * dz;
        if (v < __ldg(b + 12 + a) || v > __ldg(b + 15 + a)) return false;
    }
    return true;
}

__device__ __forceinline__ bool inside_boxes32(const ElemBox32* __restrict__ bp, float x, float y, float z)
{
    const float* b = reinterpret_cast<const float*>(bp);
    // ElemBox32 layout: c[0..2], Ai[3..11], olo[12..14], ohi[15..17], blo[18..20], bhi[21..23]
    if (x < __ldg(b + 18) || x > __ldg(b + 21) || y < __ldg(b + 19) || y > __ldg(b + 22) ||
        z < __ldg(b + 20) || z > __ldg(b + 23))
        return false;
    const float dx = x - __ldg(b + 0), dy = y - __ldg(b + 1), dz = z - __ldg(b + 2);
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float v = __ldg(b + 3 + 3 * a) * dx + __ldg(b + 4 + 3 * a) * dy + __ldg(b + 5 + 3 * a) * dz;
        if (v < __ldg(b + 12 + a) || v > __ldg(b + 15 + a)) return false;
    }
    return true;
}

struct ScreenArgs {
    int64_t P;
    const double* pts;
    const int32_t* qsess;
    const int32_t* sub;
    const ElemBox* boxes;
    const ElemBox32* boxes32;
    HashGrid g;
    const int32_t* cell_start;
    const int32_t* cell_elems;
    int32_t* cnt;
    const int32_t* off;
    int32_t* pair_elem;
    int32_t* pair_pt;
    int64_t cap;          // pair capacity: pairs at positions >= cap are not written
    int64_t stride;       // row stride of pts (and offset of y, z rows); 0 means P
    int32_t pt_base;      // added to the point index written into pair_pt
    int32_t elem_base;    // added to the element index written into pair_elem
    uint32_t* mask;       // optional [P]: the count pass records which entries of the point's cell list
                          //   passed (bit q - start), so the emit pass need not test them again;
                          //   kMaskOverflow marks lists longer than 31 entries (tested again)
};

constexpr uint32_t kMaskOverflow = 0x80000000u;

// the hash cell of a point (-1: not finite or outside the grid); the FP32
// screen hashes in FP32
template <bool F32>
__device__ __forceinline__ int64_t hash_cell(const HashGrid& g, double x, double y, double z)
{
    if (!(isfinite(x) && isfinite(y) && isfinite(z))) return -1;
    double u0, u1, u2;
    if (F32) {
        u0 = (double)(((float)x - (float)g.org[0]) * (float)g.inv[0]);
        u1 = (double)(((float)y - (float)g.org[1]) * (float)g.inv[1]);
        u2 = (double)(((float)z - (float)g.org[2]) * (float)g.inv[2]);
    } else {
        u0 = (x - g.org[0]) * g.inv[0];
        u1 = (y - g.org[1]) * g.inv[1];
        u2 = (z - g.org[2]) * g.inv[2];
    }
    if (!(u0 >= 0.0 && u1 >= 0.0 && u2 >= 0.0 && u0 <= (double)g.dim[0] && u1 <= (double)g.dim[1] &&
          u2 <= (double)g.dim[2]))
        return -1;
    const int i = min((int)u0, g.dim[0] - 1);
    const int j = min((int)u1, g.dim[1] - 1);
    const int k = min((int)u2, g.dim[2] - 1);
    return i + (int64_t)g.dim[0] * (j + (int64_t)g.dim[1] * k);
}

template <bool EMIT, bool F32>
__device__ __forceinline__ void screen_point(const ScreenArgs& A, int64_t p)
{
    const int64_t ld = A.stride ? A.stride : A.P;
    const double x = A.pts[p], y = A.pts[ld + p], z = A.pts[2 * ld + p];
    const int tag = A.qsess ? A.qsess[p] : -1;
    int c = 0;
    int base = EMIT ? A.off[p] : 0;
    uint32_t m = 0;
    if (EMIT && A.mask) m = A.mask[p];
    if (EMIT && A.mask && !(m & kMaskOverflow)) {
        // the count pass found these entries of the point's cell list
        if (m) {
            const int b = __ldg(A.cell_start + hash_cell<F32>(A.g, x, y, z));
            while (m) {
                const int bit = __ffs(m) - 1;
                m &= m - 1;
                if (base + c < A.cap) {
                    A.pair_elem[base + c] = A.elem_base + __ldg(A.cell_elems + b + bit);
                    A.pair_pt[base + c] = A.pt_base + (int32_t)p;
                }
                ++c;
            }
        }
        return;
    }
    const int64_t cell = hash_cell<F32>(A.g, x, y, z);
    if (cell >= 0) {
        const int b = __ldg(A.cell_start + cell), en = __ldg(A.cell_start + cell + 1);
        if (!EMIT && en - b > 31) m = kMaskOverflow;
        for (int q = b; q < en; ++q) {
            const int e = __ldg(A.cell_elems + q);
            if (tag >= 0 && __ldg(A.sub + e) == tag) continue;
            if (F32) {
                if (!inside_boxes32(A.boxes32 + e, (float)x, (float)y, (float)z)) continue;
            } else if (!inside_boxes(A.boxes + e, x, y, z)) {
                continue;
            }
            if (EMIT && base + c < A.cap) {
                A.pair_elem[base + c] = A.elem_base + e;
                A.pair_pt[base + c] = A.pt_base + (int32_t)p;
            }
            if (!EMIT && !(m & kMaskOverflow)) m |= 1u << (q - b);
            ++c;
        }
    }
    if (!EMIT) {
        A.cnt[p] = c;
        if (A.mask) A.mask[p] = m;
    }
}

template <bool EMIT, bool F32>
__global__ void __launch_bounds__(256) k_screen(ScreenArgs A)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= A.P) return;
    screen_point<EMIT, F32>(A, p);
}

// Batches: one thread per point of all instances; the point's instance (the
// last one whose first point is <= p) gives the hash grid, boxes and element
// numbering it is screened against.
template <bool EMIT, bool F32>
__global__ void __launch_bounds__(256) k_bscreen(BScreenArgs B)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= B.P) return;
    int lo = 0, hi = B.ninst;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(B.p0 + mid) <= p) lo = mid;
        else hi = mid;
    }
    const BInst& I = B.inst[lo];
    ScreenArgs A;
    A.P = B.P;
    A.pts = B.pts;
    A.qsess = nullptr;
    A.sub = I.sub;
    A.boxes = I.boxes;
    A.boxes32 = I.boxes32;
    A.g = I.g;
    A.cell_start = I.cell_start;
    A.cell_elems = I.cell_elems;
    A.cnt = B.cnt;
    A.off = B.off;
    A.pair_elem = B.pair_elem;
    A.pair_pt = B.pair_pt;
    A.cap = B.cap;
    A.stride = B.P;
    A.pt_base = 0;
    A.elem_base = I.ebase;
    A.mask = B.mask;
    screen_point<EMIT, F32>(A, p);
}

cudaError_t launch_bscreen(const BScreenArgs& b, bool emit, bool f32, cudaStream_t s)
{
    if (b.P == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((b.P + 255) / 256);
    if (emit) {
        if (f32) k_bscreen<true, true><<<grid, 256, 0, s>>>(b);
        else k_bscreen<true, false><<<grid, 256, 0, s>>>(b);
    } else {
        if (f32) k_bscreen<false, true><<<grid, 256, 0, s>>>(b);
        else k_bscreen<false, false><<<grid, 256, 0, s>>>(b);
    }
    count_launch();
    return cudaGetLastError();
}

// number of pairs to process: the device-side total, capped by the capacity
__device__ __forceinline__ int64_t live_pairs(const int32_t* __restrict__ dcount, int64_t cap)
{
    const int64_t t = *dcount;
    return t < cap ? t : cap;
}

__global__ void k_ehist(const int32_t* __restrict__ dcount, int64_t cap, const int32_t* __restrict__ pair_elem,
                        int32_t* __restrict__ ecount)
{
    const int64_t npairs = live_pairs(dcount, cap);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npairs; q += (int64_t)gridDim.x * blockDim.x)
        atomicAdd(ecount + pair_elem[q], 1);
}

__global__ void k_escatter(const int32_t* __restrict__ dcount, int64_t cap, const int32_t* __restrict__ pair_elem,
                           const int32_t* __restrict__ estart, int32_t* __restrict__ cursor, int32_t* __restrict__ order,
                           int32_t* __restrict__ inv)
{
    const int64_t npairs = live_pairs(dcount, cap);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < npairs; q += (int64_t)gridDim.x * blockDim.x) {
        const int e = pair_elem[q];
        const int pos = estart[e] + atomicAdd(cursor + e, 1);
        order[pos] = (int32_t)q;
        if (inv) inv[q] = pos;
    }
}

// ---------------------------------------------------------------------------
// Newton machinery
// ---------------------------------------------------------------------------
template <typename T>
struct ElemPtr {
    const T* X0;
    const T* X1;
    const T* X2;
};

template <int n, typename T>
__device__ __forceinline__ void eval_fJ(const ElemPtr<T>& el, const BasisTab& tab, const T (&r)[3],
                                        const T (&xs)[3], T (&f)[3], T (&J)[9])
{
    T hr[n], dr[n], hs[n], ds[n], ht[n], dt[n];
    lagrange_hd<n, T>(Tab<T>::xi(tab), Tab<T>::ci(tab), r[0], hr, dr);
    lagrange_hd<n, T>(Tab<T>::xi(tab), Tab<T>::ci(tab), r[1], hs, ds);
    lagrange_hd<n, T>(Tab<T>::xi(tab), Tab<T>::ci(tab), r[2], ht, dt);
    T x[3];
    map_jac<n, T>(el.X0, el.X1, el.X2, hr, dr, hs, ds, ht, dt, x, J);
#pragma unroll
    for (int a = 0; a < 3; ++a) f[a] = x[a] - xs[a];
}

template <int n, typename T>
__device__ __forceinline__ void eval_f(const ElemPtr<T>& el, const BasisTab& tab, const T (&r)[3],
                                       const T (&xs)[3], T (&f)[3])
{
    T hr[n], hs[n], ht[n];
    lagrange_h<n, T>(Tab<T>::xi(tab), Tab<T>::ci(tab), r[0], hr);
    lagrange_h<n, T>(Tab<T>::xi(tab), Tab<T>::ci(tab), r[1], hs);
    lagrange_h<n, T>(Tab<T>::xi(tab), Tab<T>::ci(tab), r[2], ht);
    f[0] = contract<n, T>(el.X0, hr, hs, ht) - xs[0];
    f[1] = contract<n, T>(el.X1, hr, hs, ht) - xs[1];
    f[2] = contract<n, T>(el.X2, hr, hs, ht) - xs[2];
}

// J d = -f by cofactors; returns false when J is singular.
template <typename T>
__device__ __forceinline__ bool newton_solve3(const T (&J)[9], const T (&f)[3], T (&d)[3])
{
    const T C00 = J[4] * J[8] - J[5] * J[7], C01 = J[5] * J[6] - J[3] * J[8], C02 = J[3] * J[7] - J[4] * J[6];
    const T det = J[0] * C00 + J[1] * C01 + J[2] * C02;
    if (det == T(0) || !isfinite(det)) return false;
    const T C10 = J[2] * J[7] - J[1] * J[8], C11 = J[0] * J[8] - J[2] * J[6], C12 = J[1] * J[6] - J[0] * J[7];
    const T C20 = J[1] * J[5] - J[2] * J[4], C21 = J[2] * J[3] - J[0] * J[5], C22 = J[0] * J[4] - J[1] * J[3];
    const T id = T(1) / det;
    d[0] = -(C00 * f[0] + C10 * f[1] + C20 * f[2]) * id;
    d[1] = -(C01 * f[0] + C11 * f[1] + C21 * f[2]) * id;
    d[2] = -(C02 * f[0] + C12 * f[1] + C22 * f[2]) * id;
    return true;
}

// Gauss-Newton step with an active set: coordinates on a bound whose
// descent direction leaves the box are frozen; the remaining ones solve the
// reduced normal equations (the plain Newton step when all three are free).
// Returns the number of free coordinates.
template <typename T>
__device__ __forceinline__ int gn_step(const T (&J)[9], const T (&f)[3], const T (&r)[3], T (&d)[3])
{
    T g[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) g[b] = J[b] * f[0] + J[3 + b] * f[1] + J[6 + b] * f[2];
    bool act[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) act[b] = (r[b] <= T(-1) && g[b] > T(0)) || (r[b] >= T(1) && g[b] < T(0));
    int nfree = 0;
    for (int pass = 0; pass < 4; ++pass) {
        d[0] = d[1] = d[2] = T(0);
        int fi[3];
        nfree = 0;
#pragma unroll
        for (int b = 0; b < 3; ++b)
            if (!act[b]) fi[nfree++] = b;
        if (nfree == 0) break;
        bool ok = false;
        if (nfree == 3) {
            ok = newton_solve3<T>(J, f, d);
        } else if (nfree == 2) {
            const int p = fi[0], q = fi[1];
            const T a00 = J[p] * J[p] + J[3 + p] * J[3 + p] + J[6 + p] * J[6 + p];
            const T a11 = J[q] * J[q] + J[3 + q] * J[3 + q] + J[6 + q] * J[6 + q];
            const T a01 = J[p] * J[q] + J[3 + p] * J[3 + q] + J[6 + p] * J[6 + q];
            const T det = a00 * a11 - a01 * a01;
            if (det > T(0)) {
                d[p] = (-a11 * g[p] + a01 * g[q]) / det;
                d[q] = (-a00 * g[q] + a01 * g[p]) / det;
                ok = true;
            }
        } else {
            const int p = fi[0];
            const T a00 = J[p] * J[p] + J[3 + p] * J[3 + p] + J[6 + p] * J[6 + p];
            if (a00 > T(0)) {
                d[p] = -g[p] / a00;
                ok = true;
            }
        }
        if (!ok) {                                   // singular: steepest descent
            for (int t = 0; t < nfree; ++t) d[fi[t]] = -g[fi[t]];
        }
        bool grew = false;
#pragma unroll
        for (int b = 0; b < 3; ++b)
            if (!act[b] && ((r[b] <= T(-1) && d[b] < T(0)) || (r[b] >= T(1) && d[b] > T(0)))) {
                act[b] = true;
                grew = true;
            }
        if (!grew) break;
    }
    return nfree;
}

template <typename T> struct Lim;
template <> struct Lim<double> {
    static constexpr double quick = 1e-4;     // full Newton step size that hands over to chord steps
    static constexpr double chord = 1e-13;    // chord correction that confirms convergence
    static constexpr double stop = 1e-13;     // accepted step that ends a constrained solve
    static constexpr double rho_min = 1e-15;
};
template <> struct Lim<float> {
    static constexpr float quick = 2e-5f;
    static constexpr float chord = 0.0f;      // unused: the FP64 phase follows
    static constexpr float stop = 1e-6f;
    static constexpr float rho_min = 1e-7f;
};

// Box truncation of a step d at r: largest t <= 1 with r + t d in the box;
// the new point lands exactly on the bound it was cut at.
template <typename T>
__device__ __forceinline__ T box_step(const T (&r)[3], const T (&d)[3], T (&rn)[3])
{
    T t = T(1);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        if (d[b] > T(0) && r[b] + d[b] > T(1)) t = fmin(t, (T(1) - r[b]) / d[b]);
        if (d[b] < T(0) && r[b] + d[b] < T(-1)) t = fmin(t, (T(-1) - r[b]) / d[b]);
    }
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        T v = r[b] + t * d[b];
        if (t < T(1)) {
            if (d[b] > T(0) && (T(1) - r[b]) / d[b] == t) v = T(1);
            if (d[b] < T(0) && (T(-1) - r[b]) / d[b] == t) v = T(-1);
        }
        rn[b] = fmin(T(1), fmax(T(-1), v));
    }
    return t;
}

// Chord iterations in FP64: value-only residuals with a fixed Jacobian J and
// the active-set step.  Converged when the next step is <= 1e-13 in every
// coordinate (r is then kept with its own residual).  Returns true on
// convergence; `res` is the residual norm at the returned r.
// Threshold of the chord check: 1e-13 in r, raised to the rounding level of a
// step where that is larger.  The residual x(r) - x* carries rounding errors
// of a few units of |x*|, which a step J^-1 f turns into ||J^-1|| times as
// much in r; on small elements far from the origin that exceeds 1e-13 and no
// step could confirm convergence.  2 eps |x*| ||J^-1||_inf bounds the noise.
__device__ __forceinline__ double chord_tol3(const double (&J)[9], const double (&xs)[3])
{
    const double C00 = J[4] * J[8] - J[5] * J[7], C01 = J[5] * J[6] - J[3] * J[8], C02 = J[3] * J[7] - J[4] * J[6];
    const double det = J[0] * C00 + J[1] * C01 + J[2] * C02;
    if (!(fabs(det) > 0.0) || !isfinite(det)) return Lim<double>::chord;
    const double C10 = J[2] * J[7] - J[1] * J[8], C11 = J[0] * J[8] - J[2] * J[6], C12 = J[1] * J[6] - J[0] * J[7];
    const double C20 = J[1] * J[5] - J[2] * J[4], C21 = J[2] * J[3] - J[0] * J[5], C22 = J[0] * J[4] - J[1] * J[3];
    const double rows = fmax(fabs(C00) + fabs(C10) + fabs(C20),
                             fmax(fabs(C01) + fabs(C11) + fabs(C21), fabs(C02) + fabs(C12) + fabs(C22)));
    const double xm = fmax(fabs(xs[0]), fmax(fabs(xs[1]), fabs(xs[2])));
    return fmax(Lim<double>::chord, 4.440892098500626e-16 * xm * rows / fabs(det));
}

// ---- one warp per pair: the n^2 rows of the contractions are split over the
// lanes, partial sums reduced to lane 0 in a fixed order and broadcast, so
// every lane holds the same bits and the Newton control flow stays uniform
// across the warp.  Used for the few pairs of the mixed form's fallback, whose
// cost is the latency of one long FP64 solve rather than throughput.
__device__ __forceinline__ double warp_sum_bcast(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return __shfl_sync(0xffffffffu, v, 0);
}

template <int n>
__device__ void eval_fJ_warp(const ElemPtr<double>& el, const BasisTab& tab, const double (&r)[3],
                             const double (&xs)[3], double (&f)[3], double (&J)[9])
{
    double hr[n], dr[n], hs[n], ds[n], ht[n], dt[n];
    lagrange_hd<n, double>(tab.xi, tab.ci, r[0], hr, dr);
    lagrange_hd<n, double>(tab.xi, tab.ci, r[1], hs, ds);
    lagrange_hd<n, double>(tab.xi, tab.ci, r[2], ht, dt);
    double x[3] = {0, 0, 0}, xr[3] = {0, 0, 0}, xsd[3] = {0, 0, 0}, xt[3] = {0, 0, 0};
    const int lane = threadIdx.x & 31;
    for (int q = lane; q < n * n; q += 32) {              // row q = j + n k
        const int j = q % n, k = q / n;
        const double hsj = hs[j], dsj = ds[j], htk = ht[k], dtk = dt[k];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double v[n];
            load_row<n>((a == 0 ? el.X0 : (a == 1 ? el.X1 : el.X2)) + n * q, v);
            double u = 0.0, w = 0.0;
#pragma unroll
            for (int i = 0; i < n; ++i) {
                u = fma(hr[i], v[i], u);
                w = fma(dr[i], v[i], w);
            }
            x[a] = fma(htk, hsj * u, x[a]);
            xr[a] = fma(htk, hsj * w, xr[a]);
            xsd[a] = fma(htk, dsj * u, xsd[a]);
            xt[a] = fma(dtk, hsj * u, xt[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        f[a] = warp_sum_bcast(x[a]) - xs[a];
        J[3 * a + 0] = warp_sum_bcast(xr[a]);
        J[3 * a + 1] = warp_sum_bcast(xsd[a]);
        J[3 * a + 2] = warp_sum_bcast(xt[a]);
    }
}

template <int n>
__device__ void eval_f_warp(const ElemPtr<double>& el, const BasisTab& tab, const double (&r)[3],
                            const double (&xs)[3], double (&f)[3])
{
    double hr[n], hs[n], ht[n];
    lagrange_h<n, double>(tab.xi, tab.ci, r[0], hr);
    lagrange_h<n, double>(tab.xi, tab.ci, r[1], hs);
    lagrange_h<n, double>(tab.xi, tab.ci, r[2], ht);
    double x[3] = {0, 0, 0};
    const int lane = threadIdx.x & 31;
    for (int q = lane; q < n * n; q += 32) {
        const double c = ht[q / n] * hs[q % n];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            double v[n];
            load_row<n>((a == 0 ? el.X0 : (a == 1 ? el.X1 : el.X2)) + n * q, v);
            double u = 0.0;
#pragma unroll
            for (int i = 0; i < n; ++i) u = fma(hr[i], v[i], u);
            x[a] = fma(c, u, x[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) f[a] = warp_sum_bcast(x[a]) - xs[a];
}

template <int n, bool WARP = false>
__device__ bool chord64(const ElemPtr<double>& el, const BasisTab& tab, const double (&xs)[3], double (&r)[3],
                        const double (&J)[9], double& res, int max_chord)
{
    const double tol = chord_tol3(J, xs);
    for (int it = 0; it < max_chord; ++it) {
        double f[3];
        if constexpr (WARP) eval_f_warp<n>(el, tab, r, xs, f);
        else eval_f<n, double>(el, tab, r, xs, f);
        res = sqrt(f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
        if (!(res > 0.0)) return true;
        double d[3];
        if (gn_step<double>(J, f, r, d) == 0) return true;         // KKT point at a vertex
        double rn[3];
        box_step<double>(r, d, rn);
        const double sn = fmax(fabs(rn[0] - r[0]), fmax(fabs(rn[1] - r[1]), fabs(rn[2] - r[2])));
        if (sn <= tol) return true;
        r[0] = rn[0]; r[1] = rn[1]; r[2] = rn[2];
    }
    return false;
}

// Box-constrained trust-region Newton (Sec. 2.1) from r (in/out); J returns
// the Jacobian at (or one small step before) the returned r.  Returns the
// residual norm ||x(r) - x*|| at the returned r.  With FINAL (FP64) a small
// full Newton step hands over to chord iterations with the current Jacobian;
// without it (FP32 phase of the mixed form) the loop stops after such a step.
// State of a solve paused between two iterations (FP64 form, two passes):
// with r, it is everything the next iteration depends on (f and J are
// recomputed at r), so a resumed solve takes exactly the steps the
// uninterrupted one would have.
struct NewtonState {
    double rho;
    int chord_fail;
    int it;
    bool paused;
};

template <int n, typename T, bool FINAL, bool WARP = false>
__device__ T newton(const ElemPtr<T>& el, const BasisTab& tab, const T (&xs)[3], T (&r)[3], T (&J)[9], int max_it,
                    bool& converged, NewtonState* st = nullptr, int budget = 0x7fffffff)
{
    static_assert(!WARP || (FINAL && sizeof(T) == 8), "the warp-cooperative solver is the FP64 one");
    auto fJ = [&](const T (&rr)[3], T (&ff)[3], T (&JJ)[9]) {
        if constexpr (WARP) eval_fJ_warp<n>(el, tab, rr, xs, ff, JJ);
        else eval_fJ<n, T>(el, tab, rr, xs, ff, JJ);
    };
    T f[3];
    fJ(r, f, J);
    T phi = T(0.5) * (f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
    T rho = st ? T(st->rho) : T(1);
    int chord_fail = st ? st->chord_fail : 0;   // after two failed chord checks the trust-region rules alone finish
    const int it0 = st ? st->it : 0;
    if (st) st->paused = false;
    converged = true;
    for (int it = it0; it < max_it; ++it) {
        if (st && it - it0 >= budget) {                   // pause: the caller resumes later
            st->rho = (double)rho;
            st->chord_fail = chord_fail;
            st->it = it;
            st->paused = true;
            converged = false;
            return sqrt(T(2) * phi);
        }
        if (!(phi > T(0))) return T(0);
        T d[3];
        const int nfree = gn_step<T>(J, f, r, d);
        if (nfree == 0) return sqrt(T(2) * phi);          // KKT point at a vertex
        const T dn = fmax(fabs(d[0]), fmax(fabs(d[1]), fabs(d[2])));
        if (!(dn > T(0))) return sqrt(T(2) * phi);
        bool full = true;
        if (dn > rho) {
            const T sc = rho / dn;
            d[0] *= sc; d[1] *= sc; d[2] *= sc;
            full = false;
        }
        T rn[3];
        if (box_step<T>(r, d, rn) < T(1)) full = false;
        T s[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) s[b] = rn[b] - r[b];
        const T sn = fmax(fabs(s[0]), fmax(fabs(s[1]), fabs(s[2])));
        if (!(sn > T(0))) return sqrt(T(2) * phi);
        // a small unconstrained Newton step: quadratic convergence from here
        if (full && nfree == 3 && dn <= Lim<T>::quick && chord_fail < 2) {
            if constexpr (!FINAL) {
                r[0] = rn[0]; r[1] = rn[1]; r[2] = rn[2];
                return sqrt(T(2) * phi);
            } else {
                T rc[3] = {rn[0], rn[1], rn[2]};
                T res;
                if (chord64<n, WARP>(el, tab, xs, rc, J, res, 3)) {
                    r[0] = rc[0]; r[1] = rc[1]; r[2] = rc[2];
                    return res;
                }
                r[0] = rc[0]; r[1] = rc[1]; r[2] = rc[2];   // not yet converged: refresh J
                ++chord_fail;
                fJ(r, f, J);
                phi = T(0.5) * (f[0] * f[0] + f[1] * f[1] + f[2] * f[2]);
                continue;
            }
        }
        T mf[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) mf[a] = f[a] + J[3 * a] * s[0] + J[3 * a + 1] * s[1] + J[3 * a + 2] * s[2];
        const T pred = phi - T(0.5) * (mf[0] * mf[0] + mf[1] * mf[1] + mf[2] * mf[2]);
        T fn[3], Jn[9];
        fJ(rn, fn, Jn);
        const T phin = T(0.5) * (fn[0] * fn[0] + fn[1] * fn[1] + fn[2] * fn[2]);
        if (sn <= Lim<T>::stop) {
            if (phin <= phi) {
                r[0] = rn[0]; r[1] = rn[1]; r[2] = rn[2];
#pragma unroll
                for (int q = 0; q < 9; ++q) J[q] = Jn[q];
                phi = phin;
            }
            return sqrt(T(2) * phi);
        }
        if (phin < phi) {
            const T ratio = pred > T(0) ? (phi - phin) / pred : T(0);
            r[0] = rn[0]; r[1] = rn[1]; r[2] = rn[2];
#pragma unroll
            for (int q = 0; q < 9; ++q) J[q] = Jn[q];
            f[0] = fn[0]; f[1] = fn[1]; f[2] = fn[2];
            phi = phin;
            if (ratio > T(0.75) && sn >= T(0.99) * rho) rho = fmin(T(2) * rho, T(2));
            else if (ratio < T(0.25)) rho = T(0.25) * sn;
        } else {
            rho = T(0.25) * sn;
            // a radius collapsed below the rounding level: converged as far as
            // this precision resolves (the FP32 phase only supplies a start)
            if (rho < Lim<T>::rho_min) return sqrt(T(2) * phi);
        }
    }
    converged = false;                                     // iteration cap
    return sqrt(T(2) * phi);
}

// nearest mapped GLL node (ties: lowest node index) -> its reference coordinates
template <int n, typename T>
__device__ __forceinline__ void seed_nearest(const ElemPtr<T>& el, const BasisTab& tab, const T (&xs)[3], T (&r)[3])
{
    constexpr int n3 = n * n * n;
    T best = T(INFINITY);
    int bq = 0;
    if constexpr (sizeof(T) == 4 && n3 % 4 == 0) {
        // four nodes per 16-byte load (every element's rows start 16-byte aligned)
        const float4* X0 = reinterpret_cast<const float4*>(el.X0);
        const float4* X1 = reinterpret_cast<const float4*>(el.X1);
        const float4* X2 = reinterpret_cast<const float4*>(el.X2);
#pragma unroll 2
        for (int q4 = 0; q4 < n3 / 4; ++q4) {
            const float4 a = __ldg(X0 + q4), b = __ldg(X1 + q4), c = __ldg(X2 + q4);
            const float ax[4] = {a.x, a.y, a.z, a.w}, bx[4] = {b.x, b.y, b.z, b.w}, cx[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
            for (int m = 0; m < 4; ++m) {
                const T dx = ax[m] - xs[0], dy = bx[m] - xs[1], dz = cx[m] - xs[2];
                const T d2 = dx * dx + dy * dy + dz * dz;
                if (d2 < best) {
                    best = d2;
                    bq = 4 * q4 + m;
                }
            }
        }
    } else {
#pragma unroll 4
        for (int q = 0; q < n3; ++q) {
            const T dx = __ldg(el.X0 + q) - xs[0];
            const T dy = __ldg(el.X1 + q) - xs[1];
            const T dz = __ldg(el.X2 + q) - xs[2];
            const T d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < best) {
                best = d2;
                bq = q;
            }
        }
    }
    const int i = bq % n, j = (bq / n) % n, k = bq / (n * n);
    r[0] = Tab<T>::xi(tab)[i];
    r[1] = Tab<T>::xi(tab)[j];
    r[2] = Tab<T>::xi(tab)[k];
}

struct NewtonArgs {
    const int32_t* dcount;  // device-side pair total (capped by cap)
    int64_t E;
    const int32_t* order;
    const int32_t* pair_elem;
    const int32_t* pair_pt;
    int64_t P;
    const double* pts;
    const double* coords;
    const float* coords32;
    const float* coords32lo;  // mixed form: low parts of the element-local coordinates
    const ElemBox* boxes;
    double* pres;
    double* prst;
    int64_t cap;
    double reject32;      // mixed: reject after FP32 when residual > reject32 * h_e
    int max_newton;
    int refine;           // mixed: compensated residuals per pair before the FP64 fallback
    int first_pass;       // FP64 form with pstate: iterations of the first pass
    unsigned long long* stats;  // optional path counters (profiling): [0] rejected after FP32,
                                // [1] FP32 not converged, [2] FP64 step converged, [3] sent to the fallback
    const int32_t* warm_elem;   // optional [P]: each point's element at the previous mesh position
    const double* warm_rst;     // [3][P]: its reference coordinates there
    int32_t* fb_count;          // mixed form: number of pairs sent to the FP64 fallback (zeroed before)
    int32_t* fb_list;           // their slots, the first fb_cap of them (batch groups: from the group's
    int64_t fb_cap;             //   first sorted position, capacity = the group's pairs)
    // batch groups: the group's pairs are the sorted positions [*s_lo, *s_hi)
    // (null: [0, live pairs)); pair_elem - ebase indexes the group's arrays
    const int32_t* s_lo;
    const int32_t* s_hi;
    int32_t ebase;
    int32_t* queue;             // work-queue counter (zeroed before the launch); null = grid-stride
    int tile;                   // sorted positions per work item (a multiple of 32)
    double2* pstate;            // FP64 form: state of solves paused after the first pass's budget
                                //   (rho, chord_fail + 4 it) per pair; null = one pass
    bool walk;                  // pair results (pres, prst, pstate) at sorted positions s (coalesced);
                                //   otherwise at pair slots q.  Fallback lists hold the same index.
};

// where pair s / q keeps its results, and the pair of a listed index
__device__ __forceinline__ int64_t result_slot(const NewtonArgs& A, int64_t s, int32_t q) { return A.walk ? s : q; }
__device__ __forceinline__ int32_t listed_pair(const NewtonArgs& A, int64_t t) { return A.walk ? A.order[t] : (int32_t)t; }

struct PairRange {
    int64_t s0, s1;
};

__device__ __forceinline__ PairRange pair_range(const NewtonArgs& A)
{
    if (A.s_lo) return {(int64_t)*A.s_lo, (int64_t)*A.s_hi};
    return {0, live_pairs(A.dcount, A.cap)};
}

// Visit the sorted pair positions of the range: grid-stride over a fixed
// grid, or (queue) work items of `tile` consecutive positions that whole
// warps draw from a device counter, so a warp whose pairs converged fast
// takes the next item instead of idling (pairs of one element stay together
// in an item).  The counter only grows; no warp waits on another.
template <typename Fn>
__device__ __forceinline__ void for_each_pair(const NewtonArgs& A, const PairRange& R, Fn&& fn)
{
    if (!A.queue) {
        for (int64_t s = R.s0 + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < R.s1;
             s += (int64_t)gridDim.x * blockDim.x)
            fn(s);
        return;
    }
    const int lane = threadIdx.x & 31;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(A.queue, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        const int64_t t0 = R.s0 + (int64_t)item * A.tile;
        if (t0 >= R.s1) break;
        const int64_t t1 = t0 + A.tile < R.s1 ? t0 + A.tile : R.s1;
        for (int64_t s = t0 + lane; s < t1; s += 32) fn(s);
    }
}

// warm start (moving meshes): a pair whose element is the point's previous
// element starts from the previous reference coordinates, clamped to the
// reference cube, instead of the nearest node.  Only the start changes; a
// non-finite previous value falls back to the nearest node.
__device__ __forceinline__ bool warm_seed(const NewtonArgs& A, int64_t p, int e, double (&r)[3])
{
    if (!A.warm_elem || A.warm_elem[p] != e) return false;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const double v = A.warm_rst[a * A.P + p];
        if (!(fabs(v) <= 2.0)) return false;
        r[a] = fmin(1.0, fmax(-1.0, v));
    }
    return true;
}

// FP64 form: nearest-node (or warm) start, full FP64 trust-region Newton;
// with A.pstate, the first pass stops a solve after A.first_pass iterations
// and lists it (fbl, capacity fbc) for the second.  Measured on the 32^3
// N=7 workload: budgets 1 / 2 / 3 / 4 / 5 / 6 gave 387 / 300 / 311 / 319 /
// 323 / 326 ms for the two passes together; the batch's per-order groups
// measured faster with 4 (82 / 88 ms for N = 5 / 7 against 105 / 104 with 2).
constexpr int kFirstPass = 2;
constexpr int kFirstPassBatch = 4;

template <int n>
__device__ __forceinline__ void solve_pair(const NewtonArgs& A, const BasisTab& tab, int64_t s, int32_t* fbl,
                                           int64_t fbc)
{
    constexpr int n3 = n * n * n;
    const int32_t q = A.order[s];
    const int e = A.pair_elem[q] - A.ebase;
    const int64_t p = pair_point(A.pair_pt[q]);
    const double xs[3] = {A.pts[p], A.pts[A.P + p], A.pts[2 * A.P + p]};
    const ElemPtr<double> el64 = {A.coords + (int64_t)e * n3, A.coords + (A.E + e) * n3,
                                  A.coords + (2 * A.E + e) * n3};
    double r[3], J[9];
    if (!warm_seed(A, p, e, r)) seed_nearest<n, double>(el64, tab, xs, r);
    bool conv64;
    NewtonState st{1.0, 0, 0, false};
    const double res = newton<n, double, true>(el64, tab, xs, r, J, A.max_newton, conv64, A.pstate ? &st : nullptr,
                                               A.first_pass);
    const int64_t w = result_slot(A, s, q);
    A.prst[w] = r[0];
    A.prst[A.cap + w] = r[1];
    A.prst[2 * A.cap + w] = r[2];
    if (st.paused) {
        // still iterating after the first pass's budget: continued by
        // k_newton_resume, so that warps of the first pass do not wait on it
        A.pres[w] = -1.0;
        A.pstate[w] = make_double2(st.rho, (double)(st.chord_fail + 4 * st.it));
        const int32_t k = atomicAdd(A.fb_count, 1);
        if (k < fbc) fbl[k] = (int32_t)w;
    } else {
        A.pres[w] = res;
    }
}

// pass 2 of the FP64 form: the solves paused by the first pass, resumed
// where they stopped, one per thread (the list is dense: every lane has a
// long solve).  If the list overflowed, the paused slots (pres < 0) are
// found by scanning the range instead.
template <int n>
__device__ __forceinline__ void resume_pair(const NewtonArgs& A, const BasisTab& tab, int64_t w)
{
    constexpr int n3 = n * n * n;
    const int32_t q = listed_pair(A, w);
    const int e = A.pair_elem[q] - A.ebase;
    const int64_t p = pair_point(A.pair_pt[q]);
    const double xs[3] = {A.pts[p], A.pts[A.P + p], A.pts[2 * A.P + p]};
    const ElemPtr<double> el64 = {A.coords + (int64_t)e * n3, A.coords + (A.E + e) * n3,
                                  A.coords + (2 * A.E + e) * n3};
    double r[3] = {A.prst[w], A.prst[A.cap + w], A.prst[2 * A.cap + w]}, J[9];
    const double2 sv = A.pstate[w];
    const int code = (int)sv.y;
    NewtonState st{sv.x, code & 3, code >> 2, false};
    bool conv;
    const double res = newton<n, double, true>(el64, tab, xs, r, J, A.max_newton, conv, &st);
    A.prst[w] = r[0];
    A.prst[A.cap + w] = r[1];
    A.prst[2 * A.cap + w] = r[2];
    A.pres[w] = res;
}

template <int n>
__global__ void __launch_bounds__(128) k_newton_resume(NewtonArgs A, BasisTab tab)
{
    const PairRange R = pair_range(A);
    const int32_t* fbl = A.fb_list + (A.s_lo ? R.s0 : 0);
    const int64_t fbc = A.s_lo ? R.s1 - R.s0 : A.fb_cap;
    const int64_t nfb = *A.fb_count;
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x, dt = (int64_t)gridDim.x * blockDim.x;
    if (nfb <= fbc) {
        for (int64_t t = t0; t < nfb; t += dt) resume_pair<n>(A, tab, fbl[t]);
    } else {
        for (int64_t s = R.s0 + t0; s < R.s1; s += dt) {
            const int64_t w = result_slot(A, s, A.order[s]);
            if (A.pres[w] < 0.0) resume_pair<n>(A, tab, w);
        }
    }
}

// FP32 value of a reference coordinate that is +-1 only when r is exactly +-1
__device__ __forceinline__ float f32_inside(double v)
{
    float f = (float)v;
    if (f >= 1.0f && v < 1.0) f = 0.99999994f;       // largest float below 1
    if (f <= -1.0f && v > -1.0) f = -0.99999994f;
    return f;
}

// ---- compensated FP32 residual for the refinement steps of the mixed form ----
// x_local(r) - x*_local with node offsets X - c held as float pairs (hi, lo),
// basis values computed in FP64 and split, products formed exactly in their
// leading part and summed with error-free two-sums (about 48 significant
// bits in element-local units).  Runs on the FP32 pipes.
// Lagrange basis at r in double-float arithmetic, on the FP32 pipes: r split
// into (hi, lo), each factor r - xi_m by an error-free difference, the
// prefix / suffix products and the normalisers c_i as double-float products.
// About 2^-45 absolute error on the basis values (measured against
// extended-precision products: 2.7e-14 at worst, 2e-15 rms, for N = 7),
// against 2^-48 for an FP64 basis split afterwards; the residuals that use it
// only steer and confirm the final Newton steps.
template <int n>
__device__ __forceinline__ void lagrange_h_df(double rv, const BasisTab& tab, float (&hh)[n], float (&hl)[n])
{
    const df r = df_split(rv);
    df dm[n];
#pragma unroll
    for (int m = 0; m < n; ++m) dm[m] = df_sub(r, df{tab.xif[m], tab.xil[m]});
    df pre[n];
    pre[0] = {1.0f, 0.0f};
#pragma unroll
    for (int i = 1; i < n; ++i) pre[i] = df_mul(pre[i - 1], dm[i - 1]);
    df suf = {1.0f, 0.0f};
#pragma unroll
    for (int i = n - 1; i >= 0; --i) {
        const df t = df_mul(df{tab.cif[i], tab.cil[i]}, df_mul(pre[i], suf));
        hh[i] = t.hi;
        hl[i] = t.lo;
        suf = df_mul(suf, dm[i]);
    }
}

template <int n>
__device__ __forceinline__ void resid_df(const ElemPtr<float>& hi, const ElemPtr<float>& lo, const BasisTab& tab,
                                         const double (&r)[3], const double (&xl)[3], float (&f)[3])
{
    float rh[n], rl[n], sh[n], sl[n], th[n], tl[n];
    lagrange_h_df<n>(r[0], tab, rh, rl);
    lagrange_h_df<n>(r[1], tab, sh, sl);
    lagrange_h_df<n>(r[2], tab, th, tl);
    df acc[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
#pragma unroll 1
    for (int k = 0; k < n; ++k) {
        df ck[3] = {{0.0f, 0.0f}, {0.0f, 0.0f}, {0.0f, 0.0f}};
#pragma unroll 1
        for (int j = 0; j < n; ++j) {
            const int off = n * (j + n * k);
            df u[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {             // three coordinates: three independent chains
                const float* Xh = (a == 0 ? hi.X0 : (a == 1 ? hi.X1 : hi.X2)) + off;
                const float* Xl = (a == 0 ? lo.X0 : (a == 1 ? lo.X1 : lo.X2)) + off;
                float vh[n], vl[n];
                load_row<n>(Xh, vh);
                load_row<n>(Xl, vl);
                u[a] = row_df<n>(vh, vl, rh, rl);
            }
#pragma unroll
            for (int a = 0; a < 3; ++a) df_fma_acc(ck[a], u[a].hi, u[a].lo, sh[j], sl[j]);
        }
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            df_norm(ck[a]);
            df_fma_acc(acc[a], ck[a].hi, ck[a].lo, th[k], tl[k]);
        }
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        const float xh = (float)xl[a];
        const float xlo = (float)(xl[a] - (double)xh);
        f[a] = (acc[a].hi - xh) + (acc[a].lo - xlo);
    }
}

// Threshold of the final step's convergence check on a double-float
// residual: 1e-13 in r, raised to the rounding level of a step where that is
// larger.  The residual is accurate to a few units of 2^-48 of the
// element-local coordinates (|x - c_e| <= h_e), which a step J^-1 f turns
// into ||J^-1|| times as much in r; 2^-46 h_e ||J^-1||_inf bounds that noise.
__device__ __forceinline__ double chord_tol_df(const double (&J)[9], double he)
{
    const double C00 = J[4] * J[8] - J[5] * J[7], C01 = J[5] * J[6] - J[3] * J[8], C02 = J[3] * J[7] - J[4] * J[6];
    const double det = J[0] * C00 + J[1] * C01 + J[2] * C02;
    if (!(fabs(det) > 0.0) || !isfinite(det)) return Lim<double>::chord;
    const double C10 = J[2] * J[7] - J[1] * J[8], C11 = J[0] * J[8] - J[2] * J[6], C12 = J[1] * J[6] - J[0] * J[7];
    const double C20 = J[1] * J[5] - J[2] * J[4], C21 = J[2] * J[3] - J[0] * J[5], C22 = J[0] * J[4] - J[1] * J[3];
    const double rows = fmax(fabs(C00) + fabs(C10) + fabs(C20),
                             fmax(fabs(C01) + fabs(C11) + fabs(C21), fabs(C02) + fabs(C12) + fabs(C22)));
    return fmax(Lim<double>::chord, 1.4210854715202004e-14 * he * rows / fabs(det));
}

// final steps of the mixed form: at most NewtonArgs::refine double-float
// residuals (3 by default); a step of at most kConfirm (computed in FP32) is
// re-solved in FP64; an FP64 step of at most kTake chord tolerances is taken
// without another residual (see solve_mixed)
constexpr double kConfirm = 1e-10;
constexpr double kTake = 1e3;

// passes 1 and 2 in one kernel: the FP32 work of some warps overlaps the
// FP64 work of others.
// Launch shape of the mixed Newton kernel.  CAP (blocks of up to 128
// threads, n <= 10, where 128 registers need no spills): registers capped so
// that four blocks of 128 threads fit an SM (measured at n = 8: 2 % faster
// than five blocks at 96 registers, which spill).
// Otherwise (persistent grids of the workspace and batch paths, larger n)
// the compiler is left free.
template <int n, bool CAP> struct MixedLB {
    static constexpr int threads = CAP ? 128 : 256;
    static constexpr int blocks = CAP ? 4 : 1;
};

template <int n>
__device__ __forceinline__ void solve_mixed(const NewtonArgs& A, const BasisTab& tab, int64_t s, int32_t* fbl,
                                            int64_t fbc)
{
    constexpr int n3 = n * n * n;
    {
        const int32_t q = A.order[s];
        const int e = A.pair_elem[q] - A.ebase;
        const int64_t p = pair_point(A.pair_pt[q]);
        const double xs[3] = {A.pts[p], A.pts[A.P + p], A.pts[2 * A.P + p]};
        const double* c = A.boxes[e].c;
        const double xd[3] = {xs[0] - c[0], xs[1] - c[1], xs[2] - c[2]};
        const float xl[3] = {(float)xd[0], (float)xd[1], (float)xd[2]};
        const ElemPtr<float> el32 = {A.coords32 + (int64_t)e * n3, A.coords32 + (A.E + e) * n3,
                                     A.coords32 + (2 * A.E + e) * n3};
        float r32[3], J32[9];
        {
            double rw[3];
            if (warm_seed(A, p, e, rw)) {
                r32[0] = (float)rw[0]; r32[1] = (float)rw[1]; r32[2] = (float)rw[2];
            } else {
                seed_nearest<n, float>(el32, tab, xl, r32);
            }
        }
        bool conv32;
        const float res32 = newton<n, float, false>(el32, tab, xl, r32, J32, A.max_newton, conv32);
        double r[3] = {r32[0], r32[1], r32[2]};
        double res = conv32 ? (double)res32 : -1.0;
        if (A.stats) {
            if (!conv32) atomicAdd(A.stats + 1, 1ULL);
            else if ((double)res32 > A.reject32 * A.boxes[e].he) atomicAdd(A.stats + 0, 1ULL);
        }
        if (conv32 && (double)res32 <= A.reject32 * A.boxes[e].he) {
            // Final Newton steps at FP64 accuracy: compensated (double-float)
            // residuals on the split element-local coordinates, on the FP32
            // pipes, with the FP32 Jacobian and the active-set step.  A step
            // that is still large is taken as computed in FP32; once it is
            // small, the 3x3 solve is repeated in FP64, and an FP64 step within
            // the tolerance confirms convergence: r is kept with its own
            // residual (as in chord64).  An FP64 step s above the tolerance ct
            // but at most kTake * ct is taken, and the residual at r + s is
            // the linear model f + J s: the Jacobian (FP32, from the last FP32
            // iterate) has a relative error eps of at most ~1e-4, so r + s is
            // within eps |s| <= 0.1 ct of the solution and f + J s within
            // eps |J s| of its residual -- a further compensated residual
            // would only confirm this.  Unconfirmed after A.refine residuals:
            // the pair goes to the full FP64 Newton.
            const ElemPtr<float> lo32 = {A.coords32lo + (int64_t)e * n3, A.coords32lo + (A.E + e) * n3,
                                         A.coords32lo + (2 * A.E + e) * n3};
            res = -1.0;
            for (int it = 0; it < A.refine; ++it) {
                float f[3], d32[3];
                resid_df<n>(el32, lo32, tab, r, xd, f);
                const double fd[3] = {(double)f[0], (double)f[1], (double)f[2]};
                if (f[0] == 0.0f && f[1] == 0.0f && f[2] == 0.0f) {   // exact hit
                    res = 0.0;
                    break;
                }
                // the active set is decided on r itself: a coordinate just inside
                // a bound must not round onto it (it would be frozen off the bound)
                const float rf[3] = {f32_inside(r[0]), f32_inside(r[1]), f32_inside(r[2])};
                if (gn_step<float>(J32, f, rf, d32) == 0) {  // KKT point at a vertex
                    res = sqrt(fd[0] * fd[0] + fd[1] * fd[1] + fd[2] * fd[2]);
                    break;
                }
                double d[3] = {(double)d32[0], (double)d32[1], (double)d32[2]};
                const bool small = fmaxf(fabsf(d32[0]), fmaxf(fabsf(d32[1]), fabsf(d32[2]))) <= (float)kConfirm;
                if (small) {
                    double J[9];
#pragma unroll
                    for (int k = 0; k < 9; ++k) J[k] = (double)J32[k];
                    if (gn_step<double>(J, fd, r, d) == 0) {
                        res = sqrt(fd[0] * fd[0] + fd[1] * fd[1] + fd[2] * fd[2]);
                        break;
                    }
                    double rn[3];
                    box_step<double>(r, d, rn);
                    const double sn = fmax(fabs(rn[0] - r[0]), fmax(fabs(rn[1] - r[1]), fabs(rn[2] - r[2])));
                    const double ct = chord_tol_df(J, A.boxes[e].he);
                    if (sn <= ct) {
                        res = sqrt(fd[0] * fd[0] + fd[1] * fd[1] + fd[2] * fd[2]);
                        break;
                    }
                    if (sn <= kTake * ct) {
                        double g[3];
#pragma unroll
                        for (int a = 0; a < 3; ++a)
                            g[a] = fd[a] + J[3 * a] * (rn[0] - r[0]) + J[3 * a + 1] * (rn[1] - r[1]) +
                                   J[3 * a + 2] * (rn[2] - r[2]);
                        r[0] = rn[0]; r[1] = rn[1]; r[2] = rn[2];
                        res = sqrt(g[0] * g[0] + g[1] * g[1] + g[2] * g[2]);
                        break;
                    }
                    r[0] = rn[0]; r[1] = rn[1]; r[2] = rn[2];
                } else {
                    double rn[3];
                    box_step<double>(r, d, rn);
                    r[0] = rn[0]; r[1] = rn[1]; r[2] = rn[2];
                }
            }
            if (A.stats) atomicAdd(A.stats + (res < 0.0 ? 3 : 2), 1ULL);
        }
        const int64_t w = result_slot(A, s, q);
        A.prst[w] = r[0];
        A.prst[A.cap + w] = r[1];
        A.prst[2 * A.cap + w] = r[2];
        A.pres[w] = res;
        if (res < 0.0) {
            const int32_t k = atomicAdd(A.fb_count, 1);
            if (k < fbc) fbl[k] = (int32_t)w;
        }
    }
}

template <int n, bool CAP>
__global__ void __launch_bounds__(MixedLB<n, CAP>::threads, MixedLB<n, CAP>::blocks)
    k_newton_mixed(NewtonArgs A, BasisTab tab)
{
    const PairRange R = pair_range(A);
    int32_t* fbl = A.fb_list + (A.s_lo ? R.s0 : 0);
    const int64_t fbc = A.s_lo ? R.s1 - R.s0 : A.fb_cap;
    for_each_pair(A, R, [&](int64_t s) { solve_mixed<n>(A, tab, s, fbl, fbc); });
}

// pass 3 (FP64): full trust-region Newton for the pairs marked -1, from the
// point the earlier passes reached.  These pairs are few and scattered, and
// each solve is a long dependent chain: the kernel is latency-bound.  The
// mixed pass listed them (fb_list); each block is one warp and solves one
// listed pair at a time with the warp-cooperative evaluators, which shortens
// the chain about 16-fold.  If the list overflowed, blocks instead gather the
// marked pairs of chunks of slots into shared memory and solve those one per
// lane.
constexpr int kFullChunk = 8192;
constexpr int kFullSub = 1024;

template <int n>
__device__ __forceinline__ void solve_full64(const NewtonArgs& A, const BasisTab& tab, int64_t w)
{
    constexpr int n3 = n * n * n;
    const int32_t q = listed_pair(A, w);
    const int e = A.pair_elem[q] - A.ebase;
    const int64_t p = pair_point(A.pair_pt[q]);
    const double xs[3] = {A.pts[p], A.pts[A.P + p], A.pts[2 * A.P + p]};
    const ElemPtr<double> el64 = {A.coords + (int64_t)e * n3, A.coords + (A.E + e) * n3,
                                  A.coords + (2 * A.E + e) * n3};
    double r[3] = {A.prst[w], A.prst[A.cap + w], A.prst[2 * A.cap + w]}, J[9];
    bool conv;
    const double res = newton<n, double, true>(el64, tab, xs, r, J, A.max_newton, conv);
    A.prst[w] = r[0];
    A.prst[A.cap + w] = r[1];
    A.prst[2 * A.cap + w] = r[2];
    A.pres[w] = res;
}

template <int n>
__global__ void __launch_bounds__(32) k_newton64_full(NewtonArgs A, BasisTab tab)
{
    const PairRange R = pair_range(A);
    const int32_t* fbl = A.fb_list + (A.s_lo ? R.s0 : 0);
    const int64_t fbc = A.s_lo ? R.s1 - R.s0 : A.fb_cap;
    const int64_t nfb = *A.fb_count;
    if (nfb <= fbc) {
        // one warp (this block) per listed pair
        constexpr int n3 = n * n * n;
        for (int64_t t = blockIdx.x; t < nfb; t += gridDim.x) {
            const int64_t w = fbl[t];
            const int32_t q = listed_pair(A, w);
            const int e = A.pair_elem[q] - A.ebase;
            const int64_t p = pair_point(A.pair_pt[q]);
            const double xs[3] = {A.pts[p], A.pts[A.P + p], A.pts[2 * A.P + p]};
            const ElemPtr<double> el64 = {A.coords + (int64_t)e * n3, A.coords + (A.E + e) * n3,
                                          A.coords + (2 * A.E + e) * n3};
            double r[3] = {A.prst[w], A.prst[A.cap + w], A.prst[2 * A.cap + w]}, J[9];
            bool conv;
            const double res = newton<n, double, true, true>(el64, tab, xs, r, J, A.max_newton, conv);
            if (threadIdx.x == 0) {
                A.prst[w] = r[0];
                A.prst[A.cap + w] = r[1];
                A.prst[2 * A.cap + w] = r[2];
                A.pres[w] = res;
            }
        }
        return;
    }
    __shared__ int32_t list[kFullSub];
    __shared__ int count;
    for (int64_t base = R.s0 + (int64_t)blockIdx.x * kFullChunk; base < R.s1; base += (int64_t)gridDim.x * kFullChunk) {
        const int64_t cend = base + kFullChunk < R.s1 ? base + kFullChunk : R.s1;
        for (int64_t sb = base; sb < cend; sb += kFullSub) {
            if (threadIdx.x == 0) count = 0;
            __syncthreads();
            const int64_t end = sb + kFullSub < cend ? sb + kFullSub : cend;
            for (int64_t s = sb + threadIdx.x; s < end; s += blockDim.x) {
                const int64_t w = result_slot(A, s, A.order[s]);
                if (A.pres[w] < 0.0) list[atomicAdd(&count, 1)] = (int32_t)w;
            }
            __syncthreads();
            const int m = count;
            for (int t = threadIdx.x; t < m; t += blockDim.x) solve_full64<n>(A, tab, list[t]);
            __syncthreads();
        }
    }
}

template <int n>
__global__ void __launch_bounds__(256) k_newton(NewtonArgs A, BasisTab tab)
{
    const PairRange R = pair_range(A);
    int32_t* fbl = A.fb_list + (A.s_lo ? R.s0 : 0);
    const int64_t fbc = A.s_lo ? R.s1 - R.s0 : A.fb_cap;
    for_each_pair(A, R, [&](int64_t s) { solve_pair<n>(A, tab, s, fbl, fbc); });
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static ScreenArgs screen_args(const FindArgs& a)
{
    ScreenArgs s;
    s.P = a.P;
    s.pts = a.pts;
    s.qsess = a.qsess;
    s.sub = a.sub;
    s.boxes = a.boxes;
    s.boxes32 = a.boxes32;
    s.g = *a.grid;
    s.cell_start = a.cell_start;
    s.cell_elems = a.cell_elems;
    s.cnt = a.cnt;
    s.off = a.off;
    s.pair_elem = a.pair_elem;
    s.pair_pt = a.pair_pt;
    s.cap = a.cap;
    s.stride = a.pts_stride;
    s.pt_base = a.pt_base;
    s.elem_base = a.elem_base;
    s.mask = a.smask;
    return s;
}

// grid for `work` items; with a persistent block count the kernels loop
// grid-stride over a count that only the device knows
static unsigned grid_for(int64_t work, int block, int persistent)
{
    int64_t g = (work + block - 1) / block;
    if (persistent > 0 && g > persistent) g = persistent;
    return (unsigned)(g < 1 ? 1 : g);
}

cudaError_t find_count(const FindArgs& a, const BasisTab&, const FindParams&, cudaStream_t s)
{
    ScreenArgs sa = screen_args(a);
    if (a.boxes32)
        k_screen<false, true><<<(unsigned)((a.P + 255) / 256), 256, 0, s>>>(sa);
    else
        k_screen<false, false><<<(unsigned)((a.P + 255) / 256), 256, 0, s>>>(sa);
    count_launch();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    return scan_exclusive(a.cnt, a.off, a.P, a.scan_tmp, s);
}

cudaError_t find_screen_count(const FindArgs& a, cudaStream_t s)
{
    ScreenArgs sa = screen_args(a);
    if (a.boxes32)
        k_screen<false, true><<<(unsigned)((a.P + 255) / 256), 256, 0, s>>>(sa);
    else
        k_screen<false, false><<<(unsigned)((a.P + 255) / 256), 256, 0, s>>>(sa);
    count_launch();
    return cudaGetLastError();
}

cudaError_t find_emit(const FindArgs& a, cudaStream_t s)
{
    ScreenArgs sa = screen_args(a);
    if (a.boxes32)
        k_screen<true, true><<<(unsigned)((a.P + 255) / 256), 256, 0, s>>>(sa);
    else
        k_screen<true, false><<<(unsigned)((a.P + 255) / 256), 256, 0, s>>>(sa);
    count_launch();
    return cudaGetLastError();
}

// Newton stage (and the mixed form's FP64 fallback) over the pairs of a:
// all live pairs, or (batch groups, a.s_lo set) the group's sorted range.
// grid == 0: sized from npairs and the block (persistent when the caller
// gave persistent_blocks).
template <int n>
static cudaError_t newton_n(const FindArgs& a, int64_t npairs, const BasisTab& tab, const FindParams& fp, int block,
                            unsigned grid, cudaStream_t s)
{
    NewtonArgs na;
    na.dcount = a.off + a.P;
    na.E = a.E;
    na.order = a.order;
    na.pair_elem = a.pair_elem;
    na.pair_pt = a.pair_pt;
    na.P = a.P;
    na.pts = a.pts;
    na.coords = a.coords;
    na.coords32 = a.coords32;
    na.coords32lo = a.coords32lo;
    na.boxes = a.boxes;
    na.pres = a.pres;
    na.prst = a.prst;
    na.cap = a.cap;
    na.reject32 = 1e-4;
    na.max_newton = fp.max_newton;
    na.refine = fp.refine;
    na.first_pass = a.batch ? kFirstPassBatch : kFirstPass;
    na.stats = a.stats;
    na.warm_elem = a.warm_elem;
    na.warm_rst = a.warm_rst;
    na.fb_count = nullptr;
    na.fb_list = nullptr;
    na.fb_cap = 0;
    na.s_lo = a.s_lo;
    na.s_hi = a.s_hi;
    na.ebase = a.ebase;
    na.queue = a.queue;
    na.tile = a.tile > 0 ? a.tile : block;
    na.pstate = nullptr;
    na.walk = a.inv != nullptr;
    cudaError_t err;
    if (a.queue && (err = cudaMemsetAsync(a.queue, 0, sizeof(int32_t), s)) != cudaSuccess) return err;
    if (grid == 0) grid = grid_for(npairs, block, a.persistent_blocks);
    if (fp.mixed) {
        if (a.s_lo) {
            // batch group: its own counter; its list from the group's first sorted position
            na.fb_count = a.fb_count;
            na.fb_list = a.fb_list;
        } else {
            // fallback list: the per-point counts (free after the scan) hold
            // the slots, the first scan scratch word (free after the sort) the count
            na.fb_count = a.scan_tmp;
            na.fb_list = a.cnt;
            na.fb_cap = a.P;
        }
        if ((err = cudaMemsetAsync(na.fb_count, 0, sizeof(int32_t), s)) != cudaSuccess) return err;
        bool capped = false;
        if constexpr (n <= 10) {
            if (block <= 128 && (a.persistent_blocks == 0 || a.queue)) {
                const unsigned g = a.persistent_blocks == 0 && !a.queue ? grid_for(npairs, block, 0) : grid;
                k_newton_mixed<n, true><<<g, block, 0, s>>>(na, tab);
                capped = true;
            }
        }
        if (!capped) k_newton_mixed<n, false><<<grid, block, 0, s>>>(na, tab);
        // blocks of one warp: enough for a list of up to 38,912 pairs in one
        // pass, and for the chunked path over every slot if it overflowed
        const unsigned gfull = (unsigned)std::max<int64_t>(
            1216, a.persistent_blocks > 0 || a.s_lo ? 0 : (npairs + kFullChunk - 1) / kFullChunk);
        k_newton64_full<n><<<gfull, 32, 0, s>>>(na, tab);
        count_launch(2);
    } else {
        na.pstate = a.pstate;
        if (a.pstate) {
            if (a.s_lo) {
                na.fb_count = a.fb_count;
                na.fb_list = a.fb_list;
            } else {
                na.fb_count = a.scan_tmp;
                na.fb_list = a.cnt;
                na.fb_cap = a.P;
            }
            if ((err = cudaMemsetAsync(na.fb_count, 0, sizeof(int32_t), s)) != cudaSuccess) return err;
        }
        k_newton<n><<<grid, block, 0, s>>>(na, tab);
        count_launch();
        if (a.pstate) {
            // the resumed solves: one per thread over the list (at most the
            // pairs of the first pass), sized like the first pass's grid
            k_newton_resume<n><<<std::max(1u, grid / 2), 128, 0, s>>>(na, tab);
            count_launch();
        }
    }
    return cudaGetLastError();
}

// Few pairs (a launch of fewer than two blocks per SM at `block` threads):
// smaller blocks, down to one warp, so that every SM gets work.  The block
// size changes only the schedule, not any pair's result.
static int spread_block(int64_t npairs, int block)
{
    static int nsm = 0;
    if (nsm == 0) {
        int dev = 0, k = 0;
        if (cudaGetDevice(&dev) == cudaSuccess &&
            cudaDeviceGetAttribute(&k, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && k > 0)
            nsm = k;
        else
            return block;
    }
    while (block > 32 && (npairs + block - 1) / block < 2 * nsm) block >>= 1;
    return block;
}

template <int n>
static cudaError_t solve_n(const FindArgs& a, int64_t npairs, const BasisTab& tab, const FindParams& fp, int block,
                           cudaStream_t s)
{
    if (npairs > 0) {
        if (a.ev[2]) cudaEventRecord(a.ev[2], s);
        if (a.persistent_blocks == 0) block = spread_block(npairs, block);
        cudaError_t err = newton_n<n>(a, npairs, tab, fp, block, 0, s);
        if (err != cudaSuccess) return err;
        if (a.ev[3]) cudaEventRecord(a.ev[3], s);
    }
    RankArgs ra;
    ra.P = a.P;
    ra.E = a.E;
    ra.off = a.off;
    ra.pair_elem = a.pair_elem;
    ra.pres = a.pres;
    ra.prst = a.prst;
    ra.cap = a.cap;
    ra.sub = a.sub;
    ra.boxes = a.boxes;
    ra.dist = a.dist;
    ra.code = a.code;
    ra.osub = a.osub;
    ra.oelem = a.oelem;
    ra.rst = a.rst;
    ra.dist2 = a.dist2;
    ra.pair_pt = a.pair_pt;
    ra.F = a.eval.F;
    ra.out = a.eval.out;
    ra.band = a.band;
    ra.inv = a.inv;
    if (a.ev[4]) cudaEventRecord(a.ev[4], s);
    k_rank<n, 3><<<(unsigned)((a.P + 127) / 128), 128, 0, s>>>(ra, fp, tab);
    count_launch();
    if (a.ev[5]) cudaEventRecord(a.ev[5], s);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || a.eval.F == 0 || npairs == 0) return err;
    if (a.ev[6]) cudaEventRecord(a.ev[6], s);
    err = launch_eval_pairs(n, a.E, a.P, a.off + a.P, a.cap, a.order, a.pair_elem, a.pair_pt, a.prst, a.eval, tab,
                            grid_for(npairs, 128, a.persistent_blocks ? 4 * a.persistent_blocks : 0), s, nullptr,
                            nullptr, 0, a.inv != nullptr);
    if (a.ev[7]) cudaEventRecord(a.ev[7], s);
    return err;
}

cudaError_t find_sort(const FindArgs& a, int64_t npairs, cudaStream_t s)
{
    cudaError_t err = cudaSuccess;
    if (npairs > 0) {
        if (a.ev[0]) cudaEventRecord(a.ev[0], s);
        err = cudaMemsetAsync(a.ecount, 0, sizeof(int32_t) * a.E, s);
        if (err != cudaSuccess) return err;
        const unsigned g256 = grid_for(npairs, 256, a.persistent_blocks ? 4 * a.persistent_blocks : 0);
        k_ehist<<<g256, 256, 0, s>>>(a.off + a.P, a.cap, a.pair_elem, a.ecount);
        count_launch();
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if ((err = scan_exclusive(a.ecount, a.estart, a.E, a.scan_tmp, s)) != cudaSuccess) return err;
        if ((err = cudaMemsetAsync(a.ecount, 0, sizeof(int32_t) * a.E, s)) != cudaSuccess) return err;
        k_escatter<<<g256, 256, 0, s>>>(a.off + a.P, a.cap, a.pair_elem, a.estart, a.ecount, a.order, a.inv);
        count_launch();
        if ((err = cudaGetLastError()) != cudaSuccess) return err;
        if (a.ev[1]) cudaEventRecord(a.ev[1], s);
    }
    return err;
}

cudaError_t find_solve(const FindArgs& a, int64_t npairs, const BasisTab& tab, const FindParams& fp, int block,
                       cudaStream_t s)
{
    cudaError_t err = find_sort(a, npairs, s);
    if (err != cudaSuccess) return err;
    switch (a.n) {
#define FP_CASE(NN) \
    case NN: return solve_n<NN>(a, npairs, tab, fp, block, s);
        FP_CASE(2) FP_CASE(3) FP_CASE(4) FP_CASE(5) FP_CASE(6) FP_CASE(7) FP_CASE(8) FP_CASE(9)
        FP_CASE(10) FP_CASE(11) FP_CASE(12) FP_CASE(13) FP_CASE(14) FP_CASE(15) FP_CASE(16)
#undef FP_CASE
        default: return cudaErrorInvalidValue;
    }
}

// Newton stage of one order-n group of a batch (a.s_lo / a.s_hi / a.ebase
// set), on `grid` blocks of `block` threads drawing work items of a.tile
// sorted positions from the counter a.queue.
cudaError_t find_newton_group(const FindArgs& a, const BasisTab& tab, const FindParams& fp, int block, unsigned grid,
                              cudaStream_t s)
{
    switch (a.n) {
#define FP_CASE(NN) \
    case NN: return newton_n<NN>(a, a.cap, tab, fp, block, grid, s);
        FP_CASE(2) FP_CASE(3) FP_CASE(4) FP_CASE(5) FP_CASE(6) FP_CASE(7) FP_CASE(8) FP_CASE(9)
        FP_CASE(10) FP_CASE(11) FP_CASE(12) FP_CASE(13) FP_CASE(14) FP_CASE(15) FP_CASE(16)
#undef FP_CASE
        default: return cudaErrorInvalidValue;
    }
}

// Blocks of `block` threads of the Newton kernel a group of order n - 1
// would launch (find_newton_group) that fit one SM at once.
template <int n>
static int newton_fit(bool mixed, int block)
{
    int k = 0;
    cudaError_t e;
    if (!mixed) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, k_newton<n>, block, 0);
    } else if (n <= 10 && block <= 128) {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, k_newton_mixed<n, true>, block, 0);
    } else {
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&k, k_newton_mixed<n, false>, block, 0);
    }
    return e == cudaSuccess ? k : 1;
}

int newton_blocks_per_sm(int n, bool mixed, int block)
{
    switch (n) {
#define FP_CASE(NN) \
    case NN: return newton_fit<NN>(mixed, block);
        FP_CASE(2) FP_CASE(3) FP_CASE(4) FP_CASE(5) FP_CASE(6) FP_CASE(7) FP_CASE(8) FP_CASE(9)
        FP_CASE(10) FP_CASE(11) FP_CASE(12) FP_CASE(13) FP_CASE(14) FP_CASE(15) FP_CASE(16)
#undef FP_CASE
        default: return 1;
    }
}

// Newton + classification on pairs already in `a.order` (no pair sort).
cudaError_t find_solve_unsorted(const FindArgs& a, int64_t npairs, const BasisTab& tab, const FindParams& fp,
                                int block, cudaStream_t s)
{
    switch (a.n) {
#define FP_CASE(NN) \
    case NN: return solve_n<NN>(a, npairs, tab, fp, block, s);
        FP_CASE(2) FP_CASE(3) FP_CASE(4) FP_CASE(5) FP_CASE(6) FP_CASE(7) FP_CASE(8) FP_CASE(9)
        FP_CASE(10) FP_CASE(11) FP_CASE(12) FP_CASE(13) FP_CASE(14) FP_CASE(15) FP_CASE(16)
#undef FP_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fpg
