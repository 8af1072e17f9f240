// fp_rank.cuh -- classification and ownership of a point's candidate pairs
// (Sec. 2.1): INSIDE / BORDER / NOT_FOUND, the lowest element id within a
// subdomain, and the owner by the largest interpolated distance D^k with a
// lower-id tie band.  Shared by the hexahedral and quadrilateral paths.
#pragma once
#include "fp_common.cuh"

namespace fpg {

// ---------------------------------------------------------------------------
// classification and ownership
// ---------------------------------------------------------------------------
struct RankArgs {
    int64_t P;
    int32_t* pair_pt;       // non-winning pairs are marked -1 for the fused eval
    int F;                  // fused eval: write NaN for points without a winner
    double* out;
    int64_t E;
    const int32_t* off;
    const int32_t* pair_elem;
    const double* pres;
    const double* prst;
    int64_t cap;
    const int32_t* sub;
    const ElemBox* boxes;
    const double* dist;
    int32_t* code;
    int32_t* osub;
    int32_t* oelem;
    double* rst;
    double* dist2;
    unsigned long long* band;   // optional [3] near-tie counters (see k_rank), null = off
    const int32_t* inv;         // pair results at sorted positions inv[q] (3D), null: at slots q (2D)
};

// Near-tie ("band") hits of a point's decisions, counted so that a result
// whose ids could depend on rounding is visible:
//   BAND_ACCEPT  a candidate's residual within a factor 2 of tol_accept*h_e
//                (INSIDE or not could differ between two FP64 evaluations)
//   BAND_BORDER  no INSIDE winner and a candidate's residual within a factor
//                2 of tol_border*h_e, or two BORDER candidates within the tie
//                band of the smallest residual (the lowest id decided)
//   BAND_OWNER   two subdomains' delta^k within twice the tie band of the
//                largest (the lower-id rule decided, or nearly did)
enum { BAND_ACCEPT = 0, BAND_BORDER = 1, BAND_OWNER = 2, BAND_KINDS = 3 };

// mark a pair that does not carry its point's result (see pair_point)
__device__ __forceinline__ void mark_loser(int32_t* pp)
{
    const int32_t v = *pp;
    if (v >= 0) *pp = ~v;
}

// D^k interpolated at (e, r) of a DIM-dimensional element (D: n^DIM values)
template <int n, int DIM>
__device__ __forceinline__ double interp_delta(const double* __restrict__ D, const BasisTab& tab, const double* prst,
                                               int64_t cap, int64_t q)
{
    double hr[n], hs[n];
    lagrange_h<n, double>(tab.xi, tab.ci, prst[q], hr);
    lagrange_h<n, double>(tab.xi, tab.ci, prst[cap + q], hs);
    if constexpr (DIM == 2) {
        double acc = 0.0;
#pragma unroll 1
        for (int j = 0; j < n; ++j) {
            double v[n];
            load_row<n>(D + n * j, v);
            double u = 0.0;
#pragma unroll
            for (int i = 0; i < n; ++i) u = fma(hr[i], v[i], u);
            acc = fma(hs[j], u, acc);
        }
        return acc;
    } else {
        double ht[n];
        lagrange_h<n, double>(tab.xi, tab.ci, prst[2 * cap + q], ht);
        return contract<n, double>(D, hr, hs, ht);
    }
}

// The decisions for point p (rst and prst hold DIM rows).  The context C
// gives the per-element data: he(e) (h_e), sub(e), has_dist() and
// delta(e, q) (D^k interpolated at pair q's r), and elem_out(e) (the element
// id written out).
template <int DIM, class Ctx>
__device__ __forceinline__ void rank_point(const RankArgs& A, const FindParams& fp, const Ctx& C, int64_t p)
{
    const int b = A.off[p], en = A.off[p + 1];
    // where pair q's results are kept
    auto W = [&](int q) -> int64_t { return A.inv ? (int64_t)A.inv[q] : (int64_t)q; };
    if (en > A.cap) {                                  // pairs dropped: not searched
        for (int q = b; q < A.cap; ++q) mark_loser(A.pair_pt + q);
        for (int f = 0; f < A.F; ++f) A.out[(int64_t)f * A.P + p] = __longlong_as_double(0x7ff8000000000000ULL);
        A.code[p] = FP_CODE_RETRY;
        A.osub[p] = -1;
        A.oelem[p] = -1;
        for (int a = 0; a < DIM; ++a) A.rst[a * A.P + p] = 0.0;
        A.dist2[p] = INFINITY;
        return;
    }
    // INSIDE winners: lowest element id per subdomain
    unsigned hit = 0;
    bool near_border = false;
    int best_q = -1, nwin = 0;
    double bmin = INFINITY;
    for (int q = b; q < en; ++q) {
        const int e = A.pair_elem[q];
        const double he = C.he(e);
        const double res = A.pres[W(q)];
        if (res >= 0.5 * fp.tol_accept * he && res <= 2.0 * fp.tol_accept * he) hit |= 1u << BAND_ACCEPT;
        if (res >= 0.5 * fp.tol_border * he && res <= 2.0 * fp.tol_border * he) near_border = true;
        if (res <= fp.tol_accept * he) {
            const int s = C.sub(e);
            bool winner = true;
            for (int q2 = b; q2 < en && winner; ++q2) {
                const int e2 = A.pair_elem[q2];
                if (q2 != q && C.sub(e2) == s && e2 < e && A.pres[W(q2)] <= fp.tol_accept * C.he(e2)) winner = false;
            }
            if (winner) {
                ++nwin;
                if (best_q < 0) best_q = q;
            }
        } else if (res <= fp.tol_border * he) {
            bmin = fmin(bmin, res);
        }
    }
    int pick = -1;
    int code = 2;
    if (nwin == 1) {
        pick = best_q;
        code = 0;
    } else if (nwin > 1) {
        // owner = argmax delta^k(x*), ties within the band -> lower subdomain id
        double dmax = -INFINITY;
        int nclose = 0;
        for (int pass = 0; pass < 2; ++pass) {
            int bs = 0x7fffffff;
            for (int q = b; q < en; ++q) {
                const int e = A.pair_elem[q];
                if (!(A.pres[W(q)] <= fp.tol_accept * C.he(e))) continue;
                const int s = C.sub(e);
                bool winner = true;
                for (int q2 = b; q2 < en && winner; ++q2) {
                    const int e2 = A.pair_elem[q2];
                    if (q2 != q && C.sub(e2) == s && e2 < e && A.pres[W(q2)] <= fp.tol_accept * C.he(e2))
                        winner = false;
                }
                if (!winner) continue;
                const double dl = C.has_dist() ? C.delta(e, W(q)) : 0.0;
                if (pass == 0) {
                    dmax = fmax(dmax, dl);
                } else {
                    if (dl >= dmax - 2.0 * fp.band) ++nclose;
                    if (dl >= dmax - fp.band && s < bs) {
                        bs = s;
                        pick = q;
                    }
                }
            }
        }
        if (nclose > 1) hit |= 1u << BAND_OWNER;
        code = 0;
    } else if (bmin < INFINITY) {
        int be = 0x7fffffff, ntie = 0;
        for (int q = b; q < en; ++q) {
            const int e = A.pair_elem[q];
            const double he = C.he(e);
            const double res = A.pres[W(q)];
            if (res > fp.tol_accept * he && res <= fp.tol_border * he && res <= bmin + fp.band) {
                ++ntie;
                if (e < be) {
                    be = e;
                    pick = q;
                }
            }
        }
        if (ntie > 1) hit |= 1u << BAND_BORDER;
        code = 1;
    }
    if (nwin == 0 && near_border) hit |= 1u << BAND_BORDER;
    if (hit && A.band) {
#pragma unroll
        for (int k = 0; k < BAND_KINDS; ++k)
            if (hit & (1u << k)) atomicAdd(A.band + k, 1ULL);
    }
    for (int q = b; q < en; ++q)
        if (q != pick) mark_loser(A.pair_pt + q);
    if (pick < 0)
        for (int f = 0; f < A.F; ++f) A.out[(int64_t)f * A.P + p] = __longlong_as_double(0x7ff8000000000000ULL);
    if (pick >= 0) {
        const int e = A.pair_elem[pick];
        A.code[p] = code;
        A.osub[p] = C.sub(e);
        A.oelem[p] = C.elem_out(e);
        for (int a = 0; a < DIM; ++a) A.rst[a * A.P + p] = A.prst[a * A.cap + W(pick)];
        const double res = A.pres[W(pick)];
        A.dist2[p] = res * res;
    } else {
        A.code[p] = 2;
        A.osub[p] = -1;
        A.oelem[p] = -1;
        for (int a = 0; a < DIM; ++a) A.rst[a * A.P + p] = 0.0;
        A.dist2[p] = INFINITY;
    }
}

// element data of one mesh (a handle)
template <int n, int DIM>
struct RankMesh {
    static constexpr int n3 = DIM == 2 ? n * n : n * n * n;
    const RankArgs& A;
    const BasisTab& tab;
    __device__ __forceinline__ double he(int e) const { return A.boxes[e].he; }
    __device__ __forceinline__ int sub(int e) const { return A.sub[e]; }
    __device__ __forceinline__ bool has_dist() const { return A.dist != nullptr; }
    __device__ __forceinline__ double delta(int e, int64_t q) const
    {
        return interp_delta<n, DIM>(A.dist + (int64_t)e * n3, tab, A.prst, A.cap, q);
    }
    __device__ __forceinline__ int elem_out(int e) const { return e; }
};

// one thread per point
template <int n, int DIM>
__global__ void __launch_bounds__(128) k_rank(RankArgs A, FindParams fp, BasisTab tab)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= A.P) return;
    const RankMesh<n, DIM> C{A, tab};
    rank_point<DIM>(A, fp, C, p);
}

}  // namespace fpg
