// fp_find2.cu -- the 2D (quadrilateral) variant of the path, for the
// paper's 2D overset examples (Sec. 3): the same steps as the hexahedral
// path with the double sum x^e(r,s) = sum_ij x_ij h_i(r) h_j(s), FP64 form.
//
//  k_hull2        per element: node box, h_e, vertex-averaged affine frame,
//                 Bernstein coefficients (a rigorous hull), padded axis box
//                 and box in the affine frame.  Written into ElemBox with a
//                 neutral third axis (c_z = 0, zero-width z bounds, identity
//                 z row of the frame), so the hash-grid and global-box
//                 kernels of the 3D path serve both.
//  k_screen2      hash cell -> candidates, session filter, both boxes;
//                 counts, then writes the (point, element) pairs.
//  (pair sort)    shared with the 3D path.
//  k_newton2<n>   box-constrained trust-region Newton in [-1,1]^2 with an
//                 active set, from the nearest mapped GLL node (or a warm
//                 start); chord steps with a fixed Jacobian confirm
//                 convergence.
//  k_rank<n,2>    classification and ownership (fp_rank.cuh).
//  k_eval2 / k_eval_pairs2   findpts_eval by sum factorisation, by point or
//                 fused in the element-sorted pair order.
#include <algorithm>

#include "fp_common.cuh"
#include "fp_internal.h"
#include "fp_rank.cuh"

namespace fpg {

// ---------------------------------------------------------------------------
// hull
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_min(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

__device__ __forceinline__ double warp_max(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// One warp per element; shared memory: per warp 3 * n^2 doubles (two
// coefficient arrays and one transform buffer).
__global__ void k_hull2(int n, int64_t E, const double* __restrict__ coords, const double* __restrict__ binv,
                        double pad_border, double pad_conv, ElemBox* __restrict__ boxes,
                        double* __restrict__ nodebox)
{
    extern __shared__ double sm2[];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t e = blockIdx.x * (int64_t)(blockDim.x >> 5) + w;
    if (e >= E) return;                                  // whole warps exit together
    const int n2 = n * n, N = n - 1;
    double* B[2] = {sm2 + (size_t)w * 3 * n2, sm2 + (size_t)w * 3 * n2 + n2};
    double* tmp = sm2 + (size_t)w * 3 * n2 + 2 * n2;
    const double* X[2] = {coords + e * n2, coords + (E + e) * n2};

    double lo[2], hi[2];
    for (int a = 0; a < 2; ++a) {
        double mn = INFINITY, mx = -INFINITY;
        for (int q = lane; q < n2; q += 32) {
            mn = fmin(mn, X[a][q]);
            mx = fmax(mx, X[a][q]);
        }
        lo[a] = warp_min(mn);
        hi[a] = warp_max(mx);
    }
    const double dx = hi[0] - lo[0], dy = hi[1] - lo[1];
    const double he = sqrt(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));

    // affine frame from the 4 vertices: c = mean, column b = (sum of the
    // vertices signed by their end along reference direction b) / 4
    double c[2], A[4];
    for (int a = 0; a < 2; ++a) {
        const double v00 = X[a][0], v10 = X[a][N], v01 = X[a][n * N], v11 = X[a][N + n * N];
        c[a] = 0.25 * (((v00 + v10) + v01) + v11);
        A[2 * a + 0] = 0.25 * (((v10 - v00) + v11) - v01);
        A[2 * a + 1] = 0.25 * (((v01 - v00) + v11) - v10);
    }
    const double det = A[0] * A[3] - A[1] * A[2];
    const double scale = fmax(dx, dy);
    double Ai[4];
    if (!(fabs(det) > 1e-12 * scale * scale)) {          // degenerate: axis frame
        Ai[0] = dx > 0 ? 2.0 / dx : 1.0;
        Ai[1] = 0.0;
        Ai[2] = 0.0;
        Ai[3] = dy > 0 ? 2.0 / dy : 1.0;
    } else {
        const double id = 1.0 / det;
        Ai[0] = A[3] * id;
        Ai[1] = -A[1] * id;
        Ai[2] = -A[2] * id;
        Ai[3] = A[0] * id;
    }

    // Bernstein coefficients of (x - c): binv along i, then along j
    double cmax = 0.0;
    for (int a = 0; a < 2; ++a) {
        for (int q = lane; q < n2; q += 32) {
            const double v = X[a][q] - c[a];
            tmp[q] = v;
            cmax = fmax(cmax, fabs(v));
        }
        __syncwarp();
        for (int q = lane; q < n2; q += 32) {
            const int i = q % n, j = q / n;
            double s = 0.0;
            for (int t = 0; t < n; ++t) s += binv[i * n + t] * tmp[t + n * j];
            B[a][q] = s;
        }
        __syncwarp();
        for (int q = lane; q < n2; q += 32) {
            const int i = q % n, j = q / n;
            double s = 0.0;
            for (int t = 0; t < n; ++t) s += binv[j * n + t] * B[a][i + n * t];
            tmp[q] = s;
        }
        __syncwarp();
        for (int q = lane; q < n2; q += 32) B[a][q] = tmp[q];
        __syncwarp();
    }
    cmax = warp_max(cmax);
    double amin[2] = {INFINITY, INFINITY}, amax[2] = {-INFINITY, -INFINITY};
    double omin[2] = {INFINITY, INFINITY}, omax[2] = {-INFINITY, -INFINITY};
    for (int q = lane; q < n2; q += 32) {
        const double b0 = B[0][q], b1 = B[1][q];
        amin[0] = fmin(amin[0], b0); amax[0] = fmax(amax[0], b0);
        amin[1] = fmin(amin[1], b1); amax[1] = fmax(amax[1], b1);
        const double y0 = Ai[0] * b0 + Ai[1] * b1, y1 = Ai[2] * b0 + Ai[3] * b1;
        omin[0] = fmin(omin[0], y0); omax[0] = fmax(omax[0], y0);
        omin[1] = fmin(omin[1], y1); omax[1] = fmax(omax[1], y1);
    }
    for (int a = 0; a < 2; ++a) {
        amin[a] = warp_min(amin[a]);
        amax[a] = warp_max(amax[a]);
        omin[a] = warp_min(omin[a]);
        omax[a] = warp_max(omax[a]);
    }
    if (lane == 0) {
        ElemBox bx;
        const double pphys = pad_border * he + pad_conv * cmax + 1e-9 * he;
        const double ainf = fmax(fabs(Ai[0]) + fabs(Ai[1]), fabs(Ai[2]) + fabs(Ai[3]));
        const double pfr = ainf * pphys + 1e-12;
        for (int a = 0; a < 2; ++a) {
            bx.c[a] = c[a];
            bx.blo[a] = c[a] + amin[a] - pphys;
            bx.bhi[a] = c[a] + amax[a] + pphys;
            bx.olo[a] = omin[a] - pfr;
            bx.ohi[a] = omax[a] + pfr;
        }
        bx.c[2] = 0.0;
        bx.blo[2] = bx.bhi[2] = 0.0;
        bx.olo[2] = bx.ohi[2] = 0.0;
        for (int q = 0; q < 9; ++q) bx.Ai[q] = 0.0;
        bx.Ai[0] = Ai[0]; bx.Ai[1] = Ai[1];
        bx.Ai[3] = Ai[2]; bx.Ai[4] = Ai[3];
        bx.Ai[8] = 1.0;
        bx.he = he;
        bx.spare = 0.0;
        boxes[e] = bx;
        nodebox[6 * e + 0] = lo[0]; nodebox[6 * e + 1] = lo[1]; nodebox[6 * e + 2] = 0.0;
        nodebox[6 * e + 3] = hi[0]; nodebox[6 * e + 4] = hi[1]; nodebox[6 * e + 5] = 0.0;
    }
}

cudaError_t launch_hull2(int n, int64_t E, const double* coords, const double* binv, double pad_border,
                         double pad_conv, ElemBox* boxes, double* nodebox, cudaStream_t s)
{
    constexpr int warps = 4;
    const size_t smem = sizeof(double) * 3 * (size_t)n * n * warps;
    cudaError_t err = cudaFuncSetAttribute(k_hull2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_hull2<<<(unsigned)((E + warps - 1) / warps), 32 * warps, smem, s>>>(n, E, coords, binv, pad_border, pad_conv,
                                                                          boxes, nodebox);
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// default distance field D^k in 2D: boundary edges of each subdomain (edges
// whose two end points match no edge of another element of the same
// subdomain), then the distance from every node to the nearest GLL node of a
// boundary edge of its own subdomain.  Edge f = 0,1: r = -1,+1 (i = 0, N),
// f = 2,3: s = -1,+1 (j = 0, N).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int edge_node2(int n, int f, int a)
{
    const int end = (f & 1) ? n - 1 : 0;
    return (f >> 1) == 0 ? end + n * a : a + n * end;
}

// end points of every edge, sorted lexicographically: ec [4E][4]
__global__ void k_edge_corners(int n, int64_t E, const double* __restrict__ coords, double* __restrict__ ec)
{
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= 4 * E) return;
    const int64_t e = f / 4;
    const int k = (int)(f % 4), n2 = n * n;
    const int i0 = edge_node2(n, k, 0), i1 = edge_node2(n, k, n - 1);
    double a0 = coords[e * n2 + i0], a1 = coords[(E + e) * n2 + i0];
    double b0 = coords[e * n2 + i1], b1 = coords[(E + e) * n2 + i1];
    if (b0 < a0 || (b0 == a0 && b1 < a1)) {
        double t = a0; a0 = b0; b0 = t;
        t = a1; a1 = b1; b1 = t;
    }
    ec[4 * f + 0] = a0; ec[4 * f + 1] = a1; ec[4 * f + 2] = b0; ec[4 * f + 3] = b1;
}

// candidates from the hash cell of the edge midpoint (a neighbour's padded
// box contains its whole edge, hence the midpoint of the chord)
__global__ void k_edge_boundary(int64_t E, const double* __restrict__ ec, const int32_t* __restrict__ sub,
                                HashGrid g, const int32_t* __restrict__ cstart, const int32_t* __restrict__ celems,
                                int32_t* __restrict__ nbnd)
{
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= 4 * E) return;
    const int64_t e = f / 4;
    const double* me = ec + 4 * f;
    const double cx = 0.5 * (me[0] + me[2]), cy = 0.5 * (me[1] + me[3]);
    const int ci = min(max((int)floor((cx - g.org[0]) * g.inv[0]), 0), g.dim[0] - 1);
    const int cj = min(max((int)floor((cy - g.org[1]) * g.inv[1]), 0), g.dim[1] - 1);
    const int64_t cidx = ci + (int64_t)g.dim[0] * cj;
    int shared = 0;
    for (int q = cstart[cidx]; q < cstart[cidx + 1] && !shared; ++q) {
        const int e2 = celems[q];
        if (e2 == e || sub[e2] != sub[e]) continue;
        for (int k2 = 0; k2 < 4 && !shared; ++k2) {
            const double* ot = ec + 4 * ((int64_t)e2 * 4 + k2);
            shared = ot[0] == me[0] && ot[1] == me[1] && ot[2] == me[2] && ot[3] == me[3];
        }
    }
    nbnd[f] = shared ? 0 : 1;
}

// the n GLL nodes of every boundary edge: positions [2][nb], subdomain [nb]
__global__ void k_edge_gather(int n, int64_t E, const double* __restrict__ coords, const int32_t* __restrict__ sub,
                              const int32_t* __restrict__ bnd_off, double* __restrict__ bx, int32_t* __restrict__ bs,
                              int64_t nb)
{
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f >= 4 * E) return;
    const int o = bnd_off[f];
    if (bnd_off[f + 1] == o) return;
    const int64_t e = f / 4;
    const int k = (int)(f % 4), n2 = n * n;
    for (int a = 0; a < n; ++a) {
        const int idx = edge_node2(n, k, a);
        const int64_t m = (int64_t)o * n + a;
        bx[m] = coords[e * n2 + idx];
        bx[nb + m] = coords[(E + e) * n2 + idx];
        bs[m] = sub[e];
    }
}

__global__ void k_dist_default2(int n2, int64_t E, const double* __restrict__ coords, const int32_t* __restrict__ sub,
                                const double* __restrict__ bx, const int32_t* __restrict__ bs, int64_t nb,
                                double* __restrict__ D)
{
    const int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= E * n2) return;
    const int64_t e = q / n2;
    const double x = coords[q], y = coords[E * n2 + q];
    const int s = sub[e];
    double best = INFINITY;
    for (int64_t b = 0; b < nb; ++b) {
        if (bs[b] != s) continue;
        const double dx = x - bx[b], dy = y - bx[nb + b];
        best = fmin(best, __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)));
    }
    D[q] = sqrt(best);
}

cudaError_t launch_dist_default2(int n, int64_t E, const double* coords, const int32_t* sub, const HashGrid& g,
                                 const int32_t* cstart, const int32_t* celems, double* D, int64_t max_pairs,
                                 bool* too_large, cudaStream_t s)
{
    *too_large = false;
    const int64_t F = 4 * E;
    double* ec = nullptr;
    int32_t *nbnd = nullptr, *off = nullptr, *tmp = nullptr;
    double* bx = nullptr;
    int32_t* bs = nullptr;
    int32_t total = 0;
    cudaError_t e = cudaMalloc(&ec, sizeof(double) * 4 * F);
    if (e == cudaSuccess) e = cudaMalloc(&nbnd, sizeof(int32_t) * F);
    if (e == cudaSuccess) e = cudaMalloc(&off, sizeof(int32_t) * (F + 1));
    if (e == cudaSuccess) e = cudaMalloc(&tmp, sizeof(int32_t) * scan_tmp_elems(F));
    if (e == cudaSuccess) {
        const unsigned gf = (unsigned)((F + 127) / 128);
        k_edge_corners<<<gf, 128, 0, s>>>(n, E, coords, ec);
        k_edge_boundary<<<gf, 128, 0, s>>>(E, ec, sub, g, cstart, celems, nbnd);
        count_launch(2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = scan_exclusive(nbnd, off, F, tmp, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, off + F, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    const int64_t nb = (int64_t)total * n;
    if (e == cudaSuccess && (double)E * n * n * (double)nb > (double)max_pairs) *too_large = true;
    if (e == cudaSuccess && !*too_large) {
        e = cudaMalloc(&bx, sizeof(double) * 2 * std::max<int64_t>(nb, 1));
        if (e == cudaSuccess) e = cudaMalloc(&bs, sizeof(int32_t) * std::max<int64_t>(nb, 1));
        if (e == cudaSuccess) {
            const unsigned gf = (unsigned)((F + 127) / 128);
            k_edge_gather<<<gf, 128, 0, s>>>(n, E, coords, sub, off, bx, bs, nb);
            k_dist_default2<<<(unsigned)((E * n * n + 127) / 128), 128, 0, s>>>(n * n, E, coords, sub, bx, bs, nb, D);
            count_launch(2);
            e = cudaGetLastError();
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    }
    cudaFree(ec); cudaFree(nbnd); cudaFree(off); cudaFree(tmp); cudaFree(bx); cudaFree(bs);
    return e;
}

// ---------------------------------------------------------------------------
// screen
// ---------------------------------------------------------------------------
__device__ __forceinline__ bool inside_boxes2(const ElemBox* __restrict__ bp, double x, double y)
{
    const double* b = reinterpret_cast<const double*>(bp);
    // ElemBox layout: c[0..2], Ai[3..11], olo[12..14], ohi[15..17], blo[18..20], bhi[21..23]
    if (x < __ldg(b + 18) || x > __ldg(b + 21) || y < __ldg(b + 19) || y > __ldg(b + 22)) return false;
    const double dx = x - __ldg(b + 0), dy = y - __ldg(b + 1);
    const double v0 = __ldg(b + 3) * dx + __ldg(b + 4) * dy;
    if (v0 < __ldg(b + 12) || v0 > __ldg(b + 15)) return false;
    const double v1 = __ldg(b + 6) * dx + __ldg(b + 7) * dy;
    return !(v1 < __ldg(b + 13) || v1 > __ldg(b + 16));
}

struct Screen2Args {
    int64_t P;
    const double* pts;
    const int32_t* qsess;
    const int32_t* sub;
    const ElemBox* boxes;
    HashGrid g;
    const int32_t* cell_start;
    const int32_t* cell_elems;
    int32_t* cnt;
    const int32_t* off;
    int32_t* pair_elem;
    int32_t* pair_pt;
    int64_t cap;
};

template <bool EMIT>
__global__ void __launch_bounds__(256) k_screen2(Screen2Args A)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= A.P) return;
    const double x = A.pts[p], y = A.pts[A.P + p];
    const int tag = A.qsess ? A.qsess[p] : -1;
    int c = 0;
    const int base = EMIT ? A.off[p] : 0;
    if (isfinite(x) && isfinite(y)) {
        const double u0 = (x - A.g.org[0]) * A.g.inv[0];
        const double u1 = (y - A.g.org[1]) * A.g.inv[1];
        if (u0 >= 0.0 && u1 >= 0.0 && u0 <= (double)A.g.dim[0] && u1 <= (double)A.g.dim[1]) {
            const int i = min((int)u0, A.g.dim[0] - 1);
            const int j = min((int)u1, A.g.dim[1] - 1);
            const int64_t cell = i + (int64_t)A.g.dim[0] * j;      // one cell layer in z
            const int b = __ldg(A.cell_start + cell), en = __ldg(A.cell_start + cell + 1);
            for (int q = b; q < en; ++q) {
                const int e = __ldg(A.cell_elems + q);
                if (tag >= 0 && __ldg(A.sub + e) == tag) continue;
                if (!inside_boxes2(A.boxes + e, x, y)) continue;
                if (EMIT && base + c < A.cap) {
                    A.pair_elem[base + c] = e;
                    A.pair_pt[base + c] = (int32_t)p;
                }
                ++c;
            }
        }
    }
    if (!EMIT) A.cnt[p] = c;
}

static Screen2Args screen2_args(const FindArgs& a)
{
    Screen2Args s;
    s.P = a.P; s.pts = a.pts; s.qsess = a.qsess; s.sub = a.sub; s.boxes = a.boxes; s.g = *a.grid;
    s.cell_start = a.cell_start; s.cell_elems = a.cell_elems; s.cnt = a.cnt; s.off = a.off;
    s.pair_elem = a.pair_elem; s.pair_pt = a.pair_pt; s.cap = a.cap;
    return s;
}

cudaError_t find_count2(const FindArgs& a, cudaStream_t s)
{
    k_screen2<false><<<(unsigned)((a.P + 255) / 256), 256, 0, s>>>(screen2_args(a));
    count_launch();
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess) return err;
    return scan_exclusive(a.cnt, a.off, a.P, a.scan_tmp, s);
}

cudaError_t find_emit2(const FindArgs& a, cudaStream_t s)
{
    k_screen2<true><<<(unsigned)((a.P + 255) / 256), 256, 0, s>>>(screen2_args(a));
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Newton in [-1,1]^2
// ---------------------------------------------------------------------------
template <int n>
__device__ __forceinline__ void eval_fJ2(const double* __restrict__ X0, const double* __restrict__ X1,
                                         const BasisTab& tab, const double (&r)[2], const double (&xs)[2],
                                         double (&f)[2], double (&J)[4])
{
    double hr[n], dr[n], hs[n], ds[n];
    lagrange_hd<n, double>(tab.xi, tab.ci, r[0], hr, dr);
    lagrange_hd<n, double>(tab.xi, tab.ci, r[1], hs, ds);
    double x[2] = {0.0, 0.0}, xr[2] = {0.0, 0.0}, xsd[2] = {0.0, 0.0};
#pragma unroll 1
    for (int j = 0; j < n; ++j) {
#pragma unroll
        for (int a = 0; a < 2; ++a) {
            double v[n];
            load_row<n>((a == 0 ? X0 : X1) + n * j, v);
            double u = 0.0, w = 0.0;
#pragma unroll
            for (int i = 0; i < n; ++i) {
                u = fma(hr[i], v[i], u);
                w = fma(dr[i], v[i], w);
            }
            x[a] = fma(hs[j], u, x[a]);
            xsd[a] = fma(ds[j], u, xsd[a]);
            xr[a] = fma(hs[j], w, xr[a]);
        }
    }
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        f[a] = x[a] - xs[a];
        J[2 * a + 0] = xr[a];
        J[2 * a + 1] = xsd[a];
    }
}

template <int n>
__device__ __forceinline__ void eval_f2(const double* __restrict__ X0, const double* __restrict__ X1,
                                        const BasisTab& tab, const double (&r)[2], const double (&xs)[2],
                                        double (&f)[2])
{
    double hr[n], hs[n];
    lagrange_h<n, double>(tab.xi, tab.ci, r[0], hr);
    lagrange_h<n, double>(tab.xi, tab.ci, r[1], hs);
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        const double* X = a == 0 ? X0 : X1;
        double acc = 0.0;
#pragma unroll 1
        for (int j = 0; j < n; ++j) {
            double v[n];
            load_row<n>(X + n * j, v);
            double u = 0.0;
#pragma unroll
            for (int i = 0; i < n; ++i) u = fma(hr[i], v[i], u);
            acc = fma(hs[j], u, acc);
        }
        f[a] = acc - xs[a];
    }
}

// Gauss-Newton step with an active set (coordinates on a bound whose descent
// direction leaves the square are frozen).  Returns the number of free ones.
__device__ __forceinline__ int gn_step2(const double (&J)[4], const double (&f)[2], const double (&r)[2],
                                        double (&d)[2])
{
    double g[2];
    g[0] = J[0] * f[0] + J[2] * f[1];
    g[1] = J[1] * f[0] + J[3] * f[1];
    bool act[2];
#pragma unroll
    for (int b = 0; b < 2; ++b) act[b] = (r[b] <= -1.0 && g[b] > 0.0) || (r[b] >= 1.0 && g[b] < 0.0);
    int nfree = 0;
    for (int pass = 0; pass < 3; ++pass) {
        d[0] = d[1] = 0.0;
        nfree = (!act[0]) + (!act[1]);
        if (nfree == 0) break;
        bool ok = false;
        if (nfree == 2) {
            const double det = J[0] * J[3] - J[1] * J[2];
            if (det != 0.0 && isfinite(det)) {
                const double id = 1.0 / det;
                d[0] = -(J[3] * f[0] - J[1] * f[1]) * id;
                d[1] = -(J[0] * f[1] - J[2] * f[0]) * id;
                ok = true;
            }
        } else {
            const int p = act[0] ? 1 : 0;
            const double a00 = J[p] * J[p] + J[2 + p] * J[2 + p];
            if (a00 > 0.0) {
                d[p] = -g[p] / a00;
                ok = true;
            }
        }
        if (!ok) {                                       // singular: steepest descent
            if (!act[0]) d[0] = -g[0];
            if (!act[1]) d[1] = -g[1];
        }
        bool grew = false;
#pragma unroll
        for (int b = 0; b < 2; ++b)
            if (!act[b] && ((r[b] <= -1.0 && d[b] < 0.0) || (r[b] >= 1.0 && d[b] > 0.0))) {
                act[b] = true;
                grew = true;
            }
        if (!grew) break;
    }
    return nfree;
}

__device__ __forceinline__ double box_step2(const double (&r)[2], const double (&d)[2], double (&rn)[2])
{
    double t = 1.0;
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        if (d[b] > 0.0 && r[b] + d[b] > 1.0) t = fmin(t, (1.0 - r[b]) / d[b]);
        if (d[b] < 0.0 && r[b] + d[b] < -1.0) t = fmin(t, (-1.0 - r[b]) / d[b]);
    }
#pragma unroll
    for (int b = 0; b < 2; ++b) {
        double v = r[b] + t * d[b];
        if (t < 1.0) {
            if (d[b] > 0.0 && (1.0 - r[b]) / d[b] == t) v = 1.0;
            if (d[b] < 0.0 && (-1.0 - r[b]) / d[b] == t) v = -1.0;
        }
        rn[b] = fmin(1.0, fmax(-1.0, v));
    }
    return t;
}

constexpr double kQuick2 = 1e-4;    // full Newton step that hands over to chord steps
constexpr double kChord2 = 1e-13;   // chord correction that confirms convergence
constexpr double kStop2 = 1e-13;    // accepted step that ends a constrained solve
constexpr double kRhoMin2 = 1e-15;

// Threshold of the chord check: 1e-13 in r, raised to the rounding level of a
// step (2 eps |x*| ||J^-1||_inf) where that is larger, as in the hexahedral
// solver: on small elements far from the origin rounding alone exceeds 1e-13.
__device__ __forceinline__ double chord_tol2(const double (&J)[4], const double (&xs)[2])
{
    const double det = J[0] * J[3] - J[1] * J[2];
    if (!(fabs(det) > 0.0) || !isfinite(det)) return kChord2;
    const double rows = fmax(fabs(J[3]) + fabs(J[1]), fabs(J[2]) + fabs(J[0]));
    const double xm = fmax(fabs(xs[0]), fabs(xs[1]));
    return fmax(kChord2, 4.440892098500626e-16 * xm * rows / fabs(det));
}

template <int n>
__device__ bool chord2(const double* X0, const double* X1, const BasisTab& tab, const double (&xs)[2],
                       double (&r)[2], const double (&J)[4], double& res, int max_chord)
{
    const double tol = chord_tol2(J, xs);
    for (int it = 0; it < max_chord; ++it) {
        double f[2];
        eval_f2<n>(X0, X1, tab, r, xs, f);
        res = sqrt(f[0] * f[0] + f[1] * f[1]);
        if (!(res > 0.0)) return true;
        double d[2];
        if (gn_step2(J, f, r, d) == 0) return true;
        double rn[2];
        box_step2(r, d, rn);
        const double sn = fmax(fabs(rn[0] - r[0]), fabs(rn[1] - r[1]));
        if (sn <= tol) return true;
        r[0] = rn[0];
        r[1] = rn[1];
    }
    return false;
}

// Box-constrained trust-region Newton (Sec. 2.1) in [-1,1]^2: the same
// radius rules, active set and chord hand-over as the hexahedral solver.
template <int n>
__device__ double newton2(const double* X0, const double* X1, const BasisTab& tab, const double (&xs)[2],
                          double (&r)[2], int max_it)
{
    double f[2], J[4];
    eval_fJ2<n>(X0, X1, tab, r, xs, f, J);
    double phi = 0.5 * (f[0] * f[0] + f[1] * f[1]);
    double rho = 1.0;
    int chord_fail = 0;   // after two failed chord checks the trust-region rules alone finish the solve
    for (int it = 0; it < max_it; ++it) {
        if (!(phi > 0.0)) return 0.0;
        double d[2];
        const int nfree = gn_step2(J, f, r, d);
        if (nfree == 0) return sqrt(2.0 * phi);
        const double dn = fmax(fabs(d[0]), fabs(d[1]));
        if (!(dn > 0.0)) return sqrt(2.0 * phi);
        bool full = true;
        if (dn > rho) {
            const double sc = rho / dn;
            d[0] *= sc;
            d[1] *= sc;
            full = false;
        }
        double rn[2];
        if (box_step2(r, d, rn) < 1.0) full = false;
        const double s[2] = {rn[0] - r[0], rn[1] - r[1]};
        const double sn = fmax(fabs(s[0]), fabs(s[1]));
        if (!(sn > 0.0)) return sqrt(2.0 * phi);
        if (full && nfree == 2 && dn <= kQuick2 && chord_fail < 2) {
            double rc[2] = {rn[0], rn[1]};
            double res;
            if (chord2<n>(X0, X1, tab, xs, rc, J, res, 3)) {
                r[0] = rc[0];
                r[1] = rc[1];
                return res;
            }
            r[0] = rc[0];
            r[1] = rc[1];
            ++chord_fail;
            eval_fJ2<n>(X0, X1, tab, r, xs, f, J);
            phi = 0.5 * (f[0] * f[0] + f[1] * f[1]);
            continue;
        }
        double mf[2];
#pragma unroll
        for (int a = 0; a < 2; ++a) mf[a] = f[a] + J[2 * a] * s[0] + J[2 * a + 1] * s[1];
        const double pred = phi - 0.5 * (mf[0] * mf[0] + mf[1] * mf[1]);
        double fn[2], Jn[4];
        eval_fJ2<n>(X0, X1, tab, rn, xs, fn, Jn);
        const double phin = 0.5 * (fn[0] * fn[0] + fn[1] * fn[1]);
        if (sn <= kStop2) {
            if (phin <= phi) {
                r[0] = rn[0];
                r[1] = rn[1];
                phi = phin;
            }
            return sqrt(2.0 * phi);
        }
        if (phin < phi) {
            const double ratio = pred > 0.0 ? (phi - phin) / pred : 0.0;
            r[0] = rn[0];
            r[1] = rn[1];
#pragma unroll
            for (int q = 0; q < 4; ++q) J[q] = Jn[q];
            f[0] = fn[0];
            f[1] = fn[1];
            phi = phin;
            if (ratio > 0.75 && sn >= 0.99 * rho) rho = fmin(2.0 * rho, 2.0);
            else if (ratio < 0.25) rho = 0.25 * sn;
        } else {
            rho = 0.25 * sn;
            if (rho < kRhoMin2) return sqrt(2.0 * phi);
        }
    }
    return sqrt(2.0 * phi);
}

struct Newton2Args {
    const int32_t* dcount;
    int64_t E, P, cap;
    const int32_t* order;
    const int32_t* pair_elem;
    const int32_t* pair_pt;
    const double* pts;
    const double* coords;
    double* pres;
    double* prst;
    int max_newton;
    const int32_t* warm_elem;
    const double* warm_rst;
};

template <int n>
__global__ void __launch_bounds__(256) k_newton2(Newton2Args A, BasisTab tab)
{
    constexpr int n2 = n * n;
    const int64_t t = *A.dcount;
    const int64_t npairs = t < A.cap ? t : A.cap;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < npairs; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = A.order[s];
        const int e = A.pair_elem[q];
        const int64_t p = pair_point(A.pair_pt[q]);
        const double xs[2] = {A.pts[p], A.pts[A.P + p]};
        const double* X0 = A.coords + (int64_t)e * n2;
        const double* X1 = A.coords + (A.E + e) * n2;
        double r[2];
        bool warm = false;
        if (A.warm_elem && A.warm_elem[p] == e) {
            const double w0 = A.warm_rst[p], w1 = A.warm_rst[A.P + p];
            if (fabs(w0) <= 2.0 && fabs(w1) <= 2.0) {
                r[0] = fmin(1.0, fmax(-1.0, w0));
                r[1] = fmin(1.0, fmax(-1.0, w1));
                warm = true;
            }
        }
        if (!warm) {                         // nearest mapped GLL node, ties to the lowest index
            double best = INFINITY;
            int bq = 0;
            for (int qq = 0; qq < n2; ++qq) {
                const double dx = __ldg(X0 + qq) - xs[0], dy = __ldg(X1 + qq) - xs[1];
                const double d2 = dx * dx + dy * dy;
                if (d2 < best) {
                    best = d2;
                    bq = qq;
                }
            }
            r[0] = tab.xi[bq % n];
            r[1] = tab.xi[bq / n];
        }
        const double res = newton2<n>(X0, X1, tab, xs, r, A.max_newton);
        A.pres[q] = res;
        A.prst[q] = r[0];
        A.prst[A.cap + q] = r[1];
    }
}

// ---------------------------------------------------------------------------
// eval
// ---------------------------------------------------------------------------
template <int n>
__device__ __forceinline__ double contract2(const double* __restrict__ F, const double (&hr)[n], const double (&hs)[n])
{
    double acc = 0.0;
#pragma unroll 1
    for (int j = 0; j < n; ++j) {
        double v[n];
        load_row<n>(F + n * j, v);
        double u = 0.0;
#pragma unroll
        for (int i = 0; i < n; ++i) u = fma(hr[i], v[i], u);
        acc = fma(hs[j], u, acc);
    }
    return acc;
}

struct Eval2dArgs {
    int64_t E, P;
    const int32_t* code;
    const int32_t* elem;
    const double* rst;
    int F;
    const double* fields;
    double* out;
};

template <int n>
__global__ void __launch_bounds__(128) k_eval2(Eval2dArgs A, BasisTab tab)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= A.P) return;
    const int e = A.elem[p];
    if (A.code[p] == FP_CODE_NOT_FOUND || A.code[p] == FP_CODE_RETRY || e < 0 || e >= A.E) {
        for (int f = 0; f < A.F; ++f) A.out[(int64_t)f * A.P + p] = __longlong_as_double(0x7ff8000000000000ULL);
        return;
    }
    double hr[n], hs[n];
    lagrange_h<n, double>(tab.xi, tab.ci, A.rst[p], hr);
    lagrange_h<n, double>(tab.xi, tab.ci, A.rst[A.P + p], hs);
    for (int f = 0; f < A.F; ++f)
        A.out[(int64_t)f * A.P + p] = contract2<n>(A.fields + ((int64_t)f * A.E + e) * (n * n), hr, hs);
}

struct EvalPairs2Args {
    int64_t E, P, cap;
    const int32_t* dcount;
    const int32_t* order;
    const int32_t* pair_elem;
    const int32_t* pair_pt;
    const double* prst;
    int F;
    const double* fields;
    double* out;
};

template <int n>
__global__ void __launch_bounds__(128) k_eval_pairs2(EvalPairs2Args A, BasisTab tab)
{
    const int64_t t = *A.dcount;
    const int64_t npairs = t < A.cap ? t : A.cap;
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < npairs; s += (int64_t)gridDim.x * blockDim.x) {
        const int32_t q = A.order[s];
        const int32_t p = A.pair_pt[q];
        if (p < 0) continue;                              // not the point's winning pair
        const int e = A.pair_elem[q];
        double hr[n], hs[n];
        lagrange_h<n, double>(tab.xi, tab.ci, A.prst[q], hr);
        lagrange_h<n, double>(tab.xi, tab.ci, A.prst[A.cap + q], hs);
        for (int f = 0; f < A.F; ++f)
            A.out[(int64_t)f * A.P + p] = contract2<n>(A.fields + ((int64_t)f * A.E + e) * (n * n), hr, hs);
    }
}

cudaError_t launch_eval2(int n, int64_t E, int64_t P, const int32_t* code, const int32_t* elem, const double* rst,
                         int F, const double* fields, double* out, const BasisTab& tab, cudaStream_t s)
{
    if (P == 0) return cudaSuccess;
    Eval2dArgs a{E, P, code, elem, rst, F, fields, out};
    const unsigned grid = (unsigned)((P + 127) / 128);
    switch (n) {
#define FP_CASE(NN) \
    case NN: k_eval2<NN><<<grid, 128, 0, s>>>(a, tab); break;
        FP_CASE(2) FP_CASE(3) FP_CASE(4) FP_CASE(5) FP_CASE(6) FP_CASE(7) FP_CASE(8) FP_CASE(9)
        FP_CASE(10) FP_CASE(11) FP_CASE(12) FP_CASE(13) FP_CASE(14) FP_CASE(15) FP_CASE(16)
#undef FP_CASE
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// solve: sort, Newton, rank, fused eval
// ---------------------------------------------------------------------------
template <int n>
static cudaError_t solve2_n(const FindArgs& a, int64_t npairs, const BasisTab& tab, const FindParams& fp, int block,
                            cudaStream_t s)
{
    if (npairs > 0) {
        Newton2Args na;
        na.dcount = a.off + a.P;
        na.E = a.E; na.P = a.P; na.cap = a.cap;
        na.order = a.order; na.pair_elem = a.pair_elem; na.pair_pt = a.pair_pt;
        na.pts = a.pts; na.coords = a.coords; na.pres = a.pres; na.prst = a.prst;
        na.max_newton = fp.max_newton;
        na.warm_elem = a.warm_elem; na.warm_rst = a.warm_rst;
        const unsigned grid = (unsigned)std::min<int64_t>((npairs + block - 1) / block, 1 << 30);
        if (a.ev[2]) cudaEventRecord(a.ev[2], s);
        k_newton2<n><<<grid, block, 0, s>>>(na, tab);
        count_launch();
        cudaError_t err = cudaGetLastError();
        if (err != cudaSuccess) return err;
        if (a.ev[3]) cudaEventRecord(a.ev[3], s);
    }
    RankArgs ra;
    ra.P = a.P; ra.E = a.E; ra.off = a.off; ra.pair_elem = a.pair_elem; ra.pres = a.pres; ra.prst = a.prst;
    ra.cap = a.cap; ra.sub = a.sub; ra.boxes = a.boxes; ra.dist = a.dist; ra.code = a.code; ra.osub = a.osub;
    ra.oelem = a.oelem; ra.rst = a.rst; ra.dist2 = a.dist2; ra.pair_pt = a.pair_pt; ra.F = a.eval.F;
    ra.out = a.eval.out; ra.band = a.band; ra.inv = nullptr;   // 2D: pair results stay at their slots
    if (a.ev[4]) cudaEventRecord(a.ev[4], s);
    k_rank<n, 2><<<(unsigned)((a.P + 127) / 128), 128, 0, s>>>(ra, fp, tab);
    count_launch();
    if (a.ev[5]) cudaEventRecord(a.ev[5], s);
    cudaError_t err = cudaGetLastError();
    if (err != cudaSuccess || a.eval.F == 0 || npairs == 0) return err;
    if (a.ev[6]) cudaEventRecord(a.ev[6], s);
    EvalPairs2Args ea{a.E, a.P, a.cap, a.off + a.P, a.order, a.pair_elem, a.pair_pt, a.prst, a.eval.F, a.eval.f64,
                      a.eval.out};
    k_eval_pairs2<n><<<(unsigned)std::min<int64_t>((npairs + 127) / 128, 1 << 30), 128, 0, s>>>(ea, tab);
    count_launch();
    if (a.ev[7]) cudaEventRecord(a.ev[7], s);
    return cudaGetLastError();
}

cudaError_t find_solve2(const FindArgs& a, int64_t npairs, const BasisTab& tab, const FindParams& fp, int block,
                        cudaStream_t s)
{
    cudaError_t err = find_sort(a, npairs, s);
    if (err != cudaSuccess) return err;
    switch (a.n) {
#define FP_CASE(NN) \
    case NN: return solve2_n<NN>(a, npairs, tab, fp, block, s);
        FP_CASE(2) FP_CASE(3) FP_CASE(4) FP_CASE(5) FP_CASE(6) FP_CASE(7) FP_CASE(8) FP_CASE(9)
        FP_CASE(10) FP_CASE(11) FP_CASE(12) FP_CASE(13) FP_CASE(14) FP_CASE(15) FP_CASE(16)
#undef FP_CASE
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace fpg
