// fp_setup.cu -- resident search structures built once per mesh
// (Sec. 2.1: elementwise bounding boxes and a hash table screen candidate
// elements before the Newton solve).
//
//  k_hull      per element: vertex-averaged affine frame, node box and h_e,
//              Bernstein coefficients of the element map (a rigorous hull:
//              the map is a convex combination of them), their axis box and
//              their box in the element's affine frame, both padded.
//  k_reduce_*  global box over all elements.
//  k_hash_*    uniform grid over the global box; CSR cell -> element lists
//              from box overlap (count, scan, fill, per-cell sort).
//  k_face_* / k_dist_default  default nodal distance-to-boundary field D^k.
#include <algorithm>

#include "fp_common.cuh"
#include "fp_internal.h"

namespace fpg {

// ---------------------------------------------------------------------------
// k_hull: one block per element.  Dynamic shared memory: 4 * n^3 doubles
// (three Bernstein coefficient arrays + one transform buffer).
// ---------------------------------------------------------------------------
__device__ __forceinline__ double block_reduce_min(double v, double* sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (l == 0) sh[w] = v;
    __syncthreads();
    double r = sh[0];
    for (int i = 1; i < nw; ++i) r = fmin(r, sh[i]);
    __syncthreads();
    return r;
}

__device__ __forceinline__ double block_reduce_max(double v, double* sh)
{
    return -block_reduce_min(-v, sh);
}

__global__ void k_hull(int n, int64_t E, const double* __restrict__ coords,
                       const double* __restrict__ binv, double pad_border, double pad_conv,
                       ElemBox* __restrict__ boxes, double* __restrict__ nodebox)
{
    extern __shared__ double sm[];
    __shared__ double red[32];
    __shared__ double frame[12];
    const int n3 = n * n * n;
    const int64_t e = blockIdx.x;
    double* B[3] = {sm, sm + n3, sm + 2 * n3};
    double* tmp = sm + 3 * n3;
    const int N = n - 1;

    // node box and h_e (no FMA contraction: matches a plain evaluation)
    double lo[3], hi[3], cmax = 0.0;
    for (int a = 0; a < 3; ++a) {
        const double* X = coords + ((int64_t)a * E + e) * n3;
        double mn = INFINITY, mx = -INFINITY;
        for (int q = threadIdx.x; q < n3; q += blockDim.x) {
            double v = X[q];
            mn = fmin(mn, v);
            mx = fmax(mx, v);
        }
        lo[a] = block_reduce_min(mn, red);
        hi[a] = block_reduce_max(mx, red);
    }
    const double dx = hi[0] - lo[0], dy = hi[1] - lo[1], dz = hi[2] - lo[2];
    const double he = sqrt(__dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)));

    // affine frame from the 8 vertices: c = mean, column b = mean edge vector
    // along reference direction b divided by 2 (r spans [-1,1])
    if (threadIdx.x == 0) {
        double V[8][3];
        for (int v = 0; v < 8; ++v) {
            int i = (v & 1) ? N : 0, j = (v & 2) ? N : 0, k = (v & 4) ? N : 0;
            int q = i + n * (j + n * k);
            for (int a = 0; a < 3; ++a) V[v][a] = coords[((int64_t)a * E + e) * n3 + q];
        }
        double c[3], A[9];
        for (int a = 0; a < 3; ++a) {
            double s = 0.0;
            for (int v = 0; v < 8; ++v) s += V[v][a];
            c[a] = 0.125 * s;
            double er = 0.0, es = 0.0, et = 0.0;
            for (int v = 0; v < 8; ++v) {
                double sr = (v & 1) ? 1.0 : -1.0, ss = (v & 2) ? 1.0 : -1.0, st = (v & 4) ? 1.0 : -1.0;
                er += sr * V[v][a];
                es += ss * V[v][a];
                et += st * V[v][a];
            }
            A[3 * a + 0] = er * 0.125;   // (sum over 4 edges of the difference) / 4 / 2
            A[3 * a + 1] = es * 0.125;
            A[3 * a + 2] = et * 0.125;
        }
        double c00 = A[4] * A[8] - A[5] * A[7];
        double c01 = A[5] * A[6] - A[3] * A[8];
        double c02 = A[3] * A[7] - A[4] * A[6];
        double det = A[0] * c00 + A[1] * c01 + A[2] * c02;
        double scale = fmax(dx, fmax(dy, dz));
        double Ai[9];
        if (!(fabs(det) > 1e-12 * scale * scale * scale)) {
            // degenerate vertex frame: fall back to the axis frame
            for (int q = 0; q < 9; ++q) Ai[q] = 0.0;
            Ai[0] = dx > 0 ? 2.0 / dx : 1.0;
            Ai[4] = dy > 0 ? 2.0 / dy : 1.0;
            Ai[8] = dz > 0 ? 2.0 / dz : 1.0;
        } else {
            double id = 1.0 / det;
            Ai[0] = c00 * id;
            Ai[3] = c01 * id;
            Ai[6] = c02 * id;
            Ai[1] = (A[2] * A[7] - A[1] * A[8]) * id;
            Ai[4] = (A[0] * A[8] - A[2] * A[6]) * id;
            Ai[7] = (A[1] * A[6] - A[0] * A[7]) * id;
            Ai[2] = (A[1] * A[5] - A[2] * A[4]) * id;
            Ai[5] = (A[2] * A[3] - A[0] * A[5]) * id;
            Ai[8] = (A[0] * A[4] - A[1] * A[3]) * id;
        }
        for (int a = 0; a < 3; ++a) frame[a] = c[a];
        for (int q = 0; q < 9; ++q) frame[3 + q] = Ai[q];
    }
    __syncthreads();
    const double c[3] = {frame[0], frame[1], frame[2]};

    // Bernstein coefficients of (x - c) per coordinate: apply binv along
    // i, then j, then k (tensor-product change of basis)
    for (int a = 0; a < 3; ++a) {
        const double* X = coords + ((int64_t)a * E + e) * n3;
        double m = 0.0;
        for (int q = threadIdx.x; q < n3; q += blockDim.x) {
            double v = X[q] - c[a];
            tmp[q] = v;
            m = fmax(m, fabs(v));
        }
        cmax = fmax(cmax, m);
        __syncthreads();
        for (int q = threadIdx.x; q < n3; q += blockDim.x) {        // along i
            int i = q % n, rest = q / n;
            double s = 0.0;
            for (int t = 0; t < n; ++t) s += binv[i * n + t] * tmp[t + n * rest];
            B[a][q] = s;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < n3; q += blockDim.x) {        // along j
            int i = q % n, j = (q / n) % n, k = q / (n * n);
            double s = 0.0;
            for (int t = 0; t < n; ++t) s += binv[j * n + t] * B[a][i + n * (t + n * k)];
            tmp[q] = s;
        }
        __syncthreads();
        for (int q = threadIdx.x; q < n3; q += blockDim.x) {        // along k
            int ij = q % (n * n), k = q / (n * n);
            double s = 0.0;
            for (int t = 0; t < n; ++t) s += binv[k * n + t] * tmp[ij + n * n * t];
            B[a][q] = s;
        }
        __syncthreads();
    }
    cmax = block_reduce_max(cmax, red);

    // boxes of the control points: axis box of c + B, frame box of Ai B
    double Ai[9];
    for (int q = 0; q < 9; ++q) Ai[q] = frame[3 + q];
    double amin[3] = {INFINITY, INFINITY, INFINITY}, amax[3] = {-INFINITY, -INFINITY, -INFINITY};
    double omin[3] = {INFINITY, INFINITY, INFINITY}, omax[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int q = threadIdx.x; q < n3; q += blockDim.x) {
        double b0 = B[0][q], b1 = B[1][q], b2 = B[2][q];
        double bb[3] = {b0, b1, b2};
        for (int a = 0; a < 3; ++a) {
            amin[a] = fmin(amin[a], bb[a]);
            amax[a] = fmax(amax[a], bb[a]);
            double y = Ai[3 * a] * b0 + Ai[3 * a + 1] * b1 + Ai[3 * a + 2] * b2;
            omin[a] = fmin(omin[a], y);
            omax[a] = fmax(omax[a], y);
        }
    }
    for (int a = 0; a < 3; ++a) {
        amin[a] = block_reduce_min(amin[a], red);
        amax[a] = block_reduce_max(amax[a], red);
        omin[a] = block_reduce_min(omin[a], red);
        omax[a] = block_reduce_max(omax[a], red);
    }
    if (threadIdx.x == 0) {
        ElemBox bx;
        // physical pad: border tolerance, conversion round-off, and a floor
        const double pphys = pad_border * he + pad_conv * cmax + 1e-9 * he;
        // frame pad: the physical pad mapped through Ai (infinity norm)
        double ainf = 0.0;
        for (int a = 0; a < 3; ++a)
            ainf = fmax(ainf, fabs(Ai[3 * a]) + fabs(Ai[3 * a + 1]) + fabs(Ai[3 * a + 2]));
        const double pfr = ainf * pphys + 1e-12;
        for (int a = 0; a < 3; ++a) {
            bx.c[a] = c[a];
            bx.blo[a] = c[a] + amin[a] - pphys;
            bx.bhi[a] = c[a] + amax[a] + pphys;
            bx.olo[a] = omin[a] - pfr;
            bx.ohi[a] = omax[a] + pfr;
        }
        for (int q = 0; q < 9; ++q) bx.Ai[q] = Ai[q];
        bx.he = he;
        bx.spare = 0.0;
        boxes[e] = bx;
        for (int a = 0; a < 3; ++a) {
            nodebox[6 * e + a] = lo[a];
            nodebox[6 * e + 3 + a] = hi[a];
        }
    }
}

// per-block min/max of the padded axis boxes and of the node boxes
__global__ void k_reduce_boxes(int64_t E, const ElemBox* __restrict__ boxes,
                               const double* __restrict__ nodebox, double* __restrict__ out)
{
    __shared__ double red[32];
    double v[12];
    for (int a = 0; a < 3; ++a) {
        v[a] = INFINITY; v[3 + a] = -INFINITY; v[6 + a] = INFINITY; v[9 + a] = -INFINITY;
    }
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < E; e += (int64_t)gridDim.x * blockDim.x) {
        for (int a = 0; a < 3; ++a) {
            v[a] = fmin(v[a], boxes[e].blo[a]);
            v[3 + a] = fmax(v[3 + a], boxes[e].bhi[a]);
            v[6 + a] = fmin(v[6 + a], nodebox[6 * e + a]);
            v[9 + a] = fmax(v[9 + a], nodebox[6 * e + 3 + a]);
        }
    }
    for (int q = 0; q < 12; ++q) {
        bool ismin = (q % 6) < 3;
        double r = ismin ? block_reduce_min(v[q], red) : block_reduce_max(v[q], red);
        if (threadIdx.x == 0) out[12 * blockIdx.x + q] = r;
    }
}

// ---------------------------------------------------------------------------
// hash grid
// ---------------------------------------------------------------------------
__device__ __forceinline__ int cell_coord(double x, double org, double inv, int dim)
{
    double u = (x - org) * inv;
    int i = (int)floor(u);
    return min(max(i, 0), dim - 1);
}

// Elements are listed in every cell their padded axis box overlaps, widened
// by `hpad` so that a query whose cell is computed in FP32 (off by at most a
// few ulps of the coordinates) still lands in a cell that lists it.
template <bool FILL>
__global__ void k_hash(int64_t E, const ElemBox* __restrict__ boxes, HashGrid g, double hpad,
                       int32_t* __restrict__ cnt, int32_t* __restrict__ cur,
                       int32_t* __restrict__ elems)
{
    int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= E) return;
    const ElemBox& b = boxes[e];
    int i0[3], i1[3];
    for (int a = 0; a < 3; ++a) {
        i0[a] = cell_coord(b.blo[a] - hpad, g.org[a], g.inv[a], g.dim[a]);
        i1[a] = cell_coord(b.bhi[a] + hpad, g.org[a], g.inv[a], g.dim[a]);
    }
    for (int k = i0[2]; k <= i1[2]; ++k)
        for (int j = i0[1]; j <= i1[1]; ++j)
            for (int i = i0[0]; i <= i1[0]; ++i) {
                int64_t cidx = i + (int64_t)g.dim[0] * (j + (int64_t)g.dim[1] * k);
                if (!FILL) {
                    atomicAdd(cnt + cidx, 1);
                } else {
                    int pos = atomicAdd(cur + cidx, 1);
                    elems[pos] = (int32_t)e;
                }
            }
}

// sort each cell's list by element id (lists are short): deterministic order
__global__ void k_hash_sort(int64_t ncell, const int32_t* __restrict__ start, int32_t* __restrict__ elems)
{
    int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (c >= ncell) return;
    int b = start[c], en = start[c + 1];
    for (int i = b + 1; i < en; ++i) {
        int v = elems[i], j = i - 1;
        while (j >= b && elems[j] > v) {
            elems[j + 1] = elems[j];
            --j;
        }
        elems[j + 1] = v;
    }
}

// ---------------------------------------------------------------------------
// default nodal distance field D^k
// ---------------------------------------------------------------------------
__device__ __forceinline__ int face_node(int n, int f, int a, int b)
{
    int end = (f & 1) ? n - 1 : 0;
    switch (f >> 1) {
        case 0: return end + n * (a + n * b);
        case 1: return a + n * (end + n * b);
        default: return a + n * (b + n * end);
    }
}

__device__ __forceinline__ bool lex_less(const double* p, const double* q)
{
    for (int a = 0; a < 3; ++a) {
        if (p[a] < q[a]) return true;
        if (p[a] > q[a]) return false;
    }
    return false;
}

// the four corner points of each face, sorted lexicographically: [6E][12]
__global__ void k_face_corners(int n, int64_t E, const double* __restrict__ coords, double* __restrict__ fc)
{
    int64_t fidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (fidx >= 6 * E) return;
    const int64_t e = fidx / 6;
    const int f = (int)(fidx % 6), N = n - 1, n3 = n * n * n;
    double c[4][3];
    const int ab[4][2] = {{0, 0}, {N, 0}, {0, N}, {N, N}};
    for (int q = 0; q < 4; ++q) {
        int idx = face_node(n, f, ab[q][0], ab[q][1]);
        for (int a = 0; a < 3; ++a) c[q][a] = coords[((int64_t)a * E + e) * n3 + idx];
    }
    for (int i = 1; i < 4; ++i)
        for (int j = i; j > 0 && lex_less(c[j], c[j - 1]); --j)
            for (int a = 0; a < 3; ++a) {
                double t = c[j][a];
                c[j][a] = c[j - 1][a];
                c[j - 1][a] = t;
            }
    for (int q = 0; q < 4; ++q)
        for (int a = 0; a < 3; ++a) fc[12 * fidx + 3 * q + a] = c[q][a];
}

// a face is a boundary face of its subdomain unless another element of the
// same subdomain has a face with the same four corners; candidates come from
// the hash cell of the face centroid (the neighbour's box contains it)
__global__ void k_face_boundary(int64_t E, const double* __restrict__ fc, const int32_t* __restrict__ sub,
                                HashGrid g, const int32_t* __restrict__ cstart,
                                const int32_t* __restrict__ celems, int32_t* __restrict__ nbnd)
{
    int64_t fidx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (fidx >= 6 * E) return;
    const int64_t e = fidx / 6;
    const double* me = fc + 12 * fidx;
    double cen[3];
    for (int a = 0; a < 3; ++a) cen[a] = 0.25 * (me[a] + me[3 + a] + me[6 + a] + me[9 + a]);
    int64_t cidx = cell_coord(cen[0], g.org[0], g.inv[0], g.dim[0]) +
                   (int64_t)g.dim[0] * (cell_coord(cen[1], g.org[1], g.inv[1], g.dim[1]) +
                                        (int64_t)g.dim[1] * cell_coord(cen[2], g.org[2], g.inv[2], g.dim[2]));
    int shared = 0;
    for (int q = cstart[cidx]; q < cstart[cidx + 1] && !shared; ++q) {
        int e2 = celems[q];
        if (e2 == e || sub[e2] != sub[e]) continue;
        for (int f2 = 0; f2 < 6 && !shared; ++f2) {
            const double* ot = fc + 12 * ((int64_t)e2 * 6 + f2);
            bool eq = true;
            for (int t = 0; t < 12; ++t) eq = eq && (ot[t] == me[t]);
            shared = eq;
        }
    }
    nbnd[fidx] = shared ? 0 : 1;
}

// gather the n^2 GLL nodes of every boundary face: positions [3][nb], subdomain [nb]
__global__ void k_face_gather(int n, int64_t E, const double* __restrict__ coords, const int32_t* __restrict__ sub,
                              const int32_t* __restrict__ bnd_off, double* __restrict__ bx,
                              int32_t* __restrict__ bs, int64_t nb)
{
    int64_t fidx = blockIdx.x;
    if (fidx >= 6 * E) return;
    int o = bnd_off[fidx];
    if (bnd_off[fidx + 1] == o) return;
    const int64_t e = fidx / 6;
    const int f = (int)(fidx % 6), n2 = n * n, n3 = n2 * n;
    for (int t = threadIdx.x; t < n2; t += blockDim.x) {
        int a = t % n, b = t / n;
        int idx = face_node(n, f, a, b);
        int64_t m = (int64_t)o * n2 + t;
        for (int c = 0; c < 3; ++c) bx[c * nb + m] = coords[((int64_t)c * E + e) * n3 + idx];
        bs[m] = sub[e];
    }
}

// D(node) = min distance to the boundary-face nodes of the node's own subdomain
__global__ void k_dist_default(int n3, int64_t E, const double* __restrict__ coords, const int32_t* __restrict__ sub,
                               const double* __restrict__ bx, const int32_t* __restrict__ bs, int64_t nb,
                               double* __restrict__ D)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= E * n3) return;
    int64_t e = q / n3;
    double x = coords[q], y = coords[E * n3 + q], z = coords[2 * E * n3 + q];
    int s = sub[e];
    double best = INFINITY;
    for (int64_t b = 0; b < nb; ++b) {
        if (bs[b] != s) continue;
        double dx = x - bx[b], dy = y - bx[nb + b], dz = z - bx[2 * nb + b];
        double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        best = fmin(best, d2);
    }
    D[q] = sqrt(best);
}

// count non-finite values (mesh validation)
__global__ void k_count_nonfinite(int64_t n, const double* __restrict__ x, int32_t* __restrict__ out)
{
    int bad = 0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        bad |= !isfinite(x[i]);
    if (__syncthreads_or(bad) && threadIdx.x == 0) atomicAdd(out, 1);
}

// FP32 boxes for the mixed form's screen.  The axis box is rounded outward
// and widened by 2^-22 max|bound| (the query coordinate is rounded to FP32
// before the comparison).  The frame box is widened by the bound on the FP32
// error of y = Ai (x - c) for x inside the axis box: rounding of x, c and
// Ai, and of the subtraction and the three-term dot product.
__global__ void k_box32(int64_t E, const ElemBox* __restrict__ boxes, ElemBox32* __restrict__ out)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= E) return;
    const ElemBox& b = boxes[e];
    ElemBox32 o;
    const double u = 5.9604644775390625e-08;           // 2^-24
    double xmax = 0.0, ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        xmax = fmax(xmax, fmax(fabs(b.blo[a]), fabs(b.bhi[a])));
        ext = fmax(ext, b.bhi[a] - b.blo[a]);
        const double m = 4.0 * u * fmax(fabs(b.blo[a]), fabs(b.bhi[a]));
        o.blo[a] = __double2float_rd(b.blo[a] - m);
        o.bhi[a] = __double2float_ru(b.bhi[a] + m);
        o.c[a] = (float)b.c[a];
    }
    for (int q = 0; q < 9; ++q) o.Ai[q] = (float)b.Ai[q];
    for (int a = 0; a < 3; ++a) {
        const double arow = fabs(b.Ai[3 * a]) + fabs(b.Ai[3 * a + 1]) + fabs(b.Ai[3 * a + 2]);
        // |dy| <= |Ai| (|dx| + |dc| + |d(x-c)|) + |dAi| |x-c| + dot-product rounding
        const double m = 16.0 * u * arow * (2.0 * xmax + 2.0 * ext) + 16.0 * u * fmax(fabs(b.olo[a]), fabs(b.ohi[a]));
        o.olo[a] = __double2float_rd(b.olo[a] - m);
        o.ohi[a] = __double2float_ru(b.ohi[a] + m);
    }
    out[e] = o;
}

cudaError_t launch_box32(int64_t E, const ElemBox* boxes, ElemBox32* out, cudaStream_t s)
{
    k_box32<<<(unsigned)((E + 255) / 256), 256, 0, s>>>(E, boxes, out);
    count_launch();
    return cudaGetLastError();
}

// element-local FP32 copy of the geometry for the mixed form: float(x - c)
__global__ void k_local32(int n3, int64_t E, const double* __restrict__ coords, const ElemBox* __restrict__ boxes,
                          float* __restrict__ c32)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= 3 * E * n3) return;
    int64_t a = q / (E * n3);
    int64_t e = (q / n3) % E;
    c32[q] = (float)(coords[q] - boxes[e].c[a]);
}

// low parts of the element-local coordinates: (x - c) - hi, rounded to FP32
__global__ void k_local32lo(int n3, int64_t E, const double* __restrict__ coords, const ElemBox* __restrict__ boxes,
                            const float* __restrict__ c32, float* __restrict__ c32lo)
{
    int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (q >= 3 * E * n3) return;
    int64_t a = q / (E * n3);
    int64_t e = (q / n3) % E;
    c32lo[q] = (float)((coords[q] - boxes[e].c[a]) - (double)c32[q]);
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
cudaError_t launch_hull(int n, int64_t E, const double* coords, const double* binv, double pad_border,
                        double pad_conv, ElemBox* boxes, double* nodebox, cudaStream_t s)
{
    size_t smem = sizeof(double) * 4 * (size_t)n * n * n;
    cudaError_t err = cudaFuncSetAttribute(k_hull, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (err != cudaSuccess) return err;
    k_hull<<<(unsigned)E, 128, smem, s>>>(n, E, coords, binv, pad_border, pad_conv, boxes, nodebox);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_reduce_boxes(int64_t E, const ElemBox* boxes, const double* nodebox, double* out,
                                int nblocks, cudaStream_t s)
{
    k_reduce_boxes<<<nblocks, 256, 0, s>>>(E, boxes, nodebox, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_hash_count(int64_t E, const ElemBox* boxes, const HashGrid& g, double hpad, int32_t* cnt,
                              cudaStream_t s)
{
    k_hash<false><<<(unsigned)((E + 255) / 256), 256, 0, s>>>(E, boxes, g, hpad, cnt, nullptr, nullptr);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_hash_fill(int64_t E, const ElemBox* boxes, const HashGrid& g, double hpad, int32_t* cur,
                             int32_t* elems, cudaStream_t s)
{
    k_hash<true><<<(unsigned)((E + 255) / 256), 256, 0, s>>>(E, boxes, g, hpad, nullptr, cur, elems);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_hash_sort(int64_t ncell, const int32_t* start, int32_t* elems, cudaStream_t s)
{
    k_hash_sort<<<(unsigned)((ncell + 255) / 256), 256, 0, s>>>(ncell, start, elems);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_face_corners(int n, int64_t E, const double* coords, double* fc, cudaStream_t s)
{
    k_face_corners<<<(unsigned)((6 * E + 127) / 128), 128, 0, s>>>(n, E, coords, fc);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_face_boundary(int64_t E, const double* fc, const int32_t* sub, const HashGrid& g,
                                 const int32_t* cstart, const int32_t* celems, int32_t* nbnd, cudaStream_t s)
{
    k_face_boundary<<<(unsigned)((6 * E + 127) / 128), 128, 0, s>>>(E, fc, sub, g, cstart, celems, nbnd);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_face_gather(int n, int64_t E, const double* coords, const int32_t* sub, const int32_t* bnd_off,
                               double* bx, int32_t* bs, int64_t nb, cudaStream_t s)
{
    k_face_gather<<<(unsigned)(6 * E), 64, 0, s>>>(n, E, coords, sub, bnd_off, bx, bs, nb);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_dist_default(int n, int64_t E, const double* coords, const int32_t* sub, const double* bx,
                                const int32_t* bs, int64_t nb, double* D, cudaStream_t s)
{
    int n3 = n * n * n;
    k_dist_default<<<(unsigned)((E * n3 + 255) / 256), 256, 0, s>>>(n3, E, coords, sub, bx, bs, nb, D);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_count_nonfinite(int64_t n, const double* x, int32_t* out, cudaStream_t s)
{
    int64_t blocks = std::min<int64_t>((n + 255) / 256, 4096);
    if (blocks < 1) blocks = 1;
    k_count_nonfinite<<<(unsigned)blocks, 256, 0, s>>>(n, x, out);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_local32lo(int n, int64_t E, const double* coords, const ElemBox* boxes, const float* c32,
                             float* c32lo, cudaStream_t s)
{
    int n3 = n * n * n;
    k_local32lo<<<(unsigned)((3 * E * n3 + 255) / 256), 256, 0, s>>>(n3, E, coords, boxes, c32, c32lo);
    count_launch();
    return cudaGetLastError();
}

cudaError_t launch_local32(int n, int64_t E, const double* coords, const ElemBox* boxes, float* c32,
                           cudaStream_t s)
{
    int n3 = n * n * n;
    k_local32<<<(unsigned)((3 * E * n3 + 255) / 256), 256, 0, s>>>(n3, E, coords, boxes, c32);
    count_launch();
    return cudaGetLastError();
}

}  // namespace fpg
