// fp_flux.cu -- mass-flux correction of interpolated interface velocity
// (Sec. 2.2, Eqs. consv1, corr, consv2).
//
// fp_bfaces_create lists the faces a caller marks on the handle's mesh
// (1 = boundary with prescribed data, 2 = interface with interpolated data),
// in (element, face) order, and computes for every face node its position,
// outward unit normal and GLL area weight dA = w_a w_b |t_1 x t_2| (tangents
// from the derivative matrix of the Lagrange basis applied along the face).
// fp_flux_correct then computes
//     flux  = sum over all listed nodes of u.n dA        (int u.n over dOmega^j)
//     area  = sum over interface nodes of n.n dA          (int n.n over dOmega_i)
//     gamma = -flux / area                                (Eq. consv2)
// and u_out = u + gamma n on interface nodes, u elsewhere (Eq. corr), with a
// fixed-order two-level reduction (the same bits on every run).
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fp_common.cuh"
#include "fp_handle.h"
#include "fp_internal.h"

using namespace fpg;

struct DerivTab {
    double D[NMAX * NMAX];   // D[a*n + i] = h_i'(xi_a)
    double w[NMAX];          // GLL quadrature weights
};

struct fp_bfaces {
    const fp_handle* owner = nullptr;
    int n = 0;
    int64_t nf = 0, M = 0;
    int32_t* face = nullptr;      // [nf] e*6 + f
    double* x = nullptr;          // [3][M]
    double* nrm = nullptr;        // [3][M]
    double* dA = nullptr;         // [M]
    int8_t* kind = nullptr;       // [M]
    int32_t* ipos = nullptr;      // [M] index of the node among the interface nodes, -1 otherwise
    int64_t Mi = 0;               // interface nodes
    double* partial = nullptr;    // [2 * nblk]
    double* result = nullptr;     // [3]: flux, area, gamma
    int nblk = 0;
    int8_t* fkind = nullptr;      // [6E] copy of the caller's face marks (for fp_bfaces_refresh)
    DerivTab tab{};
};

namespace fpg {

__global__ void k_face_flags(int64_t F, const int8_t* __restrict__ kind, int32_t* __restrict__ flag)
{
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f < F) flag[f] = kind[f] != 0;
}

__global__ void k_face_list(int64_t F, const int8_t* __restrict__ kind, const int32_t* __restrict__ off,
                            int32_t* __restrict__ face)
{
    const int64_t f = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (f < F && kind[f] != 0) face[off[f]] = (int32_t)f;
}

__device__ __forceinline__ int fnode(int n, int f, int a, int b)
{
    const int end = (f & 1) ? n - 1 : 0;
    switch (f >> 1) {
        case 0: return end + n * (a + n * b);
        case 1: return a + n * (end + n * b);
        default: return a + n * (b + n * end);
    }
}

template <int n>
__global__ void k_bface_geom(int64_t E, int64_t M, const double* __restrict__ coords, const ElemBox* __restrict__ boxes,
                             const int8_t* __restrict__ kind, const int32_t* __restrict__ face, DerivTab tab,
                             double* __restrict__ x, double* __restrict__ nrm, double* __restrict__ dA,
                             int8_t* __restrict__ nkind)
{
    constexpr int n2 = n * n, n3 = n2 * n;
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int fid = face[m / n2];
    const int64_t e = fid / 6;
    const int f = fid % 6;
    const int a = (int)(m % n2) % n, b = (int)(m % n2) / n;
    // handedness of the element: sign of det of its affine frame (det Ai has the sign of det A)
    const double* Ai = boxes[e].Ai;
    const double detAi = Ai[0] * (Ai[4] * Ai[8] - Ai[5] * Ai[7]) - Ai[1] * (Ai[3] * Ai[8] - Ai[5] * Ai[6]) +
                         Ai[2] * (Ai[3] * Ai[7] - Ai[4] * Ai[6]);
    const double hand = detAi < 0.0 ? -1.0 : 1.0;
    double t1[3], t2[3], xn[3];
    for (int c = 0; c < 3; ++c) {
        const double* X = coords + ((int64_t)c * E + e) * n3;
        double s1 = 0.0, s2 = 0.0;
#pragma unroll
        for (int q = 0; q < n; ++q) {
            s1 = fma(tab.D[a * n + q], X[fnode(n, f, q, b)], s1);
            s2 = fma(tab.D[b * n + q], X[fnode(n, f, a, q)], s2);
        }
        t1[c] = s1;
        t2[c] = s2;
        xn[c] = X[fnode(n, f, a, b)];
    }
    // cyclic orientation of the face variables: r-faces (s,t), s-faces (t,r), t-faces (r,s)
    double nv[3] = {t1[1] * t2[2] - t1[2] * t2[1], t1[2] * t2[0] - t1[0] * t2[2], t1[0] * t2[1] - t1[1] * t2[0]};
    const double o = ((f >> 1) == 1 ? -1.0 : 1.0) * ((f & 1) ? 1.0 : -1.0) * hand;
    const double len = sqrt(nv[0] * nv[0] + nv[1] * nv[1] + nv[2] * nv[2]);
    for (int c = 0; c < 3; ++c) {
        x[c * M + m] = xn[c];
        nrm[c * M + m] = o * nv[c] / len;
    }
    dA[m] = tab.w[a] * tab.w[b] * len;
    nkind[m] = kind[fid];
}

constexpr int FLUX_THREADS = 256;

// velocity component c at face node m: from u [3][M], or -- split form --
// from the interpolated interface values ui [3][Mi] on interface nodes and
// the prescribed values up [3][M] elsewhere
struct UView {
    const double* u;
    const double* ui;
    const int32_t* ipos;
    int64_t M, Mi;
    __device__ __forceinline__ double at(int c, int64_t m) const
    {
        if (ui) {
            const int32_t k = ipos[m];
            if (k >= 0) return ui[c * Mi + k];
        }
        return u[c * M + m];
    }
};

// per block: sum of u.n dA and of interface n.n dA over a contiguous chunk
__global__ void __launch_bounds__(FLUX_THREADS) k_flux_partial(int64_t M, int64_t chunk, UView u,
                                                               const double* __restrict__ nrm,
                                                               const double* __restrict__ dA,
                                                               const int8_t* __restrict__ kind,
                                                               double* __restrict__ partial)
{
    __shared__ double s0[FLUX_THREADS], s1[FLUX_THREADS];
    const int64_t lo = blockIdx.x * chunk, hi = min(M, lo + chunk);
    double a0 = 0.0, a1 = 0.0;
    for (int64_t m = lo + threadIdx.x; m < hi; m += blockDim.x) {
        const double nx = nrm[m], ny = nrm[M + m], nz = nrm[2 * M + m];
        const double un = u.at(0, m) * nx + u.at(1, m) * ny + u.at(2, m) * nz;
        a0 += un * dA[m];
        if (kind[m] == 2) a1 += (nx * nx + ny * ny + nz * nz) * dA[m];
    }
    s0[threadIdx.x] = a0;
    s1[threadIdx.x] = a1;
    __syncthreads();
    for (int w = FLUX_THREADS / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            s0[threadIdx.x] += s0[threadIdx.x + w];
            s1[threadIdx.x] += s1[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        partial[2 * blockIdx.x] = s0[0];
        partial[2 * blockIdx.x + 1] = s1[0];
    }
}

__global__ void k_flux_final(int nblk, const double* __restrict__ partial, double* __restrict__ result)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double fl = 0.0, area = 0.0;
    for (int b = 0; b < nblk; ++b) {
        fl += partial[2 * b];
        area += partial[2 * b + 1];
    }
    result[0] = fl;
    result[1] = area;
    result[2] = area > 0.0 ? -fl / area : 0.0;
}

__global__ void k_flux_apply(int64_t M, UView u, const double* __restrict__ nrm, const int8_t* __restrict__ kind,
                             const double* __restrict__ result, double* __restrict__ u_out)
{
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= M) return;
    const double g = kind[m] == 2 ? result[2] : 0.0;
    for (int c = 0; c < 3; ++c) u_out[c * M + m] = u.at(c, m) + g * nrm[c * M + m];
}

__global__ void k_iface_pos(int64_t M, const int8_t* __restrict__ kind, const int32_t* __restrict__ off,
                            int32_t* __restrict__ ipos)
{
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m < M) ipos[m] = kind[m] == 2 ? off[m] : -1;
}

// interface numbering sorted by donor element (counting sort; points of one
// element keep an arbitrary order among themselves)
__global__ void k_key_hist(int64_t Mi, int64_t E, const int32_t* __restrict__ elem, int32_t* __restrict__ cnt)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= Mi) return;
    const int32_t e = elem[k];
    atomicAdd(cnt + ((e >= 0 && e < E) ? e : E), 1);
}

__global__ void k_key_scatter(int64_t Mi, int64_t E, const int32_t* __restrict__ elem,
                              const int32_t* __restrict__ start, int32_t* __restrict__ cursor,
                              int32_t* __restrict__ newpos)
{
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= Mi) return;
    const int32_t e = elem[k];
    const int64_t key = (e >= 0 && e < E) ? e : E;
    newpos[k] = start[key] + atomicAdd(cursor + key, 1);
}

__global__ void k_ipos_remap(int64_t M, const int32_t* __restrict__ newpos, int32_t* __restrict__ ipos)
{
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m < M && ipos[m] >= 0) ipos[m] = newpos[ipos[m]];
}

__global__ void k_iface_flags(int64_t M, const int8_t* __restrict__ kind, int32_t* __restrict__ flag)
{
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m < M) flag[m] = kind[m] == 2;
}

__global__ void k_iface_points(int64_t M, int64_t Mi, const int32_t* __restrict__ ipos, const double* __restrict__ x,
                               double* __restrict__ pts)
{
    const int64_t m = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (m >= M) return;
    const int32_t k = ipos[m];
    if (k >= 0)
        for (int c = 0; c < 3; ++c) pts[c * Mi + k] = x[c * M + m];
}

// out = sum_j c_j hist_j (temporal extrapolation of interface data)
struct ExtArgs {
    const double* h[3];
    double c[3];
    int m;
};

__global__ void k_extrapolate(int64_t len, ExtArgs A, double* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        double v = A.c[0] * A.h[0][i];
        if (A.m > 1) v = fma(A.c[1], A.h[1][i], v);
        if (A.m > 2) v = fma(A.c[2], A.h[2][i], v);
        out[i] = v;
    }
}

__global__ void k_flux_out(const double* __restrict__ result, double* gamma, double* flux)
{
    if (gamma) *gamma = result[2];
    if (flux) *flux = result[0];
}

}  // namespace fpg

static void bf_release(fp_bfaces* b)
{
    cudaFree(b->ipos);
    cudaFree(b->fkind);
    cudaFree(b->face); cudaFree(b->x); cudaFree(b->nrm); cudaFree(b->dA); cudaFree(b->kind);
    cudaFree(b->partial); cudaFree(b->result);
}

// node positions, normals and weights of the listed faces from the owner's
// current coordinates
static cudaError_t bf_geom(fp_bfaces* b, const fp_handle* h, const int8_t* kind, cudaStream_t s)
{
    if (b->M == 0) return cudaSuccess;
    const unsigned grid = (unsigned)((b->M + 127) / 128);
    switch (b->n) {
#define FP_CASE(NN) \
    case NN: k_bface_geom<NN><<<grid, 128, 0, s>>>(h->E, b->M, h->coords, h->boxes, kind, b->face, b->tab, b->x, b->nrm, b->dA, b->kind); break;
        FP_CASE(2) FP_CASE(3) FP_CASE(4) FP_CASE(5) FP_CASE(6) FP_CASE(7) FP_CASE(8) FP_CASE(9)
        FP_CASE(10) FP_CASE(11) FP_CASE(12) FP_CASE(13) FP_CASE(14) FP_CASE(15) FP_CASE(16)
#undef FP_CASE
        default: return cudaErrorInvalidValue;
    }
    count_launch();
    return cudaGetLastError();
}

extern "C" fp_status fp_bfaces_create(const fp_handle* h, const int8_t* kind, fp_bfaces** out, void* stream)
{
    if (!out) return FP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    if (!kind || h->dim != 3) return FP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const int n = h->n;
    const int64_t F = 6 * h->E;
    fp_bfaces* b = new fp_bfaces();
    b->owner = h;
    b->n = n;
    int32_t *flag = nullptr, *off = nullptr, *tmp = nullptr;
    int32_t total = 0;
    cudaError_t e = cudaMalloc(&flag, sizeof(int32_t) * F);
    if (e == cudaSuccess) e = cudaMalloc(&off, sizeof(int32_t) * (F + 1));
    if (e == cudaSuccess) e = cudaMalloc(&tmp, sizeof(int32_t) * scan_tmp_elems(F));
    if (e == cudaSuccess) e = cudaMalloc(&b->fkind, F);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->fkind, kind, F, cudaMemcpyDeviceToDevice, s);
    if (e == cudaSuccess) {
        k_face_flags<<<(unsigned)((F + 255) / 256), 256, 0, s>>>(F, kind, flag);
        count_launch();
        e = scan_exclusive(flag, off, F, tmp, s);
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&total, off + F, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    b->nf = total;
    b->M = (int64_t)total * n * n;
    if (e == cudaSuccess) e = cudaMalloc(&b->face, sizeof(int32_t) * std::max<int64_t>(b->nf, 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->x, sizeof(double) * 3 * std::max<int64_t>(b->M, 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->nrm, sizeof(double) * 3 * std::max<int64_t>(b->M, 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->dA, sizeof(double) * std::max<int64_t>(b->M, 1));
    if (e == cudaSuccess) e = cudaMalloc(&b->kind, std::max<int64_t>(b->M, 1));
    b->nblk = (int)std::max<int64_t>(1, std::min<int64_t>(1024, (b->M + 511) / 512));   // ~2 nodes per thread
    if (e == cudaSuccess) e = cudaMalloc(&b->partial, sizeof(double) * 2 * b->nblk);
    if (e == cudaSuccess) e = cudaMalloc(&b->result, sizeof(double) * 3);
    if (e == cudaSuccess && b->nf > 0) {
        k_face_list<<<(unsigned)((F + 255) / 256), 256, 0, s>>>(F, kind, off, b->face);
        count_launch();
        DerivTab t;
        memset(&t, 0, sizeof(t));
        const double* xi = h->tab.xi;
        const int N = n - 1;
        for (int a = 0; a < n; ++a) {
            double dsum = 0.0;
            for (int i = 0; i < n; ++i) {
                if (i == a) continue;
                // h_i'(xi_a) for i != a: the factor (r - xi_a) is the only one that vanishes
                double p = h->tab.ci[i];
                for (int m = 0; m < n; ++m)
                    if (m != i && m != a) p *= (xi[a] - xi[m]);
                t.D[a * n + i] = p;
                dsum += 1.0 / (xi[a] - xi[i]);
            }
            t.D[a * n + a] = dsum;
            // GLL weight 2 / (N (N+1) P_N(xi_a)^2), P_N by the three-term recurrence
            double p0 = 1.0, p1 = xi[a];
            for (int k = 1; k < N; ++k) {
                double p2 = ((2 * k + 1) * xi[a] * p1 - k * p0) / (k + 1);
                p0 = p1;
                p1 = p2;
            }
            const double PN = N == 0 ? 1.0 : p1;
            t.w[a] = 2.0 / (N * (N + 1.0) * PN * PN);
        }
        b->tab = t;
        e = bf_geom(b, h, b->fkind, s);
    }
    // positions of the interface nodes among themselves (listing order)
    if (e == cudaSuccess) e = cudaMalloc(&b->ipos, sizeof(int32_t) * std::max<int64_t>(b->M, 1));
    if (e == cudaSuccess && b->M > 0) {
        int32_t *nf = nullptr, *noff = nullptr, *ntmp = nullptr;
        e = cudaMalloc(&nf, sizeof(int32_t) * b->M);
        if (e == cudaSuccess) e = cudaMalloc(&noff, sizeof(int32_t) * (b->M + 1));
        if (e == cudaSuccess) e = cudaMalloc(&ntmp, sizeof(int32_t) * scan_tmp_elems(b->M));
        if (e == cudaSuccess) {
            k_iface_flags<<<(unsigned)((b->M + 255) / 256), 256, 0, s>>>(b->M, b->kind, nf);
            count_launch();
            e = scan_exclusive(nf, noff, b->M, ntmp, s);
        }
        if (e == cudaSuccess) {
            k_iface_pos<<<(unsigned)((b->M + 255) / 256), 256, 0, s>>>(b->M, b->kind, noff, b->ipos);
            count_launch();
            int32_t mi = 0;
            e = cudaMemcpyAsync(&mi, noff + b->M, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            b->Mi = mi;
        }
        cudaFree(nf);
        cudaFree(noff);
        cudaFree(ntmp);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(flag);
    cudaFree(off);
    cudaFree(tmp);
    if (e != cudaSuccess) {
        bf_release(b);
        delete b;
        return e == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA;
    }
    *out = b;
    return FP_OK;
}

extern "C" void fp_bfaces_free(fp_bfaces* b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    bf_release(b);
    delete b;
}

extern "C" fp_status fp_bfaces_sort_iface(fp_bfaces* b, const int32_t* elem, void* stream)
{
    if (!b || !elem) return FP_ERR_INVALID_ARG;
    if (!fp_live(b->owner)) return FP_ERR_NOT_SETUP;
    const int64_t Mi = b->Mi, E = b->owner->E;
    if (Mi == 0) return FP_OK;
    cudaStream_t s = (cudaStream_t)stream;
    int32_t *cnt = nullptr, *start = nullptr, *tmp = nullptr, *newpos = nullptr;
    cudaError_t e = cudaMalloc(&cnt, sizeof(int32_t) * (E + 1));
    if (e == cudaSuccess) e = cudaMalloc(&start, sizeof(int32_t) * (E + 2));
    if (e == cudaSuccess) e = cudaMalloc(&tmp, sizeof(int32_t) * scan_tmp_elems(E + 1));
    if (e == cudaSuccess) e = cudaMalloc(&newpos, sizeof(int32_t) * Mi);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (E + 1), s);
    if (e == cudaSuccess) {
        k_key_hist<<<(unsigned)((Mi + 255) / 256), 256, 0, s>>>(Mi, E, elem, cnt);
        count_launch();
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = scan_exclusive(cnt, start, E + 1, tmp, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(int32_t) * (E + 1), s);
    if (e == cudaSuccess) {
        k_key_scatter<<<(unsigned)((Mi + 255) / 256), 256, 0, s>>>(Mi, E, elem, start, cnt, newpos);
        k_ipos_remap<<<(unsigned)((b->M + 255) / 256), 256, 0, s>>>(b->M, newpos, b->ipos);
        count_launch(2);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(cnt); cudaFree(start); cudaFree(tmp); cudaFree(newpos);
    return e == cudaSuccess ? FP_OK : (e == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA);
}

extern "C" fp_status fp_bfaces_refresh(fp_bfaces* b, void* stream)
{
    if (!b) return FP_ERR_INVALID_ARG;
    if (!fp_live(b->owner)) return FP_ERR_NOT_SETUP;
    return bf_geom(b, b->owner, b->fkind, (cudaStream_t)stream) == cudaSuccess ? FP_OK : FP_ERR_CUDA;
}

extern "C" fp_status fp_bfaces_info(const fp_bfaces* b, int64_t* nfaces, int64_t* nnodes)
{
    if (!b) return FP_ERR_INVALID_ARG;
    if (nfaces) *nfaces = b->nf;
    if (nnodes) *nnodes = b->M;
    return FP_OK;
}

extern "C" fp_status fp_bfaces_iface(const fp_bfaces* b, int64_t* n_iface, double* pts, void* stream)
{
    if (!b) return FP_ERR_INVALID_ARG;
    if (n_iface) *n_iface = b->Mi;
    if (pts && b->M > 0) {
        k_iface_points<<<(unsigned)((b->M + 255) / 256), 256, 0, (cudaStream_t)stream>>>(b->M, b->Mi, b->ipos, b->x,
                                                                                          pts);
        count_launch();
        if (cudaGetLastError() != cudaSuccess) return FP_ERR_CUDA;
    }
    return FP_OK;
}

extern "C" fp_status fp_extrapolate(int m, int64_t len, const double* const* hist, double* out, void* stream)
{
    if (m < 1 || m > 3 || len < 0 || !hist || !out) return FP_ERR_INVALID_ARG;
    ExtArgs a;
    memset(&a, 0, sizeof(a));
    a.m = m;
    static const double coef[3][3] = {{1.0, 0.0, 0.0}, {2.0, -1.0, 0.0}, {3.0, -3.0, 1.0}};
    for (int j = 0; j < m; ++j) {
        if (!hist[j]) return FP_ERR_INVALID_ARG;
        a.h[j] = hist[j];
        a.c[j] = coef[m - 1][j];
    }
    if (len == 0) return FP_OK;
    const int64_t blocks = std::min<int64_t>((len + 255) / 256, 4096);
    k_extrapolate<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(len, a, out);
    count_launch();
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ERR_CUDA;
}

extern "C" fp_status fp_bfaces_nodes(const fp_bfaces* b, double* x, double* normal, double* dA, int8_t* kind,
                                     void* stream)
{
    if (!b) return FP_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    if (x && b->M) e = cudaMemcpyAsync(x, b->x, sizeof(double) * 3 * b->M, cudaMemcpyDeviceToDevice, s);
    if (normal && b->M && e == cudaSuccess)
        e = cudaMemcpyAsync(normal, b->nrm, sizeof(double) * 3 * b->M, cudaMemcpyDeviceToDevice, s);
    if (dA && b->M && e == cudaSuccess) e = cudaMemcpyAsync(dA, b->dA, sizeof(double) * b->M, cudaMemcpyDeviceToDevice, s);
    if (kind && b->M && e == cudaSuccess) e = cudaMemcpyAsync(kind, b->kind, b->M, cudaMemcpyDeviceToDevice, s);
    return e == cudaSuccess ? FP_OK : FP_ERR_CUDA;
}

static fp_status flux_impl(const fp_bfaces* b, UView u, double* u_out, double* gamma, double* flux, cudaStream_t s)
{
    if (b->M == 0) {
        k_flux_final<<<1, 1, 0, s>>>(0, b->partial, b->result);
        k_flux_out<<<1, 1, 0, s>>>(b->result, gamma, flux);
        count_launch(2);
        return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ERR_CUDA;
    }
    const int64_t chunk = (b->M + b->nblk - 1) / b->nblk;
    k_flux_partial<<<b->nblk, FLUX_THREADS, 0, s>>>(b->M, chunk, u, b->nrm, b->dA, b->kind, b->partial);
    k_flux_final<<<1, 1, 0, s>>>(b->nblk, b->partial, b->result);
    k_flux_apply<<<(unsigned)((b->M + 255) / 256), 256, 0, s>>>(b->M, u, b->nrm, b->kind, b->result, u_out);
    k_flux_out<<<1, 1, 0, s>>>(b->result, gamma, flux);
    count_launch(4);
    return cudaGetLastError() == cudaSuccess ? FP_OK : FP_ERR_CUDA;
}

extern "C" fp_status fp_flux_correct(const fp_bfaces* b, const double* u, double* u_out, double* gamma, double* flux,
                                     void* stream)
{
    if (!b || !u || !u_out) return FP_ERR_INVALID_ARG;
    UView v{u, nullptr, nullptr, b->M, b->Mi};
    return flux_impl(b, v, u_out, gamma, flux, (cudaStream_t)stream);
}

extern "C" fp_status fp_flux_correct_iface(const fp_bfaces* b, const double* u_iface, const double* u_pres,
                                           double* u_out, double* gamma, double* flux, void* stream)
{
    if (!b || !u_iface || !u_pres || !u_out) return FP_ERR_INVALID_ARG;
    UView v{u_pres, u_iface, b->ipos, b->M, b->Mi};
    return flux_impl(b, v, u_out, gamma, flux, (cudaStream_t)stream);
}
