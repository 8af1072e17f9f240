// fp_host.cu -- the C ABI (include/findpts_gb.h): handle, validation,
// resident mesh state, workspace, and the orchestration of the setup, find
// and eval kernels.
#include <math.h>

#include <cmath>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <string>
#include <utility>
#include <vector>

#include "fp_common.cuh"
#include "fp_internal.h"
#include "fp_handle.h"

using namespace fpg;

namespace fpg {
static std::atomic<int64_t> g_launches{0};
void count_launch(int k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
}  // namespace fpg


static thread_local std::string g_setup_err;

namespace {

fp_status fail(fp_handle* h, fp_status s, const std::string& msg)
{
    if (h) h->err = msg;
    else g_setup_err = msg;
    return s;
}

fp_status cuda_fail(fp_handle* h, cudaError_t e, const char* where)
{
    std::string m = std::string(where) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA, m);
}

template <typename T>
cudaError_t dalloc(T** p, size_t count)
{
    *p = nullptr;
    if (count == 0) count = 1;
    return cudaMalloc((void**)p, sizeof(T) * count);
}

template <typename T>
void dfree(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

// ---- GLL points: -1, +1 and the interior roots of P_{N+1} - P_{N-1}, which
// vanish exactly where (1 - x^2) P_N' does; Newton with the derivative
// identity (P_{N+1} - P_{N-1})' = (2N+1) P_N.
void legendre3(int N, double x, double* pm1, double* p0, double* pp1)
{
    double a = 1.0, b = x;          // P_0, P_1
    if (N == 0) { *pm1 = 0.0; *p0 = 1.0; *pp1 = x; return; }
    for (int k = 1; k < N; ++k) {
        double c = ((2 * k + 1) * x * b - k * a) / (k + 1);
        a = b;
        b = c;
    }
    *pm1 = a;   // P_{N-1}
    *p0 = b;    // P_N
    *pp1 = ((2 * N + 1) * x * b - N * a) / (N + 1);
}

void gll_points(int N, double* xi)
{
    xi[0] = -1.0;
    xi[N] = 1.0;
    for (int i = 1; i < N; ++i) {
        double x = -cos(M_PI * i / N);
        for (int it = 0; it < 200; ++it) {
            double pm1, p0, pp1;
            legendre3(N, x, &pm1, &p0, &pp1);
            double dx = (pp1 - pm1) / ((2 * N + 1) * p0);
            x -= dx;
            if (fabs(dx) <= 1e-16) break;
        }
        xi[i] = x;
    }
    for (int i = 0; i < (N + 1) / 2; ++i) {
        double a = 0.5 * (xi[N - i] - xi[i]);
        xi[i] = -a;
        xi[N - i] = a;
    }
    if (N % 2 == 0) xi[N / 2] = 0.0;
}

// inverse of the Bernstein collocation matrix V[i][k] = C(N,k) u_i^k (1-u_i)^(N-k),
// u_i = (xi_i + 1)/2, by Gauss-Jordan elimination with partial pivoting
bool bernstein_inverse(int N, const double* xi, std::vector<double>& inv, double* norm_inf)
{
    const int n = N + 1;
    std::vector<double> M((size_t)n * 2 * n, 0.0);
    for (int i = 0; i < n; ++i) {
        double u = 0.5 * (xi[i] + 1.0);
        double binom = 1.0;
        for (int k = 0; k < n; ++k) {
            if (k > 0) binom = binom * (N - k + 1) / k;
            M[(size_t)i * 2 * n + k] = binom * pow(u, k) * pow(1.0 - u, N - k);
        }
        M[(size_t)i * 2 * n + n + i] = 1.0;
    }
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(M[(size_t)r * 2 * n + c]) > fabs(M[(size_t)piv * 2 * n + c])) piv = r;
        if (M[(size_t)piv * 2 * n + c] == 0.0) return false;
        if (piv != c)
            for (int k = 0; k < 2 * n; ++k) std::swap(M[(size_t)c * 2 * n + k], M[(size_t)piv * 2 * n + k]);
        double d = M[(size_t)c * 2 * n + c];
        for (int k = 0; k < 2 * n; ++k) M[(size_t)c * 2 * n + k] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = M[(size_t)r * 2 * n + c];
            if (f == 0.0) continue;
            for (int k = 0; k < 2 * n; ++k) M[(size_t)r * 2 * n + k] -= f * M[(size_t)c * 2 * n + k];
        }
    }
    inv.assign((size_t)n * n, 0.0);
    double nm = 0.0;
    for (int i = 0; i < n; ++i) {
        double row = 0.0;
        for (int k = 0; k < n; ++k) {
            inv[(size_t)i * n + k] = M[(size_t)i * 2 * n + n + k];
            row += fabs(inv[(size_t)i * n + k]);
        }
        nm = std::max(nm, row);
    }
    *norm_inf = nm;
    return true;
}

void make_tab(int N, BasisTab* t)
{
    memset(t, 0, sizeof(*t));
    double xi[NMAX];
    gll_points(N, xi);
    for (int i = 0; i <= N; ++i) {
        double p = 1.0;
        for (int m = 0; m <= N; ++m)
            if (m != i) p *= (xi[i] - xi[m]);
        t->xi[i] = xi[i];
        t->ci[i] = 1.0 / p;
        t->xif[i] = (float)xi[i];
        t->cif[i] = (float)(1.0 / p);
        t->xil[i] = (float)(xi[i] - (double)t->xif[i]);
        t->cil[i] = (float)(1.0 / p - (double)t->cif[i]);
    }
}

cudaEvent_t ev_get(fp_handle* h)
{
    if (!h->ev_free.empty()) {
        cudaEvent_t e = h->ev_free.back();
        h->ev_free.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
    return e;
}

void release(fp_handle* h)
{
    if (h->host_stream) {
        host_stream_free(h->host_stream);
        h->host_stream = nullptr;
    }
    for (int k = 0; k < PROF_KINDS; ++k) {
        for (auto& pr : h->ev_pend[k]) {
            cudaEventDestroy(pr.first);
            cudaEventDestroy(pr.second);
        }
        h->ev_pend[k].clear();
    }
    for (auto e : h->ev_free) cudaEventDestroy(e);
    h->ev_free.clear();
    dfree(h->stats);
    dfree(h->band);
    dfree(h->coords); dfree(h->coords32); dfree(h->coords32lo); dfree(h->sub); dfree(h->dist); dfree(h->boxes); dfree(h->boxes32);
    dfree(h->cell_start); dfree(h->cell_elems); dfree(h->ecount); dfree(h->estart); dfree(h->escan_tmp);
    dfree(h->cnt); dfree(h->smask); dfree(h->off); dfree(h->scan_tmp); dfree(h->pair_elem); dfree(h->pair_pt);
    dfree(h->order); dfree(h->pres); dfree(h->prst); dfree(h->pstate); dfree(h->inv);
    dfree(h->binv); dfree(h->nodebox); dfree(h->red); dfree(h->hcnt); dfree(h->htmp); dfree(h->flag);
    if (h->h_total) cudaFreeHost(h->h_total);
    h->h_total = nullptr;
}

fp_status grow_points(fp_handle* h, int64_t P)
{
    if (P <= h->cap_pts) return FP_OK;
    int64_t cap = std::max<int64_t>(P, 1024);
    cudaDeviceSynchronize();
    dfree(h->cnt); dfree(h->smask); dfree(h->off); dfree(h->scan_tmp);
    cudaError_t e;
    if ((e = dalloc(&h->cnt, cap)) != cudaSuccess || (e = dalloc(&h->smask, cap)) != cudaSuccess ||
        (e = dalloc(&h->off, cap + 1)) != cudaSuccess ||
        (e = dalloc(&h->scan_tmp, std::max(scan_tmp_elems(cap), scan_tmp_elems(h->E)))) != cudaSuccess) {
        h->cap_pts = 0;
        return cuda_fail(h, e, "workspace (points)");
    }
    h->cap_pts = cap;
    return FP_OK;
}

fp_status grow_pairs(fp_handle* h, int64_t np)
{
    if (np <= h->cap_pairs) return FP_OK;
    int64_t cap = std::max<int64_t>(np + np / 4, 2048);
    cudaDeviceSynchronize();
    dfree(h->pair_elem); dfree(h->pair_pt); dfree(h->order); dfree(h->pres); dfree(h->prst); dfree(h->pstate);
    dfree(h->inv);
    const bool two_pass = h->dim == 3 && h->opts.precision == FP_PREC_FP64;
    cudaError_t e;
    if ((e = dalloc(&h->pair_elem, cap)) != cudaSuccess || (e = dalloc(&h->pair_pt, cap)) != cudaSuccess ||
        (e = dalloc(&h->order, cap)) != cudaSuccess || (e = dalloc(&h->pres, cap)) != cudaSuccess ||
        (e = dalloc(&h->prst, 3 * cap)) != cudaSuccess ||
        (h->dim == 3 && (e = dalloc(&h->inv, cap)) != cudaSuccess) ||
        (two_pass && (e = dalloc(&h->pstate, cap)) != cudaSuccess)) {
        h->cap_pairs = 0;
        return cuda_fail(h, e, "workspace (pairs)");
    }
    h->cap_pairs = cap;
    return FP_OK;
}

}  // namespace

namespace fpg {
cudaError_t launch_count_nonfinite(int64_t n, const double* x, int32_t* out, cudaStream_t s);
}
namespace {

// A1 (element hulls), A2 (hash grid), the default distance field when asked
// for, and the mixed form's element-local FP32 geometry, all from h->coords.
// Used by fp_setup and by fp_update_coords; scratch lives in the handle and
// only grows, so an update of a mesh whose hash needs no more room than
// before allocates nothing.
fp_status build_geometry(fp_handle* h, cudaStream_t s, bool default_dist)
{
    const int n = h->n, n3 = h->dim == 2 ? n * n : n * n * n;
    const int64_t E = h->E;
    const fp_opts& o = h->opts;
    cudaError_t err;
#define GK(call, where) do { if ((err = (call)) != cudaSuccess) return cuda_fail(h, err, where); } while (0)
    if (!h->boxes) GK(dalloc(&h->boxes, E), "alloc boxes");
    if (!h->nodebox) GK(dalloc(&h->nodebox, 6 * E), "alloc nodebox");
    if (!h->red) {
        h->nred = (int)std::min<int64_t>(1024, (E + 255) / 256);
        GK(dalloc(&h->red, 12 * h->nred), "alloc red");
    }
    if (h->dim == 2)
        GK(launch_hull2(n, E, h->coords, h->binv, o.tol_border, h->pad_conv, h->boxes, h->nodebox, s), "hull");
    else
        GK(launch_hull(n, E, h->coords, h->binv, o.tol_border, h->pad_conv, h->boxes, h->nodebox, s), "hull");
    GK(launch_reduce_boxes(E, h->boxes, h->nodebox, h->red, h->nred, s), "reduce boxes");
    std::vector<double> red(12 * h->nred);
    GK(cudaMemcpyAsync(red.data(), h->red, sizeof(double) * 12 * h->nred, cudaMemcpyDeviceToHost, s), "read red");
    GK(cudaStreamSynchronize(s), "sync hull");
    double glo[3], ghi[3], nlo[3], nhi[3];
    for (int a = 0; a < 3; ++a) {
        glo[a] = INFINITY; ghi[a] = -INFINITY; nlo[a] = INFINITY; nhi[a] = -INFINITY;
        for (int b = 0; b < h->nred; ++b) {
            glo[a] = std::min(glo[a], red[12 * b + a]);
            ghi[a] = std::max(ghi[a], red[12 * b + 3 + a]);
            nlo[a] = std::min(nlo[a], red[12 * b + 6 + a]);
            nhi[a] = std::max(nhi[a], red[12 * b + 9 + a]);
        }
    }
    {
        double dx = nhi[0] - nlo[0], dy = nhi[1] - nlo[1], dz = nhi[2] - nlo[2];
        double sq = dx * dx;
        sq = sq + dy * dy;
        sq = sq + dz * dz;
        h->L = sqrt(sq);
    }

    // A2: hash grid over the global padded box, widened by hpad, the margin
    // that keeps FP32 cell lookups (mixed form) inside a listing cell
    double hpad;
    {
        double xmax = 0.0, extm = 0.0;
        for (int a = 0; a < 3; ++a) {
            xmax = std::max(xmax, std::max(fabs(glo[a]), fabs(ghi[a])));
            extm = std::max(extm, ghi[a] - glo[a]);
        }
        hpad = 9.5367431640625e-07 * (2.0 * xmax + extm);   // 2^-20 (2 max|x| + extent)
        for (int a = 0; a < 3; ++a) {
            glo[a] -= hpad;
            ghi[a] += hpad;
        }
    }
    h->hpad = hpad;
    {
        double ext[3], vol = 1.0;
        int nd = 0;
        for (int a = 0; a < 3; ++a) {
            ext[a] = ghi[a] - glo[a];
            if (a >= h->dim) ext[a] = 0.0;                   // 2D: one cell layer in z
            if (ext[a] > 0) { vol *= ext[a]; ++nd; }
        }
        double target = std::max(1.0, o.hash_cells_per_elem * (double)E);
        double hc = nd > 0 ? pow(vol / target, 1.0 / nd) : 1.0;
        int64_t dims[3];
        for (int it = 0; it < 64; ++it) {
            int64_t tot = 1;
            for (int a = 0; a < 3; ++a) {
                dims[a] = ext[a] > 0 ? std::max<int64_t>(1, (int64_t)ceil(ext[a] / hc)) : 1;
                dims[a] = std::min<int64_t>(dims[a], 1 << 20);
                tot *= dims[a];
            }
            if (tot <= (int64_t(1) << 26)) break;
            hc *= 1.25;
        }
        for (int a = 0; a < 3; ++a) {
            h->grid.org[a] = glo[a];
            h->grid.dim[a] = (int)dims[a];
            h->grid.inv[a] = ext[a] > 0 ? (double)dims[a] / ext[a] : 0.0;
        }
        h->grid.ncell = dims[0] * dims[1] * dims[2];
    }
    const int64_t ncell = h->grid.ncell;
    if (ncell > h->ncell_cap) {
        const int64_t cap = ncell + ncell / 8;
        cudaStreamSynchronize(s);
        dfree(h->hcnt); dfree(h->cell_start); dfree(h->htmp);
        h->ncell_cap = 0;
        GK(dalloc(&h->hcnt, cap), "alloc hash count");
        GK(dalloc(&h->cell_start, cap + 1), "alloc cell start");
        GK(dalloc(&h->htmp, scan_tmp_elems(cap)), "alloc scan tmp");
        h->ncell_cap = cap;
    }
    GK(cudaMemsetAsync(h->hcnt, 0, sizeof(int32_t) * ncell, s), "zero hash count");
    GK(launch_hash_count(E, h->boxes, h->grid, hpad, h->hcnt, s), "hash count");
    GK(scan_exclusive(h->hcnt, h->cell_start, ncell, h->htmp, s), "hash scan");
    GK(cudaMemcpyAsync(h->h_total, h->cell_start + ncell, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "read nnz");
    GK(cudaStreamSynchronize(s), "sync hash");
    h->nnz = h->h_total[0];
    if (h->nnz < 0) return fail(h, FP_ERR_INVALID_ARG, "hash grid overflow");
    if (h->nnz > h->nnz_cap || !h->cell_elems) {
        const int64_t cap = std::max<int64_t>(h->nnz + h->nnz / 8, 1);
        dfree(h->cell_elems);
        h->nnz_cap = 0;
        GK(dalloc(&h->cell_elems, cap), "alloc cell elems");
        h->nnz_cap = cap;
    }
    GK(cudaMemcpyAsync(h->hcnt, h->cell_start, sizeof(int32_t) * ncell, cudaMemcpyDeviceToDevice, s), "copy cursor");
    GK(launch_hash_fill(E, h->boxes, h->grid, hpad, h->hcnt, h->cell_elems, s), "hash fill");
    GK(launch_hash_sort(ncell, h->cell_start, h->cell_elems, s), "hash sort");

    // default distance field for the owner rule
    if (default_dist && h->dim == 2) {
        GK(cudaStreamSynchronize(s), "sync hash fill");
        if (!h->dist) GK(dalloc(&h->dist, (size_t)E * n3), "alloc dist");
        bool too_large = false;
        GK(launch_dist_default2(n, E, h->coords, h->sub, h->grid, h->cell_start, h->cell_elems, h->dist,
                                int64_t(1) << 37, &too_large, s), "dist default 2d");
        if (too_large) return fail(h, FP_ERR_INVALID_ARG, "mesh too large for the default distance field; pass dist");
        h->dist_default = true;
    } else if (default_dist) {
        double* fc = nullptr;
        int32_t *nb = nullptr, *nboff = nullptr, *tmp2 = nullptr;
        double* bx = nullptr;
        int32_t* bs = nullptr;
        auto cleanup = [&]() { dfree(fc); dfree(nb); dfree(nboff); dfree(tmp2); dfree(bx); dfree(bs); };
#define DK(call, where) do { if ((err = (call)) != cudaSuccess) { cleanup(); return cuda_fail(h, err, where); } } while (0)
        DK(cudaStreamSynchronize(s), "sync hash fill");
        DK(dalloc(&fc, 72 * E), "alloc face corners");
        DK(dalloc(&nb, 6 * E), "alloc face flags");
        DK(dalloc(&nboff, 6 * E + 1), "alloc face offsets");
        DK(dalloc(&tmp2, scan_tmp_elems(6 * E)), "alloc face scan");
        DK(launch_face_corners(n, E, h->coords, fc, s), "face corners");
        DK(launch_face_boundary(E, fc, h->sub, h->grid, h->cell_start, h->cell_elems, nb, s), "face boundary");
        DK(scan_exclusive(nb, nboff, 6 * E, tmp2, s), "face scan");
        DK(cudaMemcpyAsync(h->h_total, nboff + 6 * E, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "read nbnd");
        DK(cudaStreamSynchronize(s), "sync faces");
        const int64_t nbf = h->h_total[0];
        const int64_t nbn = nbf * n * n;
        if ((double)E * n3 * (double)nbn > 137438953472.0) {   // 2^37 node x boundary-node pairs
            cleanup();
            return fail(h, FP_ERR_INVALID_ARG, "mesh too large for the default distance field; pass dist");
        }
        DK(dalloc(&bx, 3 * std::max<int64_t>(nbn, 1)), "alloc boundary nodes");
        DK(dalloc(&bs, std::max<int64_t>(nbn, 1)), "alloc boundary subs");
        if (!h->dist) DK(dalloc(&h->dist, (size_t)E * n3), "alloc dist");
        DK(launch_face_gather(n, E, h->coords, h->sub, nboff, bx, bs, nbn, s), "face gather");
        DK(launch_dist_default(n, E, h->coords, h->sub, bx, bs, nbn, h->dist, s), "dist default");
        DK(cudaStreamSynchronize(s), "sync dist");
        cleanup();
#undef DK
        h->dist_default = true;
    }

    // mixed form: element-local FP32 geometry
    if (o.precision == FP_PREC_MIXED) {
        const size_t ncoord = (size_t)3 * E * n3;
        if (!h->coords32) GK(dalloc(&h->coords32, ncoord), "alloc coords32");
        if (!h->coords32lo) GK(dalloc(&h->coords32lo, ncoord), "alloc coords32lo");
        if (!h->boxes32) GK(dalloc(&h->boxes32, E), "alloc boxes32");
        GK(launch_local32(n, E, h->coords, h->boxes, h->coords32, s), "local32");
        GK(launch_local32lo(n, E, h->coords, h->boxes, h->coords32, h->coords32lo, s), "local32lo");
        GK(launch_box32(E, h->boxes, h->boxes32, s), "box32");
    }
#undef GK
    return FP_OK;
}
}  // namespace


extern "C" {

void fp_default_opts(fp_opts* o)
{
    if (!o) return;
    o->precision = FP_PREC_FP64;
    o->tol_accept = 1e-12;
    o->tol_border = 1e-6;
    o->max_newton = 40;
    o->hash_cells_per_elem = 1.0;
    o->tie_band = 1e-10;
    o->points_per_block = 0;
}

const char* fp_error_string(fp_status s)
{
    switch (s) {
        case FP_OK: return "ok";
        case FP_ERR_INVALID_ARG: return "invalid argument";
        case FP_ERR_OOM: return "device out of memory";
        case FP_ERR_CUDA: return "CUDA error";
        case FP_ERR_TIMEOUT: return "device-side wait timed out";
        case FP_ERR_NOT_SETUP: return "handle not set up";
    }
    return "unknown status";
}

const char* fp_last_error(const fp_handle* h)
{
    return h ? h->err.c_str() : g_setup_err.c_str();
}

static fp_status setup_impl(fp_handle** hout, int dim, const double* coords, int64_t E, int N, const int32_t* sub,
                            const double* dist, const fp_opts* opts_in, void* stream)
{
    if (!hout) return fail(nullptr, FP_ERR_INVALID_ARG, "fp_setup: null handle pointer");
    *hout = nullptr;
    g_setup_err.clear();
    if (!coords) return fail(nullptr, FP_ERR_INVALID_ARG, "fp_setup: null coords");
    if (E < 1 || E >= (int64_t(1) << 31)) return fail(nullptr, FP_ERR_INVALID_ARG, "fp_setup: E out of range");
    if (N < 1 || N >= NMAX) return fail(nullptr, FP_ERR_INVALID_ARG, "fp_setup: N must be in [1,15]");
    fp_opts o;
    fp_default_opts(&o);
    if (opts_in) o = *opts_in;
    if ((o.precision != FP_PREC_FP64 && o.precision != FP_PREC_MIXED) || !(o.tol_accept > 0) ||
        !(o.tol_border >= o.tol_accept) || o.max_newton < 1 || o.max_newton > 1000 ||
        !(o.hash_cells_per_elem > 0) || !(o.tie_band >= 0) || o.points_per_block < 0 ||
        o.points_per_block > 256 || (o.points_per_block % 32) != 0)
        return fail(nullptr, FP_ERR_INVALID_ARG, "fp_setup: options out of range");
    if (dim == 2 && o.precision != FP_PREC_FP64)
        return fail(nullptr, FP_ERR_INVALID_ARG, "fp_setup_2d: 2D meshes support the FP64 form only");
    const int n = N + 1, n3 = dim == 2 ? n * n : n * n * n;
    if ((int64_t)E * n3 * dim >= (int64_t(1) << 40)) return fail(nullptr, FP_ERR_INVALID_ARG, "fp_setup: mesh too large");
    cudaStream_t s = (cudaStream_t)stream;

    fp_handle* h = new fp_handle();
    h->N = N; h->n = n; h->E = E; h->opts = o; h->dim = dim;
    if (cudaGetDevice(&h->device) != cudaSuccess) h->device = -1;
    make_tab(N, &h->tab);
    cudaError_t err;
    const size_t ncoord = (size_t)dim * E * n3;
#define CK(call, where) do { if ((err = (call)) != cudaSuccess) { fp_status st = cuda_fail(nullptr, err, where); release(h); delete h; return st; } } while (0)
#define BAD(msg) do { fail(nullptr, FP_ERR_INVALID_ARG, msg); release(h); delete h; return FP_ERR_INVALID_ARG; } while (0)

    CK(dalloc(&h->coords, ncoord), "alloc coords");
    CK(cudaMemcpyAsync(h->coords, coords, sizeof(double) * ncoord, cudaMemcpyDefault, s), "copy coords");
    CK(dalloc(&h->sub, E), "alloc sub");
    if (sub) CK(cudaMemcpyAsync(h->sub, sub, sizeof(int32_t) * E, cudaMemcpyDefault, s), "copy sub");
    else CK(cudaMemsetAsync(h->sub, 0, sizeof(int32_t) * E, s), "zero sub");
    CK(cudaMallocHost((void**)&h->h_total, sizeof(int32_t) * 4), "alloc pinned");

    // validation: finite coordinates, subdomain ids in range
    {
        CK(dalloc(&h->flag, 1), "alloc flag");
        CK(cudaMemsetAsync(h->flag, 0, sizeof(int32_t), s), "zero flag");
        err = launch_count_nonfinite((int64_t)ncoord, h->coords, h->flag, s);
        if (err == cudaSuccess) err = cudaMemcpyAsync(h->h_total, h->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        CK(err, "check coords");
        if (h->h_total[0] != 0) BAD("fp_setup: non-finite coordinates");
        std::vector<int32_t> hs(E);
        CK(cudaMemcpy(hs.data(), h->sub, sizeof(int32_t) * E, cudaMemcpyDeviceToHost), "read sub");
        std::vector<char> seen(65536, 0);
        int ns = 0;
        for (int64_t e = 0; e < E; ++e) {
            if (hs[e] < 0 || hs[e] >= 65536) BAD("fp_setup: subdomain id out of [0,65536)");
            if (!seen[hs[e]]) { seen[hs[e]] = 1; ++ns; }
        }
        h->nsub = ns;
    }

    {
        double xi[NMAX];
        std::vector<double> binv;
        for (int i = 0; i < n; ++i) xi[i] = h->tab.xi[i];
        double binv_norm = 1.0;
        if (!bernstein_inverse(N, xi, binv, &binv_norm)) BAD("fp_setup: Bernstein matrix singular");
        h->pad_conv = 64.0 * 2.220446049250313e-16 * binv_norm * n;
        CK(dalloc(&h->binv, binv.size()), "alloc binv");
        CK(cudaMemcpyAsync(h->binv, binv.data(), sizeof(double) * binv.size(), cudaMemcpyHostToDevice, s),
           "copy binv");
        CK(cudaStreamSynchronize(s), "sync binv");
    }
    if (dist) {
        CK(dalloc(&h->dist, (size_t)E * n3), "alloc dist");
        CK(cudaMemcpyAsync(h->dist, dist, sizeof(double) * E * n3, cudaMemcpyDefault, s), "copy dist");
    }
    {
        fp_status st = build_geometry(h, s, !dist && h->nsub > 1);
        if (st != FP_OK) {
            g_setup_err = h->err;
            release(h);
            delete h;
            return st;
        }
    }
    CK(dalloc(&h->band, 3), "alloc band counters");
    CK(cudaMemsetAsync(h->band, 0, 3 * sizeof(unsigned long long), s), "zero band counters");
    CK(dalloc(&h->ecount, E), "alloc ecount");
    CK(dalloc(&h->estart, E + 1), "alloc estart");
    CK(cudaStreamSynchronize(s), "sync setup");
#undef CK
#undef BAD
    *hout = h;
    return FP_OK;
}

fp_status fp_setup(fp_handle** hout, const double* coords, int64_t E, int N, const int32_t* sub,
                   const double* dist, const fp_opts* opts, void* stream)
{
    return setup_impl(hout, 3, coords, E, N, sub, dist, opts, stream);
}

fp_status fp_setup_2d(fp_handle** hout, const double* coords, int64_t E, int N, const int32_t* sub,
                      const double* dist, const fp_opts* opts, void* stream)
{
    return setup_impl(hout, 2, coords, E, N, sub, dist, opts, stream);
}

fp_status fp_reserve(fp_handle* h, int64_t P)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    if (P < 0) return fail(h, FP_ERR_INVALID_ARG, "fp_reserve: P < 0");
    fp_status st = grow_points(h, P);
    if (st != FP_OK) return st;
    return grow_pairs(h, 2 * P);
}

static fp_status find_impl(fp_handle* h, int64_t P, const double* pts, const int32_t* qsess, int32_t* code,
                           int32_t* sub, int32_t* elem, double* rst, double* dist2, const EvalSpec& ev, void* stream,
                           const int32_t* warm_elem = nullptr, const double* warm_rst = nullptr)
{
    if (P < 0 || P >= (int64_t(1) << 31)) return fail(h, FP_ERR_INVALID_ARG, "fp_find: P out of range");
    if (P == 0) return FP_OK;
    if (!pts || !code || !sub || !elem || !rst || !dist2)
        return fail(h, FP_ERR_INVALID_ARG, "fp_find: null pointer argument");
    cudaStream_t s = (cudaStream_t)stream;
    fp_status st = grow_points(h, P);
    if (st != FP_OK) return st;
    FindArgs a;
    memset(&a, 0, sizeof(a));
    a.n = h->n; a.E = h->E; a.P = P; a.pts = pts; a.qsess = qsess;
    a.coords = h->coords; a.coords32 = h->coords32; a.coords32lo = h->coords32lo; a.sub = h->sub;
    a.dist = h->nsub > 1 ? h->dist : nullptr;
    a.boxes = h->boxes; a.boxes32 = h->boxes32; a.grid = &h->grid;
    a.cell_start = h->cell_start; a.cell_elems = h->cell_elems;
    a.cnt = h->cnt; a.off = h->off; a.ecount = h->ecount; a.estart = h->estart; a.scan_tmp = h->scan_tmp;
    a.smask = h->dim == 3 ? h->smask : nullptr;
    a.code = code; a.osub = sub; a.oelem = elem; a.rst = rst; a.dist2 = dist2;
    a.eval = ev;
    a.stats = h->prof ? h->stats : nullptr;
    a.band = h->band;
    a.warm_elem = warm_elem;
    a.warm_rst = warm_rst;
    cudaEvent_t scr0 = nullptr, scr1 = nullptr;
    if (h->prof) {
        for (int q = 0; q < (ev.F > 0 ? 8 : 6); ++q) a.ev[q] = ev_get(h);
        scr0 = ev_get(h);
        scr1 = ev_get(h);
        cudaEventRecord(scr0, s);
    }
    FindParams fp;
    fp.tol_accept = h->opts.tol_accept;
    fp.tol_border = h->opts.tol_border;
    fp.band = h->opts.tie_band * h->L;
    fp.max_newton = h->opts.max_newton;
    fp.mixed = h->opts.precision == FP_PREC_MIXED;
    fp.refine = h->refine;
    const bool d2 = h->dim == 2;
    cudaError_t err = d2 ? find_count2(a, s) : find_count(a, h->tab, fp, s);
    if (err != cudaSuccess) return cuda_fail(h, err, "fp_find count");
    err = cudaMemcpyAsync(h->h_total, h->off + P, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) return cuda_fail(h, err, "fp_find pair count");
    const int64_t npairs = h->h_total[0];
    if (npairs < 0) return fail(h, FP_ERR_INVALID_ARG, "fp_find: candidate pairs overflow int32");
    h->last_pairs = npairs;
    st = grow_pairs(h, npairs);
    if (st != FP_OK) return st;
    a.pair_elem = h->pair_elem; a.pair_pt = h->pair_pt; a.order = h->order;
    a.pres = h->pres; a.prst = h->prst; a.cap = h->cap_pairs; a.pstate = h->pstate;
    a.inv = d2 ? nullptr : h->inv;
    if (npairs > 0) {
        err = d2 ? find_emit2(a, s) : find_emit(a, s);
        if (err != cudaSuccess) return cuda_fail(h, err, "fp_find emit");
    }
    if (h->prof) {
        cudaEventRecord(scr1, s);
        h->ev_pend[PROF_SCREEN].push_back({scr0, scr1});
    }
    const int block = h->opts.points_per_block > 0 ? h->opts.points_per_block
                                                   : (d2 ? kDefaultBlock : kDefaultBlockFind3);
    err = d2 ? find_solve2(a, npairs, h->tab, fp, block, s) : find_solve(a, npairs, h->tab, fp, block, s);
    if (h->prof) {
        if (npairs > 0) {
            h->ev_pend[PROF_SORT].push_back({a.ev[0], a.ev[1]});
            h->ev_pend[PROF_NEWTON].push_back({a.ev[2], a.ev[3]});
            if (ev.F > 0) h->ev_pend[PROF_EVAL].push_back({a.ev[6], a.ev[7]});
        } else {
            for (int q = 0; q < 4; ++q) h->ev_free.push_back(a.ev[q]);
            if (ev.F > 0) { h->ev_free.push_back(a.ev[6]); h->ev_free.push_back(a.ev[7]); }
        }
        h->ev_pend[PROF_RANK].push_back({a.ev[4], a.ev[5]});
    }
    if (err != cudaSuccess) return cuda_fail(h, err, "fp_find solve");
    return FP_OK;
}

fp_status fp_find(fp_handle* h, int64_t P, const double* pts, const int32_t* qsess, int32_t* code, int32_t* sub,
                  int32_t* elem, double* rst, double* dist2, void* stream)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    h->err.clear();
    EvalSpec ev{0, nullptr, nullptr, nullptr};
    return find_impl(h, P, pts, qsess, code, sub, elem, rst, dist2, ev, stream);
}

struct fp_fields {
    const fp_handle* owner = nullptr;
    int F = 0;
    float2* data = nullptr;
};

// fused-eval arguments: posted double-float fields, else FP64 fields
static fp_status eval_spec(fp_handle* h, int F, const double* fields, const fp_fields* posted, double* out,
                           EvalSpec* ev)
{
    if (!out) return fail(h, FP_ERR_INVALID_ARG, "fp_find_eval: null out");
    if (posted) {
        if (posted->owner != h) return fail(h, FP_ERR_INVALID_ARG, "fp_find_eval: fields posted for another handle");
        if (F != posted->F) return fail(h, FP_ERR_INVALID_ARG, "fp_find_eval: F differs from the posted fields");
        *ev = EvalSpec{posted->F, nullptr, posted->data, out, h->stage_eval};
        return FP_OK;
    }
    if (!fields || F < 1) return fail(h, FP_ERR_INVALID_ARG, "fp_find_eval: no fields");
    if ((h->n % 2 == 0) && ((uintptr_t)fields % 16) != 0)
        return fail(h, FP_ERR_INVALID_ARG, "fp_find_eval: fields must be 16-byte aligned for even n");
    *ev = EvalSpec{F, fields, nullptr, out};
    return FP_OK;
}

fp_status fp_find_eval(fp_handle* h, int64_t P, const double* pts, const int32_t* qsess, int F, const double* fields,
                       const fp_fields* posted, int32_t* code, int32_t* sub, int32_t* elem, double* rst, double* dist2,
                       double* out, void* stream)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    h->err.clear();
    EvalSpec ev;
    fp_status st = eval_spec(h, F, fields, posted, out, &ev);
    if (st != FP_OK) return st;
    return find_impl(h, P, pts, qsess, code, sub, elem, rst, dist2, ev, stream);
}

fp_status fp_find_warm(fp_handle* h, int64_t P, const double* pts, const int32_t* qsess, const int32_t* warm_elem,
                       const double* warm_rst, int F, const double* fields, const fp_fields* posted, int32_t* code,
                       int32_t* sub, int32_t* elem, double* rst, double* dist2, double* out, void* stream)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    h->err.clear();
    if ((warm_elem == nullptr) != (warm_rst == nullptr))
        return fail(h, FP_ERR_INVALID_ARG, "fp_find_warm: warm_elem and warm_rst must both be given or both be null");
    EvalSpec ev{0, nullptr, nullptr, nullptr};
    if (F != 0 || posted) {
        fp_status st = eval_spec(h, F, fields, posted, out, &ev);
        if (st != FP_OK) return st;
    }
    return find_impl(h, P, pts, qsess, code, sub, elem, rst, dist2, ev, stream, warm_elem, warm_rst);
}

fp_status fp_update_coords(fp_handle* h, const double* coords, const double* dist, int flags, void* stream)
{
    if (!h || !h->coords) return FP_ERR_NOT_SETUP;
    h->err.clear();
    if (!coords) return fail(h, FP_ERR_INVALID_ARG, "fp_update_coords: null coords");
    if ((flags & ~FP_UPDATE_DEFAULT_DIST) != 0 || (dist && (flags & FP_UPDATE_DEFAULT_DIST)))
        return fail(h, FP_ERR_INVALID_ARG, "fp_update_coords: bad flags");
    const int n3 = h->dim == 2 ? h->n * h->n : h->n * h->n * h->n;
    const size_t ncoord = (size_t)h->dim * h->E * n3;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t err;
    // validate the new coordinates before the handle changes
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, coords) != cudaSuccess) {
        cudaGetLastError();
        at.type = cudaMemoryTypeUnregistered;
    }
    int64_t bad = 0;
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) {
        err = cudaMemsetAsync(h->flag, 0, sizeof(int32_t), s);
        if (err == cudaSuccess) err = launch_count_nonfinite((int64_t)ncoord, coords, h->flag, s);
        if (err == cudaSuccess) err = cudaMemcpyAsync(h->h_total, h->flag, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
        if (err != cudaSuccess) return cuda_fail(h, err, "fp_update_coords: check coords");
        bad = h->h_total[0];
    } else {
        for (size_t i = 0; i < ncoord; ++i) bad += !std::isfinite(coords[i]);
    }
    if (bad) return fail(h, FP_ERR_INVALID_ARG, "fp_update_coords: non-finite coordinates");
    h->stale = true;
    err = cudaMemcpyAsync(h->coords, coords, sizeof(double) * ncoord, cudaMemcpyDefault, s);
    if (err != cudaSuccess) return cuda_fail(h, err, "fp_update_coords: copy coords");
    if (dist) {
        if (!h->dist && (err = dalloc(&h->dist, (size_t)h->E * n3)) != cudaSuccess)
            return cuda_fail(h, err, "fp_update_coords: alloc dist");
        err = cudaMemcpyAsync(h->dist, dist, sizeof(double) * h->E * n3, cudaMemcpyDefault, s);
        if (err != cudaSuccess) return cuda_fail(h, err, "fp_update_coords: copy dist");
        h->dist_default = false;
    }
    fp_status st = build_geometry(h, s, (flags & FP_UPDATE_DEFAULT_DIST) && h->nsub > 1);
    if (st != FP_OK) return st;
    h->stale = false;
    return FP_OK;
}

struct fp_workspace {
    const fp_handle* owner = nullptr;
    int64_t max_points = 0, max_pairs = 0, last_P = 0;
    int persistent_blocks = 0;
    int64_t grid_pairs = 0;     // without a persistent grid: pairs the launches cover (0: max_pairs)
    int32_t *cnt = nullptr, *off = nullptr, *scan_tmp = nullptr;
    uint32_t* smask = nullptr;
    int32_t *pair_elem = nullptr, *pair_pt = nullptr, *order = nullptr;
    int32_t *ecount = nullptr, *estart = nullptr;
    double *pres = nullptr, *prst = nullptr;
    double2* pstate = nullptr;  // FP64 form: state of solves paused by the first Newton pass
    int32_t* inv = nullptr;     // sorted position of each pair slot
};

static void ws_release(fp_workspace* w)
{
    dfree(w->cnt); dfree(w->smask); dfree(w->off); dfree(w->scan_tmp); dfree(w->pair_elem); dfree(w->pair_pt);
    dfree(w->order); dfree(w->ecount); dfree(w->estart); dfree(w->pres); dfree(w->prst); dfree(w->pstate);
    dfree(w->inv);
}

fp_status fp_workspace_create(const fp_handle* h, int64_t max_points, int64_t max_pairs, fp_workspace** out)
{
    if (!out) return FP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    if (h->dim != 3) return FP_ERR_INVALID_ARG;          // workspaces serve hexahedral meshes
    if (max_points < 1 || max_points >= (int64_t(1) << 31)) return FP_ERR_INVALID_ARG;
    if (max_pairs <= 0) max_pairs = 2 * max_points;
    if (max_pairs >= (int64_t(1) << 31)) return FP_ERR_INVALID_ARG;
    fp_workspace* w = new fp_workspace();
    w->owner = h;
    w->max_points = max_points;
    w->max_pairs = max_pairs;
    int dev = 0, nsm = 1;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    w->persistent_blocks = 4 * nsm;
    cudaError_t e;
    if ((e = dalloc(&w->cnt, max_points)) != cudaSuccess || (e = dalloc(&w->smask, max_points)) != cudaSuccess ||
        (e = dalloc(&w->off, max_points + 1)) != cudaSuccess ||
        (e = dalloc(&w->scan_tmp, std::max(scan_tmp_elems(max_points), scan_tmp_elems(h->E)))) != cudaSuccess ||
        (e = dalloc(&w->pair_elem, max_pairs)) != cudaSuccess || (e = dalloc(&w->pair_pt, max_pairs)) != cudaSuccess ||
        (e = dalloc(&w->order, max_pairs)) != cudaSuccess || (e = dalloc(&w->ecount, h->E)) != cudaSuccess ||
        (e = dalloc(&w->estart, h->E + 1)) != cudaSuccess || (e = dalloc(&w->pres, max_pairs)) != cudaSuccess ||
        (e = dalloc(&w->prst, 3 * max_pairs)) != cudaSuccess || (e = dalloc(&w->inv, max_pairs)) != cudaSuccess ||
        (h->opts.precision == FP_PREC_FP64 && (e = dalloc(&w->pstate, max_pairs)) != cudaSuccess)) {
        ws_release(w);
        delete w;
        return e == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA;
    }
    *out = w;
    return FP_OK;
}

fp_status fp_workspace_bytes(const fp_handle* h, int64_t max_points, int64_t max_pairs, int64_t* bytes)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    if (!bytes || max_points < 1 || max_points >= (int64_t(1) << 31)) return FP_ERR_INVALID_ARG;
    if (max_pairs <= 0) max_pairs = 2 * max_points;
    if (max_pairs >= (int64_t(1) << 31)) return FP_ERR_INVALID_ARG;
    *bytes = 4 * max_points + 4 * max_points + 4 * (max_points + 1) + 4 * std::max(scan_tmp_elems(max_points), scan_tmp_elems(h->E)) +
             max_pairs * (4 + 4 + 4 + 4 + 8 + 24 + (h->opts.precision == FP_PREC_FP64 ? 16 : 0)) + 4 * h->E +
             4 * (h->E + 1);
    return FP_OK;
}

void fp_workspace_free(fp_workspace* w)
{
    if (!w) return;
    cudaDeviceSynchronize();
    ws_release(w);
    delete w;
}

}  // extern "C"

// a workspace whose launches cover its whole pair capacity with one block per
// 128 pairs (blocks past the device-side count exit at once) instead of a
// persistent grid: no host wait, and the Newton work balances like a launch
// sized on the host (used by the host-memory streaming path)
void fpg::workspace_unpersist(fp_workspace* w)
{
    if (w) w->persistent_blocks = 0;
}

// the pairs one block per 128 covers in the next launches of a workspace
// without a persistent grid (<= 0: the whole capacity).  The pair kernels loop
// grid-stride over the device-side count, so a count above the hint is still
// solved completely, with a second pass for the pairs beyond it.
void fpg::workspace_grid_hint(fp_workspace* w, int64_t pairs)
{
    if (w) w->grid_pairs = pairs;
}

cudaError_t fpg::workspace_pair_count_async(fp_workspace* w, int32_t* host_dst, cudaStream_t s)
{
    if (!w || w->last_P <= 0) return cudaErrorInvalidValue;
    return cudaMemcpyAsync(host_dst, w->off + w->last_P, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
}

extern "C" {

fp_status fp_workspace_last_pairs(fp_workspace* w, int64_t* npairs)
{
    if (!w) return FP_ERR_INVALID_ARG;
    int32_t t = 0;
    if (w->last_P > 0) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(&t, w->off + w->last_P, sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return FP_ERR_CUDA;
    }
    if (npairs) *npairs = t;
    return FP_OK;
}

static fp_status find_ws_impl(fp_handle* h, fp_workspace* w, int64_t P, const double* pts, const int32_t* qsess,
                              int32_t* code, int32_t* sub, int32_t* elem, double* rst, double* dist2,
                              const EvalSpec& ev, void* stream)
{
    if (!w || w->owner != h) return fail(h, FP_ERR_INVALID_ARG, "fp_find_ws: workspace belongs to another handle");
    if (P < 0 || P > w->max_points) return fail(h, FP_ERR_INVALID_ARG, "fp_find_ws: P outside [0, max_points]");
    if (P == 0) return FP_OK;
    if (!pts || !code || !sub || !elem || !rst || !dist2)
        return fail(h, FP_ERR_INVALID_ARG, "fp_find_ws: null pointer argument");
    cudaStream_t s = (cudaStream_t)stream;
    FindArgs a;
    memset(&a, 0, sizeof(a));
    a.n = h->n; a.E = h->E; a.P = P; a.pts = pts; a.qsess = qsess;
    a.coords = h->coords; a.coords32 = h->coords32; a.coords32lo = h->coords32lo; a.sub = h->sub;
    a.dist = h->nsub > 1 ? h->dist : nullptr;
    a.boxes = h->boxes; a.boxes32 = h->boxes32; a.grid = &h->grid;
    a.cell_start = h->cell_start; a.cell_elems = h->cell_elems;
    a.cnt = w->cnt; a.off = w->off; a.scan_tmp = w->scan_tmp; a.ecount = w->ecount; a.estart = w->estart;
    a.smask = w->smask;
    a.pair_elem = w->pair_elem; a.pair_pt = w->pair_pt; a.order = w->order; a.pres = w->pres; a.prst = w->prst;
    a.pstate = w->pstate;
    a.inv = w->inv;
    a.cap = w->max_pairs;
    a.persistent_blocks = w->persistent_blocks;
    a.code = code; a.osub = sub; a.oelem = elem; a.rst = rst; a.dist2 = dist2;
    a.eval = ev;
    a.band = h->band;
    FindParams fp;
    fp.tol_accept = h->opts.tol_accept;
    fp.tol_border = h->opts.tol_border;
    fp.band = h->opts.tie_band * h->L;
    fp.max_newton = h->opts.max_newton;
    fp.mixed = h->opts.precision == FP_PREC_MIXED;
    fp.refine = h->refine;
    const int block = h->opts.points_per_block > 0 ? h->opts.points_per_block : kDefaultBlock;
    cudaError_t err = find_count(a, h->tab, fp, s);
    if (err == cudaSuccess) err = find_emit(a, s);
    const int64_t grid_pairs = w->persistent_blocks == 0 && w->grid_pairs > 0 ? std::min(w->grid_pairs, w->max_pairs)
                                                                              : w->max_pairs;
    if (err == cudaSuccess) err = find_solve(a, grid_pairs, h->tab, fp, block, s);
    if (err != cudaSuccess) return cuda_fail(h, err, "fp_find_ws");
    w->last_P = P;
    return FP_OK;
}

fp_status fp_find_ws(fp_handle* h, fp_workspace* w, int64_t P, const double* pts, const int32_t* qsess,
                     int32_t* code, int32_t* sub, int32_t* elem, double* rst, double* dist2, void* stream)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    h->err.clear();
    EvalSpec ev{0, nullptr, nullptr, nullptr};
    return find_ws_impl(h, w, P, pts, qsess, code, sub, elem, rst, dist2, ev, stream);
}

fp_status fp_find_eval_ws(fp_handle* h, fp_workspace* w, int64_t P, const double* pts, const int32_t* qsess, int F,
                          const double* fields, const fp_fields* posted, int32_t* code, int32_t* sub, int32_t* elem,
                          double* rst, double* dist2, double* out, void* stream)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    h->err.clear();
    EvalSpec ev;
    fp_status st = eval_spec(h, F, fields, posted, out, &ev);
    if (st != FP_OK) return st;
    return find_ws_impl(h, w, P, pts, qsess, code, sub, elem, rst, dist2, ev, stream);
}

fp_status fp_fields_create(const fp_handle* h, int F, const double* fields, fp_fields** out, void* stream)
{
    if (!out) return FP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    if (F < 1 || !fields || h->dim != 3) return FP_ERR_INVALID_ARG;   // the mixed form is 3D only
    const int64_t n = (int64_t)F * h->E * h->n * h->n * h->n;
    fp_fields* f = new fp_fields();
    f->owner = h;
    f->F = F;
    cudaError_t e = dalloc(&f->data, n);
    if (e == cudaSuccess) e = launch_split_df(n, h->n, fields, f->data, (cudaStream_t)stream);
    if (e != cudaSuccess) {
        dfree(f->data);
        delete f;
        return e == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA;
    }
    *out = f;
    return FP_OK;
}

void fp_fields_free(fp_fields* f)
{
    if (!f) return;
    cudaDeviceSynchronize();
    dfree(f->data);
    delete f;
}

fp_status fp_eval_df(fp_handle* h, const fp_fields* f, int64_t P, const int32_t* code, const int32_t* elem,
                     const double* rst, double* out, void* stream)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    h->err.clear();
    if (!f || f->owner != h) return fail(h, FP_ERR_INVALID_ARG, "fp_eval_df: fields posted for another handle");
    if (P < 0) return fail(h, FP_ERR_INVALID_ARG, "fp_eval_df: P < 0");
    if (P == 0) return FP_OK;
    if (!code || !elem || !rst || !out) return fail(h, FP_ERR_INVALID_ARG, "fp_eval_df: null pointer");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->prof) {
        e0 = ev_get(h);
        e1 = ev_get(h);
        cudaEventRecord(e0, (cudaStream_t)stream);
    }
    cudaError_t err = launch_eval_df(h->n, h->E, P, code, elem, rst, f->F, f->data, out, h->tab, (cudaStream_t)stream);
    if (h->prof) {
        cudaEventRecord(e1, (cudaStream_t)stream);
        h->ev_pend[PROF_EVAL].push_back({e0, e1});
    }
    if (err != cudaSuccess) return cuda_fail(h, err, "fp_eval_df");
    return FP_OK;
}

struct fp_points {
    const fp_handle* owner = nullptr;
    int64_t P = 0;
    float* basis = nullptr;    // [6n][P]
    int32_t* elem = nullptr;   // [P], -1 = no value
};

fp_status fp_points_create(const fp_handle* h, int64_t P, fp_points** out)
{
    if (!out) return FP_ERR_INVALID_ARG;
    *out = nullptr;
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    if (P < 0 || P >= (int64_t(1) << 31) || h->dim != 3) return FP_ERR_INVALID_ARG;
    fp_points* q = new fp_points();
    q->owner = h;
    q->P = P;
    cudaError_t e = dalloc(&q->basis, (size_t)6 * h->n * std::max<int64_t>(P, 1));
    if (e == cudaSuccess) e = dalloc(&q->elem, std::max<int64_t>(P, 1));
    if (e != cudaSuccess) {
        dfree(q->basis);
        dfree(q->elem);
        delete q;
        return e == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA;
    }
    *out = q;
    return FP_OK;
}

void fp_points_free(fp_points* q)
{
    if (!q) return;
    cudaDeviceSynchronize();
    dfree(q->basis);
    dfree(q->elem);
    delete q;
}

fp_status fp_points_set(fp_handle* h, fp_points* q, const int32_t* code, const int32_t* elem, const double* rst,
                        void* stream)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    h->err.clear();
    if (!q || q->owner != h) return fail(h, FP_ERR_INVALID_ARG, "fp_points_set: points made for another handle");
    if (q->P == 0) return FP_OK;
    if (!code || !elem || !rst) return fail(h, FP_ERR_INVALID_ARG, "fp_points_set: null pointer");
    cudaError_t err = launch_points_basis(h->n, q->P, code, elem, rst, q->basis, q->elem, h->tab,
                                          (cudaStream_t)stream);
    if (err != cudaSuccess) return cuda_fail(h, err, "fp_points_set");
    return FP_OK;
}

fp_status fp_eval_points(fp_handle* h, const fp_fields* f, const fp_points* q, double* out, void* stream)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    h->err.clear();
    if (!f || f->owner != h) return fail(h, FP_ERR_INVALID_ARG, "fp_eval_points: fields posted for another handle");
    if (!q || q->owner != h) return fail(h, FP_ERR_INVALID_ARG, "fp_eval_points: points made for another handle");
    if (q->P == 0) return FP_OK;
    if (!out) return fail(h, FP_ERR_INVALID_ARG, "fp_eval_points: null out");
    cudaError_t err = launch_eval_points_df(h->n, h->E, q->P, f->F, q->elem, q->basis, f->data, out,
                                            (cudaStream_t)stream);
    if (err != cudaSuccess) return cuda_fail(h, err, "fp_eval_points");
    return FP_OK;
}

fp_status fp_eval(fp_handle* h, int64_t P, const int32_t* code, const int32_t* elem, const double* rst, int F,
                  const double* fields, double* out, void* stream)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    h->err.clear();
    if (P < 0 || F < 1) return fail(h, FP_ERR_INVALID_ARG, "fp_eval: P < 0 or F < 1");
    if (P == 0) return FP_OK;
    if (!code || !elem || !rst || !fields || !out) return fail(h, FP_ERR_INVALID_ARG, "fp_eval: null pointer");
    if ((h->n % 2 == 0) && ((uintptr_t)fields % 16) != 0)
        return fail(h, FP_ERR_INVALID_ARG, "fp_eval: fields must be 16-byte aligned for even n");
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->prof) {
        e0 = ev_get(h);
        e1 = ev_get(h);
        cudaEventRecord(e0, (cudaStream_t)stream);
    }
    cudaError_t err = h->dim == 2
                          ? launch_eval2(h->n, h->E, P, code, elem, rst, F, fields, out, h->tab, (cudaStream_t)stream)
                          : launch_eval(h->n, h->E, P, code, elem, rst, F, fields, out, h->tab, (cudaStream_t)stream);
    if (h->prof) {
        cudaEventRecord(e1, (cudaStream_t)stream);
        h->ev_pend[PROF_EVAL].push_back({e0, e1});
    }
    if (err != cudaSuccess) return cuda_fail(h, err, "fp_eval");
    return FP_OK;
}

void fp_free(fp_handle* h)
{
    if (!h) return;
    cudaDeviceSynchronize();
    release(h);
    delete h;
}

fp_status fp_profile(fp_handle* h, int enable)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    h->prof = enable != 0;
    if (h->prof && !h->stats) {
        cudaError_t e = dalloc(&h->stats, 4);
        if (e == cudaSuccess) e = cudaMemset(h->stats, 0, 4 * sizeof(unsigned long long));
        if (e != cudaSuccess) return cuda_fail(h, e, "fp_profile");
    }
    return FP_OK;
}

fp_status fp_set_eval_staging(fp_handle* h, int enable)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    h->stage_eval = enable != 0;
    return FP_OK;
}

fp_status fp_set_mixed_refine(fp_handle* h, int max_residuals)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    if (max_residuals < 0 || max_residuals > 8) return FP_ERR_INVALID_ARG;
    h->refine = max_residuals;
    return FP_OK;
}

fp_status fp_profile_read(fp_handle* h, int kind, double* total_ms, int64_t* launches)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    if (kind < 0 || kind >= PROF_KINDS) return fail(h, FP_ERR_INVALID_ARG, "fp_profile_read: kind out of range");
    double tot = 0.0;
    int64_t cnt = 0;
    for (auto& pr : h->ev_pend[kind]) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(pr.second);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, pr.first, pr.second);
        if (e != cudaSuccess) return cuda_fail(h, e, "fp_profile_read");
        tot += ms;
        ++cnt;
        h->ev_free.push_back(pr.first);
        h->ev_free.push_back(pr.second);
    }
    h->ev_pend[kind].clear();
    if (total_ms) *total_ms = tot;
    if (launches) *launches = cnt;
    return FP_OK;
}

int64_t fp_launch_count(void) { return fpg::g_launches.load(); }

fp_status fp_last_find_stats(const fp_handle* h, int64_t* npairs)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    if (npairs) *npairs = h->last_pairs;
    return FP_OK;
}

fp_status fp_newton_paths(fp_handle* h, int64_t* counts)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    unsigned long long c[4] = {0, 0, 0, 0};
    if (h->stats) {
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(c, h->stats, sizeof(c), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemset(h->stats, 0, sizeof(c));
        if (e != cudaSuccess) return cuda_fail(h, e, "fp_newton_paths");
    }
    for (int k = 0; k < 4; ++k) counts[k] = (int64_t)c[k];
    return FP_OK;
}

fp_status fp_memory(const fp_handle* h, int64_t* resident, int64_t* workspace)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    const int64_t n3 = h->dim == 2 ? (int64_t)h->n * h->n : (int64_t)h->n * h->n * h->n;
    const int64_t nc = h->dim * h->E * n3;
    if (resident) {
        int64_t b = 8 * nc + 4 * h->E + (int64_t)sizeof(ElemBox) * h->E + 48 * h->E + 4 * (h->ncell_cap + 1) +
                    4 * h->ncell_cap + 4 * scan_tmp_elems(h->ncell_cap) + 4 * h->nnz_cap + 8 * (int64_t)h->n * h->n +
                    96 * (int64_t)h->nred + 4 * h->E + 4 * (h->E + 1);
        if (h->dist) b += 8 * h->E * n3;
        if (h->coords32) b += 8 * nc + (int64_t)sizeof(ElemBox32) * h->E;
        *resident = b;
    }
    if (workspace)
        *workspace = 4 * h->cap_pts + 4 * h->cap_pts + 4 * (h->cap_pts + 1) +
                     4 * (h->cap_pts > 0 ? std::max(scan_tmp_elems(h->cap_pts), scan_tmp_elems(h->E)) : 0) +
                     h->cap_pairs * (4 + 4 + 4 + 8 + 24 + (h->pstate ? 16 : 0) + (h->inv ? 4 : 0));
    return FP_OK;
}

fp_status fp_band_hits(fp_handle* h, int64_t* counts)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    if (!counts) return fail(h, FP_ERR_INVALID_ARG, "fp_band_hits: null counts");
    unsigned long long c[3] = {0, 0, 0};
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(c, h->band, sizeof(c), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(h->band, 0, sizeof(c));
    if (e != cudaSuccess) return cuda_fail(h, e, "fp_band_hits");
    for (int k = 0; k < 3; ++k) counts[k] = (int64_t)c[k];
    return FP_OK;
}

fp_status fp_info(const fp_handle* h, int64_t* E, int* N, int64_t* ncell, int64_t* nnz, int* nsub)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    if (E) *E = h->E;
    if (N) *N = h->N;
    if (ncell) *ncell = h->grid.ncell;
    if (nnz) *nnz = h->nnz;
    if (nsub) *nsub = h->nsub;
    return FP_OK;
}

fp_status fp_debug_boxes(const fp_handle* h, double* aabb, double* grid, int32_t* cell_start, int32_t* cell_elems,
                         void* stream)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t err = cudaSuccess;
    if (aabb) {
        for (int a = 0; a < 3 && err == cudaSuccess; ++a) {
            err = cudaMemcpy2DAsync(aabb + a, 6 * sizeof(double), (const char*)h->boxes + offsetof(ElemBox, blo) + a * sizeof(double),
                                    sizeof(ElemBox), sizeof(double), h->E, cudaMemcpyDeviceToDevice, s);
            if (err == cudaSuccess)
                err = cudaMemcpy2DAsync(aabb + 3 + a, 6 * sizeof(double),
                                        (const char*)h->boxes + offsetof(ElemBox, bhi) + a * sizeof(double),
                                        sizeof(ElemBox), sizeof(double), h->E, cudaMemcpyDeviceToDevice, s);
        }
    }
    if (grid && err == cudaSuccess) {
        double g[9];
        for (int a = 0; a < 3; ++a) {
            g[a] = h->grid.org[a];
            g[3 + a] = h->grid.inv[a];
            g[6 + a] = (double)h->grid.dim[a];
        }
        err = cudaMemcpyAsync(grid, g, sizeof(g), cudaMemcpyHostToDevice, s);
        if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    }
    if (cell_start && err == cudaSuccess)
        err = cudaMemcpyAsync(cell_start, h->cell_start, sizeof(int32_t) * (h->grid.ncell + 1), cudaMemcpyDeviceToDevice, s);
    if (cell_elems && err == cudaSuccess)
        err = cudaMemcpyAsync(cell_elems, h->cell_elems, sizeof(int32_t) * std::max<int64_t>(h->nnz, 0),
                              cudaMemcpyDeviceToDevice, s);
    if (err != cudaSuccess) return FP_ERR_CUDA;
    return FP_OK;
}

}  // extern "C"
