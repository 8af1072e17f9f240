// fp_batch.cu -- many independent meshes (instances) of different E and N
// located and interpolated together.
//
// Instances of the same order N form a group.  At creation each group gets
// device-resident concatenations of its instances' geometry, element boxes,
// subdomain ids and fields.  One run then, per group:
//   gathers the group's points (one 2-D copy per instance),
//   screens each instance against its own hash grid and boxes (one launch
//   per instance, pair indices offset into the group),
//   scans the group's pair counts and emits the pairs,
//   sorts all pairs of the group by element, solves them with one
//   grid-stride Newton launch (the device alone knows the pair count),
//   classifies, evaluates, and scatters the results back to the caller's
//   instance-ordered arrays.
// Nothing waits on the host, so a run can be captured into one CUDA graph and
// replayed with a single launch.  The Newton schedule (threads per block,
// blocks per SM of the grid-stride loop) is chosen by fp_batch_tune, which
// times every candidate on the caller's data and keeps the fastest.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <string>
#include <vector>

#include "fp_common.cuh"
#include "fp_handle.h"
#include "fp_internal.h"

using namespace fpg;

namespace {

struct Group {
    int N = 0, n = 0;
    std::vector<int> inst;        // batch instance indices, in batch order
    std::vector<int64_t> eoff;    // element offset of each member (size + 1)
    std::vector<int64_t> goff;    // point offset of each member (size + 1)
    int64_t E = 0, P = 0, cap = 0;
    BasisTab tab{};
    FindParams fp{};
    double* coords = nullptr;
    float* coords32 = nullptr;
    float* coords32lo = nullptr;
    int32_t* sub = nullptr;
    ElemBox* boxes = nullptr;
    double* dist = nullptr;
    double* fields = nullptr;
    float2* fields_df = nullptr;  // mixed form: double-float copy of the fields
    // per-run buffers
    double* pts = nullptr;
    int32_t *code = nullptr, *osub = nullptr, *oelem = nullptr;
    double *rst = nullptr, *dist2 = nullptr, *out = nullptr;
    int32_t *cnt = nullptr, *off = nullptr, *scan_tmp = nullptr;
    int32_t *pair_elem = nullptr, *pair_pt = nullptr, *order = nullptr, *ecount = nullptr, *estart = nullptr;
    double *pres = nullptr, *prst = nullptr;
};

template <typename T>
cudaError_t alloc(T** p, int64_t n)
{
    *p = nullptr;
    return cudaMalloc((void**)p, sizeof(T) * (size_t)std::max<int64_t>(n, 1));
}

template <typename T>
void release(T*& p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

void release_group(Group& g)
{
    release(g.coords); release(g.coords32); release(g.coords32lo); release(g.sub); release(g.boxes); release(g.dist); release(g.fields);
    release(g.fields_df);
    release(g.pts); release(g.code); release(g.osub); release(g.oelem); release(g.rst); release(g.dist2);
    release(g.out); release(g.cnt); release(g.off); release(g.scan_tmp); release(g.pair_elem); release(g.pair_pt);
    release(g.order); release(g.ecount); release(g.estart); release(g.pres); release(g.prst);
}

}  // namespace

namespace fpg {
// copy element ids of one instance back to the caller, from group to instance numbering
__global__ void k_elem_unshift(int64_t n, const int32_t* __restrict__ src, int32_t shift, int32_t* __restrict__ dst)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) {
        const int32_t e = src[i];
        dst[i] = e >= 0 ? e - shift : e;
    }
}
}  // namespace fpg

struct fp_batch {
    int ninst = 0, F = 0;
    std::vector<fp_handle*> h;
    std::vector<int64_t> npts, uoff;
    int64_t Ptot = 0;
    std::vector<Group> groups;
    int nsm = 1;
    int block = 128;              // Newton threads per block
    int bps = 4;                  // Newton blocks per SM (grid-stride)
    cudaStream_t cap_stream = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int64_t graph_kernels = 0;    // library kernels inside the captured graph
    std::string err;
};

static fp_status bfail(fp_batch* b, fp_status s, const std::string& m)
{
    if (b) b->err = m;
    return s;
}

static void batch_release(fp_batch* b)
{
    for (auto& g : b->groups) release_group(g);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    b->exec = nullptr;
    b->graph = nullptr;
    b->cap_stream = nullptr;
}

extern "C" fp_status fp_batch_create(fp_batch** out, int ninst, fp_handle* const* handles, const int64_t* npts, int F,
                                     const double* const* fields, double pairs_per_point)
{
    if (!out) return FP_ERR_INVALID_ARG;
    *out = nullptr;
    if (ninst < 1 || !handles || !npts || F < 0 || (F > 0 && !fields)) return FP_ERR_INVALID_ARG;
    if (!(pairs_per_point > 0)) pairs_per_point = 2.0;
    fp_batch* b = new fp_batch();
    b->ninst = ninst;
    b->F = F;
    b->h.assign(handles, handles + ninst);
    b->npts.assign(npts, npts + ninst);
    b->uoff.assign(ninst + 1, 0);
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev);
    for (int i = 0; i < ninst; ++i) {
        fp_handle* h = handles[i];
        if (!h || !h->coords || h->dim != 3 || npts[i] < 0) {
            delete b;
            return FP_ERR_INVALID_ARG;
        }
        const fp_opts& o0 = handles[0]->opts;
        if (h->opts.precision != o0.precision || h->opts.tol_accept != o0.tol_accept ||
            h->opts.tol_border != o0.tol_border || h->opts.max_newton != o0.max_newton ||
            h->opts.tie_band != o0.tie_band) {
            delete b;
            return FP_ERR_INVALID_ARG;
        }
        b->uoff[i + 1] = b->uoff[i] + npts[i];
    }
    b->Ptot = b->uoff[ninst];
    if (b->Ptot >= (int64_t(1) << 31)) {
        delete b;
        return FP_ERR_INVALID_ARG;
    }
    // group instances by order N, groups in order of first appearance
    std::map<int, int> gid;
    for (int i = 0; i < ninst; ++i) {
        int N = handles[i]->N;
        if (!gid.count(N)) {
            gid[N] = (int)b->groups.size();
            b->groups.emplace_back();
            b->groups.back().N = N;
            b->groups.back().n = N + 1;
            b->groups.back().tab = handles[i]->tab;
        }
        b->groups[gid[N]].inst.push_back(i);
    }
    cudaError_t e = cudaSuccess;
    const fp_opts& o = handles[0]->opts;
    for (auto& g : b->groups) {
        const int n3 = g.n * g.n * g.n;
        g.eoff.assign(g.inst.size() + 1, 0);
        g.goff.assign(g.inst.size() + 1, 0);
        double Lmax = 0.0;
        bool multi = false;
        for (size_t k = 0; k < g.inst.size(); ++k) {
            fp_handle* h = handles[g.inst[k]];
            g.eoff[k + 1] = g.eoff[k] + h->E;
            g.goff[k + 1] = g.goff[k] + npts[g.inst[k]];
            Lmax = std::max(Lmax, h->L);
            multi = multi || h->nsub > 1;
        }
        g.E = g.eoff.back();
        g.P = g.goff.back();
        g.cap = std::max<int64_t>((int64_t)ceil(pairs_per_point * (double)g.P), 1024);
        if (g.E >= (int64_t(1) << 31) || g.cap >= (int64_t(1) << 31)) e = cudaErrorInvalidValue;
        g.fp.tol_accept = o.tol_accept;
        g.fp.tol_border = o.tol_border;
        g.fp.band = o.tie_band * Lmax;
        g.fp.max_newton = o.max_newton;
        g.fp.mixed = o.precision == FP_PREC_MIXED;
        if (e == cudaSuccess) e = alloc(&g.coords, 3 * g.E * n3);
        if (e == cudaSuccess && g.fp.mixed) e = alloc(&g.coords32, 3 * g.E * n3);
        if (e == cudaSuccess && g.fp.mixed) e = alloc(&g.coords32lo, 3 * g.E * n3);
        if (e == cudaSuccess) e = alloc(&g.sub, g.E);
        if (e == cudaSuccess) e = alloc(&g.boxes, g.E);
        if (e == cudaSuccess && multi) e = alloc(&g.dist, g.E * n3);
        if (e == cudaSuccess && F > 0) e = alloc(&g.fields, (int64_t)F * g.E * n3);
        for (size_t k = 0; k < g.inst.size() && e == cudaSuccess; ++k) {
            fp_handle* h = handles[g.inst[k]];
            const int64_t eo = g.eoff[k], Ei = h->E;
            for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
                e = cudaMemcpy(g.coords + (a * g.E + eo) * n3, h->coords + a * Ei * n3, sizeof(double) * Ei * n3,
                               cudaMemcpyDeviceToDevice);
                if (e == cudaSuccess && g.fp.mixed)
                    e = cudaMemcpy(g.coords32 + (a * g.E + eo) * n3, h->coords32 + a * Ei * n3,
                                   sizeof(float) * Ei * n3, cudaMemcpyDeviceToDevice);
                if (e == cudaSuccess && g.fp.mixed)
                    e = cudaMemcpy(g.coords32lo + (a * g.E + eo) * n3, h->coords32lo + a * Ei * n3,
                                   sizeof(float) * Ei * n3, cudaMemcpyDeviceToDevice);
            }
            if (e == cudaSuccess) e = cudaMemcpy(g.sub + eo, h->sub, sizeof(int32_t) * Ei, cudaMemcpyDeviceToDevice);
            if (e == cudaSuccess)
                e = cudaMemcpy(g.boxes + eo, h->boxes, sizeof(ElemBox) * Ei, cudaMemcpyDeviceToDevice);
            if (e == cudaSuccess && g.dist) {
                if (h->nsub > 1 && h->dist)
                    e = cudaMemcpy(g.dist + eo * n3, h->dist, sizeof(double) * Ei * n3, cudaMemcpyDeviceToDevice);
                else
                    e = cudaMemset(g.dist + eo * n3, 0, sizeof(double) * Ei * n3);
            }
            for (int f = 0; f < F && e == cudaSuccess; ++f) {
                const double* src = fields[g.inst[k]];
                if (!src) { e = cudaErrorInvalidValue; break; }
                e = cudaMemcpy(g.fields + ((int64_t)f * g.E + eo) * n3, src + (int64_t)f * Ei * n3,
                               sizeof(double) * Ei * n3, cudaMemcpyDeviceToDevice);
            }
        }
        if (e == cudaSuccess && F > 0 && g.fp.mixed) {
            const int64_t nv = (int64_t)F * g.E * n3;
            e = alloc(&g.fields_df, nv);
            if (e == cudaSuccess) e = launch_split_df(nv, g.fields, g.fields_df, 0);
            if (e == cudaSuccess) e = cudaDeviceSynchronize();
        }
        if (e == cudaSuccess) e = alloc(&g.pts, 3 * g.P);
        if (e == cudaSuccess) e = alloc(&g.code, g.P);
        if (e == cudaSuccess) e = alloc(&g.osub, g.P);
        if (e == cudaSuccess) e = alloc(&g.oelem, g.P);
        if (e == cudaSuccess) e = alloc(&g.rst, 3 * g.P);
        if (e == cudaSuccess) e = alloc(&g.dist2, g.P);
        if (e == cudaSuccess && F > 0) e = alloc(&g.out, (int64_t)F * g.P);
        if (e == cudaSuccess) e = alloc(&g.cnt, g.P);
        if (e == cudaSuccess) e = alloc(&g.off, g.P + 1);
        if (e == cudaSuccess) e = alloc(&g.scan_tmp, std::max(scan_tmp_elems(g.P), scan_tmp_elems(g.E)));
        if (e == cudaSuccess) e = alloc(&g.pair_elem, g.cap);
        if (e == cudaSuccess) e = alloc(&g.pair_pt, g.cap);
        if (e == cudaSuccess) e = alloc(&g.order, g.cap);
        if (e == cudaSuccess) e = alloc(&g.ecount, g.E);
        if (e == cudaSuccess) e = alloc(&g.estart, g.E + 1);
        if (e == cudaSuccess) e = alloc(&g.pres, g.cap);
        if (e == cudaSuccess) e = alloc(&g.prst, 3 * g.cap);
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        batch_release(b);
        delete b;
        return e == cudaErrorMemoryAllocation ? FP_ERR_OOM : (e == cudaErrorInvalidValue ? FP_ERR_INVALID_ARG : FP_ERR_CUDA);
    }
    *out = b;
    return FP_OK;
}

// one run of the whole batch on stream s (no host waits)
static cudaError_t batch_run(fp_batch* b, const double* pts, int32_t* code, int32_t* sub, int32_t* elem, double* rst,
                             double* dist2, double* out, cudaStream_t s)
{
    cudaError_t e = cudaSuccess;
    const int64_t Pt = b->Ptot;
    for (auto& g : b->groups) {
        if (g.P == 0) continue;
        const int m = (int)g.inst.size();
        // gather the group's points
        for (int k = 0; k < m && e == cudaSuccess; ++k) {
            const int i = g.inst[k];
            if (b->npts[i] == 0) continue;
            e = cudaMemcpy2DAsync(g.pts + g.goff[k], sizeof(double) * g.P, pts + b->uoff[i], sizeof(double) * Pt,
                                  sizeof(double) * b->npts[i], 3, cudaMemcpyDeviceToDevice, s);
        }
        // per-instance screen against the instance's own grid and boxes
        FindArgs a;
        memset(&a, 0, sizeof(a));
        for (int k = 0; k < m && e == cudaSuccess; ++k) {
            const int i = g.inst[k];
            if (b->npts[i] == 0) continue;
            fp_handle* h = b->h[i];
            a.n = g.n; a.E = h->E; a.P = b->npts[i];
            a.pts = g.pts + g.goff[k]; a.pts_stride = g.P; a.qsess = nullptr;
            a.sub = h->sub; a.boxes = h->boxes; a.boxes32 = h->boxes32; a.grid = &h->grid;
            a.cell_start = h->cell_start; a.cell_elems = h->cell_elems;
            a.cnt = g.cnt + g.goff[k];
            e = find_screen_count(a, s);
        }
        if (e == cudaSuccess) e = scan_exclusive(g.cnt, g.off, g.P, g.scan_tmp, s);
        for (int k = 0; k < m && e == cudaSuccess; ++k) {
            const int i = g.inst[k];
            if (b->npts[i] == 0) continue;
            fp_handle* h = b->h[i];
            a.n = g.n; a.E = h->E; a.P = b->npts[i];
            a.pts = g.pts + g.goff[k]; a.pts_stride = g.P; a.qsess = nullptr;
            a.sub = h->sub; a.boxes = h->boxes; a.boxes32 = h->boxes32; a.grid = &h->grid;
            a.cell_start = h->cell_start; a.cell_elems = h->cell_elems;
            a.off = g.off + g.goff[k];
            a.pair_elem = g.pair_elem; a.pair_pt = g.pair_pt; a.cap = g.cap;
            a.pt_base = (int32_t)g.goff[k]; a.elem_base = (int32_t)g.eoff[k];
            e = find_emit(a, s);
        }
        if (e != cudaSuccess) return e;
        // one pipeline over the whole group
        FindArgs c;
        memset(&c, 0, sizeof(c));
        c.n = g.n; c.E = g.E; c.P = g.P; c.pts = g.pts;
        c.coords = g.coords; c.coords32 = g.coords32; c.coords32lo = g.coords32lo; c.sub = g.sub; c.dist = g.dist; c.boxes = g.boxes;
        c.cnt = g.cnt; c.off = g.off; c.scan_tmp = g.scan_tmp; c.ecount = g.ecount; c.estart = g.estart;
        c.pair_elem = g.pair_elem; c.pair_pt = g.pair_pt; c.order = g.order; c.pres = g.pres; c.prst = g.prst;
        c.cap = g.cap;
        c.persistent_blocks = b->bps * b->nsm;
        c.code = g.code; c.osub = g.osub; c.oelem = g.oelem; c.rst = g.rst; c.dist2 = g.dist2;
        if (b->F > 0 && out)   // fused eval in the element-sorted pair order
            c.eval = EvalSpec{b->F, g.fields_df ? nullptr : g.fields, g.fields_df, g.out};
        e = find_solve(c, g.cap, g.tab, g.fp, b->block, s);
        // scatter back to instance order
        for (int k = 0; k < m && e == cudaSuccess; ++k) {
            const int i = g.inst[k];
            const int64_t Pi = b->npts[i], go = g.goff[k], uo = b->uoff[i];
            if (Pi == 0) continue;
            e = cudaMemcpyAsync(code + uo, g.code + go, sizeof(int32_t) * Pi, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(sub + uo, g.osub + go, sizeof(int32_t) * Pi, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) {
                k_elem_unshift<<<(unsigned)((Pi + 255) / 256), 256, 0, s>>>(Pi, g.oelem + go, (int32_t)g.eoff[k],
                                                                          elem + uo);
                count_launch();
                e = cudaGetLastError();
            }
            if (e == cudaSuccess)
                e = cudaMemcpy2DAsync(rst + uo, sizeof(double) * Pt, g.rst + go, sizeof(double) * g.P,
                                      sizeof(double) * Pi, 3, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(dist2 + uo, g.dist2 + go, sizeof(double) * Pi, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess && b->F > 0 && out)
                e = cudaMemcpy2DAsync(out + uo, sizeof(double) * Pt, g.out + go, sizeof(double) * g.P,
                                      sizeof(double) * Pi, b->F, cudaMemcpyDeviceToDevice, s);
        }
        if (e != cudaSuccess) return e;
    }
    return e;
}

static fp_status check_run_args(fp_batch* b, const double* pts, int32_t* code, int32_t* sub, int32_t* elem,
                                double* rst, double* dist2)
{
    if (!b) return FP_ERR_INVALID_ARG;
    b->err.clear();
    if (b->Ptot > 0 && (!pts || !code || !sub || !elem || !rst || !dist2))
        return bfail(b, FP_ERR_INVALID_ARG, "fp_batch: null pointer argument");
    return FP_OK;
}

extern "C" fp_status fp_batch_run(fp_batch* b, const double* pts, int32_t* code, int32_t* sub, int32_t* elem,
                                  double* rst, double* dist2, double* out, void* stream)
{
    fp_status st = check_run_args(b, pts, code, sub, elem, rst, dist2);
    if (st != FP_OK) return st;
    cudaError_t e = batch_run(b, pts, code, sub, elem, rst, dist2, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return bfail(b, FP_ERR_CUDA, std::string("fp_batch_run: ") + cudaGetErrorString(e));
    return FP_OK;
}

extern "C" fp_status fp_batch_tune(fp_batch* b, const double* pts, int32_t* code, int32_t* sub, int32_t* elem,
                                   double* rst, double* dist2, double* out, void* stream, int reps, double* best_ms)
{
    fp_status st = check_run_args(b, pts, code, sub, elem, rst, dist2);
    if (st != FP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (reps < 1) reps = 2;
    const int blocks[] = {64, 128, 256};
    const int per_sm[] = {1, 2, 4, 8};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bfail(b, FP_ERR_CUDA, "fp_batch_tune: events");
    float best = INFINITY;
    int bb = b->block, bs = b->bps;
    cudaError_t e = cudaSuccess;
    for (int blk : blocks) {
        for (int ps : per_sm) {
            b->block = blk;
            b->bps = ps;
            e = batch_run(b, pts, code, sub, elem, rst, dist2, out, s);     // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(e0, s);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = batch_run(b, pts, code, sub, elem, rst, dist2, out, s);
            if (e == cudaSuccess) e = cudaEventRecord(e1, s);
            if (e == cudaSuccess) e = cudaEventSynchronize(e1);
            float ms = 0.0f;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
            if (e != cudaSuccess) break;
            ms /= reps;
            if (ms < best) {
                best = ms;
                bb = blk;
                bs = ps;
            }
        }
        if (e != cudaSuccess) break;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->block = bb;
    b->bps = bs;
    if (e != cudaSuccess) return bfail(b, FP_ERR_CUDA, std::string("fp_batch_tune: ") + cudaGetErrorString(e));
    if (best_ms) *best_ms = best;
    return FP_OK;
}

extern "C" fp_status fp_batch_schedule(fp_batch* b, int* block, int* blocks_per_sm)
{
    if (!b) return FP_ERR_INVALID_ARG;
    if (block) {
        if (*block > 0) {
            if (*block % 32 != 0 || *block > 256) return bfail(b, FP_ERR_INVALID_ARG, "fp_batch_schedule: block");
            b->block = *block;
        }
        *block = b->block;
    }
    if (blocks_per_sm) {
        if (*blocks_per_sm > 0) b->bps = std::min(*blocks_per_sm, 64);
        *blocks_per_sm = b->bps;
    }
    return FP_OK;
}

extern "C" fp_status fp_batch_capture(fp_batch* b, const double* pts, int32_t* code, int32_t* sub, int32_t* elem,
                                      double* rst, double* dist2, double* out)
{
    fp_status st = check_run_args(b, pts, code, sub, elem, rst, dist2);
    if (st != FP_OK) return st;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bfail(b, FP_ERR_CUDA, std::string("fp_batch_capture: ") + cudaGetErrorString(e));
    const int64_t k0 = fp_launch_count();
    cudaError_t er = batch_run(b, pts, code, sub, elem, rst, dist2, out, b->cap_stream);
    b->graph_kernels = fp_launch_count() - k0;
    e = cudaStreamEndCapture(b->cap_stream, &b->graph);
    if (er != cudaSuccess) e = er;
    if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
    if (e != cudaSuccess) return bfail(b, FP_ERR_CUDA, std::string("fp_batch_capture: ") + cudaGetErrorString(e));
    return FP_OK;
}

extern "C" fp_status fp_batch_launch(fp_batch* b, void* stream)
{
    if (!b || !b->exec) return bfail(b, FP_ERR_NOT_SETUP, "fp_batch_launch: no captured graph");
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return bfail(b, FP_ERR_CUDA, std::string("fp_batch_launch: ") + cudaGetErrorString(e));
    count_launch((int)b->graph_kernels);
    return FP_OK;
}

extern "C" const char* fp_batch_last_error(const fp_batch* b)
{
    return b ? b->err.c_str() : "";
}

extern "C" void fp_batch_free(fp_batch* b)
{
    if (!b) return;
    cudaDeviceSynchronize();
    batch_release(b);
    delete b;
}
