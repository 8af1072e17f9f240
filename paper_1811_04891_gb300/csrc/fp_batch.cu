// fp_batch.cu -- many independent meshes (instances) of different E and N
// located and interpolated together (the paper posts every session's mesh to
// one findpts_setup and queries them in one call, Sec. 2.1).
//
// Elements of all instances share one batch numbering, grouped by order N
// (group g owns the ids [ebase_g, ebase_g + E_g)); each group keeps
// device-resident concatenations of its instances' geometry, boxes and
// fields.  One run is a fixed launch sequence that never waits on the host:
//   k_bscreen (count)   one thread per point of every instance, screened
//                       against its own instance's hash grid and boxes
//   scan                pair offsets over all points
//   k_bscreen (emit)    (point, batch element) pairs in point order
//   sort                counting sort of all pairs by batch element, so each
//                       group's pairs are one contiguous range of positions
//   Newton, per group   a persistent launch whose warps draw work items of
//                       `tile` sorted positions from a device counter (the
//                       groups' launches run concurrently on their own
//                       streams); mixed form: its FP64 fallback after it
//   k_rank_batch        classification / ownership of every point, each
//                       with its instance's tie band; results written in the
//                       caller's order with instance-local element ids
//   eval, per group     fused evaluation of the winning pairs
// The Newton stage is one launch per order N because its register budget
// and unrolled contractions depend on N.  fp_batch_tune chooses, per group,
// the threads per block, blocks per SM and work-item size by timing the
// group's Newton stage on the caller's data, and caches the choice per
// (form, N, E bucket, pairs bucket) for later batches.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "fp_common.cuh"
#include "fp_handle.h"
#include "fp_internal.h"
#include "fp_rank.cuh"

using namespace fpg;

namespace {

struct Sched {
    int block = 128;      // Newton threads per block
    int bps = 4;          // Newton blocks per SM (persistent grid)
    int tile = 128;       // sorted positions per work item (one warp's)
};

struct Group {
    int N = 0, n = 0;
    std::vector<int> inst;        // batch instance indices, in batch order
    int64_t E = 0, P = 0;
    int32_t ebase = 0;
    BasisTab tab{};
    FindParams fp{};
    double* coords = nullptr;
    float* coords32 = nullptr;
    float* coords32lo = nullptr;
    ElemBox* boxes = nullptr;
    double* dist = nullptr;
    double* fields = nullptr;
    float2* fields_df = nullptr;  // mixed form: double-float copy of the fields
    BasisTab* d_tab = nullptr;    // device copy for the batch classification
    Sched sched;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr, done2 = nullptr;
    cudaEvent_t t[4] = {nullptr, nullptr, nullptr, nullptr};   // profiling: Newton, eval
    double newton_ms = 0.0, eval_ms = 0.0;
};

// per-point data of the batch classification: an instance's point range,
// element base, group and tie band
struct BRankInst {
    int64_t p0;
    int32_t ebase;
    int32_t grp;
    double band;
};

// per-group data of the batch classification (distance fields)
struct BRankGroup {
    int n;
    int32_t ebase;
    const double* dist;           // [E_g][n^3] or null
    const BasisTab* tab;
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
    release(g.coords); release(g.coords32); release(g.coords32lo); release(g.boxes); release(g.dist);
    release(g.fields); release(g.fields_df); release(g.d_tab);
    if (g.st) cudaStreamDestroy(g.st);
    if (g.done) cudaEventDestroy(g.done);
    if (g.done2) cudaEventDestroy(g.done2);
    for (auto& e : g.t)
        if (e) cudaEventDestroy(e);
    g.st = nullptr;
    g.done = g.done2 = nullptr;
    for (auto& e : g.t) e = nullptr;
}

// process-wide cache of tuned schedules: (mixed, N, log2 E, log2 pairs)
std::mutex g_tune_mu;
std::map<std::tuple<int, int, int, int>, Sched> g_tune_cache;

int ilog2(int64_t v)
{
    int k = 0;
    while (v > 1) {
        v >>= 1;
        ++k;
    }
    return k;
}

}  // namespace

namespace fpg {

// Lagrange basis at r for an order known only at run time (n <= NMAX)
__device__ __forceinline__ void lagrange_rt(int n, const double* xi, const double* ci, double r, double* h)
{
    double pre = 1.0;
    for (int i = 0; i < n; ++i) {
        h[i] = pre;
        pre *= r - xi[i];
    }
    double suf = 1.0;
    for (int i = n - 1; i >= 0; --i) {
        h[i] = ci[i] * (h[i] * suf);
        suf *= r - xi[i];
    }
}

// element data of a batch: batch-wide h_e and subdomain ids; D^k of the
// point's group, interpolated with the group's run-time order
struct RankBatch {
    const double* he_all;
    const int32_t* sub_all;
    const BRankGroup* grp;
    const RankArgs& A;
    int32_t ebase_inst;
    int g;
    __device__ __forceinline__ double he(int e) const { return he_all[e]; }
    __device__ __forceinline__ int sub(int e) const { return sub_all[e]; }
    __device__ __forceinline__ bool has_dist() const { return grp[g].dist != nullptr; }
    __device__ double delta(int e, int64_t q) const
    {
        const BRankGroup G = grp[g];
        const int n = G.n;
        double hr[NMAX], hs[NMAX], ht[NMAX];
        lagrange_rt(n, G.tab->xi, G.tab->ci, A.prst[q], hr);
        lagrange_rt(n, G.tab->xi, G.tab->ci, A.prst[A.cap + q], hs);
        lagrange_rt(n, G.tab->xi, G.tab->ci, A.prst[2 * A.cap + q], ht);
        const double* D = G.dist + (int64_t)(e - G.ebase) * n * n * n;
        double acc = 0.0;
        for (int k = 0; k < n; ++k) {
            double c = 0.0;
            for (int j = 0; j < n; ++j) {
                double u = 0.0;
                for (int i = 0; i < n; ++i) u = fma(hr[i], D[i + n * (j + n * k)], u);
                c = fma(hs[j], u, c);
            }
            acc = fma(ht[k], c, acc);
        }
        return acc;
    }
    __device__ __forceinline__ int elem_out(int e) const { return e - ebase_inst; }
};

__global__ void __launch_bounds__(128) k_rank_batch(RankArgs A, FindParams fp, int ninst, const BRankInst* inst,
                                                    const int64_t* p0, const double* he_all, const int32_t* sub_all,
                                                    const BRankGroup* grp)
{
    const int64_t p = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (p >= A.P) return;
    int lo = 0, hi = ninst;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(p0 + mid) <= p) lo = mid;
        else hi = mid;
    }
    const BRankInst I = inst[lo];
    FindParams f = fp;
    f.band = I.band;
    const RankBatch C{he_all, sub_all, grp, A, I.ebase, I.grp};
    rank_point<3>(A, f, C, p);
}

__global__ void k_fill_he(int64_t E, const ElemBox* __restrict__ boxes, double* __restrict__ he)
{
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e < E) he[e] = boxes[e].he;
}

}  // namespace fpg

struct fp_batch {
    int ninst = 0, F = 0;
    bool mixed = false;
    std::vector<fp_handle*> h;
    std::vector<int64_t> npts, uoff;
    int64_t Ptot = 0, Etot = 0, cap = 0;
    std::vector<Group> groups;
    int nsm = 1;
    // device
    BInst* d_inst = nullptr;
    int64_t* d_p0 = nullptr;
    BRankInst* d_rinst = nullptr;
    BRankGroup* d_rgrp = nullptr;
    double* he_all = nullptr;
    int32_t* sub_all = nullptr;
    int32_t *cnt = nullptr, *off = nullptr, *scan_tmp = nullptr;
    uint32_t* smask = nullptr;
    int32_t *pair_elem = nullptr, *pair_pt = nullptr, *order = nullptr, *ecount = nullptr, *estart = nullptr;
    int32_t* fb_list = nullptr;
    int32_t* gcount = nullptr;    // [2 * groups]: Newton work-queue counter, fallback counter
    double *pres = nullptr, *prst = nullptr;
    double2* pstate = nullptr;    // FP64 form: state of solves paused by the first Newton pass
    int32_t* inv = nullptr;       // sorted position of each pair slot
    unsigned long long* band = nullptr;
    cudaEvent_t fork = nullptr, fork2 = nullptr;
    bool prof = false;
    bool sequential = false;      // groups' Newton / eval launches one after another on the run's stream
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
    release(b->d_inst); release(b->d_p0); release(b->d_rinst); release(b->d_rgrp); release(b->he_all);
    release(b->sub_all); release(b->cnt); release(b->smask); release(b->off); release(b->scan_tmp); release(b->pair_elem);
    release(b->pair_pt); release(b->order); release(b->ecount); release(b->estart); release(b->fb_list);
    release(b->gcount); release(b->pres); release(b->prst); release(b->pstate); release(b->inv); release(b->band);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->fork2) cudaEventDestroy(b->fork2);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap_stream) cudaStreamDestroy(b->cap_stream);
    b->fork = b->fork2 = nullptr;
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
        if (!fp_live(h) || h->dim != 3 || npts[i] < 0 || h->device != dev) {
            delete b;
            return FP_ERR_INVALID_ARG;
        }
        const fp_opts& o0 = handles[0]->opts;
        if (h->opts.precision != o0.precision || h->opts.tol_accept != o0.tol_accept ||
            h->opts.tol_border != o0.tol_border || h->opts.max_newton != o0.max_newton ||
            h->opts.tie_band != o0.tie_band || h->refine != handles[0]->refine) {
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
    const fp_opts& o = handles[0]->opts;
    b->mixed = o.precision == FP_PREC_MIXED;
    // group instances by order N, groups in order of first appearance
    std::map<int, int> gid;
    for (int i = 0; i < ninst; ++i) {
        const int N = handles[i]->N;
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
    // batch element numbering: group-major, instances in batch order within a group
    std::vector<int32_t> inst_ebase(ninst, 0), inst_grp(ninst, 0);
    int64_t ecur = 0;
    for (size_t gi = 0; gi < b->groups.size(); ++gi) {
        Group& g = b->groups[gi];
        g.ebase = (int32_t)ecur;
        for (int i : g.inst) {
            inst_ebase[i] = (int32_t)ecur;
            inst_grp[i] = (int)gi;
            ecur += handles[i]->E;
            g.E += handles[i]->E;
            g.P += npts[i];
        }
        if (ecur >= (int64_t(1) << 31)) e = cudaErrorInvalidValue;
    }
    b->Etot = ecur;
    b->cap = std::max<int64_t>((int64_t)ceil(pairs_per_point * (double)b->Ptot), 1024);
    if (b->cap >= (int64_t(1) << 31)) e = cudaErrorInvalidValue;
    for (auto& g : b->groups) {
        if (e != cudaSuccess) break;
        const int n3 = g.n * g.n * g.n;
        bool multi = false;
        for (int i : g.inst) multi = multi || handles[i]->nsub > 1;
        g.fp.tol_accept = o.tol_accept;
        g.fp.tol_border = o.tol_border;
        g.fp.band = 0.0;                  // per instance, in the classification
        g.fp.max_newton = o.max_newton;
        g.fp.mixed = b->mixed;
        g.fp.refine = handles[0]->refine;
        e = alloc(&g.coords, 3 * g.E * n3);
        if (e == cudaSuccess && b->mixed) e = alloc(&g.coords32, 3 * g.E * n3);
        if (e == cudaSuccess && b->mixed) e = alloc(&g.coords32lo, 3 * g.E * n3);
        if (e == cudaSuccess) e = alloc(&g.boxes, g.E);
        if (e == cudaSuccess && multi) e = alloc(&g.dist, g.E * n3);
        if (e == cudaSuccess && F > 0) e = alloc(&g.fields, (int64_t)F * g.E * n3);
        if (e == cudaSuccess) e = alloc(&g.d_tab, 1);
        if (e == cudaSuccess) e = cudaMemcpy(g.d_tab, &g.tab, sizeof(BasisTab), cudaMemcpyHostToDevice);
        int64_t eo = 0;
        for (int i : g.inst) {
            if (e != cudaSuccess) break;
            fp_handle* h = handles[i];
            const int64_t Ei = h->E;
            for (int a = 0; a < 3 && e == cudaSuccess; ++a) {
                e = cudaMemcpy(g.coords + (a * g.E + eo) * n3, h->coords + a * Ei * n3, sizeof(double) * Ei * n3,
                               cudaMemcpyDeviceToDevice);
                if (e == cudaSuccess && b->mixed)
                    e = cudaMemcpy(g.coords32 + (a * g.E + eo) * n3, h->coords32 + a * Ei * n3,
                                   sizeof(float) * Ei * n3, cudaMemcpyDeviceToDevice);
                if (e == cudaSuccess && b->mixed)
                    e = cudaMemcpy(g.coords32lo + (a * g.E + eo) * n3, h->coords32lo + a * Ei * n3,
                                   sizeof(float) * Ei * n3, cudaMemcpyDeviceToDevice);
            }
            if (e == cudaSuccess)
                e = cudaMemcpy(g.boxes + eo, h->boxes, sizeof(ElemBox) * Ei, cudaMemcpyDeviceToDevice);
            if (e == cudaSuccess && g.dist) {
                if (h->nsub > 1 && h->dist)
                    e = cudaMemcpy(g.dist + eo * n3, h->dist, sizeof(double) * Ei * n3, cudaMemcpyDeviceToDevice);
                else
                    e = cudaMemset(g.dist + eo * n3, 0, sizeof(double) * Ei * n3);
            }
            for (int f = 0; f < F && e == cudaSuccess; ++f) {
                const double* src = fields[i];
                if (!src) {
                    e = cudaErrorInvalidValue;
                    break;
                }
                e = cudaMemcpy(g.fields + ((int64_t)f * g.E + eo) * n3, src + (int64_t)f * Ei * n3,
                               sizeof(double) * Ei * n3, cudaMemcpyDeviceToDevice);
            }
            eo += Ei;
        }
        if (e == cudaSuccess && F > 0 && b->mixed) {
            const int64_t nv = (int64_t)F * g.E * n3;
            e = alloc(&g.fields_df, nv);
            if (e == cudaSuccess) e = launch_split_df(nv, g.n, g.fields, g.fields_df, 0);
        }
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g.st, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g.done2, cudaEventDisableTiming);
        for (auto& ev : g.t)
            if (e == cudaSuccess) e = cudaEventCreate(&ev);
    }
    // batch-wide tables and scratch
    if (e == cudaSuccess) {
        std::vector<BInst> bi(ninst);
        std::vector<BRankInst> ri(ninst);
        for (int i = 0; i < ninst; ++i) {
            fp_handle* h = handles[i];
            memset(&bi[i], 0, sizeof(BInst));
            bi[i].g = h->grid;
            bi[i].cell_start = h->cell_start;
            bi[i].cell_elems = h->cell_elems;
            bi[i].sub = h->sub;
            bi[i].boxes = h->boxes;
            bi[i].boxes32 = h->boxes32;
            bi[i].p0 = b->uoff[i];
            bi[i].ebase = inst_ebase[i];
            ri[i] = BRankInst{b->uoff[i], inst_ebase[i], inst_grp[i], o.tie_band * h->L};
        }
        std::vector<BRankGroup> rg;
        for (auto& g : b->groups) rg.push_back(BRankGroup{g.n, g.ebase, g.dist, g.d_tab});
        e = alloc(&b->d_inst, ninst);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_inst, bi.data(), sizeof(BInst) * ninst, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = alloc(&b->d_p0, ninst + 1);
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_p0, b->uoff.data(), sizeof(int64_t) * (ninst + 1), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = alloc(&b->d_rinst, ninst);
        if (e == cudaSuccess) e = cudaMemcpy(b->d_rinst, ri.data(), sizeof(BRankInst) * ninst, cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = alloc(&b->d_rgrp, (int64_t)rg.size());
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_rgrp, rg.data(), sizeof(BRankGroup) * rg.size(), cudaMemcpyHostToDevice);
        if (e == cudaSuccess) e = alloc(&b->he_all, b->Etot);
        if (e == cudaSuccess) e = alloc(&b->sub_all, b->Etot);
        for (int i = 0; i < ninst && e == cudaSuccess; ++i) {
            fp_handle* h = handles[i];
            k_fill_he<<<(unsigned)((h->E + 255) / 256), 256>>>(h->E, h->boxes, b->he_all + inst_ebase[i]);
            count_launch();
            e = cudaGetLastError();
            if (e == cudaSuccess)
                e = cudaMemcpy(b->sub_all + inst_ebase[i], h->sub, sizeof(int32_t) * h->E, cudaMemcpyDeviceToDevice);
        }
        const int64_t P = b->Ptot, ng = (int64_t)b->groups.size();
        if (e == cudaSuccess) e = alloc(&b->cnt, P);
        if (e == cudaSuccess) e = alloc(&b->smask, P);
        if (e == cudaSuccess) e = alloc(&b->off, P + 1);
        if (e == cudaSuccess) e = alloc(&b->scan_tmp, std::max(scan_tmp_elems(P), scan_tmp_elems(b->Etot)));
        if (e == cudaSuccess) e = alloc(&b->pair_elem, b->cap);
        if (e == cudaSuccess) e = alloc(&b->pair_pt, b->cap);
        if (e == cudaSuccess) e = alloc(&b->order, b->cap);
        if (e == cudaSuccess) e = alloc(&b->fb_list, b->cap);
        if (e == cudaSuccess) e = alloc(&b->ecount, b->Etot);
        if (e == cudaSuccess) e = alloc(&b->estart, b->Etot + 1);
        if (e == cudaSuccess) e = alloc(&b->gcount, 2 * ng);
        if (e == cudaSuccess) e = alloc(&b->pres, b->cap);
        if (e == cudaSuccess) e = alloc(&b->prst, 3 * b->cap);
        if (e == cudaSuccess && !b->mixed) e = alloc(&b->pstate, b->cap);
        if (e == cudaSuccess) e = alloc(&b->inv, b->cap);
        if (e == cudaSuccess) e = alloc(&b->band, 3);
        if (e == cudaSuccess) e = cudaMemset(b->band, 0, 3 * sizeof(unsigned long long));
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->fork2, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->cap_stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaDeviceSynchronize();
    }
    if (e != cudaSuccess) {
        batch_release(b);
        delete b;
        return e == cudaErrorMemoryAllocation ? FP_ERR_OOM : (e == cudaErrorInvalidValue ? FP_ERR_INVALID_ARG : FP_ERR_CUDA);
    }
    // default schedules, from the tuning cache where a group's bucket was tuned before
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        for (auto& g : b->groups) {
            const int64_t pairs_est = (int64_t)(1.05 * (double)g.P) + 1;
            auto it = g_tune_cache.find({b->mixed ? 1 : 0, g.N, ilog2(g.E), ilog2(pairs_est)});
            if (it != g_tune_cache.end()) g.sched = it->second;
        }
    }
    *out = b;
    return FP_OK;
}

// the arrays of group g for its Newton stage / evaluation
static FindArgs group_args(const fp_batch* b, const Group& g, const double* pts)
{
    FindArgs a;
    memset(&a, 0, sizeof(a));
    a.batch = 1;
    a.n = g.n;
    a.E = g.E;
    a.P = b->Ptot;
    a.pts = pts;
    a.coords = g.coords;
    a.coords32 = g.coords32;
    a.coords32lo = g.coords32lo;
    a.boxes = g.boxes;
    a.off = b->off;
    a.pair_elem = b->pair_elem;
    a.pair_pt = b->pair_pt;
    a.order = b->order;
    a.pres = b->pres;
    a.prst = b->prst;
    a.cap = b->cap;
    a.s_lo = b->estart + g.ebase;
    a.s_hi = b->estart + g.ebase + g.E;
    a.ebase = g.ebase;
    const int64_t gi = &g - b->groups.data();
    a.queue = b->gcount + 2 * gi;
    a.fb_count = b->gcount + 2 * gi + 1;
    a.fb_list = b->fb_list;
    a.pstate = b->pstate;
    a.inv = b->inv;
    a.tile = g.sched.tile;
    a.persistent_blocks = g.sched.bps * b->nsm;
    return a;
}

static cudaError_t group_newton(const fp_batch* b, const Group& g, const double* pts, cudaStream_t s)
{
    const FindArgs a = group_args(b, g, pts);
    return find_newton_group(a, g.tab, g.fp, g.sched.block, (unsigned)(g.sched.bps * b->nsm), s);
}

// one run of the whole batch on stream s (no host waits)
static cudaError_t batch_run(fp_batch* b, const double* pts, int32_t* code, int32_t* sub, int32_t* elem, double* rst,
                             double* dist2, double* out, cudaStream_t s)
{
    const int64_t P = b->Ptot;
    if (P == 0) return cudaSuccess;
    BScreenArgs sa;
    sa.ninst = b->ninst;
    sa.inst = b->d_inst;
    sa.p0 = b->d_p0;
    sa.P = P;
    sa.pts = pts;
    sa.cnt = b->cnt;
    sa.mask = b->smask;
    sa.off = b->off;
    sa.pair_elem = b->pair_elem;
    sa.pair_pt = b->pair_pt;
    sa.cap = b->cap;
    cudaError_t e = launch_bscreen(sa, false, b->mixed, s);
    if (e == cudaSuccess) e = scan_exclusive(b->cnt, b->off, P, b->scan_tmp, s);
    if (e == cudaSuccess) e = launch_bscreen(sa, true, b->mixed, s);
    if (e != cudaSuccess) return e;
    {   // all pairs sorted by batch element: each group's pairs become one range
        FindArgs a;
        memset(&a, 0, sizeof(a));
        a.E = b->Etot;
        a.P = P;
        a.off = b->off;
        a.pair_elem = b->pair_elem;
        a.order = b->order;
        a.inv = b->inv;
        a.ecount = b->ecount;
        a.estart = b->estart;
        a.scan_tmp = b->scan_tmp;
        a.cap = b->cap;
        a.persistent_blocks = b->nsm;
        if ((e = find_sort(a, b->cap, s)) != cudaSuccess) return e;
    }
    // Newton: the groups' launches run concurrently on their own streams
    // (profiled runs: one after another on s, so each group's time is its own)
    if ((e = cudaEventRecord(b->fork, s)) != cudaSuccess) return e;
    for (auto& g : b->groups) {
        if (g.P == 0) continue;
        const bool serial = b->prof || b->sequential;
        cudaStream_t gs = serial ? s : g.st;
        if (!serial && (e = cudaStreamWaitEvent(gs, b->fork, 0)) != cudaSuccess) return e;
        if (b->prof) cudaEventRecord(g.t[0], gs);
        if ((e = group_newton(b, g, pts, gs)) != cudaSuccess) return e;
        if (b->prof) cudaEventRecord(g.t[1], gs);
        if (!serial) {
            if ((e = cudaEventRecord(g.done, gs)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, g.done, 0)) != cudaSuccess) return e;
        }
    }
    // classification of every point, results in the caller's order
    {
        RankArgs ra;
        memset(&ra, 0, sizeof(ra));
        ra.P = P;
        ra.E = b->Etot;
        ra.off = b->off;
        ra.pair_elem = b->pair_elem;
        ra.pres = b->pres;
        ra.prst = b->prst;
        ra.cap = b->cap;
        ra.code = code;
        ra.osub = sub;
        ra.oelem = elem;
        ra.rst = rst;
        ra.dist2 = dist2;
        ra.pair_pt = b->pair_pt;
        ra.F = out ? b->F : 0;
        ra.out = out;
        ra.band = b->band;
        ra.inv = b->inv;
        FindParams fp = b->groups[0].fp;
        k_rank_batch<<<(unsigned)((P + 127) / 128), 128, 0, s>>>(ra, fp, b->ninst, b->d_rinst, b->d_p0, b->he_all,
                                                                b->sub_all, b->d_rgrp);
        count_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (b->F == 0 || !out) return cudaSuccess;
    // fused evaluation of the winning pairs, per group
    if ((e = cudaEventRecord(b->fork2, s)) != cudaSuccess) return e;
    for (auto& g : b->groups) {
        if (g.P == 0) continue;
        const bool serial = b->prof || b->sequential;
        cudaStream_t gs = serial ? s : g.st;
        if (!serial && (e = cudaStreamWaitEvent(gs, b->fork2, 0)) != cudaSuccess) return e;
        if (b->prof) cudaEventRecord(g.t[2], gs);
        const EvalSpec ev{b->F, g.fields_df ? nullptr : g.fields, g.fields_df, out};
        e = launch_eval_pairs(g.n, g.E, P, nullptr, b->cap, b->order, b->pair_elem, b->pair_pt, b->prst, ev, g.tab,
                              (unsigned)(4 * b->nsm), gs, b->estart + g.ebase, b->estart + g.ebase + g.E, g.ebase,
                              true);
        if (e != cudaSuccess) return e;
        if (b->prof) cudaEventRecord(g.t[3], gs);
        if (!serial) {
            if ((e = cudaEventRecord(g.done2, gs)) != cudaSuccess) return e;
            if ((e = cudaStreamWaitEvent(s, g.done2, 0)) != cudaSuccess) return e;
        }
    }
    return cudaSuccess;
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

// per-group Newton times of a profiled run (waits for its events)
static void read_group_times(fp_batch* b)
{
    for (auto& g : b->groups) {
        if (g.P == 0) continue;
        float ms = 0.0f;
        if (cudaEventSynchronize(g.t[1]) == cudaSuccess && cudaEventElapsedTime(&ms, g.t[0], g.t[1]) == cudaSuccess)
            g.newton_ms = ms;
        if (b->F > 0 && cudaEventSynchronize(g.t[3]) == cudaSuccess &&
            cudaEventElapsedTime(&ms, g.t[2], g.t[3]) == cudaSuccess)
            g.eval_ms = ms;
    }
}

extern "C" fp_status fp_batch_run(fp_batch* b, const double* pts, int32_t* code, int32_t* sub, int32_t* elem,
                                  double* rst, double* dist2, double* out, void* stream)
{
    fp_status st = check_run_args(b, pts, code, sub, elem, rst, dist2);
    if (st != FP_OK) return st;
    cudaError_t e = batch_run(b, pts, code, sub, elem, rst, dist2, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return bfail(b, FP_ERR_CUDA, std::string("fp_batch_run: ") + cudaGetErrorString(e));
    if (b->prof) read_group_times(b);
    return FP_OK;
}

extern "C" fp_status fp_batch_tune(fp_batch* b, const double* pts, int32_t* code, int32_t* sub, int32_t* elem,
                                   double* rst, double* dist2, double* out, void* stream, int reps, double* best_ms)
{
    fp_status st = check_run_args(b, pts, code, sub, elem, rst, dist2);
    if (st != FP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    if (reps < 1) reps = 1;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const bool prof = b->prof;
    b->prof = false;
    // one full run: the sorted pairs the Newton stage is timed on
    if (e == cudaSuccess) e = batch_run(b, pts, code, sub, elem, rst, dist2, out, s);
    std::vector<int32_t> es(2);
    auto time_group = [&](Group& g, const Sched& c, float* ms) -> cudaError_t {
        const Sched keep = g.sched;
        g.sched = c;
        cudaError_t r = group_newton(b, g, pts, s);                           // warm-up
        if (r == cudaSuccess) r = cudaEventRecord(e0, s);
        for (int k = 0; k < reps && r == cudaSuccess; ++k) r = group_newton(b, g, pts, s);
        if (r == cudaSuccess) r = cudaEventRecord(e1, s);
        if (r == cudaSuccess) r = cudaEventSynchronize(e1);
        if (r == cudaSuccess) r = cudaEventElapsedTime(ms, e0, e1);
        *ms /= reps;
        g.sched = keep;
        return r;
    };
    for (auto& g : b->groups) {
        if (e != cudaSuccess) break;
        if (g.P == 0) continue;
        e = cudaMemcpyAsync(es.data(), b->estart + g.ebase, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(es.data() + 1, b->estart + g.ebase + g.E, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) break;
        const int64_t pairs = std::max<int64_t>(es[1] - es[0], 1);
        const auto key = std::make_tuple(b->mixed ? 1 : 0, g.N, ilog2(g.E), ilog2(pairs));
        {
            std::lock_guard<std::mutex> lk(g_tune_mu);
            auto it = g_tune_cache.find(key);
            if (it != g_tune_cache.end()) {
                g.sched = it->second;
                continue;
            }
        }
        // threads per block x blocks per SM (blocks beyond what fits an SM only queue), then the work-item size
        Sched best = g.sched;
        float best_t = INFINITY;
        for (int blk : {64, 128, 256}) {
            const int fit = std::max(1, newton_blocks_per_sm(g.n, b->mixed, blk));
            for (int bps : {1, 2, 4, 8}) {
                if (bps > 2 * fit || e != cudaSuccess) continue;
                Sched c{blk, bps, 128};
                float ms = 0.0f;
                e = time_group(g, c, &ms);
                if (e == cudaSuccess && ms < best_t) {
                    best_t = ms;
                    best = c;
                }
            }
        }
        for (int t : {32, 512}) {
            if (e != cudaSuccess) break;
            Sched c = best;
            c.tile = t;
            float ms = 0.0f;
            e = time_group(g, c, &ms);
            if (e == cudaSuccess && ms < best_t) {
                best_t = ms;
                best = c;
            }
        }
        if (e != cudaSuccess) break;
        g.sched = best;
        g.newton_ms = best_t;
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_cache[key] = best;
    }
    // the whole run with the chosen schedules, the groups concurrently on
    // their streams or one after another (the persistent launches of one
    // group can hold every SM, leaving nothing for the others to overlap):
    // the faster of the two is kept
    float total = INFINITY;
    bool best_seq = false;
    for (int mode = 0; mode < 2 && e == cudaSuccess; ++mode) {
        b->sequential = mode == 1;
        float t = 0.0f;
        e = batch_run(b, pts, code, sub, elem, rst, dist2, out, s);
        if (e == cudaSuccess) e = cudaEventRecord(e0, s);
        for (int k = 0; k < reps && e == cudaSuccess; ++k) e = batch_run(b, pts, code, sub, elem, rst, dist2, out, s);
        if (e == cudaSuccess) e = cudaEventRecord(e1, s);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && t < total) {
            total = t;
            best_seq = b->sequential;
        }
    }
    b->sequential = best_seq;
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    b->prof = prof;
    if (e != cudaSuccess) return bfail(b, FP_ERR_CUDA, std::string("fp_batch_tune: ") + cudaGetErrorString(e));
    if (best_ms) *best_ms = total / reps;
    return FP_OK;
}

extern "C" fp_status fp_batch_schedule(fp_batch* b, int group, int* block, int* blocks_per_sm, int* tile)
{
    if (!b) return FP_ERR_INVALID_ARG;
    if (group < 0 || group >= (int)b->groups.size()) return bfail(b, FP_ERR_INVALID_ARG, "fp_batch_schedule: group");
    Sched& c = b->groups[group].sched;
    Sched n = c;
    if (block && *block > 0) {
        if (*block % 32 != 0 || *block > 256) return bfail(b, FP_ERR_INVALID_ARG, "fp_batch_schedule: block");
        n.block = *block;
    }
    if (blocks_per_sm && *blocks_per_sm > 0) n.bps = std::min(*blocks_per_sm, 64);
    if (tile && *tile > 0) {
        if (*tile % 32 != 0) return bfail(b, FP_ERR_INVALID_ARG, "fp_batch_schedule: tile");
        n.tile = *tile;
    }
    c = n;
    if (block) *block = c.block;
    if (blocks_per_sm) *blocks_per_sm = c.bps;
    if (tile) *tile = c.tile;
    return FP_OK;
}

extern "C" fp_status fp_batch_mode(fp_batch* b, int* sequential)
{
    if (!b || !sequential) return FP_ERR_INVALID_ARG;
    if (*sequential == 0 || *sequential == 1) b->sequential = *sequential == 1;
    else if (*sequential != -1) return bfail(b, FP_ERR_INVALID_ARG, "fp_batch_mode: -1, 0 or 1");
    *sequential = b->sequential ? 1 : 0;
    return FP_OK;
}

extern "C" fp_status fp_batch_groups(const fp_batch* b, int* ngroups)
{
    if (!b || !ngroups) return FP_ERR_INVALID_ARG;
    *ngroups = (int)b->groups.size();
    return FP_OK;
}

extern "C" fp_status fp_batch_group_info(fp_batch* b, int group, int* N, int64_t* E, int64_t* P, int64_t* pairs,
                                         double* newton_ms, double* eval_ms)
{
    if (!b) return FP_ERR_INVALID_ARG;
    if (group < 0 || group >= (int)b->groups.size()) return bfail(b, FP_ERR_INVALID_ARG, "fp_batch_group_info: group");
    const Group& g = b->groups[group];
    if (N) *N = g.N;
    if (E) *E = g.E;
    if (P) *P = g.P;
    if (pairs) {
        int32_t es[2] = {0, 0};
        cudaError_t e = cudaDeviceSynchronize();
        if (e == cudaSuccess) e = cudaMemcpy(es, b->estart + g.ebase, sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e == cudaSuccess) e = cudaMemcpy(es + 1, b->estart + g.ebase + g.E, sizeof(int32_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return bfail(b, FP_ERR_CUDA, std::string("fp_batch_group_info: ") + cudaGetErrorString(e));
        *pairs = es[1] - es[0];
    }
    if (newton_ms) *newton_ms = g.newton_ms;
    if (eval_ms) *eval_ms = g.eval_ms;
    return FP_OK;
}

extern "C" fp_status fp_batch_profile(fp_batch* b, int enable)
{
    if (!b) return FP_ERR_INVALID_ARG;
    b->prof = enable != 0;
    return FP_OK;
}

extern "C" fp_status fp_batch_band_hits(fp_batch* b, int64_t* counts)
{
    if (!b || !counts) return FP_ERR_INVALID_ARG;
    unsigned long long c[3] = {0, 0, 0};
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(c, b->band, sizeof(c), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(b->band, 0, sizeof(c));
    if (e != cudaSuccess) return bfail(b, FP_ERR_CUDA, std::string("fp_batch_band_hits: ") + cudaGetErrorString(e));
    for (int k = 0; k < 3; ++k) counts[k] = (int64_t)c[k];
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
    const bool prof = b->prof;
    b->prof = false;                                   // no timing events inside the graph
    cudaError_t e = cudaStreamBeginCapture(b->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        b->prof = prof;
        return bfail(b, FP_ERR_CUDA, std::string("fp_batch_capture: ") + cudaGetErrorString(e));
    }
    const int64_t k0 = fp_launch_count();
    cudaError_t er = batch_run(b, pts, code, sub, elem, rst, dist2, out, b->cap_stream);
    b->graph_kernels = fp_launch_count() - k0;
    e = cudaStreamEndCapture(b->cap_stream, &b->graph);
    b->prof = prof;
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
