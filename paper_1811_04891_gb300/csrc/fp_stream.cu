// fp_stream.cu -- fp_find_eval_host: find (+ eval) over points and results in
// host memory, streamed through the device in chunks.
//
// A caller whose query points arrive in host memory (a solver that assembles
// interface points on the CPU, a service receiving requests over the network)
// pays for two copies per call besides the search.  This entry point hides
// them: the points are cut into chunks; while the compute stream searches
// chunk i, a copy stream brings chunk i+1 in and another takes the results
// of chunk i-1 out.  Two sets of device buffers and two workspaces alternate
// between chunks, so the copies of one chunk never touch the buffers the
// search of the other is using; events order the three streams.  Each chunk
// runs the workspace find (+ fused eval): the pair count stays on the device
// and no call waits on the host.  The launches give one block to 128 pairs,
// which balances the Newton work like a launch sized on the host, over the
// pairs the chunk is expected to have: the largest pairs per point of the
// previous call's chunks, plus 1/8 and 4096 (the first call covers the whole
// capacity).  The pair kernels loop grid-stride over the count on the device,
// so a chunk with more pairs than expected is still solved completely.  The pair count of every chunk comes back with its results; a chunk
// whose pairs overflowed its workspace has its RETRY points searched again
// with fp_find_eval before the call returns.
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "fp_common.cuh"
#include "fp_handle.h"
#include "fp_internal.h"

namespace {

struct Slot {
    fp_workspace* ws = nullptr;
    double* pts = nullptr;      // [3][chunk]
    int32_t* qs = nullptr;      // [chunk]
    int32_t* code = nullptr;
    int32_t* sub = nullptr;
    int32_t* elem = nullptr;
    double* rst = nullptr;      // [3][chunk]
    double* dist2 = nullptr;
    double* out = nullptr;      // [F][chunk]
    cudaEvent_t in_done = nullptr, comp_done = nullptr, out_done = nullptr;
};

template <typename T>
cudaError_t dmalloc(T** p, int64_t n)
{
    *p = nullptr;
    return cudaMalloc((void**)p, sizeof(T) * (size_t)std::max<int64_t>(n, 1));
}

}  // namespace

struct fp_host_stream {
    int64_t chunk = 0, max_pairs = 0;
    int F = 0;
    Slot slot[2];
    cudaStream_t cin = nullptr, cout = nullptr;
    int32_t* h_pairs = nullptr;   // pinned: device pair count of each chunk
    int64_t h_pairs_cap = 0;
    double pairs_per_point = 0;   // largest of the previous call's chunks (0: none yet)
};

namespace fpg {

void host_stream_free(fp_host_stream* hs)
{
    if (!hs) return;
    if (hs->cin) cudaStreamSynchronize(hs->cin);
    if (hs->cout) cudaStreamSynchronize(hs->cout);
    for (Slot& S : hs->slot) {
        if (S.ws) fp_workspace_free(S.ws);
        cudaFree(S.pts); cudaFree(S.qs); cudaFree(S.code); cudaFree(S.sub); cudaFree(S.elem);
        cudaFree(S.rst); cudaFree(S.dist2); cudaFree(S.out);
        if (S.in_done) cudaEventDestroy(S.in_done);
        if (S.comp_done) cudaEventDestroy(S.comp_done);
        if (S.out_done) cudaEventDestroy(S.out_done);
    }
    if (hs->cin) cudaStreamDestroy(hs->cin);
    if (hs->cout) cudaStreamDestroy(hs->cout);
    if (hs->h_pairs) cudaFreeHost(hs->h_pairs);
    delete hs;
}

}  // namespace fpg

static fp_status stream_state(fp_handle* h, int64_t chunk, int64_t max_pairs, int F, int64_t nchunks,
                              fp_host_stream** out)
{
    fp_host_stream* hs = h->host_stream;
    if (hs && (hs->chunk < chunk || hs->max_pairs < max_pairs || hs->F < F)) {
        fpg::host_stream_free(hs);
        h->host_stream = hs = nullptr;
    }
    if (!hs) {
        cudaError_t e = cudaSuccess;
        hs = new fp_host_stream();
        hs->chunk = chunk;
        hs->max_pairs = max_pairs;
        hs->F = F;
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hs->cin, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hs->cout, cudaStreamNonBlocking);
        for (Slot& S : hs->slot) {
            if (e == cudaSuccess && fp_workspace_create(h, chunk, max_pairs, &S.ws) != FP_OK)
                e = cudaErrorMemoryAllocation;
            if (e == cudaSuccess) fpg::workspace_unpersist(S.ws);
            if (e == cudaSuccess) e = dmalloc(&S.pts, 3 * chunk);
            if (e == cudaSuccess) e = dmalloc(&S.qs, chunk);
            if (e == cudaSuccess) e = dmalloc(&S.code, chunk);
            if (e == cudaSuccess) e = dmalloc(&S.sub, chunk);
            if (e == cudaSuccess) e = dmalloc(&S.elem, chunk);
            if (e == cudaSuccess) e = dmalloc(&S.rst, 3 * chunk);
            if (e == cudaSuccess) e = dmalloc(&S.dist2, chunk);
            if (e == cudaSuccess) e = dmalloc(&S.out, (int64_t)std::max(F, 1) * chunk);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S.in_done, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S.comp_done, cudaEventDisableTiming);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&S.out_done, cudaEventDisableTiming);
        }
        if (e != cudaSuccess) {
            fpg::host_stream_free(hs);
            h->err = std::string("fp_find_eval_host: device buffers: ") + cudaGetErrorString(e);
            return e == cudaErrorMemoryAllocation ? FP_ERR_OOM : FP_ERR_CUDA;
        }
        h->host_stream = hs;
    }
    if (hs->h_pairs_cap < nchunks) {
        if (hs->h_pairs) cudaFreeHost(hs->h_pairs);
        hs->h_pairs = nullptr;
        hs->h_pairs_cap = 0;
        if (cudaMallocHost((void**)&hs->h_pairs, sizeof(int32_t) * (size_t)nchunks) != cudaSuccess) {
            h->err = "fp_find_eval_host: pinned pair counts";
            return FP_ERR_OOM;
        }
        hs->h_pairs_cap = nchunks;
    }
    *out = hs;
    return FP_OK;
}

// search again, with the growing (synchronous) path, the RETRY points of one chunk
static fp_status redo_retry(fp_handle* h, int64_t P, int64_t i0, int64_t c, const double* pts, const int32_t* qsess,
                            bool eval, int F, const double* fields, const fp_fields* posted, int32_t* code,
                            int32_t* sub, int32_t* elem, double* rst, double* dist2, double* out, cudaStream_t s)
{
    std::vector<int64_t> idx;
    for (int64_t k = 0; k < c; ++k)
        if (code[i0 + k] == FP_CODE_RETRY) idx.push_back(i0 + k);
    const int64_t m = (int64_t)idx.size();
    if (m == 0) return FP_OK;
    std::vector<double> hp(3 * m), hr(3 * m), hd(m), ho((size_t)std::max(F, 1) * m);
    std::vector<int32_t> hq(m), hc(m), hsb(m), he(m);
    for (int64_t k = 0; k < m; ++k) {
        for (int a = 0; a < 3; ++a) hp[a * m + k] = pts[a * P + idx[k]];
        hq[k] = qsess ? qsess[idx[k]] : -1;
    }
    double *dp = nullptr, *dr = nullptr, *dd = nullptr, *dout = nullptr;
    int32_t *dq = nullptr, *dc = nullptr, *dsu = nullptr, *de = nullptr;
    cudaError_t e = dmalloc(&dp, 3 * m);
    if (e == cudaSuccess) e = dmalloc(&dr, 3 * m);
    if (e == cudaSuccess) e = dmalloc(&dd, m);
    if (e == cudaSuccess) e = dmalloc(&dout, (int64_t)std::max(F, 1) * m);
    if (e == cudaSuccess) e = dmalloc(&dq, m);
    if (e == cudaSuccess) e = dmalloc(&dc, m);
    if (e == cudaSuccess) e = dmalloc(&dsu, m);
    if (e == cudaSuccess) e = dmalloc(&de, m);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dp, hp.data(), sizeof(double) * 3 * m, cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dq, hq.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, s);
    fp_status st = FP_ERR_CUDA;
    if (e == cudaSuccess) {
        st = eval ? fp_find_eval(h, m, dp, dq, F, fields, posted, dc, dsu, de, dr, dd, dout, s)
                  : fp_find(h, m, dp, dq, dc, dsu, de, dr, dd, s);
        if (st == FP_OK) {
            e = cudaMemcpyAsync(hc.data(), dc, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hsb.data(), dsu, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(he.data(), de, sizeof(int32_t) * m, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hr.data(), dr, sizeof(double) * 3 * m, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaMemcpyAsync(hd.data(), dd, sizeof(double) * m, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess && eval)
                e = cudaMemcpyAsync(ho.data(), dout, sizeof(double) * F * m, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) st = FP_ERR_CUDA;
        }
    }
    cudaFree(dp); cudaFree(dr); cudaFree(dd); cudaFree(dout); cudaFree(dq); cudaFree(dc); cudaFree(dsu); cudaFree(de);
    if (st != FP_OK) {
        if (h->err.empty()) h->err = "fp_find_eval_host: searching the RETRY points again failed";
        return st;
    }
    for (int64_t k = 0; k < m; ++k) {
        const int64_t p = idx[k];
        code[p] = hc[k];
        sub[p] = hsb[k];
        elem[p] = he[k];
        dist2[p] = hd[k];
        for (int a = 0; a < 3; ++a) rst[a * P + p] = hr[a * m + k];
        if (eval)
            for (int f = 0; f < F; ++f) out[(int64_t)f * P + p] = ho[(size_t)f * m + k];
    }
    return FP_OK;
}

extern "C" fp_status fp_find_eval_host(fp_handle* h, int64_t P, const double* pts, const int32_t* qsess, int F,
                                       const double* fields, const fp_fields* posted, int32_t* code, int32_t* sub,
                                       int32_t* elem, double* rst, double* dist2, double* out, int64_t chunk,
                                       int64_t max_pairs, void* stream)
{
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    h->err.clear();
    if (h->dim != 3) {
        h->err = "fp_find_eval_host: hexahedral meshes only";
        return FP_ERR_INVALID_ARG;
    }
    if (P < 0 || P >= (int64_t(1) << 31)) {
        h->err = "fp_find_eval_host: P out of range";
        return FP_ERR_INVALID_ARG;
    }
    if (P == 0) return FP_OK;
    const bool eval = F != 0 || posted != nullptr;
    if (!pts || !code || !sub || !elem || !rst || !dist2 || (eval && (!out || F < 1))) {
        h->err = "fp_find_eval_host: null pointer or F < 1 with fields";
        return FP_ERR_INVALID_ARG;
    }
    if (chunk <= 0) chunk = int64_t(1) << 22;
    chunk = std::min(chunk, P);
    if (max_pairs <= 0) max_pairs = 4 * chunk;
    if (max_pairs >= (int64_t(1) << 31)) {
        h->err = "fp_find_eval_host: max_pairs out of range";
        return FP_ERR_INVALID_ARG;
    }
    const int64_t nch = (P + chunk - 1) / chunk;
    fp_host_stream* hs = nullptr;
    fp_status st = stream_state(h, chunk, max_pairs, eval ? F : 0, nch, &hs);
    if (st != FP_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaSuccess;
    // the copy-in stream starts after the work already queued on the caller's stream
    e = cudaEventRecord(hs->slot[1].comp_done, s);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(hs->cin, hs->slot[1].comp_done, 0);
    for (int64_t i = 0; i < nch && e == cudaSuccess; ++i) {
        Slot& S = hs->slot[i & 1];
        const int64_t i0 = i * chunk, c = std::min(chunk, P - i0);
        if (i >= 2) e = cudaStreamWaitEvent(hs->cin, S.out_done, 0);   // this slot's results are out
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(S.pts, sizeof(double) * c, pts + i0, sizeof(double) * P, sizeof(double) * c, 3,
                                  cudaMemcpyHostToDevice, hs->cin);
        if (e == cudaSuccess && qsess)
            e = cudaMemcpyAsync(S.qs, qsess + i0, sizeof(int32_t) * c, cudaMemcpyHostToDevice, hs->cin);
        if (e == cudaSuccess) e = cudaEventRecord(S.in_done, hs->cin);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(s, S.in_done, 0);
        if (e != cudaSuccess) break;
        fpg::workspace_grid_hint(S.ws, hs->pairs_per_point > 0
                                           ? (int64_t)(1.125 * hs->pairs_per_point * (double)c) + 4096 : 0);
        st = eval ? fp_find_eval_ws(h, S.ws, c, S.pts, qsess ? S.qs : nullptr, F, fields, posted, S.code, S.sub,
                                    S.elem, S.rst, S.dist2, S.out, s)
                  : fp_find_ws(h, S.ws, c, S.pts, qsess ? S.qs : nullptr, S.code, S.sub, S.elem, S.rst, S.dist2, s);
        if (st != FP_OK) {
            cudaStreamSynchronize(hs->cout);
            cudaStreamSynchronize(hs->cin);
            return st;
        }
        e = fpg::workspace_pair_count_async(S.ws, hs->h_pairs + i, s);
        if (e == cudaSuccess) e = cudaEventRecord(S.comp_done, s);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(hs->cout, S.comp_done, 0);
        if (e == cudaSuccess) e = cudaMemcpyAsync(code + i0, S.code, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, hs->cout);
        if (e == cudaSuccess) e = cudaMemcpyAsync(sub + i0, S.sub, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, hs->cout);
        if (e == cudaSuccess) e = cudaMemcpyAsync(elem + i0, S.elem, sizeof(int32_t) * c, cudaMemcpyDeviceToHost, hs->cout);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(dist2 + i0, S.dist2, sizeof(double) * c, cudaMemcpyDeviceToHost, hs->cout);
        if (e == cudaSuccess)
            e = cudaMemcpy2DAsync(rst + i0, sizeof(double) * P, S.rst, sizeof(double) * c, sizeof(double) * c, 3,
                                  cudaMemcpyDeviceToHost, hs->cout);
        if (e == cudaSuccess && eval)
            e = cudaMemcpy2DAsync(out + i0, sizeof(double) * P, S.out, sizeof(double) * c, sizeof(double) * c, F,
                                  cudaMemcpyDeviceToHost, hs->cout);
        if (e == cudaSuccess) e = cudaEventRecord(S.out_done, hs->cout);
    }
    cudaError_t e2 = cudaStreamSynchronize(hs->cout);
    if (e == cudaSuccess) e = e2;
    e2 = cudaStreamSynchronize(s);
    if (e == cudaSuccess) e = e2;
    if (e != cudaSuccess) {
        h->err = std::string("fp_find_eval_host: ") + cudaGetErrorString(e);
        return FP_ERR_CUDA;
    }
    double ppp = 0;
    for (int64_t i = 0; i < nch; ++i) {
        const int64_t c = std::min(chunk, P - i * chunk);
        ppp = std::max(ppp, (double)hs->h_pairs[i] / (double)c);
    }
    hs->pairs_per_point = ppp;
    for (int64_t i = 0; i < nch; ++i) {
        if (hs->h_pairs[i] <= max_pairs) continue;               // every pair of the chunk fitted
        const int64_t i0 = i * chunk, c = std::min(chunk, P - i0);
        st = redo_retry(h, P, i0, c, pts, qsess, eval, F, fields, posted, code, sub, elem, rst, dist2, out, s);
        if (st != FP_OK) return st;
    }
    return FP_OK;
}
