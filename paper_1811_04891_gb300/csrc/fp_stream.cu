// fp_stream.cu -- fp_find_eval_host: find (+ eval) over points and results in
// host memory, streamed through the device in chunks.
//
// A caller whose query points arrive in host memory (a solver that assembles
// interface points on the CPU, a service receiving requests over the network)
// pays for two copies per call besides the search.  This entry point hides
// them: the points are cut into chunks; while the compute stream searches
// chunk i, a copy stream brings chunk i+1 in and another takes the results
// of chunk i-1 out.  Two sets of device buffers alternate between chunks, so
// the copies of one chunk never touch the buffers the search of the other
// is using; events order the three streams.  Each chunk runs the ordinary
// find (+ fused eval) on the compute stream, which waits on the host only to
// size its pair arrays, early in the chunk; the copy streams keep moving
// meanwhile.  (The workspace path would avoid that wait, but its persistent
// grids balance the Newton work of a chunk less well than one block per 128
// pairs does.)
#include <string.h>

#include <algorithm>
#include <string>

#include "fp_common.cuh"
#include "fp_handle.h"
#include "fp_internal.h"

namespace {

struct Slot {
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
    int64_t chunk = 0;
    int F = 0;
    Slot slot[2];
    cudaStream_t cin = nullptr, cout = nullptr;
};

namespace fpg {

void host_stream_free(fp_host_stream* hs)
{
    if (!hs) return;
    if (hs->cin) cudaStreamSynchronize(hs->cin);
    if (hs->cout) cudaStreamSynchronize(hs->cout);
    for (Slot& S : hs->slot) {
        cudaFree(S.pts); cudaFree(S.qs); cudaFree(S.code); cudaFree(S.sub); cudaFree(S.elem);
        cudaFree(S.rst); cudaFree(S.dist2); cudaFree(S.out);
        if (S.in_done) cudaEventDestroy(S.in_done);
        if (S.comp_done) cudaEventDestroy(S.comp_done);
        if (S.out_done) cudaEventDestroy(S.out_done);
    }
    if (hs->cin) cudaStreamDestroy(hs->cin);
    if (hs->cout) cudaStreamDestroy(hs->cout);
    delete hs;
}

}  // namespace fpg

static fp_status stream_state(fp_handle* h, int64_t chunk, int F, fp_host_stream** out)
{
    fp_host_stream* hs = h->host_stream;
    if (hs && (hs->chunk < chunk || hs->F < F)) {
        fpg::host_stream_free(hs);
        h->host_stream = hs = nullptr;
    }
    if (!hs) {
        cudaError_t e = cudaSuccess;
        hs = new fp_host_stream();
        hs->chunk = chunk;
        hs->F = F;
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hs->cin, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&hs->cout, cudaStreamNonBlocking);
        for (Slot& S : hs->slot) {
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
    *out = hs;
    return FP_OK;
}

extern "C" fp_status fp_find_eval_host(fp_handle* h, int64_t P, const double* pts, const int32_t* qsess, int F,
                                       const double* fields, const fp_fields* posted, int32_t* code, int32_t* sub,
                                       int32_t* elem, double* rst, double* dist2, double* out, int64_t chunk,
                                       void* stream)
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
    const int64_t nch = (P + chunk - 1) / chunk;
    fp_host_stream* hs = nullptr;
    fp_status st = stream_state(h, chunk, eval ? F : 0, &hs);
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
        st = eval ? fp_find_eval(h, c, S.pts, qsess ? S.qs : nullptr, F, fields, posted, S.code, S.sub, S.elem,
                                 S.rst, S.dist2, S.out, s)
                  : fp_find(h, c, S.pts, qsess ? S.qs : nullptr, S.code, S.sub, S.elem, S.rst, S.dist2, s);
        if (st != FP_OK) {
            cudaStreamSynchronize(hs->cout);
            cudaStreamSynchronize(hs->cin);
            return st;
        }
        e = cudaEventRecord(S.comp_done, s);
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
    return FP_OK;
}
