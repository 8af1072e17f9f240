// fp_static.cu -- fp_find_static: point location that allocates nothing.
//
// Some callers cannot allocate device memory at the moment they need to
// locate points: a solver that has handed all free device memory to its own
// pool allocator (cudaMalloc would fail or fragment that pool), or a
// latency-bound time-step loop that cannot take the implicit device-wide
// synchronisation of cudaMalloc / cudaFree.  For them this entry point runs
// the same screen / Newton / classification kernels as fp_find, with all
// per-call scratch (pair offsets, pair lists, per-pair results) carved out of
// one file-scope device array of fixed size, g_fp_static_scratch.  The array
// exists on every GPU that loads the library and is held until the process
// exits.  Like fp_find, the call waits once on its stream, to read the number
// of candidate pairs back to the host.
//
// Limits: at most FP_STATIC_MAX_POINTS points and FP_STATIC_MAX_PAIRS
// (point, candidate element) pairs per call.  The point limit is checked
// before any device work; the pair count is only known after the screen has
// counted the candidates, so a request over the pair limit is rejected with
// FP_ERR_INVALID_ARG after that counting pass (its outputs are then left
// unwritten).  Pairs are solved in point order (no sort by element), which
// changes only the schedule, not the result of any pair.
//
// Sharing: every call on a device uses the same array and leaves the last
// call's contents in it.  Nothing in it needs to start at zero (every word a
// kernel reads was written earlier in the same call).  Calls whose work
// overlaps on the GPU (for example on two streams at once) race on the array
// and must be serialised by the caller.
//
// Set-up: the first call on each device, with that device current, looks up
// the array's device address with cudaGetSymbolAddress (in host code the
// symbol is only a host-side stand-in, not a device address).  Make that
// first call before starting any stream capture.  A handle is used on the
// device it was set up on; a call made while another device is current is
// refused, since the scratch address would belong to the wrong GPU.
#include <mutex>

#include "fp_common.cuh"
#include "fp_handle.h"
#include "fp_internal.h"

namespace {

constexpr int64_t kMaxPoints = FP_STATIC_MAX_POINTS;
constexpr int64_t kMaxPairs = FP_STATIC_MAX_PAIRS;
constexpr int64_t kScanTmp = 8192;   // int32 words; scan_tmp_elems(kMaxPoints) is 4116

constexpr size_t al256(size_t b) { return (b + 255) & ~size_t(255); }
constexpr size_t kOffCnt = 0;
constexpr size_t kOffOff = kOffCnt + al256(4 * kMaxPoints);
constexpr size_t kOffScan = kOffOff + al256(4 * (kMaxPoints + 1));
constexpr size_t kOffPe = kOffScan + al256(4 * kScanTmp);
constexpr size_t kOffPp = kOffPe + al256(4 * kMaxPairs);
constexpr size_t kOffOrd = kOffPp + al256(4 * kMaxPairs);
constexpr size_t kOffRes = kOffOrd + al256(4 * kMaxPairs);
constexpr size_t kOffRst = kOffRes + al256(8 * kMaxPairs);
constexpr size_t kBytes = kOffRst + al256(24 * kMaxPairs);   // about 2.8 MB

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

}  // namespace

static __device__ __align__(256) unsigned char g_fp_static_scratch[kBytes];

namespace fpg {

__global__ void k_iota(int64_t n, int32_t* __restrict__ out)
{
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i < n) out[i] = (int32_t)i;
}

}  // namespace fpg

// device address of the scratch array on the current device (looked up once)
static cudaError_t static_scratch(void** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_fp_static_scratch);
        if (e != cudaSuccess) return e;
        g_addr[dev] = p;
    }
    *out = g_addr[dev];
    return cudaSuccess;
}

extern "C" fp_status fp_find_static(fp_handle* h, int64_t P, const double* pts, const int32_t* qsess, int32_t* code,
                                    int32_t* sub, int32_t* elem, double* rst, double* dist2, void* stream)
{
    using namespace fpg;
    if (!fp_live(h)) return FP_ERR_NOT_SETUP;
    h->err.clear();
    if (h->dim != 3) {
        h->err = "fp_find_static: hexahedral meshes only";
        return FP_ERR_INVALID_ARG;
    }
    if (P < 0 || P > kMaxPoints) {
        h->err = "fp_find_static: P must be in [0, FP_STATIC_MAX_POINTS = 16384]";
        return FP_ERR_INVALID_ARG;
    }
    if (P == 0) return FP_OK;
    if (!pts || !code || !sub || !elem || !rst || !dist2) {
        h->err = "fp_find_static: null pointer argument";
        return FP_ERR_INVALID_ARG;
    }
    int cur = -1;
    if (cudaGetDevice(&cur) != cudaSuccess || cur != h->device) {
        h->err = "fp_find_static: the current device is not the handle's device";
        return FP_ERR_INVALID_ARG;
    }
    if (scan_tmp_elems(P) > kScanTmp) {
        h->err = "fp_find_static: scan scratch too small";
        return FP_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    void* base = nullptr;
    cudaError_t err = static_scratch(&base);
    if (err != cudaSuccess) {
        h->err = std::string("fp_find_static: scratch address: ") + cudaGetErrorString(err);
        return FP_ERR_CUDA;
    }
    unsigned char* b = static_cast<unsigned char*>(base);
    FindArgs a;
    memset(&a, 0, sizeof(a));
    a.n = h->n; a.E = h->E; a.P = P; a.pts = pts; a.qsess = qsess;
    a.coords = h->coords; a.coords32 = h->coords32; a.coords32lo = h->coords32lo; a.sub = h->sub;
    a.dist = h->nsub > 1 ? h->dist : nullptr;
    a.boxes = h->boxes; a.boxes32 = h->boxes32; a.grid = &h->grid;
    a.cell_start = h->cell_start; a.cell_elems = h->cell_elems;
    a.cnt = reinterpret_cast<int32_t*>(b + kOffCnt);
    a.off = reinterpret_cast<int32_t*>(b + kOffOff);
    a.scan_tmp = reinterpret_cast<int32_t*>(b + kOffScan);
    a.pair_elem = reinterpret_cast<int32_t*>(b + kOffPe);
    a.pair_pt = reinterpret_cast<int32_t*>(b + kOffPp);
    a.order = reinterpret_cast<int32_t*>(b + kOffOrd);
    a.pres = reinterpret_cast<double*>(b + kOffRes);
    a.prst = reinterpret_cast<double*>(b + kOffRst);
    a.cap = kMaxPairs;
    a.code = code; a.osub = sub; a.oelem = elem; a.rst = rst; a.dist2 = dist2;
    a.stats = h->prof ? h->stats : nullptr;
    a.band = h->band;
    a.inv = a.order;    // pairs stay in point order: order and its inverse are both the identity
    FindParams fp;
    fp.tol_accept = h->opts.tol_accept;
    fp.tol_border = h->opts.tol_border;
    fp.band = h->opts.tie_band * h->L;
    fp.max_newton = h->opts.max_newton;
    fp.mixed = h->opts.precision == FP_PREC_MIXED;
    fp.refine = h->refine;

    err = find_count(a, h->tab, fp, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(h->h_total, a.off + P, sizeof(int32_t), cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    if (err != cudaSuccess) {
        h->err = std::string("fp_find_static count: ") + cudaGetErrorString(err);
        return FP_ERR_CUDA;
    }
    const int64_t npairs = h->h_total[0];
    h->last_pairs = npairs;
    if (npairs < 0 || npairs > kMaxPairs) {
        h->err = "fp_find_static: more than FP_STATIC_MAX_PAIRS = 65536 candidate pairs";
        return FP_ERR_INVALID_ARG;
    }
    if (npairs > 0) {
        err = find_emit(a, s);
        if (err == cudaSuccess) {
            k_iota<<<(unsigned)((npairs + 255) / 256), 256, 0, s>>>(npairs, a.order);
            count_launch();
            err = cudaGetLastError();
        }
    }
    const int block = h->opts.points_per_block > 0 ? h->opts.points_per_block : kDefaultBlock;
    if (err == cudaSuccess) err = find_solve_unsorted(a, npairs, h->tab, fp, block, s);
    if (err != cudaSuccess) {
        h->err = std::string("fp_find_static: ") + cudaGetErrorString(err);
        return FP_ERR_CUDA;
    }
    return FP_OK;
}
