// fp_handle.h -- the opaque handle behind the C ABI (shared by the
// translation units that implement entry points).
#pragma once
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "fp_common.cuh"

struct fp_host_stream;   // fp_find_eval_host state (fp_stream.cu)

enum { PROF_SCREEN = 0, PROF_SORT = 1, PROF_NEWTON = 2, PROF_RANK = 3, PROF_EVAL = 4, PROF_KINDS = 5 };

struct fp_handle {
    int device = -1;               // CUDA device the handle was set up on
    int dim = 3;                   // 3: hexahedra, coords [3][E][n^3]; 2: quadrilaterals, [2][E][n^2]
    int N = 0, n = 0;
    int64_t E = 0;
    int nsub = 0;
    fp_opts opts{};
    int refine = 3;                // mixed form: compensated residuals per pair (fp_set_mixed_refine)
    int stage_eval = 0;            // fused eval of posted fields from shared memory (fp_set_eval_staging)
    fpg::BasisTab tab{};
    fpg::HashGrid grid{};
    int64_t nnz = 0;
    double L = 0.0;
    // resident device state
    double* coords = nullptr;      // [3][E][n3]
    float* coords32 = nullptr;     // [3][E][n3] element-local FP32 (mixed form)
    float* coords32lo = nullptr;   // [3][E][n3] low parts: (x - c) - coords32 (mixed form)
    int32_t* sub = nullptr;        // [E]
    double* dist = nullptr;        // [E][n3] or null
    fpg::ElemBox* boxes = nullptr;      // [E]
    fpg::ElemBox32* boxes32 = nullptr;  // [E] mixed form only
    int32_t* cell_start = nullptr; // [ncell+1]
    int32_t* cell_elems = nullptr; // [nnz]
    int32_t* ecount = nullptr;     // [E]
    int32_t* estart = nullptr;     // [E+1]
    int32_t* escan_tmp = nullptr;
    // find workspace
    int64_t cap_pts = 0, cap_pairs = 0;
    int32_t* cnt = nullptr;
    uint32_t* smask = nullptr;     // [cap_pts] screen: count-pass candidate masks
    int32_t* off = nullptr;
    int32_t* scan_tmp = nullptr;
    int32_t* pair_elem = nullptr;
    int32_t* pair_pt = nullptr;
    int32_t* order = nullptr;
    double* pres = nullptr;
    double* prst = nullptr;
    double2* pstate = nullptr;     // FP64 form: state of solves paused by the first Newton pass
    int32_t* inv = nullptr;        // [cap] sorted position of each pair slot (hexahedral handles)
    int32_t* h_total = nullptr;    // pinned host word for the pair count
    // geometry scratch kept for fp_update_coords (moving meshes)
    double* binv = nullptr;        // [n][n] inverse Bernstein-to-Lagrange matrix
    double pad_conv = 0.0;         // hull padding for the rounding of the conversion
    double hpad = 0.0;             // hash widening for FP32 lookups (mixed form)
    double* nodebox = nullptr;     // [6E]
    double* red = nullptr;         // [12 * nred]
    int nred = 0;
    int32_t* hcnt = nullptr;       // [ncell_cap] hash counts / fill cursor
    int32_t* htmp = nullptr;       // scan scratch for ncell_cap cells
    int32_t* flag = nullptr;       // [1] non-finite counter
    int64_t ncell_cap = 0, nnz_cap = 0;
    bool dist_default = false;     // dist was computed by the library (default field)
    bool stale = false;            // a failed fp_update_coords left the geometry inconsistent
    fp_host_stream* host_stream = nullptr;   // buffers and streams of fp_find_eval_host
    int64_t last_pairs = 0;
    std::string err;
    // optional per-kernel timing with CUDA events on the launching stream
    bool prof = false;
    unsigned long long* stats = nullptr;   // device [4] Newton path counters while profiling
    unsigned long long* band = nullptr;    // device [3] near-tie counters of the classification (always on)
    std::vector<cudaEvent_t> ev_free;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_pend[PROF_KINDS];
};

// a handle that holds a complete, consistent mesh
inline bool fp_live(const fp_handle* h) { return h && h->coords && !h->stale; }

