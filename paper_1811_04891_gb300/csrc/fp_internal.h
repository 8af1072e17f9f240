// fp_internal.h -- launcher declarations shared between the library's
// translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace fpg {

// number of kernels this library has launched (process-wide, for reporting)
void count_launch(int k = 1);

struct ElemBox;
struct ElemBox32;
struct HashGrid;
struct BasisTab;
struct FindParams;

// setup (fp_setup.cu)
cudaError_t launch_hull(int n, int64_t E, const double* coords, const double* binv, double pad_border,
                        double pad_conv, ElemBox* boxes, double* nodebox, cudaStream_t s);
cudaError_t launch_reduce_boxes(int64_t E, const ElemBox* boxes, const double* nodebox, double* out,
                                int nblocks, cudaStream_t s);
cudaError_t launch_hash_count(int64_t E, const ElemBox* boxes, const HashGrid& g, double hpad, int32_t* cnt,
                              cudaStream_t s);
cudaError_t launch_hash_fill(int64_t E, const ElemBox* boxes, const HashGrid& g, double hpad, int32_t* cur,
                             int32_t* elems, cudaStream_t s);
cudaError_t launch_box32(int64_t E, const ElemBox* boxes, ElemBox32* out, cudaStream_t s);
cudaError_t launch_hash_sort(int64_t ncell, const int32_t* start, int32_t* elems, cudaStream_t s);
cudaError_t launch_face_corners(int n, int64_t E, const double* coords, double* fc, cudaStream_t s);
cudaError_t launch_face_boundary(int64_t E, const double* fc, const int32_t* sub, const HashGrid& g,
                                 const int32_t* cstart, const int32_t* celems, int32_t* nbnd, cudaStream_t s);
cudaError_t launch_face_gather(int n, int64_t E, const double* coords, const int32_t* sub, const int32_t* bnd_off,
                               double* bx, int32_t* bs, int64_t nb, cudaStream_t s);
cudaError_t launch_dist_default(int n, int64_t E, const double* coords, const int32_t* sub, const double* bx,
                                const int32_t* bs, int64_t nb, double* D, cudaStream_t s);
cudaError_t launch_local32(int n, int64_t E, const double* coords, const ElemBox* boxes, float* c32,
                           cudaStream_t s);
cudaError_t launch_local32lo(int n, int64_t E, const double* coords, const ElemBox* boxes, const float* c32,
                             float* c32lo, cudaStream_t s);

// scans (fp_scan.cu): out[0..n] = exclusive prefix sums of in[0..n), out[n] = total.
// tmp must hold scan_tmp_elems(n) int32 entries.
int64_t scan_tmp_elems(int64_t n);
cudaError_t scan_exclusive(const int32_t* in, int32_t* out, int64_t n, int32_t* tmp, cudaStream_t s);

// find (fp_find.cu)
// Optional fused evaluation after classification, in the element-sorted pair
// order: F fields, FP64 ([F][E][n3]) or double-float pairs; out [F][P].
// threads per block of the Newton kernels when fp_opts.points_per_block is 0:
// 64 for fp_find / fp_find_eval on hexahedra (measured 1 % faster than 128
// for the FP64 form, the same for the mixed form, whose capped kernel takes
// blocks of at most 128); 128 for quadrilaterals and for the workspace and
// allocation-free calls, whose persistent grids are sized for it
constexpr int kDefaultBlockFind3 = 64;
constexpr int kDefaultBlock = 128;

struct EvalSpec {
    int F;
    const double* f64;
    const float2* fdf;
    double* out;
    int staged = 0;     // posted fields: stage each element's fields in shared memory (fp_set_eval_staging)
};

struct FindArgs {
    int n;
    int64_t E;
    int64_t P;
    const double* pts;
    const int32_t* qsess;
    const double* coords;
    const float* coords32;
    const float* coords32lo;
    const int32_t* sub;
    const double* dist;
    const ElemBox* boxes;
    const ElemBox32* boxes32;     // non-null: screen with FP32 boxes and FP32 hashing
    const HashGrid* grid;         // host copy
    const int32_t* cell_start;
    const int32_t* cell_elems;
    // scratch
    int32_t* cnt;                 // [P]
    int32_t* off;                 // [P+1]
    int32_t* pair_elem;           // [cap]
    int32_t* pair_pt;             // [cap]
    int32_t* ecount;              // [E]  (zeroed by the launcher)
    int32_t* estart;              // [E+1]
    int32_t* order;               // [cap]
    int32_t* inv;                 // [cap] sorted position of each pair slot; set (3D): the Newton stage keeps
                                  //   pair results in sorted order (coalesced), null (2D): in slot order
    double* pres;                 // [cap]
    double* prst;                 // [3][cap]
    int32_t* scan_tmp;
    int64_t cap;                  // pair capacity
    int persistent_blocks;        // 0: pair count known on the host; >0: device-side count, this many blocks
    int64_t pts_stride;           // screen only: row stride of pts (0 = P)
    int32_t pt_base;              // screen only: offset added to emitted point indices
    int32_t elem_base;            // screen only: offset added to emitted element indices
    // optional timing events (null = off): [0,1] sort, [2,3] newton, [4,5] rank, [6,7] fused eval
    cudaEvent_t ev[8];
    EvalSpec eval;                // eval.F == 0: find only
    unsigned long long* stats;    // optional Newton path counters (4 words), null = off
    unsigned long long* band;     // optional near-tie counters (3 words, see fp_rank.cuh), null = off
    const int32_t* warm_elem;     // optional warm start: previous element [P] (null = off)
    const double* warm_rst;       // and previous reference coordinates [3][P]
    // batch groups (fp_batch.cu): the group's pairs are the sorted positions
    // [*s_lo, *s_hi); pair_elem - ebase indexes the group's arrays
    const int32_t* s_lo;
    const int32_t* s_hi;
    int32_t ebase;
    int32_t* queue;               // Newton work-queue counter (zeroed by the launcher), null = grid-stride
    int tile;                     // sorted positions per work item (0: one block's worth)
    int32_t* fb_count;            // mixed form, batch groups: fallback counter and list (group slice
    int32_t* fb_list;             //   from the group's first sorted position)
    double2* pstate;              // FP64 form: [cap] state of solves paused by the first pass (null: one pass)
    // outputs
    int32_t* code;
    int32_t* osub;
    int32_t* oelem;
    double* rst;
    double* dist2;
    uint32_t* smask = nullptr;    // [P] screen: candidates that passed the count pass, by bit of the
                                  //   cell list (bit 31: list too long, test again); null = test again
    int batch = 0;                // 1: a batch group (its own FP64 first-pass budget)
};
cudaError_t find_count(const FindArgs& a, const BasisTab& tab, const FindParams& fp, cudaStream_t s);
cudaError_t find_screen_count(const FindArgs& a, cudaStream_t s);   // counts only, no scan
cudaError_t find_emit(const FindArgs& a, cudaStream_t s);
cudaError_t find_solve(const FindArgs& a, int64_t npairs, const BasisTab& tab, const FindParams& fp,
                       int block, cudaStream_t s);
cudaError_t find_solve_unsorted(const FindArgs& a, int64_t npairs, const BasisTab& tab, const FindParams& fp,
                                int block, cudaStream_t s);
struct BScreenArgs;
cudaError_t launch_bscreen(const BScreenArgs& b, bool emit, bool f32, cudaStream_t s);
int newton_blocks_per_sm(int n, bool mixed, int block);
cudaError_t find_newton_group(const FindArgs& a, const BasisTab& tab, const FindParams& fp, int block, unsigned grid,
                              cudaStream_t s);

// host streaming state of fp_find_eval_host (fp_stream.cu), freed with the handle
}  // namespace fpg
struct fp_host_stream;
struct fp_workspace;
namespace fpg {
void host_stream_free(fp_host_stream* hs);
// workspace launches over its whole pair capacity instead of a persistent grid
void workspace_unpersist(fp_workspace* w);
void workspace_grid_hint(fp_workspace* w, int64_t pairs);
// copy the workspace's device pair count of its latest find to *host_dst on s
cudaError_t workspace_pair_count_async(fp_workspace* w, int32_t* host_dst, cudaStream_t s);

// counting sort of the pairs by element (fp_find.cu), shared by both dimensions
cudaError_t find_sort(const FindArgs& a, int64_t npairs, cudaStream_t s);

// 2D quadrilateral variant (fp_find2.cu): coords [2][E][n^2], pts / rst [2][P]
cudaError_t launch_hull2(int n, int64_t E, const double* coords, const double* binv, double pad_border,
                         double pad_conv, ElemBox* boxes, double* nodebox, cudaStream_t s);
// default D^k from the boundary edges of each subdomain; *too_large when the
// node x boundary-node pairs exceed max_pairs (nothing computed then)
cudaError_t launch_dist_default2(int n, int64_t E, const double* coords, const int32_t* sub, const HashGrid& g,
                                 const int32_t* cstart, const int32_t* celems, double* D, int64_t max_pairs,
                                 bool* too_large, cudaStream_t s);
cudaError_t find_count2(const FindArgs& a, cudaStream_t s);
cudaError_t find_emit2(const FindArgs& a, cudaStream_t s);
cudaError_t find_solve2(const FindArgs& a, int64_t npairs, const BasisTab& tab, const FindParams& fp, int block,
                        cudaStream_t s);
cudaError_t launch_eval2(int n, int64_t E, int64_t P, const int32_t* code, const int32_t* elem, const double* rst,
                         int F, const double* fields, double* out, const BasisTab& tab, cudaStream_t s);

// eval (fp_eval.cu)
// s_lo / s_hi / ebase: batch groups, as in FindArgs (null: all live pairs)
cudaError_t launch_eval_pairs(int n, int64_t E, int64_t P, const int32_t* dcount, int64_t cap, const int32_t* order,
                              const int32_t* pair_elem, const int32_t* pair_pt, const double* prst,
                              const EvalSpec& ev, const BasisTab& tab, unsigned grid, cudaStream_t s,
                              const int32_t* s_lo = nullptr, const int32_t* s_hi = nullptr, int32_t ebase = 0,
                              bool walk = false);
cudaError_t launch_split_df(int64_t count, int n, const double* src, float2* dst, cudaStream_t s);
cudaError_t launch_eval_df(int n, int64_t E, int64_t P, const int32_t* code, const int32_t* elem, const double* rst,
                           int F, const float2* fields, double* out, const BasisTab& tab, cudaStream_t s);
cudaError_t launch_points_basis(int n, int64_t P, const int32_t* code, const int32_t* elem, const double* rst,
                                float* basis, int32_t* pe, const BasisTab& tab, cudaStream_t s);
cudaError_t launch_eval_points_df(int n, int64_t E, int64_t P, int F, const int32_t* pe, const float* basis,
                                  const float2* fields, double* out, cudaStream_t s);
cudaError_t launch_eval(int n, int64_t E, int64_t P, const int32_t* code, const int32_t* elem, const double* rst,
                        int F, const double* fields, double* out, const BasisTab& tab, cudaStream_t s);

}  // namespace fpg
