/*
 * findpts_gb.h -- C ABI of the GB300 point-location / interpolation library.
 *
 * The library finds, for query points x* in R^3, the computational
 * coordinates q* = (subdomain, element e, r, s, t) on a set of overlapping
 * hexahedral spectral-element meshes, and interpolates nodal fields there
 * (arXiv 1811.04891, Sec. 2.1: findpts_setup / findpts / findpts_eval with a
 * session discriminator and the distance-to-boundary owner rule).
 *
 * Conventions shared by every entry point
 *  - N is the polynomial order, n = N + 1 GLL points per direction,
 *    n3 = n^3 nodes per element, 1 <= N <= 15.
 *  - Node (i,j,k) of an element sits at local index i + n*(j + n*k), i fastest.
 *  - All array arguments are DEVICE pointers (cudaMalloc'd or from a device
 *    allocator such as PyTorch's) on the current CUDA device unless stated.
 *    The caller owns every pointer it passes; the library never frees them.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Every call only enqueues work on that stream; outputs are valid once the
 *    stream has been synchronised.  No call synchronises the device, except
 *    fp_setup and workspace growth (see fp_reserve), which allocate.
 *  - No C++ exception crosses this boundary.  Every call returns an
 *    fp_status; the text of the last failure is kept in the handle and
 *    returned by fp_last_error().
 *  - A handle is not thread-safe: calls on one handle must be serialised by
 *    the caller (they may use different streams, but one at a time; find
 *    calls share the handle's workspace).
 */
#ifndef FINDPTS_GB_H
#define FINDPTS_GB_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct fp_handle fp_handle;   /* opaque; owns all resident device state */

typedef enum {
    FP_OK = 0,
    FP_ERR_INVALID_ARG = 1,   /* bad sizes, null required pointer, non-finite mesh  */
    FP_ERR_OOM = 2,           /* device allocation failed                            */
    FP_ERR_CUDA = 3,          /* a CUDA runtime call or kernel launch failed         */
    FP_ERR_TIMEOUT = 4,       /* a bounded device-side wait gave up (reserved: no
                                 kernel of this library waits on another block)    */
    FP_ERR_NOT_SETUP = 5      /* null handle or handle without a mesh                */
} fp_status;

/* Per-point result codes (Sec. 2.1: found inside an element, on a border, or
   not found within the mesh).  FP_CODE_RETRY only comes from fp_find_ws: the
   workspace ran out of candidate-pair capacity before this point's pairs, so
   the point was not searched (sub = elem = -1, r = 0, dist2 = +inf). */
enum { FP_CODE_INSIDE = 0, FP_CODE_BORDER = 1, FP_CODE_NOT_FOUND = 2, FP_CODE_RETRY = 3 };

/* Arithmetic forms of fp_find. */
enum {
    FP_PREC_FP64 = 0,         /* every step in FP64                                      */
    FP_PREC_MIXED = 1         /* FP32 seed and early Newton steps on element-local
                                 coordinates, FP64 final Newton step(s), residual,
                                 classification, owner comparison and eval          */
};

typedef struct {
    int precision;              /* FP_PREC_FP64 (default) or FP_PREC_MIXED               */
    double tol_accept;          /* INSIDE if ||x^e(r)-x*|| <= tol_accept*h_e (1e-12)     */
    double tol_border;          /* BORDER if residual <= tol_border*h_e (1e-6)           */
    int max_newton;             /* Newton iteration cap per candidate (40)               */
    double hash_cells_per_elem; /* hash-grid cells per element (1.0); result-invariant   */
    double tie_band;            /* owner and border ties within tie_band*L (1e-10)       */
    int points_per_block;       /* threads per block of the Newton kernel: 0 (= 64 for
                                   fp_find / fp_find_eval on hexahedra, 128 for
                                   quadrilaterals and for the workspace and
                                   allocation-free calls) or a multiple of 32 up to
                                   256; result-invariant                              */
} fp_opts;
/* h_e = diagonal of the axis-aligned box spanned by element e's nodes;
   L = diagonal of the box spanned by all nodes. */

/* Fill *o with the defaults above. */
void fp_default_opts(fp_opts *o);

/* fp_setup -- post the meshes (Sec. 2.1, findpts_setup with a per-element
 * session discriminator) and build the resident search structures: per
 * element bounding boxes from the Bernstein form of the element map (an axis
 * box and a box in the element's own affine frame) and a uniform hash grid
 * over the global box with a cell -> element list.
 *   h      out: new handle (set to NULL on failure)
 *   coords [3][E][n3] FP64 node coordinates x, y, z of every element
 *   E      number of elements (>= 1, < 2^31)
 *   N      polynomial order (1..15)
 *   sub    [E] int32 subdomain (session) id per element, 0 <= sub < 65536;
 *          NULL = all elements in subdomain 0
 *   dist   [E][n3] FP64 nodal distance-to-own-boundary field D^k used by the
 *          owner rule, or NULL.  When NULL and the mesh has more than one
 *          subdomain, the library computes D (distance from each node to the
 *          nearest boundary-face GLL node of its own subdomain); that
 *          brute-force pass is limited to meshes with at most 2^37
 *          node x boundary-node pairs, beyond which FP_ERR_INVALID_ARG is
 *          returned and D must be supplied.
 *   opts   NULL = defaults
 * The library copies everything it keeps; the caller may free its buffers
 * once `stream` has been synchronised.  Synchronises `stream` before return.
 * Errors: FP_ERR_INVALID_ARG (E, N, sub or opts out of range, null coords,
 * non-finite coordinates), FP_ERR_OOM, FP_ERR_CUDA. */
fp_status fp_setup(fp_handle **h, const double *coords, int64_t E, int N,
                   const int32_t *sub, const double *dist, const fp_opts *opts,
                   void *stream);

/* fp_setup_2d -- the 2D (quadrilateral) variant (the paper's 2D overset
 * examples, Sec. 3): the same set-up on a mesh of quads with
 * x^e(r,s) = sum_ij x_ij h_i(r) h_j(s).
 *   coords [2][E][n2] FP64 node coordinates x, y, node (i,j) at i + n*j,
 *          n2 = n^2
 *   dist   [E][n2] D^k, or NULL: with more than one subdomain the library
 *          computes the default (distance from each node to the nearest GLL
 *          node of a boundary edge of its own subdomain; the same 2^37
 *          node x boundary-node limit as fp_setup)
 *   opts   the FP64 form only (FP_PREC_MIXED gives FP_ERR_INVALID_ARG)
 * On a 2D handle fp_find, fp_find_eval, fp_find_warm and fp_eval take
 * points and reference coordinates as [2][P] and fields as [F][E][n2], with
 * the same rules, codes and errors; fp_update_coords takes [2][E][n2].  The
 * workspace, static, batch, posted-field and boundary-face calls accept
 * hexahedral handles only (FP_ERR_INVALID_ARG otherwise). */
fp_status fp_setup_2d(fp_handle **h, const double *coords, int64_t E, int N,
                      const int32_t *sub, const double *dist, const fp_opts *opts,
                      void *stream);

/* fp_reserve -- pre-size the find workspace for up to P points, so that
 * later fp_find calls with at most P points allocate nothing (required before
 * capturing fp_find into a CUDA graph).  Synchronises the device.
 * Errors: FP_ERR_NOT_SETUP, FP_ERR_INVALID_ARG (P < 0), FP_ERR_OOM,
 * FP_ERR_CUDA. */
fp_status fp_reserve(fp_handle *h, int64_t P);

/* fp_find -- locate P points (Sec. 2.1, findpts).
 *   pts    [3][P] FP64 query coordinates
 *   qsess  [P] int32 session tag per point: a point tagged j searches only
 *          elements with sub != j; -1 searches all.  NULL = all -1.
 * Outputs (all [P] unless stated):
 *   code   int32 FP_CODE_*;  non-finite points give FP_CODE_NOT_FOUND
 *   sub    int32 owning subdomain (-1 when not found)
 *   elem   int32 element index in [0,E) (-1 when not found)
 *   rst    [3][P] FP64 reference coordinates in [-1,1]^3 (0 when not found)
 *   dist2  FP64 squared residual ||x^e(r)-x*||^2 (+inf when not found)
 * Rules: INSIDE elements within a subdomain -> lowest element id; between
 * subdomains -> largest interpolated D^k(x*), ties within tie_band*L to the
 * lower subdomain id; no INSIDE element but a constrained residual within
 * tol_border*h_e -> BORDER at the element of smallest residual (lowest id
 * within tie_band*L).  P = 0 is a no-op.  May grow the workspace (allocates
 * and synchronises) when P exceeds what fp_reserve or an earlier call sized.
 * Errors: FP_ERR_NOT_SETUP, FP_ERR_INVALID_ARG (P < 0, null pointers),
 * FP_ERR_OOM, FP_ERR_CUDA. */
fp_status fp_find(fp_handle *h, int64_t P, const double *pts, const int32_t *qsess,
                  int32_t *code, int32_t *sub, int32_t *elem, double *rst,
                  double *dist2, void *stream);

/* fp_eval -- interpolate F nodal fields at located points (Sec. 2.1,
 * findpts_eval): out[f][p] = sum_ijk fields[f][elem[p]][ijk] h_i(r) h_j(s) h_k(t)
 * evaluated by sum factorisation in FP64.
 *   code, elem, rst  as written by fp_find (rst is [3][P])
 *   fields  [F][E][n3] FP64 nodal values on the handle's mesh
 *   out     [F][P] FP64; quiet NaN where code is FP_CODE_NOT_FOUND
 * `fields` must be 16-byte aligned when n is even (rows are read as 16-byte
 * vectors).  Allocates nothing.  Errors: FP_ERR_NOT_SETUP,
 * FP_ERR_INVALID_ARG (P < 0, F < 1, null pointers, misaligned fields),
 * FP_ERR_CUDA. */
fp_status fp_eval(fp_handle *h, int64_t P, const int32_t *code, const int32_t *elem,
                  const double *rst, int F, const double *fields, double *out,
                  void *stream);

/* fp_find_static -- fp_find for callers that cannot allocate device memory
 * at call time: a solver whose device memory is all handed to its own pool
 * allocator, or a latency-bound loop that cannot afford the implicit device
 * synchronisation of cudaMalloc / cudaFree.  The paper has no counterpart;
 * this is a deployment variant of fp_find.
 * Same arguments, outputs, rules and results as fp_find, for at most
 * FP_STATIC_MAX_POINTS points and FP_STATIC_MAX_PAIRS candidate pairs per
 * call.  A request over the point limit returns FP_ERR_INVALID_ARG before any
 * device work; the pair count is known only after the screen has counted the
 * candidates, so a request over the pair limit returns FP_ERR_INVALID_ARG
 * after that counting pass, with the outputs unwritten.
 * All per-call scratch lives in one file-scope device array of about 2.8 MB
 * that every GPU loading the library holds until exit; the call makes no
 * cudaMalloc / cudaFree or other allocating call.  The first call on each
 * device looks up the array's device address (cudaGetSymbolAddress) and
 * should come before any stream capture.  The handle's device must be the
 * current device (FP_ERR_INVALID_ARG otherwise).  All calls share the array
 * and it keeps the last call's contents (no part of it needs to start at
 * zero); calls that overlap on the GPU race on it and must be serialised.
 * Like fp_find it waits for `stream` once, to read the number of pairs.
 * Band hits and (while profiling) Newton path counts are counted as for
 * fp_find; fp_profile does not time the kernels of static calls.
 * fp_last_find_stats reports the pairs of the latest static call too.
 * Errors: FP_ERR_NOT_SETUP, FP_ERR_INVALID_ARG, FP_ERR_CUDA. */
#define FP_STATIC_MAX_POINTS 16384
#define FP_STATIC_MAX_PAIRS 65536
fp_status fp_find_static(fp_handle *h, int64_t P, const double *pts, const int32_t *qsess,
                         int32_t *code, int32_t *sub, int32_t *elem, double *rst,
                         double *dist2, void *stream);

/* Workspaces for asynchronous finds.  A workspace holds all per-call scratch
 * of fp_find_ws for up to max_points points and max_pairs candidate pairs on
 * one handle's mesh; several workspaces let several finds run at once on
 * different streams (each workspace must be used by one call at a time).
 * fp_workspace_create allocates (max_pairs <= 0 picks 2 * max_points) and
 * writes the new workspace to *ws (NULL on failure); it serves hexahedral
 * handles only.  Errors: FP_ERR_NOT_SETUP, FP_ERR_INVALID_ARG (ws NULL,
 * max_points outside [1, 2^31), max_pairs >= 2^31, a 2D handle), FP_ERR_OOM,
 * FP_ERR_CUDA.  fp_workspace_free synchronises the device, then frees (NULL
 * is a no-op); the handle must outlive its workspaces. */
typedef struct fp_workspace fp_workspace;
fp_status fp_workspace_create(const fp_handle *h, int64_t max_points, int64_t max_pairs,
                              fp_workspace **ws);
void fp_workspace_free(fp_workspace *ws);
/* Device bytes a workspace of max_points points and max_pairs pairs
 * (<= 0: 2 * max_points) on this handle's mesh holds, for callers that
 * budget device memory (the per-point, per-pair and per-element arrays;
 * allocator rounding not included).  Errors: FP_ERR_NOT_SETUP,
 * FP_ERR_INVALID_ARG (bytes NULL, sizes out of range). */
fp_status fp_workspace_bytes(const fp_handle *h, int64_t max_points, int64_t max_pairs,
                             int64_t *bytes);

/* fp_find_ws -- fp_find with its scratch in `ws`.  Never waits on the host
 * and never allocates, so a sequence of fp_find_ws / fp_eval calls can be
 * captured into a CUDA graph and replayed.  The number of candidate pairs
 * stays on the device; if it exceeds the workspace's max_pairs, the points
 * whose pairs did not fit come back as FP_CODE_RETRY (all others are
 * complete and identical to fp_find).  Errors: FP_ERR_NOT_SETUP,
 * FP_ERR_INVALID_ARG (P outside [0, max_points], null pointers, a workspace
 * made for another handle), FP_ERR_CUDA. */
fp_status fp_find_ws(fp_handle *h, fp_workspace *ws, int64_t P, const double *pts,
                     const int32_t *qsess, int32_t *code, int32_t *sub, int32_t *elem,
                     double *rst, double *dist2, void *stream);

/* Number of candidate pairs of the workspace's most recent fp_find_ws
 * (synchronises the device; for diagnostics).  Errors: FP_ERR_INVALID_ARG
 * (ws NULL), FP_ERR_CUDA. */
fp_status fp_workspace_last_pairs(fp_workspace *ws, int64_t *npairs);

/* Batches: many independent meshes (instances) of different E and N located
 * and interpolated in one launch sequence (the paper posts all meshes of all
 * sessions to one findpts_setup, Sec. 2.1; here independent problems share
 * the device).  Instances of the same N form a group whose geometry, boxes
 * and fields are copied into group-resident arrays at creation.  A run
 * screens every point against its own instance's hash grid and boxes in one
 * launch, sorts all candidate pairs by element in one pass, solves each
 * group's pairs with one persistent Newton launch whose warps draw work
 * items (runs of `tile` element-sorted pairs) from a device counter, the
 * groups' launches running concurrently, classifies every point (with its
 * own instance's tie band, so each result equals fp_find on that instance
 * alone) and evaluates the winning pairs, writing the results directly in
 * instance order.  A run never waits on the host, so it can be captured into
 * one CUDA graph.
 *   handles  [ninst] set-up handles on the current device (same precision,
 *            tolerances and max_newton); they must outlive the batch
 *   npts     [ninst] host array: points per instance (instance i owns points
 *            [sum_{k<i} npts_k, sum_{k<=i} npts_k) of every run)
 *   F        fields per instance (0 = find only)
 *   fields   [ninst] host array of device pointers, instance i's fields laid
 *            out [F][E_i][n_i^3] (NULL when F = 0); copied at creation
 *   pairs_per_point  pair capacity per point of the whole batch (<= 0: 2.0);
 *            points beyond it come back as FP_CODE_RETRY
 * fp_batch_run: pts [3][Ptot], outputs as fp_find over Ptot points plus
 * out [F][Ptot] (may be NULL); element ids are instance-local.
 * fp_batch_tune: per group, times the Newton stage on the given data for
 * every schedule -- threads per block 64/128/256 x blocks per SM 1/2/4/8
 * (those that fit), then work items of 32, 128 or 512 pairs per warp --
 * keeps the fastest, and caches it for the process by (form, N, log2 E,
 * log2 pairs): a later batch or call whose group falls in a tuned bucket
 * takes the cached schedule without timing.  It then times whole runs with
 * the groups' launches concurrent and one after another, keeps the faster
 * mode, and returns that run's time (synchronises).
 * fp_batch_schedule reads (and, for positive inputs, sets) one group's
 * schedule; tile must be a multiple of 32.  fp_batch_groups gives the
 * number of groups; fp_batch_group_info a group's N, elements, points,
 * candidate pairs of the latest run (synchronises) and the Newton and eval
 * times (ms) of the latest profiled run (with fp_batch_profile(b, 1), runs
 * record events around each group's Newton and eval launches and run the
 * groups one after another on the caller's stream, so that each time is the
 * group's own; graphs are captured without them) or, for the Newton stage,
 * of the tuning.  fp_batch_band_hits reads and resets the
 * batch's near-tie counts (as fp_band_hits).
 * fp_batch_capture records one run on the given buffers into a CUDA graph;
 * fp_batch_launch replays it on `stream` (same buffers, new contents).
 * The batch copies what it needs at creation and owns it; fp_batch_free
 * releases it (NULL is a no-op); fp_batch_last_error gives the text of the
 * batch's last failure.  Errors: fp_batch_create FP_ERR_INVALID_ARG (b NULL,
 * ninst < 1, NULL arrays, F < 0 or fields missing, a NULL, unset, 2D or
 * other-device handle, npts < 0, handles whose precision, tolerances or
 * max_newton differ, 2^31 points, elements or pairs or more), FP_ERR_OOM,
 * FP_ERR_CUDA; fp_batch_run / _tune / _capture FP_ERR_INVALID_ARG (NULL batch
 * or pointer), FP_ERR_CUDA; fp_batch_schedule FP_ERR_INVALID_ARG (NULL batch,
 * group out of range, a block size that is not a multiple of 32 up to 256, a
 * tile that is not a multiple of 32); fp_batch_groups /
 * fp_batch_group_info / fp_batch_profile / fp_batch_band_hits
 * FP_ERR_INVALID_ARG (NULL batch or pointer, group out of range),
 * FP_ERR_CUDA; fp_batch_launch FP_ERR_NOT_SETUP (nothing captured),
 * FP_ERR_CUDA. */
typedef struct fp_batch fp_batch;
fp_status fp_batch_create(fp_batch **b, int ninst, fp_handle *const *handles, const int64_t *npts,
                          int F, const double *const *fields, double pairs_per_point);
fp_status fp_batch_run(fp_batch *b, const double *pts, int32_t *code, int32_t *sub, int32_t *elem,
                       double *rst, double *dist2, double *out, void *stream);
fp_status fp_batch_tune(fp_batch *b, const double *pts, int32_t *code, int32_t *sub, int32_t *elem,
                        double *rst, double *dist2, double *out, void *stream, int reps,
                        double *best_ms);
fp_status fp_batch_schedule(fp_batch *b, int group, int *block, int *blocks_per_sm, int *tile);
fp_status fp_batch_groups(const fp_batch *b, int *ngroups);
/* Whether the groups' Newton and eval launches run concurrently on their
 * own streams (0) or one after another (1): *sequential = -1 reads the mode,
 * 0 or 1 sets it first (fp_batch_tune sets it to the faster).  Captured
 * graphs keep the mode they were captured with.  Errors: FP_ERR_INVALID_ARG
 * (NULL pointer, another value). */
fp_status fp_batch_mode(fp_batch *b, int *sequential);
fp_status fp_batch_group_info(fp_batch *b, int group, int *N, int64_t *E, int64_t *P, int64_t *pairs,
                              double *newton_ms, double *eval_ms);
fp_status fp_batch_profile(fp_batch *b, int enable);
fp_status fp_batch_band_hits(fp_batch *b, int64_t *counts);
fp_status fp_batch_capture(fp_batch *b, const double *pts, int32_t *code, int32_t *sub,
                           int32_t *elem, double *rst, double *dist2, double *out);
fp_status fp_batch_launch(fp_batch *b, void *stream);
const char *fp_batch_last_error(const fp_batch *b);
void fp_batch_free(fp_batch *b);

typedef struct fp_fields fp_fields;

/* Posted fields for the mixed form's evaluation.  fp_fields_create copies F
 * nodal fields [F][E][n3] (FP64, the handle's mesh) to the device as pairs of
 * floats (hi, lo) with hi + lo equal to the value to 48 bits (allocates;
 * enqueued on `stream`).  fp_eval_df interpolates them at located points like
 * fp_eval, but with double-float arithmetic on the FP32 pipes: exact leading
 * products, error-free two-sums, basis values computed in FP64 and split the
 * same way.  The result is rounded to FP64; its error is a few 2^-48 times
 * the sum of |f_ijk h_i h_j h_k| (measured against the FP64 oracle: below
 * 1e-13 of the field's largest nodal magnitude on the test meshes).  NaN
 * where code is NOT_FOUND or RETRY.  Allocates nothing. */
fp_status fp_fields_create(const fp_handle *h, int F, const double *fields, fp_fields **out,
                           void *stream);
void fp_fields_free(fp_fields *f);
fp_status fp_eval_df(fp_handle *h, const fp_fields *f, int64_t P, const int32_t *code,
                     const int32_t *elem, const double *rst, double *out, void *stream);

/* fp_find_eval / fp_find_eval_ws -- fp_find (or fp_find_ws) followed by the
 * interpolation of F fields, fused into the same launch sequence: after
 * classification each point's winning (point, element) pair is evaluated in
 * the element-sorted pair order of the Newton stage, so neighbouring threads
 * share an element's field rows.  Fields are either posted double-float
 * fields (`posted`, see fp_fields_create; F must equal its count) or FP64
 * fields [F][E][n3] (`fields`, 16-byte aligned for even n) when posted is
 * NULL.  out [F][P] FP64; NaN for points not found (or RETRY).  The other
 * arguments, outputs and errors are those of fp_find / fp_find_ws. */
fp_status fp_find_eval(fp_handle *h, int64_t P, const double *pts, const int32_t *qsess, int F,
                       const double *fields, const fp_fields *posted, int32_t *code, int32_t *sub,
                       int32_t *elem, double *rst, double *dist2, double *out, void *stream);
fp_status fp_find_eval_ws(fp_handle *h, fp_workspace *ws, int64_t P, const double *pts,
                          const int32_t *qsess, int F, const double *fields,
                          const fp_fields *posted, int32_t *code, int32_t *sub, int32_t *elem,
                          double *rst, double *dist2, double *out, void *stream);

/* Moving meshes (Sec. 1: donor elements are found again after every time
 * step when meshes move or deform).
 *
 * fp_update_coords -- replace the node coordinates of the handle's mesh (same
 * E, N, subdomain ids and options) and rebuild what depends on them: element
 * boxes, global box, hash grid and, in the mixed form, the element-local FP32
 * geometry.  A later fp_find gives exactly what fp_find on a new handle set
 * up with these coordinates gives.
 *   coords [3][E][n3] FP64, device or host memory; checked for non-finite
 *          values before the handle changes
 *   dist   [E][n3] new D^k field, or NULL to keep the current one (exact
 *          when every subdomain moves rigidly: D^k moves with its mesh)
 *   flags  0, or FP_UPDATE_DEFAULT_DIST to recompute the library's default D
 *          (only with dist == NULL; brute force, see fp_setup)
 * Work is enqueued on `stream` after what is already there; the call
 * synchronises `stream` twice (global box, hash size).  Scratch is kept in
 * the handle and only grows: an update whose hash grid fits the room of an
 * earlier one allocates nothing.  Objects that copied geometry at creation
 * (fp_bfaces, fp_batch) and CUDA graphs captured before the update must be
 * created or captured again.  Errors: FP_ERR_NOT_SETUP, FP_ERR_INVALID_ARG
 * (null or non-finite coords, bad flags; the handle is unchanged),
 * FP_ERR_OOM, FP_ERR_CUDA (the handle is then unusable until an update
 * succeeds).
 *
 * fp_find_warm -- fp_find (F == 0 and posted == NULL; out may be NULL) or
 * fp_find_eval with a warm start: warm_elem [P] and warm_rst [3][P] are each
 * point's element and reference coordinates from an earlier find (typically
 * the previous time step).  The candidate pair (p, warm_elem[p]), if the
 * screen keeps it, starts Newton from warm_rst[p] clamped to [-1,1]^3 instead
 * of the nearest GLL node; elem = -1 or a non-finite warm_rst means no warm
 * start for that point.  Only Newton's starting point changes, so INSIDE
 * results equal fp_find's up to the Newton tolerance (the root in an element
 * is unique); a BORDER point's clamped r is the local minimiser reached from
 * the start.  warm_elem / warm_rst may be the same buffers as elem / rst (the
 * warm values are read before the outputs are written).  Both NULL = cold
 * start.  Errors as fp_find / fp_find_eval. */
#define FP_UPDATE_DEFAULT_DIST 1
fp_status fp_update_coords(fp_handle *h, const double *coords, const double *dist, int flags,
                           void *stream);
fp_status fp_find_warm(fp_handle *h, int64_t P, const double *pts, const int32_t *qsess,
                       const int32_t *warm_elem, const double *warm_rst, int F,
                       const double *fields, const fp_fields *posted, int32_t *code,
                       int32_t *sub, int32_t *elem, double *rst, double *dist2, double *out,
                       void *stream);

/* fp_find_eval_host -- fp_find_eval (F == 0 and posted == NULL: fp_find) for
 * points and results in HOST memory.  The points are cut into chunks of
 * `chunk` points (<= 0: 2^22); while the device searches one chunk, a copy
 * stream brings the next one in and another takes the results of the
 * previous one out, so the copies overlap the search.  Two workspaces of
 * `chunk` points and `max_pairs` candidate pairs (<= 0: 4 * chunk) and two
 * sets of device buffers alternate; they are kept in the handle for later
 * calls (grown when a call asks for more) and freed with it.  A call sizes
 * its launches on the pairs per point of the previous call (any count is
 * still solved completely).  The searches never wait on the host; a chunk whose pairs overflowed its workspace has
 * its RETRY points searched again with fp_find_eval before the call
 * returns, so no FP_CODE_RETRY comes back.
 *   pts [3][P], qsess [P] or NULL: host memory (pinned memory copies fastest)
 *   fields / posted: device, as for fp_find_eval
 *   code, sub, elem [P], rst [3][P], dist2 [P], out [F][P]: host memory
 * Results are those of fp_find_eval on the same points.  The call waits for
 * its work (work queued earlier on `stream` runs first) and returns with
 * the host outputs complete.  Allocates on its first call and when it grows.
 * Hexahedral handles only.  Errors: FP_ERR_NOT_SETUP, FP_ERR_INVALID_ARG,
 * FP_ERR_OOM, FP_ERR_CUDA. */
fp_status fp_find_eval_host(fp_handle *h, int64_t P, const double *pts, const int32_t *qsess, int F,
                            const double *fields, const fp_fields *posted, int32_t *code,
                            int32_t *sub, int32_t *elem, double *rst, double *dist2, double *out,
                            int64_t chunk, int64_t max_pairs, void *stream);

/* Posted points: the split Lagrange basis values of P located points, for
 * repeated evaluation at the same (e, r) -- the interface points of a
 * Schwarz step are evaluated once per sub-iteration while the mesh stands
 * still (Sec. 2: kappa sub-iterations per step).
 * fp_points_create: room for P points of the handle's mesh (allocates;
 *   hexahedral handles).  fp_points_free: release (NULL is a no-op).
 * fp_points_set: compute and keep the basis values of the points
 *   code/elem/rst (as written by fp_find, rst [3][P]); call again after the
 *   points are found anew; the buffers stay where they are, so a graph that
 *   captured fp_eval_points stays valid.  Enqueued on `stream`.
 * fp_eval_points: out [F][P] = the posted double-float fields interpolated at
 *   the posted points, bit-identical to fp_eval_df at the same (e, r); NaN for
 *   points not found.  Allocates nothing, never waits.
 * The points belong to the handle they were made for and must be freed
 * before it.  Errors: fp_points_create FP_ERR_NOT_SETUP, FP_ERR_INVALID_ARG
 * (out NULL, P outside [0, 2^31), a 2D handle), FP_ERR_OOM, FP_ERR_CUDA;
 * fp_points_set and fp_eval_points FP_ERR_NOT_SETUP, FP_ERR_INVALID_ARG (NULL
 * pointers, points or fields made for another handle), FP_ERR_CUDA. */
typedef struct fp_points fp_points;
fp_status fp_points_create(const fp_handle *h, int64_t P, fp_points **out);
void fp_points_free(fp_points *q);
fp_status fp_points_set(fp_handle *h, fp_points *q, const int32_t *code, const int32_t *elem,
                        const double *rst, void *stream);
fp_status fp_eval_points(fp_handle *h, const fp_fields *f, const fp_points *q, double *out,
                         void *stream);

/* Mass-flux correction of interpolated interface velocity (Sec. 2.2,
 * Eqs. consv1, corr, consv2).
 * fp_bfaces_create: kind [E][6] int8 on the device marks faces of the
 * handle's mesh: 0 = not used, 1 = boundary face of the subdomain with
 * prescribed (Dirichlet) data, 2 = interface face whose data is
 * interpolated.  The marked faces are listed in (element, face) order; for
 * each, its (N+1)^2 GLL nodes (node (a,b) of face f numbered with a fastest
 * along the face's first reference direction: r-faces (s,t), s-faces (r,t),
 * t-faces (r,s)) get their position, outward unit normal and area weight
 * dA = w_a w_b |t_1 x t_2|.  Allocates; synchronises `stream`.
 * fp_bfaces_info: number of listed faces and of face nodes M.
 * fp_bfaces_nodes: copy positions [3][M], normals [3][M], dA [M], node kinds
 * [M] (int8) to device buffers (any may be NULL).  The interface nodes are
 * the query points for the interpolation of boundary data.
 * fp_flux_correct: u [3][M] velocity at the face nodes (prescribed or
 * interpolated); writes u_out [3][M] = u + gamma n on interface nodes and u
 * elsewhere, with gamma = -(sum u.n dA over all nodes) / (sum n.n dA over
 * interface nodes) (0 when there is no interface), so that the corrected flux
 * through the listed faces vanishes.  gamma and flux (before correction) are
 * written to device scalars if non-NULL.  Deterministic fixed-order sums;
 * allocates nothing; enqueued on `stream`.  Edge and corner nodes appear once
 * per face, each with its own face's normal.
 * The face set keeps a pointer to its handle (which must outlive it) and
 * owns its device arrays; fp_bfaces_free releases them (NULL is a no-op).
 * Errors: fp_bfaces_create FP_ERR_NOT_SETUP, FP_ERR_INVALID_ARG (out or kind
 * NULL, a 2D handle), FP_ERR_OOM, FP_ERR_CUDA; fp_bfaces_info,
 * fp_bfaces_nodes and fp_flux_correct FP_ERR_INVALID_ARG (NULL face set, or
 * u / u_out NULL), FP_ERR_CUDA. */
typedef struct fp_bfaces fp_bfaces;
fp_status fp_bfaces_create(const fp_handle *h, const int8_t *kind, fp_bfaces **out, void *stream);
void fp_bfaces_free(fp_bfaces *b);
fp_status fp_bfaces_info(const fp_bfaces *b, int64_t *nfaces, int64_t *nnodes);
fp_status fp_bfaces_nodes(const fp_bfaces *b, double *x, double *normal, double *dA, int8_t *kind,
                          void *stream);
fp_status fp_flux_correct(const fp_bfaces *b, const double *u, double *u_out, double *gamma,
                          double *flux, void *stream);
/* fp_bfaces_refresh: recompute positions, normals and weights of the listed
 * face nodes from the owner handle's current coordinates (after
 * fp_update_coords on a moving mesh); the face list, node kinds and the
 * interface numbering stay.  Allocates nothing; enqueued on `stream`.
 * Errors: FP_ERR_INVALID_ARG (b NULL), FP_ERR_NOT_SETUP (its handle freed),
 * FP_ERR_CUDA. */
fp_status fp_bfaces_refresh(fp_bfaces *b, void *stream);
/* fp_bfaces_sort_iface: renumber the interface nodes so that nodes with the
 * same donor element are consecutive.  elem [Mi] (device) holds each
 * interface node's donor element in the current numbering (as found at the
 * fp_bfaces_iface points; -1 = not found, placed last).  Afterwards
 * fp_bfaces_iface lists the points in the new order and
 * fp_flux_correct_iface reads u_iface in it.  Only the order changes: an
 * evaluation at the reordered points reads each element's field rows from
 * cache for neighbouring threads.  Nodes of one element keep an unspecified
 * order among themselves (results do not depend on it).  Allocates and
 * synchronises `stream`.  Errors: FP_ERR_INVALID_ARG (b or elem NULL),
 * FP_ERR_NOT_SETUP (its handle freed), FP_ERR_OOM, FP_ERR_CUDA. */
fp_status fp_bfaces_sort_iface(fp_bfaces *b, const int32_t *elem, void *stream);

/* Interface-data pipeline helpers.
 * fp_bfaces_iface: number of interface nodes Mi and (if pts != NULL) their
 * positions [3][Mi] in listing order -- the query points of the
 * interpolation of interface data.
 * fp_flux_correct_iface: fp_flux_correct with the velocity given as the
 * interpolated values at the interface nodes u_iface [3][Mi] (e.g. the
 * first three rows of an fp_eval output at the fp_bfaces_iface points) and
 * the prescribed values u_pres [3][M] (read at the other nodes only).
 * fp_extrapolate: out[i] = sum_{j=1..m} c_j hist[j-1][i] for i < len, the
 * order-m extrapolation in time of interface data over equal time steps from
 * the m newest values (hist: host array of m device pointers, newest first),
 * c = (1), (2,-1), (3,-3,1) for m = 1, 2, 3 (Sec. 2: lagged or extrapolated
 * boundary data, refined by kappa sub-iterations).  These calls allocate
 * nothing and never wait, so an eval + correction sub-iteration can be
 * captured in a CUDA graph and replayed kappa times.  Errors:
 * FP_ERR_INVALID_ARG (NULL face set or arrays; for fp_extrapolate m outside
 * 1..3, len < 0 or a NULL history pointer), FP_ERR_CUDA. */
fp_status fp_bfaces_iface(const fp_bfaces *b, int64_t *n_iface, double *pts, void *stream);
fp_status fp_flux_correct_iface(const fp_bfaces *b, const double *u_iface, const double *u_pres,
                                double *u_out, double *gamma, double *flux, void *stream);
fp_status fp_extrapolate(int m, int64_t len, const double *const *hist, double *out, void *stream);

/* Release every device resource of the handle (synchronises it first).
   NULL is a no-op. */
void fp_free(fp_handle *h);

/* Static text for a status code. */
const char *fp_error_string(fp_status s);

/* Text of the handle's most recent failure ("" if none); valid until the next
   call on the handle. */
const char *fp_last_error(const fp_handle *h);

/* Measurement support.  With fp_profile(h, 1) the library brackets its own
 * kernels with CUDA events recorded on the launching stream; fp_profile_read
 * waits for the recorded events of one kernel class and returns the summed
 * device time (ms) and number of timed launches since the previous read.
 * kind: 0 screen (hash + boxes + pair emission, with the offset scan),
 * 1 pair sort by element, 2 Newton, 3 classification / ownership, 4 eval. */
fp_status fp_profile(fp_handle *h, int enable);
fp_status fp_profile_read(fp_handle *h, int kind, double *total_ms, int64_t *launches);

/* Mixed form, while profiling is enabled: how many pairs took each Newton
 * path since the previous read -- counts[0] rejected after the FP32 phase
 * (converged away from the element), [1] FP32 phase not converged, [2]
 * finished by the compensated final steps, [3] sent to the full FP64
 * Newton.  Synchronises the device and resets the counters. */
fp_status fp_newton_paths(fp_handle *h, int64_t *counts);

/* Mixed form (Sec. 2.1 Newton solve, final steps at FP64 accuracy): the
 * number of compensated (double-float) residuals a pair may use in its final
 * steps before it is handed to the full FP64 Newton, 0..8 (3 after
 * fp_setup).  0 sends every pair whose FP32 phase converged near its element
 * to the full FP64 Newton: slower, with results within the same tolerance.
 * Applies to later fp_find / fp_find_eval / fp_find_static calls and to
 * batches created afterwards (all handles of a batch must agree).
 * Errors: FP_ERR_NOT_SETUP, FP_ERR_INVALID_ARG (out of range). */
fp_status fp_set_mixed_refine(fp_handle *h, int max_residuals);

/* Fused evaluation of posted (double-float) fields (Sec. 2.1 findpts_eval):
 * with enable != 0, each block copies the fields of every element its 128
 * sorted (point, element) pairs touch into shared memory once and reads the
 * rows from there; with 0 (after fp_setup) the rows are read through L1,
 * where the threads of one element share them.  Results are identical either
 * way; elements whose F fields exceed 48 KB are always read through L1.
 * Applies to later fp_find_eval / fp_find_eval_ws / fp_find_warm calls with
 * posted fields.  Errors: FP_ERR_NOT_SETUP. */
fp_status fp_set_eval_staging(fp_handle *h, int enable);

/* Device bytes the handle holds: *resident = the posted mesh and its search
 * structures (coordinates and their FP32 copies, boxes, hash grid, distance
 * field, per-element sort arrays); *workspace = the handle's own fp_find
 * workspace as grown so far (either pointer may be NULL; allocator rounding
 * not included).  Errors: FP_ERR_NOT_SETUP. */
fp_status fp_memory(const fp_handle *h, int64_t *resident, int64_t *workspace);

/* Near-tie ("band") hits of the classification since the previous read
 * (Sec. 2.1 decides INSIDE / BORDER by residual thresholds and the owner by
 * comparing interpolated distances; where two of those numbers lie close
 * together, ids could depend on rounding).  Counted on every find, workspace
 * and static call of the handle, one count per point and kind:
 *   counts[0]  a candidate's residual within a factor 2 of tol_accept*h_e
 *   counts[1]  no INSIDE element, and a candidate's residual within a factor
 *              2 of tol_border*h_e, or two BORDER candidates within
 *              tie_band*L of the smallest residual
 *   counts[2]  two subdomains' interpolated D^k within 2*tie_band*L of the
 *              largest (the lower-id rule decided the owner, or nearly did)
 * Synchronises the device and resets the counters.  Errors:
 * FP_ERR_NOT_SETUP, FP_ERR_INVALID_ARG (counts NULL), FP_ERR_CUDA. */
fp_status fp_band_hits(fp_handle *h, int64_t *counts);

/* Arithmetic peak probes (measurement support; the paper has no
 * counterpart).  The location stage is bound by arithmetic, so its roofline
 * needs this GPU's multiply-add rates.  fp_fma_probe enqueues one launch of
 * blocks_per_sm (1..8) blocks of 256 threads per SM; every thread runs 8
 * independent chains of `iters` dependent steps:
 *   kind 0  FP64 fma             kind 1  FP32 fma
 *   kind 2  double-float multiply-add on the FP32 pipes (the operation the
 *           mixed form uses for its FP64-accuracy residuals and eval)
 *   kind 3  packed FP32 pair fma (two lanes of a float2 per instruction)
 *   kind 4  two double-float multiply-adds in packed FP32 pairs
 * and stores one double per thread to `sink` (device, fp_probe_threads()
 * doubles).  *flops (may be NULL) receives the launch's flop count (2 per
 * fma, 4 per packed pair fma; a double-float step counts as one FP64-class
 * multiply-add).  Time it with events on `stream`.  Errors:
 * FP_ERR_INVALID_ARG (kind outside 0..4,
 * iters < 1, blocks_per_sm outside 1..8, sink NULL), FP_ERR_CUDA.
 * fp_probe_threads returns the threads of one launch (-1 on a CUDA error). */
fp_status fp_fma_probe(int kind, int64_t iters, int blocks_per_sm, double *sink, double *flops,
                       void *stream);
int64_t fp_probe_threads(int blocks_per_sm);

/* Number of kernels the library has launched in this process. */
int64_t fp_launch_count(void);

/* Number of (point, candidate element) pairs that survived the box screen in
   the handle's most recent fp_find (each pair gets one Newton solve). */
fp_status fp_last_find_stats(const fp_handle *h, int64_t *npairs);

/* Introspection for tests: E, N, number of hash cells, number of
   cell -> element entries, number of subdomains. */
fp_status fp_info(const fp_handle *h, int64_t *E, int *N, int64_t *ncell, int64_t *nnz,
                  int *nsub);

/* Introspection for tests: copy the per-element axis boxes [E][6]
   (xmin,ymin,zmin,xmax,ymax,zmax, padded) and the hash grid to DEVICE
   buffers.  grid[9] = origin xyz, inverse cell size xyz, dims xyz (as
   doubles); cell_start [ncell+1] and cell_elems [nnz] int32.  Any output may
   be NULL.  Enqueued on `stream`. */
fp_status fp_debug_boxes(const fp_handle *h, double *aabb, double *grid,
                         int32_t *cell_start, int32_t *cell_elems, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* FINDPTS_GB_H */
