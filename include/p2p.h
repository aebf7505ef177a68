/*
 * p2p.h -- C ABI of the GB300 near-field P2P library (libp2p.so).
 *
 * The near-field (P2P) operator of MLFMA (Sec. 1: A = A_near + A_far; the
 * near part is evaluated directly): for every target point x_i,
 *
 *     out_i = sum over sources y_j in the leaf box of x_i and in the (up to 26)
 *             leaf boxes adjacent to it, r_ij = |x_i - y_j| > 0, of G(r_ij) lambda_j
 *
 * with G(r) = exp(i k r) / (4 pi r) (Helmholtz) or 1 / (4 pi r) (Laplace).
 * Sources and targets are one point set, as in the paper's symmetric setup
 * (Sec. 3.1).  Leaf boxes form a uniform grid of ng^3 cubes of edge h starting
 * at lo; boxes are numbered in Morton order over the non-empty boxes only
 * (Sec. 3.2 stores box data "in the order of the box's Morton index").
 *
 * Two source layouts are offered (Sec. 3.2 "indexing", Sec. 3.3 "repetition"):
 *   P2P_LAYOUT_INDEXED    every box reads its neighbours' sources through the
 *                         neighbour lists from one box-sorted point array;
 *   P2P_LAYOUT_REDUNDANT  every box owns a contiguous copy of all sources of its
 *                         neighbourhood (the redundancy of Sec. 3.3, kept per box
 *                         rather than per target), so each thread block reads one
 *                         contiguous tile independent of all others.
 *   P2P_LAYOUT_SYMMETRIC  the indexed gather over half of each neighbourhood: a box
 *                         lists its own sources and those of its neighbours with a
 *                         higher id, and every pair of points in different boxes is
 *                         evaluated once and added to both ends (G(x, y) = G(y, x)).
 *                         Same results, about half the kernel evaluations; results
 *                         are accumulated with atomics.  p2p_grad_points needs an
 *                         indexed or redundant plan.
 *   P2P_LAYOUT_REPETITION the paper's own repetition layout (Sec. 3.3, eq. 8 - 9):
 *                         every TARGET owns one contiguous record -- its coordinates,
 *                         then a copy of every source of its box's neighbourhood --
 *                         and one thread evaluates one target by reading its record
 *                         front to back; the strengths are repacked into the records
 *                         at every apply.  Records are not padded to 27 CT entries
 *                         (each is 1 + S_b long, offsets kept per target).  One
 *                         point set, max_nrhs 1; see p2p_repetition_records for the
 *                         workspace.  Other calls on such a plan (batched launch,
 *                         coordinate gradient) run on its indexed lists.
 *
 * Conventions shared by every entry point
 *   - Memory.  Pointers marked [dev] are CUDA device pointers, [host] are host
 *     pointers.  The caller allocates and owns every buffer, including the
 *     workspaces whose sizes the *_workspace_size queries return.  The library
 *     never frees caller memory.  A plan stores pointers to the arrays it was
 *     created from; they must stay valid and unchanged for the plan's lifetime.
 *   - Streams.  Every call enqueues its work on `stream` (a cudaStream_t; NULL
 *     is the legacy default stream) and returns without waiting, except where a
 *     call says it synchronises (it then waits for `stream` only).
 *   - Point order.  Coordinates, strengths, results and gradients are in the
 *     caller's original point order.  perm maps sorted position -> original index.
 *   - Complex numbers are two consecutive floats (re, im) (C99 float complex,
 *     CUDA float2); a complex array of n rows and nrhs columns with leading
 *     dimension ld stores element (i, q) at index i*ld + q, ld >= nrhs.
 *   - Errors.  Every call returns a p2p_status and never throws or aborts.
 *     Invalid arguments return P2P_ERR_INVALID before any work is enqueued.  A
 *     CUDA launch or runtime failure returns P2P_ERR_CUDA; p2p_last_error_string
 *     gives the CUDA message.  Anomalies detected inside kernels (a bounded wait
 *     that ran out, an out-of-range index in the input structure) set a device
 *     status word that p2p_last_async_status reads.
 */
#ifndef P2P_H
#define P2P_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define P2P_API __attribute__((visibility("default")))
#else
#define P2P_API
#endif

typedef struct CUstream_st* p2p_stream_t; /* same type as cudaStream_t */

typedef enum {
    P2P_OK = 0,
    P2P_ERR_INVALID = 1,     /* bad argument, size, pointer alignment or input value */
    P2P_ERR_WORKSPACE = 2,   /* workspace smaller than the size query returned */
    P2P_ERR_CUDA = 3,        /* a CUDA call failed; see p2p_last_error_string */
    P2P_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out */
    P2P_ERR_UNSUPPORTED = 5, /* valid request that this build/device does not support */
    P2P_ERR_ALLOC = 6,       /* host memory for the plan object could not be allocated */
    P2P_ERR_STALE = 7        /* new coordinates move a point out of its leaf box: rebuild the plan */
} p2p_status;

typedef enum { P2P_HELMHOLTZ = 0, P2P_LAPLACE = 1 } p2p_kernel;

typedef enum {
    P2P_LAYOUT_INDEXED = 0,
    P2P_LAYOUT_REDUNDANT = 1,
    P2P_LAYOUT_SYMMETRIC = 2,
    P2P_LAYOUT_REPETITION = 3
} p2p_layout;

/* Evaluation path of p2p_apply_path (the plain p2p_apply picks P2P_PATH_AUTO). */
typedef enum {
    P2P_PATH_AUTO = 0,        /* FP32 shared-G for nrhs < 16, tensor-core path otherwise (when available) */
    P2P_PATH_FP32_PER_RHS = 1,/* FP32; G re-evaluated for every right-hand side */
    P2P_PATH_FP32_SHARED = 2, /* FP32; each G evaluated once and applied to up to 4 RHS at a time */
    P2P_PATH_TC_BF16X3 = 3,   /* G tile and strengths split into BF16 hi + lo, 3 tcgen05 MMAs per 16
                                 sources, FP32 accumulation in tensor memory; plans with max_nrhs >= 16
                                 on an sm_103 device, else P2P_ERR_UNSUPPORTED */
    P2P_PATH_TC_BF16X6 = 4    /* as P2P_PATH_TC_BF16X3 with three BF16 parts (hi + mid + lo, ~24 bits)
                                 and the 6 MMAs whose part products are not below 2^-24 of the term:
                                 FP32-level accuracy on the tensor cores, same availability */
} p2p_path;

/* Launch tuning of a plan (the autotuner's knobs).  Zero fields take defaults.  With
 * chunk and warps_per_cta both zero (or a NULL tuning) the plan chooses them: 192
 * sources per item and 8 warps per block, or 256 and 6 when more than half of the
 * boxes' source lists hold 193 .. 256 sources (a 192-source item would leave each of
 * them a short tail item of the same fixed cost), or 128 and 8 when the plan would
 * have fewer than 2.5 items per resident warp (16 warps per SM; the last items
 * would leave most warps idle).  The workspace size covers all three.
 *
 * warp_boxes selects the kernel of one-right-hand-side FP32 applies.  The staged
 * pipeline stages chunks of a box's source list in shared memory and suits boxes
 * of many targets; the direct kernel gives each warp 1, 2, 4, 8, 16 or 32 whole
 * boxes (32 / warp_boxes lanes each) and reads the sources through the L1, which
 * suits sparse boxes (a few targets each), where a staged item carries too little
 * work for its fixed cost.  0: the plan decides from its mean box occupancy D (the
 * direct kernel with 32, 16, 8 or 4 boxes per warp up to D = 1.3, 2.5, 6 and 12,
 * the box-group kernel for 12 < D <= 24 on the indexed layout, the staged pipeline
 * above); -1: the staged pipeline; 1 .. 32: the direct kernel with that many boxes
 * per warp; -2 (indexed layout only): the box-group
 * kernel, in which groups of 16 consecutive target boxes stage the union of their
 * neighbourhoods in shared memory once and every box sweeps its own neighbour
 * boxes inside it (a plan whose largest union exceeds 8 192 sources, or of another
 * layout, runs the staged pipeline instead and reports -1).
 * Multi-RHS applies, the symmetric layout and the batched launch always use the
 * staged pipeline. */
typedef struct {
    int32_t chunk;         /* sources staged per work item, multiple of 32, 32..1024 (default 192) */
    int32_t warps_per_cta; /* warps per thread block of the pair kernel, 1..16 (default 8) */
    int32_t target_group;  /* targets swept per pass, multiple of 32, 32..128 (default 32) */
    int32_t warp_boxes;    /* 0 (plan decides), -1 (staged pipeline), 1, 2, 4, 8, 16 or 32 (direct kernel),
                              -2 (box-group kernel) */
} p2p_tuning;

typedef struct p2p_plan p2p_plan;

/* ------------------------------------------------------------ messages --- */

/* Static description of a status code. */
P2P_API const char* p2p_status_string(p2p_status status);

/* Message of the last CUDA failure seen by this thread ("" if none). */
P2P_API const char* p2p_last_error_string(void);

/* Library version as major*10000 + minor*100 + patch. */
P2P_API int32_t p2p_version(void);

/* ------------------------------------------------------- leaf binning --- */
/*
 * Sec. 3.1 (points assigned to the boxes of the last tree level) and Sec. 3.2
 * (box data in Morton order).  For every point, per axis
 *     cell = clamp(floor((double(x) - lo) / h), 0, ng - 1)
 * computed as one IEEE double subtraction and one double division (so the
 * result equals a host computation bit for bit); the Morton key interleaves
 * the cell bits with x at bit 0, y at bit 1, z at bit 2 of every triple.  A
 * point on a face between cells belongs to the upper cell; points outside the
 * grid are clamped into the boundary boxes.  Points are stably sorted by key
 * (ties keep the original order) and run-length encoded into boxes.
 *
 *   pts        [dev]  n x 3 float, xyz of each point (row-major, 4-byte aligned)
 *   n                 number of points, 0 <= n < 2^31 - 1
 *   lo         [host] 3 doubles, grid origin
 *   h                 leaf box edge, > 0 and finite
 *   ng                boxes per axis, 1 <= ng <= 2^21
 *   perm       [dev]  out, n int32: perm[s] = original index of the s-th sorted point
 *   point_box  [dev]  out, n int32: box id of each original point
 *   box_keys   [dev]  out, capacity n int64: Morton key of each box (ascending)
 *   box_ptr    [dev]  out, capacity n + 1 int32: box b holds sorted points box_ptr[b] .. box_ptr[b+1]-1
 *   num_boxes  [host] out, number of non-empty boxes
 *   work       [dev]  scratch of at least p2p_bin_workspace_size(n) bytes, 256-byte aligned
 *
 * Synchronises: waits for `stream` to read back num_boxes and the input check.
 * Returns P2P_ERR_INVALID if a coordinate is NaN or infinite (outputs are then
 * undefined).
 */
P2P_API p2p_status p2p_bin_workspace_size(int64_t n, size_t* bytes);
P2P_API p2p_status p2p_bin_points(const float* pts, int64_t n, const double lo[3], double h, int32_t ng,
                                  int32_t* perm, int32_t* point_box, int64_t* box_keys, int32_t* box_ptr,
                                  int32_t* num_boxes, void* work, size_t work_bytes, p2p_stream_t stream);

/*
 * Allocation-free variant of p2p_bin_points.  The paper has no counterpart;
 * this entry point exists for callers that cannot allocate device memory when
 * they bin points: real-time or embedded hosts that fix their device memory
 * budget up front and refuse allocations afterwards, and plug-ins whose host
 * application owns every allocation and forbids device allocations from inside
 * a callback.
 *
 * Inputs, outputs and results are those of p2p_bin_points; there is no work
 * argument.  The scratch lives in one fixed device array inside the library,
 * sized for at most P2P_BIN_STATIC_MAX_POINTS points (about 2 MiB); every GPU
 * that loads the library keeps that array until the process exits.  n above
 * the maximum returns P2P_ERR_INVALID without touching the device.  The call
 * performs no cudaMalloc, cudaFree or other allocation.
 *
 * The first call on a device looks up the array's device address (with that
 * device current) and keeps it; make that first call before any stream
 * capture begins.  The kept address belongs to the device's current context:
 * after cudaDeviceReset (or any other teardown of the primary context) it is
 * stale, and the next call must not be made in that process.  All calls on a
 * device share the array, which keeps the previous call's contents (the call
 * clears what it needs zeroed): calls that overlap on the GPU -- on different
 * streams, or from different host threads on the same device -- race on it and
 * must be serialised by the caller.  Like p2p_bin_points, the call
 * synchronises `stream` before it returns (it reads the box count back).
 */
#define P2P_BIN_STATIC_MAX_POINTS 65536
P2P_API p2p_status p2p_bin_points_static(const float* pts, int64_t n, const double lo[3], double h, int32_t ng,
                                         int32_t* perm, int32_t* point_box, int64_t* box_keys, int32_t* box_ptr,
                                         int32_t* num_boxes, p2p_stream_t stream);

/* ---------------------------------------------------- neighbour lists --- */
/*
 * Sec. 3.2 (the per-box list of neighbouring sources and its "second order
 * index") with the 9 adjacent boxes of the paper's 2D quadtree replaced by
 * the 27 boxes of a 3D grid: the neighbours of box b are the non-empty boxes
 * whose cells lie within Chebyshev distance 1 of b's cell, b itself included,
 * with no periodic wrap, listed in ascending box id.
 *
 *   box_keys   [dev]  num_boxes int64 from p2p_bin_points (strictly ascending)
 *   box_ptr    [dev]  num_boxes + 1 int32 from p2p_bin_points
 *   num_boxes, ng     as returned / passed to p2p_bin_points
 *   nbr_ptr    [dev]  out, num_boxes + 1 int32 (CSR row pointer)
 *   nbr_idx    [dev]  out, capacity 27 * num_boxes int32 (CSR column indices)
 *   nnz        [host] out, number of (box, neighbour) entries = nbr_ptr[num_boxes]
 *   sources    [host] out, sum over boxes of the number of sources in the
 *                     box's neighbourhood (the size of the redundant layout)
 *   work       [dev]  scratch of at least p2p_neighbors_workspace_size bytes
 *
 * Synchronises to read back nnz and sources.
 */
P2P_API p2p_status p2p_neighbors_workspace_size(int32_t num_boxes, size_t* bytes);
P2P_API p2p_status p2p_build_neighbors(const int64_t* box_keys, const int32_t* box_ptr, int32_t num_boxes,
                                       int32_t ng, int32_t* nbr_ptr, int32_t* nbr_idx, int64_t* nnz,
                                       int64_t* sources, void* work, size_t work_bytes, p2p_stream_t stream);

/*
 * Neighbour lists between two point sets binned on the same grid (targets and
 * sources kept as separate arrays, as the paper's tree object does, Sec. 3.1):
 * for target box b, the non-empty SOURCE boxes whose cells lie within
 * Chebyshev distance 1 of b's cell, in ascending source box id, and the
 * position in that list of the source box of b's own cell (the only sources
 * that can coincide with one of b's targets), or -1 if that cell holds no
 * source.
 *
 *   tgt_keys, num_tgt_boxes  [dev] target box keys from p2p_bin_points on the targets (strictly ascending)
 *   src_keys, src_box_ptr    [dev] source box keys and box pointers from p2p_bin_points on the sources
 *   num_src_boxes, ng              as returned / passed to the two p2p_bin_points calls (same lo, h, ng)
 *   nbr_ptr    [dev]  out, num_tgt_boxes + 1 int32
 *   nbr_idx    [dev]  out, capacity 27 * num_tgt_boxes int32 (source box ids)
 *   nbr_self   [dev]  out, num_tgt_boxes int32
 *   nnz, sources [host] out, entries of the lists and the total of their source counts
 *   work       [dev]  scratch of at least p2p_neighbors_workspace_size(num_tgt_boxes) bytes
 *
 * Synchronises to read back nnz and sources.
 */
P2P_API p2p_status p2p_build_neighbors_st(const int64_t* tgt_keys, int32_t num_tgt_boxes, const int64_t* src_keys,
                                          const int32_t* src_box_ptr, int32_t num_src_boxes, int32_t ng,
                                          int32_t* nbr_ptr, int32_t* nbr_idx, int32_t* nbr_self, int64_t* nnz,
                                          int64_t* sources, void* work, size_t work_bytes, p2p_stream_t stream);

/* ------------------------------------------------------------- plans --- */
/*
 * A plan binds one point set and its box structure to a kernel, a wavenumber,
 * a source layout and launch tuning, and lays the device data out for the
 * apply calls: box-sorted coordinates, the work-item list (target group x
 * source chunk of one box), and for P2P_LAYOUT_REDUNDANT the per-box packed
 * copy of the neighbourhood's source coordinates (the data collection of Sec.
 * 3.3, eq. 6 - 8, done on the device).
 *
 *   pts                    [dev] n x 3 float (the array given to p2p_bin_points)
 *   perm, box_ptr          [dev] from p2p_bin_points
 *   nbr_ptr, nbr_idx       [dev] from p2p_build_neighbors
 *   nnz, sources                 from p2p_build_neighbors
 *   kernel, k                    Green's function and wavenumber (k finite; ignored for Laplace)
 *   layout                       source layout
 *   max_nrhs                     largest nrhs any apply on this plan will use, 1..256; from 16 up
 *                                the workspace also holds the tensor-core path's per-box group lists
 *                                and its strength records, (n / 16 + num_boxes) x
 *                                (ceil(max_nrhs / 64) x 8192 + 256) bytes
 *   tuning                 [host] NULL for defaults
 *   workspace              [dev] at least p2p_plan_workspace_size bytes, 256-byte aligned;
 *                                owned by the caller, must outlive the plan
 *
 * Synchronises to read back the number of work items.  The plan object
 * itself is host memory released by p2p_plan_destroy.
 */
P2P_API p2p_status p2p_plan_workspace_size(int64_t n, int32_t num_boxes, int64_t nnz, int64_t sources,
                                           p2p_layout layout, int32_t max_nrhs, const p2p_tuning* tuning,
                                           size_t* bytes);

/*
 * Size of the per-target records of P2P_LAYOUT_REPETITION: records = sum over
 * boxes b of n_b (1 + S_b) entries (the paper's memory estimate, eq. 8, without
 * its padding), computed from the box pointers and neighbour lists of
 * p2p_bin_points / p2p_build_neighbors (copied to the host; synchronises).
 * p2p_plan_workspace_size_rep gives the workspace of such a plan; records must
 * stay below 2^31.
 */
P2P_API p2p_status p2p_repetition_records(const int32_t* box_ptr, int32_t num_boxes, const int32_t* nbr_ptr,
                                          const int32_t* nbr_idx, int64_t* records, p2p_stream_t stream);
P2P_API p2p_status p2p_plan_workspace_size_rep(int64_t n, int32_t num_boxes, int64_t nnz, int64_t sources,
                                               int64_t records, const p2p_tuning* tuning, size_t* bytes);
P2P_API p2p_status p2p_plan_create(p2p_plan** plan, const float* pts, int64_t n, const int32_t* perm,
                                   const int32_t* box_ptr, int32_t num_boxes, const int32_t* nbr_ptr,
                                   const int32_t* nbr_idx, int64_t nnz, int64_t sources, p2p_kernel kernel,
                                   float k, p2p_layout layout, int32_t max_nrhs, const p2p_tuning* tuning,
                                   void* workspace, size_t workspace_bytes, p2p_stream_t stream);

/*
 * A plan between two point sets: out (n_tgt rows) = A lambda (n_src rows), the
 * near-field operator from the sources to the targets, with the target boxes,
 * source boxes and lists of p2p_bin_points (once per set, same lo, h and ng)
 * and p2p_build_neighbors_st.  A target and a source at the same position
 * (r = 0) are skipped.  Layouts INDEXED and REDUNDANT (SYMMETRIC returns
 * P2P_ERR_UNSUPPORTED); every apply path, the batched launch and the host-buffer
 * apply take such plans, with strengths of n_src rows and results of n_tgt rows.
 * p2p_apply_adjoint and p2p_grad_points return P2P_ERR_UNSUPPORTED: the adjoint
 * A^H g (n_src rows) is the plan with the two sets exchanged applied with
 * adjoint = 1 in p2p_apply_path, since G(x, y) = G(y, x) (p2p_apply_path with
 * adjoint = 1 on a two-set plan computes conj(A) lambda).  The tensor-core
 * workspace term counts n_src / 16 + num_src_boxes groups.  Other arguments as
 * for p2p_plan_create.
 */
P2P_API p2p_status p2p_plan_workspace_size_st(int64_t n_tgt, int32_t num_tgt_boxes, int64_t n_src,
                                              int32_t num_src_boxes, int64_t nnz, int64_t sources, p2p_layout layout,
                                              int32_t max_nrhs, const p2p_tuning* tuning, size_t* bytes);
P2P_API p2p_status p2p_plan_create_st(p2p_plan** plan, const float* tgt_pts, int64_t n_tgt, const int32_t* tgt_perm,
                                      const int32_t* tgt_box_ptr, int32_t num_tgt_boxes, const float* src_pts,
                                      int64_t n_src, const int32_t* src_perm, const int32_t* src_box_ptr,
                                      int32_t num_src_boxes, const int32_t* nbr_ptr, const int32_t* nbr_idx,
                                      const int32_t* nbr_self, int64_t nnz, int64_t sources, p2p_kernel kernel,
                                      float k, p2p_layout layout, int32_t max_nrhs, const p2p_tuning* tuning,
                                      void* workspace, size_t workspace_bytes, p2p_stream_t stream);

P2P_API p2p_status p2p_plan_destroy(p2p_plan* plan);

/*
 * New coordinates for the points of a one-set plan whose box structure stays
 * valid: every point must lie in the same leaf box (the same grid cell under
 * lo, h, ng, the grid the structure was binned on) as the coordinates the plan
 * holds now.  A shape-optimisation step that moves points by less than their
 * distance to the box faces keeps the binning, the neighbour lists and the work
 * items; only the box-sorted coordinates (and, for the redundant layout, the
 * per-box copies of Sec. 3.3) are gathered again.
 *
 *   pts        [dev] n x 3 float, the new coordinates in original point order
 *   lo, h, ng        the grid passed to p2p_bin_points for this plan
 *   moved      [host] out (may be NULL): points whose cell would change
 *
 * Returns P2P_ERR_STALE, leaving the plan unchanged, if any point would change
 * cell (rebuild the structure and the plan from the new coordinates);
 * P2P_ERR_INVALID for a non-finite coordinate; P2P_ERR_UNSUPPORTED for a
 * two-set plan.  On success the plan reads its coordinates from `pts` from now
 * on (the previous array may be released).  Synchronises.
 */
P2P_API p2p_status p2p_plan_update_points(p2p_plan* plan, const float* pts, const double lo[3], double h, int32_t ng,
                                          int64_t* moved, p2p_stream_t stream);

/* Number of work items, ordered (target, source) pairs with r > 0 are not
 * counted here; see p2p_plan_pair_count. */
P2P_API p2p_status p2p_plan_info(const p2p_plan* plan, int64_t* n, int32_t* num_boxes, int64_t* sources,
                                 int64_t* work_items, p2p_layout* layout, p2p_tuning* tuning);

/* Number of ordered (target, source) pairs in the neighbourhoods with r > 0
 * (the work of one apply per right-hand side).  Synchronises. */
P2P_API p2p_status p2p_plan_pair_count(const p2p_plan* plan, int64_t* pairs, p2p_stream_t stream);

/* ------------------------------------------------------------- apply --- */
/*
 * out = A lambda (p2p_apply), out = A^H g (p2p_apply_adjoint).  A is complex
 * symmetric (G(x, y) = G(y, x) and the neighbour relation is symmetric), so
 * A^H = conj(A): the adjoint uses exp(-i k r) / (4 pi r).  This is the
 * gradient dL/dlambda of a real loss whose gradient with respect to out is g
 * (convention dL/dRe + i dL/dIm).
 *
 *   lambda, g  [dev] n x nrhs complex64, leading dimension ld, 8-byte aligned
 *   out        [dev] n x nrhs complex64, leading dimension ld; fully overwritten
 *                    in its first nrhs columns, other columns untouched
 *   nrhs             1 .. the plan's max_nrhs
 *
 * lambda and out must not overlap.  Calls on one plan must not overlap in
 * time (they share the plan's staging buffers): issue them on one stream.
 */
P2P_API p2p_status p2p_apply(const p2p_plan* plan, const void* lambda, void* out, int32_t nrhs, int64_t ld,
                             p2p_stream_t stream);
P2P_API p2p_status p2p_apply_adjoint(const p2p_plan* plan, const void* g, void* out, int32_t nrhs, int64_t ld,
                                     p2p_stream_t stream);

/* p2p_apply / p2p_apply_adjoint with an explicit evaluation path. */
P2P_API p2p_status p2p_apply_path(const p2p_plan* plan, const void* lambda, void* out, int32_t nrhs, int64_t ld,
                                  int32_t adjoint, p2p_path path, p2p_stream_t stream);

/*
 * The two phases of p2p_apply_path, for callers that overlap or time them
 * separately.  p2p_apply_stage gathers lambda into the plan's staging buffer
 * in the order the chosen path reads it (box-sorted rows, or the per-box
 * packed rows of the redundant layout, Sec. 3.3; for the tensor-core path, the
 * BF16 hi/lo record of every 16-source group); p2p_apply_staged then runs the
 * pair kernel (or the tensor-core kernel) on the staged strengths and writes
 * out.  Both must be given the same nrhs and path; no other call on the plan
 * may come between them.  The arguments mean what they mean for
 * p2p_apply_path.
 */
P2P_API p2p_status p2p_apply_stage(const p2p_plan* plan, const void* lambda, int32_t nrhs, int64_t ld, p2p_path path,
                                   p2p_stream_t stream);
P2P_API p2p_status p2p_apply_staged(const p2p_plan* plan, void* out, int32_t nrhs, int64_t ld, int32_t adjoint,
                                    p2p_path path, p2p_stream_t stream);

/*
 * Gradient with respect to the point coordinates of a real loss L whose
 * gradient with respect to out = A lambda is g, box membership held fixed:
 *
 *   dL/dx_m = sum_{j in nbr(m), r > 0} sum_q Re[G'(r) (conj(g_mq) lambda_jq + conj(g_jq) lambda_mq)] (x_m - x_j) / r
 *
 * with G'(r) = exp(ikr)(ikr - 1)/(4 pi r^2) (Helmholtz) or -1/(4 pi r^2) (Laplace).
 *
 *   lambda, g  [dev] n x nrhs complex64, leading dimension ld
 *   grad       [dev] out, n x 3 float, overwritten
 */
P2P_API p2p_status p2p_grad_points(const p2p_plan* plan, const void* lambda, const void* g, float* grad,
                                   int32_t nrhs, int64_t ld, p2p_stream_t stream);

/*
 * Guarded apply: p2p_apply_path with every result within a relative tolerance
 * of the exact sum (an FP64 final evaluation wherever the FP32 result's error
 * could exceed the tolerance, decided per target).  An evaluation whose terms G lambda are
 * each accurate to a relative delta has |out_i - exact_i| <= delta S_i with
 * S_i = sum_j |G(r_ij) lambda_j|; the call computes S (a Laplace sweep over
 * |lambda|), flags every target with delta S_i > tol |out_i| for some right-hand
 * side (the sums that cancel: S_i / |out_i| large), and re-evaluates the flagged
 * targets in FP64 on the GPU (their whole neighbourhood, every right-hand side),
 * overwriting their FP32 results.  delta: 2^-20 for the FP32 paths and
 * P2P_PATH_TC_BF16X6, 2^-14 for P2P_PATH_TC_BF16X3; path AUTO takes the FP32
 * path for nrhs < 16 or without tensor-core support, else P2P_PATH_TC_BF16X3
 * when 32 * 2^-14 <= tol and P2P_PATH_TC_BF16X6 below.  For strengths with random phases most targets have
 * S_i / |out_i| of 10 - 30, so tol = 1e-6 re-evaluates most of them; tol = 1e-4
 * picks out the strongly cancelling ones.
 *
 *   tol          relative tolerance per target and right-hand side, >= 0
 *   work   [dev] at least p2p_apply_guarded_workspace_size bytes, 256-byte aligned
 *   refined [host] out (may be NULL): targets re-evaluated in FP64
 *
 * Other arguments as for p2p_apply_path.  Not for symmetric-layout plans
 * (P2P_ERR_UNSUPPORTED).  Synchronises once (to read the number of flagged
 * targets).
 */
P2P_API p2p_status p2p_apply_guarded_workspace_size(const p2p_plan* plan, int32_t nrhs, size_t* bytes);
P2P_API p2p_status p2p_apply_guarded(const p2p_plan* plan, const void* lambda, void* out, int32_t nrhs, int64_t ld,
                                     int32_t adjoint, p2p_path path, double tol, void* work, size_t work_bytes,
                                     int64_t* refined, p2p_stream_t stream);

/* ----------------------------------------------------- batched apply --- */
/*
 * Several independent geometries (plans) applied in one persistent launch.
 * The paper splits large problems into pieces of 50k - 150k points to keep its
 * repetition kernel near its optimum (Sec. 4.3); a batch runs such pieces, or
 * unrelated geometries of uneven box occupancy, together: the plans' work items
 * (each plan's own list, heaviest first) form one queue, plan after plan in the
 * order given, and warp w of a persistent grid of W warps takes items w, w + W, ...
 * Giving the plans from smallest to largest leaves the tail to the largest
 * geometry's lightest items.
 *
 *   plans           [host] count plan pointers, 1 <= count <= 16; the plans must
 *                          outlive the batch and are applied with nrhs columns
 *   nrhs                   1 .. min over plans of max_nrhs
 *   warps_per_cta          0 (default 8) or 1 .. 16
 *   workspace       [dev]  at least p2p_batch_workspace_size bytes, 256-byte aligned
 *
 * p2p_batch_create synchronises once (it builds the work queue on the device).
 * p2p_batch_apply takes host arrays of count device pointers: lambdas[g] and
 * outs[g] are plan g's n_g x nrhs complex64 strengths and results, leading
 * dimension ld (same for all).  It enqueues two kernels and no allocation or
 * synchronisation, so it may be captured in a CUDA graph;
 * p2p_batch_graph_create does exactly that for fixed buffers (the graph reads
 * lambdas and writes outs every time p2p_batch_graph_launch replays it; update
 * the buffers' contents in place between replays).  A batch shares its plans'
 * staging buffers: do not apply those plans concurrently with the batch.
 */
typedef struct p2p_batch p2p_batch;
P2P_API p2p_status p2p_batch_workspace_size(const p2p_plan* const* plans, int32_t count, int32_t nrhs,
                                            size_t* bytes);
P2P_API p2p_status p2p_batch_create(p2p_batch** batch, const p2p_plan* const* plans, int32_t count, int32_t nrhs,
                                    int32_t warps_per_cta, void* workspace, size_t workspace_bytes,
                                    p2p_stream_t stream);
P2P_API p2p_status p2p_batch_apply(const p2p_batch* batch, const void* const* lambdas, void* const* outs, int64_t ld,
                                   p2p_stream_t stream);
P2P_API p2p_status p2p_batch_graph_create(p2p_batch* batch, const void* const* lambdas, void* const* outs,
                                          int64_t ld);
P2P_API p2p_status p2p_batch_graph_launch(const p2p_batch* batch, p2p_stream_t stream);
P2P_API p2p_status p2p_batch_info(const p2p_batch* batch, int64_t* work_items, int32_t* grid,
                                  int32_t* warps_per_cta);
P2P_API p2p_status p2p_batch_destroy(p2p_batch* batch);

/* ------------------------------------------------- host-buffer apply --- */
/*
 * out_g = A_g lambda_g for a sequence of plans g = 0 .. count-1 whose strengths
 * and results live in host memory.  Each plan's strengths are copied into one of
 * two device staging slots, gathered and applied (as p2p_apply, path AUTO), and
 * the results copied back; the copies run on the pipe's own copy stream, so the
 * upload of plan g+1 and the download of plan g-1 overlap the kernels of plan g.
 *
 *   max_n            largest plan size (points) the pipe will carry, >= 1
 *   nrhs             right-hand sides per point, 1 .. 256
 *   workspace  [dev] at least p2p_host_pipe_workspace_size bytes, 256-byte aligned
 *                    (two strength slots and two result slots of max_n x nrhs
 *                    complex64)
 *   lambdas    [host] count host pointers; lambdas[g] is plan g's n_g x nrhs
 *                    complex64 strengths, contiguous (ld = nrhs)
 *   outs       [host] count host pointers, same shape; fully overwritten
 *   count            1 .. 64; every plan has n_g <= max_n and max_nrhs >= nrhs
 *
 * Host buffers should be page-locked (cudaHostAlloc / cudaHostRegister); pageable
 * memory gives the same results without the overlap.  p2p_apply_host enqueues
 * everything and returns; the outs are complete once `stream` reaches the end of
 * the call (the caller's stream waits for the last download), so synchronising
 * `stream`, or an event recorded on it after the call, covers them.  Calls on one
 * pipe must be issued on one stream; the plans must not be applied concurrently
 * elsewhere meanwhile (they share their staging buffers).  p2p_host_pipe_create
 * creates the copy stream and events (host-side objects released by
 * p2p_host_pipe_destroy, which synchronises the copy stream first).
 */
typedef struct p2p_host_pipe p2p_host_pipe;
P2P_API p2p_status p2p_host_pipe_workspace_size(int64_t max_n, int32_t nrhs, size_t* bytes);
P2P_API p2p_status p2p_host_pipe_create(p2p_host_pipe** pipe, int64_t max_n, int32_t nrhs, void* workspace,
                                        size_t workspace_bytes);
P2P_API p2p_status p2p_apply_host(p2p_host_pipe* pipe, const p2p_plan* const* plans, int32_t count,
                                  const void* const* lambdas, void* const* outs, p2p_stream_t stream);
P2P_API p2p_status p2p_host_pipe_destroy(p2p_host_pipe* pipe);

/*
 * Self-check of the tensor-core operand path (not part of the operator): one
 * thread block computes D = A . B^T through the same BF16 hi/lo split, shared-
 * memory layout, descriptors and tcgen05 MMAs as the multi-RHS P2P path.
 *
 *   A       [dev] 128 x K float, row-major
 *   B       [dev] n x K float, row-major
 *   D       [dev] out, 128 x n float, row-major
 *   K             multiple of 64, >= 64
 *   n             multiple of 16, 16 .. 256
 *   status  [dev] one unsigned int; bit 2 is set if a bounded wait ran out
 */
P2P_API p2p_status p2p_diag_tc_gemm(const float* A, const float* B, float* D, int32_t K, int32_t n,
                                    unsigned int* status, p2p_stream_t stream);
/*
 * Self-check of the bounded waits (not part of the operator): one warp waits
 * on an mbarrier that nothing arrives at, with the poll loop of the pipelined
 * kernels capped at `limit` polls (>= 1).  The wait runs out, bit 1
 * (P2P_ERR_TIMEOUT's device flag) is set in *status [dev], the kernel returns
 * and the CUDA context remains usable.
 */
P2P_API p2p_status p2p_diag_wait_timeout(unsigned int* status, int32_t limit, p2p_stream_t stream);

/*
 * Self-check of the tensor-core path's abort handling (not part of the
 * operator): every pipeline wait of the plan's later tensor-core launches polls
 * at most `polls` times (0: it gives up at once; negative: the normal bound).
 * A wait that runs out sets P2P_ERR_TIMEOUT in the status word; the roles stop,
 * the producers and MMA issuers wait (bounded) for their own copies and MMAs in
 * flight, the block frees its tensor memory and returns.  The results of such a
 * launch are not valid; restore the bound before relying on the plan again.
 */
P2P_API p2p_status p2p_diag_tc_wait_limit(p2p_plan* plan, int32_t polls);

/* Reads and clears the plan's device status word.  Synchronises. */
P2P_API p2p_status p2p_last_async_status(const p2p_plan* plan, p2p_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* P2P_H */
