/*
 * rsi.h -- C ABI of librsi: line-segment / triangle-mesh intersection on one
 * NVIDIA GB300 (sm_103a).
 *
 * Method: arXiv 2209.02878 (Leung, "GPU implementation of a ray-surface
 * intersection algorithm in CUDA").  The problem (Sec. 1): N_r segments
 * l_i = (r_start_i, r_end_i) against a mesh of N_t triangles t_j indexing
 * vertices V; result per segment is a crossing flag (default), a crossing
 * count (Sec. 2.4 "intercept_count") or the intersecting point and triangle
 * (Sec. 2.4 "barycentric").  The segment/triangle predicate is
 * Moller-Trumbore (Sec. 2); the acceleration structure is a linear BVH over
 * Morton-sorted triangle centroids (Sec. 2: centroids, quantisation, Morton
 * codes, sort, binary radix tree, bottom-up boxes) searched per segment with
 * a stack (Sec. 3.2, bvhTraverse / bvhFindCollisions).
 *
 * Conventions shared by every call:
 *  - Layouts follow Sec. 2.5: vertices float32 [nV][3], triangles int32
 *    [nT][3] (0-based vertex indices), segment starts / ends float32 [nR][3],
 *    all C-contiguous, x y z interleaved.
 *  - Pointers named d* are DEVICE pointers of the current CUDA device; the
 *    caller owns them, must keep them alive until the stream work using them
 *    has finished, and the library never frees them.  Pointers without the d
 *    prefix are host pointers.
 *  - rsi_stream is a cudaStream_t (NULL = legacy default stream).  Every
 *    compute call is asynchronous on that stream unless stated otherwise.
 *  - A handle (rsi_bvh, rsi_batch) holds its tree, work counters,
 *    workspaces and internal streams: calls on one handle must not run
 *    concurrently from several host threads, and their GPU work must not
 *    overlap -- queue them on one stream, or order the streams with events
 *    (rsi_intersect_host orders its own internal streams).  Different
 *    handles are independent.
 *  - Calls never throw, never abort and never trap the GPU; they return an
 *    rsi_status.  Errors that can only be seen on the device (a triangle index
 *    outside [0, nV)) are latched in a device status word and returned by
 *    rsi_bvh_status / rsi_batch_status (which synchronise the stream).
 *  - Arithmetic: FP32 with certified error bounds; every boolean decision
 *    whose FP32 error bound does not settle it is recomputed in FP64 in the
 *    exact operation order of the definition below, so flags, counts and
 *    triangle ids equal those of the FP64 definition.  t, u, v, points and
 *    distances are within 1e-5 of the definition's FP64 values (relative to
 *    max(1, |x|)): FP32 values stand where a rigorous bound shows them
 *    within that, the rest are recomputed in double-float, or with the FP64
 *    definition itself at grazing angles (det not separable from zero in
 *    FP32) and on long segments.  Gradients are within 1e-5 of the FP64
 *    adjoint (relative to max(|g|, 1e-3 max |g|)).
 *
 * Definition computed (Sec. 2, Moller-Trumbore without division):
 *   d = b - a, e1 = v1 - v0, e2 = v2 - v0, p = d x e2, det = e1.p,
 *   s0 = a - v0, q = s0 x e1, nU = s0.p, nV = d.q, nT = e2.q;
 *   if det < 0 negate det, nU, nV, nT;
 *   hit <=> det > 0, nU >= 0, nV >= 0, nU + nV <= det, 0 <= nT <= det;
 *   t = nT/det, u = nU/det, v = nV/det, P = a + t d, dist = t |d|.
 *   A segment or triangle with a non-finite coordinate never hits.
 */
#ifndef RSI_H
#define RSI_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* rsi_stream; /* == cudaStream_t */
typedef struct rsi_bvh_s* rsi_bvh;      /* opaque, library-owned */
typedef struct rsi_batch_s* rsi_batch;  /* opaque, library-owned */

typedef enum {
    RSI_OK = 0,
    RSI_ERR_ARG = 1,            /* invalid argument (null, negative size, bad mode) */
    RSI_ERR_CUDA = 2,           /* a CUDA runtime call failed */
    RSI_ERR_OOM = 3,            /* device allocation failed */
    RSI_ERR_BAD_INDEX = 4,      /* a triangle index is outside [0, nV), or a
                                   processing-order entry outside [0, nR) */
    RSI_ERR_STACK_OVERFLOW = 5, /* traversal stack too small (never with depth >= 64) */
    RSI_ERR_TIMEOUT = 6,        /* a bounded device-side wait gave up */
    RSI_ERR_NOT_BUILT = 7,      /* handle has no built tree */
    RSI_ERR_INTERNAL = 8,       /* a device-side consistency bound was hit (a
                                   tree slot or leaf range out of its mesh,
                                   or more node visits than nodes); the work
                                   stopped */
    RSI_ERR_CAPACITY = 9        /* the problem exceeds the fixed scratch of an
                                   allocation-free entry point */
} rsi_status;

typedef enum {
    RSI_MODE_BOOL = 0,    /* Sec. 1: crossing flag y_i in {0,1} */
    RSI_MODE_COUNT = 1,   /* Sec. 2.4 intercept_count: number of crossings */
    RSI_MODE_NEAREST = 2  /* Sec. 2.4 barycentric: nearest crossing (min t,
                             ties to the lower triangle index) */
} rsi_mode;

/* Options fixed when a tree is built.  Zero-initialised = defaults. */
typedef struct {
    int32_t leaf_size;  /* max triangles per leaf, 1..8 (0 -> 1, the paper's
                           one-triangle leaves, Sec. 3.1) */
    int32_t top_levels; /* breadth-first levels of the tree copied into a
                           compact top "treelet" (at most 2048 nodes) that
                           traversal can stage in shared memory (launch
                           option smem_nodes), 1..12; 0 or -1 -> no treelet
                           (the default: L1 serves the top levels as well on
                           the paper-scale workload) */
    int32_t height_axis; /* 0: the paper's Morton code over the centroids'
                           x, y, z (10 bits each).  1, 2, 3: for a mesh that
                           is a height field over the plane of the other two
                           axes (a terrain: z = f(x, y) is 3), that
                           coordinate is left out and the other two take 15
                           bits each.  Only the tree's shape changes, not a
                           result; on height fields it avoids the splits
                           along the height that put both children across a
                           segment's path (131,072-triangle terrain,
                           near-vertical segments: 29.2 -> 18.8 node visits,
                           nearest 0.227 -> 0.127 ms).  Not in the paper. */
} rsi_build_opts;

/* Options of one traversal launch.  Zero-initialised = defaults. */
typedef struct {
    int32_t block_size;  /* threads per block, multiple of 32 in [32, 1024]
                            (0 -> 128); capped at what the kernel's register
                            use allows */
    int32_t stack_depth; /* per-segment traversal stack entries: 8, 32 or 64
                            (0 -> 64).  Radix trees over 64-bit keys are at
                            most 63 levels deep, so 64 never overflows; a
                            smaller stack re-runs overflowed segments with a
                            deeper one. */
    int32_t smem_nodes;  /* treelet nodes staged in shared memory per block
                            (64 B each, at most 2048); 0 or -1 -> none (the
                            top levels then live in L1, which measured
                            faster on the paper-scale workload) */
    int32_t stats;       /* nonzero: count node visits, triangle tests and
                            FP64 fallbacks (slower; see rsi_intersect_stats) */
    int32_t sort_bits;   /* coherent segment order (the paper's Morton-sorted
                            rays, Sec. 4.1): segments are processed in the
                            order of a key of this many bits (midpoint Morton
                            code + direction octant), 6..30; 0 or -1 -> input
                            order (measured faster for random segments).
                            Results do not depend on the order.  Needs a
                            workspace of 16 B per segment, allocated by the
                            handle on first use (device allocator, on s) and
                            kept for later calls of the same or smaller nR. */
    int32_t node_width;  /* traversal node arity: 2 (the binary tree, as in
                            the paper) or 4 (each visit tests the four
                            grandchildren of a binary node: half the chain of
                            dependent node fetches, twice the box tests;
                            its records are built by one extra kernel on the
                            first 4-wide traversal after each build or
                            refit); 0 -> 2.  smem_nodes > 0 implies 2. */
    int32_t packet;      /* 1: warp-cooperative traversal (f4, for coherent
                            segments): each warp takes 32 consecutive
                            segments in processing order and walks the tree
                            once for all of them, descending into a child
                            when any lane's segment enters it; results are
                            the same.  Costs the union of the 32 paths, so
                            use it with sort_bits or with inputs already
                            ordered in space.  Requires node_width 0 / 2 and
                            smem_nodes <= 0 (else RSI_ERR_ARG); block_size
                            and stack_depth are ignored (128, 64).  0 -> one
                            stack per segment. */
    const int32_t* order; /* DEVICE int32[nR] processing order, used instead
                            of sort_bits: pool position k processes segment
                            order[k] (outputs still go to the segment's own
                            index), so an order computed once by
                            rsi_segment_order serves every later call on
                            the same segments (e.g. fixed rays while the
                            mesh moves).  Must be a permutation of [0, nR);
                            an entry outside [0, nR) is skipped and latches
                            RSI_ERR_BAD_INDEX (rsi_bvh_status).  Only
                            rsi_intersect takes it: the host, inside and
                            batch calls return RSI_ERR_ARG.  NULL -> none. */
} rsi_launch_opts;

/* Per-segment outputs, all DEVICE pointers owned by the caller.  Which must be
 * non-NULL depends on the mode; the others may be NULL and are ignored.
 *   BOOL:    flag  uint8[nR]   (1 = the segment crosses the surface)
 *   COUNT:   count int32[nR]   (number of triangles crossed)
 *   NEAREST: tri   int32[nR]   (original triangle index, -1 = no crossing)
 *            tuv   float[nR][3] (t, u, v; 0 on a miss)      optional
 *            point float[nR][3] (a + t d; 0 on a miss)       optional
 *            dist  float[nR]    (t |b - a|; 0 on a miss)     optional
 * Compaction (COUNT and NEAREST; optional): when hit_idx != NULL, the index
 * of every segment with at least one crossing is appended to hit_idx[0..cap)
 * by a warp-aggregated atomic; *n_hits (device int64, zeroed by the call)
 * receives the total, which may exceed cap (entries past cap are dropped).
 * Order across warps is unspecified; for NEAREST the parallel arrays
 * hit_tri / hit_dist / hit_point, and for COUNT hit_count, are filled at the
 * same positions when non-NULL (the paper's (intersecting_rays, distances,
 * intersecting_triangles, intersecting_points), Sec. 2.4). */
typedef struct {
    uint8_t* flag;
    int32_t* count;
    int32_t* tri;
    float* tuv;
    float* point;
    float* dist;
    int32_t* hit_idx;
    int64_t hit_cap;
    int64_t* n_hits;
    int32_t* hit_tri;
    float* hit_dist;
    float* hit_point;
    int32_t* hit_count;
} rsi_output;

typedef struct {
    int64_t n_vertices;
    int64_t n_triangles;
    int32_t leaf_size;
    int32_t treelet_nodes;  /* nodes in the breadth-first top treelet */
    int64_t device_bytes;   /* device memory held by the handle */
} rsi_bvh_info;

typedef struct {
    int64_t segments;
    int64_t node_visits;   /* internal nodes fetched */
    int64_t tri_tests;     /* FP32 segment/triangle tests */
    int64_t fp64_tests;    /* tests decided by the FP64 recomputation */
    int64_t df_refines;    /* nearest hits whose outputs were recomputed in
                              double-float (the FP32 bound too loose for the
                              output tolerance) */
    int64_t overflows;     /* segments re-run with a deeper stack */
    int64_t fp64_values;   /* nearest hits whose outputs were recomputed with
                              the FP64 definition (grazing crossings whose det
                              FP32 cannot separate from zero, or directions
                              outside the FP32 filter's range) */
} rsi_stats;

/* Library and status helpers. */
const char* rsi_version(void);
const char* rsi_status_string(rsi_status s);

/* ------------------------------------------------------ device memory --- */

/* Caller-supplied device allocator (optional).  alloc returns `bytes` of
 * device memory on `device`, usable in stream order on s, at least 256-byte
 * aligned, or NULL when it cannot; free releases a pointer that alloc
 * returned, in stream order on s (work already queued on s may still use
 * it, as with cudaFreeAsync).  ctx is passed back unchanged. */
typedef void* (*rsi_alloc_fn)(size_t bytes, int device, rsi_stream s, void* ctx);
typedef void (*rsi_free_fn)(void* p, int device, rsi_stream s, void* ctx);

/* Route every device allocation of the library (handle storage, workspaces,
 * host-path staging, the adjoint's accumulator) through alloc / free, e.g.
 * PyTorch's caching allocator, instead of cudaMallocAsync / cudaFreeAsync;
 * both NULL restores the default.  Process-wide; a handle or batch keeps
 * the pair that was set when it was created for all its memory, including
 * the final free.  A NULL from alloc gives RSI_ERR_OOM, memory that is not
 * 256-byte aligned is handed back and gives RSI_ERR_CUDA.  Not part of the
 * paper.  Errors: RSI_ERR_ARG (exactly one of alloc, free NULL). */
rsi_status rsi_set_allocator(rsi_alloc_fn alloc, rsi_free_fn free, void* ctx);

/* ---------------------------------------------------------------- BVH --- */

/* Allocate a handle for meshes of nV vertices and nT triangles (device memory
 * from the device allocator -- rsi_set_allocator, else cudaMallocAsync --
 * on stream s, ordered on s).  No tree is built yet.
 * Sec. 2 / Sec. 3.1: the paper's internalNodes (N_t - 1) and leafNodes (N_t)
 * arrays; here one 64-byte node per internal node holding both child boxes,
 * plus a root slot, and the triangles re-stored in leaf order.
 * Errors: RSI_ERR_ARG (nV < 0, nT < 0, nT >= 2^31, out == NULL, bad opts),
 * RSI_ERR_OOM. */
rsi_status rsi_bvh_create(int64_t nV, int64_t nT, const rsi_build_opts* opt,
                          rsi_stream s, rsi_bvh* out);

/* Build the LBVH of (dV, dT) into h, asynchronously on s, without allocating
 * (capturable in a CUDA graph).  Steps (Sec. 2): centroid support interval,
 * 10-bit-per-axis quantisation and 30-bit Morton codes, on-device radix sort,
 * Karras binary radix tree, bottom-up boxes merged with per-node atomics
 * (Sec. 3.1 `atomic` field), optional leaf collapse and the top treelet.
 * dV float32[nV][3], dT int32[nT][3] with the sizes given at create time.
 * Index errors are latched for rsi_bvh_status.  Errors: RSI_ERR_ARG,
 * RSI_ERR_CUDA. */
rsi_status rsi_bvh_build(rsi_bvh h, const float* dV, const int32_t* dT, rsi_stream s);

/* rsi_bvh_create followed by rsi_bvh_build. */
rsi_status rsi_build_bvh(const float* dV, int64_t nV, const int32_t* dT, int64_t nT,
                         const rsi_build_opts* opt, rsi_stream s, rsi_bvh* out);

/* Re-fit the boxes of a built tree to new vertex positions dV (same nV, same
 * triangles as the last build): the bottom-up box pass of Sec. 2 without the
 * sort and hierarchy steps.  Results stay exact; only traversal speed depends
 * on how far the vertices moved.  Asynchronous, no allocation.  dT must be
 * the triangle array of the last build.  Errors: RSI_ERR_ARG,
 * RSI_ERR_NOT_BUILT, RSI_ERR_CUDA. */
rsi_status rsi_refit(rsi_bvh h, const float* dV, const int32_t* dT, rsi_stream s);

/* Synchronise s and return the device-side status latched by builds and
 * traversals on h since the last call (RSI_OK; RSI_ERR_BAD_INDEX: a triangle
 * index outside [0, nV); RSI_ERR_INTERNAL: a traversal exceeded its visit
 * bound, i.e. a corrupt tree; RSI_ERR_TIMEOUT: a streamed host call's wait
 * for its data gave up), then clear it. */
rsi_status rsi_bvh_status(rsi_bvh h, rsi_stream s);

rsi_status rsi_bvh_get_info(rsi_bvh h, rsi_bvh_info* info);

/* Free a handle: its internal streams are synchronised, then its memory is
 * released stream-ordered on the stream of the last call made with it
 * (every earlier use of the memory precedes that call), which must still
 * exist. */
rsi_status rsi_bvh_destroy(rsi_bvh h);

/* Debug / validation: synchronise s and copy the tree of h to HOST buffers,
 * each NULL-able:
 *   bounds  float[6]        centroid support interval (lo xyz, hi xyz)
 *   codes   uint32[nT]      Morton codes in sorted (leaf) order
 *   order   int32[nT]       sorted position -> original triangle index
 *   left, right int32[nT-1] children of Karras internal node i: >= 0 internal
 *                           node, < 0 leaf -(pos+1)
 *   range   int32[nT-1][2]  first, last leaf of internal node i
 *   nbox    float[nT-1][6]  internal node boxes (lo xyz, hi xyz)
 *   lbox    float[nT][6]    leaf (triangle) boxes by sorted position
 *   nodes   float[nT][16]   the traversal nodes (slot nT-1 is the root slot),
 *                           the children's coordinates in pairs:
 *                           lo.x0 lo.x1 lo.y0 lo.y1 | lo.z0 lo.z1 hi.x0 hi.x1 |
 *                           hi.y0 hi.y1 hi.z0 hi.z1 | ref0 ref1 cnt0 cnt1
 *                           (refs and counts as int32 bit patterns) */
rsi_status rsi_bvh_export(rsi_bvh h, rsi_stream s, float* bounds, uint32_t* codes,
                          int32_t* order, int32_t* left, int32_t* right, int32_t* range,
                          float* nbox, float* lbox, float* nodes);

/* ---------------------------------------------------------- traversal --- */

/* Test nR segments (dA[i] -> dB[i]) against the tree in h (Sec. 3.2-3.3,
 * bvhIntersectionKernel): one persistent launch with warp-granular dynamic
 * work distribution, stack traversal testing both child boxes of each node
 * with a conservative slab test, triangles tested inline at the leaves.
 * BOOL stops at the first crossing (Sec. 3.2, detected[rayIdx]); COUNT visits
 * every candidate; NEAREST prunes boxes beyond the best crossing so far.
 * out: see rsi_output.  lo: NULL = defaults.  nR == 0 is a no-op; an empty
 * mesh gives all misses.  Errors: RSI_ERR_ARG (null required output, bad
 * mode or options), RSI_ERR_NOT_BUILT, RSI_ERR_CUDA. */
rsi_status rsi_intersect(rsi_bvh h, const float* dA, const float* dB, int64_t nR,
                         rsi_mode mode, const rsi_output* out,
                         const rsi_launch_opts* lo, rsi_stream s);

/* Coherent processing order of nR segments (dA[i] -> dB[i], device), for
 * rsi_launch_opts.order: the order sort_bits computes on every call (paper
 * Sec. 4.1, Morton-sorted rays: the midpoint's Morton code over the tree's
 * root box grown by its extent on every side, then the direction octant, a
 * key of `bits` bits, 6..30, 0 -> 30), computed once and written to order
 * (DEVICE int32[nR], a permutation of [0, nR)) on s.  Uses the handle's
 * segment-order workspace (16 B per segment, allocated on first use from the
 * device allocator, on s).  Measured on 262,144 near-vertical segments over
 * a 131,072-triangle heightfield: nearest traversal 0.227 -> 0.185 ms against
 * input order; random segments gain nothing.  Errors: RSI_ERR_ARG (NULL pointer,
 * nR < 0 or >= 2^31, bits out of range), RSI_ERR_NOT_BUILT, RSI_ERR_OOM,
 * RSI_ERR_CUDA. */
rsi_status rsi_segment_order(rsi_bvh h, const float* dA, const float* dB, int64_t nR,
                             int32_t bits, int32_t* dOrder, rsi_stream s);

/* rsi_intersect from HOST buffers: hA, hB float[nR][3] and the outputs in
 * *hout (flag / count / tri, tuv, point, dist as for rsi_intersect) are host
 * pointers; compaction (hout->hit_idx) is not supported.  The segments go
 * through in chunks of `chunk` (0 -> 2^21) on two internal streams with
 * double-buffered device staging (56 B per segment per buffer, allocated by
 * the handle on first use from the device allocator, on s), so that the traversal of
 * one chunk and the copy of the previous chunk's results back overlap.
 * When hA and hB both lie in page-locked memory the device can address
 * (cudaHostAlloc / cudaHostRegister, unified addressing): in BOOL mode one
 * persistent traversal starts at once while the copy engine streams the
 * segments into device staging in chunks of `chunk` (0 -> 2^20, rounded up
 * to 32) and flags each chunk as it lands, the warps waiting (bounded:
 * RSI_ERR_TIMEOUT in the handle's status) for the chunks they take (two
 * staging slots used in turn, 25 B per segment each); in COUNT / NEAREST
 * the traversal kernel reads the segments in place over the CPU-GPU link.
 * Otherwise each chunk is first copied to the staging buffer, overlapped
 * with the previous chunk's traversal.  The traversal is ordered after
 * everything already on s, and s waits for the whole call: the host outputs
 * are complete once s is synchronised (hA and hB must stay unchanged until
 * then).  In the streamed BOOL path the copies of hA and hB wait only for
 * their staging slot (the call before the previous one), not for s, so
 * that they overlap the work already on s (a build, the previous call's
 * traversal): hA and hB must hold their data when the call is made.
 * Pageable host memory is staged by the driver and overlaps less.  Segments
 * are processed in input order (lo->sort_bits is ignored; lo->order gives
 * RSI_ERR_ARG).  Errors as rsi_intersect, plus RSI_ERR_OOM. */
rsi_status rsi_intersect_host(rsi_bvh h, const float* hA, const float* hB, int64_t nR,
                              rsi_mode mode, const rsi_output* hout, int64_t chunk,
                              const rsi_launch_opts* lo, rsi_stream s);

/* Odd-parity inside test for a CLOSED mesh (Sec. 2.6: the crossing count of
 * the intercept_count mode tells which segment starting points lie inside a
 * closed surface).  For each point dP[i] (float[nP][3], device) the segment
 * from the point to a far point along a fixed oblique direction, beyond the
 * mesh box, is counted in COUNT mode; dInside[i] (uint8[nP], device) = count
 * mod 2.  A point whose test segment passes within the near-degenerate band
 * of an edge or vertex can get the wrong parity, as with any parity test.
 * Uses a workspace of 16 B per point held by the handle (allocated on first
 * use from the device allocator, on s).  lo as for rsi_intersect (may be NULL).
 * Errors: RSI_ERR_ARG, RSI_ERR_NOT_BUILT, RSI_ERR_OOM, RSI_ERR_CUDA. */
rsi_status rsi_points_inside(rsi_bvh h, const float* dP, int64_t nP, uint8_t* dInside,
                             const rsi_launch_opts* lo, rsi_stream s);

/* Like rsi_intersect with lo->stats set; synchronises s and returns the
 * counters of that launch in *st (host). */
rsi_status rsi_intersect_stats(rsi_bvh h, const float* dA, const float* dB, int64_t nR,
                               rsi_mode mode, const rsi_output* out,
                               const rsi_launch_opts* lo, rsi_stream s, rsi_stats* st);

/* ----------------------------------------------------------- backward --- */

/* Adjoint of the NEAREST outputs with the crossing triangle held fixed (not
 * in the paper; implicit differentiation of a + t d = v0 + u e1 + v e2).
 * With M = [-d, e1, e2], x = (t,u,v) = M^-1 (a - v0) (recomputed from the
 * geometry, exact input differences), g_x = (gt + gP.d, gu, gv),
 * lambda = M^-T g_x:
 *   dA[i] = (1-t)(gP + lambda),  dB[i] = t (gP + lambda),
 *   dGradV[T[j][0]] += -(1-u-v) lambda, dGradV[T[j][1]] += -u lambda,
 *   dGradV[T[j][2]] += -v lambda,
 * and zero for segments with dTri[i] < 0.  The per-segment algebra runs in
 * double-float (about 44 bits), and in FP64 for crossings at grazing angles
 * (|det M| <= 2^-16 of its componentwise magnitude, where lambda grows like
 * 1/det M); the vertex sums use FP64 atomics into a stream-ordered FP64
 * scratch of 24 nV bytes (freed on s), rounded to FP32 once.  Within the
 * gradient tolerance stated at the top of this header.
 * Inputs: dV, dT as for the build; dA, dB the segments; dTri int32[nR] saved
 * from the NEAREST forward; dGradPoint float[nR][3] and dGradTuv float[nR][3]
 * (either may be NULL = zero).  Outputs: dGradV float[nV][3] ACCUMULATED into
 * (caller zeroes it), dGradA / dGradB float[nR][3] overwritten (each may be
 * NULL).  Errors: RSI_ERR_ARG, RSI_ERR_OOM, RSI_ERR_CUDA; a dTri entry >= nT
 * or a vertex index outside [0, nV) contributes nothing. */
rsi_status rsi_intersect_backward(const float* dV, int64_t nV, const int32_t* dT, int64_t nT,
                                  const float* dA, const float* dB, int64_t nR,
                                  const int32_t* dTri, const float* dGradPoint,
                                  const float* dGradTuv, float* dGradV, float* dGradA,
                                  float* dGradB, rsi_stream s);

/* Largest nV accepted by rsi_intersect_backward_static. */
#define RSI_STATIC_MAX_VERTICES 262144

/* Allocation-free variant of rsi_intersect_backward (the paper has no
 * counterpart; it has no backward pass).  For callers that cannot allocate
 * device memory when they call it -- hosts that reserve all device memory at
 * start-up and forbid later allocation, code running while a CUDA graph is
 * captured into a memory pool it does not own, or code called from inside an
 * allocator -- the FP64 vertex accumulator lives in a fixed device array
 * compiled into the library (RSI_STATIC_MAX_VERTICES vertices, 6 MiB per
 * device, held until the process exits) instead of a per-call allocation.
 * Same arguments, outputs and arithmetic as rsi_intersect_backward; no
 * cudaMalloc / cudaFree or other allocating call is made.
 *  - nV > RSI_STATIC_MAX_VERTICES returns RSI_ERR_CAPACITY and enqueues
 *    nothing.
 *  - The first call on a device (that device current) looks up the array's
 *    device address.  Under lazy module loading (CUDA_MODULE_LOADING=LAZY,
 *    the default since CUDA 12) that first call is also what loads the
 *    module holding the array, and so commits its 6 MiB of device memory:
 *    make the first call before reserving the rest of device memory and
 *    before any stream capture begins.
 *  - All calls share the array: each call clears what it uses first, and
 *    the array keeps the last call's sums.  Calls whose work overlaps on the
 *    GPU (e.g. on two unordered streams) race and give wrong gradients. */
rsi_status rsi_intersect_backward_static(const float* dV, int64_t nV, const int32_t* dT,
                                         int64_t nT, const float* dA, const float* dB,
                                         int64_t nR, const int32_t* dTri,
                                         const float* dGradPoint, const float* dGradTuv,
                                         float* dGradV, float* dGradA, float* dGradB,
                                         rsi_stream s);

/* ------------------------------------------------------------ batched --- */

/* One independent problem of a batch: a mesh, its segments, a mode and the
 * outputs (same meaning as for rsi_intersect).  Device pointers. */
typedef struct {
    const float* dV;
    int64_t nV;
    const int32_t* dT;
    int64_t nT;
    const float* dA;
    const float* dB;
    int64_t nR;
    int32_t mode;   /* rsi_mode */
    int32_t height_axis; /* 1, 2, 3: this mesh's Morton code leaves that axis
                            out (rsi_build_opts.height_axis, per item); 0:
                            the batch's build option */
    rsi_output out;
} rsi_batch_item;

/* Plan a batch of n items (host array, copied): allocates one concatenated
 * tree storage for all meshes and a work list of (item, segment chunk) tiles
 * ordered by estimated cost (N_r log N_t), largest first.  The item pointers
 * are stored: they must stay valid for the plan's lifetime.  From lo the
 * batch uses block_size and stack_depth (the batched kernel traverses binary
 * nodes with one stack per segment, in input order); the other fields are
 * validated and otherwise ignored.
 * Errors: RSI_ERR_ARG, RSI_ERR_OOM, RSI_ERR_CUDA. */
rsi_status rsi_batch_create(const rsi_batch_item* items, int32_t n,
                            const rsi_build_opts* bo, const rsi_launch_opts* lo,
                            rsi_stream s, rsi_batch* out);

/* Build every mesh of the batch: the same build steps as rsi_bvh_build run
 * once over all meshes (segmented by a mesh id in the sort key).
 * Asynchronous, no allocation, capturable. */
rsi_status rsi_batch_build(rsi_batch b, rsi_stream s);

/* Traverse every item in ONE persistent launch (tiles pulled from an atomic
 * work counter, per-tile mode).  Asynchronous, no allocation, capturable. */
rsi_status rsi_batch_intersect(rsi_batch b, rsi_stream s);

/* Capture build + intersect of the batch into a CUDA graph once (on s) and
 * launch it; later calls replay the graph.  rebuild = 0 replays only the
 * traversal graph. */
rsi_status rsi_batch_run_graph(rsi_batch b, int32_t rebuild, rsi_stream s);

/* As rsi_bvh_status for a batch: synchronise s, return and clear the status
 * latched by the batch's build and traversals. */
rsi_status rsi_batch_status(rsi_batch b, rsi_stream s);

rsi_status rsi_batch_destroy(rsi_batch b);

/* -------------------------------------------------------------- tuning --- */

/* One timed configuration of the tuner. */
typedef struct {
    int32_t block_size, stack_depth, smem_nodes, leaf_size;
    float ms;  /* median traversal time of `reps` launches */
} rsi_tune_entry;

/* Autotuner: for every combination of the candidate lists (leaf sizes need a
 * rebuild of h with those options), time `reps` traversals of the given
 * segments in `mode` with CUDA events on s, write up to cap entries to
 * table (host) and the fastest launch options / leaf size to *best_lo /
 * *best_leaf.  The handle is left built with the best leaf size.  dV, dT
 * must be the mesh h was built from.  Synchronous. */
rsi_status rsi_autotune(rsi_bvh h, const float* dV, const int32_t* dT,
                        const float* dA, const float* dB, int64_t nR, rsi_mode mode,
                        const rsi_output* out,
                        const int32_t* block_sizes, int32_t n_bs,
                        const int32_t* stack_depths, int32_t n_sd,
                        const int32_t* smem_nodes, int32_t n_sm,
                        const int32_t* leaf_sizes, int32_t n_ls, int32_t reps,
                        rsi_stream s, rsi_tune_entry* table, int32_t cap,
                        int32_t* n_written, rsi_launch_opts* best_lo, int32_t* best_leaf);

/* Autotuner for the build option height_axis (not in the paper): rebuilds h
 * from dV, dT with each of the Morton codes 0 (x, y, z), 1, 2, 3 (that axis
 * left out), times `reps` traversals of the given segments in `mode` with
 * launch options lo (NULL = defaults) under each (median, CUDA events on s),
 * writes the four medians to ms[4] (host) and the fastest axis to
 * *best_axis, and leaves h built with it (its later builds and refits keep
 * it).  Results never depend on the choice.  Synchronous.  Errors:
 * RSI_ERR_ARG (NULL pointer, nR <= 0, reps < 1), RSI_ERR_NOT_BUILT, and
 * those of rsi_bvh_build / rsi_intersect. */
rsi_status rsi_autotune_height_axis(rsi_bvh h, const float* dV, const int32_t* dT,
                                    const float* dA, const float* dB, int64_t nR,
                                    rsi_mode mode, const rsi_output* out,
                                    const rsi_launch_opts* lo, int32_t reps, rsi_stream s,
                                    float* ms, int32_t* best_axis);

/* --------------------------------------------------------- measurement --- */

/* FP32 peak probe (not part of the paper's method): launches an FMA-only
 * kernel that fills every SM of the current device (8 independent chains
 * per thread, `iters` FMAs per chain), times it with CUDA events on s after
 * one short warm-up launch, and writes the measured FP32 rate in TFLOP/s
 * (2 flops per FMA) to *tflops (host).  It is the ceiling the benchmark
 * compares the traversal's box-test and triangle-test arithmetic with.
 * Synchronises s; allocates 4 bytes (device allocator, on s).  Errors:
 * RSI_ERR_ARG (iters < 1, tflops NULL), RSI_ERR_CUDA. */
rsi_status rsi_fp32_peak(int64_t iters, double* tflops, rsi_stream s);

/* Self-test of the bounded device-side wait (not part of the paper's
 * method): one warp waits, with the wait the streamed host path uses, on a
 * device flag that nothing sets; after `polls` polls (about 0.25 us each) it
 * gives up and latches RSI_ERR_TIMEOUT into a status word, which is written
 * to *status_out (host).  The context stays usable.  Synchronises s;
 * allocates 8 bytes (device allocator, on s).  Errors: RSI_ERR_ARG
 * (polls < 1, status_out NULL), RSI_ERR_OOM, RSI_ERR_CUDA. */
rsi_status rsi_selftest_wait(int32_t polls, rsi_stream s, int32_t* status_out);

/* Self-test of the streamed host path giving up (not part of the paper's
 * method): one persistent BOOL traversal over nR zero-length segments (no
 * mesh), launched exactly as the streamed path launches it, whose warps wait
 * for ready flags that no copy ever sets, each wait bounded by `polls`
 * polls.  The first wait that gives up latches RSI_ERR_TIMEOUT and ends the
 * launch for every warp (no warp takes another chunk), so the launch lasts
 * about one wait, not one per chunk.  Writes the latched status to
 * *status_out and the launch's event-timed duration in ms to *ms_out
 * (host).  Synchronises s; allocates about 13 nR bytes (device allocator,
 * on s).  Errors: RSI_ERR_ARG (polls < 1, nR outside [1, 2^26], a NULL
 * output), RSI_ERR_OOM, RSI_ERR_CUDA. */
rsi_status rsi_selftest_stream_wait(int32_t polls, int64_t nR, rsi_stream s,
                                    int32_t* status_out, float* ms_out);

#ifdef __cplusplus
}
#endif
#endif /* RSI_H */
