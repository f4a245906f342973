/*
 * rsi.h -- C ABI of the GB300 (sm_103a) ray-segment / triangle-surface
 * intersection library (librsi.so).
 *
 * The method (R. Leung, "An experience with PyCUDA: Refactoring an existing
 * implementation of a ray-surface intersection algorithm", 2023):
 *   build  -- surface extent (Sec. 3.3), Morton codes of triangle centroids
 *             (Sec. 3.2), sort (Sec. 3.2), binary radix tree (Sec. 1, after
 *             Karras 2012; Sec. 4.2) and bottom-up bounding boxes (Sec. 4.1,
 *             4.2), all on the GPU;
 *   query  -- per-segment BVH search with Moller-Trumbore segment/triangle
 *             tests (Sec. 1), returning the boolean result or the number of
 *             crossings (the "boolean" and "intercept_count" modes of Sec. 1).
 * Tests run in FP32; segments whose FP32 result could differ from an FP64
 * evaluation (the Epilogue's near-parallel precision loss) are re-tested on
 * the GPU in FP64.
 *
 * Conventions
 *   - A "segment" (the paper's ray) runs from `from[i]` to `to[i]`; both are
 *     row-major float32 [n_rays][3].  Vertices are float32 [n_vertices][3];
 *     triangles are int32 [n_triangles][3] vertex indices (int64 indices are
 *     a different layout and are not accepted, Sec. 4.1.2).
 *   - Pointers named d_* are device pointers, h_* host pointers.  The caller
 *     owns every buffer it passes; the library owns a handle and its buffers.
 *   - `stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Work is stream-ordered: a call returns after enqueueing unless
 *     stated otherwise.  Calls that share a handle must be ordered on one
 *     stream (they share the handle's scratch memory).
 *   - Device memory of handles and their scratch comes from a private
 *     stream-ordered pool per device: up to 4 GiB of freed blocks stay cached
 *     for later handles, and frees do not synchronize the device.
 *   - A handle, plan or network belongs to the device that was current when
 *     it was created; the library never switches devices, so that device
 *     must be current (and the buffers and stream must be on it) for every
 *     later call on it.
 *   - Every function returns RSI_OK (0) or a negative RSI_ERR_* code and
 *     never throws; rsi_last_error() then describes the failure.
 */
#ifndef RSI_H_
#define RSI_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RSI_OK 0
#define RSI_ERR_INVALID_ARG (-1) /* null pointer, negative size, bad mode   */
#define RSI_ERR_DTYPE (-2)       /* element size other than the documented  */
#define RSI_ERR_OOM (-3)         /* device allocation failed                */
#define RSI_ERR_CUDA (-4)        /* a CUDA runtime call failed              */
#define RSI_ERR_TIMEOUT (-5)     /* a bounded device wait ran out           */
#define RSI_ERR_STACK (-6)       /* tree deeper than the traversal stack    */
#define RSI_ERR_NAN (-7)         /* NaN vertex coordinate                   */
#define RSI_ERR_INDEX (-8)       /* triangle vertex index out of range      */
#define RSI_ERR_OVERFLOW (-9)    /* a bounded per-segment list overflowed   */

/* Query modes (Sec. 1). */
#define RSI_ANY_HIT 0 /* "boolean": does the segment meet the surface       */
#define RSI_COUNT 1   /* "intercept_count": number of distinct crossings    */
#define RSI_NEAREST 2 /* "barycentric": nearest crossing (rsi_query_nearest) */
#define RSI_BOTH 3    /* boolean and intercept_count answers from one pass    */

typedef struct rsi_bvh_s* rsi_bvh_t;
typedef struct rsi_mlp_s* rsi_mlp_t;

/* Options of a query; a NULL pointer means all defaults (zeros). */
typedef struct rsi_options {
    int fp32_only;      /* 1: skip the FP64 re-test (results may flip near
                           edges and for nearly parallel segments)          */
    int block;          /* threads per block of the traversal: a multiple
                           of 32 in [32, 256]; 0 = tuned                    */
    int blocks_per_sm;  /* resident blocks per SM for the persistent grid,
                           0 = tuned                                         */
    int collect_stats;  /* 1: count node visits and triangle tests          */
    int64_t timeout_ns; /* batched plans: > 0 bounds the device waits of a
                           streaming plan (0 = 2 s); < 0 makes the plan
                           streaming with a |timeout_ns| bound             */
    int time_kernels;   /* 1: record CUDA events around the traversal and
                           re-test kernels on `stream` (rsi_last_query_ms) */
    int ray_sort_tile;  /* 0: segments traversed in input order; 256..8192:
                           each tile of this many segments is first grouped
                           by a coarse Morton cell of the segment midpoints
                           (better warp coherence; results are unchanged)  */
    int node_width;     /* nodes the FP32 traversal fetches: 2 (or 0, the
                           default) = child-pair nodes; 4 = four-wide nodes
                           (up to four child boxes per 128-byte fetch; trees
                           of height > 82 fall back to 2); 3 = compressed
                           child-pair nodes (32 bytes: child boxes on an
                           8-bit grid, rebuilt rounded outward; single
                           queries of single builds, else 2).  Results are
                           the same in every case.                          */
    int fp64_all;       /* 1: skip the FP32 traversal and settle every
                           segment with the FP64 re-test (a validation mode:
                           its answers must equal the default path's; slow).
                           Device-buffer queries only; not with fp32_only. */
    int stack;          /* entries of the FP32 traversal's stack: 0 = the
                           smallest of 32 / 64 / 128 that holds the walk of
                           the tree; 32, 64 or 128 = at least that many (a
                           tuning choice; results are unchanged)            */
    const int32_t* order; /* device [n_rays]: the order in which the FP32
                           traversal takes the segments, a permutation of
                           0 .. n_rays - 1 such as rsi_segment_order writes
                           (NULL = input order).  Results are unchanged and
                           stay at the segments' own indices.  Device-buffer
                           rsi_query / rsi_query_nearest only; not with
                           ray_sort_tile.                                   */
} rsi_options;

/* Per-query counters, filled on the host when a non-NULL pointer is given
 * (the call then synchronizes `stream`). */
typedef struct rsi_stats {
    int64_t n_rays;
    int64_t node_visits;   /* nodes fetched by the FP32 traversal, four-wide
                              or child-pair (collect_stats only)            */
    int64_t tri_tests;     /* FP32 segment/triangle tests (collect_stats)    */
    int64_t band_rays;     /* segments re-tested in FP64                     */
    int64_t ambiguous;     /* segments left ambiguous by the FP64 re-test    */
    int32_t tree_height;
    int32_t device_error;  /* RSI_OK or the RSI_ERR_* a kernel raised        */
    int64_t proposal_confirmed; /* learned query: hits settled by the proposal */
    int64_t fallback_rays;      /* learned query: segments left to the tree   */
} rsi_stats;

/* Static description of a built hierarchy. */
typedef struct rsi_bvh_info {
    int64_t n_triangles;
    int64_t n_vertices;
    int32_t morton_bits;
    int32_t height;          /* edges on the longest root-to-leaf path      */
    int64_t device_bytes;    /* bytes the handle holds on the device        */
    float extent_lo[3], extent_hi[3];
    float max_tri_extent[3]; /* largest triangle box side per axis          */
} rsi_bvh_info;

/* Host-side copy of the hierarchy for inspection (the BVH dump of Sec.
 * 4.1.1).  The caller allocates every array with the sizes given
 * (n = n_triangles); NULL members are skipped.  Internal node i has children
 * left[i], right[i]: an internal node index, or a leaf j tagged as
 * (int32)(0x80000000u | j); leaf j holds triangle perm[j].  Numbering follows
 * Karras 2012: the root is internal node 0.  parent[] lists internal nodes
 * then leaves (root: -1).  box[] is 6 floats (min xyz, max xyz) per node,
 * internal nodes then leaves. */
typedef struct rsi_bvh_host_view {
    uint64_t* sorted_keys; /* [n]     Morton codes in sorted order          */
    int32_t* perm;         /* [n]     triangle id of each leaf              */
    int32_t* left;         /* [n-1]                                         */
    int32_t* right;        /* [n-1]                                         */
    int32_t* parent;       /* [2n-1]                                        */
    float* box;            /* [6(2n-1)]                                     */
} rsi_bvh_host_view;

/*
 * Build the hierarchy over a triangle mesh (Sec. 3.2, 3.3, 4.1, 4.2): extent,
 * Morton codes of the centroids ((v0 + v1) + v2) / 3 in FP32
 * round-to-nearest, a stable radix sort by (code, triangle id), a Karras
 * radix tree and bottom-up boxes.
 *   d_vertices  [n_vertices][3] float32, device; d_triangles [n_triangles][3]
 *   int32, device.  index_bytes must be 4 (RSI_ERR_DTYPE otherwise: the
 *   int64 mix-up of Sec. 4.1.2).  morton_bits is 30 or 63.
 * The inputs are read during the call and may be freed afterwards.  The call
 * synchronizes `stream` once to check for NaN coordinates (RSI_ERR_NAN) and
 * out-of-range indices (RSI_ERR_INDEX).  n_triangles >= 1.
 * On success *out holds a new handle; release it with lbvh_free.
 */
int lbvh_build(const float* d_vertices, int64_t n_vertices, const int32_t* d_triangles,
               int64_t n_triangles, int index_bytes, int morton_bits, void* stream,
               rsi_bvh_t* out);

/* Tree construction of lbvh_build_ex. */
#define RSI_TREE_KARRAS 0  /* radix tree top-down, one thread per internal node
                              (Karras 2012), then a separate bottom-up refit */
#define RSI_TREE_APETREI 1 /* one bottom-up pass that builds the tree and its
                              boxes together (Apetrei 2014; the bottom-up
                              construction of Sec. 4.2)                      */
/* Or-ed into tree_builder: after the build, `passes` (1 .. 3) bottom-up
 * restructuring passes rewire groups of 7 subtrees so that the summed box
 * surface of the internal nodes goes down (treelet restructuring, Karras &
 * Aila 2013; not in the paper).  Leaves, their order and the triangles stay;
 * children, parents and boxes of internal nodes change (lbvh_export shows
 * the restructured tree), queries answer exactly as on the plain tree and
 * meet fewer nodes (c2 heightfield: 35 -> 28 child-pair nodes per segment
 * after one pass).  Such handles have no compressed nodes (node_width 3 is
 * served by child-pair nodes). */
#define RSI_TREE_TREELETS(passes) ((passes) << 8)

/*
 * As lbvh_build, with the tree construction chosen by tree_builder
 * (RSI_TREE_KARRAS or RSI_TREE_APETREI, optionally | RSI_TREE_TREELETS(p)
 * with p in 1 .. 3; anything else: RSI_ERR_INVALID_ARG).  The two builders
 * give the same hierarchy bit for bit -- the binary radix tree over the
 * sorted (code, triangle id) pairs is unique -- in the same numbering
 * (lbvh_export), so queries answer identically; only the build time differs.
 * RSI_TREE_APETREI replaces the tree and refit kernels with one kernel.
 */
int lbvh_build_ex(const float* d_vertices, int64_t n_vertices, const int32_t* d_triangles,
                  int64_t n_triangles, int index_bytes, int morton_bits, int tree_builder, void* stream,
                  rsi_bvh_t* out);

/*
 * Build the hierarchies of n_meshes independent meshes at once (the many
 * meshes of a batched query; building many at once has no counterpart in the
 * paper).  Mesh m: d_vertices[m] [n_vertices[m]][3] float32 and
 * d_triangles[m] [n_triangles[m]][3] int32, device (host arrays of device
 * pointers and counts).  Each stage of the build runs as one launch over all
 * meshes -- extent, Morton codes, a stable sort by code and then by mesh,
 * the single bottom-up pass of lbvh_build_ex(RSI_TREE_APETREI) and the
 * four-wide collapse -- and the call synchronizes `stream` once.  out[m]
 * receives mesh m's handle, identical to what lbvh_build would give it
 * (release each with lbvh_free).  Errors: as lbvh_build, naming the mesh;
 * on any error no handle is returned.  At most 2^30 triangles in all.
 */
int lbvh_build_batched(int n_meshes, const float* const* d_vertices, const int64_t* n_vertices,
                       const int32_t* const* d_triangles, const int64_t* n_triangles, int index_bytes,
                       int morton_bits, void* stream, rsi_bvh_t* out);

/* As lbvh_build_batched, then treelet_passes (0 .. 3; else
 * RSI_ERR_INVALID_ARG) restructuring passes over all meshes at once, each a
 * few launches over all meshes' nodes: every handle equals what
 * lbvh_build_ex(RSI_TREE_TREELETS(treelet_passes)) gives its mesh. */
int lbvh_build_batched_ex(int n_meshes, const float* const* d_vertices, const int64_t* n_vertices,
                          const int32_t* const* d_triangles, const int64_t* n_triangles, int index_bytes,
                          int morton_bits, int treelet_passes, void* stream, rsi_bvh_t* out);

/* As lbvh_build, with the mesh in host memory: h_vertices and h_triangles
 * are copied in on `stream` (page-locked arrays copy asynchronously) and may
 * be freed when the call returns; the call synchronizes `stream` as
 * lbvh_build does.  Errors as lbvh_build, plus RSI_ERR_OOM for the copies. */
int lbvh_build_host(const float* h_vertices, int64_t n_vertices, const int32_t* h_triangles,
                    int64_t n_triangles, int index_bytes, int morton_bits, void* stream,
                    rsi_bvh_t* out);

/* As lbvh_build_host, with tree_builder as in lbvh_build_ex. */
int lbvh_build_host_ex(const float* h_vertices, int64_t n_vertices, const int32_t* h_triangles,
                       int64_t n_triangles, int index_bytes, int morton_bits, int tree_builder, void* stream,
                       rsi_bvh_t* out);

/* Release a handle (synchronizes the device first).  NULL is a no-op. */
int lbvh_free(rsi_bvh_t h);

/* Describe a built hierarchy (host read of values kept in the handle; no
 * device work).  device_bytes counts the hierarchy plus the query scratch
 * the handle holds now.  RSI_ERR_INVALID_ARG for a NULL argument. */
int lbvh_info(rsi_bvh_t h, rsi_bvh_info* out);

/* Copy the hierarchy to the caller's host arrays (layout and sizes in
 * rsi_bvh_host_view; 30-bit codes are widened to uint64).  Synchronizes
 * `stream` first, so every build and query enqueued there is complete, and
 * returns after the copies.  RSI_ERR_INVALID_ARG for a NULL argument,
 * RSI_ERR_CUDA if a copy fails. */
int lbvh_export(rsi_bvh_t h, void* stream, rsi_bvh_host_view* out);

/* sizeof of one packed hierarchy node on the device (the paper's
 * bytesInBVHNode query, Sec. 3.2: sizes are asked of the library, never
 * hard-coded). */
size_t lbvh_node_bytes(void);

/*
 * Query n_rays segments against the hierarchy (Sec. 1 modes).
 *   mode RSI_ANY_HIT: d_hit[i] = 1 if segment i meets the surface, else 0.
 *   mode RSI_COUNT  : d_count[i] = number of distinct crossings; d_hit, if
 *                     not NULL, gets count > 0.
 *   mode RSI_BOTH   : both answers from one traversal (the count pass):
 *                     d_count as RSI_COUNT and d_hit (required) the boolean
 *                     answer, which is count > 0; d_ambiguous gets bit 0 =
 *                     the boolean mode's flag, bit 1 = the count mode's.
 *                     Every value equals what the two separate queries
 *                     write.
 *   d_ambiguous (optional): 1 where the segment lies within the 1e-6
 *   relative margin band even in FP64 (an end point, edge or vertex on the
 *   surface, or nearly parallel and touching); those results are the
 *   closed-interval reading with crossings closer than 1e-9 in t merged.
 *   In the boolean mode a decisive hit settles a segment whatever its other
 *   pairs are, so fewer segments are flagged than in the count mode.
 * Segments: d_from, d_to [n_rays][3] float32, device.  n_rays == 0 is a
 * no-op.  Asynchronous unless `stats` is given.  The handle grows its
 * scratch (the FP64 re-test's queue and pair lists, about 22 B per segment
 * of the largest batch queried so far) on demand; lbvh_free releases it.
 */
/* Errors: RSI_ERR_INVALID_ARG for a NULL handle or segment pointer, n_rays
 * outside [0, 2^31), a mode other than the three above, the output the mode
 * writes missing, or option values out of range; RSI_ERR_OOM when the
 * scratch cannot grow; RSI_ERR_STACK for a tree of height 127 or more
 * (a Karras tree over n < 2^30 leaves is at most 63 + 30 high); RSI_ERR_CUDA
 * for a failed launch.  A kernel's own error (RSI_ERR_OVERFLOW: a segment
 * with more than 64 inclusive crossings to de-duplicate in the FP64 pass) is
 * returned in stats->device_error. */
int rsi_query(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n_rays, int mode,
              const rsi_options* opt, uint8_t* d_hit, int32_t* d_count, uint8_t* d_ambiguous,
              rsi_stats* stats, void* stream);

/*
 * Barycentric mode (Sec. 1: for each intersecting ray, the intersecting
 * triangle and the distance to and location of the nearest intersecting
 * point; Sec. 3.3 moves the distance and point computations onto the GPU).
 * Per segment i, over the inclusive (closed-interval) crossings:
 *   d_tri[i]   int32, required: index (into the caller's triangle array) of
 *              the triangle of the smallest t (equal t: the lower index), or
 *              -1 when the segment meets no triangle;
 *   d_t[i]     float, optional: that t in [0, 1] (fraction of to - from),
 *              evaluated by the Moller-Trumbore definition in FP64 and
 *              rounded once; -1 when there is no hit;
 *   d_point    float [n_rays][3], optional: from + t (to - from), FP64 then
 *              rounded; NaN when there is no hit;
 *   d_dist[i]  float, optional: t |to - from|, the distance from the start
 *              point; -1 when there is no hit;
 *   d_ambiguous[i] uint8, optional: 1 where some pair lies in the 1e-6
 *              margin band in FP64 (as in RSI_COUNT); the result there is
 *              the closed-interval reading.
 * The search visits every pair like RSI_COUNT; segments whose nearest pair
 * is not certain in FP32 are settled in FP64.  Device buffers; n_rays == 0
 * is a no-op; asynchronous unless `stats` is given.  Errors as rsi_query.
 */
int rsi_query_nearest(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n_rays,
                      const rsi_options* opt, int32_t* d_tri, float* d_t, float* d_point, float* d_dist,
                      uint8_t* d_ambiguous, rsi_stats* stats, void* stream);

/*
 * The paper's barycentric result form (Sec. 2.3: intersecting rays,
 * distances, hit triangles, hit points): the segments with d_tri[i] >= 0,
 * in increasing index order, gathered from rsi_query_nearest's outputs.
 *   d_rays [n]: segment indices; d_tri_out [n]: triangle indices;
 *   d_dist_out [n] from d_dist; d_point_out [n][3] from d_point.
 * Every output is optional (NULL skips it) and must hold n_rays entries (the
 * most there can be).  *n_hits (host) receives n.  Device buffers; returns
 * after `stream` has finished the compaction.  RSI_ERR_INVALID_ARG when an
 * output is asked for without its input, or n_rays is outside [0, 2^31).
 */
int rsi_nearest_compact(const int32_t* d_tri, const float* d_dist, const float* d_point, int64_t n_rays,
                        int32_t* d_rays, int32_t* d_tri_out, float* d_dist_out, float* d_point_out,
                        int64_t* n_hits, void* stream);

/*
 * A traversal order for the segments of a batch (no counterpart in the
 * paper; the answers do not depend on the order): d_order [n_rays] (device,
 * caller-owned) receives 0 .. n_rays - 1 sorted by the Morton cell of each
 * segment's midpoint on a 32 x 32 x 32 grid over the hierarchy's extent
 * (order inside a cell arbitrary).  Pass it as rsi_options.order to any
 * number of queries of the same segments: neighbouring segments then cross
 * the same part of the tree and share node fetches.  Three launches and a
 * 128 KB counter array kept by the handle (allocated on first use);
 * asynchronous.  Errors: RSI_ERR_INVALID_ARG for a NULL handle or pointer
 * or n_rays outside [0, 2^31).
 */
int rsi_segment_order(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n_rays, int32_t* d_order,
                      void* stream);

/*
 * As rsi_query with segments and results in HOST memory; returns after the
 * results are in host memory.  Batches of up to 2^28 segments are staged
 * whole on the device (30 B per segment, kept for later calls): the segments
 * are copied in at most 64 chunks on an internal stream (2^16 segments,
 * then doubling up to 2^21) while one persistent FP32 traversal on `stream`
 * takes each chunk as it lands, then one FP64 re-test settles the whole
 * batch and the results are copied back.
 * Larger batches, batches whose staging does not fit in device memory, and
 * queries with opt->ray_sort_tile stream chunks of 2^21 through two recycled
 * staging slots (copies and traversal overlapped; the re-test runs per
 * chunk).  Page-locked host buffers give asynchronous copies; with
 * page-locked outputs (and child-pair nodes, no statistics) the traversal
 * counts its finished segments per chunk of 2^21 and the calling thread,
 * polling those counts, copies each chunk's FP32 answers out while the
 * traversal and the FP64 re-test go on; the re-tested segments' answers are
 * then written into the host arrays by the device.  The
 * staging is shared by all handles of a device: concurrent host-buffer
 * queries on one device run one after the other.
 */
int rsi_query_host(rsi_bvh_t h, const float* h_from, const float* h_to, int64_t n_rays, int mode,
                   const rsi_options* opt, uint8_t* h_hit, int32_t* h_count, uint8_t* h_ambiguous,
                   rsi_stats* stats, void* stream);

/*
 * Query without any device allocation.  The paper has no counterpart: this
 * is for callers that cannot allocate device memory while they query -- for
 * example a plugin whose host application owns all device memory through
 * its own allocator, or a real-time loop that must not pay for (or risk the
 * failure of) a cudaMalloc.  The hierarchy must already be built.
 *
 * Same arguments and results as rsi_query, except that no statistics are
 * returned and opt->time_kernels and opt->ray_sort_tile are ignored.  The per-call scratch (the
 * queue of segments re-tested in FP64 and the call's counters) lives in one
 * fixed device array of 256 B + 4 B x RSI_NOALLOC_MAX_RAYS (about 8 MiB)
 * that every GPU which loads the library keeps until the process exits.
 * n_rays above RSI_NOALLOC_MAX_RAYS is rejected with RSI_ERR_INVALID_ARG;
 * split larger batches into several calls.
 *
 * The first call on a device looks up that device's address of the array
 * (cudaGetSymbolAddress) with the device current; make that first call
 * before any stream capture.  The looked-up address is kept for the life of
 * the process: cudaDeviceReset (or anything else that destroys the device's
 * primary context) invalidates it, as it invalidates every handle built
 * before, so do not call this entry point on that device afterwards.  All calls share the one array: each call
 * clears the counters it needs, but calls whose work overlaps on the GPU
 * (different streams, or different threads without ordering) race on it and
 * must be serialized by the caller.  Device-side errors are not reported.
 */
#define RSI_NOALLOC_MAX_RAYS (1 << 21)
int rsi_query_noalloc(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n_rays, int mode,
                      const rsi_options* opt, uint8_t* d_hit, int32_t* d_count, uint8_t* d_ambiguous,
                      void* stream);

/*
 * Batched queries: many independent meshes, each with its own segments.
 * Each segment gets the boolean or intercept_count answer of Sec. 1 against
 * its own mesh, exactly as rsi_query would give it; batching (one persistent
 * launch over all batches, a device work queue, a CUDA graph) has no
 * counterpart in the paper.
 *   bvh       built hierarchy (must outlive the plan)
 *   d_from/d_to/n_rays, d_hit/d_count/d_ambiguous: as in rsi_query, device.
 */
typedef struct rsi_ray_batch {
    rsi_bvh_t bvh;
    const float* d_from;
    const float* d_to;
    int64_t n_rays;
    uint8_t* d_hit;
    int32_t* d_count;
    uint8_t* d_ambiguous;
} rsi_ray_batch;

typedef struct rsi_batch_s* rsi_batch_t;

/* Plan a batched query: validates the batches, uploads a descriptor table
 * (total segments < 2^31), and captures reset + traversal + FP64 pass into a
 * CUDA graph.  The buffers named in `batches` are fixed for the plan's life.
 * opt->timeout_ns < 0 selects streaming: the work queue starts empty and the
 * caller makes segments available with rsi_batch_post (|timeout_ns| bounds
 * each wait of the kernel for a post, then RSI_ERR_TIMEOUT is raised and the
 * unposted segments are left untouched).  opt->ray_sort_tile (256..8192)
 * groups each batch's segments tile by tile as rsi_query does (the graph
 * then starts with one reordering launch per batch); streaming plans
 * ignore it.  opt->node_width 3 is treated as 2.  Synchronizes `stream`. */
int rsi_batch_create(const rsi_ray_batch* batches, int n_batches, int mode, const rsi_options* opt,
                     void* stream, rsi_batch_t* out);

/* A plan whose graph first rebuilds every batch's hierarchy in place from
 * its mesh and then answers the query: build and query in one graph launch,
 * with the batched build's kernels and no host synchronization between them.
 *   d_vertices[i], d_triangles[i]  device float32 [n][3] / int32 [m][3] with
 *       the vertex and triangle counts of batches[i].bvh's own build; read at
 *       every launch, so the caller may change them between launches.
 * Otherwise as rsi_batch_create (no streaming; each hierarchy at most once;
 * all hierarchies of one Morton width).  The rebuild repeats the
 * restructuring passes the hierarchies were built with (the most any of them
 * had).  The heights of the rebuilt trees
 * are not known when the graph is captured, so every walk uses a 128-entry
 * stack and child-pair nodes.  Mesh errors (a NaN vertex, an index out of
 * range) are reported by rsi_batch_stats, which also brings the
 * hierarchies' host-side summaries (extent, padding, height, which lbvh_info
 * and single queries read) up to date: call it before using a rebuilt
 * hierarchy outside the plan.  Rebuilding has no counterpart in the paper. */
int rsi_batch_create_rebuild(const rsi_ray_batch* batches, int n_batches, const float* const* d_vertices,
                             const int32_t* const* d_triangles, int mode, const rsi_options* opt, void* stream,
                             rsi_batch_t* out);

/* Replay the plan on `stream` (one graph launch, asynchronous). */
int rsi_batch_launch(rsi_batch_t plan, void* stream);

/*
 * The batched query in one call: batch i's segments against hierarchy
 * hs[i], each with the boolean or intercept_count answer of Sec. 1 (mode),
 * exactly as rsi_query would give it.
 *   hs        [n_meshes] built hierarchies (host array of handles)
 *   batches   [n_meshes] segments and outputs (device buffers, as in
 *             rsi_batch_create); batches[i].bvh must be NULL or hs[i]
 *   opt       as for rsi_batch_create (streaming plans are not available
 *             here: opt->timeout_ns < 0 is rejected)
 * The library plans the call (rsi_batch_create: descriptor table, scratch,
 * graph capture; this synchronizes `stream`) and keeps the plan: a later
 * call with the same hierarchies, buffers, sizes, mode and options replays
 * it with one graph launch and returns without waiting.  Up to 4 plans are
 * kept per process (least recently used first out); lbvh_free drops the
 * plans that name the freed hierarchy.  A call's scratch is its plan's, so
 * two calls with identical arguments must not overlap on the GPU.
 */
int rsi_query_batched(const rsi_bvh_t* hs, int n_meshes, const rsi_ray_batch* batches, int mode,
                      const rsi_options* opt, void* stream);

/* Streaming plans only: segments [0, n_ready) of the concatenated batches
 * (batch 0's, then batch 1's, ...) are now in device memory.  Call after
 * rsi_batch_launch for the run being fed, on a stream other than the one
 * running the plan, after the copies of those segments on that stream
 * (stream order makes them visible first; the post also waits for the run's
 * queue reset, not for the run).  Counts must not decrease; at most 256
 * posts per plan may be pending. */
int rsi_batch_post(rsi_batch_t plan, int64_t n_ready, void* stream);

/* Counters of the plan's last run (synchronizes `stream`); returns the
 * device error (e.g. RSI_ERR_TIMEOUT) if a kernel raised one. */
int rsi_batch_stats(rsi_batch_t plan, rsi_stats* out, void* stream);

/* Release a plan (synchronizes the device first).  NULL is a no-op. */
int rsi_batch_free(rsi_batch_t plan);

/* Result of rsi_autotune. */
typedef struct rsi_tuning {
    int block;          /* threads per block chosen                          */
    int blocks_per_sm;  /* resident blocks per SM chosen                     */
    int ray_sort_tile;  /* in-tile reordering chosen (0 = off)               */
    int stack;          /* traversal stack entries the tree needs (32/64/128,
                           the smallest above the tree height)               */
    float ms;           /* time of the best candidate on the sample          */
    int from_cache;     /* 1 if the choice came from the cache file          */
    int candidates;     /* candidates timed (0 on a cache hit)               */
    int node_width;     /* node width chosen (2, 3 or 4, see rsi_options)    */
} rsi_tuning;

/*
 * Choose the traversal launch shape, node width and the in-tile segment reordering for
 * queries like this one (the method's query of Sec. 1; tuning has no
 * counterpart in the paper).  Times candidate options on the first
 * min(n_rays, 2^21) segments with CUDA events (running rsi_query, so it
 * allocates and synchronizes `stream`), writes the winner into *inout, and
 * records it in `cache_path` (a JSON object keyed by device, mode and log2
 * buckets of the triangle and segment counts; NULL = no cache).  A cached
 * key is reused without timing.  Concurrent writers of one cache file may
 * lose entries.
 */
int rsi_autotune(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n_rays, int mode,
                 const char* cache_path, rsi_options* inout, rsi_tuning* result, void* stream);

/*
 * The same tuning for batched plans (tuning has no counterpart in the
 * paper): times plans of the batches (each batch cut to its first 2^17
 * segments, outputs in scratch the call allocates) over threads per block,
 * resident blocks per SM, node width (2 or 4), the in-tile reordering
 * (0 or 8192) and the traversal stack (the smallest bucket that holds the
 * deepest tree, or the next one), writes the winner into *inout and
 * result->(block, blocks_per_sm, node_width, ray_sort_tile, stack), and
 * caches it in `cache_path` keyed by device, mode, the number of batches and
 * log2 buckets of their total triangles and segments.  Synchronizes `stream`.
 */
int rsi_batch_autotune(const rsi_ray_batch* batches, int n_batches, int mode, const char* cache_path,
                       rsi_options* inout, rsi_tuning* result, void* stream);

/*
 * Learned cluster proposal for boolean queries (no counterpart in the paper;
 * the answers stay the paper's, see rsi_query_learned).  A small network maps
 * a segment's end points (normalised by the mesh extent) through
 * 6 -> 128 -> 128 -> 256 units with GELU to logits over 256 clusters: equal
 * ranges of the Morton-ordered leaves of the hierarchy.  Weights and layer
 * inputs are BF16, accumulation FP32; inference runs on the tensor cores.
 * Parameters are one FP32 array of rsi_mlp_num_params() values:
 *   W1 [16][128] (rows 6..15 unused), b1 [128], W2 [128][128], b2 [128],
 *   W3 [128][256], b3 [256]   (row-major, y = x W + b).
 */
/* New network with seeded He-normal weights and zero biases (one device
 * allocation: weights, gradients, Adam moments, BF16 images).  RSI_ERR_OOM
 * if it fails.  rsi_mlp_free releases it (NULL is a no-op);
 * rsi_mlp_num_params is the parameter count (51,712). */
int rsi_mlp_create(uint64_t seed, rsi_mlp_t* out);
int rsi_mlp_free(rsi_mlp_t m);
int rsi_mlp_num_params(void);
/* Copy parameters in / out (host arrays of rsi_mlp_num_params() floats;
 * h_grads receives the gradient of the last training step; both
 * synchronize `stream`). */
int rsi_mlp_set_params(rsi_mlp_t m, const float* h_params, void* stream);
int rsi_mlp_get_params(rsi_mlp_t m, float* h_params, float* h_grads, void* stream);

/* Tensor-core inference for n segments against the extent of hierarchy h:
 * d_logits [n][256] float (nullable) and/or d_top4 [n][4] cluster ids, best
 * first (nullable).  The top 4 are chosen on keys made of the FP32 logit
 * with its low 8 bits replaced by 255 - cluster, compared as floats.
 * Asynchronous; rsi_mlp_status reports a tensor-core wait that ran out
 * (RSI_ERR_TIMEOUT). */
int rsi_mlp_forward(rsi_mlp_t m, rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n,
                    float* d_logits, uint8_t* d_top4, void* stream);
/* Synchronizes `stream` and returns RSI_ERR_TIMEOUT if a tensor-core wait of
 * an earlier forward on the network ran out (its outputs are then not
 * valid), else RSI_OK. */
int rsi_mlp_status(rsi_mlp_t m, void* stream);

/* The network's activation on n device floats z (for tests): GELU in its
 * tanh form, 0.5 z (1 + tanh(sqrt(2/pi) (z + 0.044715 z^3))) (Hendrycks &
 * Gimpel 2016).  d_tanh gets tanh(z) by the hardware approximation inference
 * uses (tanh.approx.f32), d_tanh_cuda CUDA's tanhf of the same z, d_gelu the
 * GELU the inference layers apply.  (Training evaluates the same formula
 * with tanhf.) */
int rsi_mlp_activation(const float* d_z, int64_t n, float* d_tanh, float* d_tanh_cuda, float* d_gelu, void* stream);

/* One training step on the GPU over a batch of n (1..65536) segments with
 * multi-hot labels d_labels [n][8] uint32 (bit c of word c/32: the segment
 * meets a triangle of cluster c, see rsi_cluster_labels): forward with the
 * inference roundings, mean binary cross-entropy over n x 256 logits,
 * backward (the BF16 roundings pass gradients unchanged), gradients kept for
 * rsi_mlp_get_params, then an Adam step (b1 0.9, b2 0.999, eps 1e-8, rate
 * lr) on the FP32 master weights if `apply`.  h_loss (nullable) gets the
 * batch loss before the step (the call then synchronizes `stream`). */
int rsi_mlp_train_step(rsi_mlp_t m, rsi_bvh_t h, const float* d_from, const float* d_to,
                       const uint32_t* d_labels, int64_t n, float lr, int apply, float* h_loss, void* stream);
/* Zero the Adam moments and step count (the weights are kept). */
int rsi_mlp_reset_optimizer(rsi_mlp_t m, void* stream);

/* Attach network m to hierarchy h (m = NULL detaches): from then on
 * rsi_query in RSI_ANY_HIT mode on h answers through the learned proposal
 * (rsi_query_learned) with the same answers; the other modes, the
 * host-buffer, batched and no-allocation queries are unaffected.  Freeing
 * either object detaches them.  A hierarchy holds at most one network; a
 * network may serve several hierarchies. */
int rsi_mlp_attach(rsi_bvh_t h, rsi_mlp_t m);

/*
 * Training labels: d_labels [n][8] uint32, bit c set when segment i meets a
 * triangle of cluster c (c = 256 * leaf / n_triangles) -- FP32 decisions,
 * the plain closed-interval one inside the error band (labels need not be
 * exact: they only steer the proposal).
 */
int rsi_cluster_labels(rsi_bvh_t h, const float* d_from, const float* d_to, int64_t n, uint32_t* d_labels,
                       void* stream);

/*
 * Boolean query with the learned proposal (Sec. 1's boolean mode; the
 * proposal has no counterpart in the paper): one tensor-core kernel runs the
 * network on tiles of 128 segments, keeps each segment's 4 proposed clusters
 * in registers and tests their triangles in FP32; a certain decisive hit
 * ends the segment with hit = 1.  Every other segment gets the plain query
 * (tree search + FP64 re-test) in a second launch.  d_hit / d_ambiguous are
 * therefore identical to rsi_query's.  Scratch as rsi_query; asynchronous
 * unless `stats` (whose tri_tests then include the proposal's tests).
 */
int rsi_query_learned(rsi_bvh_t h, rsi_mlp_t m, const float* d_from, const float* d_to, int64_t n_rays,
                      const rsi_options* opt, uint8_t* d_hit, uint8_t* d_ambiguous, rsi_stats* stats,
                      void* stream);

/* Durations of the FP32 traversal kernel and of the FP64 re-test kernel of
 * the last query on `h` that ran with time_kernels = 1, from CUDA events
 * recorded on that query's stream (waits for them); in the nearest mode the
 * second figure includes the pass that writes t, points and distances.
 * -1 if none. */
int rsi_last_query_ms(rsi_bvh_t h, float* traverse_ms, float* retest_ms);

/* Number of kernels this library has launched since it was loaded (all
 * threads, all devices): lets a caller count the device work of a region. */
uint64_t rsi_kernel_launches(void);

/* Message of the last failure on the calling thread ("" if none). */
const char* rsi_last_error(void);

/*
 * Failure injection for tests of the callers' error paths (no counterpart in
 * the paper).  With after >= 0, the next `after` device or pinned allocations
 * the library makes (all threads, all devices) succeed and every later one
 * fails as if the memory were exhausted: the call that needed it returns
 * RSI_ERR_OOM, releases what it had taken and leaves its handle usable.
 * after < 0 switches injection off (the default).  Always returns RSI_OK.
 */
int rsi_debug_fail_allocations(int64_t after);

#ifdef __cplusplus
}
#endif

#endif /* RSI_H_ */
