/*
 * vicp.h -- C ABI of the GB300 (sm_103a) dilation-based ICP library.
 *
 * The library implements the data-parallel hot path of dilation-based ICP
 * (VANICP) with per-voxel dynamic memory assignment, arXiv 2512.04996:
 * voxelise the target and count points per voxel (Alg. 1, GPU part), turn
 * the counts into segment offsets (Alg. 1, CPU part -- here a parallel
 * exclusive scan on the GPU), scatter point indices into a compact CSR store
 * (Alg. 2), dilate root-voxel labels into empty neighbours (Alg. 3), search
 * each transformed source point's root voxel with a global fallback
 * (Alg. 4), and solve the rigid update of Eq. 1.
 *
 * Conventions shared by every entry point
 *   - Point clouds are arrays of N x 4 float (x, y, z, w), 16-byte aligned,
 *     w ignored.  "dev" pointers are CUDA device pointers, "host" pointers
 *     are host memory (pinned or pageable).
 *   - Poses are 4x4 row-major double matrices mapping source coordinates
 *     into the target frame: q = R p + t with R = pose[0..2][0..2],
 *     t = pose[0..2][3].
 *   - The caller owns every input and output buffer.  The context owns its
 *     workspace (grid arrays, scratch), allocated through the allocator given
 *     to vicp_create and freed by vicp_destroy.
 *   - Calls are asynchronous on the context's CUDA stream unless stated
 *     otherwise.  Argument errors are returned immediately and launch
 *     nothing.  Errors detected on the device (a bounded wait that gave up,
 *     degenerate geometry in a solve) are recorded in a device status word
 *     and returned by the next synchronising call (vicp_sync, vicp_register,
 *     vicp_register_host, vicp_get_grid, vicp_memory_report,
 *     vicp_profile_read).
 *   - No entry point aborts, traps or throws across the ABI.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef VICP_H
#define VICP_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VICP_ABI_VERSION 2

#if defined(__GNUC__)
#define VICP_API __attribute__((visibility("default")))
#else
#define VICP_API
#endif

/* Status codes. */
typedef enum vicp_status {
    VICP_OK = 0,
    VICP_ERR_INVALID = 1,         /* bad argument: NULL, misaligned, size or range */
    VICP_ERR_CUDA = 2,            /* a CUDA runtime call failed (see vicp_last_error) */
    VICP_ERR_OOM = 3,             /* the allocator returned NULL */
    VICP_ERR_GRID_TOO_LARGE = 4,  /* nx*ny*nz >= 2^31 voxels */
    VICP_ERR_TIMEOUT = 5,         /* a bounded device-side wait gave up (no current kernel waits) */
    VICP_ERR_STATE = 6,           /* call order: e.g. correspond before build_grid */
    VICP_ERR_DEGENERATE = 7       /* rank(H) < 2 in the rigid solve; pose left unchanged */
} vicp_status;

typedef struct vicp_ctx vicp_ctx;

/* Device-memory allocator.  alloc returns a device pointer aligned to at
 * least 256 bytes, or NULL on failure; free releases it.  `stream` is the
 * context's stream (stream-ordered allocators may use it).  A NULL allocator
 * in vicp_create selects cudaMalloc / cudaFree. */
typedef struct vicp_allocator {
    void *(*alloc)(size_t bytes, void *stream, void *user);
    void (*free)(void *ptr, size_t bytes, void *stream, void *user);
    void *user;
} vicp_allocator;

/* Flags for vicp_params.flags. */
#define VICP_FLAG_KEEP_GRID         (1u << 0) /* auto grid: fit once, reuse for later builds */
#define VICP_FLAG_REBUILD_EACH_ITER (1u << 1) /* vicp_register: rebuild + dilate every iteration */
#define VICP_FLAG_FP64_SOLVE        (1u << 2) /* vicp_step / vicp_register: centroid and cross-covariance
                                                 sums in FP64 and the rigid solve in FP64 (Horn's
                                                 quaternion by Jacobi sweeps); default: double-float
                                                 (~48-bit) sums and solve on the FP32 pipes */
#define VICP_FLAG_SPARSE_GRID       (1u << 3) /* the sparse (hashed) grid, see vicp_get_sparse_grid: no
                                                 per-voxel count, offset, root or ring arrays */
#define VICP_FLAG_NO_GRAPH          (1u << 4) /* vicp_register / vicp_register_host: never replay the
                                                 call from a captured CUDA graph */


/* Run parameters (Sec. 4.1 "Parameter": voxelisation scale, dilation
 * layers L, maximum iteration count, RMSE-difference threshold). */
typedef struct vicp_params {
    float voxel_size;        /* > 0: voxel edge h.  <= 0: h = target extent / grid_divisions */
    int32_t grid_divisions;  /* used when voxel_size <= 0 (2^N in the paper; any value >= 1) */
    float origin[3];         /* explicit grid origin, used when dims[0] > 0 */
    int32_t dims[3];         /* explicit grid dims; dims[0] <= 0: origin = min corner of the
                                target, dims_a = floor(extent_a / h) + 1 */
    int32_t dilation_layers; /* L, 0..31 (paper: 10) */
    int32_t max_iters;       /* ICP iterations of vicp_register (paper: 50) */
    double rmse_eps;         /* stop once |rmse_k - rmse_(k-1)| < rmse_eps (paper: 1e-5); <= 0: never */
    uint32_t flags;          /* VICP_FLAG_* */
} vicp_params;

/* Read-only view of the grid built by the last vicp_build_grid / vicp_dilate.
 * All pointers are device pointers owned by the context and valid until the
 * next build or vicp_destroy. */
typedef struct vicp_grid_view {
    float origin[3];
    float voxel_size;
    float inv_voxel_size;      /* (float)(1.0 / (double)voxel_size) */
    int32_t dims[3];
    int64_t n_voxels;          /* V = dims[0]*dims[1]*dims[2] */
    int32_t n_target;          /* points passed to the last build */
    int32_t n_stored;          /* points inside the grid = offsets[V] */
    int32_t dilation_layers;   /* L of the last vicp_dilate, -1 before any */
    const int32_t *keys;       /* [n_target] voxel key x + nx*(y + ny*z), -1 outside */
    const uint32_t *offsets;   /* [V+1] exclusive scan of the per-voxel counts (all entries) */
    const int32_t *ids;        /* [n_stored] point indices grouped by voxel; the order inside
                                  one voxel's segment is unspecified */
    const float *csr_points;   /* [n_stored x 4] x, y, z of ids[k]; w holds the bits of ids[k] */
    const int32_t *root;       /* [V] root voxel of each voxel, -1 if farther than L */
    const uint8_t *ring;       /* [V] Manhattan distance to the root, 255 if unlabelled */
    const uint32_t *occupancy; /* [ceil(V/32)] bit v set iff voxel v holds a point */
} vicp_grid_view;

/* Device-memory accounting of one context (bytes). */
typedef struct vicp_memory {
    uint64_t current_bytes;          /* held now through the allocator */
    uint64_t peak_bytes;             /* high-water mark since vicp_create */
    uint64_t static_bytes;           /* per-voxel count + offset arrays (Table 1 note 1's
                                        "histogram and address offsets") */
    uint64_t csr_store_bytes;        /* offsets + ids + root + ring: the dynamic store */
    uint64_t fixed_capacity_bytes;   /* V * C_max * 4 for a fixed-capacity layout with C_max =
                                        the largest voxel count (the monolithic alternative) */
    uint64_t paper_static_layout_bytes; /* V * 65536: a 64 KB block per voxel (Sec. 2.2) */
    uint32_t max_voxel_count;        /* C_max */
    uint32_t occupied_voxels;
    uint32_t nonempty_bricks;        /* 8x8x8-voxel bricks holding a point (global-search index) */
    uint32_t labelled_voxels;        /* sparse grid: voxels within L of a point (the labelled-voxel
                                        table's entries); 0 for the dense grid */
} vicp_memory;

/* Work counters of the searches since the last reset. */
typedef struct vicp_stats {
    uint64_t queries;            /* source points searched */
    uint64_t fallbacks;          /* of which took the global search (Alg. 4, count == 0) */
    uint64_t local_candidates;   /* target points examined in root voxels */
    uint64_t global_candidates;  /* target points examined by global searches */
} vicp_stats;

/* ---------------------------------------------------------------------- */

VICP_API int32_t vicp_abi_version(void);
VICP_API const char *vicp_status_string(vicp_status s);

/* Fills *p with the paper's parameters: h = extent/16 (N = 4), L = 10,
 * 50 iterations, RMSE difference 1e-5 (Sec. 4.1 "Parameter"). */
VICP_API void vicp_default_params(vicp_params *p);

/* Creates a context bound to the current CUDA device and to `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream).  `params` is copied.
 * `alloc` may be NULL (cudaMalloc).  Errors: VICP_ERR_INVALID for NULL
 * out/params or out-of-range parameters; VICP_ERR_CUDA. */
VICP_API vicp_status vicp_create(vicp_ctx **out, const vicp_params *params, const vicp_allocator *alloc,
                        void *cuda_stream);

/* Synchronises the stream and frees everything the context allocated. */
VICP_API void vicp_destroy(vicp_ctx *ctx);

/* Rebinds the context to another stream (work already issued stays on the
 * old one, and the internal dilation stream's ordering refers to it:
 * synchronise first). */
VICP_API vicp_status vicp_set_stream(vicp_ctx *ctx, void *cuda_stream);

/* Grid build = Alg. 1 + Alg. 2: quantise every target point into its voxel
 * key (x fastest), count points per voxel with warp-aggregated atomics,
 * exclusive-scan the counts into segment offsets (the paper's MOC, done on
 * the GPU by a single-pass decoupled-lookback scan instead of serially on
 * the host), and scatter point indices into the CSR store.
 *   target_xyzw: dev, n_target x 4 floats, 16-byte aligned; read only.
 *   n_target >= 1.
 * In auto-grid mode (params.dims[0] <= 0) the bounding box is reduced on the
 * device and read back (this call then synchronises once) unless
 * VICP_FLAG_KEEP_GRID is set and a grid was already fitted.  Target points
 * outside an explicit grid are not stored.  Errors: VICP_ERR_INVALID,
 * VICP_ERR_GRID_TOO_LARGE, VICP_ERR_OOM, VICP_ERR_CUDA. */
VICP_API vicp_status vicp_build_grid(vicp_ctx *ctx, const float *target_xyzw, int32_t n_target);

/* Dilation = Alg. 3 and Sec. 3's description of it: every empty voxel
 * within Manhattan distance `layers` of an occupied voxel receives the
 * occupied root voxel at the smallest distance (ties: smallest voxel index)
 * and that distance as its ring; the result equals `layers` synchronous
 * rounds of six-neighbour propagation.  layers < 0 uses
 * params.dilation_layers; 0 <= layers <= 31.  The dilation depends only on
 * the build's first kernel, so it runs on a second, internal stream,
 * concurrently with the rest of the build; the context's stream then waits
 * for it, so work issued on that stream after this call sees its results.
 * Errors: VICP_ERR_STATE before a build, VICP_ERR_INVALID, VICP_ERR_CUDA. */
VICP_API vicp_status vicp_dilate(vicp_ctx *ctx, int32_t layers);

/* NNS = Alg. 4: transform each source point by the pose (entries rounded to
 * float), quantise it, follow its voxel's root label and search that root
 * voxel's points; a point outside the grid or in an unlabelled voxel takes
 * the global search over all target points (exact nearest neighbour).
 * Squared distance ((dx*dx + dy*dy) + dz*dz) in float; ties go to the smaller
 * target index.
 *   src_xyzw: dev, n_src x 4, 16-byte aligned.  pose_dev: dev, 16 doubles.
 *   nn_out: dev int32[n_src] target index.  d2_out: dev float[n_src].
 *   n_fallback_out: dev int32, number of global searches; may be NULL.
 * Needs vicp_build_grid and vicp_dilate first (VICP_ERR_STATE). */
VICP_API vicp_status vicp_correspond(vicp_ctx *ctx, const float *src_xyzw, int32_t n_src,
                            const double *pose_dev, int32_t *nn_out, float *d2_out,
                            int32_t *n_fallback_out);

/* One ICP iteration on the built grid (Sec. 2.1, Eq. 1): NNS as above, the
 * centroids and cross-covariance reduced deterministically, the optimal
 * rotation (Horn's quaternion method) and translation, and pose <- dT * pose
 * in place (FP64).  The sums and the solve run in double-float arithmetic
 * (about 48 significant bits on the FP32 pipes), or in FP64 when the
 * context was created with VICP_FLAG_FP64_SOLVE.
 *   pose_dev: dev, 16 doubles, read and written.  rmse_dev: dev double, the
 *   RMSE of this iteration's correspondences (before the update); may be
 *   NULL.  Degenerate geometry (rank(H) < 2) leaves the pose unchanged and
 *   is reported as VICP_ERR_DEGENERATE by the next synchronising call. */
VICP_API vicp_status vicp_step(vicp_ctx *ctx, const float *src_xyzw, int32_t n_src, double *pose_dev,
                      double *rmse_dev);

/* Full registration, synchronous: build the grid on the target, dilate,
 * then up to params.max_iters iterations of vicp_step, stopping early once
 * |rmse_k - rmse_(k-1)| < params.rmse_eps (Sec. 4.1).  The stopping test
 * runs on the device; the host reads the result once at the end.
 *   src_xyzw / tgt_xyzw: dev, 16-byte aligned.
 *   pose_host: in = initial pose, out = result (left at the last good pose
 *   on VICP_ERR_DEGENERATE).  iters_out, rmse_out: host, may be NULL
 *   (iterations applied; RMSE of the last iteration). */
VICP_API vicp_status vicp_register(vicp_ctx *ctx, const float *src_xyzw, int32_t n_src,
                          const float *tgt_xyzw, int32_t n_tgt, double pose_host[16],
                          int32_t *iters_out, double *rmse_out);

/* Graph replay of vicp_register and vicp_register_host: the second call in
 * a row with the same clouds (the same pointers and sizes) and parameters is
 * captured into a CUDA graph -- the copies, every kernel of the builds, the
 * dilations and the iterations, and the read-back -- and that call and
 * every later one with the same arguments replay the graph (one launch)
 * instead of launching the kernels one by one.  The contents of the clouds
 * and the initial pose are read anew at every replay, and the results equal
 * those of the launches one by one bit for bit.  Only where nothing in the
 * call synchronises or allocates: the dense grid, an explicit grid or
 * VICP_FLAG_KEEP_GRID after the grid was fitted, kernel timing off, and not
 * VICP_FLAG_NO_GRAPH.  If a capture fails (vicp_register_host with pageable
 * host clouds, for one) the context launches directly from then on. */

/* vicp_register with both clouds in host memory: copies them to
 * context-owned device buffers -- the target on the context's stream before
 * the grid build, the source on an internal copy stream while the grid is
 * built (ordered after all work issued earlier on the context's stream; the
 * first search waits for it).  Host buffers should be pinned for the copies
 * to run asynchronously.  A replayed call (above) with a page-locked target
 * (cudaHostAlloc / cudaHostRegister, 16-byte aligned) does not copy it
 * first: the first build's histogram reads the points through their
 * device-mapped address and stores the device copy, and the source cloud's
 * copy follows that histogram.  Either way both buffers are read during the
 * call only and must not change until it returns. */
VICP_API vicp_status vicp_register_host(vicp_ctx *ctx, const float *src_xyzw_host, int32_t n_src,
                               const float *tgt_xyzw_host, int32_t n_tgt, double pose_host[16],
                               int32_t *iters_out, double *rmse_out);

/* Synchronous: waits for the stream and fills *out (n_stored is read back).
 * The build itself writes only the offsets its searches read (those of the
 * occupied voxels and the ones just past them, every 32nd, and offsets[V]);
 * the first vicp_get_grid or vicp_memory_report after a build completes the
 * array (one kernel on the context's stream), so out->offsets holds all
 * V + 1 entries. */
VICP_API vicp_status vicp_get_grid(vicp_ctx *ctx, vicp_grid_view *out);

/* The sparse (hashed) grid, a context created with VICP_FLAG_SPARSE_GRID.
 * The paper's dynamic assignment (Sec. 3) makes the point store compact but
 * keeps per-voxel count / address words for every voxel (Table 1 note 1),
 * and VANICP's dilation labels every voxel; at fine voxel sizes those dense
 * arrays dominate the memory (Sec. 2.2's argument, one level up).  The
 * sparse grid keeps, instead, only
 *   - the occupied voxels, in an open-addressing table (voxel key -> slot;
 *     at least 2 n_target slots, so at most half full) whose slots carry the
 *     counts and the segment offsets (an exclusive scan in slot order, so
 *     segments lie in the store in slot order), and
 *   - the labelled voxels (within L of a point), by row segment: a segment
 *     is 32 voxels along x of one row of one plane (voxel x, y, z lies in
 *     segment x/32 + nxb (y + ny z), nxb = ceil(nx / 32)); a second table
 *     holds every segment with a labelled voxel (segment -> the mask of its
 *     labelled voxels, bit x mod 32, and the index of its first root), and
 *     the labelled voxels' root voxel keys lie segment after segment in a
 *     root array, a segment's in the order of their x (the ring is the
 *     Manhattan distance between a voxel and its root).  The table is sized
 *     after a dilation to keep it at most half full, the root array to hold
 *     every label (vicp_dilate synchronises once: pass Z counts them, and
 *     what was too small is grown and the dilation run again).  Under
 *     VICP_FLAG_KEEP_GRID the sizes found by the first dilation of the kept
 *     grid are kept and later dilations run without that synchronisation; a
 *     cloud that then needs more room is reported by the next synchronising
 *     call as VICP_ERR_STATE (its labels are incomplete), and the next
 *     vicp_dilate checks and grows them again.
 * Keys, CSR ids and points, the occupancy bits, the dilation's pass-Y words
 * and the global search's brick level are as in the dense grid, and every
 * search result equals the dense grid's.  Not available with the
 * fixed-capacity store (VICP_ERR_STATE) or vicp_get_grid.
 * All pointers are device pointers owned by the context, valid until the
 * next build or vicp_destroy. */
typedef struct vicp_sparse_view {
    float origin[3];
    float voxel_size;
    float inv_voxel_size;
    int32_t dims[3];
    int64_t n_voxels;
    int32_t n_target;
    int32_t n_stored;
    int32_t dilation_layers;           /* -1 before any dilation */
    int64_t occupied_slots;            /* slots of the occupied-voxel table (a power of two) */
    const uint32_t *occupied_keys;     /* [occupied_slots] voxel key, 0xffffffff for an empty slot */
    const uint32_t *occupied_offsets;  /* [occupied_slots + 1]: the points of the voxel in slot s are
                                          ids[occupied_offsets[s] .. occupied_offsets[s + 1]); valid for
                                          occupied slots s (and s + 1), and [occupied_slots] = n_stored */
    int64_t labelled_slots;            /* slots of the labelled-segment table (0 before a dilation) */
    const uint32_t *labelled_keys;     /* [labelled_slots] segment, 0xffffffff for an empty slot */
    const uint32_t *labelled_segments; /* [labelled_slots x 2]: the segment's label mask (bit i: voxel
                                          32 (segment mod nxb) + i of its row) and the index in
                                          labelled_root of its first labelled voxel's root */
    const int32_t *labelled_root;      /* [labelled_voxels] root voxel keys, segment by segment */
    int64_t labelled_voxels;           /* labelled voxels */
    int64_t labelled_segment_count;    /* entries in the labelled-segment table */
    const int32_t *keys;               /* [n_target] voxel key of each target point, -1 outside */
    const int32_t *ids;                /* [n_stored] point indices grouped by voxel */
    const float *csr_points;           /* [n_stored x 4] x, y, z of ids[k]; w holds the bits of ids[k] */
    const uint32_t *occupancy;         /* [ceil(V/32)] bit v set iff voxel v holds a point */
} vicp_sparse_view;

/* Synchronous: the sparse grid of the last build / dilation.  Errors:
 * VICP_ERR_STATE (not a sparse-grid context, or no build). */
VICP_API vicp_status vicp_get_sparse_grid(vicp_ctx *ctx, vicp_sparse_view *out);

/* Synchronous: waits for the stream, returns and clears the device status. */
VICP_API vicp_status vicp_sync(vicp_ctx *ctx);

/* Synchronous: device-memory accounting of the current grid. */
VICP_API vicp_status vicp_memory_report(vicp_ctx *ctx, vicp_memory *out);

/* Kernel timing: while enabled, every kernel launch is bracketed by CUDA
 * events on the context's stream.  vicp_profile_read synchronises, writes
 * per-kernel launch counts and summed milliseconds into arrays of
 * vicp_kernel_count() entries (either may be NULL) and resets the tallies. */
VICP_API vicp_status vicp_profile_enable(vicp_ctx *ctx, int32_t enable);
VICP_API int32_t vicp_kernel_count(void);
VICP_API const char *vicp_kernel_name(int32_t kernel);
VICP_API vicp_status vicp_profile_read(vicp_ctx *ctx, int64_t *launches, double *total_ms);

/* Synchronous: the search work counters; reset != 0 clears them. */
VICP_API vicp_status vicp_read_stats(vicp_ctx *ctx, vicp_stats *out, int32_t reset);

/* Kernels this context has launched since vicp_create. */
VICP_API int64_t vicp_launch_count(const vicp_ctx *ctx);

/* 1 if the last vicp_register / vicp_register_host call on this context
 * replayed its captured CUDA graph, 0 if it launched its kernels one by one
 * (or no registration has run yet); -1 for a NULL context. */
VICP_API int32_t vicp_graph_replayed(const vicp_ctx *ctx);

/* Text of the last error on this context ("" if none). */
VICP_API const char *vicp_last_error(const vicp_ctx *ctx);

/* Fixed-capacity voxel store, a measured alternative to the CSR store: each
 * voxel owns `capacity` slots at v * capacity (direct addressing, the
 * monolithic layout whose memory cost the paper's dynamic assignment
 * removes, Sec. 2.2 and Sec. 3), filled by one scatter with no histogram and
 * no scan; points past a voxel's capacity are dropped and counted.  It
 * replaces the voxel store only: the geometry, the dilation labels and the
 * global search's brick level are those of the context's CSR build.
 *   vicp_fixed_build: target_xyzw / n must be the last vicp_build_grid's
 *     target (else VICP_ERR_STATE); capacity >= 1 and V * capacity < 2^32;
 *     allocates V * capacity * 16 + 4V bytes (slots of x, y, z, index and
 *     fill counts).  Synchronous: overflow_out (host, may be NULL) = points
 *     dropped; store_bytes_out (host, may be NULL) = bytes of the store.
 *   vicp_fixed_correspond: as vicp_correspond, with the localised search
 *     reading the fixed store; with capacity >= the largest voxel count the
 *     results equal vicp_correspond's.  Needs vicp_dilate after the CSR build.
 * Errors: VICP_ERR_INVALID, VICP_ERR_STATE, VICP_ERR_GRID_TOO_LARGE,
 * VICP_ERR_OOM, VICP_ERR_CUDA. */
VICP_API vicp_status vicp_fixed_build(vicp_ctx *ctx, const float *target_xyzw, int32_t n, int32_t capacity,
                                      uint32_t *overflow_out, uint64_t *store_bytes_out);
VICP_API vicp_status vicp_fixed_correspond(vicp_ctx *ctx, const float *src_xyzw, int32_t n_src,
                                           const double *pose_dev, int32_t *nn_out, float *d2_out,
                                           int32_t *n_fallback_out);
/* Read-only view of the fixed-capacity store of the last vicp_fixed_build
 * (Sec. 2.2's monolithic layout): *slots_out (dev, V * capacity x 4 floats:
 * voxel v's slots at v * capacity, each x, y, z and the bits of the target
 * index in w), *fill_out (dev uint32[V]: points that fell into voxel v; the
 * first min(fill, capacity) slots are stored, which of a full voxel's points
 * they are depends on the order the scatter's atomics ran in), and
 * *capacity_out.  Any output may be NULL.  Valid until the next
 * vicp_fixed_build or vicp_destroy.  Synchronous.  Errors: VICP_ERR_STATE
 * before vicp_fixed_build. */
VICP_API vicp_status vicp_fixed_view(vicp_ctx *ctx, const float **slots_out, const uint32_t **fill_out,
                                     int32_t *capacity_out);

/* Voxel keys and segment offsets of a target cloud -- the keys and offsets
 * steps of vicp_build_grid -- computed WITHOUT allocating any device memory.
 * The paper has no counterpart: it is for callers that may not allocate at
 * the point of the call, such as a loop that has committed a fixed
 * device-memory plan (cudaMalloc can block and synchronise the device) or a
 * plug-in whose host framework owns all device memory.  No context is
 * needed.
 *
 * Working memory is one static device array inside the library (about
 * 70 MiB on every GPU the library is loaded on, held until the process
 * exits); the grid is therefore limited to VICP_STATIC_MAX_VOXELS voxels and
 * VICP_STATIC_MAX_BRICK_SLOTS 8^3-voxel brick slots (bricks padded to whole
 * 4x4x4-brick groups per axis); larger grids return VICP_ERR_GRID_TOO_LARGE.
 * Every call, on any stream or host thread, shares that one array: calls on
 * one device that overlap in time race and give wrong results, so callers
 * must serialise them.  Each call clears the parts that must start at zero.
 * The first call on a device looks up the array's device address (once per
 * device, with that device current).  The address is kept for the life of
 * the process, so the library must not be used on a device after
 * cudaDeviceReset (or any other teardown of the device's primary context)
 * in the same process.  The call
 * synchronises `cuda_stream` before returning, and runs on the device that
 * is current when it is called: `cuda_stream`, the target and the outputs
 * must belong to that device.
 *   target_xyzw: dev, n x 4 floats (w ignored), 16-byte aligned; n >= 1.
 *   origin[3], voxel_size, dims[3]: host; the explicit grid (as
 *     params.origin / voxel_size / dims of vicp_build_grid), dims >= 1.
 *   keys_out: dev int32[n], 4-byte aligned; key x + nx*(y + ny*z) of each
 *     point, -1 outside the grid.
 *   offsets_out: dev uint32[V + 1], 16-byte aligned, V = dims product;
 *     exclusive prefix sum of the per-voxel counts, offsets_out[V] = points
 *     inside the grid.  Equal to vicp_get_grid's keys and offsets after
 *     vicp_build_grid with the same grid.
 * Errors: VICP_ERR_INVALID (NULL or misaligned pointer, n < 1, bad grid),
 * VICP_ERR_GRID_TOO_LARGE, VICP_ERR_CUDA. */
#define VICP_STATIC_MAX_VOXELS (1ll << 24)
#define VICP_STATIC_MAX_BRICK_SLOTS (1ll << 20)
VICP_API vicp_status vicp_offsets_static(const float *target_xyzw, int32_t n, const float origin[3],
                                         float voxel_size, const int32_t dims[3], int32_t *keys_out,
                                         uint32_t *offsets_out, void *cuda_stream);

/* ---------------------------------------------------------------------- */
/* Batched registration: many independent (source, target) pairs of uneven
 * sizes registered together.  The pairs' clouds are pooled (concatenated in
 * pair order: pair k's points follow pair k-1's), every pair gets its own
 * grid fitted to its target exactly as vicp_build_grid fits one, and all
 * pairs' grids are built by a few launches over the pooled store (one
 * exclusive scan over all pairs' counts gives every pair's segments).  Each
 * ICP iteration of all pairs is ONE persistent cooperative launch: the
 * localised search of Alg. 4 for every (pair, tile) item, the global
 * searches and dense segments shared out over all warps, and per pair the
 * deterministic reduction and the update of Eq. 1.  The paper registers one
 * pair at a time; this extends its kernels (Algs. 1-4) to many pairs.  The
 * result of each pair is that of vicp_register on the pair alone up to the
 * rounding order of the reduction (the sums are split differently).  */

typedef struct vicp_batch vicp_batch;

#define VICP_BATCH_MAX_PAIRS 65536
#define VICP_BATCH_SHAPES 7                     /* iteration kernel shapes (see vicp_batch_shape_info) */
#define VICP_BATCH_FLAG_NO_GRAPH (1u << 0)      /* launch the iterations one by one instead of
                                                   replaying them as a captured CUDA graph */
#define VICP_BATCH_FLAG_TEST_BARRIER_TIMEOUT (1u << 1) /* test hook: block 0 of the iteration kernel
                                                   leaves before the first grid barrier, so the
                                                   other blocks' bounded wait (1 s) runs out and
                                                   the call returns VICP_ERR_TIMEOUT */
#define VICP_BATCH_FLAG_FP64 (1u << 2)          /* per-pair centroid / cross-covariance sums and
                                                   the rigid solve in FP64 (as VICP_FLAG_FP64_SOLVE);
                                                   default: double-float */

typedef struct vicp_batch_params {
    int32_t dilation_layers;  /* L of every pair, 0..31 */
    int32_t max_iters;        /* iterations of vicp_batch_register */
    double rmse_eps;          /* a pair stops once |rmse_k - rmse_(k-1)| < rmse_eps; <= 0: never */
    int32_t shape;            /* iteration kernel shape 0..VICP_BATCH_SHAPES-1; < 0: the one
                                 vicp_batch_tune chose, else shape 0 */
    uint32_t flags;           /* VICP_BATCH_FLAG_* */
} vicp_batch_params;

/* Fills *p: L = 10, 40 iterations, rmse_eps = 0 (fixed iteration count),
 * shape -1, flags 0. */
VICP_API void vicp_batch_default_params(vicp_batch_params *p);

/* Threads per block, source points per thread and resident blocks (on the
 * current device; of the double-float variant) of iteration kernel shape
 * `shape`.  Errors: VICP_ERR_INVALID. */
VICP_API vicp_status vicp_batch_shape_info(int32_t shape, int32_t *threads, int32_t *points_per_thread,
                                           int32_t *resident_blocks);

/* Creates a batch context on the current device and `cuda_stream`
 * (NULL = legacy default stream); `alloc` as for vicp_create. */
VICP_API vicp_status vicp_batch_create(vicp_batch **out, const vicp_batch_params *params,
                                       const vicp_allocator *alloc, void *cuda_stream);
VICP_API void vicp_batch_destroy(vicp_batch *b);

/* Builds and dilates the grids of n_pairs targets (Alg. 1-3 per pair).
 *   tgt_xyzw: dev, pooled targets, sum(n_tgt) x 4 floats, 16-byte aligned;
 *     must stay valid and unchanged until the next build (the searches read it).
 *   n_tgt: host int32[n_pairs], each >= 1; sum < 2^31.
 *   voxel_size: host float[n_pairs] or NULL; where > 0 it is the pair's
 *     voxel edge, else h = target extent / grid_divisions[k].
 *   grid_divisions: host int32[n_pairs] (>= 1 where used) or NULL.
 * Synchronises once (the bounding boxes are read back).  Errors:
 * VICP_ERR_INVALID, VICP_ERR_GRID_TOO_LARGE (a pair's grid, or all pairs'
 * voxels together, reach 2^31 - 1), VICP_ERR_OOM, VICP_ERR_CUDA. */
VICP_API vicp_status vicp_batch_build(vicp_batch *b, int32_t n_pairs, const float *tgt_xyzw, const int32_t *n_tgt,
                                      const float *voxel_size, const int32_t *grid_divisions);

/* Registers every pair on the built grids, synchronously: up to
 * params.max_iters iterations, each pair stopping on its own RMSE test.
 *   src_xyzw: dev, pooled sources (pair order), 16-byte aligned.
 *   n_src: host int32[n_pairs], each >= 1.
 *   poses: host double[n_pairs * 16], row-major 4x4 each; in = initial,
 *     out = result (a degenerate pair keeps its last good pose).
 *   iters_out (int32[n_pairs]), rmse_out (double[n_pairs], RMSE of the last
 *   iteration), status_out (int32[n_pairs]: VICP_OK or VICP_ERR_DEGENERATE):
 *   host, each may be NULL.
 * Errors: VICP_ERR_STATE before a build, VICP_ERR_INVALID, VICP_ERR_OOM,
 * VICP_ERR_TIMEOUT (a grid barrier gave up), VICP_ERR_CUDA; with status_out
 * NULL, VICP_ERR_DEGENERATE if any pair was degenerate. */
VICP_API vicp_status vicp_batch_register(vicp_batch *b, const float *src_xyzw, const int32_t *n_src, double *poses,
                                         int32_t *iters_out, double *rmse_out, int32_t *status_out);

/* Build + register with every cloud in host memory (copied to
 * context-owned device buffers on the context's stream first). */
VICP_API vicp_status vicp_batch_register_host(vicp_batch *b, int32_t n_pairs, const float *src_xyzw_host,
                                              const int32_t *n_src, const float *tgt_xyzw_host,
                                              const int32_t *n_tgt, const float *voxel_size,
                                              const int32_t *grid_divisions, double *poses, int32_t *iters_out,
                                              double *rmse_out, int32_t *status_out);

/* NNS of every pair (Alg. 4, as vicp_correspond per pair) at the given
 * poses, without an update.
 *   src_xyzw, n_src: as for vicp_batch_register.  poses_dev: dev,
 *   double[n_pairs * 16].  nn_out: dev int32[sum n_src], the pair's own
 *   target index of each source point; d2_out: dev float[sum n_src]. */
VICP_API vicp_status vicp_batch_correspond(vicp_batch *b, const float *src_xyzw, const int32_t *n_src,
                                           const double *poses_dev, int32_t *nn_out, float *d2_out);

/* Autotuner: runs `iters` iterations of every pair from `poses` (host, as
 * for vicp_batch_register; left unchanged) with each iteration kernel shape,
 * timing each with CUDA events (best of `trials`), and keeps the fastest for
 * later registrations whose params.shape < 0.  shape_out (host int32) and
 * ms_out (host float[VICP_BATCH_SHAPES], -1 for a shape that cannot run)
 * may be NULL. */
VICP_API vicp_status vicp_batch_tune(vicp_batch *b, const float *src_xyzw, const int32_t *n_src,
                                     const double *poses, int32_t iters, int32_t trials, int32_t *shape_out,
                                     float *ms_out);

/* Pair k's grid after vicp_batch_build, as vicp_get_grid gives a single
 * grid, with one difference: offsets hold positions in the POOLED store, so
 * offsets[0] is the pair's first position (not 0) and ids / csr_points point
 * at the start of the pooled store; ids and the csr w fields hold the pair's
 * own target indices.  As with vicp_get_grid, the first call after a build
 * completes the pooled offsets array (one kernel).  Synchronous.  Errors:
 * VICP_ERR_STATE, VICP_ERR_INVALID. */
VICP_API vicp_status vicp_batch_pair_grid(vicp_batch *b, int32_t pair, vicp_grid_view *out);

/* Synchronous: device bytes held by the batch context now and at peak,
 * and the search work counters (reset != 0 clears them); either may be NULL. */
VICP_API vicp_status vicp_batch_report(vicp_batch *b, uint64_t *current_bytes, uint64_t *peak_bytes,
                                       vicp_stats *stats, int32_t reset);

/* Replaces params.flags of the context (for example to clear a test hook);
 * takes effect at the next call. */
VICP_API vicp_status vicp_batch_set_flags(vicp_batch *b, uint32_t flags);

/* Kernels the batch context has launched since vicp_batch_create (a graph
 * replay counts its kernels). */
VICP_API int64_t vicp_batch_launch_count(const vicp_batch *b);

/* How the last registration's iterations ran: 1 replayed from the captured
 * CUDA graph, 0 launched one by one (VICP_BATCH_FLAG_NO_GRAPH, or the
 * capture of the cooperative launches failed once on this context), -1 no
 * registration yet (or b NULL). */
VICP_API int32_t vicp_batch_graph_replayed(const vicp_batch *b);

/* Text of the last error on this batch context ("" if none). */
VICP_API const char *vicp_batch_last_error(const vicp_batch *b);

/* ---------------------------------------------------------------------- */
/* Differentiable loss.  The point-to-point objective of Eq. 1 as a loss per
 * pair, L_k = (1/M) sum_i |T p_i - q_nn(i)|^2, at pose T with the
 * correspondences nn of the localised NNS held fixed (they carry no
 * gradient).  Poses are parameterised in se(3) with a left perturbation:
 * T = Exp(xi) T0, xi = (rho, phi), translation part first.  The paper
 * minimises Eq. 1 by the closed-form update only; the gradients serve
 * callers that put the loss into a larger differentiable objective. */

/* T = Exp(xi) T0 for n poses (FP64, on the device, stream-ordered).
 *   xi_dev: dev double[n * 6]; T0_dev, T_dev: dev double[n * 16] row-major.
 * Errors: VICP_ERR_INVALID, VICP_ERR_CUDA. */
VICP_API vicp_status vicp_se3_exp(int32_t n, const double *xi_dev, const double *T0_dev, double *T_dev,
                                  void *cuda_stream);

/* out = J(xi)^T g for n poses, J the 6x6 left Jacobian of SE(3)
 * (Exp(xi + e) = Exp(J(xi) e) Exp(xi) to first order): turns the
 * left-perturbation gradient at Exp(xi) T0 into the gradient in xi.
 *   xi_dev, g_dev, out_dev: dev double[n * 6]. */
VICP_API vicp_status vicp_se3_left_jacobian_t(int32_t n, const double *xi_dev, const double *g_dev, double *out_dev,
                                              void *cuda_stream);

/* Loss and gradients of every pair of a built batch (stream-ordered, no
 * synchronisation).
 *   src_xyzw, n_src: the pooled sources (as for vicp_batch_register).
 *   poses_dev: dev double[n_pairs * 16], the poses T.
 *   nn_dev: dev int32[sum n_src], each source point's target index within
 *     its pair (vicp_batch_correspond at the same poses).
 *   dloss_dev: dev double[n_pairs], weights of the pairs' losses in the
 *     gradients (the incoming gradient); NULL = all 1.
 *   loss_out: dev double[n_pairs].
 *   grad_pose_out: dev double[n_pairs * 6] or NULL: dloss_k * dL_k/dd at
 *     d = 0 for T <- Exp(d) T: (2/M) (sum r_i, sum s_i x r_i) with
 *     s_i = T p_i, r_i = s_i - q_nn(i).
 *   grad_src_out: dev float[sum n_src * 4], 16-byte aligned, or NULL:
 *     dloss_k (2/M) R^T r_i in x, y, z and 0 in w.
 * s_i and r_i are formed in double-float arithmetic from the FP64 pose; the
 * sums are double-float and deterministic. */
VICP_API vicp_status vicp_batch_loss(vicp_batch *b, const float *src_xyzw, const int32_t *n_src,
                                     const double *poses_dev, const int32_t *nn_dev, const double *dloss_dev,
                                     double *loss_out, double *grad_pose_out, float *grad_src_out);

/* Voxel occupancy histogram (VOH, Alg. 1 GPU part) as a standalone
 * ablation of two designs; no allocation, stream-ordered (no
 * synchronisation).  method VICP_HIST_WARP_AGGREGATED: lanes of a warp with
 * the same voxel add their group size with one atomic (the design the grid
 * build uses).  method VICP_HIST_SHARED_HASH: the paper's per-block
 * shared-memory hash table (one slot per thread, slot = key modulo the
 * block size, linear probing by atomicCAS, count by atomicAdd on the same
 * packed word, one global atomicAdd per used slot), with the word widened to
 * [key + 1 : 32 | count : 32] so that voxel 0 is not the empty word and any
 * grid size fits (the paper's 16-bit key field limits grids to 2^16 voxels).
 *   target_xyzw: dev, n x 4 floats, 16-byte aligned; n >= 1.
 *   origin[3], voxel_size, dims[3]: host, the explicit grid, V < 2^31 - 1.
 *   keys_out: dev int32[n], key x + nx*(y + ny*z) of each point, -1 outside.
 *   counts_out: dev uint32[V]; the call ADDS the counts (pass zeros for a
 *     histogram).
 * Errors: VICP_ERR_INVALID, VICP_ERR_GRID_TOO_LARGE, VICP_ERR_CUDA. */
#define VICP_HIST_WARP_AGGREGATED 0
#define VICP_HIST_SHARED_HASH 1
VICP_API vicp_status vicp_voxel_histogram(const float *target_xyzw, int32_t n, const float origin[3],
                                          float voxel_size, const int32_t dims[3], int32_t method,
                                          int32_t *keys_out, uint32_t *counts_out, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* VICP_H */
