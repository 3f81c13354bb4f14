// vicp_batch.h -- batched registration: many independent (source, target)
// pairs of uneven sizes registered together over one pooled store.  Device
// layouts and the host-side launchers of vicp_batch.cu.
//
// Pooling.  The pairs' target clouds are concatenated (pair p's n_tgt points
// start at tbase), and so are the source clouds (sbase).  Each pair has its
// own voxel grid, fitted to its target like a single-pair grid; the grids'
// per-voxel arrays are concatenated too (pair p's V voxels start at vbase, a
// multiple of 32 so that no occupancy word is shared by two pairs), and so
// are the brick slots (bbase) and super-brick records (sbbase).  One
// exclusive scan over the concatenated counts gives every pair's segment
// offsets at once, as positions in one pooled CSR store.  Inside a pair,
// voxel keys, root labels and target indices are the pair's own (local),
// exactly as in a single-pair grid.
#pragma once

#include "vicp_device.cuh"

namespace vicp {

// Per-pair descriptor (written by the host; read-only on the device).
struct BatchPair {
    GridGeom g;            // the pair's grid
    long long vbase;       // first voxel in the pooled voxel arrays (multiple of 32)
    int tbase, n_tgt;      // target points [tbase, tbase + n_tgt) of the pooled target array
    int sbase, n_src;      // source points [sbase, sbase + n_src) of the pooled source array
    int bbase;             // first brick slot (pooled brick arrays)
    int sbbase;            // first super-brick record
    int uxy, uz;           // first dilation units (pass XY, pass Z)
    int item0, n_items;    // the pair's iteration items [item0, item0 + n_items)
    float cx, cy, cz;      // reduction centre: the grid centre rounded to float
    int pad;
};
static_assert(sizeof(BatchPair) == 128, "BatchPair layout");

// Per-pair device state.
struct BatchState {
    int n_bricks;          // brick scan: non-empty bricks
    int n_super;           // brick boxes: super-brick records
    int n_outside;         // scatter: target points outside the grid
    unsigned items_done;   // iteration: items reduced (the last one solves and resets it)
    int stop;              // 1 once converged or degenerate
    int iters;             // iterations applied
    unsigned err;          // DEVERR_* bits of this pair
    int pad;
    double prev_rmse;
    double last_rmse;
};
static_assert(sizeof(BatchState) == 48, "BatchState layout");

// A tile of one pair's points: pooled indices [i0, i1), local index of i0.
struct BatchItem {
    int pair, i0, i1, l0;
};

constexpr int BATCH_TILE = 256;          // target points per build item (one block)
constexpr int BATCH_SMEM_PAIRS = 2048;   // unit-start tables up to this many pairs go to shared memory

// Iteration kernel shapes the autotuner chooses from: threads per block,
// source points per thread (the item tile is their product) and the blocks
// per SM the registers are budgeted for.
struct BatchShape {
    int threads, ppt, min_blocks;
};
constexpr int BATCH_N_SHAPES = 7;
extern const BatchShape BATCH_SHAPES[BATCH_N_SHAPES];

// Arguments of one iteration of all pairs.
struct BatchIterArgs {
    const float4 *src;          // pooled source points
    const float4 *tgt;          // pooled target points
    const BatchPair *pairs;
    BatchState *state;
    double *pose;               // [P][16] row-major 4x4, FP64
    const BatchItem *items;     // source tiles, grouped by pair
    int n_items;
    int n_pairs;
    int n_stored;               // points in the pooled CSR store
    const int *root;            // pooled, pair-local voxel labels
    const unsigned *off;        // pooled offsets (positions in the CSR store)
    const float4 *csr;          // pooled CSR points, w = pair-local target index
    const float4 *bpts;         // pooled brick-ordered points, w = pair-local target index
    const float4 *bbox;         // pooled brick records
    const float4 *sb_box;       // pooled super-brick records
    const int *outside;         // pooled (at tbase) lists of target points outside each grid
    int *nn;                    // [M] pair-local target index of each source point
    float *d2;                  // [M] squared distance
    int2 *fb_list;              // global-search queries (pair, pooled source index)
    int4 *hv_list;              // dense segments (pair, pooled source index, begin, end)
    int list_cap;               // capacity of each list (M)
    float2 *partials;           // [n_items][16] double-float sums per item
    DevCtl *ctl;                // fb_count, hv_count, barrier, stats, err
    double eps;                 // stopping threshold on the RMSE difference (<= 0: never)
    int search_only;            // 1: phases 1-2 only (nn, d2), no reduction or update
    int test_leave_early;       // test hook: block 0 leaves before the first barrier
};

cudaError_t launch_batch_bbox(const float4 *pts, const BatchItem *items, int n_items, int P, unsigned *bbox,
                              cudaStream_t st);
cudaError_t launch_batch_histogram(const float4 *pts, const BatchItem *items, int n_items, const BatchPair *pairs,
                                   int *keys, unsigned *counts, unsigned *bcounts, unsigned *occ, unsigned *tile_sum,
                                   DevCtl *ctl, cudaStream_t st);
cudaError_t launch_batch_brick_scan(const unsigned *bcounts, const BatchPair *pairs, int P, const unsigned *off,
                                    unsigned *boff, int *list, uint2 *range, int *bslot, uint4 *boxord,
                                    BatchState *state, cudaStream_t st);
cudaError_t launch_batch_scatter(const float4 *pts, const int *keys, const BatchItem *items, int n_items,
                                 const BatchPair *pairs, int n_total, const unsigned *off, unsigned *counts,
                                 const unsigned *boff, unsigned *bcounts, const int *bslot, unsigned *boxord, int *ids,
                                 float4 *csr, float4 *bpts, int *outside, unsigned *tile_sum, int n_tiles,
                                 BatchState *state, DevCtl *ctl, cudaStream_t st);
cudaError_t launch_batch_brick_boxes(const uint4 *boxord, const int *list, const uint2 *range,
                                     const BatchPair *pairs, int P, BatchState *state, float4 *box, float4 *sb_box,
                                     cudaStream_t st);
// ustart_xy / ustart_z: [P + 1] first dilation unit of each pair (and the total).
cudaError_t launch_batch_dilate(const unsigned *occ, const BatchPair *pairs, int P, const int *ustart_xy,
                                const int *ustart_z, int L, void *inter, unsigned *rows, unsigned char *dirty,
                                int *root, unsigned char *ring, cudaStream_t st);
// Resident blocks of the iteration kernel of a shape (0 if it cannot run);
// f64: the variant with FP64 sums and solve.
int batch_iter_blocks(int shape, bool f64);
// One iteration of every pair (or the search alone): a cooperative
// persistent launch of `blocks` blocks (<= batch_iter_blocks(shape, f64)).
cudaError_t launch_batch_iter(int shape, bool f64, int blocks, const BatchIterArgs &a, cudaStream_t st);

// Differentiable loss (vicp_diff.cu): SE(3) exponential T = Exp(xi) T0 and
// J(xi)^T g (J the left Jacobian), one thread per pose; the loss of Eq. 1
// per pair with its left-perturbation and per-point gradients.
cudaError_t launch_se3_exp(int n, const double *xi, const double *T0, double *T, cudaStream_t st);
cudaError_t launch_se3_jlt(int n, const double *xi, const double *g, double *out, cudaStream_t st);
cudaError_t launch_batch_loss(const float4 *src, const float4 *tgt, const BatchPair *pairs, BatchState *state,
                              const BatchItem *items, int n_items, const double *pose, const int *nn,
                              const double *dloss, float2 *partials, double *loss_out, double *grad_pose,
                              float4 *grad_src, DevCtl *ctl, cudaStream_t st);

}  // namespace vicp
