// vicp_launch.h -- host-side launchers of the library's kernels, called by the
// C ABI runtime (vicp_api.cu).  Each returns the launch's cudaError_t.
#pragma once

#include <utility>

#include "vicp_device.cuh"

namespace vicp {

// Launch with programmatic stream serialisation allowed (the kernel itself
// waits for its predecessor in pdl_begin()).
template <typename... KArgs, typename... Args>
inline cudaError_t launch_kernel(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                                 Args &&...args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// Kernel identifiers for launch accounting and event timing.
enum KernelId {
    K_BBOX = 0,
    K_HISTOGRAM,
    K_SCAN,
    K_SCATTER,
    K_BRICK_SCAN,
    K_DILATE,
    K_CORRESPOND,
    K_FALLBACK,
    K_REDUCE_SOLVE,
    K_MAXCOUNT,
    K_FIXED_SCATTER,
    K_FIXED_CORRESPOND,
    K_OFFSETS_FILL,
    K_REDUCE_SOLVE_F64,
    K_COUNT
};
const char *kernel_name(int k);

// Scan tiling (voxels per CTA, 32 per thread) -- sizes the descriptor array
// and the per-tile sums.
constexpr int SCAN_TILE = 16384;
// Reduction blocks of one ICP iteration (two per SM) -- sizes the partial sums.
constexpr int REDUCE_MAX_BLOCKS = 1024;
constexpr int REDUCE_VALUES = 16;
// Largest dilation depth L the kernels support.
constexpr int DILATE_MAX_L = 31;

inline long long scan_tiles(long long V) { return (V + SCAN_TILE - 1) / SCAN_TILE; }
inline long long occ_words(long long V) { return (V + 31) / 32 + 2; }   // +2: window reads
inline int reduce_blocks(int m, int sms)
{
    const int cap = 2 * sms < REDUCE_MAX_BLOCKS ? 2 * sms : REDUCE_MAX_BLOCKS;
    const int b = (m + 255) / 256;
    return b < 1 ? 1 : (b > cap ? cap : b);
}

cudaError_t launch_bbox(const float4 *pts, int n, unsigned *bbox6, cudaStream_t st);
// occ must hold zeros (the previous build's scatter clears it).
// sb_left and boxk (may be null): per super-brick, its non-empty bricks are
// counted up (the scatter counts them down again); per brick key, 8 words of
// bounds are merged into boxk (all ones before the build).  after_solve:
// the kernel launched just before it on `st` is the reduction + solve, and
// the histogram does not wait for it (any other predecessor: it waits).
// ho (the sparse grid; null: dense): counts, tile_sum and socc are indexed
// by the voxel's slot in the occupied-voxel table ho, and pslot[j] receives
// point j's slot (-1 outside the grid); occ is still indexed by voxel key.
// copy_out (may be null): pts is a page-locked host cloud (its device-mapped
// address), and every point is also stored to copy_out[j] (device memory),
// so that the cloud crosses the host link once, inside the histogram.
cudaError_t launch_histogram(const float4 *pts, int n, const GridGeom &g, int *keys, unsigned *counts,
                             unsigned *bcounts, unsigned *occ, unsigned *tile_sum, unsigned *sb_left,
                             unsigned *boxk, DevCtl *ctl, cudaStream_t st, bool after_solve,
                             const HashTable *ho = nullptr, unsigned *socc = nullptr, int *pslot = nullptr,
                             float4 *copy_out = nullptr);
// dense: every off[v]; sparse: only off[v] and off[v + 1] of occupied voxels,
// off[32 k] and off[V] (what the build and the searches read) -- the rest
// is completed by launch_offsets_fill on the same occupancy bits.
cudaError_t launch_scan(const unsigned *counts, const GridGeom &g, unsigned *off, const unsigned *occ,
                        const unsigned *tile_sum, unsigned long long *desc, const DevCtl *ctl, cudaStream_t st,
                        bool dense);
cudaError_t launch_offsets_fill(unsigned *off, const unsigned *occ, long long V, cudaStream_t st);
cudaError_t launch_brick_scan(const unsigned *bcounts, const GridGeom &g, unsigned *boff, int *list, uint2 *range,
                              int *bslot, DevCtl *ctl, cudaStream_t st);
// The scatter also zeroes the tile totals and the occupancy buffer of the
// next build (occ_next, occ_next_words words), writes the brick and
// super-brick float boxes from the histogram's bounds (boxk) and sets the
// next build's whole bound buffer (boxk_next, boxk_next_words words) to all
// ones.  keys index off / counts: voxel keys (dense grid) or the points'
// slots in the occupied-voxel table (sparse grid; n_tiles then counts the
// slots' scan tiles, and the next build's table keys (empty_next, set to
// HASH_EMPTY) and slot occupancy bits (zero_next, zeroed) are reset too).
cudaError_t launch_scatter(const float4 *pts, const int *keys, int n, const GridGeom &g, const unsigned *off,
                           unsigned *counts, const unsigned *boff, unsigned *bcounts, const int *bslot,
                           const unsigned *boxk, unsigned *boxk_next, long long boxk_next_words, const uint2 *range,
                           float4 *box, unsigned *sb_left, float4 *sb_box, int *ids, float4 *csr, float4 *bpts,
                           int *outside, unsigned *tile_sum, unsigned *occ_next, long long occ_next_words,
                           DevCtl *ctl, cudaStream_t st, long long n_tiles = -1, unsigned *empty_next = nullptr,
                           long long empty_next_words = 0, unsigned *zero_next = nullptr,
                           long long zero_next_words = 0);
// keys (may be null): the sparse grid's occupied-voxel table over g.V slots.
cudaError_t launch_maxcount(const unsigned *off, const GridGeom &g, DevCtl *ctl, cudaStream_t st,
                            const unsigned *keys = nullptr);
// Dilation: `inter` holds V words of pass Y (V x 4 bytes suffices for any
// L), `rows` dilate_units(g) 32-bit row masks (neither needs clearing),
// `dirty` dilate_column_units(g) bytes marking the column units whose voxels
// hold labels.  root/ring must hold "unlabelled" (all bytes 0xff) wherever
// `dirty` is 0: clear all three when they are new or the dimensions change.
cudaError_t launch_dilate(const unsigned *occ, const GridGeom &g, int L, void *inter, unsigned *rows,
                          unsigned char *dirty, int *root, unsigned char *ring, cudaStream_t st);
// The sparse grid's dilation: passes X and Y as above (the kernel also sets
// the keys of `labels` to HASH_EMPTY and counts[0 .. B + 2) to zero), then
// pass Z enters every row
// segment (32 voxels along x of one row of one plane) holding labelled
// voxels into `labels` with seg[slot] = (label mask, index of the segment's
// first root), and the labelled voxels' root keys into root[0 .. cap_root),
// segment by segment.  Block b of pass Z writes its segment count to
// counts[b], b < B = dilate_hashed_blocks(g, L); if an insert gave up or the
// roots did not fit, it sets counts[B] to 1 and DEVERR_CAPACITY in *err;
// counts[B + 1] ends as the number of labelled voxels.
cudaError_t launch_dilate_hashed(const unsigned *occ, const GridGeom &g, int L, void *inter, unsigned *rows,
                                 const HashTable &labels, uint2 *seg, int *root, unsigned cap_root, unsigned *counts,
                                 unsigned *err, cudaStream_t st);
// *word &= ~bits, atomically.
cudaError_t launch_clear_bits(unsigned *word, unsigned bits, cudaStream_t st);
int dilate_hashed_blocks(const GridGeom &g, int L);
long long dilate_units(const GridGeom &g);
long long dilate_column_units(const GridGeom &g);
// The localised search lists queries whose root segment is long (with the
// segment) in hv_list / hv_range and queries without a root in fb_list; the
// fallback kernel then answers both lists.
cudaError_t launch_correspond(const float4 *src, int m, const double *pose, const GridGeom &g, const int *root,
                              const unsigned *off, const float4 *csr, int n_cap, int *nn, float *d2,
                              int *fb_list, int *hv_list, uint2 *hv_range, DevCtl *ctl, int honor_stop,
                              cudaStream_t st);
// The localised search on the sparse grid: root labels from the
// labelled-segment table (segment ids in `labelled`, (mask, first root
// index) in lseg, root keys in lroot), segments [off[slot], off[slot + 1])
// by the root's slot in the occupied-voxel table.
cudaError_t launch_correspond_hashed(const float4 *src, int m, const double *pose, const GridGeom &g,
                                     const HashTable &labelled, const uint2 *lseg, const int *lroot,
                                     const HashTable &occupied, const unsigned *off, const float4 *csr, int n_cap,
                                     int *nn, float *d2, int *fb_list, int *hv_list, uint2 *hv_range, DevCtl *ctl,
                                     int honor_stop, cudaStream_t st);
// The localised search over a fixed-capacity store (C slots per voxel at
// v * C, fill counts in count), listing like launch_correspond; the global
// search then takes the slots as its dense-segment store.
cudaError_t launch_correspond_fixed(const float4 *src, int m, const double *pose, const GridGeom &g, const int *root,
                                    const unsigned *count, unsigned C, const float4 *slots, int *nn, float *d2,
                                    int *fb_list, int *hv_list, uint2 *hv_range, DevCtl *ctl, cudaStream_t st);
// Fixed-capacity build (vicp_fixed.cu): count must hold zeros; overflow
// (one word) is added to.
cudaError_t launch_fixed_scatter(const float4 *pts, int n, const GridGeom &g, unsigned C, unsigned *count,
                                 float4 *slots, unsigned *overflow, cudaStream_t st);
cudaError_t launch_fallback(const float4 *src, const double *pose, const float4 *bpts, const float4 *bbox,
                            const float4 *sb_box, const float4 *tgt, int n_tgt, const int *outside, const int *fb_list,
                            const int *hv_list, const uint2 *hv_range, const float4 *csr, DevCtl *ctl, int *nn,
                            float *d2, int m, int honor_stop, cudaStream_t st);
// Standalone voxel histogram (vicp_hist.cu): method 0 warp-aggregated,
// 1 per-block shared-memory hash; adds to counts.
cudaError_t launch_voxel_histogram(const float4 *pts, int n, const GridGeom &g, int method, int *keys,
                                   unsigned *counts, cudaStream_t st);
cudaError_t launch_reduce_solve(const float4 *src, int m, double *pose, const float4 *tgt, int n_tgt, const int *nn,
                                float3 center, float2 *partials, int nparts, double *rmse_out, DevCtl *ctl,
                                int honor_stop, double eps, cudaStream_t st);
// The same update with FP64 sums and an FP64 solve (vicp_solve64.cu);
// partials holds nparts x 16 doubles.
cudaError_t launch_reduce_solve_f64(const float4 *src, int m, double *pose, const float4 *tgt, int n_tgt,
                                    const int *nn, float3 center, double *partials, int nparts, double *rmse_out,
                                    DevCtl *ctl, int honor_stop, double eps, cudaStream_t st);

}  // namespace vicp
