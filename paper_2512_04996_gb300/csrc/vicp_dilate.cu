// vicp_dilate.cu -- DDMA, dilation of root-voxel labels into empty voxels
// (Alg. 3 and its description in Sec. 3).
//
// What is computed.  L synchronous rounds of six-neighbour propagation, with
// the smallest root kept where several labelled neighbours meet, label every
// voxel v within Manhattan distance L of an occupied voxel with
//     ring[v] = d(v) = min over occupied u of |u - v|_1,
//     root[v] = the smallest linear index among occupied u at that distance,
// and leave the rest at root -1 / ring 255.  (On a box grid every monotone
// lattice path between two voxels stays inside the box, so the rounds reach
// exactly the voxels at Manhattan distance r in round r.)
//
// How.  Instead of L rounds over the dense grid, the kernels evaluate that
// closed form as a separable lexicographic minimum.  A candidate is packed
// into one 32-bit word (dist:6 | dz+31:6 | dy+31:6 | dx+31:6), the root's
// offset from the voxel holding the word.  Because the linear index
// x + nx*(y + ny*z) orders in-grid voxels as (z, y, x) lexicographically, for
// a fixed voxel the unsigned order of these words is the order (distance,
// root index).  Moving a word one voxel along an axis adds one to the
// distance and shifts one offset field: a single integer add.  Words whose
// distance passes L are dropped (they cannot end within L).
//
//   pass X: nearest occupied voxel along the row, from the occupancy bitmask
//           with clz/ffs on a 64-bit window (ties go to the left, the smaller
//           index);
//   pass Y: forward and backward running minimum along y;
//   pass Z: the same along z, then the word is decoded into root and ring.
//
// Most of a grid is far from every point (typically over 90% of the voxels
// of a depth scene at L = 10), so the work is organised around skipping it.
// k_dilate_xy runs passes X and Y for units of 32 x 32 voxels of one
// z-plane (a warp each, a lane per x): the lanes load the occupancy bits of
// the unit's rows grown by L, and a unit with no occupied voxel in reach only
// records a zero row mask.  The others write their pass-Y words to an
// intermediate array (16 bits a word while L <= 15).  All words a warp needs
// are loaded (or shuffled in) before its sweeps, so each sweep is a chain of
// register operations rather than of memory latencies.  k_dilate_z then runs
// pass Z for columns of 32 voxels (a warp per 32 x 32 columns of one row y,
// a lane per x), reading only planes whose row mask is set, and writes root
// and ring.  root and ring keep "unlabelled" between dilations everywhere
// but where the last dilation wrote labels (a flag per column unit), so a
// column unit with nothing in reach now and no labels before writes nothing;
// the host clears both arrays in full only when they are new or the grid's
// dimensions change.  L <= 31.
#include "vicp_dilate.cuh"
#include "vicp_launch.h"

namespace vicp {

using namespace dil;

// `clear` (sparse grid: the labelled-segment table's keys, which pass Z fills)
// is set to HASH_EMPTY and `zero` (pass Z's counters) to zero on the way:
// pass Z starts only after this kernel.
template <class W>
__global__ void __launch_bounds__(THREADS) k_dilate_xy(const unsigned *__restrict__ occ, long long n_words, GridGeom g,
                                                       int L, int nxb, int nyb, int units,
                                                       typename W::Stored *__restrict__ inter,
                                                       unsigned *__restrict__ rows, unsigned *__restrict__ clear,
                                                       long long clear_words, unsigned *__restrict__ zero,
                                                       int zero_words)
{
    pdl_begin();
    for (long long w = (long long)blockIdx.x * THREADS + threadIdx.x; w < clear_words; w += (long long)gridDim.x * THREADS)
        clear[w] = HASH_EMPTY;
    for (int w = blockIdx.x * THREADS + threadIdx.x; w < zero_words; w += gridDim.x * THREADS)
        zero[w] = 0u;
    for (int u = blockIdx.x * WARPS + (threadIdx.x >> 5); u < units; u += gridDim.x * WARPS)
        dilate_xy_unit<W>(u, occ, n_words, g, L, nxb, nyb, inter, rows);
}

template <class W>
__global__ void __launch_bounds__(THREADS) k_dilate_z(const typename W::Stored *__restrict__ inter,
                                                      const unsigned *__restrict__ rows,
                                                      unsigned char *__restrict__ dirty, GridGeom g, int L, int nxb,
                                                      int nyb, int units, int *__restrict__ root,
                                                      unsigned char *__restrict__ ring)
{
    pdl_begin();
    const DenseLabels out{dirty, root, ring};
    for (int u = blockIdx.x * WARPS + (threadIdx.x >> 5); u < units; u += gridDim.x * WARPS)
        dilate_z_unit<W>(u, inter, rows, out, g, L, nxb, nyb);
}

// Pass Z into the labelled-segment table; each block writes the number of
// segments it entered to counts[blockIdx.x], counts[gridDim.x] (zero
// beforehand) is set to 1 if an insert gave up or the roots ran out, and
// counts[gridDim.x + 1] (zero beforehand) counts the roots handed out.
template <class W>
__global__ void __launch_bounds__(THREADS) k_dilate_z_hashed(const typename W::Stored *__restrict__ inter,
                                                             const unsigned *__restrict__ rows, GridGeom g, int L,
                                                             int nxb, int nyb, int units, HashTable table,
                                                             uint2 *__restrict__ seg, int *__restrict__ root,
                                                             unsigned cap_root, unsigned *__restrict__ counts,
                                                             unsigned *__restrict__ err)
{
    pdl_begin();
    __shared__ unsigned s_count;
    if (threadIdx.x == 0)
        s_count = 0u;
    __syncthreads();
    const HashLabels out{table, seg, root, cap_root, counts + gridDim.x + 1, counts + gridDim.x, err};
    unsigned n = 0u;
    for (int u = blockIdx.x * WARPS + (threadIdx.x >> 5); u < units; u += gridDim.x * WARPS)
        n += dilate_z_unit<W>(u, inter, rows, out, g, L, nxb, nyb);   // the same on every lane
    if ((threadIdx.x & 31) == 0 && n)
        atomicAdd(&s_count, n);
    __syncthreads();
    if (threadIdx.x == 0)
        counts[blockIdx.x] = s_count;
}

// Blocks that can be resident at once (the kernels loop over their units).
template <typename K>
static int resident_blocks(K kernel)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, THREADS, 0) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return sms * per_sm;
}

template <class W>
static cudaError_t run_dilate(const unsigned *occ, const GridGeom &g, int L, void *inter, unsigned *rows,
                              unsigned char *dirty, int *root, unsigned char *ring, const HashTable *labels,
                              uint2 *seg, unsigned cap_root, unsigned *counts, unsigned *err, cudaStream_t st)
{
    using S = typename W::Stored;
    static const int xy_blocks = resident_blocks(k_dilate_xy<W>), z_blocks = resident_blocks(k_dilate_z<W>),
                     zh_blocks = resident_blocks(k_dilate_z_hashed<W>);
    const int nxb = (g.nx + UX - 1) / UX, nyb = (g.ny + UY - 1) / UY, nzb = (g.nz + UZ - 1) / UZ;
    const int u_xy = nxb * nyb * g.nz;   // < V < 2^31
    const int u_z = nxb * g.ny * nzb;    // < V < 2^31
    const int zh_grid = min(zh_blocks, (u_z + WARPS - 1) / WARPS);
    cudaError_t e = launch_kernel(k_dilate_xy<W>, dim3(min(xy_blocks, (u_xy + WARPS - 1) / WARPS)), dim3(THREADS), 0,
                                  st, occ, occ_words(g.V), g, L, nxb, nyb, u_xy, static_cast<S *>(inter), rows,
                                  labels ? labels->keys : nullptr, labels ? (long long)labels->mask + 1 : 0ll,
                                  labels ? counts : nullptr, labels ? zh_grid + 2 : 0);
    if (e != cudaSuccess)
        return e;
    if (labels)
        return launch_kernel(k_dilate_z_hashed<W>, dim3(zh_grid), dim3(THREADS), 0, st, static_cast<const S *>(inter),
                             rows, g, L, nxb, nyb, u_z, *labels, seg, root, cap_root, counts, err);
    return launch_kernel(k_dilate_z<W>, dim3(min(z_blocks, (u_z + WARPS - 1) / WARPS)), dim3(THREADS), 0, st,
                         static_cast<const S *>(inter), rows, dirty, g, L, nxb, nyb, u_z, root, ring);
}

int dilate_hashed_blocks(const GridGeom &g, int L)
{
    const int nxb = (g.nx + UX - 1) / UX, nzb = (g.nz + UZ - 1) / UZ;
    const int u_z = nxb * g.ny * nzb;
    const int res = L <= L_COMPACT_MAX ? resident_blocks(k_dilate_z_hashed<Words16>)
                                       : resident_blocks(k_dilate_z_hashed<Words32>);
    return min(res, (u_z + WARPS - 1) / WARPS);
}

long long dilate_units(const GridGeom &g)
{
    return (long long)((g.nx + UX - 1) / UX) * ((g.ny + UY - 1) / UY) * g.nz;
}

long long dilate_column_units(const GridGeom &g)
{
    return (long long)((g.nx + UX - 1) / UX) * g.ny * ((g.nz + UZ - 1) / UZ);
}

cudaError_t launch_dilate(const unsigned *occ, const GridGeom &g, int L, void *inter, unsigned *rows,
                          unsigned char *dirty, int *root, unsigned char *ring, cudaStream_t st)
{
    if (L <= L_COMPACT_MAX)
        return run_dilate<Words16>(occ, g, L, inter, rows, dirty, root, ring, nullptr, nullptr, 0u, nullptr, nullptr,
                                   st);
    return run_dilate<Words32>(occ, g, L, inter, rows, dirty, root, ring, nullptr, nullptr, 0u, nullptr, nullptr, st);
}

cudaError_t launch_dilate_hashed(const unsigned *occ, const GridGeom &g, int L, void *inter, unsigned *rows,
                                 const HashTable &labels, uint2 *seg, int *root, unsigned cap_root, unsigned *counts,
                                 unsigned *err, cudaStream_t st)
{
    if (L <= L_COMPACT_MAX)
        return run_dilate<Words16>(occ, g, L, inter, rows, nullptr, root, nullptr, &labels, seg, cap_root, counts,
                                   err, st);
    return run_dilate<Words32>(occ, g, L, inter, rows, nullptr, root, nullptr, &labels, seg, cap_root, counts, err,
                               st);
}

// Clears bits of a device word (atomically, so that concurrent kernels'
// bits are kept).
__global__ void k_clear_bits(unsigned *word, unsigned bits) { atomicAnd(word, ~bits); }

cudaError_t launch_clear_bits(unsigned *word, unsigned bits, cudaStream_t st)
{
    k_clear_bits<<<1, 1, 0, st>>>(word, bits);
    return cudaGetLastError();
}

}  // namespace vicp
