// vicp_batch.cu -- batched registration of many pairs over one pooled store
// (layouts in vicp_batch.h).  The grid build of every pair (Alg. 1, Alg. 2,
// the brick levels of the global search, Alg. 3) runs as a handful of
// launches over all pairs at once, and each ICP iteration of every pair
// (Alg. 4 and the update of Eq. 1) is one persistent launch.
//
// The iteration kernel is cooperative: all its blocks are resident together
// and pass two grid-wide barriers.
//   phase 1  each block takes (pair, tile) items in turn and runs the
//            localised search of the tile's points (a thread per point); a
//            query whose root segment is long, or that has no root, is
//            listed for phase 2 (one global atomic per block and list);
//   phase 2  every warp of the grid takes listed queries in turn: all lanes
//            scan one dense segment, or run one exact global search over the
//            query's pair;
//   phase 3  each block reduces the items it searched in phase 1 into
//            per-item double-float sums; the block that finishes a pair's
//            last item adds the pair's item sums in item order and solves
//            Eq. 1 for that pair (one warp), so every pair's update is
//            bit-identical from run to run.
// The barriers wait with a time limit (one second): a block that gives up
// sets DEVERR_TIMEOUT and leaves the kernel.
#include "vicp_batch.h"
#include "vicp_df.cuh"
#include "vicp_f64.cuh"
#include "vicp_dilate.cuh"
#include "vicp_launch.h"
#include "vicp_search.cuh"

namespace vicp {

// ---------------------------------------------------------------------------
// Per-pair bounding boxes: one block per 256-point tile; warp-reduced bounds
// merged with one atomic per axis, bound and warp.  bbox: [3P] minima then
// [3P] maxima (order-preserving images).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BATCH_TILE) k_batch_bbox(const float4 *__restrict__ pts,
                                                           const BatchItem *__restrict__ items, int P,
                                                           unsigned *__restrict__ bbox)
{
    pdl_begin();
    const BatchItem it = items[blockIdx.x];
    const int j = it.i0 + threadIdx.x;
    const float inf = __int_as_float(0x7f800000);
    float lo[3] = {inf, inf, inf}, hi[3] = {-inf, -inf, -inf};
    if (j < it.i1) {
        const float4 q = __ldg(pts + j);
        lo[0] = fminf(lo[0], q.x); hi[0] = fmaxf(hi[0], q.x);
        lo[1] = fminf(lo[1], q.y); hi[1] = fmaxf(hi[1], q.y);
        lo[2] = fminf(lo[2], q.z); hi[2] = fmaxf(hi[2], q.z);
    }
#pragma unroll
    for (int a = 0; a < 3; ++a) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(FULL_MASK, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(FULL_MASK, hi[a], o));
        }
    }
    if ((threadIdx.x & 31) == 0) {
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            atomicMin(bbox + 3 * it.pair + a, float_to_ordered(lo[a]));
            atomicMax(bbox + 3 * P + 3 * it.pair + a, float_to_ordered(hi[a]));
        }
    }
}

cudaError_t launch_batch_bbox(const float4 *pts, const BatchItem *items, int n_items, int P, unsigned *bbox,
                              cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(bbox, 0xff, 3 * (size_t)P * sizeof(unsigned), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(bbox + 3 * P, 0x00, 3 * (size_t)P * sizeof(unsigned), st);
    if (e != cudaSuccess)
        return e;
    return launch_kernel(k_batch_bbox, dim3(n_items), dim3(BATCH_TILE), 0, st, pts, items, P, bbox);
}

// ---------------------------------------------------------------------------
// VOH over all pairs: as the single-grid histogram, with a block per tile of
// one pair.  Keys are the pair's own; counts, occupancy bits and the scan's
// tile totals are indexed by the pooled voxel vbase + key, brick counts by
// bbase + brick.  All lanes of a warp belong to one pair, so grouping by the
// local key groups by the pooled one.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BATCH_TILE) k_batch_histogram(const float4 *__restrict__ pts,
                                                                const BatchItem *__restrict__ items,
                                                                const BatchPair *__restrict__ pairs,
                                                                int *__restrict__ keys, unsigned *__restrict__ counts,
                                                                unsigned *__restrict__ bcounts,
                                                                unsigned *__restrict__ occ,
                                                                unsigned *__restrict__ tile_sum,
                                                                DevCtl *__restrict__ ctl)
{
    pdl_begin();
    if (blockIdx.x == 0 && threadIdx.x == 0)
        ctl->scan_epoch = ctl->scan_epoch + 1u;
    const BatchItem it = items[blockIdx.x];
    const GridGeom g = pairs[it.pair].g;
    const int vbase = (int)pairs[it.pair].vbase;
    const int bbase = pairs[it.pair].bbase;
    const int j = it.i0 + threadIdx.x;
    int key = -2, bk = -2;   // lanes past the end match only each other and add nothing
    if (j < it.i1) {
        const float4 q = __ldg(pts + j);
        int ix, iy, iz;
        if (voxel_coords(g, q.x, q.y, q.z, ix, iy, iz)) {
            key = ix + g.nx * (iy + g.ny * iz);
            bk = brick_key(g, ix, iy, iz);
        } else {
            key = bk = -1;
        }
        keys[j] = key;
    }
    const int lane = threadIdx.x & 31;
    const int gv = key >= 0 ? vbase + key : -1;
    const unsigned peers = __match_any_sync(FULL_MASK, key);
    if (key >= 0 && lane == __ffs(peers) - 1)
        atomicAdd(counts + gv, (unsigned)__popc(peers));
    const unsigned bpeers = __match_any_sync(FULL_MASK, bk);
    if (bk >= 0 && lane == __ffs(bpeers) - 1)
        atomicAdd(bcounts + bbase + bk, (unsigned)__popc(bpeers));
    const int word = key >= 0 ? (gv >> 5) : -2;
    const unsigned wpeers = __match_any_sync(FULL_MASK, word);
    const unsigned wbits = __reduce_or_sync(wpeers, key >= 0 ? 1u << (gv & 31) : 0u);
    if (word >= 0 && lane == __ffs(wpeers) - 1)
        atomicOr(occ + word, wbits);
    const int tile = key >= 0 ? (gv / SCAN_TILE) : -2;
    const unsigned tpeers = __match_any_sync(FULL_MASK, tile);
    if (tile >= 0 && lane == __ffs(tpeers) - 1)
        atomicAdd(tile_sum + tile, (unsigned)__popc(tpeers));
}

cudaError_t launch_batch_histogram(const float4 *pts, const BatchItem *items, int n_items, const BatchPair *pairs,
                                   int *keys, unsigned *counts, unsigned *bcounts, unsigned *occ, unsigned *tile_sum,
                                   DevCtl *ctl, cudaStream_t st)
{
    return launch_kernel(k_batch_histogram, dim3(n_items), dim3(BATCH_TILE), 0, st, pts, items, pairs, keys, counts,
                         bcounts, occ, tile_sum, ctl);
}

// ---------------------------------------------------------------------------
// Brick offsets, one block per pair: the pair's brick counts scanned
// together with their non-empty flags (as the single-grid brick scan), from
// the pair's first position in the pooled store (off[vbase]).  Brick slots
// are the pair's own, stored at bbase + slot; list holds the pair's own
// brick index, bslot the pooled slot.
// ---------------------------------------------------------------------------
constexpr int BBS_THREADS = 1024;
constexpr int BBS_PER = 8;   // bricks per thread and round

__global__ void __launch_bounds__(BBS_THREADS) k_batch_brick_scan(const unsigned *__restrict__ bcounts,
                                                                  const BatchPair *__restrict__ pairs,
                                                                  const unsigned *__restrict__ off,
                                                                  unsigned *__restrict__ boff, int *__restrict__ list,
                                                                  uint2 *__restrict__ range, int *__restrict__ bslot,
                                                                  uint4 *__restrict__ boxord,
                                                                  BatchState *__restrict__ state)
{
    pdl_begin();
    __shared__ unsigned long long s_w[BBS_THREADS / 32];
    __shared__ unsigned long long s_carry;
    const int p = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const GridGeom g = pairs[p].g;
    const int bbase = pairs[p].bbase;
    const int nbt = brick_slots(g);
    if (tid == 0)
        s_carry = (unsigned long long)__ldg(off + pairs[p].vbase);   // slot count 0, first position
    __syncthreads();
    for (int c0 = 0; c0 < nbt; c0 += BBS_THREADS * BBS_PER) {
        // thread t owns the contiguous bricks [c0 + t*PER, c0 + t*PER + PER)
        unsigned c[BBS_PER];
        unsigned long long sum = 0ull;
#pragma unroll
        for (int k = 0; k < BBS_PER; ++k) {
            const int b = c0 + tid * BBS_PER + k;
            c[k] = b < nbt ? __ldg(bcounts + bbase + b) : 0u;
        }
#pragma unroll
        for (int k = 0; k < BBS_PER; ++k)
            sum += (unsigned long long)c[k] | ((unsigned long long)(c[k] != 0u) << 32);
        unsigned long long incl = sum;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const unsigned long long y = __shfl_up_sync(FULL_MASK, incl, d);
            if (lane >= d)
                incl += y;
        }
        if (lane == 31)
            s_w[warp] = incl;
        __syncthreads();
        if (warp == 0) {
            const unsigned long long w = s_w[lane];
            unsigned long long wi = w;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const unsigned long long y = __shfl_up_sync(FULL_MASK, wi, d);
                if (lane >= d)
                    wi += y;
            }
            s_w[lane] = wi - w;
        }
        __syncthreads();
        unsigned long long run = s_carry + s_w[warp] + (incl - sum);
#pragma unroll
        for (int k = 0; k < BBS_PER; ++k) {
            const int b = c0 + tid * BBS_PER + k;
            if (b < nbt) {
                const unsigned start = (unsigned)run;
                boff[bbase + b] = start;
                if (c[k]) {
                    const int slot = bbase + (int)(run >> 32);
                    list[slot] = b;
                    range[slot] = make_uint2(start, start + c[k]);
                    bslot[bbase + b] = slot;
                    boxord[2 * slot] = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0u);   // min
                    boxord[2 * slot + 1] = make_uint4(0u, 0u, 0u, 0u);                          // max
                }
                run += (unsigned long long)c[k] | ((unsigned long long)(c[k] != 0u) << 32);
            }
        }
        __syncthreads();
        if (tid == BBS_THREADS - 1)
            s_carry = run;
        __syncthreads();
    }
    if (tid == 0)
        state[p].n_bricks = (int)(s_carry >> 32);
}

cudaError_t launch_batch_brick_scan(const unsigned *bcounts, const BatchPair *pairs, int P, const unsigned *off,
                                    unsigned *boff, int *list, uint2 *range, int *bslot, uint4 *boxord,
                                    BatchState *state, cudaStream_t st)
{
    return launch_kernel(k_batch_brick_scan, dim3(P), dim3(BBS_THREADS), 0, st, bcounts, pairs, off, boff, list, range,
                         bslot, boxord, state);
}

// ---------------------------------------------------------------------------
// VDMA over all pairs: as the single-grid scatter, a block per tile of one
// pair.  Segment slots come from the pooled voxel vbase + key; the stored
// index (ids, and the w field of csr and bpts) is the pair's own; target
// points outside the pair's grid are listed at outside + tbase.  Zeroes the
// scan's tile totals for the next build.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(BATCH_TILE) k_batch_scatter(const float4 *__restrict__ pts,
                                                              const int *__restrict__ keys,
                                                              const BatchItem *__restrict__ items,
                                                              const BatchPair *__restrict__ pairs, int n_total,
                                                              const unsigned *__restrict__ off,
                                                              unsigned *__restrict__ counts,
                                                              const unsigned *__restrict__ boff,
                                                              unsigned *__restrict__ bcounts,
                                                              const int *__restrict__ bslot,
                                                              unsigned *__restrict__ boxord, int *__restrict__ ids,
                                                              float4 *__restrict__ csr, float4 *__restrict__ bpts,
                                                              int *__restrict__ outside,
                                                              unsigned *__restrict__ tile_sum, int n_tiles,
                                                              BatchState *__restrict__ state,
                                                              DevCtl *__restrict__ ctl)
{
    pdl_begin();
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x)
        tile_sum[t] = 0u;
    const BatchItem it = items[blockIdx.x];
    const GridGeom g = pairs[it.pair].g;
    const int vbase = (int)pairs[it.pair].vbase;
    const int bbase = pairs[it.pair].bbase;
    const int tbase = pairs[it.pair].tbase;
    const int j = it.i0 + threadIdx.x;
    const int jl = it.l0 + threadIdx.x;   // the pair's own index
    const int lane = threadIdx.x & 31;
    const int key = (j < it.i1) ? __ldg(keys + j) : -2;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    int bk = key;
    if (key >= 0) {
        q = __ldg(pts + j);
        int ix, iy, iz;
        bk = voxel_coords(g, q.x, q.y, q.z, ix, iy, iz) ? brick_key(g, ix, iy, iz) : -1;
        q.w = __int_as_float(jl);
    }
    {
        const unsigned peers = __match_any_sync(FULL_MASK, key);
        const int leader = __ffs(peers) - 1;
        const unsigned rank = __popc(peers & lanemask_lt());
        const unsigned cnt = __popc(peers);
        unsigned old = 0u;
        if (lane == leader) {
            if (key >= 0)
                old = atomicSub(counts + vbase + key, cnt);
            else if (key == -1)
                old = (unsigned)atomicAdd(&state[it.pair].n_outside, (int)cnt);
        }
        old = __shfl_sync(FULL_MASK, old, leader);
        if (key >= 0) {
            const unsigned pos = __ldg(off + vbase + key) + old - 1u - rank;
            if (pos < (unsigned)n_total) {
                ids[pos] = jl;
                csr[pos] = q;
            } else {
                atomicOr(&ctl->err, DEVERR_BOUNDS);
            }
        } else if (key == -1) {
            outside[tbase + old + rank] = jl;
        }
    }
    {
        const unsigned peers = __match_any_sync(FULL_MASK, bk);
        const int leader = __ffs(peers) - 1;
        const unsigned rank = __popc(peers & lanemask_lt());
        const unsigned ox = float_to_ordered(q.x), oy = float_to_ordered(q.y), oz = float_to_ordered(q.z);
        const unsigned mnx = __reduce_min_sync(peers, ox), mny = __reduce_min_sync(peers, oy),
                       mnz = __reduce_min_sync(peers, oz);
        const unsigned mxx = __reduce_max_sync(peers, ox), mxy = __reduce_max_sync(peers, oy),
                       mxz = __reduce_max_sync(peers, oz);
        unsigned old = 0u;
        if (lane == leader && bk >= 0) {
            old = atomicSub(bcounts + bbase + bk, (unsigned)__popc(peers));
            unsigned *b = boxord + 8 * __ldg(bslot + bbase + bk);
            atomicMin(b + 0, mnx);
            atomicMin(b + 1, mny);
            atomicMin(b + 2, mnz);
            atomicMax(b + 4, mxx);
            atomicMax(b + 5, mxy);
            atomicMax(b + 6, mxz);
        }
        old = __shfl_sync(FULL_MASK, old, leader);
        if (bk >= 0) {
            const unsigned pos = __ldg(boff + bbase + bk) + old - 1u - rank;
            if (pos < (unsigned)n_total)
                bpts[pos] = q;
            else
                atomicOr(&ctl->err, DEVERR_BOUNDS);
        }
    }
}

cudaError_t launch_batch_scatter(const float4 *pts, const int *keys, const BatchItem *items, int n_items,
                                 const BatchPair *pairs, int n_total, const unsigned *off, unsigned *counts,
                                 const unsigned *boff, unsigned *bcounts, const int *bslot, unsigned *boxord, int *ids,
                                 float4 *csr, float4 *bpts, int *outside, unsigned *tile_sum, int n_tiles,
                                 BatchState *state, DevCtl *ctl, cudaStream_t st)
{
    return launch_kernel(k_batch_scatter, dim3(n_items), dim3(BATCH_TILE), 0, st, pts, keys, items, pairs, n_total,
                         off, counts, boff, bcounts, bslot, boxord, ids, csr, bpts, outside, tile_sum, n_tiles, state,
                         ctl);
}

// ---------------------------------------------------------------------------
// Brick and super-brick records of every pair, one block per pair (as the
// single-grid kernel, on the pair's slots bbase..; super-brick records at
// sbbase.. carry the pair's own brick-record ranges).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_batch_brick_boxes(const uint4 *__restrict__ boxord,
                                                           const int *__restrict__ list,
                                                           const uint2 *__restrict__ range,
                                                           const BatchPair *__restrict__ pairs,
                                                           BatchState *__restrict__ state, float4 *__restrict__ box,
                                                           float4 *__restrict__ sb_box)
{
    pdl_begin();
    const int p = blockIdx.x;
    const int bbase = pairs[p].bbase, sbbase = pairs[p].sbbase;
    const int nb = state[p].n_bricks;
    const uint4 *bo = boxord + 2 * bbase;
    const int *li = list + bbase;
    const uint2 *ra = range + bbase;
    float4 *bx = box + 2 * bbase;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        const uint4 lo = bo[2 * k], hi = bo[2 * k + 1];
        const uint2 r = ra[k];
        bx[2 * k] = make_float4(ordered_to_float(lo.x), ordered_to_float(lo.y), ordered_to_float(lo.z),
                                __uint_as_float(r.x));
        bx[2 * k + 1] = make_float4(ordered_to_float(hi.x), ordered_to_float(hi.y), ordered_to_float(hi.z),
                                    __uint_as_float(r.y));
        const int sb = __ldg(li + k) / SUPER_BRICKS;
        if (k == 0 || __ldg(li + k - 1) / SUPER_BRICKS != sb) {
            uint4 l = lo, h = hi;
            int e = k + 1;
            while (e < nb && __ldg(li + e) / SUPER_BRICKS == sb) {
                const uint4 bl = bo[2 * e], bh = bo[2 * e + 1];
                l = make_uint4(min(l.x, bl.x), min(l.y, bl.y), min(l.z, bl.z), 0u);
                h = make_uint4(max(h.x, bh.x), max(h.y, bh.y), max(h.z, bh.z), 0u);
                ++e;
            }
            const int slot = sbbase + atomicAdd(&state[p].n_super, 1);
            sb_box[2 * slot] = make_float4(ordered_to_float(l.x), ordered_to_float(l.y), ordered_to_float(l.z),
                                           __uint_as_float((unsigned)k));
            sb_box[2 * slot + 1] = make_float4(ordered_to_float(h.x), ordered_to_float(h.y), ordered_to_float(h.z),
                                               __uint_as_float((unsigned)e));
        }
    }
}

cudaError_t launch_batch_brick_boxes(const uint4 *boxord, const int *list, const uint2 *range,
                                     const BatchPair *pairs, int P, BatchState *state, float4 *box, float4 *sb_box,
                                     cudaStream_t st)
{
    return launch_kernel(k_batch_brick_boxes, dim3(P), dim3(256), 0, st, boxord, list, range, pairs, state, box,
                         sb_box);
}

// ---------------------------------------------------------------------------
// Dilation of every pair's grid: the single-grid passes (vicp_dilate.cuh)
// over the concatenated units of all pairs.  A warp finds the pair of its
// unit by binary search in the pairs' first-unit table (kept in shared
// memory for up to BATCH_SMEM_PAIRS pairs) and runs the unit on the pair's
// slices of the pooled arrays.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_pair(const int *starts, int P, int u)
{
    int lo = 0, hi = P - 1;   // starts[lo] <= u < starts[hi + 1]
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (starts[mid] <= u)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ const int *stage_starts(const int *starts, int P, int *s_buf)
{
    if (P + 1 > BATCH_SMEM_PAIRS)
        return starts;
    for (int k = threadIdx.x; k <= P; k += blockDim.x)
        s_buf[k] = __ldg(starts + k);
    __syncthreads();
    return s_buf;
}

template <class W>
__global__ void __launch_bounds__(dil::THREADS) k_batch_dilate_xy(const unsigned *__restrict__ occ,
                                                                  const BatchPair *__restrict__ pairs, int P,
                                                                  const int *__restrict__ ustart, int L,
                                                                  typename W::Stored *__restrict__ inter,
                                                                  unsigned *__restrict__ rows)
{
    pdl_begin();
    extern __shared__ int s_starts[];
    const int *starts = stage_starts(ustart, P, s_starts);
    const int units = __ldg(ustart + P);
    for (int u = blockIdx.x * dil::WARPS + (threadIdx.x >> 5); u < units; u += gridDim.x * dil::WARPS) {
        const int p = find_pair(starts, P, u);
        const GridGeom g = pairs[p].g;
        const long long vb = pairs[p].vbase;
        const int nxb = (g.nx + dil::UX - 1) / dil::UX, nyb = (g.ny + dil::UY - 1) / dil::UY;
        const int u0 = starts[p];
        dil::dilate_xy_unit<W>(u - u0, occ + (vb >> 5), (g.V + 31) / 32, g, L, nxb, nyb, inter + vb, rows + u0);
    }
}

template <class W>
__global__ void __launch_bounds__(dil::THREADS) k_batch_dilate_z(const typename W::Stored *__restrict__ inter,
                                                                 const unsigned *__restrict__ rows,
                                                                 unsigned char *__restrict__ dirty,
                                                                 const BatchPair *__restrict__ pairs, int P,
                                                                 const int *__restrict__ ustart_xy,
                                                                 const int *__restrict__ ustart, int L,
                                                                 int *__restrict__ root,
                                                                 unsigned char *__restrict__ ring)
{
    pdl_begin();
    extern __shared__ int s_starts[];
    const int *starts = stage_starts(ustart, P, s_starts);
    const int units = __ldg(ustart + P);
    for (int u = blockIdx.x * dil::WARPS + (threadIdx.x >> 5); u < units; u += gridDim.x * dil::WARPS) {
        const int p = find_pair(starts, P, u);
        const GridGeom g = pairs[p].g;
        const long long vb = pairs[p].vbase;
        const int nxb = (g.nx + dil::UX - 1) / dil::UX, nyb = (g.ny + dil::UY - 1) / dil::UY;
        const int u0 = starts[p];
        dil::dilate_z_unit<W>(u - u0, inter + vb, rows + __ldg(ustart_xy + p),
                              dil::DenseLabels{dirty + u0, root + vb, ring + vb}, g, L, nxb, nyb);
    }
}

template <typename K>
static int resident_blocks_of(K kernel, int threads, size_t smem)
{
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem) != cudaSuccess || per_sm < 1)
        per_sm = 1;
    return sms * per_sm;
}

template <class W>
static cudaError_t run_batch_dilate(const unsigned *occ, const BatchPair *pairs, int P, const int *ustart_xy,
                                    const int *ustart_z, int L, void *inter, unsigned *rows, unsigned char *dirty,
                                    int *root, unsigned char *ring, int units_xy, int units_z, cudaStream_t st)
{
    using S = typename W::Stored;
    const size_t smem = P + 1 <= BATCH_SMEM_PAIRS ? (size_t)(P + 1) * sizeof(int) : 0;
    const int xy_blocks = resident_blocks_of(k_batch_dilate_xy<W>, dil::THREADS, smem);
    const int z_blocks = resident_blocks_of(k_batch_dilate_z<W>, dil::THREADS, smem);
    cudaError_t e = launch_kernel(k_batch_dilate_xy<W>, dim3(min(xy_blocks, (units_xy + dil::WARPS - 1) / dil::WARPS)),
                                  dim3(dil::THREADS), smem, st, occ, pairs, P, ustart_xy, L, static_cast<S *>(inter),
                                  rows);
    if (e != cudaSuccess)
        return e;
    return launch_kernel(k_batch_dilate_z<W>, dim3(min(z_blocks, (units_z + dil::WARPS - 1) / dil::WARPS)),
                         dim3(dil::THREADS), smem, st, static_cast<const S *>(inter), rows, dirty, pairs, P, ustart_xy,
                         ustart_z, L, root, ring);
}

cudaError_t launch_batch_dilate(const unsigned *occ, const BatchPair *pairs, int P, const int *ustart_xy,
                                const int *ustart_z, int L, void *inter, unsigned *rows, unsigned char *dirty,
                                int *root, unsigned char *ring, cudaStream_t st)
{
    // unit totals: read back by the caller would cost a synchronisation, so
    // the grids are sized from the resident block count alone
    const int big = 1 << 30;
    if (L <= dil::L_COMPACT_MAX)
        return run_batch_dilate<dil::Words16>(occ, pairs, P, ustart_xy, ustart_z, L, inter, rows, dirty, root, ring,
                                              big, big, st);
    return run_batch_dilate<dil::Words32>(occ, pairs, P, ustart_xy, ustart_z, L, inter, rows, dirty, root, ring, big,
                                          big, st);
}

// ---------------------------------------------------------------------------
// Grid-wide barrier of the cooperative iteration kernel, with a time limit.
// One thread per block arrives (atomic ticket after a fence that publishes
// the block's writes); the last one resets the ticket and advances the
// generation with a release store; the others poll the generation with
// acquire loads.  Returns false, with DEVERR_TIMEOUT set, when the
// generation has not moved for BARRIER_LIMIT_NS.
// ---------------------------------------------------------------------------
constexpr unsigned long long BARRIER_LIMIT_NS = 1000000000ull;

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned *p)
{
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned *p, unsigned v)
{
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long globaltimer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ bool grid_barrier(DevCtl *ctl, int *s_flag)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        const unsigned gen = ld_acquire_u32(&ctl->bar_gen);
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->bar_count, 1u);
        if (arrived == gridDim.x - 1) {
            ctl->bar_count = 0u;
            st_release_u32(&ctl->bar_gen, gen + 1u);
        } else {
            const unsigned long long t0 = globaltimer_ns();
            unsigned polls = 0;
            while (ld_acquire_u32(&ctl->bar_gen) == gen) {
                __nanosleep(64);
                if ((++polls & 255u) == 0u && globaltimer_ns() - t0 > BARRIER_LIMIT_NS) {
                    atomicOr(&ctl->err, DEVERR_TIMEOUT);
                    ok = 0;
                    break;
                }
            }
        }
        __threadfence();
        *s_flag = ok;
    }
    __syncthreads();
    return *s_flag != 0;
}

// The float pose of a pair, on every lane of a warp (lanes 0..11 convert one
// entry each).
__device__ __forceinline__ PoseF pose_f_warp(const double *__restrict__ pose)
{
    const int lane = threadIdx.x & 31;
    const float v = lane < 12 ? __double2float_rn(pose[lane]) : 0.0f;
    PoseF P;
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const float x = __shfl_sync(FULL_MASK, v, k);
        const int a = k >> 2, b = k & 3;
        if (b < 3)
            P.r[3 * a + b] = x;
        else
            P.t[a] = x;
    }
    return P;
}

// ---------------------------------------------------------------------------
// Phase 3 of the iteration kernel with FP64 sums and an FP64 solve: the same
// items and the same fixed summation order (thread, warp, block per item,
// then the pair's items in item order by the block of its last item) as the
// double-float phase 3 of k_batch_iter, in doubles.  s_dyn_f holds
// WARPS x 16 x 33 doubles; the partials one double per (item, sum).
// ---------------------------------------------------------------------------
template <int TH, int PPT>
__device__ __forceinline__ void batch_phase3_f64(const BatchIterArgs &a, float *s_dyn_f, BatchItem &s_item,
                                                 int &s_skip, int &s_last, PoseF &s_pose)
{
    constexpr int WARPS = TH / 32;
    __shared__ double s_w[WARPS][F64_SUMS];
    __shared__ double s_tot[F64_SUMS];
    double(*s_t)[F64_SUMS][33] = reinterpret_cast<double(*)[F64_SUMS][33]>(s_dyn_f);
    double *partials = reinterpret_cast<double *>(a.partials);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    DevCtl *const ctl = a.ctl;
    for (int itx = blockIdx.x; itx < a.n_items; itx += gridDim.x) {
        if (tid == 0) {
            s_item = a.items[itx];
            s_skip = *(volatile const int *)&a.state[s_item.pair].stop;
        }
        __syncthreads();
        const BatchItem it = s_item;
        if (s_skip) {
            __syncthreads();
            continue;
        }
        load_pose_f_block(a.pose + 16 * it.pair, s_pose);
        const PoseF P = s_pose;
        const BatchPair *bp = a.pairs + it.pair;
        const double3 c = make_double3((double)bp->cx, (double)bp->cy, (double)bp->cz);
        const int tbase = bp->tbase, n_tgt = bp->n_tgt;
        double acc[F64_SUMS];
#pragma unroll
        for (int k = 0; k < F64_SUMS; ++k)
            acc[k] = 0.0;
        int j[PPT];
        float4 p[PPT], q[PPT];
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            const int i = it.i0 + tid + TH * u;
            j[u] = -1;
            if (i < it.i1) {
                j[u] = __ldcg(a.nn + i);
                p[u] = __ldg(a.src + i);
            }
        }
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            if ((unsigned)j[u] < (unsigned)n_tgt)
                q[u] = __ldg(a.tgt + tbase + j[u]);
            else if (it.i0 + tid + TH * u < it.i1)   // no valid match: report, leave it out
                atomicOr(&ctl->err, DEVERR_BOUNDS);
        }
#pragma unroll
        for (int u = 0; u < PPT; ++u)
            if ((unsigned)j[u] < (unsigned)n_tgt)
                accumulate_corr_f64(acc, transform_pt(P, p[u]), q[u], c);
        // warp sums through shared memory: lane l adds value l % 16 over
        // lanes 16 (l / 16) .. 16 (l / 16) + 15 in order, then the halves
#pragma unroll
        for (int k = 0; k < F64_SUMS; ++k)
            s_t[warp][k][lane] = acc[k];
        __syncwarp();
        {
            const int k = lane & 15, h = (lane >> 4) * 16;
            double v = s_t[warp][k][h];
#pragma unroll
            for (int t = 1; t < 16; ++t)
                v += s_t[warp][k][h + t];
            v += __shfl_xor_sync(FULL_MASK, v, 16);
            if (lane < 16)
                s_w[warp][k] = v;
        }
        __syncthreads();
        if (tid < F64_SUMS) {   // the block's warps, in order
            double v = s_w[0][tid];
#pragma unroll
            for (int w = 1; w < WARPS; ++w)
                v += s_w[w][tid];
            partials[(size_t)itx * F64_SUMS + tid] = v;
            __threadfence();
        }
        __syncthreads();
        if (tid == 0)
            s_last = atomicAdd(&a.state[it.pair].items_done, 1u) == (unsigned)(bp->n_items - 1);
        __syncthreads();
        if (s_last) {
            __threadfence();
            // the pair's item sums in item order, as in the double-float phase 3
            const int item0 = bp->item0, n_items = bp->n_items;
            {
                const int k = tid & 15, grp = tid >> 4;
                double v = 0.0;
                for (int b = grp; b < n_items; b += TH / 16)
                    v += __ldcg(partials + (size_t)(item0 + b) * F64_SUMS + k);
                v += __shfl_xor_sync(FULL_MASK, v, 16);
                if (lane < 16)
                    s_w[warp][lane] = v;
            }
            __syncthreads();
            if (tid < F64_SUMS) {
                double t = s_w[0][tid];
#pragma unroll
                for (int w = 1; w < WARPS; ++w)
                    t += s_w[w][tid];
                s_tot[tid] = t;
            }
            __syncthreads();
            if (warp == 0) {
                double rmse;
                BatchState *stp = a.state + it.pair;
                const bool ok = solve_update_f64(s_tot, bp->n_src, c, a.pose + 16 * it.pair, rmse);
                if (lane == 0) {
                    stp->items_done = 0u;
                    stp->last_rmse = rmse;
                    if (!ok) {
                        stp->err |= DEVERR_DEGENERATE;
                        stp->stop = 1;
                        atomicOr(&ctl->err, DEVERR_DEGENERATE);
                    } else {
                        const int k = stp->iters;
                        stp->iters = k + 1;
                        if (a.eps > 0.0 && k >= 1 && fabs(rmse - stp->prev_rmse) < a.eps)
                            stp->stop = 1;
                        stp->prev_rmse = rmse;
                    }
                }
            }
        }
        __syncthreads();   // s_item, s_pose and the sums are rewritten for the next item
    }
}

// ---------------------------------------------------------------------------
// The iteration kernel (see the top of this file).  Dynamic shared memory:
// the transposed per-lane sums of phase 3, WARPS x 16 x 33 words of 8 bytes
// (a float pair per word for double-float sums, a double for FP64 sums).
// With F64 the sums of phase 3 and the solve are FP64 (vicp_f64.cuh).
// ---------------------------------------------------------------------------
template <int TH, int PPT, int MINB, bool F64>
__global__ void __launch_bounds__(TH, MINB) k_batch_iter(const BatchIterArgs a)
{
    constexpr int WARPS = TH / 32;
    __shared__ PoseF s_pose;
    __shared__ BatchItem s_item;
    __shared__ int s_skip, s_flag, s_last;
    __shared__ unsigned long long s_cand;
    __shared__ int s_fb, s_fb_base, s_hv, s_hv_base;
    __shared__ float s_whi[WARPS][N_SUMS], s_wlo[WARPS][N_SUMS];
    __shared__ dfl s_tot[N_SUMS];
    extern __shared__ float s_dyn[];   // [2][WARPS][N_SUMS][33]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    DevCtl *const ctl = a.ctl;
    // After a barrier gave up, the arrival count no longer matches the
    // blocks in the barrier: the remaining launches of the registration do
    // nothing (the host clears the status and the count).
    if (*(volatile const unsigned *)&ctl->err & DEVERR_TIMEOUT)
        return;
    if (a.test_leave_early && blockIdx.x == 0)
        return;   // the others' first barrier runs out of time (test of the time limit)

    // ---- phase 1: localised search, item by item --------------------------
    for (int itx = blockIdx.x; itx < a.n_items; itx += gridDim.x) {
        if (tid == 0) {
            s_item = a.items[itx];
            s_skip = *(volatile const int *)&a.state[s_item.pair].stop;
            s_cand = 0ull;
            s_fb = s_hv = 0;
        }
        __syncthreads();
        const BatchItem it = s_item;
        if (s_skip) {
            __syncthreads();
            continue;
        }
        load_pose_f_block(a.pose + 16 * it.pair, s_pose);
        const PoseF P = s_pose;
        const BatchPair *bp = a.pairs + it.pair;
        const GridGeom g = bp->g;
        const long long vb = bp->vbase;
        bool fall[PPT], heavy[PPT];
        unsigned ra[PPT], rb[PPT];
        unsigned cand = 0u;
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            const int i = it.i0 + tid + TH * u;
            fall[u] = heavy[u] = false;
            ra[u] = rb[u] = 0u;
            if (i < it.i1) {
                const float3 s = transform_pt(P, __ldg(a.src + i));
                const int v = voxel_key(g, s.x, s.y, s.z);
                const int r = (v >= 0) ? __ldg(a.root + vb + v) : -1;
                if (r >= 0) {
                    const unsigned x0 = __ldg(a.off + vb + r);
                    const unsigned x1 = max(x0, min(__ldg(a.off + vb + r + 1), (unsigned)a.n_stored));
                    ra[u] = x0;
                    rb[u] = x1;
                    cand += x1 - x0;
                    heavy[u] = x1 - x0 > HEAVY;
                    if (!heavy[u]) {
                        const unsigned long long best = segment_min(a.csr, x0, x1, s);
                        a.nn[i] = (int)(unsigned)best;
                        a.d2[i] = __uint_as_float((unsigned)(best >> 32));
                    }
                } else {
                    fall[u] = true;
                }
            }
        }
        // list the queries for phase 2: warp slots by shared atomics, one
        // global atomic per list and block
        unsigned fm[PPT], hm[PPT];
        int fb_w[PPT], hv_w[PPT];
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            fm[u] = __ballot_sync(FULL_MASK, fall[u]);
            hm[u] = __ballot_sync(FULL_MASK, heavy[u]);
            fb_w[u] = hv_w[u] = 0;
            if (lane == 0) {
                if (fm[u])
                    fb_w[u] = atomicAdd(&s_fb, __popc(fm[u]));
                if (hm[u])
                    hv_w[u] = atomicAdd(&s_hv, __popc(hm[u]));
            }
        }
        const unsigned long long wc = warp_sum_u64(cand);
        if (lane == 0 && wc)
            atomicAdd(&s_cand, wc);
        __syncthreads();
        if (tid == 0) {
            if (s_cand)
                atomicAdd(&ctl->stat_local_cand, s_cand);
            atomicAdd(&ctl->stat_queries, (unsigned long long)(it.i1 - it.i0));
            if (s_fb)
                s_fb_base = atomicAdd(&ctl->fb_count, s_fb);
            if (s_hv)
                s_hv_base = atomicAdd(&ctl->hv_count, s_hv);
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            const int i = it.i0 + tid + TH * u;
            const int fbw = __shfl_sync(FULL_MASK, fb_w[u], 0), hvw = __shfl_sync(FULL_MASK, hv_w[u], 0);
            if (fall[u]) {
                const int slot = s_fb_base + fbw + __popc(fm[u] & lanemask_lt());
                if (slot < a.list_cap)
                    a.fb_list[slot] = make_int2(it.pair, i);
                else
                    atomicOr(&ctl->err, DEVERR_BOUNDS);
            }
            if (heavy[u]) {
                const int slot = s_hv_base + hvw + __popc(hm[u] & lanemask_lt());
                if (slot < a.list_cap)
                    a.hv_list[slot] = make_int4(it.pair, i, (int)ra[u], (int)rb[u]);
                else
                    atomicOr(&ctl->err, DEVERR_BOUNDS);
            }
        }
        __syncthreads();   // s_item and the counters are rewritten for the next item
    }
    if (!grid_barrier(ctl, &s_flag))
        return;

    // ---- phase 2: dense segments, then global searches, a warp each -------
    {
        const int F = min(*(volatile int *)&ctl->fb_count, a.list_cap);
        const int Hv = min(*(volatile int *)&ctl->hv_count, a.list_cap);
        const int n_warps = gridDim.x * WARPS, gw = blockIdx.x * WARPS + warp;
        unsigned long long examined = 0ull;
        for (int qi = n_warps - 1 - gw; qi < Hv; qi += n_warps) {
            const int4 e = a.hv_list[qi];
            if ((unsigned)e.x >= (unsigned)a.n_pairs || (unsigned)e.y >= (unsigned)a.list_cap || e.z > e.w ||
                (unsigned)e.w > (unsigned)a.n_stored) {   // a stale entry: skip it, report it
                if (lane == 0)
                    atomicOr(&ctl->err, DEVERR_BOUNDS);
                continue;
            }
            const PoseF P = pose_f_warp(a.pose + 16 * e.x);
            const float3 s = transform_pt(P, __ldg(a.src + e.y));
            unsigned long long unused = 0ull;
            const unsigned long long best = scan_run(a.csr, (unsigned)e.z, (unsigned)e.w, s, lane, ~0ull, unused);
            if (lane == 0) {
                a.nn[e.y] = (int)(unsigned)best;
                a.d2[e.y] = __uint_as_float((unsigned)(best >> 32));
            }
        }
        // global queries in chunks of FB_CHUNK, each chunk to whichever warp is
        // free (a ticket per chunk): their costs vary widely, and a fixed share
        // per warp leaves the whole grid waiting at the barrier for the warp
        // that drew the slowest ones
        constexpr int FB_CHUNK = 4;
        for (;;) {
            int q0 = 0;
            if (lane == 0)
                q0 = FB_CHUNK * (int)atomicAdd(&ctl->fb_next, 1u);
            q0 = __shfl_sync(FULL_MASK, q0, 0);
            if (q0 >= F)
                break;
            for (int qi = q0; qi < min(q0 + FB_CHUNK, F); ++qi) {
            const int2 e = a.fb_list[qi];
            if ((unsigned)e.x >= (unsigned)a.n_pairs || (unsigned)e.y >= (unsigned)a.list_cap) {
                if (lane == 0)   // a stale entry: skip it, report it
                    atomicOr(&ctl->err, DEVERR_BOUNDS);
                continue;
            }
            const BatchPair *bp = a.pairs + e.x;
            const PoseF P = pose_f_warp(a.pose + 16 * e.x);
            const float3 s = transform_pt(P, __ldg(a.src + e.y));
            const int tbase = bp->tbase;
            const unsigned long long best =
                global_search(s, a.bpts, a.bbox + 2 * bp->bbase, a.sb_box + 2 * bp->sbbase, a.state[e.x].n_super,
                              a.tgt + tbase, bp->n_tgt, a.outside + tbase, a.state[e.x].n_outside, lane, examined);
            if (lane == 0) {
                a.nn[e.y] = (int)(unsigned)best;
                a.d2[e.y] = __uint_as_float((unsigned)(best >> 32));
            }
            }
        }
        if (lane == 0 && examined)
            atomicAdd(&ctl->stat_global_cand, examined);
        if (!grid_barrier(ctl, &s_flag))
            return;
        if (blockIdx.x == 0 && tid == 0) {   // every block has read the list lengths
            ctl->stat_fallbacks += (unsigned long long)F;
            ctl->fb_count = 0;
            ctl->hv_count = 0;
            ctl->fb_next = 0u;
        }
    }
    if (a.search_only)
        return;

    // ---- phase 3: per-item sums; the last item of a pair solves it --------
    if constexpr (F64) {
        batch_phase3_f64<TH, PPT>(a, s_dyn, s_item, s_skip, s_last, s_pose);
        return;
    }
    float(*s_thi)[N_SUMS][33] = reinterpret_cast<float(*)[N_SUMS][33]>(s_dyn);
    float(*s_tlo)[N_SUMS][33] = reinterpret_cast<float(*)[N_SUMS][33]>(s_dyn + WARPS * N_SUMS * 33);
    for (int itx = blockIdx.x; itx < a.n_items; itx += gridDim.x) {
        if (tid == 0) {
            s_item = a.items[itx];
            s_skip = *(volatile const int *)&a.state[s_item.pair].stop;
        }
        __syncthreads();
        const BatchItem it = s_item;
        if (s_skip) {
            __syncthreads();
            continue;
        }
        load_pose_f_block(a.pose + 16 * it.pair, s_pose);
        const PoseF P = s_pose;
        const BatchPair *bp = a.pairs + it.pair;
        const float3 cf = make_float3(bp->cx, bp->cy, bp->cz);
        const int tbase = bp->tbase, n_tgt = bp->n_tgt;
        dfl acc[N_SUMS];
#pragma unroll
        for (int k = 0; k < N_SUMS; ++k)
            acc[k] = {0.0f, 0.0f};
        int j[PPT];
        float4 p[PPT], q[PPT];
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            const int i = it.i0 + tid + TH * u;
            j[u] = -1;
            if (i < it.i1) {
                j[u] = __ldcg(a.nn + i);
                p[u] = __ldg(a.src + i);
            }
        }
#pragma unroll
        for (int u = 0; u < PPT; ++u) {
            if ((unsigned)j[u] < (unsigned)n_tgt)
                q[u] = __ldg(a.tgt + tbase + j[u]);
            else if (it.i0 + tid + TH * u < it.i1)   // no valid match: report, leave it out
                atomicOr(&ctl->err, DEVERR_BOUNDS);
        }
#pragma unroll
        for (int u = 0; u < PPT; ++u)
            if ((unsigned)j[u] < (unsigned)n_tgt)
                accumulate_corr(acc, transform_pt(P, p[u]), q[u], cf);
        // warp sums through shared memory: lane l adds value l % 16 over
        // lanes 16 (l / 16) .. 16 (l / 16) + 15 in order, then the halves
#pragma unroll
        for (int k = 0; k < N_SUMS; ++k) {
            s_thi[warp][k][lane] = acc[k].hi;
            s_tlo[warp][k][lane] = acc[k].lo;
        }
        __syncwarp();
        {
            const int k = lane & 15, h = (lane >> 4) * 16;
            dfl v = {s_thi[warp][k][h], s_tlo[warp][k][h]};
#pragma unroll
            for (int t = 1; t < 16; ++t)
                v = df_acc(v, dfl{s_thi[warp][k][h + t], s_tlo[warp][k][h + t]});
            v = df_acc(v, df_shfl_xor(v, 16));
            if (lane < 16) {
                s_whi[warp][k] = v.hi;
                s_wlo[warp][k] = v.lo;
            }
        }
        __syncthreads();
        if (tid < N_SUMS) {   // the block's warps, in order
            dfl v = {s_whi[0][tid], s_wlo[0][tid]};
#pragma unroll
            for (int w = 1; w < WARPS; ++w)
                v = df_acc(v, dfl{s_whi[w][tid], s_wlo[w][tid]});
            a.partials[(size_t)itx * N_SUMS + tid] = make_float2(v.hi, v.lo);
            __threadfence();
        }
        __syncthreads();
        if (tid == 0)
            s_last = atomicAdd(&a.state[it.pair].items_done, 1u) == (unsigned)(bp->n_items - 1);
        __syncthreads();
        if (s_last) {
            __threadfence();
            // the pair's item sums in item order: thread t adds value t % 16
            // of items t/16, t/16 + TH/16, ...; the groups are then added in
            // order (pairs of groups by a shuffle, then the warps)
            const int item0 = bp->item0, n_items = bp->n_items;
            {
                const int k = tid & 15, grp = tid >> 4;
                dfl v = {0.0f, 0.0f};
                for (int b = grp; b < n_items; b += TH / 16) {
                    const float2 x = __ldcg(a.partials + (size_t)(item0 + b) * N_SUMS + k);
                    v = df_acc(v, dfl{x.x, x.y});
                }
                v = df_acc(v, df_shfl_xor(v, 16));
                if (lane < 16) {
                    s_whi[warp][lane] = v.hi;
                    s_wlo[warp][lane] = v.lo;
                }
            }
            __syncthreads();
            if (tid < N_SUMS) {
                dfl t = {s_whi[0][tid], s_wlo[0][tid]};
#pragma unroll
                for (int w = 1; w < WARPS; ++w)
                    t = df_acc(t, dfl{s_whi[w][tid], s_wlo[w][tid]});
                s_tot[tid] = t;
            }
            __syncthreads();
            if (warp == 0) {
                double rmse;
                BatchState *stp = a.state + it.pair;
                const bool ok = solve_update(s_tot, bp->n_src, cf, a.pose + 16 * it.pair, rmse);
                if (lane == 0) {
                    stp->items_done = 0u;
                    stp->last_rmse = rmse;
                    if (!ok) {
                        stp->err |= DEVERR_DEGENERATE;
                        stp->stop = 1;
                        atomicOr(&ctl->err, DEVERR_DEGENERATE);
                    } else {
                        const int k = stp->iters;
                        stp->iters = k + 1;
                        if (a.eps > 0.0 && k >= 1 && fabs(rmse - stp->prev_rmse) < a.eps)
                            stp->stop = 1;
                        stp->prev_rmse = rmse;
                    }
                }
            }
        }
        __syncthreads();   // s_item, s_pose and the sums are rewritten for the next item
    }
}

const BatchShape BATCH_SHAPES[BATCH_N_SHAPES] = {
    {256, 4, 2},   // 1024-point items
    {256, 2, 3},   // 512-point items, more warps per SM
    {512, 2, 1},   // 1024-point items, wide blocks
    {128, 4, 4},   // 512-point items, narrow blocks
    {256, 8, 2},   // 2048-point items
    {256, 2, 4},   // 512-point items, 64 registers: more warps per SM
    {256, 2, 5},   // 512-point items, 48 registers (spills some of the reduction's sums)
};

using IterKernel = void (*)(const BatchIterArgs);

static IterKernel iter_kernel(int shape, bool f64)
{
    switch (shape) {
    case 0: return f64 ? k_batch_iter<256, 4, 2, true> : k_batch_iter<256, 4, 2, false>;
    case 1: return f64 ? k_batch_iter<256, 2, 3, true> : k_batch_iter<256, 2, 3, false>;
    case 2: return f64 ? k_batch_iter<512, 2, 1, true> : k_batch_iter<512, 2, 1, false>;
    case 3: return f64 ? k_batch_iter<128, 4, 4, true> : k_batch_iter<128, 4, 4, false>;
    case 4: return f64 ? k_batch_iter<256, 8, 2, true> : k_batch_iter<256, 8, 2, false>;
    case 5: return f64 ? k_batch_iter<256, 2, 4, true> : k_batch_iter<256, 2, 4, false>;
    case 6: return f64 ? k_batch_iter<256, 2, 5, true> : k_batch_iter<256, 2, 5, false>;
    }
    return nullptr;
}

// 2 x WARPS x 16 x 33 floats = WARPS x 16 x 33 doubles
static size_t iter_smem(int shape) { return (size_t)2 * (BATCH_SHAPES[shape].threads / 32) * N_SUMS * 33 * 4; }

int batch_iter_blocks(int shape, bool f64)
{
    if (shape < 0 || shape >= BATCH_N_SHAPES)
        return 0;
    IterKernel k = iter_kernel(shape, f64);
    const size_t smem = iter_smem(shape);
    if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    int dev = 0, sms = 0, per_sm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, BATCH_SHAPES[shape].threads, smem) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return sms * per_sm;
}

cudaError_t launch_batch_iter(int shape, bool f64, int blocks, const BatchIterArgs &a, cudaStream_t st)
{
    IterKernel k = iter_kernel(shape, f64);
    if (!k || blocks < 1)
        return cudaErrorInvalidValue;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(blocks);
    cfg.blockDim = dim3(BATCH_SHAPES[shape].threads);
    cfg.dynamicSmemBytes = iter_smem(shape);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k, a);
}

}  // namespace vicp
