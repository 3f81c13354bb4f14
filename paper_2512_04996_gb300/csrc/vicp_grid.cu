// vicp_grid.cu -- grid build: bounding box, voxel occupancy histogram
// (Alg. 1, GPU part), offsets by a single-pass decoupled-lookback exclusive
// scan (the paper's memory-offset computation, Alg. 1 CPU part, moved onto
// the GPU), scatter of point indices into the CSR store (Alg. 2) and the
// brick list used by the exact global search.
#include "vicp_launch.h"

namespace vicp {

// ---------------------------------------------------------------------------
// Bounding box of the target (auto grid): per-axis atomicMin/atomicMax on the
// order-preserving unsigned images of the coordinates; NaN coordinates are
// skipped by fminf/fmaxf.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bbox(const float4 *__restrict__ pts, int n, unsigned *__restrict__ out)
{
    pdl_begin();
    float lo[3] = {__int_as_float(0x7f800000), __int_as_float(0x7f800000), __int_as_float(0x7f800000)};
    float hi[3] = {-lo[0], -lo[1], -lo[2]};
    for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n; j += gridDim.x * blockDim.x) {
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
            atomicMin(out + a, float_to_ordered(lo[a]));
            atomicMax(out + 3 + a, float_to_ordered(hi[a]));
        }
    }
}

cudaError_t launch_bbox(const float4 *pts, int n, unsigned *bbox6, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(bbox6, 0xff, 3 * sizeof(unsigned), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(bbox6 + 3, 0x00, 3 * sizeof(unsigned), st);
    if (e != cudaSuccess)
        return e;
    int blocks = (n + 255) / 256;
    if (blocks > 1216)
        blocks = 1216;
    return launch_kernel(k_bbox, dim3(blocks), dim3(256), 0, st, pts, n, bbox6);
}

// ---------------------------------------------------------------------------
// VOH: one thread per target point; lanes of a warp holding the same voxel
// key are grouped with __match_any_sync and their leader adds the group size
// (warp-aggregated atomics).  The same grouping feeds the per-brick counts
// (brick level of the global search), the occupancy bitmask (one atomicOr
// per word) and the per-tile totals the scan starts from.  Block 0 also
// bumps the scan's descriptor epoch and clears the outside counter for this
// build.
//
// SPARSE (the hashed grid): the voxel's group leader inserts the key into the
// occupied-voxel table `ho` (its slot is broadcast to the group and stored
// per point in `pslot`), and the counts, the occupancy bits the scan reads
// (`socc`) and the tile totals are indexed by that slot instead of by the
// voxel key; the voxel occupancy bits (`occ`, read by the dilation) are set
// as in the dense grid.
// ---------------------------------------------------------------------------
// Slot tables of at most this many scan tiles keep each block's tile totals
// in shared memory: a voxel's slot is a hash, so the keys of one warp fall
// into many tiles, and per-warp atomics would pile onto the few tile words.
constexpr int HIST_SMEM_TILES = 1024;

template <bool AFTER_SOLVE, bool SPARSE>
__global__ void __launch_bounds__(256) k_histogram(const float4 *__restrict__ pts, int n, GridGeom g,
                                                   int *__restrict__ keys, unsigned *__restrict__ counts,
                                                   unsigned *__restrict__ bcounts, unsigned *__restrict__ occ,
                                                   unsigned *__restrict__ tile_sum, unsigned *__restrict__ sb_left,
                                                   unsigned *__restrict__ boxk, DevCtl *__restrict__ ctl,
                                                   HashTable ho, unsigned *__restrict__ socc,
                                                   int *__restrict__ pslot, float4 *__restrict__ copy_out)
{
    // In the ICP loop a build follows the previous iteration's reduction and
    // solve (AFTER_SOLVE), whose single-block tail leaves the GPU idle; the
    // histogram touches none of the arrays (nor control words) that the
    // solve reads or writes, and every kernel before the solve has completed
    // by the time the solve lets this launch start, so it does not wait and
    // the next build overlaps that tail.  Every reader of the solve's pose is
    // still ordered after it: the event recorded after the histogram
    // completes only after all earlier work of the stream, the dilation waits
    // for that event, and the search waits for the dilation.  After any
    // other kernel (a previous build's scatter, for one, which resets the
    // buffers this build fills) the histogram waits as every kernel does.
    if (AFTER_SOLVE)
        pdl_begin_nowait();
    else
        pdl_begin();
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->scan_epoch = ctl->scan_epoch + 1u;
        ctl->n_outside = 0;
        ctl->n_super = 0;
    }
    __shared__ unsigned s_tile[SPARSE ? HIST_SMEM_TILES : 1];
    const int n_tiles = SPARSE ? (int)((ho.mask + 1u) / SCAN_TILE) : 0;
    const bool block_tiles = SPARSE && n_tiles <= HIST_SMEM_TILES;
    if (block_tiles) {
        for (int t = threadIdx.x; t < n_tiles; t += blockDim.x)
            s_tile[t] = 0u;
        __syncthreads();
    }
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    int key = -2, bk = -2;   // lanes past the end match only each other and add nothing
    float4 q = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    if (j < n) {
        q = __ldg(pts + j);
        if (copy_out)   // pts is the caller's page-locked host cloud: keep a device copy
            copy_out[j] = q;
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
    const unsigned peers = __match_any_sync(FULL_MASK, key);
    int idx = key;   // index of the voxel's count: its key, or its slot in the table
    if (SPARSE) {
        int slot = -1;
        if (key >= 0 && lane == __ffs(peers) - 1) {
            slot = hash_insert(ho, (unsigned)key);
            if (slot < 0)
                atomicOr(&ctl->err, DEVERR_CAPACITY);
        }
        slot = __shfl_sync(FULL_MASK, slot, __ffs(peers) - 1);
        idx = key >= 0 ? slot : key;
        if (j < n)
            pslot[j] = idx;   // -1 outside the grid (or, with a full table, uncounted)
    }
    if (idx >= 0 && lane == __ffs(peers) - 1)
        atomicAdd(counts + idx, (unsigned)__popc(peers));
    const unsigned bpeers = __match_any_sync(FULL_MASK, bk);
    // the brick's exact bounds: the group's min and max of each coordinate
    // (order-preserving unsigned images of the floats; maxima as their
    // complements, so every word is an atomicMin from all ones)
    const unsigned ox = float_to_ordered(q.x), oy = float_to_ordered(q.y), oz = float_to_ordered(q.z);
    const unsigned mnx = __reduce_min_sync(bpeers, ox), mny = __reduce_min_sync(bpeers, oy),
                   mnz = __reduce_min_sync(bpeers, oz);
    const unsigned cmx = __reduce_min_sync(bpeers, ~ox), cmy = __reduce_min_sync(bpeers, ~oy),
                   cmz = __reduce_min_sync(bpeers, ~oz);
    if (bk >= 0 && lane == __ffs(bpeers) - 1) {
        // the group that makes a brick non-empty counts it for its super-brick
        // (the scatter writes a super-brick's box when its last brick is done)
        if (atomicAdd(bcounts + bk, (unsigned)__popc(bpeers)) == 0u && sb_left)
            atomicAdd(sb_left + bk / SUPER_BRICKS, 1u);
        if (boxk) {
            unsigned *b = boxk + 8 * bk;
            atomicMin(b + 0, mnx);
            atomicMin(b + 1, mny);
            atomicMin(b + 2, mnz);
            atomicMin(b + 4, cmx);
            atomicMin(b + 5, cmy);
            atomicMin(b + 6, cmz);
        }
    }
    // occupancy bit of the voxel (one atomicOr per word and warp)
    const int word = key >= 0 ? (key >> 5) : -2;
    const unsigned wpeers = __match_any_sync(FULL_MASK, word);
    const unsigned wbits = __reduce_or_sync(wpeers, key >= 0 ? 1u << (key & 31) : 0u);
    if (word >= 0 && lane == __ffs(wpeers) - 1)
        atomicOr(occ + word, wbits);
    if (SPARSE) {   // the scan's occupancy bit of the slot
        const int sw = idx >= 0 ? (idx >> 5) : -2;
        const unsigned spe = __match_any_sync(FULL_MASK, sw);
        const unsigned sbits = __reduce_or_sync(spe, idx >= 0 ? 1u << (idx & 31) : 0u);
        if (sw >= 0 && lane == __ffs(spe) - 1)
            atomicOr(socc + sw, sbits);
    }
    // per-tile totals for the scan (one atomicAdd per tile and warp; for a
    // small slot table per tile and block, through shared memory)
    const int tile = idx >= 0 ? (idx / SCAN_TILE) : -2;
    const unsigned tpeers = __match_any_sync(FULL_MASK, tile);
    if (tile >= 0 && lane == __ffs(tpeers) - 1)
        atomicAdd(block_tiles ? s_tile + tile : tile_sum + tile, (unsigned)__popc(tpeers));
    if (block_tiles) {
        __syncthreads();
        for (int t = threadIdx.x; t < n_tiles; t += blockDim.x)
            if (s_tile[t])
                atomicAdd(tile_sum + t, s_tile[t]);
    }
}

cudaError_t launch_histogram(const float4 *pts, int n, const GridGeom &g, int *keys, unsigned *counts,
                             unsigned *bcounts, unsigned *occ, unsigned *tile_sum, unsigned *sb_left,
                             unsigned *boxk, DevCtl *ctl, cudaStream_t st, bool after_solve, const HashTable *ho,
                             unsigned *socc, int *pslot, float4 *copy_out)
{
    // occ must hold zeros: the caller clears it beforehand
    const HashTable h = ho ? *ho : HashTable{nullptr, 0u, 32};
    if (ho)
        return launch_kernel(after_solve ? k_histogram<true, true> : k_histogram<false, true>, dim3((n + 255) / 256),
                             dim3(256), 0, st, pts, n, g, keys, counts, bcounts, occ, tile_sum, sb_left, boxk, ctl, h,
                             socc, pslot, copy_out);
    return launch_kernel(after_solve ? k_histogram<true, false> : k_histogram<false, false>, dim3((n + 255) / 256),
                         dim3(256), 0, st, pts, n, g, keys, counts, bcounts, occ, tile_sum, sb_left, boxk, ctl, h,
                         socc, pslot, copy_out);
}

// ---------------------------------------------------------------------------
// Brick offsets: one CTA scans the per-brick counts (few: V / 512) into
// brick offsets, and lists the non-empty bricks in ascending order with their
// point ranges and slot numbers.  The
// count and the non-empty flag are scanned together as one 64-bit value
// (flag count in the high half).  The counts are staged in shared memory with
// coalesced loads; each thread sums a contiguous run of bricks, one
// block-wide scan offsets the runs, and a second pass writes them.
// ---------------------------------------------------------------------------
constexpr int BS_THREADS = 1024;

__device__ __forceinline__ unsigned long long brick_pair(unsigned c)
{
    return (unsigned long long)c | ((unsigned long long)(c != 0u) << 32);
}

constexpr int BS_CHUNK = 24576;   // bricks staged in shared memory per pass (96 KB)

__global__ void __launch_bounds__(BS_THREADS) k_brick_scan(const unsigned *__restrict__ bcounts, int nbt,
                                                           unsigned *__restrict__ boff, int *__restrict__ list,
                                                           uint2 *__restrict__ range, int *__restrict__ bslot,
                                                           DevCtl *__restrict__ ctl)
{
    pdl_begin();
    extern __shared__ unsigned s_c[];   // [BS_CHUNK]
    __shared__ unsigned long long s_w[BS_THREADS / 32];
    __shared__ unsigned long long s_carry;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0)
        s_carry = 0ull;
    for (int c0 = 0; c0 < nbt; c0 += BS_CHUNK) {
        const int cn = min(BS_CHUNK, nbt - c0);
        for (int i0 = tid; i0 < cn; i0 += 8 * BS_THREADS) {   // coalesced, eight loads in flight
            unsigned v[8];
#pragma unroll
            for (int k = 0; k < 8; ++k)
                v[k] = (i0 + k * BS_THREADS < cn) ? __ldg(bcounts + c0 + i0 + k * BS_THREADS) : 0u;
#pragma unroll
            for (int k = 0; k < 8; ++k)
                if (i0 + k * BS_THREADS < cn)
                    s_c[i0 + k * BS_THREADS] = v[k];
        }
        __syncthreads();
        // thread t owns the contiguous bricks [t*per, (t+1)*per) of the chunk
        const int per = (cn + BS_THREADS - 1) / BS_THREADS;
        const int i0 = min(tid * per, cn), i1 = min(i0 + per, cn);
        unsigned long long sum = 0ull;
        for (int i = i0; i < i1; ++i)
            sum += brick_pair(s_c[i]);
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
        for (int i = i0; i < i1; ++i) {
            const unsigned c = s_c[i];
            const int bi = c0 + i;
            const unsigned start = (unsigned)run;
            boff[bi] = start;
            if (c) {
                const int slot = (int)(run >> 32);
                list[slot] = bi;
                range[slot] = make_uint2(start, start + c);
                bslot[bi] = slot;
            }
            run += brick_pair(c);
        }
        __syncthreads();
        if (tid == BS_THREADS - 1)
            s_carry = run;
        __syncthreads();
    }
    if (tid == 0) {
        boff[nbt] = (unsigned)s_carry;
        ctl->n_bricks = (int)(s_carry >> 32);
    }
}

// Many bricks per CTA in parallel: CTA b owns bricks [1024 b, 1024 b + 1024)
// and finds its starting offset and slot by summing the counts of all
// earlier bricks itself (cheap while bricks are few: at most 64 CTAs).
constexpr int BM_THREADS = 1024;
constexpr int BM_MAX_BRICKS = 64 * BM_THREADS;

__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v, unsigned long long *s_w)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULL_MASK, v, o);
    if (lane == 0)
        s_w[warp] = v;
    __syncthreads();
    unsigned long long t = 0ull;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w)
        t += s_w[w];
    __syncthreads();
    return t;
}

__global__ void __launch_bounds__(BM_THREADS) k_brick_scan_multi(const unsigned *__restrict__ bcounts, int nbt,
                                                                 unsigned *__restrict__ boff, int *__restrict__ list,
                                                                 uint2 *__restrict__ range, int *__restrict__ bslot,
                                                                 DevCtl *__restrict__ ctl)
{
    pdl_begin();
    __shared__ unsigned long long s_w[BM_THREADS / 32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int b0 = blockIdx.x * BM_THREADS;
    // the predecessors' counts, eight independent loads per round
    unsigned long long before = 0ull;
    for (int i0 = tid; i0 < b0; i0 += 8 * BM_THREADS) {
        unsigned v[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
            const int i = i0 + u * BM_THREADS;
            v[u] = i < b0 ? __ldg(bcounts + i) : 0u;
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
            before += brick_pair(v[u]);
    }
    before = block_sum_u64(before, s_w);
    const int i = b0 + tid;
    const unsigned c = i < nbt ? __ldg(bcounts + i) : 0u;
    const unsigned long long pc = brick_pair(c);
    unsigned long long incl = pc;
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
    const unsigned long long run = before + s_w[warp] + (incl - pc);
    if (i < nbt) {
        const unsigned start = (unsigned)run;
        boff[i] = start;
        if (c) {
            const int slot = (int)(run >> 32);
            list[slot] = i;
            range[slot] = make_uint2(start, start + c);
            bslot[i] = slot;
        }
        if (i == nbt - 1) {
            boff[nbt] = (unsigned)(run + pc);
            ctl->n_bricks = (int)((run + pc) >> 32);
        }
    }
}

cudaError_t launch_brick_scan(const unsigned *bcounts, const GridGeom &g, unsigned *boff, int *list, uint2 *range,
                              int *bslot, DevCtl *ctl, cudaStream_t st)
{
    const int nbt = brick_slots(g);
    if (nbt <= BM_MAX_BRICKS) {
        return launch_kernel(k_brick_scan_multi, dim3((nbt + BM_THREADS - 1) / BM_THREADS), dim3(BM_THREADS), 0, st,
                             bcounts, nbt, boff, list, range, bslot, ctl);
    }
    const size_t smem = BS_CHUNK * sizeof(unsigned);
    cudaError_t e = cudaFuncSetAttribute(k_brick_scan, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    return launch_kernel(k_brick_scan, dim3(1), dim3(BS_THREADS), smem, st, bcounts, nbt, boff, list, range, bslot,
                         ctl);
}

// ---------------------------------------------------------------------------
// MOC as a single-pass exclusive scan with lookback, without waiting.
//
// A tile is 16384 voxels; CTA t scans tile t, each thread owning WPT
// consecutive occupancy words (32 WPT voxels).  It reads its occupancy
// words, gathers the counts of the occupied voxels only (loads in flight
// together) and scans them.  Its exclusive prefix is the sum of every
// earlier tile's total, and the histogram has already written those totals,
// so nothing ever has to be waited for: the CTA looks back over its
// predecessors, 512 per round, and adds their totals down to the
// nearest predecessor that has already published its inclusive prefix (any
// one that has not is simply summed through).  Up to SCAN_DIRECT_TILES
// tiles, the CTA instead adds all earlier totals itself (a few L1-cached
// 16-byte loads per thread): every CTA reading its 512 nearest descriptors
// from L2 put hundreds of thousands of loads on a few lines, and the
// occupancy and count loads queued behind them (on the 226k scene the last
// tiles ended 12 us after the median one).  A published prefix is one
// 64-bit word [epoch:30 | flag:2 | value:32], so flag and value are read
// together; the epoch (bumped by the histogram each build) retires the
// previous build's words without clearing them.  The tile totals stay
// untouched while the scan runs (predecessors are read throughout); the
// scatter, which runs next, zeroes them for the following build.
//
// Output.  Dense (512 threads x 1 word): every off[v], staged in shared
// memory and written with coalesced 16-byte stores.  Sparse (256 threads x
// 2 words, the build's form): only the entries the build and the searches
// read -- off[v] and off[v + 1] of every occupied voxel v, off[32 k] for
// every occupancy word k, and off[V] -- about 1/15 of the array's bytes at
// the scene workloads' 0.5% occupancy.  Every other entry equals the nearest
// written entry before it in its word (an empty voxel adds nothing), which
// is how k_offsets_fill completes the array when a caller asks for it.
// ---------------------------------------------------------------------------
constexpr unsigned long long DESC_PREFIX = 2ull << 32;
constexpr int LOOKBACK = 512;   // predecessors examined per lookback round
constexpr int SCAN_DIRECT_TILES = 4096;   // up to this many tiles: no lookback, earlier totals summed directly

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long *p, unsigned long long v)
{
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ unsigned warp_sum_u32(unsigned v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// Exclusive block-wide scan of one value per thread (WARPS warps); returns
// the thread's exclusive prefix, *total gets the block total.  Uses
// s_w[WARPS + 1].
template <int WARPS>
__device__ __forceinline__ unsigned block_excl_scan(unsigned v, unsigned *s_w, unsigned *total)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned incl = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned y = __shfl_up_sync(FULL_MASK, incl, d);
        if (lane >= d)
            incl += y;
    }
    if (lane == 31)
        s_w[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned w = lane < WARPS ? s_w[lane] : 0u;
        unsigned wi = w;
#pragma unroll
        for (int d = 1; d < WARPS; d <<= 1) {
            const unsigned y = __shfl_up_sync(FULL_MASK, wi, d);
            if (lane >= d)
                wi += y;
        }
        if (lane < WARPS)
            s_w[lane] = wi - w;
        if (lane == WARPS - 1)
            s_w[WARPS] = wi;
    }
    __syncthreads();
    *total = s_w[WARPS];
    return s_w[warp] + (incl - v);
}

// Sum of the counts of the set bits of `bits` (voxels base + i), four loads
// in flight per round.
__device__ __forceinline__ unsigned word_count_sum(const unsigned *__restrict__ counts, long long base, unsigned bits)
{
    unsigned sum = 0u;
    while (bits) {
        unsigned c[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            c[u] = 0u;
            if (bits) {
                c[u] = __ldg(counts + base + (__ffs(bits) - 1));
                bits &= bits - 1u;
            }
        }
        sum += (c[0] + c[1]) + (c[2] + c[3]);
    }
    return sum;
}

// A word with more than this many occupied voxels takes its 32 counts with
// eight 16-byte loads (one round trip; the counts of empty voxels are zero
// at scan time) instead of one load per occupied voxel.  A plane of the
// cloud facing the grid's z axis fills whole scan tiles, and their threads
// would otherwise take 16 rounds of loads per word to sum the counts and
// then 32 dependent load-add steps to write the offsets: on the 226k depth
// scene those few tiles ended 13 us after all others.
constexpr int SCAN_DENSE_BITS = 4;

// Sum of the 32 counts of the word at voxel b (b a multiple of 32).
__device__ __forceinline__ unsigned word_count_sum_vec(const unsigned *__restrict__ counts, long long b)
{
    const uint4 *c4 = reinterpret_cast<const uint4 *>(counts + b);
    unsigned sum = 0u;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint4 c[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            c[q] = __ldg(c4 + 4 * h + q);
#pragma unroll
        for (int q = 0; q < 4; ++q)
            sum += (c[q].x + c[q].y) + (c[q].z + c[q].w);
    }
    return sum;
}

// All 32 offsets of the word at voxel b from its first one, `run`, written
// with 16-byte stores; returns the offset after the word.
__device__ __forceinline__ unsigned word_offsets_vec(const unsigned *__restrict__ counts, unsigned *__restrict__ off,
                                                     long long b, unsigned run)
{
    const uint4 *c4 = reinterpret_cast<const uint4 *>(counts + b);
    uint4 *o4 = reinterpret_cast<uint4 *>(off + b);
#pragma unroll
    for (int h = 0; h < 2; ++h) {
        uint4 c[4];
#pragma unroll
        for (int q = 0; q < 4; ++q)
            c[q] = __ldg(c4 + 4 * h + q);   // from L1
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            uint4 o;
            o.x = run;
            run += c[q].x;
            o.y = run;
            run += c[q].y;
            o.z = run;
            run += c[q].z;
            o.w = run;
            run += c[q].w;
            o4[4 * h + q] = o;
        }
    }
    return run;
}

template <int THREADS, int WPT, bool DENSE>
__global__ void __launch_bounds__(THREADS, DENSE ? 3 : 1024 / THREADS)
    k_scan(const unsigned *__restrict__ counts, long long V, unsigned *__restrict__ off,
           const unsigned *__restrict__ occ, const unsigned *__restrict__ tile_sum,
           unsigned long long *__restrict__ desc, const DevCtl *__restrict__ ctl)
{
    static_assert(THREADS * WPT * 32 == SCAN_TILE, "tile");
    static_assert(!DENSE || WPT == 1, "the dense output stages one word per thread");
    constexpr int WARPS = THREADS / 32;
    pdl_begin();
    __shared__ unsigned s_epoch, s_w[WARPS + 1], s_first[WARPS], s_sum[WARPS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const unsigned tile = blockIdx.x;
    if (tid == 0)   // read by one thread per CTA (a hot line otherwise)
        s_epoch = *(volatile const unsigned *)&ctl->scan_epoch & 0x3fffffffu;

    // this thread's words and the counts of their occupied voxels; the first
    // lookback round's loads go out at the same time (they depend on the
    // tile index only)
    const long long base = (long long)tile * SCAN_TILE + 32ll * WPT * tid;
    unsigned bits[WPT];
#pragma unroll
    for (int w = 0; w < WPT; ++w)
        bits[w] = base + 32 * w < V ? __ldg(occ + (base >> 5) + w) : 0u;
    constexpr int CPT = LOOKBACK / THREADS;   // predecessors per thread and round
    const bool direct = gridDim.x <= SCAN_DIRECT_TILES;
    unsigned long long d0[CPT];
    unsigned t0[CPT];
    unsigned before = 0u;   // direct: this thread's part of the earlier tiles' totals
    if (direct) {
        if ((reinterpret_cast<uintptr_t>(tile_sum) & 15u) == 0u) {
            for (int j = 4 * tid; j < (int)tile; j += 4 * THREADS) {
                if (j + 4 <= (int)tile) {
                    const uint4 q = __ldg(reinterpret_cast<const uint4 *>(tile_sum + j));
                    before += (q.x + q.y) + (q.z + q.w);
                } else {
                    for (int k = j; k < (int)tile; ++k)
                        before += __ldg(tile_sum + k);
                }
            }
        } else {
            for (int j = tid; j < (int)tile; j += THREADS)
                before += __ldg(tile_sum + j);
        }
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            d0[c] = 0ull;
            t0[c] = 0u;
        }
    } else {
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const long long idx = (long long)tile - 1 - (c * THREADS + tid);
            d0[c] = idx >= 0 ? ld_relaxed_u64(desc + idx) : 0ull;
            t0[c] = idx >= 0 ? __ldg(tile_sum + idx) : 0u;
        }
    }
    unsigned sum = 0u;
    if (DENSE) {
#pragma unroll
        for (int i = 0; i < 32; ++i)
            sum += ((bits[0] >> i) & 1u) ? __ldg(counts + base + i) : 0u;
    } else {
#pragma unroll
        for (int w = 0; w < WPT; ++w) {
            const long long b = base + 32 * w;
            if (__popc(bits[w]) > SCAN_DENSE_BITS && b + 32 <= V)
                sum += word_count_sum_vec(counts, b);
            else
                sum += word_count_sum(counts, b, bits[w]);
        }
    }
    if (direct) {
        before = warp_sum_u32(before);
        if (lane == 0)
            s_sum[warp] = before;   // read after the block scan's barriers
    }
    unsigned tile_total;
    const unsigned thread_excl = block_excl_scan<WARPS>(sum, s_w, &tile_total);   // also orders s_epoch
    const unsigned long long tag = (unsigned long long)s_epoch << 34;

    // lookback: LOOKBACK predecessors per round, nearest first (thread i
    // looks at tile - 1 - (c THREADS + i), c < CPT); sum the totals before the
    // nearest published prefix
    unsigned excl = 0u;
    if (direct) {
#pragma unroll
        for (int w = 0; w < WARPS; ++w)
            excl += s_sum[w];
    }
    for (long long look = direct ? -1ll : (long long)tile - 1; look >= 0; look -= LOOKBACK) {
        bool pre[CPT];
        unsigned v[CPT];
        unsigned mine = LOOKBACK;   // this warp's nearest published prefix
#pragma unroll
        for (int c = 0; c < CPT; ++c) {
            const long long idx = look - (c * THREADS + tid);
            pre[c] = false;
            v[c] = 0u;
            if (idx >= 0) {
                unsigned long long d = d0[c];
                unsigned t = t0[c];
                if (look != (long long)tile - 1) {
                    d = ld_relaxed_u64(desc + idx);
                    t = __ldg(tile_sum + idx);
                }
                pre[c] = (d >> 34) == (tag >> 34) && (d & DESC_PREFIX);
                v[c] = pre[c] ? (unsigned)d : t;
            }
            const unsigned pm = __ballot_sync(FULL_MASK, pre[c]);
            if (pm)
                mine = min(mine, (unsigned)(c * THREADS + warp * 32 + __ffs(pm) - 1));
        }
        if (lane == 0)
            s_first[warp] = mine;
        __syncthreads();
        unsigned first = LOOKBACK;
#pragma unroll
        for (int w = 0; w < WARPS; ++w)
            first = min(first, s_first[w]);
        unsigned part = 0u;
#pragma unroll
        for (int c = 0; c < CPT; ++c)
            part += (unsigned)(c * THREADS + tid) <= first ? v[c] : 0u;
        const unsigned ws = warp_sum_u32(part);
        if (lane == 0)
            s_sum[warp] = ws;
        __syncthreads();
        unsigned round = 0u;
#pragma unroll
        for (int w = 0; w < WARPS; ++w)
            round += s_sum[w];
        excl += round;
        __syncthreads();   // s_first / s_sum are reused
        if (first < LOOKBACK)
            break;
    }
    if (tid == 0 && !direct)
        st_relaxed_u64(desc + tile, tag | DESC_PREFIX | (unsigned)(excl + tile_total));

    unsigned run = excl + thread_excl;
    if (!DENSE) {
        // the entries the build and the searches read, straight from registers
#pragma unroll
        for (int w = 0; w < WPT; ++w) {
            const long long b = base + 32 * w;
            if (b > V)
                break;
            if (__popc(bits[w]) > SCAN_DENSE_BITS && b + 32 <= V) {   // every entry of the word
                run = word_offsets_vec(counts, off, b, run);
                if (b + 32 == V)
                    off[V] = run;
                continue;
            }
            off[b] = run;   // the word's first entry (off[V] itself when b == V)
            for (unsigned m = bits[w]; m; m &= m - 1u) {
                const int i = __ffs(m) - 1;
                if (i)
                    off[b + i] = run;
                run += __ldg(counts + b + i);   // from L1
                if (i < 31 && !((bits[w] >> (i + 1)) & 1u))
                    off[b + i + 1] = run;
            }
            if (b < V && b + 32 >= V)   // the word holding voxel V-1 closes the array
                off[V] = run;
        }
        return;
    }

    // the 32 offsets of this thread, staged in shared memory (row stride 33
    // words: conflict-free both ways) and written out with coalesced 16-byte
    // stores
    extern __shared__ unsigned s_off[];   // [THREADS][33]
#pragma unroll
    for (int i = 0; i < 32; ++i) {   // the counts again, from L1
        s_off[tid * 33 + i] = run;
        run += ((bits[0] >> i) & 1u) ? __ldg(counts + base + i) : 0u;
    }
    if (base < V && base + 32 >= V)   // the thread holding voxel V-1 closes the array
        off[V] = run;
    __syncthreads();
    const long long tbase = (long long)tile * SCAN_TILE;
#pragma unroll
    for (int j = 0; j < SCAN_TILE / (4 * THREADS); ++j) {
        const int v = 4 * tid + 4 * THREADS * j;   // voxel within the tile
        const unsigned *r = s_off + (v >> 5) * 33 + (v & 31);
        const long long gv = tbase + v;
        if (gv + 4 <= V) {
            *reinterpret_cast<uint4 *>(off + gv) = make_uint4(r[0], r[1], r[2], r[3]);
        } else {
#pragma unroll
            for (int i = 0; i < 4; ++i)
                if (gv + i < V)
                    off[gv + i] = r[i];
        }
    }
}

cudaError_t launch_scan(const unsigned *counts, const GridGeom &g, unsigned *off, const unsigned *occ,
                        const unsigned *tile_sum, unsigned long long *desc, const DevCtl *ctl, cudaStream_t st,
                        bool dense)
{
    const long long tiles = scan_tiles(g.V);
    if (!dense)
        return launch_kernel(k_scan<256, 2, false>, dim3((unsigned)tiles), dim3(256), 0, st, counts, g.V, off, occ,
                             tile_sum, desc, ctl);
    constexpr int T = 512;
    const size_t smem = (size_t)T * 33 * sizeof(unsigned);
    cudaError_t e = cudaFuncSetAttribute(k_scan<T, 1, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    return launch_kernel(k_scan<T, 1, true>, dim3((unsigned)tiles), dim3(T), smem, st, counts, g.V, off, occ,
                         tile_sum, desc, ctl);
}

// ---------------------------------------------------------------------------
// Completes a sparse offsets array (k_scan's sparse output): an entry the
// scan did not write equals the nearest written one before it in its
// occupancy word.  Thread per voxel; reads only written entries and writes
// only the others, so threads never touch an entry another one writes.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_offsets_fill(unsigned *__restrict__ off, const unsigned *__restrict__ occ,
                                                      long long V)
{
    pdl_begin();
    const long long v = (long long)blockIdx.x * 256 + threadIdx.x;
    if (v >= V)
        return;
    const unsigned bits = __ldg(occ + (v >> 5));
    const unsigned written = 1u | bits | (bits << 1);
    const int i = (int)(v & 31);
    if ((written >> i) & 1u)
        return;
    const int j = 31 - __clz(written & ((1u << i) - 1u));   // i >= 1 here
    off[v] = off[(v & ~31ll) + j];
}

cudaError_t launch_offsets_fill(unsigned *off, const unsigned *occ, long long V, cudaStream_t st)
{
    return launch_kernel(k_offsets_fill, dim3((unsigned)((V + 255) / 256)), dim3(256), 0, st, off, occ, V);
}

// ---------------------------------------------------------------------------
// Brick boxes as floats for the global search, written inside the scatter.
// The histogram has merged every brick's exact bounds into boxk (by brick
// key: min x, y, z and the complements of max x, y, z, each an atomicMin
// from all ones), so they are complete when the scatter runs.  The group
// whose slot reservation brings a brick's count to zero writes the brick's
// float box (every stored point lies inside it as float values, which is
// what the search's lower bound needs), with the brick's point range
// [lo.w, hi.w) in the w fields as integer bits, then counts its super-brick
// down (sb_left, counted up by the histogram); the last brick's warp writes
// the super-brick's union box with its brick-slot range (bricks of a
// super-brick hold consecutive slots).  Everything read here was written by
// an earlier kernel, so no fence is needed.  The scatter also resets the
// other boxk buffer, which the next build's histogram fills.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void finish_brick(int slot, int bk, const unsigned *__restrict__ boxk,
                                             const uint2 *__restrict__ range, float4 *__restrict__ box)
{
    const uint4 lo = __ldg(reinterpret_cast<const uint4 *>(boxk) + 2 * bk);
    const uint4 hi = __ldg(reinterpret_cast<const uint4 *>(boxk) + 2 * bk + 1);
    const uint2 r = __ldg(range + slot);
    box[2 * slot] = make_float4(ordered_to_float(lo.x), ordered_to_float(lo.y), ordered_to_float(lo.z),
                                __uint_as_float(r.x));
    box[2 * slot + 1] = make_float4(ordered_to_float(~hi.x), ordered_to_float(~hi.y), ordered_to_float(~hi.z),
                                    __uint_as_float(r.y));
}

// Super-brick sb's box by the whole warp: its bricks' bounds (two brick keys
// per lane; a brick is non-empty when its offsets differ), their union, and
// the slot range from the first non-empty brick's slot and their number.
__device__ __forceinline__ void finish_super(int sb, const unsigned *__restrict__ boxk,
                                             const unsigned *__restrict__ boff, const int *__restrict__ bslot,
                                             float4 *__restrict__ sb_box, DevCtl *__restrict__ ctl)
{
    static_assert(SUPER_BRICKS == 64, "two bricks per lane");
    const int lane = threadIdx.x & 31;
    unsigned lx = 0xffffffffu, ly = 0xffffffffu, lz = 0xffffffffu;
    unsigned hx = 0xffffffffu, hy = 0xffffffffu, hz = 0xffffffffu, first = 0xffffffffu;
    int n = 0;
#pragma unroll
    for (int t = 0; t < 2; ++t) {
        const int k = sb * SUPER_BRICKS + 32 * t + lane;
        const bool ne = __ldg(boff + k + 1) > __ldg(boff + k);
        if (ne) {
            const uint4 lo = __ldg(reinterpret_cast<const uint4 *>(boxk) + 2 * k);
            const uint4 hi = __ldg(reinterpret_cast<const uint4 *>(boxk) + 2 * k + 1);
            lx = min(lx, lo.x);
            ly = min(ly, lo.y);
            lz = min(lz, lo.z);
            hx = min(hx, hi.x);
            hy = min(hy, hi.y);
            hz = min(hz, hi.z);
            first = min(first, (unsigned)__ldg(bslot + k));
        }
        n += __popc(__ballot_sync(FULL_MASK, ne));
    }
    lx = __reduce_min_sync(FULL_MASK, lx);
    ly = __reduce_min_sync(FULL_MASK, ly);
    lz = __reduce_min_sync(FULL_MASK, lz);
    hx = __reduce_min_sync(FULL_MASK, hx);
    hy = __reduce_min_sync(FULL_MASK, hy);
    hz = __reduce_min_sync(FULL_MASK, hz);
    first = __reduce_min_sync(FULL_MASK, first);
    if (lane == 0) {
        const int s = atomicAdd(&ctl->n_super, 1);
        sb_box[2 * s] = make_float4(ordered_to_float(lx), ordered_to_float(ly), ordered_to_float(lz),
                                    __uint_as_float(first));
        sb_box[2 * s + 1] = make_float4(ordered_to_float(~hx), ordered_to_float(~hy), ordered_to_float(~hz),
                                        __uint_as_float(first + (unsigned)n));
    }
}

// ---------------------------------------------------------------------------
// VDMA without locks: a warp's points of one voxel reserve their slots with
// one atomicSub on the voxel's count (which the histogram left at the final
// count), so the counts return to zero for the next build.  Slots fill from
// the end of each segment; the order inside a segment is unspecified.  The
// scatter also writes each point's coordinates and index next to its slot
// (csr), does the same per brick (bpts, brick-ordered), finalises the brick
// and super-brick boxes (above), and lists target points outside an
// explicit grid.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_scatter(const float4 *__restrict__ pts, const int *__restrict__ keys, int n,
                                                 GridGeom g, const unsigned *__restrict__ off,
                                                 unsigned *__restrict__ counts, const unsigned *__restrict__ boff,
                                                 unsigned *__restrict__ bcounts, const int *__restrict__ bslot,
                                                 const unsigned *__restrict__ boxk, unsigned *__restrict__ boxk_next,
                                                 long long boxk_words, const uint2 *__restrict__ range,
                                                 float4 *__restrict__ box, unsigned *__restrict__ sb_left,
                                                 float4 *__restrict__ sb_box, int *__restrict__ ids,
                                                 float4 *__restrict__ csr, float4 *__restrict__ bpts,
                                                 int *__restrict__ outside, unsigned *__restrict__ tile_sum,
                                                 int n_tiles, unsigned *__restrict__ occ_next,
                                                 long long occ_next_words, DevCtl *__restrict__ ctl,
                                                 unsigned *__restrict__ empty_next, long long empty_next_words,
                                                 unsigned *__restrict__ zero_next, long long zero_next_words)
{
    pdl_begin();
    // the scan is done with the tile totals: zero them for the next build,
    // and clear the occupancy and brick-bound buffers the next build will fill
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_tiles; t += gridDim.x * blockDim.x)
        tile_sum[t] = 0u;
    for (long long w = blockIdx.x * blockDim.x + threadIdx.x; w < empty_next_words; w += gridDim.x * blockDim.x)
        empty_next[w] = HASH_EMPTY;
    for (long long w = blockIdx.x * blockDim.x + threadIdx.x; w < zero_next_words; w += gridDim.x * blockDim.x)
        zero_next[w] = 0u;
    for (long long w = blockIdx.x * blockDim.x + threadIdx.x; w < boxk_words; w += gridDim.x * blockDim.x)
        boxk_next[w] = 0xffffffffu;
    for (long long w = blockIdx.x * blockDim.x + threadIdx.x; w < occ_next_words; w += gridDim.x * blockDim.x)
        occ_next[w] = 0u;
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int key = (j < n) ? __ldg(keys + j) : -2;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    int bk = key;
    if (key >= 0) {
        q = __ldg(pts + j);
        int ix, iy, iz;
        // inside, so the same quantisation as the histogram's gives the brick
        bk = voxel_coords(g, q.x, q.y, q.z, ix, iy, iz) ? brick_key(g, ix, iy, iz) : -1;
        q.w = __int_as_float(j);
    }
    // voxel segment
    {
        const unsigned peers = __match_any_sync(FULL_MASK, key);
        const int leader = __ffs(peers) - 1;
        const unsigned rank = __popc(peers & lanemask_lt());
        const unsigned cnt = __popc(peers);
        unsigned old = 0u;
        if (lane == leader) {
            if (key >= 0)
                old = atomicSub(counts + key, cnt);
            else if (key == -1)
                old = (unsigned)atomicAdd(&ctl->n_outside, (int)cnt);
        }
        old = __shfl_sync(FULL_MASK, old, leader);
        if (key >= 0) {
            const unsigned pos = __ldg(off + key) + old - 1u - rank;
            if (pos < (unsigned)n) {
                ids[pos] = j;
                csr[pos] = q;
            } else {
                atomicOr(&ctl->err, DEVERR_BOUNDS);
            }
        } else if (key == -1) {
            outside[old + rank] = j;
        }
    }
    // brick segment; the group that brings the brick's count to zero writes
    // its float box, and the one that finishes a super-brick has its warp
    // write the super-brick's box (above)
    {
        const unsigned peers = __match_any_sync(FULL_MASK, bk);
        const int leader = __ffs(peers) - 1;
        const unsigned rank = __popc(peers & lanemask_lt());
        unsigned old = 0u;
        int fin = -1;   // a super-brick this lane's group finished
        if (lane == leader && bk >= 0) {
            const unsigned cnt = (unsigned)__popc(peers);
            old = atomicSub(bcounts + bk, cnt);
            if (old == cnt) {   // the brick's last points
                finish_brick(__ldg(bslot + bk), bk, boxk, range, box);
                const int sb = bk / SUPER_BRICKS;
                if (atomicSub(sb_left + sb, 1u) == 1u)
                    fin = sb;
            }
        }
        old = __shfl_sync(FULL_MASK, old, leader);
        if (bk >= 0) {
            const unsigned pos = __ldg(boff + bk) + old - 1u - rank;
            if (pos < (unsigned)n)
                bpts[pos] = q;
            else
                atomicOr(&ctl->err, DEVERR_BOUNDS);
        }
        for (unsigned fm = __ballot_sync(FULL_MASK, fin >= 0); fm; fm &= fm - 1u)
            finish_super(__shfl_sync(FULL_MASK, fin, __ffs(fm) - 1), boxk, boff, bslot, sb_box, ctl);
    }
}

cudaError_t launch_scatter(const float4 *pts, const int *keys, int n, const GridGeom &g, const unsigned *off,
                           unsigned *counts, const unsigned *boff, unsigned *bcounts, const int *bslot,
                           const unsigned *boxk, unsigned *boxk_next, long long boxk_next_words, const uint2 *range,
                           float4 *box, unsigned *sb_left, float4 *sb_box, int *ids, float4 *csr, float4 *bpts,
                           int *outside, unsigned *tile_sum, unsigned *occ_next, long long occ_next_words,
                           DevCtl *ctl, cudaStream_t st, long long n_tiles, unsigned *empty_next,
                           long long empty_next_words, unsigned *zero_next, long long zero_next_words)
{
    return launch_kernel(k_scatter, dim3((n + 255) / 256), dim3(256), 0, st, pts, keys, n, g, off, counts, boff,
                         bcounts, bslot, boxk, boxk_next, boxk_next_words, range, box, sb_left, sb_box, ids, csr,
                         bpts, outside, tile_sum, (int)(n_tiles >= 0 ? n_tiles : scan_tiles(g.V)), occ_next,
                         occ_next_words, ctl, empty_next, empty_next_words, zero_next, zero_next_words);
}

// ---------------------------------------------------------------------------
// Memory report helper: largest voxel count and number of occupied voxels.
// ---------------------------------------------------------------------------
// keys (sparse grid: the occupied-voxel table, whose offsets are valid at
// occupied slots and just past them only): empty slots are skipped.
__global__ void __launch_bounds__(256) k_maxcount(const unsigned *__restrict__ off, long long V,
                                                  DevCtl *__restrict__ ctl, const unsigned *__restrict__ keys)
{
    pdl_begin();
    unsigned mx = 0u, occupied = 0u;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
        if (keys && keys[v] == HASH_EMPTY)
            continue;
        const unsigned c = off[v + 1] - off[v];
        mx = max(mx, c);
        occupied += c != 0u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mx = max(mx, __shfl_xor_sync(FULL_MASK, mx, o));
        occupied += __shfl_xor_sync(FULL_MASK, occupied, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&ctl->max_count, mx);
        atomicAdd(&ctl->occupied, occupied);
    }
}

cudaError_t launch_maxcount(const unsigned *off, const GridGeom &g, DevCtl *ctl, cudaStream_t st,
                            const unsigned *keys)
{
    long long blocks = (g.V + 255) / 256;
    if (blocks > 2432)
        blocks = 2432;
    return launch_kernel(k_maxcount, dim3((unsigned)blocks), dim3(256), 0, st, off, g.V, ctl, keys);
}

}  // namespace vicp
