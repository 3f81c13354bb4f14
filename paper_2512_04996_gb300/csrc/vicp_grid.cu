// vicp_grid.cu -- grid build: bounding box, voxel occupancy histogram
// (Alg. 1, GPU part), offsets by a single-pass decoupled-lookback exclusive
// scan (the paper's memory-offset computation, Alg. 1 CPU part, moved onto
// the GPU), scatter of point indices into the CSR store (Alg. 2) and the
// brick list used by the exact global search.
#include "vicp_launch.h"

namespace vicp {

// ---------------------------------------------------------------------------
// Bounding box of the target (auto grid).  Floats are mapped to unsigned
// integers whose order matches the float order, so atomicMin/atomicMax
// reduce them; NaN coordinates are skipped by fminf/fmaxf.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned float_to_ordered(float f)
{
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__global__ void __launch_bounds__(256) k_bbox(const float4 *__restrict__ pts, int n, unsigned *__restrict__ out)
{
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
    k_bbox<<<blocks, 256, 0, st>>>(pts, n, bbox6);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// VOH: one thread per target point; lanes of a warp holding the same voxel
// key are grouped with __match_any_sync and their leader adds the group size
// (warp-aggregated atomics).  Block 0 also resets the scan's ticket, bumps
// its descriptor epoch and clears the outside/brick counters for this build.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_histogram(const float4 *__restrict__ pts, int n, GridGeom g,
                                                   int *__restrict__ keys, unsigned *__restrict__ counts,
                                                   DevCtl *__restrict__ ctl)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        ctl->scan_ticket = 0u;
        ctl->scan_epoch = ctl->scan_epoch + 1u;
        ctl->n_outside = 0;
        ctl->n_bricks = 0;
    }
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    int key = -2;   // lanes past the end match only each other and add nothing
    if (j < n) {
        const float4 q = __ldg(pts + j);
        key = voxel_key(g, q.x, q.y, q.z);
        keys[j] = key;
    }
    const unsigned peers = __match_any_sync(FULL_MASK, key);
    if (key >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1)
        atomicAdd(counts + key, (unsigned)__popc(peers));
}

cudaError_t launch_histogram(const float4 *pts, int n, const GridGeom &g, int *keys, unsigned *counts,
                             DevCtl *ctl, cudaStream_t st)
{
    k_histogram<<<(n + 255) / 256, 256, 0, st>>>(pts, n, g, keys, counts, ctl);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// MOC as a single-pass exclusive scan with decoupled lookback.
//
// Each CTA takes the next tile of 4096 counts from an atomic ticket (so
// every tile it waits on has already started), scans it, publishes its
// aggregate, then looks back over its predecessors' descriptors, 32 at a
// time, until it meets an inclusive prefix.  A descriptor is one 64-bit word
// [epoch:30 | flag:2 | value:32], so flag and value are read together; the
// epoch (bumped by the histogram kernel each build) makes the previous
// build's descriptors invalid without clearing them.  The wait is bounded by
// the global timer: on expiry the tile sets DEVERR_TIMEOUT and publishes a
// prefix anyway, so no successor waits on it.
//
// The same pass writes the occupancy bitmask (bit v set iff count[v] > 0).
// ---------------------------------------------------------------------------
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = SCAN_TILE / SCAN_THREADS;   // 16
constexpr int SCAN_WARPS = SCAN_THREADS / 32;
constexpr unsigned long long DESC_AGG = 1ull << 32;
constexpr unsigned long long DESC_PREFIX = 2ull << 32;
constexpr unsigned long long SCAN_TIMEOUT_NS = 200ull * 1000ull * 1000ull;   // 200 ms

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

__device__ __forceinline__ unsigned long long global_timer_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned warp_sum_u32(unsigned v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

__global__ void __launch_bounds__(SCAN_THREADS) k_scan(const unsigned *__restrict__ counts, long long V,
                                                       unsigned *__restrict__ off, unsigned *__restrict__ occ,
                                                       unsigned long long *__restrict__ desc,
                                                       DevCtl *__restrict__ ctl, int skip_tile)
{
    __shared__ unsigned s_tile, s_excl;
    __shared__ unsigned s_warp[SCAN_WARPS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (tid == 0)
        s_tile = atomicAdd(&ctl->scan_ticket, 1u);
    __syncthreads();
    const unsigned tile = s_tile;
    const unsigned long long epoch = (unsigned long long)(*(volatile unsigned *)&ctl->scan_epoch & 0x3fffffffu);
    const unsigned long long tag = epoch << 34;

    const long long base = (long long)tile * SCAN_TILE + (long long)tid * SCAN_ITEMS;
    unsigned c[SCAN_ITEMS];
    if (base + SCAN_ITEMS <= V) {
        const uint4 *p = reinterpret_cast<const uint4 *>(counts + base);
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS / 4; ++k) {
            const uint4 u = __ldcs(p + k);
            c[4 * k + 0] = u.x; c[4 * k + 1] = u.y; c[4 * k + 2] = u.z; c[4 * k + 3] = u.w;
        }
    } else {
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i)
            c[i] = (base + i < V) ? counts[base + i] : 0u;
    }
    unsigned bits = 0u, sum = 0u;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        bits |= (c[i] != 0u ? 1u : 0u) << i;
        const unsigned t = c[i];
        c[i] = sum;   // exclusive within the thread
        sum += t;
    }
    unsigned incl = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned y = __shfl_up_sync(FULL_MASK, incl, d);
        if (lane >= d)
            incl += y;
    }
    if (lane == 31)
        s_warp[warp] = incl;
    __syncthreads();

    if (warp == 0) {
        const unsigned w = (lane < SCAN_WARPS) ? s_warp[lane] : 0u;
        unsigned wi = w;
#pragma unroll
        for (int d = 1; d < SCAN_WARPS; d <<= 1) {
            const unsigned y = __shfl_up_sync(FULL_MASK, wi, d);
            if (lane >= d)
                wi += y;
        }
        const unsigned agg = __shfl_sync(FULL_MASK, wi, SCAN_WARPS - 1);
        if (lane < SCAN_WARPS)
            s_warp[lane] = wi - w;
        unsigned excl = 0u;
        if (tile == 0) {
            if (lane == 0 && skip_tile != 0)
                st_relaxed_u64(desc, tag | DESC_PREFIX | agg);
        } else {
            if (lane == 0 && (int)tile != skip_tile)
                st_relaxed_u64(desc + tile, tag | DESC_AGG | agg);
            long long look = (long long)tile - 1;
            const unsigned long long t0 = global_timer_ns();
            bool gave_up = false;
            for (;;) {
                const long long idx = look - lane;   // lane 0 is the nearest predecessor
                unsigned long long d;
                for (;;) {
                    d = (idx >= 0) ? ld_relaxed_u64(desc + idx) : (tag | DESC_PREFIX);
                    const bool ready = ((d >> 34) == epoch) && ((d & (3ull << 32)) != 0ull);
                    if (__all_sync(FULL_MASK, ready))
                        break;
                    const bool late = (global_timer_ns() - t0 > SCAN_TIMEOUT_NS) ||
                                      (*(volatile unsigned *)&ctl->err != 0u);
                    if (__any_sync(FULL_MASK, late)) {
                        gave_up = true;
                        break;
                    }
                    __nanosleep(32);
                }
                if (gave_up)
                    break;
                const unsigned pmask = __ballot_sync(FULL_MASK, (d & DESC_PREFIX) != 0ull);
                unsigned val = (unsigned)d;
                if (pmask) {
                    const int first = __ffs(pmask) - 1;
                    excl += warp_sum_u32(lane <= first ? val : 0u);
                    break;
                }
                excl += warp_sum_u32(val);
                look -= 32;
            }
            if (lane == 0) {
                if (gave_up)
                    atomicOr(&ctl->err, DEVERR_TIMEOUT);
                st_relaxed_u64(desc + tile, tag | DESC_PREFIX | (unsigned)(excl + agg));
            }
        }
        if (lane == 0)
            s_excl = excl;
    }
    __syncthreads();

    const unsigned prefix = s_excl + s_warp[warp] + (incl - sum);
    if (base + SCAN_ITEMS <= V) {
        uint4 *p = reinterpret_cast<uint4 *>(off + base);
#pragma unroll
        for (int k = 0; k < SCAN_ITEMS / 4; ++k)
            p[k] = make_uint4(prefix + c[4 * k], prefix + c[4 * k + 1], prefix + c[4 * k + 2], prefix + c[4 * k + 3]);
    } else {
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i)
            if (base + i < V)
                off[base + i] = prefix + c[i];
    }
    if (base <= V - 1 && V - 1 < base + SCAN_ITEMS)
        off[V] = prefix + sum;
    // Occupancy: threads 2k and 2k+1 hold the 32 bits of one word.
    const unsigned hi_bits = __shfl_down_sync(FULL_MASK, bits, 1);
    if ((tid & 1) == 0 && base < V)
        occ[base >> 5] = bits | (hi_bits << 16);
}

cudaError_t launch_scan(const unsigned *counts, const GridGeom &g, unsigned *off, unsigned *occ,
                        unsigned long long *desc, DevCtl *ctl, int skip_tile, cudaStream_t st)
{
    const long long tiles = scan_tiles(g.V);
    k_scan<<<(unsigned)tiles, SCAN_THREADS, 0, st>>>(counts, g.V, off, occ, desc, ctl, skip_tile);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// VDMA without locks: a warp's points of one voxel reserve their slots with
// one atomicSub on the voxel's count (which the histogram left at the final
// count), so the counts return to zero for the next build.  Slots fill from
// the end of each segment; the order inside a segment is unspecified.  The
// scatter also writes each point's coordinates and index next to its slot
// (csr), and lists target points outside an explicit grid.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_scatter(const float4 *__restrict__ pts, const int *__restrict__ keys, int n,
                                                 const unsigned *__restrict__ off, unsigned *__restrict__ counts,
                                                 int *__restrict__ ids, float4 *__restrict__ csr,
                                                 int *__restrict__ outside, DevCtl *__restrict__ ctl)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int key = (j < n) ? __ldg(keys + j) : -2;
    const unsigned peers = __match_any_sync(FULL_MASK, key);
    const int leader = __ffs(peers) - 1;
    const unsigned rank = __popc(peers & lanemask_lt());
    const unsigned cnt = __popc(peers);
    unsigned old = 0u;
    if ((int)(threadIdx.x & 31) == leader) {
        if (key >= 0)
            old = atomicSub(counts + key, cnt);
        else if (key == -1)
            old = (unsigned)atomicAdd(&ctl->n_outside, (int)cnt);
    }
    old = __shfl_sync(FULL_MASK, old, leader);
    if (key >= 0) {
        const unsigned pos = __ldg(off + key) + old - 1u - rank;
        if (pos < (unsigned)n) {
            const float4 q = __ldg(pts + j);
            ids[pos] = j;
            csr[pos] = make_float4(q.x, q.y, q.z, __int_as_float(j));
        } else {
            atomicOr(&ctl->err, DEVERR_BOUNDS);
        }
    } else if (key == -1) {
        outside[old + rank] = j;
    }
}

cudaError_t launch_scatter(const float4 *pts, const int *keys, int n, const unsigned *off, unsigned *counts,
                           int *ids, float4 *csr, int *outside, DevCtl *ctl, cudaStream_t st)
{
    k_scatter<<<(n + 255) / 256, 256, 0, st>>>(pts, keys, n, off, counts, ids, csr, outside, ctl);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Brick list for the exact global search: one warp per 8x8x8 brick reads the
// brick's 64 occupancy rows; a non-empty brick is appended with its box in
// float, widened outward so that it contains every point stored in the brick
// (the widening covers the rounding of the quantisation).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_bricks(const unsigned *__restrict__ occ, GridGeom g,
                                                int *__restrict__ list, float4 *__restrict__ box,
                                                DevCtl *__restrict__ ctl, long long n_bricks)
{
    const long long wid = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (wid >= n_bricks)
        return;   // whole warp
    const int bxi = (int)(wid % g.bx);
    const int byi = (int)((wid / g.bx) % g.by);
    const int bzi = (int)(wid / ((long long)g.bx * g.by));
    const int x0 = bxi * BRICK, y0 = byi * BRICK, z0 = bzi * BRICK;
    const int xw = min(BRICK, g.nx - x0);
    bool any = false;
#pragma unroll
    for (int r = lane; r < BRICK * BRICK; r += 32) {
        const int y = y0 + (r % BRICK), z = z0 + (r / BRICK);
        if (y < g.ny && z < g.nz) {
            const long long b = (long long)g.nx * (y + (long long)g.ny * z) + x0;
            any |= extract_bits(occ, b, xw) != 0u;
        }
    }
    if (__any_sync(FULL_MASK, any) && lane == 0) {
        const int slot = atomicAdd(&ctl->n_bricks, 1);
        list[slot] = (int)wid;
        const int x1 = min(x0 + BRICK, g.nx), y1 = min(y0 + BRICK, g.ny), z1 = min(z0 + BRICK, g.nz);
        // Exact bounds o + i*h in double, widened by 2^-20 of the grid's reach.
        const double h = (double)g.h;
        const double reach = fabs((double)g.ox) + fabs((double)g.oy) + fabs((double)g.oz) +
                             h * (double)(g.nx + g.ny + g.nz);
        const double m = reach * 0x1p-20;
        box[2 * slot + 0] = make_float4(__double2float_rd((double)g.ox + x0 * h - m),
                                        __double2float_rd((double)g.oy + y0 * h - m),
                                        __double2float_rd((double)g.oz + z0 * h - m), 0.0f);
        box[2 * slot + 1] = make_float4(__double2float_ru((double)g.ox + x1 * h + m),
                                        __double2float_ru((double)g.oy + y1 * h + m),
                                        __double2float_ru((double)g.oz + z1 * h + m), 0.0f);
    }
}

cudaError_t launch_bricks(const unsigned *occ, const GridGeom &g, int *brick_list, float4 *brick_box,
                          DevCtl *ctl, cudaStream_t st)
{
    const long long nb = (long long)g.bx * g.by * g.bz;
    const long long blocks = (nb * 32 + 255) / 256;
    k_bricks<<<(unsigned)blocks, 256, 0, st>>>(occ, g, brick_list, brick_box, ctl, nb);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Memory report helper: largest voxel count and number of occupied voxels.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_maxcount(const unsigned *__restrict__ off, long long V,
                                                  DevCtl *__restrict__ ctl)
{
    unsigned mx = 0u, occupied = 0u;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < V;
         v += (long long)gridDim.x * blockDim.x) {
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

cudaError_t launch_maxcount(const unsigned *off, const GridGeom &g, DevCtl *ctl, cudaStream_t st)
{
    long long blocks = (g.V + 255) / 256;
    if (blocks > 2432)
        blocks = 2432;
    k_maxcount<<<(unsigned)blocks, 256, 0, st>>>(off, g.V, ctl);
    return cudaGetLastError();
}

}  // namespace vicp
