// vicp_device.cuh -- types, constants and device helpers shared by the CUDA
// translation units of the library (not by the host API's callers).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace vicp {

constexpr unsigned FULL_MASK = 0xffffffffu;

// Programmatic dependent launch.  Every kernel of the library starts with
// pdl_begin(): it waits until the kernel before it in the stream has
// completed and its writes are visible (so each kernel sees exactly what
// plain stream order gives it), then lets the next kernel's blocks be
// scheduled onto the SMs while this one runs, which takes the launch latency
// out of the gap between the two.
__device__ __forceinline__ void pdl_begin()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The start of a kernel that does not wait for the kernel before it: only
// for a kernel that reads nothing that kernel writes and writes nothing it
// reads.  It starts once every block of the kernel before it has passed that
// kernel's own wait, so everything older has completed.
__device__ __forceinline__ void pdl_begin_nowait()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// Voxel grid geometry passed by value to kernels.  Keys are
// x + nx*(y + ny*z) (x fastest, the neighbour offsets +-1, +-2^N, +-2^2N of
// Alg. 3); V < 2^31 so keys fit int32.
struct GridGeom {
    float ox, oy, oz;   // origin (minimum corner)
    float inv_h;        // (float)(1.0 / (double)h)
    float h;
    int nx, ny, nz;
    long long V;
    int bx, by, bz;     // brick grid: ceil(dims / BRICK)
    int sx, sy, sz;     // super-brick grid: ceil(brick dims / SUPER)
};

// Brick edge (voxels) of the coarse level used by the exact global search,
// and super-brick edge (bricks) of the level above it.
constexpr int BRICK = 8;
constexpr int SUPER = 4;
constexpr int SUPER_BRICKS = SUPER * SUPER * SUPER;

// Bits of the device status word.
constexpr unsigned DEVERR_TIMEOUT = 1u;      // a bounded wait gave up
constexpr unsigned DEVERR_DEGENERATE = 2u;   // rank(H) < 2 in a solve
constexpr unsigned DEVERR_BOUNDS = 4u;       // an index failed its bounds check (write skipped)
constexpr unsigned DEVERR_CAPACITY = 8u;     // a hashed voxel table could not take a key (insert skipped)

// Per-context control block in device memory.  Kernels of one stream use it
// in launch order; the comments say which kernel writes each field.
struct DevCtl {
    unsigned bar_count;     // batched iteration: blocks arrived at the grid barrier
    unsigned scan_epoch;    // scan: descriptor epoch; bumped by the histogram kernel
    int n_outside;          // scatter: target points outside the grid; reset by histogram
    int n_bricks;           // brick list length; reset by histogram
    int fb_count;           // correspond: fallback queries; reset by the fallback kernel
    unsigned fb_done;       // fallback: finished blocks (the last one resets fb_count)
    unsigned err;           // DEVERR_* bits; cleared by the host
    unsigned max_count;     // memory report: largest voxel count
    unsigned occupied;      // memory report: occupied voxels
    unsigned red_done;      // reduction: finished blocks (the last one solves and resets it)
    int hv_count;           // correspond: dense segments listed; reset by the fallback kernel
    unsigned bar_gen;       // batched iteration: grid barrier generation
    int n_super;            // non-empty super-bricks; reset by the histogram
    unsigned fb_next;       // batched iteration: next chunk of listed global queries; reset with fb_count
    // Work counters (added by the search kernels, read and cleared by the host).
    unsigned long long stat_queries;       // source points searched
    unsigned long long stat_fallbacks;     // of which took the global search
    unsigned long long stat_local_cand;    // target points examined by local searches
    unsigned long long stat_global_cand;   // target points examined by global searches
    // Registration loop state, reset together by the host before a run.
    int stop;               // 1 once converged or failed
    int iters;              // iterations applied
    double prev_rmse;
    double last_rmse;
};
static_assert(sizeof(DevCtl) == 112, "DevCtl layout");

// Rigid transform rounded to float: R row-major, t.
struct PoseF {
    float r[9];
    float t[3];
};

// The 3x4 upper part of a row-major 4x4 double pose, each entry rounded to
// the nearest float, loaded into shared memory by threads 0..11 (one entry
// each: the conversion runs on the FP64 pipe, so twelve lanes of one
// instruction rather than twelve instructions of one thread).  Contains
// __syncthreads(); every thread of the block must call it.
__device__ __forceinline__ void load_pose_f_block(const double *__restrict__ pose, PoseF &sp)
{
    if (threadIdx.x < 12) {
        const int a = threadIdx.x >> 2, b = threadIdx.x & 3;
        const float v = __double2float_rn(pose[4 * a + b]);
        if (b < 3)
            sp.r[3 * a + b] = v;
        else
            sp.t[a] = v;
    }
    __syncthreads();
}

// s_a = ((R_a0*x + R_a1*y) + R_a2*z) + t_a, every operation rounded to
// nearest on its own (no contraction into FMA).
__device__ __forceinline__ float3 transform_pt(const PoseF &P, float4 p)
{
    float s[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        float acc = __fmul_rn(P.r[3 * a + 0], p.x);
        acc = __fadd_rn(acc, __fmul_rn(P.r[3 * a + 1], p.y));
        acc = __fadd_rn(acc, __fmul_rn(P.r[3 * a + 2], p.z));
        s[a] = __fadd_rn(acc, P.t[a]);
    }
    return make_float3(s[0], s[1], s[2]);
}

// Quantize (Alg. 1/2/4): scaled coordinate s = (p - o) * inv_h per axis,
// each operation rounded once; the point is outside when a scaled coordinate
// is NaN, < 0 or >= dims.  Returns false outside.
__device__ __forceinline__ bool voxel_coords(const GridGeom &g, float x, float y, float z, int &ix, int &iy, int &iz)
{
    const float sx = __fmul_rn(__fsub_rn(x, g.ox), g.inv_h);
    const float sy = __fmul_rn(__fsub_rn(y, g.oy), g.inv_h);
    const float sz = __fmul_rn(__fsub_rn(z, g.oz), g.inv_h);
    if (!(sx >= 0.0f) || !(sy >= 0.0f) || !(sz >= 0.0f))
        return false;
    if (sx >= __int2float_rn(g.nx) || sy >= __int2float_rn(g.ny) || sz >= __int2float_rn(g.nz))
        return false;
    ix = (int)floorf(sx);
    iy = (int)floorf(sy);
    iz = (int)floorf(sz);
    return true;
}

// Concat: key = x + nx*(y + ny*z), or -1 outside the grid.
__device__ __forceinline__ int voxel_key(const GridGeom &g, float x, float y, float z)
{
    int ix, iy, iz;
    if (!voxel_coords(g, x, y, z, ix, iy, iz))
        return -1;
    return ix + g.nx * (iy + g.ny * iz);
}

// Linear index of brick (bx, by, bz): super-brick major (x fastest at both
// levels), so the bricks of one 4x4x4 super-brick are consecutive.
__host__ __device__ __forceinline__ int brick_index(const GridGeom &g, int bx, int by, int bz)
{
    const int sb = (bx / SUPER) + g.sx * ((by / SUPER) + g.sy * (bz / SUPER));
    return sb * SUPER_BRICKS + (bx % SUPER) + SUPER * ((by % SUPER) + SUPER * (bz % SUPER));
}

// Brick of a voxel (8x8x8 voxels per brick).
__device__ __forceinline__ int brick_key(const GridGeom &g, int ix, int iy, int iz)
{
    return brick_index(g, ix / BRICK, iy / BRICK, iz / BRICK);
}

// Length of the brick index space (padded to whole super-bricks).
__host__ __device__ __forceinline__ int brick_slots(const GridGeom &g) { return g.sx * g.sy * g.sz * SUPER_BRICKS; }

// ---------------------------------------------------------------------------
// Hashed voxel tables (the sparse grid): open addressing with linear
// probing over a power-of-two number of slots, keyed by voxel key (>= 0);
// an empty slot holds HASH_EMPTY.  The home slot is the top bits of the key
// times 2^32 / golden ratio (Fibonacci hashing), so that neighbouring voxel
// keys land far apart.
// ---------------------------------------------------------------------------
constexpr unsigned HASH_EMPTY = 0xffffffffu;
// Longest probe sequence: an insert that meets this many other keys gives up
// (the table is too full; the library keeps tables at most half full, where
// linear probing's runs stay far shorter), and a lookup never looks further.
constexpr unsigned HASH_MAX_PROBE = 256u;

struct HashTable {
    unsigned *keys;   // [mask + 1]
    unsigned mask;    // slots - 1
    int shift;        // 32 - log2(slots)
};

__host__ __device__ __forceinline__ unsigned hash_home(unsigned key, unsigned mask, int shift)
{
    return shift >= 32 ? 0u : ((key * 2654435769u) >> shift) & mask;
}

// Slot of `key`, inserted if absent; -1 after HASH_MAX_PROBE slots taken by
// other keys (the caller records DEVERR_CAPACITY).
__device__ __forceinline__ int hash_insert(const HashTable &h, unsigned key)
{
    unsigned s = hash_home(key, h.mask, h.shift);
    for (unsigned probe = 0; probe <= h.mask && probe < HASH_MAX_PROBE; ++probe, s = (s + 1u) & h.mask) {
        const unsigned k = atomicCAS(h.keys + s, HASH_EMPTY, key);
        if (k == HASH_EMPTY || k == key)
            return (int)s;
    }
    return -1;
}

// Slot of `key`, or -1 if it is absent (the probe stops at the first empty
// slot, or where an insert would have given up).
__device__ __forceinline__ int hash_find(const unsigned *__restrict__ keys, unsigned mask, int shift, unsigned key)
{
    unsigned s = hash_home(key, mask, shift);
    for (unsigned probe = 0; probe <= mask && probe < HASH_MAX_PROBE; ++probe, s = (s + 1u) & mask) {
        const unsigned k = __ldg(keys + s);
        if (k == key)
            return (int)s;
        if (k == HASH_EMPTY)
            return -1;
    }
    return -1;
}

// Floats mapped to unsigned integers whose order matches the float order, so
// atomicMin/atomicMax reduce them (and back).
__device__ __forceinline__ unsigned float_to_ordered(float f)
{
    const unsigned b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float ordered_to_float(unsigned o)
{
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}

// Squared distance ((dx*dx + dy*dy) + dz*dz), each operation rounded once.
__device__ __forceinline__ float dist2(float3 s, float4 q)
{
    const float dx = __fsub_rn(s.x, q.x);
    const float dy = __fsub_rn(s.y, q.y);
    const float dz = __fsub_rn(s.z, q.z);
    return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(dz, dz));
}

// Candidate key for the nearest-neighbour argmin: squared distance bits
// above the target index.  A distance is a sum of squares, so it is +0, a
// positive number, +inf or the canonical NaN 0x7fffffff; the unsigned order
// of the bits is then the order "numbers ascending, NaN last", and equal
// distances fall to the smaller index.
__device__ __forceinline__ unsigned long long nn_key(float d, int id)
{
    return ((unsigned long long)__float_as_uint(d) << 32) | (unsigned)id;
}

__device__ __forceinline__ unsigned long long umin64(unsigned long long a, unsigned long long b)
{
    return a < b ? a : b;
}

__device__ __forceinline__ unsigned long long warp_min_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = umin64(v, __shfl_xor_sync(FULL_MASK, v, o));
    return v;
}

__device__ __forceinline__ unsigned long long warp_sum_u64(unsigned long long v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// `width` (1..32) bits of a linear bitmask starting at bit `b`; needs one
// readable word past the last word touched.
__device__ __forceinline__ unsigned extract_bits(const unsigned *__restrict__ bits, long long b, int width)
{
    const long long w = b >> 5;
    const int sh = (int)(b & 31);
    const unsigned lo = __ldg(bits + w);
    const unsigned hi = (sh + width > 32) ? __ldg(bits + w + 1) : 0u;
    const unsigned v = __funnelshift_r(lo, hi, sh);
    return width >= 32 ? v : (v & ((1u << width) - 1u));
}

}  // namespace vicp
