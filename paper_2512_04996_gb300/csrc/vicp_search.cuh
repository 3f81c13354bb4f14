// vicp_search.cuh -- device code of the NNS (Alg. 4) shared by the
// single-grid kernels and the batched iteration kernel: the scan of a root
// voxel's CSR segment, and the exact global search over the brick levels.
#pragma once

#include "vicp_device.cuh"

namespace vicp {

// A root segment longer than this is scanned by a whole warp, not by the
// query's own thread (a warp waits for its longest segment).  On the 226k
// scene 48 leaves 9-18k of the 226k queries to whole warps (32: 27-38k)
// while the longest light segment of a warp grows by a sixth: measured step
// 107.5 -> 105.9 us.
constexpr unsigned HEAVY = 48;

// Nearest point of the CSR run [a, b) to s by one thread: 16-byte loads of
// (x, y, z, index), eight in flight.  Returns the (distance bits, index) key;
// ~0 for an empty run.
__device__ __forceinline__ unsigned long long segment_min(const float4 *__restrict__ csr, unsigned a, unsigned b,
                                                          float3 s)
{
    unsigned long long best = ~0ull;
    unsigned k = a;
    for (; k + 8 <= b; k += 8) {
        float4 q[8];
#pragma unroll
        for (int u = 0; u < 8; ++u)
            q[u] = __ldg(csr + k + u);
#pragma unroll
        for (int u = 0; u < 8; ++u)
            best = umin64(best, nn_key(dist2(s, q[u]), __float_as_int(q[u].w)));
    }
    for (; k < b; ++k) {
        const float4 q = __ldg(csr + k);
        best = umin64(best, nn_key(dist2(s, q), __float_as_int(q.w)));
    }
    return best;
}

// ---------------------------------------------------------------------------
// Global search ("Globalsearch" of Alg. 4): the exact nearest target point,
// found without scanning every point.
//
// The grid build groups the stored target points per non-empty 8x8x8 brick
// (contiguous runs of (x, y, z, index)) with each brick's exact float
// bounding box, and groups the bricks per 4x4x4-brick super-brick (a
// contiguous range of brick slots) with the union of their boxes.  For a
// query s, the box bound lb = ((ex*ex + ey*ey) + ez*ez), with e the rounded
// gap between s and the box on each axis, is never larger than the computed
// squared distance from s to any point in the box: rounding is monotone, so
// every operation of the bound is <= the same operation of the distance
// formula.  A warp per query
//   (1) takes the super-brick of smallest bound, and in it the brick of
//       smallest bound, and scans that brick's points (lanes split the run),
//       which gives a first best distance D;
//   (2) visits every super-brick whose bound is <= D, and in it scans each
//       brick whose bound is still <= D, tightening D as it goes;
//   (3) scans the target points that lie outside the grid.
// The result is the same (distance, index) minimum as a scan of all target
// points.  A query with a non-finite coordinate scans all target points.
// ---------------------------------------------------------------------------

// The gap on an axis is max(lo - s, s - hi, 0): at most one difference is
// positive, and rounding keeps each difference's sign.
__device__ __forceinline__ float box_lb2(float3 s, float4 lo, float4 hi)
{
    const float ex = fmaxf(fmaxf(__fsub_rn(lo.x, s.x), __fsub_rn(s.x, hi.x)), 0.0f);
    const float ey = fmaxf(fmaxf(__fsub_rn(lo.y, s.y), __fsub_rn(s.y, hi.y)), 0.0f);
    const float ez = fmaxf(fmaxf(__fsub_rn(lo.z, s.z), __fsub_rn(s.z, hi.z)), 0.0f);
    return __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
}

// Record index of the smallest bound over the warp (lane values lb, k; any
// lane holding the minimum may win: the choice only orders the search).
__device__ __forceinline__ int warp_argmin(unsigned lb, int k)
{
    const unsigned mn = __reduce_min_sync(FULL_MASK, lb);
    return __shfl_sync(FULL_MASK, k, __ffs(__ballot_sync(FULL_MASK, lb == mn)) - 1);
}

// Warp minimum of (distance bits, index) keys: the smallest distance, then
// the smallest index at it -- two single-instruction warp reductions.
__device__ __forceinline__ unsigned long long warp_min_key(unsigned long long v)
{
    const unsigned d = __reduce_min_sync(FULL_MASK, (unsigned)(v >> 32));
    const unsigned i = __reduce_min_sync(FULL_MASK, (unsigned)(v >> 32) == d ? (unsigned)v : 0xffffffffu);
    return ((unsigned long long)d << 32) | i;
}

// Bound of box record k (as order-preserving bits), and its index range
// [a, b) (the boxes carry their ranges in the w fields).
__device__ __forceinline__ unsigned box_bound(const float4 *__restrict__ box, int k, float3 s)
{
    return __float_as_uint(box_lb2(s, __ldg(box + 2 * k), __ldg(box + 2 * k + 1)));
}

__device__ __forceinline__ uint2 box_range(const float4 *__restrict__ box, int k)
{
    return make_uint2(__float_as_uint(__ldg(box + 2 * k).w), __float_as_uint(__ldg(box + 2 * k + 1).w));
}

// Bound and index range of box record k.
__device__ __forceinline__ void load_rec(const float4 *__restrict__ box, int k, float3 s, unsigned &lb, unsigned &a,
                                         unsigned &b)
{
    const float4 lo = __ldg(box + 2 * k), hi = __ldg(box + 2 * k + 1);
    lb = __float_as_uint(box_lb2(s, lo, hi));
    a = __float_as_uint(lo.w);
    b = __float_as_uint(hi.w);
}

// All lanes scan the run [a, b) of brick-ordered points (four loads in
// flight per lane); returns the warp-wide minimum key (every lane gets it).
__device__ __forceinline__ unsigned long long scan_run(const float4 *__restrict__ bpts, unsigned a, unsigned b,
                                                       float3 s, int lane, unsigned long long best,
                                                       unsigned long long &examined)
{
    unsigned i = a + lane;
    for (; i + 96 < b; i += 128) {
        const float4 q0 = __ldg(bpts + i), q1 = __ldg(bpts + i + 32);
        const float4 q2 = __ldg(bpts + i + 64), q3 = __ldg(bpts + i + 96);
        best = umin64(best, nn_key(dist2(s, q0), __float_as_int(q0.w)));
        best = umin64(best, nn_key(dist2(s, q1), __float_as_int(q1.w)));
        best = umin64(best, nn_key(dist2(s, q2), __float_as_int(q2.w)));
        best = umin64(best, nn_key(dist2(s, q3), __float_as_int(q3.w)));
    }
    for (; i < b; i += 32) {
        const float4 q = __ldg(bpts + i);
        best = umin64(best, nn_key(dist2(s, q), __float_as_int(q.w)));
    }
    examined += b - a;
    return warp_min_key(best);
}

// Scan, in ascending lane order, the bricks of one 32-record chunk whose bound
// (lb, per lane) is <= the current best distance; (ra, rb) are the bricks'
// point ranges.
__device__ __forceinline__ unsigned long long scan_chunk(const float4 *__restrict__ bpts, unsigned lb, unsigned ra,
                                                         unsigned rb, float3 s, int lane, unsigned long long best,
                                                         unsigned long long &examined)
{
    unsigned c = __ballot_sync(FULL_MASK, lb <= (unsigned)(best >> 32));
    while (c) {
        const int l = __ffs(c) - 1;
        c &= c - 1u;
        if (__shfl_sync(FULL_MASK, lb, l) > (unsigned)(best >> 32))
            continue;   // the bound was overtaken by a closer point
        const unsigned a = __shfl_sync(FULL_MASK, ra, l), b = __shfl_sync(FULL_MASK, rb, l);
        best = scan_run(bpts, a, b, s, lane, best, examined);
    }
    return best;
}

constexpr int SB_CACHED = 4;   // super-brick records kept in registers: 32 per chunk

// The global search of one query s by the whole warp (every lane calls it
// with the same s; every lane gets the result key).  One grid's levels:
// brick records bbox (their w fields: point ranges in bpts), `ns`
// super-brick records sb_box (w fields: brick-record ranges), and the `no`
// target points outside the grid (indices into tgt); tgt holds all n_tgt
// target points.  `examined` counts the candidates (the same on every lane).
__device__ __forceinline__ unsigned long long global_search(float3 s, const float4 *__restrict__ bpts,
                                                            const float4 *__restrict__ bbox,
                                                            const float4 *__restrict__ sb_box, int ns,
                                                            const float4 *__restrict__ tgt, int n_tgt,
                                                            const int *__restrict__ outside, int no, int lane,
                                                            unsigned long long &examined)
{
    unsigned long long best = ~0ull;
    if (!(isfinite(s.x) && isfinite(s.y) && isfinite(s.z))) {
        for (int j = lane; j < n_tgt; j += 32)
            best = umin64(best, nn_key(dist2(s, __ldg(tgt + j)), j));
        examined += (unsigned long long)n_tgt;
        return warp_min_key(best);
    }
    if (ns > 0) {
        // (1) super-brick bounds (the first SB_CACHED chunks kept in
        //     registers; ranges are fetched from L1 when a record is
        //     picked), the nearest super-brick S0 ...
        unsigned sl[SB_CACHED];
        unsigned lmin = 0xffffffffu;
        int kmin = lane;
#pragma unroll
        for (int t = 0; t < SB_CACHED; ++t) {
            const int k = 32 * t + lane;
            sl[t] = 0xffffffffu;
            if (k < ns)
                sl[t] = box_bound(sb_box, k, s);
            if (sl[t] < lmin) {
                lmin = sl[t];
                kmin = k;
            }
        }
        for (int k = 32 * SB_CACHED + lane; k < ns; k += 32) {
            const unsigned lb = box_bound(sb_box, k, s);
            if (lb < lmin) {
                lmin = lb;
                kmin = k;
            }
        }
        const int s0 = min(warp_argmin(lmin, kmin), ns - 1);
        uint2 r0 = box_range(sb_box, s0);
        // ... its bricks' bounds (at most 64: two chunks, kept), and the
        //     nearest brick K0 in it, scanned first for a first distance
        unsigned bl[2];
        unsigned bmin = 0xffffffffu;
        int bk = lane;
#pragma unroll
        for (int t = 0; t < 2; ++t) {
            const int k = 32 * t + lane;   // relative to the super-brick's first brick
            bl[t] = (int)r0.x + k < (int)r0.y ? box_bound(bbox, (int)r0.x + k, s) : 0xffffffffu;
            if (bl[t] < bmin) {
                bmin = bl[t];
                bk = k;
            }
        }
        int k0 = min(warp_argmin(bmin, bk), (int)(r0.y - r0.x) - 1);
        {
            const uint2 pr = box_range(bbox, (int)r0.x + k0);
            best = scan_run(bpts, pr.x, pr.y, s, lane, best, examined);
        }
        // (2) best first: the unvisited super-brick of smallest bound
        //     while that bound is <= D, and in it the unvisited brick
        //     of smallest bound while that bound is <= D
#pragma unroll
        for (int t = 0; t < SB_CACHED; ++t)
            if (32 * t + lane == s0)
                sl[t] = 0xffffffffu;
        if ((k0 & 31) == lane) {   // K0 is done
            if (k0 < 32)
                bl[0] = 0xffffffffu;
            else
                bl[1] = 0xffffffffu;
        }
        for (;;) {
            // bricks of the current super-brick (first r0.x), nearest first
            for (;;) {
                const bool first = bl[0] <= bl[1];
                const unsigned v = first ? bl[0] : bl[1];
                const unsigned mn = __reduce_min_sync(FULL_MASK, v);
                if (mn > (unsigned)(best >> 32))
                    break;
                const int w = __ffs(__ballot_sync(FULL_MASK, v == mn)) - 1;
                const int rel = __shfl_sync(FULL_MASK, first ? lane : 32 + lane, w);
                if (lane == w) {
                    if (first)
                        bl[0] = 0xffffffffu;
                    else
                        bl[1] = 0xffffffffu;
                }
                const uint2 pr = box_range(bbox, (int)r0.x + rel);
                best = scan_run(bpts, pr.x, pr.y, s, lane, best, examined);
            }
            // the next super-brick
            unsigned v = 0xffffffffu;
            int vk = lane;
#pragma unroll
            for (int t = 0; t < SB_CACHED; ++t)
                if (sl[t] < v) {
                    v = sl[t];
                    vk = 32 * t + lane;
                }
            const unsigned mn = __reduce_min_sync(FULL_MASK, v);
            if (mn > (unsigned)(best >> 32))
                break;
            const int w = __ffs(__ballot_sync(FULL_MASK, v == mn)) - 1;
            const int sk = __shfl_sync(FULL_MASK, vk, w);
#pragma unroll
            for (int t = 0; t < SB_CACHED; ++t)
                if (lane == w && 32 * t + lane == sk)
                    sl[t] = 0xffffffffu;
            r0 = box_range(sb_box, sk);
#pragma unroll
            for (int t = 0; t < 2; ++t) {   // at most 64 bricks in a super-brick
                const int k = (int)r0.x + 32 * t + lane;
                bl[t] = k < (int)r0.y ? box_bound(bbox, k, s) : 0xffffffffu;
            }
        }
        // super-bricks past the cached chunks, in index order
        for (int c0 = 32 * SB_CACHED; c0 < ns; c0 += 32) {
            unsigned lbs = 0xffffffffu, ra = 0u, rb = 0u;
            if (c0 + lane < ns)
                load_rec(sb_box, c0 + lane, s, lbs, ra, rb);
            unsigned cs = __ballot_sync(FULL_MASK, lbs <= (unsigned)(best >> 32));
            while (cs) {
                const int l = __ffs(cs) - 1;
                cs &= cs - 1u;
                if (__shfl_sync(FULL_MASK, lbs, l) > (unsigned)(best >> 32))
                    continue;   // the bound was overtaken by a closer point
                const unsigned xa = __shfl_sync(FULL_MASK, ra, l), xb = __shfl_sync(FULL_MASK, rb, l);
                for (int kb = (int)xa; kb < (int)xb; kb += 32) {
                    const int k = kb + lane;
                    unsigned lbb = 0xffffffffu, pa = 0u, pb = 0u;
                    if (k < (int)xb)
                        load_rec(bbox, k, s, lbb, pa, pb);
                    best = scan_chunk(bpts, lbb, pa, pb, s, lane, best, examined);
                }
            }
        }
    }
    // (3) target points outside the grid
    for (int k = lane; k < no; k += 32) {
        const int j = __ldg(outside + k);
        best = umin64(best, nn_key(dist2(s, __ldg(tgt + j)), j));
    }
    examined += (unsigned long long)no;
    return warp_min_key(best);
}

}  // namespace vicp
