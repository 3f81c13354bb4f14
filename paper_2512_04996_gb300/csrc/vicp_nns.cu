// vicp_nns.cu -- NNS (Alg. 4): localised search in the root voxel, and the
// global search for source points outside the grid or in unlabelled voxels.
#include "vicp_launch.h"

namespace vicp {

// ---------------------------------------------------------------------------
// Localised search: one thread per source point.  The point is transformed
// by the float-rounded pose, quantised, and its voxel's root label followed
// once (Alg. 4); the root voxel's CSR segment is scanned with 16-byte loads
// of (x, y, z, index).  Points that need the global search are compacted
// into a list with one warp-aggregated atomic per warp.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_correspond(const float4 *__restrict__ src, int m,
                                                    const double *__restrict__ pose, GridGeom g,
                                                    const int *__restrict__ root, const unsigned *__restrict__ off,
                                                    const float4 *__restrict__ csr, int n_cap,
                                                    int *__restrict__ nn, float *__restrict__ d2,
                                                    int *__restrict__ fb_list, DevCtl *__restrict__ ctl,
                                                    int honor_stop)
{
    if (honor_stop && *(volatile int *)&ctl->stop)
        return;
    __shared__ PoseF sp;
    if (threadIdx.x == 0)
        load_pose_f(pose, sp);
    __syncthreads();
    const PoseF P = sp;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool fall = false;
    unsigned cand = 0u;
    if (i < m) {
        const float3 s = transform_pt(P, __ldg(src + i));
        const int v = voxel_key(g, s.x, s.y, s.z);
        const int r = (v >= 0) ? __ldg(root + v) : -1;
        if (r >= 0) {
            const unsigned a = __ldg(off + r);
            const unsigned b = min(__ldg(off + r + 1), (unsigned)n_cap);
            cand = b > a ? b - a : 0u;
            unsigned long long best = ~0ull;
            unsigned k = a;
            for (; k + 4 <= b; k += 4) {   // four independent loads in flight
                const float4 q0 = __ldg(csr + k), q1 = __ldg(csr + k + 1);
                const float4 q2 = __ldg(csr + k + 2), q3 = __ldg(csr + k + 3);
                best = umin64(best, nn_key(dist2(s, q0), __float_as_int(q0.w)));
                best = umin64(best, nn_key(dist2(s, q1), __float_as_int(q1.w)));
                best = umin64(best, nn_key(dist2(s, q2), __float_as_int(q2.w)));
                best = umin64(best, nn_key(dist2(s, q3), __float_as_int(q3.w)));
            }
            for (; k < b; ++k) {
                const float4 q = __ldg(csr + k);
                best = umin64(best, nn_key(dist2(s, q), __float_as_int(q.w)));
            }
            nn[i] = (int)(unsigned)best;
            d2[i] = __uint_as_float((unsigned)(best >> 32));
        } else {
            fall = true;
        }
    }
    const unsigned long long wc = warp_sum_u64(cand);
    if ((threadIdx.x & 31) == 0 && wc)
        atomicAdd(&ctl->stat_local_cand, wc);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd(&ctl->stat_queries, (unsigned long long)m);
    const unsigned fm = __ballot_sync(FULL_MASK, fall);
    if (fm) {
        const int lane = threadIdx.x & 31, leader = __ffs(fm) - 1;
        int base = 0;
        if (lane == leader)
            base = atomicAdd(&ctl->fb_count, __popc(fm));
        base = __shfl_sync(FULL_MASK, base, leader);
        if (fall) {
            const int slot = base + __popc(fm & lanemask_lt());
            if (slot < m)
                fb_list[slot] = i;
            else
                atomicOr(&ctl->err, DEVERR_BOUNDS);
        }
    }
}

cudaError_t launch_correspond(const float4 *src, int m, const double *pose, const GridGeom &g, const int *root,
                              const unsigned *off, const float4 *csr, int n_cap, int *nn, float *d2,
                              int *fb_list, DevCtl *ctl, int honor_stop, cudaStream_t st)
{
    k_correspond<<<(m + 255) / 256, 256, 0, st>>>(src, m, pose, g, root, off, csr, n_cap, nn, d2, fb_list, ctl,
                                                  honor_stop);
    return cudaGetLastError();
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
constexpr int FB_THREADS = 256;
constexpr int FB_WARPS = FB_THREADS / 32;

__device__ __forceinline__ float box_lb2(float3 s, float4 lo, float4 hi)
{
    const float ex = s.x < lo.x ? __fsub_rn(lo.x, s.x) : (s.x > hi.x ? __fsub_rn(s.x, hi.x) : 0.0f);
    const float ey = s.y < lo.y ? __fsub_rn(lo.y, s.y) : (s.y > hi.y ? __fsub_rn(s.y, hi.y) : 0.0f);
    const float ez = s.z < lo.z ? __fsub_rn(lo.z, s.z) : (s.z > hi.z ? __fsub_rn(s.z, hi.z) : 0.0f);
    return __fadd_rn(__fadd_rn(__fmul_rn(ex, ex), __fmul_rn(ey, ey)), __fmul_rn(ez, ez));
}

__device__ __forceinline__ unsigned lb_bits(float3 s, const float4 *__restrict__ box, int k)
{
    return __float_as_uint(box_lb2(s, __ldg(box + 2 * k), __ldg(box + 2 * k + 1)));
}

// All lanes scan the run [r.x, r.y) of brick-ordered points; returns the
// warp-wide minimum key (every lane gets it).
__device__ __forceinline__ unsigned long long scan_run(const float4 *__restrict__ bpts, uint2 r, float3 s, int lane,
                                                       unsigned long long best, unsigned long long &examined)
{
    for (unsigned i = r.x + lane; i < r.y; i += 32) {
        const float4 q = __ldg(bpts + i);
        best = umin64(best, nn_key(dist2(s, q), __float_as_int(q.w)));
    }
    examined += r.y - r.x;
    return warp_min_u64(best);
}

__global__ void __launch_bounds__(FB_THREADS) k_fallback(const float4 *__restrict__ src,
                                                         const double *__restrict__ pose,
                                                         const float4 *__restrict__ bpts,
                                                         const uint2 *__restrict__ brange,
                                                         const float4 *__restrict__ bbox,
                                                         const uint2 *__restrict__ sb_range,
                                                         const float4 *__restrict__ sb_box,
                                                         const float4 *__restrict__ tgt, int n_tgt,
                                                         const int *__restrict__ outside,
                                                         const int *__restrict__ fb_list,
                                                         DevCtl *__restrict__ ctl, int *__restrict__ nn,
                                                         float *__restrict__ d2, int m, int honor_stop)
{
    if (honor_stop && *(volatile int *)&ctl->stop)
        return;   // the correspond kernel appended nothing either
    __shared__ PoseF sp;
    if (threadIdx.x == 0)
        load_pose_f(pose, sp);
    __syncthreads();
    const PoseF P = sp;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int F = min(*(volatile int *)&ctl->fb_count, m);
    const int ns = *(volatile int *)&ctl->n_super;
    const int no = *(volatile int *)&ctl->n_outside;
    unsigned long long examined = 0ull;   // every lane counts the same; lane 0 reports

    for (int qi = blockIdx.x * FB_WARPS + warp; qi < F; qi += gridDim.x * FB_WARPS) {
        const int i = __ldg(fb_list + qi);
        if ((unsigned)i >= (unsigned)m) {   // a stale entry: skip it, report it
            if (lane == 0)
                atomicOr(&ctl->err, DEVERR_BOUNDS);
            continue;
        }
        const float3 s = transform_pt(P, __ldg(src + i));
        unsigned long long best = ~0ull;
        if (!(isfinite(s.x) && isfinite(s.y) && isfinite(s.z))) {
            for (int j = lane; j < n_tgt; j += 32)
                best = umin64(best, nn_key(dist2(s, __ldg(tgt + j)), j));
            examined += (unsigned long long)n_tgt;
        } else {
            if (ns > 0) {
                // (1) nearest super-brick, nearest brick in it, scan it
                unsigned long long m0 = ~0ull;
                for (int k = lane; k < ns; k += 32)
                    m0 = umin64(m0, ((unsigned long long)lb_bits(s, sb_box, k) << 32) | (unsigned)k);
                m0 = warp_min_u64(m0);
                const uint2 r0 = __ldg(sb_range + (int)(unsigned)m0);
                unsigned long long m1 = ~0ull;
                for (int k = (int)r0.x + lane; k < (int)r0.y; k += 32)
                    m1 = umin64(m1, ((unsigned long long)lb_bits(s, bbox, k) << 32) | (unsigned)k);
                m1 = warp_min_u64(m1);
                const int k0 = (int)(unsigned)m1;
                best = scan_run(bpts, __ldg(brange + k0), s, lane, best, examined);
                // (2) every super-brick, and brick in it, that could hold a point at distance <= D
                for (int sb0 = 0; sb0 < ns; sb0 += 32) {
                    const int sbk = sb0 + lane;
                    const unsigned lbs = sbk < ns ? lb_bits(s, sb_box, sbk) : 0xffffffffu;
                    unsigned cs = __ballot_sync(FULL_MASK, lbs <= (unsigned)(best >> 32));
                    while (cs) {
                        const int sl = __ffs(cs) - 1;
                        cs &= cs - 1u;
                        if (__shfl_sync(FULL_MASK, lbs, sl) > (unsigned)(best >> 32))
                            continue;   // the bound was overtaken by a closer point
                        const uint2 r = __ldg(sb_range + sb0 + sl);
                        for (int kb = (int)r.x; kb < (int)r.y; kb += 32) {
                            const int k = kb + lane;
                            const unsigned lbb =
                                (k < (int)r.y && k != k0) ? lb_bits(s, bbox, k) : 0xffffffffu;
                            unsigned cb = __ballot_sync(FULL_MASK, lbb <= (unsigned)(best >> 32));
                            while (cb) {
                                const int bl = __ffs(cb) - 1;
                                cb &= cb - 1u;
                                if (__shfl_sync(FULL_MASK, lbb, bl) > (unsigned)(best >> 32))
                                    continue;
                                best = scan_run(bpts, __ldg(brange + kb + bl), s, lane, best, examined);
                            }
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
        }
        best = warp_min_u64(best);
        if (lane == 0) {
            nn[i] = (int)(unsigned)best;
            d2[i] = __uint_as_float((unsigned)(best >> 32));
        }
    }
    if (lane == 0 && examined)
        atomicAdd(&ctl->stat_global_cand, examined);
    // The last block to finish clears the fallback counter for the next search.
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const unsigned done = atomicAdd(&ctl->fb_done, 1u);
        if (done == gridDim.x - 1) {
            ctl->stat_fallbacks += (unsigned long long)F;
            ctl->fb_count = 0;
            ctl->fb_done = 0u;
        }
    }
}

cudaError_t launch_fallback(const float4 *src, const double *pose, const float4 *bpts, const uint2 *brange,
                            const float4 *bbox, const uint2 *sb_range, const float4 *sb_box, const float4 *tgt,
                            int n_tgt, const int *outside, const int *fb_list, DevCtl *ctl, int *nn, float *d2, int m,
                            int honor_stop, cudaStream_t st)
{
    k_fallback<<<152 * 4, FB_THREADS, 0, st>>>(src, pose, bpts, brange, bbox, sb_range, sb_box, tgt, n_tgt, outside,
                                               fb_list, ctl, nn, d2, m, honor_stop);
    return cudaGetLastError();
}

}  // namespace vicp
