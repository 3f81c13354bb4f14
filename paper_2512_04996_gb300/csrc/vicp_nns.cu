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
    pdl_begin();
    if (honor_stop && *(volatile int *)&ctl->stop)
        return;
    __shared__ PoseF sp;
    __shared__ unsigned long long s_cand;   // block totals: one global atomic each
    __shared__ int s_fb, s_fb_base;
    if (threadIdx.x == 0) {
        s_cand = 0ull;
        s_fb = 0;
    }
    load_pose_f_block(pose, sp);   // also orders the initialisation above
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
    // The block's fallback queries and work counts are gathered in shared
    // memory first: same-address global atomics from every warp would
    // serialise in one L2 slice.
    const int lane = threadIdx.x & 31;
    const unsigned fm = __ballot_sync(FULL_MASK, fall);
    const unsigned long long wc = warp_sum_u64(cand);
    int wbase = 0;
    if (lane == 0) {
        if (wc)
            atomicAdd(&s_cand, wc);
        if (fm)
            wbase = atomicAdd(&s_fb, __popc(fm));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_cand)
            atomicAdd(&ctl->stat_local_cand, s_cand);
        if (blockIdx.x == 0)
            atomicAdd(&ctl->stat_queries, (unsigned long long)m);
        if (s_fb)
            s_fb_base = atomicAdd(&ctl->fb_count, s_fb);
    }
    __syncthreads();
    wbase = __shfl_sync(FULL_MASK, wbase, 0);
    if (fall) {
        const int slot = s_fb_base + wbase + __popc(fm & lanemask_lt());
        if (slot < m)
            fb_list[slot] = i;
        else
            atomicOr(&ctl->err, DEVERR_BOUNDS);
    }
}

cudaError_t launch_correspond(const float4 *src, int m, const double *pose, const GridGeom &g, const int *root,
                              const unsigned *off, const float4 *csr, int n_cap, int *nn, float *d2,
                              int *fb_list, DevCtl *ctl, int honor_stop, cudaStream_t st)
{
    return launch_kernel(k_correspond, dim3((m + 255) / 256), dim3(256), 0, st, src, m, pose, g, root, off, csr, n_cap,
                         nn, d2, fb_list, ctl, honor_stop);
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

// Bound (as order-preserving bits) and index range [a, b) of box record k:
// the boxes carry their ranges in the w fields.
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
    return warp_min_u64(best);
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

__global__ void __launch_bounds__(FB_THREADS, 4) k_fallback(const float4 *__restrict__ src,
                                                         const double *__restrict__ pose,
                                                         const float4 *__restrict__ bpts,
                                                         const float4 *__restrict__ bbox,
                                                         const float4 *__restrict__ sb_box,
                                                         const float4 *__restrict__ tgt, int n_tgt,
                                                         const int *__restrict__ outside,
                                                         const int *__restrict__ fb_list,
                                                         DevCtl *__restrict__ ctl, int *__restrict__ nn,
                                                         float *__restrict__ d2, int m, int honor_stop)
{
    pdl_begin();
    if (honor_stop && *(volatile int *)&ctl->stop)
        return;   // the correspond kernel appended nothing either
    __shared__ PoseF sp;
    __shared__ unsigned long long s_examined;   // block total: one global atomic
    if (threadIdx.x == 0)
        s_examined = 0ull;
    load_pose_f_block(pose, sp);   // also orders the initialisation above
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
                // (1) super-brick records (the first SB_CACHED chunks kept in
                //     registers), the nearest super-brick S0 ...
                unsigned sl[SB_CACHED], sa[SB_CACHED], sb[SB_CACHED];
                unsigned long long m0 = ~0ull;
#pragma unroll
                for (int t = 0; t < SB_CACHED; ++t) {
                    const int k = 32 * t + lane;
                    sl[t] = 0xffffffffu;
                    sa[t] = sb[t] = 0u;
                    if (k < ns)
                        load_rec(sb_box, k, s, sl[t], sa[t], sb[t]);
                    m0 = umin64(m0, ((unsigned long long)sl[t] << 32) | (unsigned)k);
                }
                for (int k = 32 * SB_CACHED + lane; k < ns; k += 32) {
                    unsigned lb, a, b;
                    load_rec(sb_box, k, s, lb, a, b);
                    m0 = umin64(m0, ((unsigned long long)lb << 32) | (unsigned)k);
                }
                m0 = warp_min_u64(m0);
                const int s0 = (int)(unsigned)m0;
                unsigned r0a, r0b;
                if (s0 < 32 * SB_CACHED) {
                    unsigned a = 0u, b = 0u;
#pragma unroll
                    for (int t = 0; t < SB_CACHED; ++t)
                        if (t == (s0 >> 5)) {
                            a = sa[t];
                            b = sb[t];
                        }
                    r0a = __shfl_sync(FULL_MASK, a, s0 & 31);
                    r0b = __shfl_sync(FULL_MASK, b, s0 & 31);
                } else {
                    r0a = __float_as_uint(__ldg(sb_box + 2 * s0).w);
                    r0b = __float_as_uint(__ldg(sb_box + 2 * s0 + 1).w);
                }
                // ... its brick records (at most 64: two chunks, kept), and the
                //     nearest brick K0 in it, scanned first for a first distance
                unsigned bl[2], ba[2], bb[2];
                unsigned long long m1 = ~0ull;
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const int k = (int)r0a + 32 * t + lane;
                    bl[t] = 0xffffffffu;
                    ba[t] = bb[t] = 0u;
                    if (k < (int)r0b)
                        load_rec(bbox, k, s, bl[t], ba[t], bb[t]);
                    m1 = umin64(m1, ((unsigned long long)bl[t] << 32) | (unsigned)k);
                }
                m1 = warp_min_u64(m1);
                const int k0 = (int)(unsigned)m1 - (int)r0a;   // chunk-relative
                {
                    const unsigned a = k0 < 32 ? ba[0] : ba[1], b = k0 < 32 ? bb[0] : bb[1];
                    best = scan_run(bpts, __shfl_sync(FULL_MASK, a, k0 & 31), __shfl_sync(FULL_MASK, b, k0 & 31), s,
                                    lane, best, examined);
                }
                // (2) every super-brick, and brick in it, that could hold a point
                //     at distance <= D
                for (int c0 = 0; c0 < ns; c0 += 32) {
                    const int t = c0 >> 5;
                    unsigned lbs = 0xffffffffu, ra = 0u, rb = 0u;
#pragma unroll
                    for (int c = 0; c < SB_CACHED; ++c)
                        if (t == c) {
                            lbs = sl[c];
                            ra = sa[c];
                            rb = sb[c];
                        }
                    if (t >= SB_CACHED && c0 + lane < ns)
                        load_rec(sb_box, c0 + lane, s, lbs, ra, rb);
                    unsigned cs = __ballot_sync(FULL_MASK, lbs <= (unsigned)(best >> 32));
                    while (cs) {
                        const int l = __ffs(cs) - 1;
                        cs &= cs - 1u;
                        if (__shfl_sync(FULL_MASK, lbs, l) > (unsigned)(best >> 32))
                            continue;   // the bound was overtaken by a closer point
                        if (c0 + l == s0) {   // S0: its records are in registers; K0 is done
#pragma unroll
                            for (int u = 0; u < 2; ++u) {
                                const bool k0_here = (k0 >> 5) == u && (k0 & 31) == lane;
                                best = scan_chunk(bpts, k0_here ? 0xffffffffu : bl[u], ba[u], bb[u], s, lane, best,
                                                  examined);
                            }
                            continue;
                        }
                        const unsigned a = __shfl_sync(FULL_MASK, ra, l), b = __shfl_sync(FULL_MASK, rb, l);
                        for (int kb = (int)a; kb < (int)b; kb += 32) {
                            const int k = kb + lane;
                            unsigned lbb = 0xffffffffu, pa = 0u, pb = 0u;
                            if (k < (int)b)
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
        }
        best = warp_min_u64(best);
        if (lane == 0) {
            nn[i] = (int)(unsigned)best;
            d2[i] = __uint_as_float((unsigned)(best >> 32));
        }
    }
    // work counter: one global atomic per block; the last block to finish
    // clears the fallback counter for the next search
    if (lane == 0 && examined)
        atomicAdd(&s_examined, examined);
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_examined)
            atomicAdd(&ctl->stat_global_cand, s_examined);
        __threadfence();
        const unsigned done = atomicAdd(&ctl->fb_done, 1u);
        if (done == gridDim.x - 1) {
            ctl->stat_fallbacks += (unsigned long long)F;
            ctl->fb_count = 0;
            ctl->fb_done = 0u;
        }
    }
}

cudaError_t launch_fallback(const float4 *src, const double *pose, const float4 *bpts, const float4 *bbox,
                            const float4 *sb_box, const float4 *tgt, int n_tgt, const int *outside, const int *fb_list,
                            DevCtl *ctl, int *nn, float *d2, int m, int honor_stop, cudaStream_t st)
{
    // as many warps as can be resident: a query per warp at most times
    static int per_sm = 0;
    if (per_sm == 0) {
        cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_fallback, FB_THREADS, 0);
        if (e != cudaSuccess || per_sm < 1)
            per_sm = 1;
    }
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return launch_kernel(k_fallback, dim3(sms * per_sm), dim3(FB_THREADS), 0, st, src, pose, bpts, bbox, sb_box, tgt,
                         n_tgt, outside, fb_list, ctl, nn, d2, m, honor_stop);
}

}  // namespace vicp
