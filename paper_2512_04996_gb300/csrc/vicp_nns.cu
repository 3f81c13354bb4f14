// vicp_nns.cu -- NNS (Alg. 4): localised search in the root voxel, and the
// global search for source points outside the grid or in unlabelled voxels.
#include "vicp_launch.h"
#include "vicp_search.cuh"

namespace vicp {

// ---------------------------------------------------------------------------
// Localised search: one thread per source point.  The point is transformed
// by the float-rounded pose, quantised, and its voxel's root label followed
// once (Alg. 4); the root voxel's CSR segment is scanned with 16-byte loads
// of (x, y, z, index), eight in flight.  A few dense voxels hold far more
// points than the rest, and a warp waits for its longest segment: a query
// whose segment has more than HEAVY points is not scanned here but listed,
// with its segment, for the next kernel, whose warps take such segments one
// at a time with all lanes.  Points that need the global search are listed
// for it.  Both lists get one global atomic per block.
// ---------------------------------------------------------------------------
constexpr int CORR_THREADS = 512;

// Segment of a root voxel in the CSR store: [off[r], off[r + 1]) (clamped to
// the store's length).
struct CsrSeg {
    const unsigned *off;
    unsigned cap;
    __device__ __forceinline__ void range(int r, unsigned &a, unsigned &b) const
    {
        a = __ldg(off + r);
        b = max(a, min(__ldg(off + r + 1), cap));
    }
};

// Segment of a root voxel in a fixed-capacity store: the first
// min(count[r], C) of the C slots that start at r * C.
struct FixedSeg {
    const unsigned *count;
    unsigned C;
    __device__ __forceinline__ void range(int r, unsigned &a, unsigned &b) const
    {
        a = (unsigned)r * C;
        b = a + min(__ldg(count + r), C);
    }
};

// Root label of voxel v, as the index of its segment in the store: the
// dense root array (the root's voxel key), or the sparse grid's two tables
// (the labelled-segment table gives v's row segment -- its label mask and
// the index of its first root -- and so the root's voxel key, at v's rank
// among the segment's labelled voxels; the occupied-voxel table gives that
// voxel's slot, which indexes the offsets).  -1: unlabelled.
struct DenseRoot {
    const int *root;
    __device__ __forceinline__ int operator()(int v) const { return __ldg(root + v); }
};

struct HashedRoot {
    const unsigned *lkeys;   // labelled row segments
    unsigned lmask;
    int lshift;
    const uint2 *lseg;       // their label masks and first-root indices
    const int *lroot;        // the labelled voxels' root keys, segment by segment
    const unsigned *okeys;   // occupied voxels
    unsigned omask;
    int oshift;
    int nx, nxb;             // grid row length, 32-voxel segments per row
    __device__ __forceinline__ int operator()(int v) const
    {
        const int x = v % nx, row = v / nx;   // row = y + ny z
        const int ls = hash_find(lkeys, lmask, lshift, (unsigned)((x >> 5) + nxb * row));
        if (ls < 0)
            return -1;
        const uint2 e = __ldg(lseg + ls);
        const unsigned bit = (unsigned)x & 31u;
        if (!((e.x >> bit) & 1u))
            return -1;
        const int r = __ldg(lroot + e.y + __popc(e.x & ((1u << bit) - 1u)));
        return hash_find(okeys, omask, oshift, (unsigned)r);
    }
};

template <class Seg, class Root>
__global__ void __launch_bounds__(CORR_THREADS) k_correspond(const float4 *__restrict__ src, int m,
                                                             const double *__restrict__ pose, GridGeom g,
                                                             Root root, Seg seg,
                                                             const float4 *__restrict__ csr,
                                                             int *__restrict__ nn, float *__restrict__ d2,
                                                             int *__restrict__ fb_list, int *__restrict__ hv_list,
                                                             uint2 *__restrict__ hv_range, DevCtl *__restrict__ ctl,
                                                             int honor_stop)
{
    pdl_begin();
    if (honor_stop && *(volatile int *)&ctl->stop)
        return;
    __shared__ PoseF sp;
    __shared__ unsigned long long s_cand;   // block totals: one global atomic each
    __shared__ int s_fb, s_fb_base, s_hv, s_hv_base;
    if (threadIdx.x == 0) {
        s_cand = 0ull;
        s_fb = s_hv = 0;
    }
    load_pose_f_block(pose, sp);   // also orders the initialisation above
    const PoseF P = sp;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool fall = false, heavy = false;
    unsigned cand = 0u, a = 0u, b = 0u;
    if (i < m) {
        const float3 s = transform_pt(P, __ldg(src + i));
        const int v = voxel_key(g, s.x, s.y, s.z);
        const int r = (v >= 0) ? root(v) : -1;
        if (r >= 0) {
            seg.range(r, a, b);
            cand = b - a;
            heavy = cand > HEAVY;
            if (!heavy) {
                const unsigned long long best = segment_min(csr, a, b, s);
                nn[i] = (int)(unsigned)best;
                d2[i] = __uint_as_float((unsigned)(best >> 32));
            }
        } else {
            fall = true;
        }
    }
    const unsigned fm = __ballot_sync(FULL_MASK, fall), hm = __ballot_sync(FULL_MASK, heavy);
    const unsigned long long wc = warp_sum_u64(cand);
    int fb_base = 0, hv_base = 0;
    if (lane == 0) {
        if (wc)
            atomicAdd(&s_cand, wc);
        if (fm)
            fb_base = atomicAdd(&s_fb, __popc(fm));
        if (hm)
            hv_base = atomicAdd(&s_hv, __popc(hm));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        if (s_cand)
            atomicAdd(&ctl->stat_local_cand, s_cand);
        if (blockIdx.x == 0)
            atomicAdd(&ctl->stat_queries, (unsigned long long)m);
        if (s_fb)
            s_fb_base = atomicAdd(&ctl->fb_count, s_fb);
        if (s_hv)
            s_hv_base = atomicAdd(&ctl->hv_count, s_hv);
    }
    __syncthreads();
    fb_base = __shfl_sync(FULL_MASK, fb_base, 0);
    hv_base = __shfl_sync(FULL_MASK, hv_base, 0);
    if (fall) {
        const int slot = s_fb_base + fb_base + __popc(fm & lanemask_lt());
        if (slot < m)
            fb_list[slot] = i;
        else
            atomicOr(&ctl->err, DEVERR_BOUNDS);
    }
    if (heavy) {
        const int slot = s_hv_base + hv_base + __popc(hm & lanemask_lt());
        if (slot < m) {
            hv_list[slot] = i;
            hv_range[slot] = make_uint2(a, b);
        } else {
            atomicOr(&ctl->err, DEVERR_BOUNDS);
        }
    }
}

cudaError_t launch_correspond(const float4 *src, int m, const double *pose, const GridGeom &g, const int *root,
                              const unsigned *off, const float4 *csr, int n_cap, int *nn, float *d2,
                              int *fb_list, int *hv_list, uint2 *hv_range, DevCtl *ctl, int honor_stop,
                              cudaStream_t st)
{
    return launch_kernel(k_correspond<CsrSeg, DenseRoot>, dim3((m + CORR_THREADS - 1) / CORR_THREADS),
                         dim3(CORR_THREADS), 0, st, src, m, pose, g, DenseRoot{root}, CsrSeg{off, (unsigned)n_cap},
                         csr, nn, d2, fb_list, hv_list, hv_range, ctl, honor_stop);
}

cudaError_t launch_correspond_hashed(const float4 *src, int m, const double *pose, const GridGeom &g,
                                     const HashTable &labelled, const uint2 *lseg, const int *lroot,
                                     const HashTable &occupied, const unsigned *off, const float4 *csr, int n_cap,
                                     int *nn, float *d2, int *fb_list, int *hv_list, uint2 *hv_range, DevCtl *ctl,
                                     int honor_stop, cudaStream_t st)
{
    const HashedRoot root{labelled.keys, labelled.mask, labelled.shift, lseg, lroot,
                          occupied.keys, occupied.mask, occupied.shift, g.nx, (g.nx + 31) / 32};
    return launch_kernel(k_correspond<CsrSeg, HashedRoot>, dim3((m + CORR_THREADS - 1) / CORR_THREADS),
                         dim3(CORR_THREADS), 0, st, src, m, pose, g, root, CsrSeg{off, (unsigned)n_cap}, csr, nn, d2,
                         fb_list, hv_list, hv_range, ctl, honor_stop);
}

cudaError_t launch_correspond_fixed(const float4 *src, int m, const double *pose, const GridGeom &g, const int *root,
                                    const unsigned *count, unsigned C, const float4 *slots, int *nn, float *d2,
                                    int *fb_list, int *hv_list, uint2 *hv_range, DevCtl *ctl, cudaStream_t st)
{
    return launch_kernel(k_correspond<FixedSeg, DenseRoot>, dim3((m + CORR_THREADS - 1) / CORR_THREADS),
                         dim3(CORR_THREADS), 0, st, src, m, pose, g, DenseRoot{root}, FixedSeg{count, C}, slots, nn,
                         d2, fb_list, hv_list, hv_range, ctl, 0);
}

// ---------------------------------------------------------------------------
// Global search ("Globalsearch" of Alg. 4) of the queries the localised
// search listed (global_search: a warp per query over the brick levels), and
// the dense root segments it left (all lanes of a warp scan one).
//
// Scheduling without global atomics: block b takes the list entries b,
// b + B, b + 2B, ... of both lists (B blocks; strided, so that a block's
// share mixes the regions of the source cloud and the shares cost about the
// same), global queries first and dense segments after them, and its warps
// take these items one at a time from a shared-memory counter.  Per-query
// costs vary several-fold, so the warps of a block balance each other; the
// shares balance the blocks.  (A single global ticket counter would put one
// same-address atomic per item, plus one per warp at the end, into the L2
// line that also holds the list lengths every block reads: on the 226k
// scene those ~17k serialised operations, not the searches, set the
// kernel's duration.)
// ---------------------------------------------------------------------------
constexpr int FB_THREADS = 256;
constexpr int FB_WARPS = FB_THREADS / 32;

// Entries b, b + B, ... below n: how many.
__device__ __forceinline__ int strided_share(int n, int b, int B) { return n > b ? (n - 1 - b) / B + 1 : 0; }

__global__ void __launch_bounds__(FB_THREADS, 4) k_fallback(const float4 *__restrict__ src,
                                                         const double *__restrict__ pose,
                                                         const float4 *__restrict__ bpts,
                                                         const float4 *__restrict__ bbox,
                                                         const float4 *__restrict__ sb_box,
                                                         const float4 *__restrict__ tgt, int n_tgt,
                                                         const int *__restrict__ outside,
                                                         const int *__restrict__ fb_list,
                                                         const int *__restrict__ hv_list,
                                                         const uint2 *__restrict__ hv_range,
                                                         const float4 *__restrict__ csr,
                                                         DevCtl *__restrict__ ctl, int *__restrict__ nn,
                                                         float *__restrict__ d2, int m, int honor_stop)
{
    pdl_begin();
    if (honor_stop && *(volatile int *)&ctl->stop)
        return;   // the correspond kernel appended nothing either
    __shared__ PoseF sp;
    __shared__ unsigned long long s_examined;   // block total: one global atomic
    __shared__ int s_F, s_Hv, s_ns, s_no;
    __shared__ unsigned s_next;                 // next item of this block's share
    if (threadIdx.x == 0) {
        s_examined = 0ull;
        s_F = min(*(volatile int *)&ctl->fb_count, m);
        s_Hv = min(*(volatile int *)&ctl->hv_count, m);
        s_ns = *(volatile int *)&ctl->n_super;
        s_no = *(volatile int *)&ctl->n_outside;
        s_next = 0u;
    }
    load_pose_f_block(pose, sp);   // also orders the initialisation above
    const PoseF P = sp;
    const int lane = threadIdx.x & 31;
    const int F = s_F, Hv = s_Hv, ns = s_ns, no = s_no;
    const int B = (int)gridDim.x, b = (int)blockIdx.x;
    const int nG = strided_share(F, b, B), nH = strided_share(Hv, b, B);
    unsigned long long examined = 0ull;   // every lane counts the same; lane 0 reports

    for (;;) {
        int k = 0;
        if (lane == 0)
            k = (int)atomicAdd(&s_next, 1u);
        k = __shfl_sync(FULL_MASK, k, 0);
        if (k >= nG + nH)
            break;
        if (k < nG) {   // a global query
            const int i = __ldg(fb_list + b + k * B);
            if ((unsigned)i >= (unsigned)m) {   // a stale entry: skip it, report it
                if (lane == 0)
                    atomicOr(&ctl->err, DEVERR_BOUNDS);
                continue;
            }
            const float3 s = transform_pt(P, __ldg(src + i));
            const unsigned long long best =
                global_search(s, bpts, bbox, sb_box, ns, tgt, n_tgt, outside, no, lane, examined);
            if (lane == 0) {
                nn[i] = (int)(unsigned)best;
                d2[i] = __uint_as_float((unsigned)(best >> 32));
            }
        } else {        // a dense root segment: all lanes scan it
            const int qi = b + (k - nG) * B;
            const int i = __ldg(hv_list + qi);
            const uint2 r = __ldg(hv_range + qi);
            if ((unsigned)i >= (unsigned)m) {
                if (lane == 0)
                    atomicOr(&ctl->err, DEVERR_BOUNDS);
                continue;
            }
            const float3 s = transform_pt(P, __ldg(src + i));
            unsigned long long unused = 0ull;
            const unsigned long long best = scan_run(csr, r.x, r.y, s, lane, ~0ull, unused);
            if (lane == 0) {
                nn[i] = (int)(unsigned)best;
                d2[i] = __uint_as_float((unsigned)(best >> 32));
            }
        }
    }
    // work counter: one global atomic per block; the last block to finish
    // clears the list lengths for the next search
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
            ctl->hv_count = 0;
            ctl->fb_done = 0u;
        }
    }
}

cudaError_t launch_fallback(const float4 *src, const double *pose, const float4 *bpts, const float4 *bbox,
                            const float4 *sb_box, const float4 *tgt, int n_tgt, const int *outside, const int *fb_list,
                            const int *hv_list, const uint2 *hv_range, const float4 *csr, DevCtl *ctl, int *nn,
                            float *d2, int m, int honor_stop, cudaStream_t st)
{
    // as many warps as can be resident
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
                         n_tgt, outside, fb_list, hv_list, hv_range, csr, ctl, nn, d2, m, honor_stop);
}

}  // namespace vicp
