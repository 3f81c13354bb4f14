// vicp_solve64.cu -- the rigid update of Eq. 1 with FP64 accumulation and an
// FP64 solve (vicp_f64.cuh), in one launch: the variant a context selects
// with VICP_FLAG_FP64_SOLVE in place of the double-float reduction of
// vicp_solve.cu.  The launch has the same shape and the same fixed summation
// order (thread, warp, block, then all blocks by the last one), so its
// results are bit-reproducible from run to run.
#include "vicp_f64.cuh"
#include "vicp_launch.h"

namespace vicp {

constexpr int R64_THREADS = 256;
constexpr int R64_WARPS = R64_THREADS / 32;
static_assert(F64_SUMS == REDUCE_VALUES, "sum layout");

__global__ void __launch_bounds__(R64_THREADS) k_reduce_solve_f64(const float4 *__restrict__ src, int m,
                                                                  double *__restrict__ pose,
                                                                  const float4 *__restrict__ tgt, int n_tgt,
                                                                  const int *__restrict__ nn, float3 cf,
                                                                  double *__restrict__ partials,
                                                                  double *__restrict__ rmse_out,
                                                                  DevCtl *__restrict__ ctl, int honor_stop,
                                                                  double eps)
{
    pdl_begin();
    if (honor_stop && *(volatile int *)&ctl->stop)
        return;
    __shared__ PoseF sp;
    __shared__ double s_w[R64_WARPS][F64_SUMS];
    __shared__ int s_last;
    load_pose_f_block(pose, sp);
    const PoseF P = sp;
    const double3 c = make_double3((double)cf.x, (double)cf.y, (double)cf.z);
    double acc[F64_SUMS];
#pragma unroll
    for (int k = 0; k < F64_SUMS; ++k)
        acc[k] = 0.0;
    // this thread's points, four per round with all their loads issued first
    const int stride = gridDim.x * R64_THREADS;
    for (int i0 = blockIdx.x * R64_THREADS + threadIdx.x; i0 < m; i0 += 4 * stride) {
        int j[4];
        float4 p[4], q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int i = i0 + u * stride;
            j[u] = -1;
            if (i < m) {
                j[u] = __ldg(nn + i);
                p[u] = __ldg(src + i);
            }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if ((unsigned)j[u] < (unsigned)n_tgt)
                q[u] = __ldg(tgt + j[u]);
            else if (i0 + u * stride < m)   // no valid match: report, leave it out
                atomicOr(&ctl->err, DEVERR_BOUNDS);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            if ((unsigned)j[u] >= (unsigned)n_tgt)
                continue;
            accumulate_corr_f64(acc, transform_pt(P, p[u]), q[u], c);
        }
    }
    // warp sums through shared memory: lane l adds value l % 16 over lanes
    // 16 (l / 16) .. 16 (l / 16) + 15 in order, and the two halves are added
    __shared__ double s_t[R64_WARPS][F64_SUMS][33];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
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
    if (threadIdx.x < F64_SUMS) {
        double v = s_w[0][threadIdx.x];
#pragma unroll
        for (int w = 1; w < R64_WARPS; ++w)
            v += s_w[w][threadIdx.x];
        partials[blockIdx.x * F64_SUMS + threadIdx.x] = v;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        s_last = (int)atomicAdd(&ctl->red_done, 1u);
    __syncthreads();
    if (s_last == 0 && gridDim.x > 2 && warp == 0) {
        // The first block to finish runs the solve once on fixed sums of a
        // well-posed problem, writing only its own shared memory, so that the
        // solve's instructions are in L2 when the last block needs them.
        __shared__ double s_warm[F64_SUMS], s_wpose[16];
        if (lane < F64_SUMS)
            s_warm[lane] = lane == 6 ? 4.0 : (lane == 10 ? 2.0 : (lane == 14 || lane == 15 ? 1.0 : (lane == 7 ? 0.5 : 0.0)));
        if (lane < 16)
            s_wpose[lane] = (lane % 5) == 0 ? 1.0 : 0.0;
        __syncwarp();
        double r;
        solve_update_f64(s_warm, 8, c, s_wpose, r);
        return;
    }
    if (s_last != (int)gridDim.x - 1)
        return;
    __threadfence();

    // Last block: fixed-order sum of all partials.  Thread t adds value t % 16
    // of partials t/16, t/16 + 16, ...; the 16 groups are then added in order.
    __shared__ double s_r[R64_WARPS][F64_SUMS];
    __shared__ double s_tot[F64_SUMS];
    {
        const int k = threadIdx.x & 15, grp = threadIdx.x >> 4;
        double v = 0.0;
        for (int b0 = grp; b0 < (int)gridDim.x; b0 += 8 * (R64_THREADS / 16)) {   // eight loads in flight
            double q[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int b = b0 + u * (R64_THREADS / 16);
                q[u] = b < (int)gridDim.x ? __ldcg(partials + b * F64_SUMS + k) : 0.0;
            }
#pragma unroll
            for (int u = 0; u < 8; ++u)
                if (b0 + u * (R64_THREADS / 16) < (int)gridDim.x)
                    v += q[u];
        }
        v += __shfl_xor_sync(FULL_MASK, v, 16);   // groups 2w and 2w+1 of warp w
        if (lane < 16)
            s_r[warp][lane] = v;
    }
    __syncthreads();
    if (threadIdx.x < F64_SUMS) {
        double t = s_r[0][threadIdx.x];
#pragma unroll
        for (int w = 1; w < R64_WARPS; ++w)
            t += s_r[w][threadIdx.x];
        s_tot[threadIdx.x] = t;
    }
    __syncthreads();
    if (warp != 0)
        return;

    double rmse;
    const bool ok = solve_update_f64(s_tot, m, c, pose, rmse);
    if (lane == 0) {
        ctl->red_done = 0u;
        if (rmse_out)
            *rmse_out = rmse;
    }
    if (!ok) {
        if (lane == 0) {
            atomicOr(&ctl->err, DEVERR_DEGENERATE);
            if (honor_stop) {
                ctl->stop = 1;
                ctl->last_rmse = rmse;
            }
        }
        return;
    }
    if (lane == 0 && honor_stop) {
        const int it = ctl->iters;
        ctl->iters = it + 1;
        ctl->last_rmse = rmse;
        if (eps > 0.0 && it >= 1 && fabs(rmse - ctl->prev_rmse) < eps)
            ctl->stop = 1;
        ctl->prev_rmse = rmse;
    }
}

cudaError_t launch_reduce_solve_f64(const float4 *src, int m, double *pose, const float4 *tgt, int n_tgt,
                                    const int *nn, float3 center, double *partials, int nparts, double *rmse_out,
                                    DevCtl *ctl, int honor_stop, double eps, cudaStream_t st)
{
    return launch_kernel(k_reduce_solve_f64, dim3(nparts), dim3(R64_THREADS), 0, st, src, m, pose, tgt, n_tgt, nn,
                         center, partials, rmse_out, ctl, honor_stop, eps);
}

}  // namespace vicp
