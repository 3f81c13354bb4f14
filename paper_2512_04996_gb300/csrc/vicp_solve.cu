// vicp_solve.cu -- rigid update of Eq. 1: deterministic FP64 reduction of the
// centroids, cross-covariance and residual, and the FP64 solve.
#include "vicp_launch.h"

namespace vicp {

// ---------------------------------------------------------------------------
// Reduction.  Every block accumulates, in FP64 and relative to a fixed
// centre c (the grid centre, to keep the single-pass covariance well
// conditioned):
//   [0..2]  sum (s - c)          [3..5]  sum (q - c)
//   [6..14] sum (s - c)(q - c)^T [15]    sum |s - q|^2
// over a fixed strided set of points, reduces them with warp shuffles and
// shared memory in a fixed order, and writes its 16 partials.  The grid size
// depends only on M, so the sums are bit-identical from run to run.
// ---------------------------------------------------------------------------
constexpr int RED_THREADS = 256;

__global__ void __launch_bounds__(RED_THREADS) k_reduce(const float4 *__restrict__ src, int m,
                                                        const double *__restrict__ pose,
                                                        const float4 *__restrict__ tgt, int n_tgt,
                                                        const int *__restrict__ nn, double3 c,
                                                        double *__restrict__ partials,
                                                        DevCtl *__restrict__ ctl, int honor_stop)
{
    if (honor_stop && *(volatile int *)&ctl->stop)
        return;
    __shared__ PoseF sp;
    __shared__ double s_red[RED_THREADS / 32][REDUCE_VALUES];
    if (threadIdx.x == 0)
        load_pose_f(pose, sp);
    __syncthreads();
    const PoseF P = sp;
    double acc[REDUCE_VALUES];
#pragma unroll
    for (int k = 0; k < REDUCE_VALUES; ++k)
        acc[k] = 0.0;
    for (int i = blockIdx.x * RED_THREADS + threadIdx.x; i < m; i += gridDim.x * RED_THREADS) {
        const int j = __ldg(nn + i);
        if ((unsigned)j >= (unsigned)n_tgt) {   // no valid match: report, leave it out
            atomicOr(&ctl->err, DEVERR_BOUNDS);
            continue;
        }
        const float3 s = transform_pt(P, __ldg(src + i));
        const float4 q = __ldg(tgt + j);
        const double sv[3] = {(double)s.x - c.x, (double)s.y - c.y, (double)s.z - c.z};
        const double qv[3] = {(double)q.x - c.x, (double)q.y - c.y, (double)q.z - c.z};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            acc[a] += sv[a];
            acc[3 + a] += qv[a];
#pragma unroll
            for (int b = 0; b < 3; ++b)
                acc[6 + 3 * a + b] = fma(sv[a], qv[b], acc[6 + 3 * a + b]);
        }
        const double ex = (double)s.x - (double)q.x, ey = (double)s.y - (double)q.y,
                     ez = (double)s.z - (double)q.z;
        acc[15] += ex * ex + ey * ey + ez * ez;
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < REDUCE_VALUES; ++k) {
        double v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(FULL_MASK, v, o);
        if (lane == 0)
            s_red[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x < REDUCE_VALUES) {
        double v = 0.0;
#pragma unroll
        for (int w = 0; w < RED_THREADS / 32; ++w)
            v += s_red[w][threadIdx.x];
        partials[blockIdx.x * REDUCE_VALUES + threadIdx.x] = v;
    }
}

cudaError_t launch_reduce(const float4 *src, int m, const double *pose, const float4 *tgt, int n_tgt,
                          const int *nn, double3 center, double *partials, DevCtl *ctl, int honor_stop,
                          cudaStream_t st)
{
    k_reduce<<<reduce_blocks(m), RED_THREADS, 0, st>>>(src, m, pose, tgt, n_tgt, nn, center, partials, ctl,
                                                       honor_stop);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Solve.  Horn's closed form: with S the 3x3 cross-covariance
// sum (s - sbar)(q - qbar)^T, the rotation minimising Eq. 1 is the unit
// quaternion of the largest eigenvalue of the symmetric 4x4
//   [ Sxx+Syy+Szz  Syz-Szy      Szx-Sxz      Sxy-Syx     ]
//   [ Syz-Szy      Sxx-Syy-Szz  Sxy+Syx      Szx+Sxz     ]
//   [ Szx-Sxz      Sxy+Syx     -Sxx+Syy-Szz  Syz+Szy     ]
//   [ Sxy-Syx      Szx+Sxz      Syz+Szy     -Sxx-Syy+Szz ]
// found here by cyclic Jacobi rotations in FP64.  A quaternion is always a
// proper rotation, so no reflection fix is needed.  t = qbar - R sbar, and
// pose <- [R t] * pose.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void jacobi_rotate(double A[4][4], double V[4][4], int p, int q)
{
    const double apq = A[p][q];
    if (apq == 0.0)
        return;
    const double theta = (A[q][q] - A[p][p]) / (2.0 * apq);
    double t;
    if (fabs(theta) > 1e150)
        t = 0.5 / theta;
    else
        t = (theta >= 0.0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
    const double c = 1.0 / sqrt(t * t + 1.0);
    const double s = t * c;
    const double tau = s / (1.0 + c);
    const double h = t * apq;
    A[p][p] -= h;
    A[q][q] += h;
    A[p][q] = A[q][p] = 0.0;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        if (r != p && r != q) {
            const double g = A[r][p], k = A[r][q];
            A[r][p] = A[p][r] = g - s * (k + g * tau);
            A[r][q] = A[q][r] = k + s * (g - k * tau);
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        const double g = V[r][p], k = V[r][q];
        V[r][p] = g - s * (k + g * tau);
        V[r][q] = k + s * (g - k * tau);
    }
}

__device__ __forceinline__ void horn_rotation(const double S[9], double R[9])
{
    const double sxx = S[0], sxy = S[1], sxz = S[2], syx = S[3], syy = S[4], syz = S[5], szx = S[6], szy = S[7],
                 szz = S[8];
    double A[4][4] = {{sxx + syy + szz, syz - szy, szx - sxz, sxy - syx},
                      {syz - szy, sxx - syy - szz, sxy + syx, szx + sxz},
                      {szx - sxz, sxy + syx, -sxx + syy - szz, syz + szy},
                      {sxy - syx, szx + sxz, syz + szy, -sxx - syy + szz}};
    double V[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
    for (int sweep = 0; sweep < 32; ++sweep) {
        double off = 0.0, dia = 0.0;
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            dia += A[p][p] * A[p][p];
#pragma unroll
            for (int q = p + 1; q < 4; ++q)
                off += A[p][q] * A[p][q];
        }
        if (off <= 1e-34 * dia)
            break;
        jacobi_rotate(A, V, 0, 1);
        jacobi_rotate(A, V, 0, 2);
        jacobi_rotate(A, V, 0, 3);
        jacobi_rotate(A, V, 1, 2);
        jacobi_rotate(A, V, 1, 3);
        jacobi_rotate(A, V, 2, 3);
    }
    int k = 0;
#pragma unroll
    for (int p = 1; p < 4; ++p)
        if (A[p][p] > A[k][k])
            k = p;
    double w = V[0][k], x = V[1][k], y = V[2][k], z = V[3][k];
    const double inv = 1.0 / sqrt(w * w + x * x + y * y + z * z);
    w *= inv; x *= inv; y *= inv; z *= inv;
    R[0] = w * w + x * x - y * y - z * z; R[1] = 2.0 * (x * y - w * z);         R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (y * x + w * z);         R[4] = w * w - x * x + y * y - z * z; R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (z * x - w * y);         R[7] = 2.0 * (z * y + w * x);         R[8] = w * w - x * x - y * y + z * z;
}

// rank(S) < 2: every 2x2 minor negligible against |S|_F^2 (a definition
// shared with the oracle, not its code).
__device__ bool rank_below_two(const double S[9])
{
    double s2 = 0.0;
#pragma unroll
    for (int k = 0; k < 9; ++k)
        s2 += S[k] * S[k];
    if (s2 == 0.0)
        return true;
    double c2 = 0.0;
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
            const double cf = S[3 * i1 + j1] * S[3 * i2 + j2] - S[3 * i1 + j2] * S[3 * i2 + j1];
            c2 += cf * cf;
        }
    return sqrt(c2) <= 1e-12 * s2;
}

constexpr int SOLVE_THREADS = 256;

__global__ void __launch_bounds__(SOLVE_THREADS) k_solve(const double *__restrict__ partials, int nparts, int m,
                                                         double3 c, double *__restrict__ pose,
                                                         double *__restrict__ rmse_out,
                                                         DevCtl *__restrict__ ctl, int honor_stop, double eps)
{
    if (honor_stop && *(volatile int *)&ctl->stop)
        return;
    __shared__ double s_sum[SOLVE_THREADS / 32][REDUCE_VALUES];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // Fixed-order sum of the block partials: thread t adds partials t, t+256, ...
#pragma unroll 1
    for (int k = 0; k < REDUCE_VALUES; ++k) {
        double v = 0.0;
        for (int b = threadIdx.x; b < nparts; b += SOLVE_THREADS)
            v += partials[b * REDUCE_VALUES + k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v += __shfl_xor_sync(FULL_MASK, v, o);
        if (lane == 0)
            s_sum[warp][k] = v;
    }
    __syncthreads();
    if (threadIdx.x != 0)
        return;
    double S[REDUCE_VALUES];
    for (int k = 0; k < REDUCE_VALUES; ++k) {
        double v = 0.0;
        for (int w = 0; w < SOLVE_THREADS / 32; ++w)
            v += s_sum[w][k];
        S[k] = v;
    }
    const double M = (double)m;
    const double pb[3] = {S[0] / M, S[1] / M, S[2] / M};   // relative to c
    const double qb[3] = {S[3] / M, S[4] / M, S[5] / M};
    double H[9];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            H[3 * a + b] = S[6 + 3 * a + b] - M * pb[a] * qb[b];
    const double rmse = sqrt(S[15] / M);
    if (rmse_out)
        *rmse_out = rmse;
    if (rank_below_two(H)) {
        atomicOr(&ctl->err, DEVERR_DEGENERATE);
        if (honor_stop) {
            ctl->stop = 1;
            ctl->last_rmse = rmse;
        }
        return;
    }
    double R[9];
    horn_rotation(H, R);
    const double pa[3] = {pb[0] + c.x, pb[1] + c.y, pb[2] + c.z};
    const double qa[3] = {qb[0] + c.x, qb[1] + c.y, qb[2] + c.z};
    double dT[12];
    for (int a = 0; a < 3; ++a) {
        dT[4 * a + 0] = R[3 * a + 0];
        dT[4 * a + 1] = R[3 * a + 1];
        dT[4 * a + 2] = R[3 * a + 2];
        dT[4 * a + 3] = qa[a] - (R[3 * a] * pa[0] + R[3 * a + 1] * pa[1] + R[3 * a + 2] * pa[2]);
    }
    double T[16];
    for (int k = 0; k < 16; ++k)
        T[k] = pose[k];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 4; ++b)
            pose[4 * a + b] = dT[4 * a] * T[b] + dT[4 * a + 1] * T[4 + b] + dT[4 * a + 2] * T[8 + b] +
                              dT[4 * a + 3] * T[12 + b];
    for (int b = 0; b < 4; ++b)
        pose[12 + b] = T[12 + b];
    if (honor_stop) {
        const int k = ctl->iters;
        ctl->iters = k + 1;
        ctl->last_rmse = rmse;
        if (eps > 0.0 && k >= 1 && fabs(rmse - ctl->prev_rmse) < eps)
            ctl->stop = 1;
        ctl->prev_rmse = rmse;
    }
}

cudaError_t launch_solve(const double *partials, int nparts, int m, double3 center, double *pose,
                         double *rmse_out, DevCtl *ctl, int honor_stop, double eps, cudaStream_t st)
{
    k_solve<<<1, SOLVE_THREADS, 0, st>>>(partials, nparts, m, center, pose, rmse_out, ctl, honor_stop, eps);
    return cudaGetLastError();
}

}  // namespace vicp
