// vicp_solve.cu -- rigid update of Eq. 1: deterministic FP64 reduction of the
// centroids, cross-covariance and residual, and the FP64 solve, in one launch.
#include "vicp_launch.h"

namespace vicp {

constexpr int RED_THREADS = 256;

__device__ __forceinline__ double det3(double a, double b, double c, double d, double e, double f, double g, double h,
                                       double i)
{
    return a * (e * i - f * h) - b * (d * i - f * g) + c * (d * h - e * g);
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

// Horn's closed form.  With S the 3x3 cross-covariance sum (s - sbar)(q - qbar)^T,
// the rotation minimising Eq. 1 is the unit quaternion (w, x, y, z) of the
// largest eigenvalue of the symmetric, traceless 4x4
//   [ Sxx+Syy+Szz  Syz-Szy      Szx-Sxz      Sxy-Syx     ]
//   [ Syz-Szy      Sxx-Syy-Szz  Sxy+Syx      Szx+Sxz     ]
//   [ Szx-Sxz      Sxy+Syx     -Sxx+Syy-Szz  Syz+Szy     ]
//   [ Sxy-Syx      Szx+Sxz      Syz+Szy     -Sxx-Syy+Szz ].
// Its characteristic polynomial is l^4 + c2 l^2 + c1 l + c0 with
// c2 = -2 |S|_F^2, c1 = -8 det S, c0 = det N.  The largest root is found by
// Newton's method from the upper bound (Ga + Gb) / 2 = E/2 + tr S (Ga, Gb the
// centred sums of squares, E the centred residual), which lies just right of
// it; from the right of the largest root of a real-rooted polynomial Newton
// decreases monotonically onto it.  The eigenvector is a column of the
// adjugate of N - l I (rank one at a simple eigenvalue); the column of the
// largest diagonal cofactor is used.  All in FP64.
__device__ void horn_rotation(const double S[9], double E, double R[9])
{
    const double sxx = S[0], sxy = S[1], sxz = S[2], syx = S[3], syy = S[4], syz = S[5], szx = S[6], szy = S[7],
                 szz = S[8];
    double N[4][4] = {{sxx + syy + szz, syz - szy, szx - sxz, sxy - syx},
                      {syz - szy, sxx - syy - szz, sxy + syx, szx + sxz},
                      {szx - sxz, sxy + syx, -sxx + syy - szz, syz + szy},
                      {sxy - syx, szx + sxz, syz + szy, -sxx - syy + szz}};
    double s2 = 0.0;
    for (int k = 0; k < 9; ++k)
        s2 += S[k] * S[k];
    const double c2 = -2.0 * s2;
    const double c1 = -8.0 * det3(sxx, sxy, sxz, syx, syy, syz, szx, szy, szz);
    // det N by Laplace expansion along rows 0 and 1 (u: 2x2 minors of rows
    // 0-1, w: of rows 2-3, over column pairs)
    const double u01 = N[0][0] * N[1][1] - N[0][1] * N[1][0], u02 = N[0][0] * N[1][2] - N[0][2] * N[1][0];
    const double u03 = N[0][0] * N[1][3] - N[0][3] * N[1][0], u12 = N[0][1] * N[1][2] - N[0][2] * N[1][1];
    const double u13 = N[0][1] * N[1][3] - N[0][3] * N[1][1], u23 = N[0][2] * N[1][3] - N[0][3] * N[1][2];
    const double w01 = N[2][0] * N[3][1] - N[2][1] * N[3][0], w02 = N[2][0] * N[3][2] - N[2][2] * N[3][0];
    const double w03 = N[2][0] * N[3][3] - N[2][3] * N[3][0], w12 = N[2][1] * N[3][2] - N[2][2] * N[3][1];
    const double w13 = N[2][1] * N[3][3] - N[2][3] * N[3][1], w23 = N[2][2] * N[3][3] - N[2][3] * N[3][2];
    const double c0 = u01 * w23 - u02 * w13 + u03 * w12 + u12 * w03 - u13 * w02 + u23 * w01;

    double l = 0.5 * E + (sxx + syy + szz);
    l += 1e-12 * fabs(l);
    const double loose = sqrt(3.0 * s2);   // l_max <= sqrt(3/4 tr N^2) = sqrt(3) |S|_F
    if (!(l > 0.0) || ((l * l + c2) * l + c1) * l + c0 < 0.0 || l > loose)
        l = loose;
    for (int it = 0; it < 64; ++it) {
        const double P = ((l * l + c2) * l + c1) * l + c0;
        const double dP = (4.0 * l * l + 2.0 * c2) * l + c1;
        if (!(dP != 0.0))
            break;
        const double step = P / dP;
        l -= step;
        if (fabs(step) <= 1e-15 * fabs(l))
            break;
    }
    // adjugate of A = N - l I (symmetric): column k is (C_k0, C_k1, C_k2, C_k3)
    // with C_ij = (-1)^(i+j) det(A without row i and column j).  The column
    // of the largest diagonal cofactor is the best-conditioned eigenvector.
    const double a00 = N[0][0] - l, a11 = N[1][1] - l, a22 = N[2][2] - l, a33 = N[3][3] - l;
    const double a01 = N[0][1], a02 = N[0][2], a03 = N[0][3], a12 = N[1][2], a13 = N[1][3], a23 = N[2][3];
    const double c00 = det3(a11, a12, a13, a12, a22, a23, a13, a23, a33);
    const double c11 = det3(a00, a02, a03, a02, a22, a23, a03, a23, a33);
    const double c22 = det3(a00, a01, a03, a01, a11, a13, a03, a13, a33);
    const double c33 = det3(a00, a01, a02, a01, a11, a12, a02, a12, a22);
    double v[4];
    const double m01 = fabs(c00) >= fabs(c11) ? fabs(c00) : fabs(c11);
    const double m23 = fabs(c22) >= fabs(c33) ? fabs(c22) : fabs(c33);
    if (m01 >= m23) {
        if (fabs(c00) >= fabs(c11)) {   // column 0
            v[0] = c00;
            v[1] = -det3(a01, a02, a03, a12, a22, a23, a13, a23, a33);
            v[2] = det3(a01, a02, a03, a11, a12, a13, a13, a23, a33);
            v[3] = -det3(a01, a02, a03, a11, a12, a13, a12, a22, a23);
        } else {                        // column 1
            v[0] = -det3(a01, a12, a13, a02, a22, a23, a03, a23, a33);
            v[1] = c11;
            v[2] = -det3(a00, a01, a03, a02, a12, a23, a03, a13, a33);
            v[3] = det3(a00, a01, a02, a02, a12, a22, a03, a13, a23);
        }
    } else {
        if (fabs(c22) >= fabs(c33)) {   // column 2
            v[0] = det3(a01, a02, a03, a11, a12, a13, a13, a23, a33);
            v[1] = -det3(a00, a02, a03, a01, a12, a13, a03, a23, a33);
            v[2] = c22;
            v[3] = -det3(a00, a01, a02, a01, a11, a12, a03, a13, a23);
        } else {                        // column 3
            v[0] = -det3(a01, a02, a03, a11, a12, a13, a12, a22, a23);
            v[1] = det3(a00, a02, a03, a01, a12, a13, a02, a22, a23);
            v[2] = -det3(a00, a01, a03, a01, a11, a13, a02, a12, a23);
            v[3] = c33;
        }
    }
    const double inv = 1.0 / sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] + v[3] * v[3]);
    const double w = v[0] * inv, x = v[1] * inv, y = v[2] * inv, z = v[3] * inv;
    R[0] = w * w + x * x - y * y - z * z; R[1] = 2.0 * (x * y - w * z);         R[2] = 2.0 * (x * z + w * y);
    R[3] = 2.0 * (y * x + w * z);         R[4] = w * w - x * x + y * y - z * z; R[5] = 2.0 * (y * z - w * x);
    R[6] = 2.0 * (z * x - w * y);         R[7] = 2.0 * (z * y + w * x);         R[8] = w * w - x * x - y * y + z * z;
}

// ---------------------------------------------------------------------------
// Extended-precision sums on the FP32 pipes.  GB300 executes FP64 at a small
// fraction of its FP32 rate, so the per-point work of the reduction is done
// with error-free float transformations ("double-float": a value is the
// unevaluated sum hi + lo of two floats, about 48 significant bits):
//   two_sum(a, b)  = (s, e) with s + e == a + b exactly (Knuth),
//   two_prod(a, b) = (p, e) with p + e == a * b exactly (one FMA).
// Every per-point term is formed exactly; sums of terms carry a relative
// error of order 2^-46 of the summed magnitudes, comparable to an FP64
// accumulation.  Warp partials are converted to FP64 and everything after
// that -- the sum over warps and blocks and the solve -- is FP64.
// ---------------------------------------------------------------------------
struct dfl {
    float hi, lo;
};

__device__ __forceinline__ dfl two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}

__device__ __forceinline__ dfl quick_two_sum(float a, float b)   // needs |a| >= |b| or a == 0
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ dfl df_add(dfl x, dfl y)
{
    const dfl s = two_sum(x.hi, y.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

// (x.hi + x.lo) * (y.hi + y.lo), the lo * lo term (2^-48 relative) dropped
__device__ __forceinline__ dfl df_mul(dfl x, dfl y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return quick_two_sum(p, e);
}

__device__ __forceinline__ dfl df_shfl_xor(dfl v, int o)
{
    return {__shfl_xor_sync(FULL_MASK, v.hi, o), __shfl_xor_sync(FULL_MASK, v.lo, o)};
}

// ---------------------------------------------------------------------------
// Reduction and solve in one launch.  Relative to a fixed centre c (the grid
// centre rounded to float; s - c is then exact as a double-float), every
// thread accumulates over a fixed strided set of points
//   [0..2]  sum (s - c)          [3..5]  sum (q - c)
//   [6..14] sum (s - c)(q - c)^T [15]    sum |s - q|^2
// in double-float, each warp reduces them with shuffles in a fixed order, and
// the warps' partials are added in FP64 per block.  The last block to finish
// (atomic ticket) adds all block partials in a fixed order and thread 0
// solves Eq. 1 and updates the pose, so the result is bit-identical from run
// to run whichever block finishes last.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(RED_THREADS) k_reduce_solve(const float4 *__restrict__ src, int m,
                                                              double *__restrict__ pose,
                                                              const float4 *__restrict__ tgt, int n_tgt,
                                                              const int *__restrict__ nn, float3 cf,
                                                              double *__restrict__ partials,
                                                              double *__restrict__ rmse_out,
                                                              DevCtl *__restrict__ ctl, int honor_stop, double eps)
{
    if (honor_stop && *(volatile int *)&ctl->stop)
        return;
    __shared__ PoseF sp;
    __shared__ double s_red[RED_THREADS / 32][REDUCE_VALUES];
    __shared__ float s_hi[RED_THREADS / 32][REDUCE_VALUES], s_lo[RED_THREADS / 32][REDUCE_VALUES];
    __shared__ int s_last;
    load_pose_f_block(pose, sp);
    const PoseF P = sp;
    dfl acc[REDUCE_VALUES];
#pragma unroll
    for (int k = 0; k < REDUCE_VALUES; ++k)
        acc[k] = {0.0f, 0.0f};
    for (int i = blockIdx.x * RED_THREADS + threadIdx.x; i < m; i += gridDim.x * RED_THREADS) {
        const int j = __ldg(nn + i);
        if ((unsigned)j >= (unsigned)n_tgt) {   // no valid match: report, leave it out
            atomicOr(&ctl->err, DEVERR_BOUNDS);
            continue;
        }
        const float3 s = transform_pt(P, __ldg(src + i));
        const float4 q = __ldg(tgt + j);
        const dfl sv[3] = {two_sum(s.x, -cf.x), two_sum(s.y, -cf.y), two_sum(s.z, -cf.z)};
        const dfl qv[3] = {two_sum(q.x, -cf.x), two_sum(q.y, -cf.y), two_sum(q.z, -cf.z)};
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            acc[a] = df_add(acc[a], sv[a]);
            acc[3 + a] = df_add(acc[3 + a], qv[a]);
#pragma unroll
            for (int b = 0; b < 3; ++b)
                acc[6 + 3 * a + b] = df_add(acc[6 + 3 * a + b], df_mul(sv[a], qv[b]));
        }
        const dfl ex = two_sum(s.x, -q.x), ey = two_sum(s.y, -q.y), ez = two_sum(s.z, -q.z);
        acc[15] = df_add(acc[15], df_add(df_add(df_mul(ex, ex), df_mul(ey, ey)), df_mul(ez, ez)));
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < REDUCE_VALUES; ++k) {
        dfl v = acc[k];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
            v = df_add(v, df_shfl_xor(v, o));
        if (lane == 0) {
            s_hi[warp][k] = v.hi;
            s_lo[warp][k] = v.lo;
        }
    }
    __syncthreads();
    // the block's warps in double-float, then one FP64 value per thread 0..15
    if (threadIdx.x < REDUCE_VALUES) {
        dfl v = {s_hi[0][threadIdx.x], s_lo[0][threadIdx.x]};
#pragma unroll
        for (int w = 1; w < RED_THREADS / 32; ++w)
            v = df_add(v, dfl{s_hi[w][threadIdx.x], s_lo[w][threadIdx.x]});
        partials[blockIdx.x * REDUCE_VALUES + threadIdx.x] = (double)v.hi + (double)v.lo;
        __threadfence();
    }
    __syncthreads();
    if (threadIdx.x == 0)
        s_last = atomicAdd(&ctl->red_done, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();

    // Last block: fixed-order sum of all partials.  Thread t adds value t % 16
    // of partials t/16, t/16 + 16, ...; the 16 groups are then added in order.
    const int k = threadIdx.x & 15, grp = threadIdx.x >> 4;
    double v = 0.0;
    for (int b = grp; b < (int)gridDim.x; b += RED_THREADS / 16)
        v += __ldcg(partials + b * REDUCE_VALUES + k);
    v += __shfl_xor_sync(FULL_MASK, v, 16);   // groups 2w and 2w+1 of warp w
    if (lane < 16)
        s_red[warp][lane] = v;
    __syncthreads();
    __shared__ double s_tot[REDUCE_VALUES];
    if (threadIdx.x < REDUCE_VALUES) {
        double t = 0.0;
#pragma unroll
        for (int w = 0; w < RED_THREADS / 32; ++w)
            t += s_red[w][threadIdx.x];
        s_tot[threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x != 0)
        return;
    ctl->red_done = 0u;
    double S[REDUCE_VALUES];
#pragma unroll
    for (int q = 0; q < REDUCE_VALUES; ++q)
        S[q] = s_tot[q];
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
    // centred residual E = sum |s - q|^2 - M |sbar - qbar|^2
    const double dm[3] = {pb[0] - qb[0], pb[1] - qb[1], pb[2] - qb[2]};
    const double E = S[15] - M * (dm[0] * dm[0] + dm[1] * dm[1] + dm[2] * dm[2]);
    double R[9];
    horn_rotation(H, E, R);
    const double pa[3] = {pb[0] + (double)cf.x, pb[1] + (double)cf.y, pb[2] + (double)cf.z};
    const double qa[3] = {qb[0] + (double)cf.x, qb[1] + (double)cf.y, qb[2] + (double)cf.z};
    double dT[12];
    for (int a = 0; a < 3; ++a) {
        dT[4 * a + 0] = R[3 * a + 0];
        dT[4 * a + 1] = R[3 * a + 1];
        dT[4 * a + 2] = R[3 * a + 2];
        dT[4 * a + 3] = qa[a] - (R[3 * a] * pa[0] + R[3 * a + 1] * pa[1] + R[3 * a + 2] * pa[2]);
    }
    double T[16];
    for (int q = 0; q < 16; ++q)
        T[q] = pose[q];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 4; ++b)
            pose[4 * a + b] = dT[4 * a] * T[b] + dT[4 * a + 1] * T[4 + b] + dT[4 * a + 2] * T[8 + b] +
                              dT[4 * a + 3] * T[12 + b];
    if (honor_stop) {
        const int it = ctl->iters;
        ctl->iters = it + 1;
        ctl->last_rmse = rmse;
        if (eps > 0.0 && it >= 1 && fabs(rmse - ctl->prev_rmse) < eps)
            ctl->stop = 1;
        ctl->prev_rmse = rmse;
    }
}

cudaError_t launch_reduce_solve(const float4 *src, int m, double *pose, const float4 *tgt, int n_tgt, const int *nn,
                                float3 center, double *partials, int nparts, double *rmse_out, DevCtl *ctl,
                                int honor_stop, double eps, cudaStream_t st)
{
    k_reduce_solve<<<nparts, RED_THREADS, 0, st>>>(src, m, pose, tgt, n_tgt, nn, center, partials, rmse_out, ctl,
                                                   honor_stop, eps);
    return cudaGetLastError();
}

}  // namespace vicp
