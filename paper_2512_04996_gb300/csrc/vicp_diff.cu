// vicp_diff.cu -- the differentiable point-to-point loss of Eq. 1 over the
// pairs of a batch, and the se(3) maps its gradient needs.
//
// Loss of pair k at pose T with fixed correspondences nn (from the NNS of
// Alg. 4; they carry no gradient):
//     L_k = (1/M) sum_i |T p_i - q_nn(i)|^2.
// Its gradient under a left perturbation T <- Exp(d) T at d = 0, with
// d = (rho, phi) (translation part first):
//     dL/drho = (2/M) sum_i r_i,   dL/dphi = (2/M) sum_i s_i x r_i,
// s_i = T p_i, r_i = s_i - q_nn(i); and in a source point dL/dp_i =
// (2/M) R^T r_i.  For a pose parameterised as T = Exp(xi) T0 the gradient
// in xi is J(xi)^T times the left-perturbation gradient, J the left
// Jacobian of SE(3).
//
// s_i and r_i are formed in double-float arithmetic from the FP64 pose (the
// pose entries split into two floats), so the residual is exact to ~2^-48
// even where it is small against the coordinates; the sums are
// double-float, per item and then per pair in item order (deterministic).
#include "vicp_batch.h"
#include "vicp_df.cuh"
#include "vicp_launch.h"

namespace vicp {

// ---------------------------------------------------------------------------
// SE(3) exponential and left Jacobian (FP64, one thread per pose).  With
// t = |phi| and P = phi^ (the cross-product matrix):
//   Exp(rho, phi) = [[I + A P + B P^2, (I + B P + C P^2) rho], [0, 1]],
//   J(rho, phi)   = [[Js, Q], [0, Js]],  Js = I + B P + C P^2,
//   Q = R/2 + C (P R + R P + P R P) + D (P P R + R P P - 3 P R P)
//       + (D + 3 E)/2 (P R P P + P P R P),  R = rho^,
// with A = sin t / t, B = (1 - cos t)/t^2, C = (t - sin t)/t^3,
// D = (t^2/2 + cos t - 1)/t^4, E = (t - sin t - t^3/6)/t^5.  B is evaluated
// as 2 (sin(t/2)/t)^2; C, D and E lose digits to cancellation at small t, so
// for t < 2 they are summed from their Taylor series (terms
// (-1)^k t^2k / (2k + n)!, n = 3, 4, 5; E with the opposite sign) until the
// terms no longer change the sum.
// ---------------------------------------------------------------------------
struct M3 {
    double m[9];
};

__device__ inline M3 m3_hat(double x, double y, double z)
{
    return {{0.0, -z, y, z, 0.0, -x, -y, x, 0.0}};
}

__device__ inline M3 m3_mul(const M3 &a, const M3 &b)
{
    M3 c;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j)
            c.m[3 * i + j] = a.m[3 * i] * b.m[j] + a.m[3 * i + 1] * b.m[3 + j] + a.m[3 * i + 2] * b.m[6 + j];
    return c;
}

__device__ inline M3 m3_axpy(double s, const M3 &a, const M3 &b)   // s a + b
{
    M3 c;
    for (int k = 0; k < 9; ++k)
        c.m[k] = s * a.m[k] + b.m[k];
    return c;
}

__device__ inline double taylor_coeff(double t2, int n, double sign)
{
    double term = sign;
    for (int j = 2; j <= n; ++j)
        term /= (double)j;
    double sum = term;
    for (int k = 1; k < 40; ++k) {
        term *= -t2 / ((double)(2 * k + n - 1) * (double)(2 * k + n));
        const double next = sum + term;
        if (next == sum)
            break;
        sum = next;
    }
    return sum;
}

struct Se3Coeffs {
    double A, B, C, D, E;
};

__device__ inline Se3Coeffs se3_coeffs(double t)
{
    const double t2 = t * t;
    Se3Coeffs k;
    if (t < 1e-4) {
        k.A = 1.0 - t2 / 6.0 + t2 * t2 / 120.0;
        k.B = 0.5 - t2 / 24.0 + t2 * t2 / 720.0;
    } else {
        const double s = sin(0.5 * t) / t;
        k.A = sin(t) / t;
        k.B = 2.0 * s * s;
    }
    if (t < 2.0) {
        k.C = taylor_coeff(t2, 3, 1.0);
        k.D = taylor_coeff(t2, 4, 1.0);
        k.E = taylor_coeff(t2, 5, -1.0);
    } else {
        const double s = sin(t), c = cos(t);
        k.C = (t - s) / (t2 * t);
        k.D = (0.5 * t2 + c - 1.0) / (t2 * t2);
        k.E = (t - s - t2 * t / 6.0) / (t2 * t2 * t);
    }
    return k;
}

__global__ void __launch_bounds__(128) k_se3_exp(int n, const double *__restrict__ xi, const double *__restrict__ T0,
                                                 double *__restrict__ T)
{
    pdl_begin();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n)
        return;
    const double *x = xi + 6 * k;
    const double t = sqrt(x[3] * x[3] + x[4] * x[4] + x[5] * x[5]);
    const Se3Coeffs c = se3_coeffs(t);
    const M3 P = m3_hat(x[3], x[4], x[5]);
    const M3 P2 = m3_mul(P, P);
    M3 I = {{1, 0, 0, 0, 1, 0, 0, 0, 1}};
    const M3 R = m3_axpy(c.B, P2, m3_axpy(c.A, P, I));
    const M3 J = m3_axpy(c.C, P2, m3_axpy(c.B, P, I));
    double E[16];
    for (int a = 0; a < 3; ++a) {
        for (int b = 0; b < 3; ++b)
            E[4 * a + b] = R.m[3 * a + b];
        E[4 * a + 3] = J.m[3 * a] * x[0] + J.m[3 * a + 1] * x[1] + J.m[3 * a + 2] * x[2];
    }
    E[12] = E[13] = E[14] = 0.0;
    E[15] = 1.0;
    const double *A0 = T0 + 16 * k;
    double *out = T + 16 * k;
    for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b)
            out[4 * a + b] = E[4 * a] * A0[b] + E[4 * a + 1] * A0[4 + b] + E[4 * a + 2] * A0[8 + b] +
                             E[4 * a + 3] * A0[12 + b];
}

__global__ void __launch_bounds__(128) k_se3_jlt(int n, const double *__restrict__ xi, const double *__restrict__ g,
                                                 double *__restrict__ out)
{
    pdl_begin();
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n)
        return;
    const double *x = xi + 6 * k;
    const double t = sqrt(x[3] * x[3] + x[4] * x[4] + x[5] * x[5]);
    const Se3Coeffs c = se3_coeffs(t);
    const M3 P = m3_hat(x[3], x[4], x[5]);
    const M3 Rh = m3_hat(x[0], x[1], x[2]);
    const M3 P2 = m3_mul(P, P);
    M3 I = {{1, 0, 0, 0, 1, 0, 0, 0, 1}};
    const M3 Js = m3_axpy(c.C, P2, m3_axpy(c.B, P, I));
    const M3 PR = m3_mul(P, Rh), RP = m3_mul(Rh, P);
    const M3 PRP = m3_mul(PR, P);
    const M3 PPR = m3_mul(P, PR), RPP = m3_mul(RP, P);
    const M3 PRPP = m3_mul(PRP, P), PPRP = m3_mul(P, PRP);
    M3 Q;
    for (int i = 0; i < 9; ++i)
        Q.m[i] = 0.5 * Rh.m[i] + c.C * (PR.m[i] + RP.m[i] + PRP.m[i]) +
                 c.D * (PPR.m[i] + RPP.m[i] - 3.0 * PRP.m[i]) + 0.5 * (c.D + 3.0 * c.E) * (PRPP.m[i] + PPRP.m[i]);
    const double *gk = g + 6 * k;
    double *o = out + 6 * k;
    // [[Js, Q], [0, Js]]^T g = (Js^T g_rho, Q^T g_rho + Js^T g_phi)
    for (int j = 0; j < 3; ++j) {
        o[j] = Js.m[j] * gk[0] + Js.m[3 + j] * gk[1] + Js.m[6 + j] * gk[2];
        o[3 + j] = Q.m[j] * gk[0] + Q.m[3 + j] * gk[1] + Q.m[6 + j] * gk[2] + Js.m[j] * gk[3] +
                   Js.m[3 + j] * gk[4] + Js.m[6 + j] * gk[5];
    }
}

cudaError_t launch_se3_exp(int n, const double *xi, const double *T0, double *T, cudaStream_t st)
{
    return launch_kernel(k_se3_exp, dim3((n + 127) / 128), dim3(128), 0, st, n, xi, T0, T);
}

cudaError_t launch_se3_jlt(int n, const double *xi, const double *g, double *out, cudaStream_t st)
{
    return launch_kernel(k_se3_jlt, dim3((n + 127) / 128), dim3(128), 0, st, n, xi, g, out);
}

// ---------------------------------------------------------------------------
// The loss and its gradients, one block per (pair, tile) item.  Per item the
// seven sums [sum |r|^2, sum r, sum s x r] go to the item's slot; the block
// that reduces a pair's last item adds the pair's slots in item order and
// writes L_k and (if asked) dL_k * (2/M)(sum r, sum s x r).  Point
// gradients dL_k * (2/M) R^T r_i are written by the thread of the point.
// ---------------------------------------------------------------------------
constexpr int LOSS_THREADS = 256;
constexpr int LOSS_SUMS = 7;

__device__ __forceinline__ dfl df_of(double x)
{
    const float hi = __double2float_rn(x);
    return {hi, __double2float_rn(x - (double)hi)};
}

__global__ void __launch_bounds__(LOSS_THREADS) k_batch_loss(const float4 *__restrict__ src,
                                                             const float4 *__restrict__ tgt,
                                                             const BatchPair *__restrict__ pairs,
                                                             BatchState *__restrict__ state,
                                                             const BatchItem *__restrict__ items,
                                                             const double *__restrict__ pose,
                                                             const int *__restrict__ nn,
                                                             const double *__restrict__ dloss,
                                                             float2 *__restrict__ partials,
                                                             double *__restrict__ loss_out,
                                                             double *__restrict__ grad_pose,
                                                             float4 *__restrict__ grad_src, DevCtl *__restrict__ ctl)
{
    pdl_begin();
    constexpr int WARPS = LOSS_THREADS / 32;
    __shared__ dfl s_T[12];
    __shared__ float s_R[9];
    __shared__ float s_hi[WARPS][LOSS_SUMS], s_lo[WARPS][LOSS_SUMS];
    __shared__ int s_last;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const BatchItem it = items[blockIdx.x];
    const BatchPair *bp = pairs + it.pair;
    const double *Tk = pose + 16 * it.pair;
    if (tid < 12) {
        const int a = tid >> 2, b = tid & 3;
        s_T[tid] = df_of(Tk[4 * a + b]);   // entry (a, b) of the 3x4 upper block
        if (b < 3)
            s_R[3 * a + b] = __double2float_rn(Tk[4 * a + b]);
    }
    __syncthreads();
    const int M = bp->n_src, tbase = bp->tbase, n_tgt = bp->n_tgt;
    const double scale = 2.0 / (double)M * (dloss ? dloss[it.pair] : 1.0);
    const float scale_f = (float)scale;
    dfl acc[LOSS_SUMS];
#pragma unroll
    for (int k = 0; k < LOSS_SUMS; ++k)
        acc[k] = {0.0f, 0.0f};
    for (int i = it.i0 + tid; i < it.i1; i += LOSS_THREADS) {
        const int j = __ldg(nn + i);
        if ((unsigned)j >= (unsigned)n_tgt) {
            atomicOr(&ctl->err, DEVERR_BOUNDS);
            continue;
        }
        const float4 p = __ldg(src + i), q = __ldg(tgt + tbase + j);
        dfl s[3], r[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            dfl v = df_mul_f(s_T[4 * a], p.x);
            v = df_add(v, df_mul_f(s_T[4 * a + 1], p.y));
            v = df_add(v, df_mul_f(s_T[4 * a + 2], p.z));
            s[a] = df_add(v, s_T[4 * a + 3]);
            r[a] = df_sub(s[a], df_f(a == 0 ? q.x : (a == 1 ? q.y : q.z)));
        }
        acc[0] = df_acc(acc[0], df_add(df_add(df_mul(r[0], r[0]), df_mul(r[1], r[1])), df_mul(r[2], r[2])));
#pragma unroll
        for (int a = 0; a < 3; ++a)
            acc[1 + a] = df_acc(acc[1 + a], r[a]);
        acc[4] = df_acc(acc[4], df_sub(df_mul(s[1], r[2]), df_mul(s[2], r[1])));
        acc[5] = df_acc(acc[5], df_sub(df_mul(s[2], r[0]), df_mul(s[0], r[2])));
        acc[6] = df_acc(acc[6], df_sub(df_mul(s[0], r[1]), df_mul(s[1], r[0])));
        if (grad_src) {
            // (2/M) dL R^T r, the residual rounded to float first (its
            // double-float low part is below float resolution of the result)
            const float rx = r[0].hi + r[0].lo, ry = r[1].hi + r[1].lo, rz = r[2].hi + r[2].lo;
            float gv[3];
#pragma unroll
            for (int b = 0; b < 3; ++b)
                gv[b] = scale_f * (s_R[b] * rx + s_R[3 + b] * ry + s_R[6 + b] * rz);
            grad_src[i] = make_float4(gv[0], gv[1], gv[2], 0.0f);
        }
    }
    // block sums in a fixed order: warps by shuffles, then the warps in order
#pragma unroll
    for (int k = 0; k < LOSS_SUMS; ++k) {
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
    if (tid < LOSS_SUMS) {
        dfl v = {s_hi[0][tid], s_lo[0][tid]};
        for (int w = 1; w < WARPS; ++w)
            v = df_add(v, dfl{s_hi[w][tid], s_lo[w][tid]});
        partials[(size_t)blockIdx.x * LOSS_SUMS + tid] = make_float2(v.hi, v.lo);
        __threadfence();
    }
    __syncthreads();
    if (tid == 0)
        s_last = atomicAdd(&state[it.pair].items_done, 1u) == (unsigned)(bp->n_items - 1);
    __syncthreads();
    if (!s_last)
        return;
    __threadfence();
    if (tid < LOSS_SUMS) {
        dfl v = {0.0f, 0.0f};
        for (int b = 0; b < bp->n_items; ++b) {
            const float2 x = __ldcg(partials + (size_t)(bp->item0 + b) * LOSS_SUMS + tid);
            v = df_add(v, dfl{x.x, x.y});
        }
        const double sum = df_to_double(v);
        if (tid == 0)
            loss_out[it.pair] = sum / (double)M;
        else if (grad_pose)
            grad_pose[6 * it.pair + tid - 1] = scale * sum;
    }
    if (tid == 0)
        state[it.pair].items_done = 0u;
}

cudaError_t launch_batch_loss(const float4 *src, const float4 *tgt, const BatchPair *pairs, BatchState *state,
                              const BatchItem *items, int n_items, const double *pose, const int *nn,
                              const double *dloss, float2 *partials, double *loss_out, double *grad_pose,
                              float4 *grad_src, DevCtl *ctl, cudaStream_t st)
{
    return launch_kernel(k_batch_loss, dim3(n_items), dim3(LOSS_THREADS), 0, st, src, tgt, pairs, state, items, pose,
                         nn, dloss, partials, loss_out, grad_pose, grad_src, ctl);
}

}  // namespace vicp
