// vicp_f64.cuh -- the reduction sums and the rigid solve of Eq. 1 in FP64,
// shared by the single-pair FP64 reduction kernel (vicp_solve64.cu) and the
// batched iteration kernel's FP64 variant.
//
// This is the precision recipe stated for the method's update: coordinates
// and distances in float, the centroid / cross-covariance accumulation and
// the 3x3 solve in FP64.  It runs beside the double-float path
// (vicp_df.cuh), selected per context by a flag, so that the two can be
// measured against each other and against the oracle.
#pragma once

#include "vicp_device.cuh"

namespace vicp {

// The 16 sums of one ICP iteration in FP64, relative to a fixed centre c
// (the grid centre, a float, so every difference s - c, q - c, s - q of two
// floats is exact in double):
//   [0..2]  sum (s - c)          [3..5]  sum (q - c)
//   [6..14] sum (s - c)(q - c)^T [15]    sum |s - q|^2
constexpr int F64_SUMS = 16;

__device__ __forceinline__ void accumulate_corr_f64(double (&acc)[F64_SUMS], float3 s, float4 q, double3 c)
{
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
    const double ex = (double)s.x - (double)q.x, ey = (double)s.y - (double)q.y, ez = (double)s.z - (double)q.z;
    acc[15] = fma(ez, ez, fma(ey, ey, fma(ex, ex, acc[15])));
}

__device__ __forceinline__ double warp_sum_f64(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v += __shfl_xor_sync(FULL_MASK, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// The rigid update of Eq. 1 in FP64 from the sums s_tot (shared memory) of m
// correspondences, by one warp:
//  * lanes 0..8 hold H = sum (s - sbar)(q - qbar)^T, entry (k / 3, k % 3),
//    and its 2x2 cofactors for the rank test; H is then scaled by a power of
//    two to |H|_F ~ 1 (the rotation does not change).
//  * Horn's closed form: the rotation is the unit quaternion (w, x, y, z) of
//    the largest eigenvalue of the symmetric 4x4 matrix N built from H.
//    Lanes 0..15 hold N, entry (k / 4, k % 4), lanes 16..31 the eigenvector
//    matrix V (starting at I), and cyclic Jacobi sweeps (Golub & Van Loan,
//    the symmetric Schur rotation) diagonalise N in place: for each pair
//    (p, q), A <- J^T A J and V <- V J with the rotation J that zeroes
//    A_pq, each lane updating its own entry from its row or column partner
//    by one shuffle.  Jacobi is backward stable, so close eigenvalues (nearly
//    symmetric geometry) cost accuracy only in the eigenvector they make
//    ambiguous, never elsewhere.
//  * R from the quaternion, t = qbar - R sbar, and lanes 0..11 compose
//    pose <- dT * pose.
// Returns false, leaving the pose untouched, when rank(H) < 2 (every 2x2
// minor negligible: |cof(H)|_F <= 1e-12 |H|_F^2).  rmse = sqrt(S15 / m) on
// every lane.  Every lane of the warp must call it.
// ---------------------------------------------------------------------------
static __device__ __noinline__ bool solve_update_f64(const double *s_tot, int m, double3 c, double *pose,
                                                     double &rmse)
{
    const int lane = threadIdx.x & 31;
    const int pc = lane & 3;
    double P0 = 0.0, P1 = 0.0, P2 = 0.0, P3 = 0.0;
    if (lane < 12) {
        P0 = pose[pc];
        P1 = pose[4 + pc];
        P2 = pose[8 + pc];
        P3 = pose[12 + pc];
    }
    const double invM = 1.0 / (double)m;
    rmse = sqrt(s_tot[15] * invM);

    // H entry (a, b) on lane 3a + b < 9
    const int a = lane < 9 ? lane / 3 : 0, b = lane < 9 ? lane - 3 * a : 0;
    double h = 0.0;
    if (lane < 9)
        h = s_tot[6 + lane] - s_tot[a] * s_tot[3 + b] * invM;
    const double hn2 = warp_sum_f64(h * h);
    if (!(hn2 > 0.0) || !isfinite(hn2))
        return false;
    // cofactor (a, b) from the cyclically next rows and columns
    double cof = 0.0;
    {
        const int a1 = a == 2 ? 0 : a + 1, a2 = a == 0 ? 2 : a - 1;
        const int b1 = b == 2 ? 0 : b + 1, b2 = b == 0 ? 2 : b - 1;
        const double h11 = __shfl_sync(FULL_MASK, h, 3 * a1 + b1), h22 = __shfl_sync(FULL_MASK, h, 3 * a2 + b2);
        const double h12 = __shfl_sync(FULL_MASK, h, 3 * a1 + b2), h21 = __shfl_sync(FULL_MASK, h, 3 * a2 + b1);
        if (lane < 9)
            cof = h11 * h22 - h12 * h21;
    }
    const double cn2 = warp_sum_f64(cof * cof);
    if (sqrt(cn2) <= 1e-12 * hn2)
        return false;
    {
        int ex;
        frexp(sqrt(hn2), &ex);
        h = ldexp(h, -ex);
    }

    // every lane gathers H and forms its entry of N (lanes 0..15) or of V = I
    const double Sxx = __shfl_sync(FULL_MASK, h, 0), Sxy = __shfl_sync(FULL_MASK, h, 1),
                 Sxz = __shfl_sync(FULL_MASK, h, 2), Syx = __shfl_sync(FULL_MASK, h, 3),
                 Syy = __shfl_sync(FULL_MASK, h, 4), Syz = __shfl_sync(FULL_MASK, h, 5),
                 Szx = __shfl_sync(FULL_MASK, h, 6), Szy = __shfl_sync(FULL_MASK, h, 7),
                 Szz = __shfl_sync(FULL_MASK, h, 8);
    const int ri = (lane >> 2) & 3, cj = lane & 3, base = lane & 16;
    double x;
    if (lane < 16) {
        const int lo = min(ri, cj), hi = max(ri, cj);
        if (lo == hi)
            x = lo == 0 ? Sxx + Syy + Szz : (lo == 1 ? Sxx - Syy - Szz : (lo == 2 ? Syy - Sxx - Szz : Szz - Sxx - Syy));
        else if (lo == 0)
            x = hi == 1 ? Syz - Szy : (hi == 2 ? Szx - Sxz : Sxy - Syx);
        else if (lo == 1)
            x = hi == 2 ? Sxy + Syx : Szx + Sxz;
        else
            x = Syz + Szy;
    } else {
        x = ri == cj ? 1.0 : 0.0;
    }

    // cyclic Jacobi sweeps until the off-diagonal part of N is negligible
#pragma unroll 1
    for (int sweep = 0; sweep < 12; ++sweep) {
        const double od = (lane < 16 && ri != cj) ? x * x : 0.0;
        const double dg = (lane < 16 && ri == cj) ? x * x : 0.0;
        const double off2 = warp_sum_f64(od), diag2 = warp_sum_f64(dg);
        if (off2 <= 1e-34 * (off2 + diag2))
            break;
#pragma unroll 1
        for (int pq = 0; pq < 6; ++pq) {
            const int p = pq < 3 ? 0 : (pq < 5 ? 1 : 2);
            const int q = pq < 3 ? pq + 1 : (pq < 5 ? pq - 1 : 3);
            const double app = __shfl_sync(FULL_MASK, x, 5 * p), aqq = __shfl_sync(FULL_MASK, x, 5 * q);
            const double apq = __shfl_sync(FULL_MASK, x, 4 * p + q);
            if (apq == 0.0)
                continue;   // the same decision on every lane
            const double th = (aqq - app) / (2.0 * apq);
            const double t = fabs(th) > 1e150 ? 0.5 / th : copysign(1.0, th) / (fabs(th) + sqrt(fma(th, th, 1.0)));
            const double cs = rsqrt(fma(t, t, 1.0)), sn = t * cs;
            // right multiplication (A and V): columns p and q
            const int jp = cj == p ? q : (cj == q ? p : cj);
            double y = __shfl_sync(FULL_MASK, x, base + 4 * ri + jp);
            if (cj == p)
                x = cs * x - sn * y;
            else if (cj == q)
                x = sn * y + cs * x;
            // left multiplication (A only): rows p and q
            const int ip = ri == p ? q : (ri == q ? p : ri);
            y = __shfl_sync(FULL_MASK, x, base + 4 * ip + cj);
            if (lane < 16) {
                if (ri == p)
                    x = cs * x - sn * y;
                else if (ri == q)
                    x = sn * y + cs * x;
                if (lane == 4 * p + q || lane == 4 * q + p)
                    x = 0.0;
            }
        }
    }

    // the eigenvector of the largest eigenvalue (lowest index on ties)
    int k = 0;
    {
        double best = __shfl_sync(FULL_MASK, x, 0);
#pragma unroll
        for (int d = 1; d < 4; ++d) {
            const double v = __shfl_sync(FULL_MASK, x, 5 * d);
            if (v > best) {
                best = v;
                k = d;
            }
        }
    }
    const double qw = __shfl_sync(FULL_MASK, x, 16 + k), qx = __shfl_sync(FULL_MASK, x, 20 + k);
    const double qy = __shfl_sync(FULL_MASK, x, 24 + k), qz = __shfl_sync(FULL_MASK, x, 28 + k);
    const double inv_n = 1.0 / (qw * qw + qx * qx + qy * qy + qz * qz);

    // row ar of [R | t] on lane 4 ar + column (lanes 0..11)
    const int ar = lane < 12 ? lane >> 2 : 0;
    double r0, r1, r2;
    if (ar == 0) {
        r0 = qw * qw + qx * qx - qy * qy - qz * qz;
        r1 = 2.0 * (qx * qy - qw * qz);
        r2 = 2.0 * (qx * qz + qw * qy);
    } else if (ar == 1) {
        r0 = 2.0 * (qx * qy + qw * qz);
        r1 = qw * qw - qx * qx + qy * qy - qz * qz;
        r2 = 2.0 * (qy * qz - qw * qx);
    } else {
        r0 = 2.0 * (qx * qz - qw * qy);
        r1 = 2.0 * (qy * qz + qw * qx);
        r2 = qw * qw - qx * qx - qy * qy + qz * qz;
    }
    r0 *= inv_n;
    r1 *= inv_n;
    r2 *= inv_n;
    const double sb0 = s_tot[0] * invM + c.x, sb1 = s_tot[1] * invM + c.y, sb2 = s_tot[2] * invM + c.z;
    const double ca = ar == 0 ? c.x : (ar == 1 ? c.y : c.z);
    const double tr = (s_tot[3 + ar] * invM + ca) - (r0 * sb0 + r1 * sb1 + r2 * sb2);
    double pnew = 0.0;
    if (lane < 12)
        pnew = r0 * P0 + r1 * P1 + r2 * P2 + tr * P3;
    __syncwarp();
    if (lane < 12)
        pose[lane] = pnew;
    return true;
}

}  // namespace vicp
