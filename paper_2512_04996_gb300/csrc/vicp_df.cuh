// vicp_df.cuh -- double-float arithmetic and the rigid solve of Eq. 1
// (Horn's closed form), shared by the single-pair reduction kernel and the
// batched iteration kernel.
//
// GB300 runs FP64 at a small fraction of its FP32 rate: a dependent chain of
// FP64 operations on one thread costs tens of cycles per operation.  The
// reduction and the solve therefore run in double-float arithmetic on the
// FP32 pipes (a value is the unevaluated sum hi + lo of two floats, about 48
// significant bits); only the final pose composition, spread over twelve
// lanes, and the RMSE test use FP64.
#pragma once

#include "vicp_device.cuh"

namespace vicp {

// ---------------------------------------------------------------------------
// Double-float arithmetic from error-free transformations:
//   two_sum(a, b)       = (s, e) with s + e == a + b exactly (Knuth),
//   quick_two_sum(a, b) the same when |a| >= |b| (Dekker),
//   two_prod(a, b)      = (p, e) with p + e == a * b exactly (one FMA).
// df_acc is the short addition used to accumulate many terms (its error is a
// small multiple of 2^-46 of the magnitudes added); df_add is the accurate
// addition of Shewchuk / Bailey (both low parts summed exactly as well),
// used wherever cancellation can occur.  df_div refines the float quotient
// twice and df_sqrt the float square root once by Newton's method.
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

__device__ __forceinline__ dfl two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ dfl df_acc(dfl x, dfl y)
{
    const dfl s = two_sum(x.hi, y.hi);
    return quick_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

__device__ __forceinline__ dfl df_add(dfl x, dfl y)
{
    dfl s = two_sum(x.hi, y.hi);
    const dfl t = two_sum(x.lo, y.lo);
    s = quick_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return quick_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}

__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dfl df_sub(dfl x, dfl y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ dfl df_f(float x) { return {x, 0.0f}; }

// (x.hi + x.lo) * (y.hi + y.lo), the lo * lo term (2^-48 relative) dropped
__device__ __forceinline__ dfl df_mul(dfl x, dfl y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return quick_two_sum(p, e);
}

__device__ __forceinline__ dfl df_mul_f(dfl x, float y)
{
    const float p = __fmul_rn(x.hi, y);
    float e = __fmaf_rn(x.hi, y, -p);
    e = __fmaf_rn(x.lo, y, e);
    return quick_two_sum(p, e);
}

__device__ __forceinline__ dfl df_div(dfl a, dfl b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    dfl r = df_sub(a, df_mul_f(b, q1));
    const float q2 = __fdiv_rn(r.hi, b.hi);
    r = df_sub(r, df_mul_f(b, q2));
    const float q3 = __fdiv_rn(r.hi, b.hi);
    return df_add(quick_two_sum(q1, q2), df_f(q3));
}

__device__ __forceinline__ dfl df_sqrt(dfl a)
{
    if (!(a.hi > 0.0f))
        return {0.0f, 0.0f};
    const float s = __fsqrt_rn(a.hi);
    const dfl r = df_sub(a, two_prod(s, s));
    return quick_two_sum(s, __fdiv_rn(r.hi, __fmul_rn(2.0f, s)));
}

__device__ __forceinline__ dfl df_scale(dfl x, float pow2) { return {x.hi * pow2, x.lo * pow2}; }   // exact
__device__ __forceinline__ bool df_lt0(dfl x) { return x.hi < 0.0f; }
__device__ __forceinline__ dfl df_abs(dfl x) { return x.hi < 0.0f ? df_neg(x) : x; }
__device__ __forceinline__ double df_to_double(dfl x) { return (double)x.hi + (double)x.lo; }

__device__ __forceinline__ dfl df_shfl_xor(dfl v, int o)
{
    return {__shfl_xor_sync(FULL_MASK, v.hi, o), __shfl_xor_sync(FULL_MASK, v.lo, o)};
}

__device__ __forceinline__ dfl det3(dfl a, dfl b, dfl c, dfl d, dfl e, dfl f, dfl g, dfl h, dfl i)
{
    const dfl m0 = df_sub(df_mul(e, i), df_mul(f, h));
    const dfl m1 = df_sub(df_mul(d, i), df_mul(f, g));
    const dfl m2 = df_sub(df_mul(d, h), df_mul(e, g));
    return df_add(df_sub(df_mul(a, m0), df_mul(b, m1)), df_mul(c, m2));
}

// Rows (columns) other than k of a 4x4 matrix, ascending.
__device__ __forceinline__ void others(int k, int &i0, int &i1, int &i2)
{
    i0 = k == 0 ? 1 : 0;
    i1 = k <= 1 ? 2 : 1;
    i2 = k <= 2 ? 3 : 2;
}

// Cofactor C_ij = (-1)^(i+j) det(A without row i and column j) of a 4x4
// double-float matrix in shared memory.  Not inlined: the solve evaluates it
// on several lanes at once and several times, from one copy of the code.
static __device__ __noinline__ dfl cofactor4(const dfl *A, int i, int j)
{
    int r0, r1, r2, c0, c1, c2;
    others(i, r0, r1, r2);
    others(j, c0, c1, c2);
    const dfl d = det3(A[4 * r0 + c0], A[4 * r0 + c1], A[4 * r0 + c2], A[4 * r1 + c0], A[4 * r1 + c1],
                       A[4 * r1 + c2], A[4 * r2 + c0], A[4 * r2 + c1], A[4 * r2 + c2]);
    return ((i + j) & 1) ? df_neg(d) : d;
}

__device__ __forceinline__ dfl warp_sum_df(dfl v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = df_add(v, df_shfl_xor(v, o));
    return v;
}

// rank(S) < 2: every 2x2 minor negligible against |S|_F^2 (a definition
// shared with the oracle, not its code): |cof(S)|_F <= 1e-12 |S|_F^2,
// tested as |cof(S)|_F^2 <= 1e-24 |S|_F^4 on S normalised to |S|_F ~ 1.
// Lanes 0..8 take one minor each; every lane of the warp must call it.
static __device__ bool rank_below_two(const dfl S[9], dfl s2)
{
    const int lane = threadIdx.x & 31;
    dfl sq = {0.0f, 0.0f};
    if (lane < 9) {
        const int i = lane / 3, j = lane % 3;
        const int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
        const dfl cf = df_sub(df_mul(S[3 * i1 + j1], S[3 * i2 + j2]), df_mul(S[3 * i1 + j2], S[3 * i2 + j1]));
        sq = df_mul(cf, cf);
    }
    const dfl c2 = warp_sum_df(sq);
    return c2.hi <= 1e-24f * (s2.hi * s2.hi);
}

// Horn's closed form, evaluated by one warp.  With S the 3x3 cross-covariance
// sum (s - sbar)(q - qbar)^T, the rotation minimising Eq. 1 is the unit
// quaternion (w, x, y, z) of the largest eigenvalue of the symmetric,
// traceless 4x4
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
// largest diagonal cofactor is used.  S and E come in scaled by one power of
// two (|S|_F ~ 1), which changes neither the rotation nor any rounding.
// Every lane of the warp must call it; sM is 16 double-floats of shared
// memory.  R is returned on every lane.
static __device__ void horn_rotation(const dfl S[9], dfl s2, dfl E, dfl R[9], dfl *sM)
{
    const int lane = threadIdx.x & 31;
    const dfl sxx = S[0], sxy = S[1], sxz = S[2], syx = S[3], syy = S[4], syz = S[5], szx = S[6], szy = S[7],
              szz = S[8];
    const dfl n00 = df_add(df_add(sxx, syy), szz);
    if (lane == 0) {
        sM[0] = n00;
        sM[5] = df_sub(df_sub(sxx, syy), szz);
        sM[10] = df_sub(df_sub(syy, sxx), szz);
        sM[15] = df_sub(df_sub(szz, sxx), syy);
        sM[1] = sM[4] = df_sub(syz, szy);
        sM[2] = sM[8] = df_sub(szx, sxz);
        sM[3] = sM[12] = df_sub(sxy, syx);
        sM[6] = sM[9] = df_add(sxy, syx);
        sM[7] = sM[13] = df_add(szx, sxz);
        sM[11] = sM[14] = df_add(syz, szy);
    }
    __syncwarp();
    const dfl c2 = df_scale(s2, -2.0f);
    const dfl c1 = df_scale(det3(sxx, sxy, sxz, syx, syy, syz, szx, szy, szz), -8.0f);
    // det N along row 0: lanes 0..3 take one term each
    dfl term = {0.0f, 0.0f};
    if (lane < 4)
        term = df_mul(sM[lane], cofactor4(sM, 0, lane));
    const dfl c0 = warp_sum_df(term);

    auto poly = [&](dfl l) { return df_add(df_mul(df_add(df_mul(df_add(df_mul(l, l), c2), l), c1), l), c0); };
    dfl l = df_add(df_scale(E, 0.5f), n00);
    l = df_add(l, df_mul_f(df_abs(l), 1e-12f));
    const dfl loose = df_sqrt(df_mul_f(s2, 3.0f));   // l_max <= sqrt(3/4 tr N^2) = sqrt(3) |S|_F
    if (!(l.hi > 0.0f) || df_lt0(poly(l)) || df_lt0(df_sub(loose, l)))
        l = loose;
    // Newton in float first (short dependency chains), from the same start;
    // its root seeds the double-float iteration when it stays in (0, l]
    {
        const float f2 = c2.hi, f1 = c1.hi, f0 = c0.hi;
        float lf = l.hi;
#pragma unroll 1
        for (int it = 0; it < 32; ++it) {
            const float P = __fmaf_rn(__fmaf_rn(__fmaf_rn(lf, lf, f2), lf, f1), lf, f0);
            const float dP = __fmaf_rn(__fmaf_rn(4.0f * lf, lf, 2.0f * f2), lf, f1);
            if (!(dP != 0.0f))
                break;
            const float step = __fdiv_rn(P, dP);
            lf -= step;
            if (fabsf(step) <= 1e-6f * fabsf(lf))
                break;
        }
        if (lf > 0.0f && lf <= l.hi && isfinite(lf))
            l = df_f(lf);
    }
#pragma unroll 1
    for (int it = 0; it < 64; ++it) {
        const dfl P = poly(l);
        const dfl dP = df_add(df_mul(df_add(df_scale(df_mul(l, l), 4.0f), df_scale(c2, 2.0f)), l), c1);
        if (!(dP.hi != 0.0f))
            break;
        const dfl step = df_div(P, dP);
        l = df_sub(l, step);
        if (fabsf(step.hi) <= 1e-13f * fabsf(l.hi))
            break;
    }
    // adjugate of A = N - l I (symmetric), in place of N
    __syncwarp();
    if (lane < 16 && (lane % 5) == 0)
        sM[lane] = df_sub(sM[lane], l);
    __syncwarp();
    // the column of the largest diagonal cofactor (lowest index on ties)
    dfl ckk = {0.0f, 0.0f};
    if (lane < 4)
        ckk = cofactor4(sM, lane, lane);
    unsigned long long key = lane < 4 ? ((unsigned long long)__float_as_uint(fabsf(ckk.hi)) << 32) | (unsigned)(3 - lane)
                                      : 0ull;
#pragma unroll
    for (int o = 2; o > 0; o >>= 1) {
        const unsigned long long y = __shfl_xor_sync(FULL_MASK, key, o);
        key = y > key ? y : key;
    }
    const int col = 3 - (int)(unsigned)__shfl_sync(FULL_MASK, key, 0);
    dfl vi = {0.0f, 0.0f};
    if (lane < 4)
        vi = lane == col ? ckk : cofactor4(sM, lane, col);
    dfl v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        v[k] = {__shfl_sync(FULL_MASK, vi.hi, k), __shfl_sync(FULL_MASK, vi.lo, k)};
    // the cofactors scale like l^3: bring them to ~1 by a power of two first
    int ex;
    frexpf(fmaxf(fmaxf(fabsf(v[0].hi), fabsf(v[1].hi)), fmaxf(fabsf(v[2].hi), fabsf(v[3].hi))), &ex);
    const float sc = ldexpf(1.0f, -ex);
#pragma unroll
    for (int k = 0; k < 4; ++k)
        v[k] = df_scale(v[k], sc);
    dfl nv = df_mul(v[0], v[0]);
    nv = df_add(nv, df_mul(v[1], v[1]));
    nv = df_add(nv, df_mul(v[2], v[2]));
    nv = df_add(nv, df_mul(v[3], v[3]));
    const dfl inv = df_div(df_f(1.0f), df_sqrt(nv));
    const dfl w = df_mul(v[0], inv), x = df_mul(v[1], inv), y = df_mul(v[2], inv), z = df_mul(v[3], inv);
    const dfl ww = df_mul(w, w), xx = df_mul(x, x), yy = df_mul(y, y), zz = df_mul(z, z);
    const dfl xy = df_mul(x, y), xz = df_mul(x, z), yz = df_mul(y, z), wx = df_mul(w, x), wy = df_mul(w, y),
              wz = df_mul(w, z);
    R[0] = df_sub(df_add(ww, xx), df_add(yy, zz));
    R[1] = df_scale(df_sub(xy, wz), 2.0f);
    R[2] = df_scale(df_add(xz, wy), 2.0f);
    R[3] = df_scale(df_add(xy, wz), 2.0f);
    R[4] = df_sub(df_add(ww, yy), df_add(xx, zz));
    R[5] = df_scale(df_sub(yz, wx), 2.0f);
    R[6] = df_scale(df_sub(xz, wy), 2.0f);
    R[7] = df_scale(df_add(yz, wx), 2.0f);
    R[8] = df_sub(df_add(ww, zz), df_add(xx, yy));
}

// The 16 sums of one ICP iteration, relative to a fixed centre c (s - c is
// then exact as a double-float):
//   [0..2]  sum (s - c)          [3..5]  sum (q - c)
//   [6..14] sum (s - c)(q - c)^T [15]    sum |s - q|^2
constexpr int N_SUMS = 16;

// Adds the correspondence (s, q) -- s the transformed source point, q its
// target point -- to the sums.
__device__ __forceinline__ void accumulate_corr(dfl (&acc)[N_SUMS], float3 s, float4 q, float3 cf)
{
    const dfl sv[3] = {two_sum(s.x, -cf.x), two_sum(s.y, -cf.y), two_sum(s.z, -cf.z)};
    const dfl qv[3] = {two_sum(q.x, -cf.x), two_sum(q.y, -cf.y), two_sum(q.z, -cf.z)};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        acc[a] = df_acc(acc[a], sv[a]);
        acc[3 + a] = df_acc(acc[3 + a], qv[a]);
#pragma unroll
        for (int b = 0; b < 3; ++b)
            acc[6 + 3 * a + b] = df_acc(acc[6 + 3 * a + b], df_mul(sv[a], qv[b]));
    }
    const dfl ex = two_sum(s.x, -q.x), ey = two_sum(s.y, -q.y), ez = two_sum(s.z, -q.z);
    acc[15] = df_acc(acc[15], df_acc(df_acc(df_mul(ex, ex), df_mul(ey, ey)), df_mul(ez, ez)));
}

// The rigid update of Eq. 1 from the sums s_tot (shared memory) of m
// correspondences, by one warp: its lanes share the scalar work and split
// the minors and cofactors; the update dT (3x4, double-float) goes through
// shared memory to lanes 0..11, which compose it with the pose in FP64:
// pose <- dT * pose.  Returns false, leaving the pose untouched, when the
// geometry is degenerate (rank(H) < 2).  rmse = the RMSE of the m
// correspondences, on every lane.  s_M (16) and s_dT (12) are shared memory.
// Every lane of the warp must call it.
static __device__ bool solve_update(const dfl *s_tot, int m, float3 cf, double *pose, dfl *s_M, dfl *s_dT,
                                    double &rmse)
{
    const int lane = threadIdx.x & 31;
    dfl S[N_SUMS];
#pragma unroll
    for (int q = 0; q < N_SUMS; ++q)
        S[q] = s_tot[q];
    const float mh = (float)m;
    const dfl M = {mh, (float)((long long)m - (long long)mh)};
    const dfl invM = df_div(df_f(1.0f), M);
    dfl pb[3], qb[3];   // centroids relative to c
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        pb[a] = df_mul(S[a], invM);
        qb[a] = df_mul(S[3 + a], invM);
    }
    // sum (s - sbar)(q - qbar)^T = sum (s - c)(q - c)^T - sbar_c * sum (q - c)^T,
    // entry `lane` on lanes 0..8, then shared by shuffles; its squares summed
    dfl h = {0.0f, 0.0f}, h2 = {0.0f, 0.0f}, e = {0.0f, 0.0f};
    if (lane < 9) {
        const int a = lane / 3, b = lane % 3;
        h = df_sub(s_tot[6 + lane], df_mul(df_mul(s_tot[a], invM), s_tot[3 + b]));
        h2 = df_mul(h, h);
    }
    dfl H[9];
#pragma unroll
    for (int k = 0; k < 9; ++k)
        H[k] = {__shfl_sync(FULL_MASK, h.hi, k), __shfl_sync(FULL_MASK, h.lo, k)};
    dfl s2 = warp_sum_df(h2);
    rmse = df_to_double(df_sqrt(df_mul(S[15], invM)));
    // centred residual E = sum |s - q|^2 - M |sbar - qbar|^2 (a term per lane 0..2)
    if (lane < 3) {
        const dfl sum_s = s_tot[lane], sum_q = s_tot[3 + lane];
        e = df_mul(df_sub(df_mul(sum_s, invM), df_mul(sum_q, invM)), df_sub(sum_s, sum_q));
    }
    dfl E = df_sub(S[15], warp_sum_df(e));
    bool ok = s2.hi > 0.0f && isfinite(s2.hi);
    if (ok) {
        int ex;
        frexpf(__fsqrt_rn(s2.hi), &ex);
        const float sc = ldexpf(1.0f, -ex);
#pragma unroll
        for (int k = 0; k < 9; ++k)
            H[k] = df_scale(H[k], sc);
        s2 = df_scale(s2, sc * sc);
        E = df_scale(E, sc);
        ok = !rank_below_two(H, s2);
    }
    if (!ok)
        return false;
    dfl R[9];
    horn_rotation(H, s2, E, R, s_M);
    // translation qa - R pa, row `lane` on lanes 0..2
    if (lane < 3) {
        const int a = lane;
        const dfl pa0 = df_add(pb[0], df_f(cf.x)), pa1 = df_add(pb[1], df_f(cf.y)), pa2 = df_add(pb[2], df_f(cf.z));
        const float ca = a == 0 ? cf.x : (a == 1 ? cf.y : cf.z);
        const dfl Ra0 = a == 0 ? R[0] : (a == 1 ? R[3] : R[6]);
        const dfl Ra1 = a == 0 ? R[1] : (a == 1 ? R[4] : R[7]);
        const dfl Ra2 = a == 0 ? R[2] : (a == 1 ? R[5] : R[8]);
        dfl r = df_mul(Ra0, pa0);
        r = df_add(r, df_mul(Ra1, pa1));
        r = df_add(r, df_mul(Ra2, pa2));
        const dfl qa = df_add(a == 0 ? qb[0] : (a == 1 ? qb[1] : qb[2]), df_f(ca));
        s_dT[4 * a + 0] = Ra0;
        s_dT[4 * a + 1] = Ra1;
        s_dT[4 * a + 2] = Ra2;
        s_dT[4 * a + 3] = df_sub(qa, r);
    }
    __syncwarp();
    // pose <- dT * pose: lane 4a + b computes entry (a, b)
    double pnew = 0.0;
    if (lane < 12) {
        const int a = lane >> 2, b = lane & 3;
        const double d0 = df_to_double(s_dT[4 * a]), d1 = df_to_double(s_dT[4 * a + 1]);
        const double d2 = df_to_double(s_dT[4 * a + 2]), d3 = df_to_double(s_dT[4 * a + 3]);
        pnew = d0 * pose[b] + d1 * pose[4 + b] + d2 * pose[8 + b] + d3 * pose[12 + b];
    }
    __syncwarp();
    if (lane < 12)
        pose[lane] = pnew;
    return true;
}

}  // namespace vicp
