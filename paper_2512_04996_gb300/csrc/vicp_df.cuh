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

__device__ __forceinline__ dfl df_shfl(dfl v, int src)
{
    return {__shfl_sync(FULL_MASK, v.hi, src), __shfl_sync(FULL_MASK, v.lo, src)};
}

// 1 / x: the correctly rounded float reciprocal q, corrected once from the
// residual 1 - x q (its x.hi part is exact in one FMA).
__device__ __forceinline__ dfl df_rcp(dfl x)
{
    const float q = __frcp_rn(x.hi);
    const float r = __fmaf_rn(-x.lo, q, __fmaf_rn(-x.hi, q, 1.0f));
    return quick_two_sum(q, __fmul_rn(r, q));
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

// Sums over the warp (xor butterfly: every lane gets the same total, since
// df_add is commutative bit for bit).
__device__ __forceinline__ dfl warp_sum_df(dfl v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1)
        v = df_add(v, df_shfl_xor(v, o));
    return v;
}

__device__ __forceinline__ void warp_sum_df2(dfl &a, dfl &b)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const dfl ya = df_shfl_xor(a, o), yb = df_shfl_xor(b, o);
        a = df_add(a, ya);
        b = df_add(b, yb);
    }
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

// ---------------------------------------------------------------------------
// The rigid update of Eq. 1 from the sums s_tot (shared memory) of m
// correspondences, by one warp, every lane holding one entry of the
// matrices involved so that the whole solve is one short stream of
// instructions (a solve is latency-bound, and its code is fetched cold once
// per iteration):
//  * lanes 0..8: H = sum (s - sbar)(q - qbar)^T, entry (k / 3, k % 3), and
//    its cofactors (rank test, det H); H, |H|_F^2 and the centred residual E
//    are scaled by one power of two to |H|_F ~ 1, which changes neither the
//    rotation nor any rounding.
//  * Horn's closed form: the rotation minimising Eq. 1 is the unit
//    quaternion (w, x, y, z) of the largest eigenvalue of the symmetric,
//    traceless 4x4
//      [ Sxx+Syy+Szz  Syz-Szy      Szx-Sxz      Sxy-Syx     ]
//      [ Syz-Szy      Sxx-Syy-Szz  Sxy+Syx      Szx+Sxz     ]
//      [ Szx-Sxz      Sxy+Syx     -Sxx+Syy-Szz  Syz+Szy     ]
//      [ Sxy-Syx      Szx+Sxz      Syz+Szy     -Sxx-Syy+Szz ]
//    (S = H), entry (k / 4, k % 4) on lane k < 16.  Its characteristic
//    polynomial is l^4 + c2 l^2 + c1 l + c0, c2 = -2 |S|_F^2, c1 = -8 det S,
//    c0 = det N (Laplace expansion over the 2x2 minors of rows 0-1 and 2-3,
//    one column pair per lane).  The largest root: Newton's method from the
//    upper bound (Ga + Gb) / 2 = E/2 + tr S, which lies just right of it
//    (from the right of the largest root of a real-rooted polynomial Newton
//    decreases monotonically onto it), in float, then polished in
//    double-float (the polynomial in double-float, the derivative in float:
//    each step gains the float precision again).
//  * The eigenvector: a column of the adjugate of N - l I (rank one at a
//    simple eigenvalue), all sixteen cofactors at once (lane k: cofactor
//    (k / 4, k % 4)), the column of the largest diagonal cofactor taken.
//  * R from the unnormalised quaternion q = (w, v), n = |q|^2:
//    R_aa = (2 (w^2 + v_a^2) - n) / n, R_ab = 2 (v_a v_b - e_abc w v_c) / n.
//  * t = qbar - R sbar, and lanes 0..11 compose pose <- dT * pose in FP64
//    (lane 4a + b: entry (a, b)).
// Returns false, leaving the pose untouched, when the geometry is degenerate
// (rank(H) < 2).  rmse = the RMSE of the m correspondences, on every lane.
// Every lane of the warp must call it.  Not inlined: one copy of its code
// per kernel, which the single-pair kernel fetches ahead of the real solve.
// ---------------------------------------------------------------------------
static __device__ __noinline__ bool solve_update(const dfl *s_tot, int m, float3 cf, double *pose, double &rmse)
{
    const int lane = threadIdx.x & 31;
    // the pose column this lane composes, loaded first
    const int pc = lane & 3;
    double P0 = 0.0, P1 = 0.0, P2 = 0.0, P3 = 0.0;
    if (lane < 12) {
        P0 = pose[pc];
        P1 = pose[4 + pc];
        P2 = pose[8 + pc];
        P3 = pose[12 + pc];
    }
    const float mh = (float)m;
    const dfl invM = df_rcp(dfl{mh, (float)((long long)m - (long long)mh)});

    // H entry (a, b) on lane 3a + b < 9:
    //   sum (s - c)_a (q - c)_b - (sum (s - c)_a)(sum (q - c)_b) / M;
    // lanes 0..2: the centring term (sum (s - q)_a)^2 / M of the residual
    const int a = lane < 9 ? lane / 3 : 0, b = lane < 9 ? lane - 3 * a : 0;
    dfl h = {0.0f, 0.0f}, e = {0.0f, 0.0f};
    if (lane < 9)
        h = df_sub(s_tot[6 + lane], df_mul(df_mul(s_tot[a], invM), s_tot[3 + b]));
    if (lane < 3) {
        const dfl d = df_sub(s_tot[lane], s_tot[3 + lane]);
        e = df_mul(df_mul(d, invM), d);
    }
    dfl s2 = df_mul(h, h);
    warp_sum_df2(s2, e);
    const dfl S15 = s_tot[15];
    rmse = df_to_double(df_sqrt(df_mul(S15, invM)));
    dfl E = df_sub(S15, e);
    if (!(s2.hi > 0.0f) || !isfinite(s2.hi))
        return false;
    {
        int ex;
        frexpf(__fsqrt_rn(s2.hi), &ex);
        const float sc = ldexpf(1.0f, -ex);
        h = df_scale(h, sc);
        s2 = df_scale(s2, sc * sc);
        E = df_scale(E, sc);
    }

    // cofactors of H (cyclic index order gives the sign), the rank test and
    // det H = sum_b H_0b C_0b
    dfl cof = {0.0f, 0.0f}, dH = {0.0f, 0.0f};
    {
        const int a1 = a == 2 ? 0 : a + 1, a2 = a == 0 ? 2 : a - 1;
        const int b1 = b == 2 ? 0 : b + 1, b2 = b == 0 ? 2 : b - 1;
        const dfl h11 = df_shfl(h, 3 * a1 + b1), h22 = df_shfl(h, 3 * a2 + b2);
        const dfl h12 = df_shfl(h, 3 * a1 + b2), h21 = df_shfl(h, 3 * a2 + b1);
        if (lane < 9) {
            cof = df_sub(df_mul(h11, h22), df_mul(h12, h21));
            if (lane < 3)
                dH = df_mul(h, cof);
        }
    }
    dfl c2s = df_mul(cof, cof);
    warp_sum_df2(c2s, dH);
    // rank(H) < 2: every 2x2 minor negligible against |H|_F^2 (a definition
    // shared with the oracle, not its code): |cof(H)|_F <= 1e-12 |H|_F^2
    if (c2s.hi <= 1e-24f * (s2.hi * s2.hi))
        return false;

    // N entry (ni, nj) on lane 4 ni + nj (lanes 16..31 repeat lanes 0..15):
    // a signed sum of two or three entries of H
    const int ni = (lane >> 2) & 3, nj = lane & 3;
    dfl nv;
    {
        const int i0 = min(ni, nj), j0 = max(ni, nj);
        int u0 = 0, u1 = 4, u2 = 8;
        float g0 = 1.0f, g1 = 1.0f, g2 = 0.0f;
        if (i0 == j0) {   // +-Sxx +-Syy +-Szz
            g0 = (i0 == 0 || i0 == 1) ? 1.0f : -1.0f;
            g1 = (i0 == 0 || i0 == 2) ? 1.0f : -1.0f;
            g2 = (i0 == 0 || i0 == 3) ? 1.0f : -1.0f;
        } else {          // (0,1) Syz-Szy, (0,2) Szx-Sxz, (0,3) Sxy-Syx; (2,3), (1,3), (1,2) the same with +
            const int k = i0 == 0 ? j0 : 6 - i0 - j0;
            u0 = k == 1 ? 5 : (k == 2 ? 6 : 1);
            u1 = k == 1 ? 7 : (k == 2 ? 2 : 3);
            g1 = i0 == 0 ? -1.0f : 1.0f;
        }
        const dfl v0 = df_shfl(h, u0), v1 = df_shfl(h, u1), v2 = df_shfl(h, u2);
        nv = df_add(df_add(df_scale(v0, g0), df_scale(v1, g1)), df_scale(v2, g2));
    }

    // c0 = det N = sum over column pairs (p, q) of rows 0-1 of
    // (-1)^(1+p+q) det N[01, pq] det N[23, rs], (r, s) the other two columns
    dfl c0;
    {
        const int t = lane < 6 ? lane : 0;
        const int p = t < 3 ? 0 : (t < 5 ? 1 : 2);
        const int q = t < 3 ? t + 1 : (t < 5 ? t - 1 : 3);
        const unsigned rest = 15u & ~((1u << p) | (1u << q));
        const int r = __ffs(rest) - 1, s = 31 - __clz(rest);
        const dfl x0p = df_shfl(nv, p), x1q = df_shfl(nv, 4 + q), x0q = df_shfl(nv, q), x1p = df_shfl(nv, 4 + p);
        const dfl x2r = df_shfl(nv, 8 + r), x3s = df_shfl(nv, 12 + s), x2s = df_shfl(nv, 8 + s),
                  x3r = df_shfl(nv, 12 + r);
        c0 = {0.0f, 0.0f};
        if (lane < 6) {
            const dfl top = df_sub(df_mul(x0p, x1q), df_mul(x0q, x1p));
            const dfl bot = df_sub(df_mul(x2r, x3s), df_mul(x2s, x3r));
            c0 = df_mul(top, bot);
            if (t == 1 || t == 4)
                c0 = df_neg(c0);
        }
        c0 = warp_sum_df(c0);
    }
    const dfl c2 = df_scale(s2, -2.0f);
    const dfl c1 = df_scale(dH, -8.0f);

    // the largest root
    auto poly = [&](dfl l) { return df_add(df_mul(df_add(df_mul(df_add(df_mul(l, l), c2), l), c1), l), c0); };
    dfl l = df_add(df_scale(E, 0.5f), df_shfl(nv, 0));
    l = df_add(l, df_mul_f(df_abs(l), 1e-12f));
    const dfl loose = df_sqrt(df_mul_f(s2, 3.0f));   // l_max <= sqrt(3/4 tr N^2) = sqrt(3) |S|_F
    if (!(l.hi > 0.0f) || df_lt0(poly(l)) || df_lt0(df_sub(loose, l)))
        l = loose;
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
    for (int it = 0; it < 8; ++it) {
        const dfl P = poly(l);
        const float lf = l.hi;
        const float dP = __fmaf_rn(__fmaf_rn(4.0f * lf, lf, 2.0f * c2.hi), lf, c1.hi);
        if (!(dP != 0.0f))
            break;
        const float step = __fdiv_rn(P.hi, dP);
        l = df_add(l, df_f(-step));
        if (fabsf(step) <= 1e-13f * fabsf(l.hi))
            break;
    }

    // cofactor (ni, nj) of A = N - l I, from the other rows and columns
    dfl ca;
    {
        const dfl av = ni == nj ? df_sub(nv, l) : nv;
        int r0, r1, r2, k0, k1, k2;
        others(ni, r0, r1, r2);
        others(nj, k0, k1, k2);
        ca = det3(df_shfl(av, 4 * r0 + k0), df_shfl(av, 4 * r0 + k1), df_shfl(av, 4 * r0 + k2),
                  df_shfl(av, 4 * r1 + k0), df_shfl(av, 4 * r1 + k1), df_shfl(av, 4 * r1 + k2),
                  df_shfl(av, 4 * r2 + k0), df_shfl(av, 4 * r2 + k1), df_shfl(av, 4 * r2 + k2));
        if ((ni + nj) & 1)
            ca = df_neg(ca);
    }
    // the column of the largest diagonal cofactor (lowest index on ties)
    int col = 0;
    {
        float best = fabsf(__shfl_sync(FULL_MASK, ca.hi, 0));
#pragma unroll
        for (int k = 1; k < 4; ++k) {
            const float x = fabsf(__shfl_sync(FULL_MASK, ca.hi, 5 * k));
            if (x > best) {
                best = x;
                col = k;
            }
        }
    }
    dfl v[4];
#pragma unroll
    for (int k = 0; k < 4; ++k)
        v[k] = df_shfl(ca, 4 * k + col);
    // the cofactors scale like l^3: bring them to ~1 by a power of two first
    {
        int ev;
        frexpf(fmaxf(fmaxf(fabsf(v[0].hi), fabsf(v[1].hi)), fmaxf(fabsf(v[2].hi), fabsf(v[3].hi))), &ev);
        const float sc = ldexpf(1.0f, -ev);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            v[k] = df_scale(v[k], sc);
    }
    const dfl nq = df_add(df_add(df_mul(v[0], v[0]), df_mul(v[1], v[1])), df_add(df_mul(v[2], v[2]), df_mul(v[3], v[3])));
    const dfl inv_nq = df_rcp(nq);

    // R entry (a, b) on lane 3a + b < 9, and its product with sbar_b + c_b
    const dfl qa = a == 0 ? v[1] : (a == 1 ? v[2] : v[3]);
    dfl rab;
    if (a == b) {
        rab = df_sub(df_scale(df_add(df_mul(v[0], v[0]), df_mul(qa, qa)), 2.0f), nq);
    } else {
        const int c = 3 - a - b;
        const dfl qb = b == 0 ? v[1] : (b == 1 ? v[2] : v[3]);
        const dfl qc = c == 0 ? v[1] : (c == 1 ? v[2] : v[3]);
        const dfl wq = df_mul(v[0], qc);
        rab = df_scale(df_add(df_mul(qa, qb), b == (a == 2 ? 0 : a + 1) ? df_neg(wq) : wq), 2.0f);
    }
    rab = df_mul(rab, inv_nq);
    const float cb = b == 0 ? cf.x : (b == 1 ? cf.y : cf.z);
    const dfl rp = df_mul(rab, df_add(df_mul(s_tot[b], invM), df_f(cb)));

    // lane 4a' + k (< 12): row a' of dT = [R | qbar + c - R (sbar + c)]
    const int ar = lane < 12 ? lane >> 2 : 0;
    const dfl d0 = df_shfl(rab, 3 * ar), d1 = df_shfl(rab, 3 * ar + 1), d2 = df_shfl(rab, 3 * ar + 2);
    const dfl p0 = df_shfl(rp, 3 * ar), p1 = df_shfl(rp, 3 * ar + 1), p2 = df_shfl(rp, 3 * ar + 2);
    const float ca_ = ar == 0 ? cf.x : (ar == 1 ? cf.y : cf.z);
    const dfl qbar = df_add(df_mul(s_tot[3 + ar], invM), df_f(ca_));
    const dfl tr = df_sub(qbar, df_add(df_add(p0, p1), p2));
    double pnew = 0.0;
    if (lane < 12)
        pnew = df_to_double(d0) * P0 + df_to_double(d1) * P1 + df_to_double(d2) * P2 + df_to_double(tr) * P3;
    __syncwarp();
    if (lane < 12)
        pose[lane] = pnew;
    return true;
}

}  // namespace vicp
