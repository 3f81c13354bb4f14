// vicp_dilate.cuh -- device code of the dilation (Alg. 3) shared by the
// single-grid kernels and the batched build: the packed candidate words, the
// sweeps, and the per-unit passes (the design is described at the top of
// vicp_dilate.cu).
#pragma once

#include "vicp_device.cuh"

namespace vicp {

namespace dil {
constexpr int UX = 32;   // x per unit: a lane each
constexpr int UY = 32;   // output rows of a pass-XY unit
constexpr int UZ = 32;   // output planes of a pass-Z unit
constexpr int WARPS = 4, THREADS = 32 * WARPS;
constexpr unsigned NONE = 0xffffffffu;
constexpr int L_COMPACT_MAX = 15;   // 16-bit intermediate words up to this L

// Move a word n voxels (n >= 0) along one axis: the distance (at bit SD)
// grows by n and one offset field shifts by n (inc = the one-voxel step).  A
// word whose distance would exceed L becomes NONE (NONE stays NONE).
template <int SD>
__device__ __forceinline__ unsigned stepn(unsigned v, int n, unsigned inc, int L)
{
    if (n > L)
        return NONE;
    return v >= ((unsigned)(L + 1 - n) << SD) ? NONE : v + (unsigned)n * inc;
}

// Word layouts, (distance, dz, dy, dx) from the most significant field down,
// offsets biased to be non-negative.  For L <= 15 passes X and Y work on
// dist:6 | dy+15:5 | dx+15:5, stored as 16 bits (NONE truncates to 0xffff,
// distance 63), and pass Z on dist:6 | dz+31:6 | dy+15:5 | dx+15:5, made from
// the stored word by a few logic operations; the stored NONE becomes a word
// of distance 63, which no step keeps and every real word beats.  For larger
// L every pass uses dist:6 | dz+31:6 | dy+31:6 | dx+31:6.
struct Words16 {
    using Stored = unsigned short;
    static constexpr int SD = 10, SY = 5;   // passes X and Y
    static constexpr int ZD = 16, ZZ = 10;  // pass Z
    static constexpr unsigned CENTER = (15u << SY) | 15u;
    __device__ static unsigned load_z(const Stored *p, int i)
    {
        const unsigned s = __ldg(p + i);
        return ((s << 6) & 0x3f0000u) | (31u << ZZ) | (s & 0x3ffu);
    }
    // root - voxel for a pass-Z word is offset - bias (modulo 2^32)
    __device__ static unsigned offset(unsigned w, unsigned nx, unsigned plane)
    {
        return (w & 31u) + nx * ((w >> 5) & 31u) + plane * ((w >> 10) & 63u);
    }
    __device__ static unsigned bias(unsigned nx, unsigned plane) { return 15u + 15u * nx + 31u * plane; }
};
struct Words32 {
    using Stored = unsigned;
    static constexpr int SD = 18, SY = 6;
    static constexpr int ZD = 18, ZZ = 12;
    static constexpr unsigned CENTER = (31u << 12) | (31u << SY) | 31u;
    __device__ static unsigned load_z(const Stored *p, int i) { return __ldg(p + i); }
    __device__ static unsigned offset(unsigned w, unsigned nx, unsigned plane)
    {
        return (w & 63u) + nx * ((w >> 6) & 63u) + plane * ((w >> 12) & 63u);
    }
    __device__ static unsigned bias(unsigned nx, unsigned plane) { return 31u + 31u * nx + 31u * plane; }
};

// Pass X for the voxel x of a row from the row's bits around it: `left` bit i
// is x - 32 + i, `right` bit i is x + i.
template <class W>
__device__ __forceinline__ unsigned row_word(unsigned left, unsigned right, int L)
{
    if (right & 1u)
        return W::CENTER;
    if (L == 0)
        return NONE;
    const unsigned lm = left & (0xffffffffu << (32 - L));
    const unsigned rm = (right >> 1) & ((1u << L) - 1u);
    const int dl = lm ? __clz(lm) + 1 : 64;
    const int dr = rm ? __ffs(rm) : 64;
    if (dl <= dr)
        return dl <= L ? (((unsigned)dl << W::SD) | (W::CENTER - (unsigned)dl)) : NONE;
    return dr <= L ? (((unsigned)dr << W::SD) | (W::CENTER + (unsigned)dr)) : NONE;
}

// One axis of passes Y and Z on 32 output positions held in registers:
// c[k] holds the words found at position k itself; `before` and `after` are
// the best words from the halo beyond each end, already moved to positions 0
// and 31.  The result is min over i of stepn(c[i], |k - i|).  A forward and
// a backward running minimum go through the array together, each in place
// (two independent dependency chains of 31 steps instead of one of 62).
// Where a chain meets a position the other has already passed, it also
// carries that value on; every value either chain holds is the word of some
// lattice path to its position, and a path that turns pays |i - j| +
// |k - j| >= |k - i|, so the minimum at every position is still the direct
// word from the nearest candidate -- the forward chain ends each position at
// or below it for k >= 16, the backward chain for k < 16.
template <unsigned INC_FWD, unsigned INC_BWD>
__device__ __forceinline__ void sweep32(unsigned (&c)[32], unsigned before, unsigned after, unsigned lim)
{
    c[0] = min(c[0], before);
    c[31] = min(c[31], after);
    unsigned f = c[0], b = c[31];
#pragma unroll
    for (int i = 1; i < 32; ++i) {
        c[i] = min(c[i], f >= lim ? NONE : f + INC_FWD);
        f = c[i];
        c[31 - i] = min(c[31 - i], b >= lim ? NONE : b + INC_BWD);
        b = c[31 - i];
    }
}

// ---------------------------------------------------------------------------
// Passes X and Y.  Warp u = xb + nxb*(yb + nyb*z) covers x in [32xb, 32xb+32),
// y in [32yb, 32yb+32) of plane z; lane l stands for x = 32xb + l.  Lane l
// loads the occupancy bits of output row y0 + l and, for l < L, of halo rows
// y0 - L + l and y0 + 32 + l: four aligned words funnel-shifted into three
// covering x in [x0-32, x0+64), masked to the grid and to [x0-L, x0+31+L].
// A row's words are broadcast by shuffles.  rows[u] bit k is set iff output
// row y0 + k holds a label after pass Y (0 for a unit with nothing in reach,
// whose words are not written).
// ---------------------------------------------------------------------------
template <class W>
__device__ __forceinline__ void dilate_xy_unit(int u, const unsigned *__restrict__ occ, long long n_words,
                                               const GridGeom &g, int L, int nxb, int nyb,
                                               typename W::Stored *__restrict__ inter, unsigned *__restrict__ rows)
{
    constexpr unsigned STEP_YF = (1u << W::SD) - (1u << W::SY);   // moved from y-1 to y: dy -= 1
    constexpr unsigned STEP_YB = (1u << W::SD) + (1u << W::SY);   // moved from y+1 to y: dy += 1
    const int lane = threadIdx.x & 31;
    const int xb = u % nxb, q = u / nxb;
    const int yb = q % nyb, z = q / nyb;
    const int x0 = xb * UX, y0 = yb * UY;
    // kept bits of the three words (the same for every row)
    const int right_room = g.nx - x0;   // >= 1
    const unsigned m0 = (x0 == 0 || L == 0) ? 0u : (0xffffffffu << (32 - L));
    const unsigned m1 = right_room >= 32 ? 0xffffffffu : ((1u << right_room) - 1u);
    const int r2 = min(L, right_room - 32);
    const unsigned m2 = r2 <= 0 ? 0u : ((1u << r2) - 1u);

    // row sets: [0] output row y0 + lane, [1] y0 - L + lane, [2] y0 + 32 + lane
    unsigned w[3][3], rm[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int y = j == 0 ? y0 + lane : (j == 1 ? y0 - L + lane : y0 + UY + lane);
        const bool mine = j == 0 || lane < L;
        unsigned a0 = 0u, a1 = 0u, a2 = 0u;
        if (mine && y >= 0 && y < g.ny) {
            const long long b = (long long)g.nx * (y + (long long)g.ny * z) + x0 - 32;
            const long long wi = b >> 5;   // floor (b >= -32)
            const int sh = (int)(b & 31);
            unsigned qw[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                qw[i] = (wi + i >= 0 && wi + i < n_words) ? __ldg(occ + wi + i) : 0u;
            a0 = __funnelshift_r(qw[0], qw[1], sh) & m0;
            a1 = __funnelshift_r(qw[1], qw[2], sh) & m1;
            a2 = __funnelshift_r(qw[2], qw[3], sh) & m2;
        }
        w[j][0] = a0;
        w[j][1] = a1;
        w[j][2] = a2;
        rm[j] = __ballot_sync(FULL_MASK, (a0 | a1 | a2) != 0u);
    }
    if ((rm[0] | rm[1] | rm[2]) == 0u) {
        if (lane == 0)
            rows[u] = 0u;
        return;
    }

    // pass-X word of row set j held by lane s, for this lane's x
    auto label = [&](int j, int s) -> unsigned {
        const unsigned b0 = __shfl_sync(FULL_MASK, w[j][0], s);
        const unsigned b1 = __shfl_sync(FULL_MASK, w[j][1], s);
        const unsigned b2 = __shfl_sync(FULL_MASK, w[j][2], s);
        return row_word<W>(__funnelshift_r(b0, b1, lane), __funnelshift_r(b1, b2, lane), L);
    };
    unsigned c[UY];
#pragma unroll
    for (int k = 0; k < UY; ++k)
        c[k] = ((rm[0] >> k) & 1u) ? label(0, k) : NONE;
    // halo rows: below (seen from output row 0) and above (from row 31)
    unsigned before = NONE, after = NONE;
    for (unsigned m = rm[1]; m; m &= m - 1u) {   // row y0 - L + s: L - s below row 0
        const int s = __ffs(m) - 1;
        before = min(before, stepn<W::SD>(label(1, s), L - s, STEP_YF, L));
    }
    for (unsigned m = rm[2]; m; m &= m - 1u) {   // row y0 + 32 + s: s + 1 above row 31
        const int s = __ffs(m) - 1;
        after = min(after, stepn<W::SD>(label(2, s), s + 1, STEP_YB, L));
    }
    sweep32<STEP_YF, STEP_YB>(c, before, after, (unsigned)L << W::SD);

    // labelled rows (the sweeps also carry labels into rows past the grid's
    // edge, which are left out)
    const int x = x0 + lane;
    const bool in = x < g.nx;
    const int y_room = g.ny - y0;   // >= 1
    unsigned labelled = 0u;
#pragma unroll
    for (int k = 0; k < UY; ++k)
        labelled |= __ballot_sync(FULL_MASK, in && c[k] != NONE) != 0u ? (1u << k) : 0u;
    if (y_room < UY)
        labelled &= (1u << y_room) - 1u;
    if (lane == 0)
        rows[u] = labelled;
    if (in) {
        const int base = x + g.nx * (y0 + g.ny * z);
#pragma unroll
        for (int k = 0; k < UY; ++k)
            if ((labelled >> k) & 1u)
                inter[base + g.nx * k] = (typename W::Stored)c[k];
    }
}

// Where pass Z puts its labels: the dense root / ring arrays (with the
// per-unit flags that let unlabelled units skip their writes), or the
// labelled-segment table of the sparse grid (row segment -> label mask and
// first root index; the roots in a packed array; the ring is the Manhattan
// distance between a voxel and its root), which holds the labelled segments
// only and starts empty at every dilation.
struct DenseLabels {
    unsigned char *dirty;
    int *root;
    unsigned char *ring;
};
struct HashLabels {
    HashTable table;       // keys: the labelled row segments (32 voxels along x of one row of one plane)
    uint2 *seg;            // [slots] the segment's label mask and the index of its first root in `root`
    int *root;             // [cap_root] root keys of the labelled voxels, segment by segment
    unsigned cap_root;
    unsigned *root_count;  // roots handed out so far (zero before the dilation)
    unsigned *overflow;    // set to 1 when an insert gave up or the roots ran out (too small) ...
    unsigned *err;         // ... and DEVERR_CAPACITY set in the device status word
};

template <class W>
__device__ __forceinline__ unsigned dilate_z_segments(unsigned (&c)[32], unsigned before, unsigned after,
                                                      const HashLabels &out, const GridGeom &g, int L, int col,
                                                      int z0, int kmax, bool in_x, int xb, int y, int nxb);

// ---------------------------------------------------------------------------
// Pass Z and the output.  Warp u = xb + nxb*(y + ny*zb) covers x in
// [32xb, 32xb+32) of row y, z in [32zb, 32zb+32).  Lane l reads whether row y
// is labelled after pass Y in output plane z0 + l and, for l < L, in halo
// planes z0 - L + l and z0 + 32 + l; only those planes are read from the
// intermediate array, all before the sweeps (halo planes four at a time).
// ---------------------------------------------------------------------------
template <class W, class Out = DenseLabels>
__device__ __forceinline__ unsigned dilate_z_unit(int u, const typename W::Stored *__restrict__ inter,
                                                  const unsigned *__restrict__ rows, const Out &out, const GridGeom &g,
                                                  int L, int nxb, int nyb)
{
    constexpr bool HASHED = !__is_same(Out, DenseLabels);
    constexpr unsigned STEP_ZF = (1u << W::ZD) - (1u << W::ZZ);   // moved from z-1 to z: dz -= 1
    constexpr unsigned STEP_ZB = (1u << W::ZD) + (1u << W::ZZ);   // moved from z+1 to z: dz += 1
    const int lane = threadIdx.x & 31;
    const int xb = u % nxb, q = u / nxb;
    const int y = q % g.ny, zb = q / g.ny;
    const int x0 = xb * UX, z0 = zb * UZ, yb = y / UY, ybit = y & (UY - 1);
    const int x = x0 + lane;
    const int plane = g.nx * g.ny;
    const int col = x + g.nx * y;   // voxel (x, y, 0)
    const int kmax = min(UZ, g.nz - z0);

    // planes: [0] output z0 + lane, [1] z0 - L + lane, [2] z0 + 32 + lane
    unsigned pm[3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        const int z = j == 0 ? z0 + lane : (j == 1 ? z0 - L + lane : z0 + UZ + lane);
        const bool mine = j == 0 || lane < L;
        bool set = false;
        if (mine && z >= 0 && z < g.nz)
            set = (__ldg(rows + (z * nyb + yb) * nxb + xb) >> ybit) & 1u;
        pm[j] = __ballot_sync(FULL_MASK, set);
    }
    const bool labels = (pm[0] | pm[1] | pm[2]) != 0u;
    if constexpr (HASHED) {
        if (!labels)   // the whole warp: the segments' ballots need every lane
            return 0u;
    } else {
        // A unit with nothing within L keeps "unlabelled" unless the previous
        // dilation labelled some of its voxels; those are reset here.
        const bool was = __ldg(out.dirty + u) != 0;
        if (lane == 0 && labels != was)
            out.dirty[u] = labels ? 1 : 0;
        if (x >= g.nx || !(labels || was))
            return 0u;
        if (!labels) {
            int v = col + plane * z0;
#pragma unroll 8
            for (int k = 0; k < kmax; ++k, v += plane) {
                out.root[v] = -1;
                out.ring[v] = 255;
            }
            return 0u;
        }
    }

    const bool in_x = x < g.nx;   // (hashed: lanes past the grid take part, with no words)
    unsigned c[UZ];
#pragma unroll
    for (int k = 0; k < UZ; ++k)
        c[k] = (in_x && ((pm[0] >> k) & 1u)) ? W::load_z(inter, col + plane * (z0 + k)) : NONE;
    unsigned before = NONE, after = NONE;
#pragma unroll 1
    for (int side = 1; side <= 2; ++side) {
        for (unsigned m = side == 1 ? pm[1] : pm[2]; m;) {
            int s[4];
            unsigned wv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                s[i] = m ? __ffs(m) - 1 : -1;
                m &= m - 1u;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int zz = side == 1 ? z0 - L + s[i] : z0 + UZ + s[i];
                wv[i] = (in_x && s[i] >= 0) ? W::load_z(inter, col + plane * zz) : NONE;
            }
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                if (s[i] >= 0) {
                    if (side == 1)   // L - s below plane 0
                        before = min(before, stepn<W::ZD>(wv[i], L - s[i], STEP_ZF, L));
                    else             // s + 1 above plane 31
                        after = min(after, stepn<W::ZD>(wv[i], s[i] + 1, STEP_ZB, L));
                }
            }
        }
    }
    if constexpr (HASHED)
        return dilate_z_segments<W>(c, before, after, out, g, L, col, z0, kmax, in_x, xb, y, nxb);
    sweep32<STEP_ZF, STEP_ZB>(c, before, after, (unsigned)L << W::ZD);

    const unsigned valid = (unsigned)(L + 1) << W::ZD;   // words below this are labels
    const int v0 = col + plane * z0;
    const unsigned vb = (unsigned)v0 - W::bias((unsigned)g.nx, (unsigned)plane);
    int v = v0;
    unsigned labelled = 0u;
#pragma unroll
    for (int k = 0; k < UZ; ++k, v += plane) {
        if (k < kmax) {
            const unsigned w = c[k];
            const bool hit = w < valid;
            const int r = (int)(vb + (unsigned)plane * k + W::offset(w, (unsigned)g.nx, (unsigned)plane));
            if constexpr (!HASHED) {
                out.root[v] = hit ? r : -1;
                out.ring[v] = hit ? (unsigned char)(w >> W::ZD) : (unsigned char)255;
                labelled += hit ? 1u : 0u;
            }
        }
    }
    return labelled;
}

// Pass Z's output into the sparse grid's labelled-segment table.  Plane k
// of the unit is one row segment (x in [32 xb, 32 xb + 32) of row y); its
// labelled voxels, a ballot over the lanes, are one entry: the label mask
// and the index of the segment's first root in the root array, whose slice
// for the whole unit one lane reserves with a single atomic.  Lane k then
// inserts segment k (at most 32 inserts per unit, all at once), and every
// lane stores the roots of its labelled voxels at their rank in the
// segment.  Returns the segments entered (for the table's size).
template <class W>
__device__ __forceinline__ unsigned dilate_z_segments(unsigned (&c)[32], unsigned before, unsigned after,
                                                      const HashLabels &out, const GridGeom &g, int L, int col,
                                                      int z0, int kmax, bool in_x, int xb, int y, int nxb)
{
    constexpr unsigned STEP_ZF = (1u << W::ZD) - (1u << W::ZZ);
    constexpr unsigned STEP_ZB = (1u << W::ZD) + (1u << W::ZZ);
    const int lane = threadIdx.x & 31;
    const int plane = g.nx * g.ny;
    sweep32<STEP_ZF, STEP_ZB>(c, before, after, (unsigned)L << W::ZD);
    const unsigned valid = (unsigned)(L + 1) << W::ZD;   // words below this are labels

    // lane k: the label mask of plane k
    unsigned my_mask = 0u;
#pragma unroll
    for (int k = 0; k < UZ; ++k) {
        const unsigned m = __ballot_sync(FULL_MASK, in_x && k < kmax && c[k] < valid);
        if (lane == k)
            my_mask = m;
    }
    const unsigned cnt = __popc(my_mask);
    unsigned incl = cnt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const unsigned t = __shfl_up_sync(FULL_MASK, incl, d);
        if (lane >= d)
            incl += t;
    }
    const unsigned total = __shfl_sync(FULL_MASK, incl, 31);
    if (total == 0u)
        return 0u;
    unsigned base = 0u;
    if (lane == 0)
        base = atomicAdd(out.root_count, total);
    base = __shfl_sync(FULL_MASK, base, 0);
    if ((unsigned long long)base + total > out.cap_root) {   // the root array is too small
        if (lane == 0) {
            atomicOr(out.overflow, 1u);
            atomicOr(out.err, DEVERR_CAPACITY);
        }
        return 0u;
    }
    const unsigned my_base = base + incl - cnt;
    if (my_mask) {
        const unsigned sid = (unsigned)xb + (unsigned)nxb * ((unsigned)y + (unsigned)g.ny * (unsigned)(z0 + lane));
        const int slot = hash_insert(out.table, sid);
        if (slot >= 0) {
            out.seg[slot] = make_uint2(my_mask, my_base);
        } else {
            atomicOr(out.overflow, 1u);
            atomicOr(out.err, DEVERR_CAPACITY);
        }
    }
    const unsigned vb = (unsigned)(col + plane * z0) - W::bias((unsigned)g.nx, (unsigned)plane);
#pragma unroll
    for (int k = 0; k < UZ; ++k) {
        const unsigned mk = __shfl_sync(FULL_MASK, my_mask, k), bk = __shfl_sync(FULL_MASK, my_base, k);
        if ((mk >> lane) & 1u) {
            const int r = (int)(vb + (unsigned)plane * k + W::offset(c[k], (unsigned)g.nx, (unsigned)plane));
            out.root[bk + __popc(mk & ((1u << lane) - 1u))] = r;
        }
    }
    return __popc(__ballot_sync(FULL_MASK, my_mask != 0u));
}

}  // namespace dil

}  // namespace vicp
