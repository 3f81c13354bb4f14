// vicp_dilate.cu -- DDMA, dilation of root-voxel labels into empty voxels
// (Alg. 3 and its description in Sec. 3).
//
// What is computed.  L synchronous rounds of six-neighbour propagation, with
// the smallest root kept where several labelled neighbours meet, label every
// voxel v within Manhattan distance L of an occupied voxel with
//     ring[v] = d(v) = min over occupied u of |u - v|_1,
//     root[v] = the smallest linear index among occupied u at that distance,
// and leave the rest at root -1 / ring 255.  (On a box grid every monotone
// lattice path between two voxels stays inside the box, so the rounds reach
// exactly the voxels at Manhattan distance r in round r.)
//
// How.  Instead of L rounds over the dense grid, the kernel evaluates that
// closed form as a separable lexicographic minimum.  A candidate is packed
// into one 32-bit word (dist:6 | dz+31:6 | dy+31:6 | dx+31:6), the root's
// offset from the voxel holding the word.  Because the linear index
// x + nx*(y + ny*z) orders in-grid voxels as (z, y, x) lexicographically, for
// a fixed voxel the unsigned order of these words is the order (distance,
// root index).  Moving a word one voxel along an axis adds one to the
// distance and shifts one offset field: a single integer add.  Words whose
// distance reaches L are dropped (they cannot end within L).
//
//   pass X: nearest occupied voxel along the row, from the occupancy bitmask
//           with clz/ffs on a 64-bit window (ties go to the left, the smaller
//           index);
//   pass Y: forward and backward running minimum along y;
//   pass Z: the same along z, then the word is decoded into root and ring.
//
// The grid is cut into 32 x 8 x 32 output tiles (32 x 8 x 8 for L > 16).  A
// tile whose L-grown box touches no occupied 8x8x8 brick is written
// "unlabelled" by a light classification kernel.  Every other tile is processed by one CTA, which
// stages the occupancy bits of the tile grown by L in y and z (three 32-bit
// words per row cover x in [x0-32, x0+64)), runs passes X and Y for eight
// z-planes at a time into shared memory, then pass Z, and writes root and
// ring with coalesced stores.  L <= 31.
#include "vicp_launch.h"

namespace vicp {

namespace {
constexpr int TX = 32, TY = 8, ZB = 8, THREADS = 256;
constexpr unsigned NONE = 0xffffffffu;
constexpr int SH_D = 18, SH_Z = 12, SH_Y = 6;
constexpr unsigned CENTER = (31u << SH_Z) | (31u << SH_Y) | 31u;   // zero offsets
constexpr unsigned STEP_D = 1u << SH_D;
constexpr unsigned STEP_YF = STEP_D - (1u << SH_Y);   // moved from y-1 to y: dy -= 1
constexpr unsigned STEP_YB = STEP_D + (1u << SH_Y);   // moved from y+1 to y: dy += 1
constexpr unsigned STEP_ZF = STEP_D - (1u << SH_Z);
constexpr unsigned STEP_ZB = STEP_D + (1u << SH_Z);
constexpr int TZ_WIDE = 32, TZ_NARROW = 8, L_WIDE_MAX = 16;   // 32-deep tiles while shared memory allows

// Move a word n voxels (n >= 0) along one axis: the distance grows by n and
// one offset field shifts by n (inc = the one-voxel step).  A word whose
// distance would exceed L becomes NONE (NONE stays NONE).
__device__ __forceinline__ unsigned stepn(unsigned v, int n, unsigned inc, int L)
{
    if (n > L)
        return NONE;
    return v >= ((unsigned)(L + 1 - n) << SH_D) ? NONE : v + (unsigned)n * inc;
}
}  // namespace

// Row-mask words per plane: bit yy of word yy/32 is set when row yy of the
// grown tile holds an occupied voxel in the staged x window.
__host__ __device__ constexpr int mask_words(int HY) { return (HY + 31) / 32; }

static int tile_depth(int L) { return L <= L_WIDE_MAX ? TZ_WIDE : TZ_NARROW; }

size_t dilate_smem_bytes(int L)
{
    const size_t TZ = tile_depth(L), HY = TY + 2 * L, HZ = TZ + 2 * L;
    return sizeof(unsigned) * (HZ * HY * 3 + HZ * mask_words((int)HY) + mask_words((int)HZ) + ZB * HY * TX +
                               HZ * TY * TX);
}

__device__ __forceinline__ bool bit_of(const unsigned *m, int i) { return (m[i >> 5] >> (i & 31)) & 1u; }

// ---------------------------------------------------------------------------
// Tile classification: a CTA per TX x TY x TZ tile checks the brick offsets
// of every 8x8x8 brick its L-grown box touches.  A tile with no point in
// reach writes "unlabelled" (root -1, ring 255) for its voxels at once (a
// warp per row); any other tile is appended to the list the shared-memory
// kernel works through.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_dilate_tiles(const unsigned *__restrict__ boff, GridGeom g, int L, int TZ,
                                                      int tiles_x, int tiles_y, int n_tiles,
                                                      int *__restrict__ active, DevCtl *__restrict__ ctl,
                                                      int *__restrict__ root, unsigned char *__restrict__ ring)
{
    const int t = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int txy = tiles_x * tiles_y;
    const int x0 = (t % tiles_x) * TX;
    const int y0 = ((t / tiles_x) % tiles_y) * TY;
    const int z0 = (t / txy) * TZ;
    const int bx0 = max(x0 - L, 0) / BRICK, bx1 = min(x0 + TX - 1 + L, g.nx - 1) / BRICK;
    const int by0 = max(y0 - L, 0) / BRICK, by1 = min(y0 + TY - 1 + L, g.ny - 1) / BRICK;
    const int bz0 = max(z0 - L, 0) / BRICK, bz1 = min(z0 + TZ - 1 + L, g.nz - 1) / BRICK;
    const int nbx = bx1 - bx0 + 1, nby = by1 - by0 + 1, nb = nbx * nby * (bz1 - bz0 + 1);
    int any = 0;
    for (int k = threadIdx.x; k < nb; k += blockDim.x) {
        const int b = brick_index(g, bx0 + k % nbx, by0 + (k / nbx) % nby, bz0 + k / (nbx * nby));
        any |= __ldg(boff + b + 1) > __ldg(boff + b);
    }
    if (__syncthreads_or(any)) {
        if (threadIdx.x == 0) {
            const int slot = atomicAdd(&ctl->n_active_tiles, 1);
            if (slot < n_tiles)
                active[slot] = t;
            else
                atomicOr(&ctl->err, DEVERR_BOUNDS);
        }
        return;
    }
    const int x = x0 + lane;
    if (x >= g.nx)
        return;
    const int ny_t = min(TY, g.ny - y0), nz_t = min(TZ, g.nz - z0);
#pragma unroll 1
    for (int r = warp; r < ny_t * nz_t; r += blockDim.x / 32) {
        const long long v = x + (long long)g.nx * (y0 + r % ny_t + (long long)g.ny * (z0 + r / ny_t));
        root[v] = -1;
        ring[v] = 255;
    }
}

// ---------------------------------------------------------------------------
// Active tiles: a persistent grid works through the list; the last block to
// finish clears the list length for the next dilation.  Work follows the
// occupied rows: pass X runs on rows holding an occupied voxel in the staged
// window; passes Y and Z step from one occupied row (plane) to the next with
// the n-voxel shift and evaluate every output row (plane) of the tile.
// ---------------------------------------------------------------------------
template <int TZ>
__global__ void __launch_bounds__(THREADS) k_dilate(const unsigned *__restrict__ occ,
                                                    const int *__restrict__ active, GridGeom g, int L,
                                                    int tiles_x, int tiles_y, int n_tiles,
                                                    int *__restrict__ root, unsigned char *__restrict__ ring,
                                                    DevCtl *__restrict__ ctl)
{
    extern __shared__ unsigned smem[];
    const int HY = TY + 2 * L, HZ = TZ + 2 * L, MW = mask_words(HY), PW = mask_words(HZ);
    unsigned *s_bits = smem;                  // [HZ][HY][3]
    unsigned *s_mask = s_bits + HZ * HY * 3;  // [HZ][MW]      rows holding an occupied voxel
    unsigned *s_pmask = s_mask + HZ * MW;     // [PW]          planes whose pass-Y output is not all NONE
    unsigned *s_a = s_pmask + PW;             // [ZB][HY][TX]  pass X, one z batch (occupied rows only)
    unsigned *s_b = s_a + ZB * HY * TX;       // [HZ][TY][TX]  pass Y (flagged planes only)
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_active = min(*(volatile int *)&ctl->n_active_tiles, n_tiles);
    const int txy = tiles_x * tiles_y;

    for (int it = blockIdx.x; it < n_active; it += gridDim.x) {
        const int t = __ldg(active + it);
        const int x0 = (t % tiles_x) * TX;
        const int y0 = ((t / tiles_x) % tiles_y) * TY;
        const int z0 = (t / txy) * TZ;

        // 1. occupancy windows of the grown tile (a lane per row, a warp per
        //    32 rows of one plane) and the per-plane masks of occupied rows
        if (tid < PW)
            s_pmask[tid] = 0u;
        for (int zz = warp; zz < HZ; zz += THREADS / 32) {
            const int z = z0 - L + zz;
            for (int yb = 0; yb < HY; yb += 32) {
                const int yy = yb + lane, y = y0 - L + yy;
                unsigned w[3] = {0u, 0u, 0u};
                if (yy < HY && y >= 0 && y < g.ny && z >= 0 && z < g.nz) {
                    const long long rowbase = (long long)g.nx * (y + (long long)g.ny * z);
#pragma unroll
                    for (int k = 0; k < 3; ++k) {
                        const int xs = x0 - 32 + 32 * k;
                        const int lo = max(xs, 0), hi = min(xs + 32, g.nx);
                        if (lo < hi)
                            w[k] = extract_bits(occ, rowbase + lo, hi - lo) << (lo - xs);
                    }
                }
                if (yy < HY) {
                    unsigned *dst = s_bits + (zz * HY + yy) * 3;
                    dst[0] = w[0];
                    dst[1] = w[1];
                    dst[2] = w[2];
                }
                const unsigned m = __ballot_sync(FULL_MASK, (w[0] | w[1] | w[2]) != 0u);
                if (lane == 0)
                    s_mask[zz * MW + (yb >> 5)] = m;
            }
        }
        __syncthreads();

        for (int zb = 0; zb < HZ; zb += ZB) {
            // 2a. pass X on the occupied rows: warp w takes plane zb + w
            const int zz = zb + warp;
            if (zz < HZ) {
                for (int mw = 0; mw < MW; ++mw) {
                    unsigned m = s_mask[zz * MW + mw];
                    while (m) {
                        const int yy = 32 * mw + __ffs(m) - 1;
                        m &= m - 1u;
                        const unsigned *wrow = s_bits + (zz * HY + yy) * 3;
                        const unsigned a0 = wrow[0], a1 = wrow[1], a2 = wrow[2];
                        const unsigned left = __funnelshift_r(a0, a1, lane);    // bit i <-> x - 32 + i
                        const unsigned right = __funnelshift_r(a1, a2, lane);   // bit i <-> x + i
                        unsigned lbl = NONE;
                        if (right & 1u) {
                            lbl = CENTER;
                        } else if (L > 0) {
                            const unsigned lm = left & (0xffffffffu << (32 - L));
                            const unsigned rm = (right >> 1) & ((1u << L) - 1u);
                            const int dl = lm ? __clz(lm) + 1 : 64;
                            const int dr = rm ? __ffs(rm) : 64;
                            if (dl <= dr) {
                                if (dl <= L)
                                    lbl = ((unsigned)dl << SH_D) | (CENTER - (unsigned)dl);
                            } else if (dr <= L) {
                                lbl = ((unsigned)dr << SH_D) | (CENTER + (unsigned)dr);
                            }
                        }
                        s_a[(warp * HY + yy) * TX + lane] = lbl;
                    }
                }
            }
            __syncthreads();
            // 2b. pass Y: thread per (x, plane of the batch), stepping over
            //     the plane's occupied rows
            if (zz < HZ) {
                const unsigned *mk = s_mask + zz * MW;
                bool any_row = false;
                for (int mw = 0; mw < MW; ++mw)
                    any_row |= mk[mw] != 0u;
                if (any_row) {
                    if (lane == 0)
                        atomicOr(s_pmask + (zz >> 5), 1u << (zz & 31));
                    const unsigned *col = s_a + warp * HY * TX + lane;
                    unsigned *ob = s_b + zz * TY * TX + lane;
                    // forward: occupied rows below the tile, then every output row
                    unsigned f = NONE;
                    int rp = 0;
                    for (int mw = 0; mw < MW && 32 * mw < L; ++mw) {
                        unsigned m = mk[mw];
                        if (32 * mw + 32 > L)
                            m &= (1u << (L - 32 * mw)) - 1u;
                        while (m) {
                            const int r = 32 * mw + __ffs(m) - 1;
                            m &= m - 1u;
                            f = min(stepn(f, r - rp, STEP_YF, L), col[r * TX]);
                            rp = r;
                        }
                    }
#pragma unroll
                    for (int k = 0; k < TY; ++k) {
                        const int y = L + k;
                        f = stepn(f, y - rp, STEP_YF, L);
                        if (bit_of(mk, y))
                            f = min(f, col[y * TX]);
                        rp = y;
                        ob[k * TX] = f;
                    }
                    // backward: occupied rows above the tile, then every output row
                    unsigned bk = NONE;
                    rp = HY - 1;
                    for (int mw = MW - 1; mw >= 0; --mw) {
                        if (32 * mw + 31 < L + TY)
                            break;
                        unsigned m = mk[mw];
                        if (32 * mw < L + TY)
                            m &= ~((1u << (L + TY - 32 * mw)) - 1u);
                        while (m) {
                            const int r = 32 * mw + 31 - __clz(m);
                            m &= ~(1u << (r - 32 * mw));
                            bk = min(stepn(bk, rp - r, STEP_YB, L), col[r * TX]);
                            rp = r;
                        }
                    }
#pragma unroll
                    for (int k = TY - 1; k >= 0; --k) {
                        const int y = L + k;
                        bk = stepn(bk, rp - y, STEP_YB, L);
                        if (bit_of(mk, y))
                            bk = min(bk, col[y * TX]);
                        rp = y;
                        ob[k * TX] = min(ob[k * TX], bk);
                    }
                }
            }
            __syncthreads();
        }

        // 3. pass Z: thread per (x, y) column, stepping over the planes whose
        //    pass-Y output is not all NONE
        unsigned out[TZ];
        {
            const unsigned *col = s_b + warp * TX + lane;
            unsigned f = NONE;
            int rp = 0;
            for (int pw = 0; pw < PW && 32 * pw < L; ++pw) {
                unsigned m = s_pmask[pw];
                if (32 * pw + 32 > L)
                    m &= (1u << (L - 32 * pw)) - 1u;
                while (m) {
                    const int r = 32 * pw + __ffs(m) - 1;
                    m &= m - 1u;
                    f = min(stepn(f, r - rp, STEP_ZF, L), col[r * TY * TX]);
                    rp = r;
                }
            }
#pragma unroll
            for (int k = 0; k < TZ; ++k) {
                const int z = L + k;
                f = stepn(f, z - rp, STEP_ZF, L);
                if (bit_of(s_pmask, z))
                    f = min(f, col[z * TY * TX]);
                rp = z;
                out[k] = f;
            }
            unsigned bk = NONE;
            rp = HZ - 1;
            for (int pw = PW - 1; pw >= 0; --pw) {
                if (32 * pw + 31 < L + TZ)
                    break;
                unsigned m = s_pmask[pw];
                if (32 * pw < L + TZ)
                    m &= ~((1u << (L + TZ - 32 * pw)) - 1u);
                while (m) {
                    const int r = 32 * pw + 31 - __clz(m);
                    m &= ~(1u << (r - 32 * pw));
                    bk = min(stepn(bk, rp - r, STEP_ZB, L), col[r * TY * TX]);
                    rp = r;
                }
            }
#pragma unroll
            for (int k = TZ - 1; k >= 0; --k) {
                const int z = L + k;
                bk = stepn(bk, rp - z, STEP_ZB, L);
                if (bit_of(s_pmask, z))
                    bk = min(bk, col[z * TY * TX]);
                rp = z;
                out[k] = min(out[k], bk);
            }
        }
        // 4. decode and store
        const int x = x0 + lane, y = y0 + warp;
        if (x < g.nx && y < g.ny) {
            const long long plane = (long long)g.nx * g.ny;
            long long v = x + (long long)g.nx * y + plane * z0;
#pragma unroll
            for (int k = 0; k < TZ; ++k, v += plane) {
                if (z0 + k < g.nz) {
                    const unsigned w = out[k];
                    int r = -1;
                    unsigned char d = 255;
                    if (w != NONE) {
                        const int dz = (int)((w >> SH_Z) & 63u) - 31;
                        const int dy = (int)((w >> SH_Y) & 63u) - 31;
                        const int dx = (int)(w & 63u) - 31;
                        r = (int)(v + dx + (long long)g.nx * dy + plane * dz);
                        d = (unsigned char)(w >> SH_D);
                    }
                    root[v] = r;
                    ring[v] = d;
                }
            }
        }
        __syncthreads();   // shared memory is reused by the next tile
    }

    if (tid == 0) {
        __threadfence();
        if (atomicAdd(&ctl->dil_done, 1u) == gridDim.x - 1) {
            ctl->n_active_tiles = 0;
            ctl->dil_done = 0u;
        }
    }
}

template <int TZ>
static cudaError_t run_dilate(const unsigned *occ, const unsigned *boff, const GridGeom &g, int L, int *active,
                              int *root, unsigned char *ring, DevCtl *ctl, int sms, cudaStream_t st)
{
    const int tiles_x = (g.nx + TX - 1) / TX, tiles_y = (g.ny + TY - 1) / TY, tiles_z = (g.nz + TZ - 1) / TZ;
    const int tiles = tiles_x * tiles_y * tiles_z;   // < V < 2^31
    k_dilate_tiles<<<tiles, 256, 0, st>>>(boff, g, L, TZ, tiles_x, tiles_y, tiles, active, ctl, root, ring);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const size_t smem = dilate_smem_bytes(L);
    e = cudaFuncSetAttribute(k_dilate<TZ>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess)
        return e;
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dilate<TZ>, THREADS, smem);
    if (e != cudaSuccess)
        return e;
    int grid = sms * (per_sm > 0 ? per_sm : 1);
    if (grid > tiles)
        grid = tiles;
    k_dilate<TZ><<<grid, THREADS, smem, st>>>(occ, active, g, L, tiles_x, tiles_y, tiles, root, ring, ctl);
    return cudaGetLastError();
}

long long dilate_tiles(const GridGeom &g, int L)
{
    const int TZ = tile_depth(L);
    return (long long)((g.nx + TX - 1) / TX) * ((g.ny + TY - 1) / TY) * ((g.nz + TZ - 1) / TZ);
}

cudaError_t launch_dilate(const unsigned *occ, const unsigned *boff, const GridGeom &g, int L, int *active,
                          int *root, unsigned char *ring, DevCtl *ctl, int sms, cudaStream_t st)
{
    if (tile_depth(L) == TZ_WIDE)
        return run_dilate<TZ_WIDE>(occ, boff, g, L, active, root, ring, ctl, sms, st);
    return run_dilate<TZ_NARROW>(occ, boff, g, L, active, root, ring, ctl, sms, st);
}

}  // namespace vicp
