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
// The grid is cut into 32 x 8 x 8 output tiles.  A tile whose L-grown box
// touches no occupied 8x8x8 brick is written "unlabelled" by a light
// classification kernel.  Every other tile is processed by one CTA, which
// stages the occupancy bits of the tile grown by L in y and z (three 32-bit
// words per row cover x in [x0-32, x0+64)), runs passes X and Y for eight
// z-planes at a time into shared memory, then pass Z, and writes root and
// ring with coalesced stores.  L <= 31.
#include "vicp_launch.h"

namespace vicp {

namespace {
constexpr int TX = 32, TY = 8, TZ = 8, ZB = 8, THREADS = 256;
constexpr unsigned NONE = 0xffffffffu;
constexpr int SH_D = 18, SH_Z = 12, SH_Y = 6;
constexpr unsigned CENTER = (31u << SH_Z) | (31u << SH_Y) | 31u;   // zero offsets
constexpr unsigned STEP_D = 1u << SH_D;
constexpr unsigned STEP_YF = STEP_D - (1u << SH_Y);   // moved from y-1 to y: dy -= 1
constexpr unsigned STEP_YB = STEP_D + (1u << SH_Y);   // moved from y+1 to y: dy += 1
constexpr unsigned STEP_ZF = STEP_D - (1u << SH_Z);
constexpr unsigned STEP_ZB = STEP_D + (1u << SH_Z);

// Move a word one voxel; words at distance >= L (and NONE) become NONE.
// `lim` = L << SH_D: a word is >= lim exactly when its distance is >= L.
__device__ __forceinline__ unsigned step(unsigned v, unsigned inc, unsigned lim)
{
    return v >= lim ? NONE : v + inc;
}
}  // namespace

// Row-mask words per plane: bit yy of word yy/32 is set when row yy of the
// grown tile holds an occupied voxel in the staged x window.
__host__ __device__ constexpr int mask_words(int HY) { return (HY + 31) / 32; }

size_t dilate_smem_bytes(int L)
{
    const size_t HY = TY + 2 * L, HZ = TZ + 2 * L;
    return sizeof(unsigned) * (HZ * HY * 3 + HZ * mask_words((int)HY) + ZB * HY * TX + HZ * TY * TX);
}

__device__ __forceinline__ bool row_bit(const unsigned *m, int yy) { return (m[yy >> 5] >> (yy & 31)) & 1u; }

// ---------------------------------------------------------------------------
// Tile classification: a warp per 32 x 8 x 8 tile checks the brick offsets of
// every 8x8x8 brick its L-grown box touches.  A tile with no point in reach
// writes "unlabelled" (root -1, ring 255) for its voxels at once; any other
// tile is appended to the list the shared-memory kernel below works through.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_dilate_tiles(const unsigned *__restrict__ boff, GridGeom g, int L,
                                                      int tiles_x, int tiles_y, long long n_tiles,
                                                      int *__restrict__ active, DevCtl *__restrict__ ctl,
                                                      int *__restrict__ root, unsigned char *__restrict__ ring)
{
    const long long t = ((long long)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (t >= n_tiles)
        return;   // whole warp
    const int x0 = (int)(t % tiles_x) * TX;
    const int y0 = (int)((t / tiles_x) % tiles_y) * TY;
    const int z0 = (int)(t / ((long long)tiles_x * tiles_y)) * TZ;
    const int bx0 = max(x0 - L, 0) / BRICK, bx1 = min(x0 + TX - 1 + L, g.nx - 1) / BRICK;
    const int by0 = max(y0 - L, 0) / BRICK, by1 = min(y0 + TY - 1 + L, g.ny - 1) / BRICK;
    const int bz0 = max(z0 - L, 0) / BRICK, bz1 = min(z0 + TZ - 1 + L, g.nz - 1) / BRICK;
    const int nbx = bx1 - bx0 + 1;
    bool any = false;
    for (int bz = bz0; bz <= bz1; ++bz)
        for (int by = by0; by <= by1; by += 1) {
            if (lane < nbx) {
                const int b = bx0 + lane + g.bx * (by + g.by * bz);
                any |= __ldg(boff + b + 1) > __ldg(boff + b);
            }
        }
    if (__any_sync(FULL_MASK, any)) {
        if (lane == 0) {
            const int slot = atomicAdd(&ctl->n_active_tiles, 1);
            if (slot < n_tiles)
                active[slot] = (int)t;
            else
                atomicOr(&ctl->err, DEVERR_BOUNDS);
        }
        return;
    }
    const int x = x0 + lane;
    if (x >= g.nx)
        return;
    const long long plane = (long long)g.nx * g.ny;
    const int ny_t = min(TY, g.ny - y0), nz_t = min(TZ, g.nz - z0);
    long long vz = x + (long long)g.nx * y0 + plane * z0;
    for (int zl = 0; zl < nz_t; ++zl, vz += plane) {
        long long v = vz;
        for (int yl = 0; yl < ny_t; ++yl, v += g.nx) {
            root[v] = -1;
            ring[v] = 255;
        }
    }
}

// ---------------------------------------------------------------------------
// Active tiles: a persistent grid works through the list; the last block to
// finish clears the list length for the next dilation.  Work is proportional
// to the occupied rows: pass X runs on the rows that hold an occupied voxel
// in the staged window, pass Y reads pass-X labels only of such rows and
// skips planes without any.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(THREADS) k_dilate(const unsigned *__restrict__ occ,
                                                    const int *__restrict__ active, GridGeom g, int L,
                                                    int tiles_x, int tiles_y, long long n_tiles,
                                                    int *__restrict__ root, unsigned char *__restrict__ ring,
                                                    DevCtl *__restrict__ ctl)
{
    extern __shared__ unsigned smem[];
    const int HY = TY + 2 * L, HZ = TZ + 2 * L, MW = mask_words(HY);
    unsigned *s_bits = smem;                  // [HZ][HY][3]
    unsigned *s_mask = s_bits + HZ * HY * 3;  // [HZ][MW]      non-empty rows
    unsigned *s_a = s_mask + HZ * MW;         // [ZB][HY][TX]  pass X, one z batch (non-empty rows only)
    unsigned *s_b = s_a + ZB * HY * TX;       // [HZ][TY][TX]  pass Y, all planes
    const unsigned lim = (unsigned)L << SH_D;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int n_active = (int)min((long long)*(volatile int *)&ctl->n_active_tiles, n_tiles);

    for (int it = blockIdx.x; it < n_active; it += gridDim.x) {
        const long long t = __ldg(active + it);
        const int x0 = (int)(t % tiles_x) * TX;
        const int y0 = (int)((t / tiles_x) % tiles_y) * TY;
        const int z0 = (int)(t / ((long long)tiles_x * tiles_y)) * TZ;

        // 1. occupancy windows of the grown tile (a lane per row, a warp per
        //    32 rows of one plane) and the per-plane masks of non-empty rows
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

        unsigned out[TZ];
        for (int zb = 0; zb < HZ; zb += ZB) {
            // 2a. pass X on the non-empty rows: warp w takes plane zb + w
            {
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
            }
            __syncthreads();
            // 2b. pass Y: thread per (x, plane of the batch); rows without an
            //     occupied voxel contribute nothing
            {
                const int zz = zb + warp;
                if (zz < HZ) {
                    const unsigned *mk = s_mask + zz * MW;
                    int first = HY, last = -1;
                    for (int mw = 0; mw < MW; ++mw) {
                        const unsigned m = mk[mw];
                        if (m) {
                            first = min(first, 32 * mw + __ffs(m) - 1);
                            last = max(last, 32 * mw + 31 - __clz(m));
                        }
                    }
                    unsigned *ob = s_b + zz * TY * TX + lane;
                    // rows farther than L from the tile's y range cannot reach it
                    if (last < 0) {   // no occupied row in reach: nothing to propagate
#pragma unroll
                        for (int k = 0; k < TY; ++k)
                            ob[k * TX] = NONE;
                    } else {
                        const unsigned *col = s_a + warp * HY * TX + lane;
                        unsigned f = NONE;
                        for (int yy = first; yy < L; ++yy)
                            f = min(step(f, STEP_YF, lim), row_bit(mk, yy) ? col[yy * TX] : NONE);
#pragma unroll
                        for (int k = 0; k < TY; ++k) {
                            const int yy = L + k;
                            f = min(step(f, STEP_YF, lim), (yy >= first && row_bit(mk, yy)) ? col[yy * TX] : NONE);
                            ob[k * TX] = f;
                        }
                        unsigned bk = NONE;
                        for (int yy = last; yy >= L + TY; --yy)
                            bk = min(step(bk, STEP_YB, lim), row_bit(mk, yy) ? col[yy * TX] : NONE);
#pragma unroll
                        for (int k = TY - 1; k >= 0; --k) {
                            const int yy = L + k;
                            bk = min(step(bk, STEP_YB, lim), (yy <= last && row_bit(mk, yy)) ? col[yy * TX] : NONE);
                            ob[k * TX] = min(ob[k * TX], bk);
                        }
                    }
                }
            }
            __syncthreads();
        }
        // 3. pass Z: thread per (x, y) column of the tile
        {
            const unsigned *col = s_b + warp * TX + lane;
            unsigned f = NONE;
            for (int zz = 0; zz < L; ++zz)
                f = min(step(f, STEP_ZF, lim), col[zz * TY * TX]);
#pragma unroll
            for (int k = 0; k < TZ; ++k) {
                f = min(step(f, STEP_ZF, lim), col[(L + k) * TY * TX]);
                out[k] = f;
            }
            unsigned bk = NONE;
            for (int zz = HZ - 1; zz >= L + TZ; --zz)
                bk = min(step(bk, STEP_ZB, lim), col[zz * TY * TX]);
#pragma unroll
            for (int k = TZ - 1; k >= 0; --k) {
                bk = min(step(bk, STEP_ZB, lim), col[(L + k) * TY * TX]);
                out[k] = min(out[k], bk);
            }
        }
        // 4. decode and store
        const int x = x0 + lane, y = y0 + warp;
        if (x < g.nx && y < g.ny) {
#pragma unroll
            for (int k = 0; k < TZ; ++k) {
                const int z = z0 + k;
                if (z < g.nz) {
                    const long long v = x + (long long)g.nx * (y + (long long)g.ny * z);
                    const unsigned w = out[k];
                    int r = -1;
                    unsigned char d = 255;
                    if (w != NONE) {
                        const int dz = (int)((w >> SH_Z) & 63u) - 31;
                        const int dy = (int)((w >> SH_Y) & 63u) - 31;
                        const int dx = (int)(w & 63u) - 31;
                        r = (int)(v + dx + (long long)g.nx * (dy + (long long)g.ny * dz));
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

cudaError_t launch_dilate(const unsigned *occ, const unsigned *boff, const GridGeom &g, int L, int *active,
                          int *root, unsigned char *ring, DevCtl *ctl, int sms, cudaStream_t st)
{
    const int tiles_x = (g.nx + TX - 1) / TX, tiles_y = (g.ny + TY - 1) / TY, tiles_z = (g.nz + TZ - 1) / TZ;
    const long long tiles = (long long)tiles_x * tiles_y * tiles_z;
    k_dilate_tiles<<<(unsigned)((tiles * 32 + 255) / 256), 256, 0, st>>>(boff, g, L, tiles_x, tiles_y, tiles, active,
                                                                         ctl, root, ring);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess)
        return e;
    const size_t smem = dilate_smem_bytes(L);
    if (smem > 48 * 1024) {   // opt in above the default limit (a per-device function attribute)
        e = cudaFuncSetAttribute(k_dilate, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess)
            return e;
    }
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_dilate, THREADS, smem);
    if (e != cudaSuccess)
        return e;
    long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
    if (grid > tiles)
        grid = tiles;
    k_dilate<<<(unsigned)grid, THREADS, smem, st>>>(occ, active, g, L, tiles_x, tiles_y, tiles, root, ring, ctl);
    return cudaGetLastError();
}

}  // namespace vicp
