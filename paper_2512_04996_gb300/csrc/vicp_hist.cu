// vicp_hist.cu -- the voxel occupancy histogram (VOH, Alg. 1 GPU part) as a
// standalone ablation of two designs, both allocation-free:
//
//   warp-aggregated  lanes of a warp with the same voxel are grouped with
//                    __match_any_sync and one leader adds the group's size
//                    (the design the grid build uses);
//   shared hash      the paper's two-layer scheme: each block builds a hash
//                    table in shared memory (one slot per thread, slot = key
//                    modulo the block size, linear probing by atomicCAS,
//                    count by atomicAdd on the same packed word), then each
//                    thread flushes its slot to the global histogram with one
//                    atomicAdd.
//
// The paper packs the key into the upper 16 bits of a 32-bit word and uses
// the all-zero word as "empty", which limits grids to 2^16 voxels and makes
// voxel 0 indistinguishable from an empty slot.  Here the word is 64 bits,
// [key + 1 : 32 | count : 32]: the +1 keeps every key away from the empty
// word, and 32-bit keys cover any grid (a count never reaches 2^32 within
// one block, so adding 1 to the word never carries into the key).
#include <cmath>

#include "vicp.h"
#include "vicp_geom.h"
#include "vicp_launch.h"

namespace vicp {

constexpr int HIST_BLOCK = 256;

__global__ void __launch_bounds__(HIST_BLOCK) k_hist_warp(const float4 *__restrict__ pts, int n, GridGeom g,
                                                          int *__restrict__ keys, unsigned *__restrict__ counts)
{
    pdl_begin();
    const int j = blockIdx.x * HIST_BLOCK + threadIdx.x;
    int key = -2;   // lanes past the end match only each other and add nothing
    if (j < n) {
        const float4 q = __ldg(pts + j);
        key = voxel_key(g, q.x, q.y, q.z);
        keys[j] = key;
    }
    const unsigned peers = __match_any_sync(FULL_MASK, key);
    if (key >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1)
        atomicAdd(counts + key, (unsigned)__popc(peers));
}

__global__ void __launch_bounds__(HIST_BLOCK) k_hist_hash(const float4 *__restrict__ pts, int n, GridGeom g,
                                                          int *__restrict__ keys, unsigned *__restrict__ counts)
{
    pdl_begin();
    __shared__ unsigned long long s_tab[HIST_BLOCK];
    s_tab[threadIdx.x] = 0ull;
    __syncthreads();
    const int j = blockIdx.x * HIST_BLOCK + threadIdx.x;
    if (j < n) {
        const float4 q = __ldg(pts + j);
        const int key = voxel_key(g, q.x, q.y, q.z);
        keys[j] = key;
        if (key >= 0) {
            const unsigned long long tag = (unsigned long long)((unsigned)key + 1u) << 32;
            unsigned slot = (unsigned)key & (HIST_BLOCK - 1);
            // a block holds at most HIST_BLOCK distinct keys, so some slot is
            // free or already holds this key within HIST_BLOCK probes
            for (int probe = 0; probe < HIST_BLOCK; ++probe) {
                const unsigned long long prev = atomicCAS(&s_tab[slot], 0ull, tag);
                if (prev == 0ull || (prev >> 32) == (tag >> 32)) {
                    atomicAdd(&s_tab[slot], 1ull);
                    break;
                }
                slot = (slot + 1u) & (HIST_BLOCK - 1);
            }
        }
    }
    __syncthreads();
    const unsigned long long e = s_tab[threadIdx.x];
    if (e)
        atomicAdd(counts + ((e >> 32) - 1ull), (unsigned)(e & 0xffffffffull));
}

cudaError_t launch_voxel_histogram(const float4 *pts, int n, const GridGeom &g, int method, int *keys,
                                   unsigned *counts, cudaStream_t st)
{
    const dim3 grid((n + HIST_BLOCK - 1) / HIST_BLOCK);
    if (method == 1)
        return launch_kernel(k_hist_hash, grid, dim3(HIST_BLOCK), 0, st, pts, n, g, keys, counts);
    return launch_kernel(k_hist_warp, grid, dim3(HIST_BLOCK), 0, st, pts, n, g, keys, counts);
}

}  // namespace vicp

extern "C" VICP_API vicp_status vicp_voxel_histogram(const float *target_xyzw, int32_t n, const float origin[3],
                                                     float voxel_size, const int32_t dims[3], int32_t method,
                                                     int32_t *keys_out, uint32_t *counts_out, void *cuda_stream)
{
    using namespace vicp;
    if (!target_xyzw || n < 1 || !origin || !dims || !keys_out || !counts_out || (method != 0 && method != 1))
        return VICP_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(target_xyzw) & 15u) != 0 || (reinterpret_cast<uintptr_t>(keys_out) & 3u) != 0 ||
        (reinterpret_cast<uintptr_t>(counts_out) & 3u) != 0)
        return VICP_ERR_INVALID;
    if (!(voxel_size > 0.0f) || !std::isfinite(voxel_size))
        return VICP_ERR_INVALID;
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || !std::isfinite(origin[a]))
            return VICP_ERR_INVALID;
    if ((long long)dims[0] * dims[1] * dims[2] >= (1ll << 31) - 1)
        return VICP_ERR_GRID_TOO_LARGE;
    const int d[3] = {dims[0], dims[1], dims[2]};
    const GridGeom g = make_geom(origin, voxel_size, d);
    const cudaError_t e = launch_voxel_histogram(reinterpret_cast<const float4 *>(target_xyzw), n, g, method,
                                                 keys_out, counts_out, static_cast<cudaStream_t>(cuda_stream));
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VICP_ERR_CUDA;
    }
    return VICP_OK;
}
