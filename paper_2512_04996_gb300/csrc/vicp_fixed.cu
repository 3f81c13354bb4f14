// vicp_fixed.cu -- the fixed-capacity voxel store, kept as a measured
// alternative to the CSR store: every voxel owns C slots at v * C (direct
// addressing, the layout the paper's dynamic assignment replaces, Sec. 2.2),
// so a build is one counter reset and one scatter with no histogram and no
// scan; points past a voxel's C-th are dropped and counted.
#include "vicp_launch.h"

namespace vicp {

// A warp's points of one voxel take consecutive slots with one atomicAdd on
// the voxel's fill count (the same grouping as the CSR scatter); a slot at or
// past C is an overflow.  Slots hold (x, y, z, index) like the CSR points.
__global__ void __launch_bounds__(256) k_fixed_scatter(const float4 *__restrict__ pts, int n, GridGeom g, unsigned C,
                                                       unsigned *__restrict__ count, float4 *__restrict__ slots,
                                                       unsigned *__restrict__ overflow)
{
    pdl_begin();
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    int key = -2;
    float4 q = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j < n) {
        q = __ldg(pts + j);
        key = voxel_key(g, q.x, q.y, q.z);
        q.w = __int_as_float(j);
    }
    const unsigned peers = __match_any_sync(FULL_MASK, key);
    const int leader = __ffs(peers) - 1;
    const unsigned rank = __popc(peers & lanemask_lt());
    unsigned base = 0u;
    if (lane == leader && key >= 0)
        base = atomicAdd(count + key, (unsigned)__popc(peers));
    base = __shfl_sync(FULL_MASK, base, leader);
    const unsigned slot = base + rank;
    const bool over = key >= 0 && slot >= C;
    if (key >= 0 && !over)
        slots[(size_t)key * C + slot] = q;
    const unsigned om = __ballot_sync(FULL_MASK, over);
    if (lane == 0 && om)
        atomicAdd(overflow, (unsigned)__popc(om));
}

cudaError_t launch_fixed_scatter(const float4 *pts, int n, const GridGeom &g, unsigned C, unsigned *count,
                                 float4 *slots, unsigned *overflow, cudaStream_t st)
{
    return launch_kernel(k_fixed_scatter, dim3((n + 255) / 256), dim3(256), 0, st, pts, n, g, C, count, slots,
                         overflow);
}

}  // namespace vicp
