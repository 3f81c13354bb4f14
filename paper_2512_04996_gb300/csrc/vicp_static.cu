// vicp_static.cu -- vicp_offsets_static: voxel keys and offsets with no device
// allocation.
//
// Some callers cannot allocate device memory where they call this library:
// code that runs after a fixed device-memory plan has been committed (for
// example a real-time loop that forbids allocation after start-up, because
// cudaMalloc can block and synchronise the device), or a plug-in running
// inside another framework that owns all device memory through its own
// allocator.  This entry point therefore uses only a scratch area that the
// library holds in static device memory: the per-voxel counts, occupancy
// bits, scan tile sums and descriptors, brick counts and a control block.
// The caller passes the inputs and the outputs.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "vicp.h"
#include "vicp_launch.h"

using namespace vicp;

namespace {

constexpr long long MAX_V = VICP_STATIC_MAX_VOXELS;
constexpr long long MAX_BRICK_SLOTS = VICP_STATIC_MAX_BRICK_SLOTS;

constexpr size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

// Scratch layout (bytes from the start of the array).
constexpr size_t OFF_CTL = 0;
constexpr size_t OFF_COUNTS = OFF_CTL + align256(sizeof(DevCtl));
constexpr size_t OFF_OCC = OFF_COUNTS + align256(MAX_V * 4);
constexpr size_t OFF_TILES = OFF_OCC + align256(((MAX_V + 31) / 32 + 2) * 4);
constexpr size_t OFF_DESC = OFF_TILES + align256(((MAX_V + SCAN_TILE - 1) / SCAN_TILE) * 4);
constexpr size_t OFF_BRICKS = OFF_DESC + align256(((MAX_V + SCAN_TILE - 1) / SCAN_TILE) * 8);
constexpr size_t SCRATCH_BYTES = OFF_BRICKS + align256(MAX_BRICK_SLOTS * 4);

// About 70 MiB, held on every GPU that loads the library until the process
// exits.  Host code never hands `g_scratch` itself to a kernel: kernels get
// the address that cudaGetSymbolAddress returns for the current device.
static __device__ __align__(256) unsigned char g_scratch[SCRATCH_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_setup_lock;
unsigned char *g_addr[MAX_DEVICES] = {};

// Device address of the scratch on the current device (looked up once per
// device, with that device current, and kept until the process exits: a
// cudaDeviceReset would leave a stale address behind, which the header
// rules out).
vicp_status scratch_address(unsigned char **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) {
        cudaGetLastError();
        return VICP_ERR_CUDA;
    }
    std::lock_guard<std::mutex> lock(g_setup_lock);
    if (!g_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return VICP_ERR_CUDA;
        }
        g_addr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_addr[dev];
    return VICP_OK;
}

}  // namespace

extern "C" VICP_API vicp_status vicp_offsets_static(const float *target_xyzw, int32_t n, const float origin[3],
                                                    float voxel_size, const int32_t dims[3], int32_t *keys_out,
                                                    uint32_t *offsets_out, void *cuda_stream)
{
    if (!target_xyzw || n < 1 || !origin || !dims || !keys_out || !offsets_out)
        return VICP_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(target_xyzw) & 15u) != 0 || (reinterpret_cast<uintptr_t>(keys_out) & 3u) != 0 ||
        (reinterpret_cast<uintptr_t>(offsets_out) & 15u) != 0)
        return VICP_ERR_INVALID;
    if (!(voxel_size > 0.0f) || !std::isfinite(voxel_size))
        return VICP_ERR_INVALID;
    for (int a = 0; a < 3; ++a)
        if (dims[a] < 1 || !std::isfinite(origin[a]))
            return VICP_ERR_INVALID;
    GridGeom g{};
    g.ox = origin[0];
    g.oy = origin[1];
    g.oz = origin[2];
    g.h = voxel_size;
    g.inv_h = (float)(1.0 / (double)voxel_size);
    g.nx = dims[0];
    g.ny = dims[1];
    g.nz = dims[2];
    g.V = (long long)dims[0] * dims[1] * dims[2];
    g.bx = (dims[0] + BRICK - 1) / BRICK;
    g.by = (dims[1] + BRICK - 1) / BRICK;
    g.bz = (dims[2] + BRICK - 1) / BRICK;
    g.sx = (g.bx + SUPER - 1) / SUPER;
    g.sy = (g.by + SUPER - 1) / SUPER;
    g.sz = (g.bz + SUPER - 1) / SUPER;
    if (g.V > MAX_V || (long long)g.sx * g.sy * g.sz * SUPER_BRICKS > MAX_BRICK_SLOTS)
        return VICP_ERR_GRID_TOO_LARGE;

    unsigned char *base = nullptr;
    vicp_status s = scratch_address(&base);
    if (s != VICP_OK)
        return s;
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    DevCtl *ctl = reinterpret_cast<DevCtl *>(base + OFF_CTL);
    unsigned *counts = reinterpret_cast<unsigned *>(base + OFF_COUNTS);
    unsigned *occ = reinterpret_cast<unsigned *>(base + OFF_OCC);
    unsigned *tiles = reinterpret_cast<unsigned *>(base + OFF_TILES);
    unsigned long long *desc = reinterpret_cast<unsigned long long *>(base + OFF_DESC);
    unsigned *bcounts = reinterpret_cast<unsigned *>(base + OFF_BRICKS);

    // The scratch keeps the last call's contents: clear everything that must
    // start at zero.
    const long long nt = scan_tiles(g.V);
    cudaError_t e = cudaMemsetAsync(ctl, 0, sizeof(DevCtl), st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(counts, 0, (size_t)g.V * 4, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(tiles, 0, (size_t)nt * 4, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(desc, 0, (size_t)nt * 8, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(bcounts, 0, (size_t)brick_slots(g) * 4, st);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(occ, 0, (size_t)occ_words(g.V) * 4, st);
    if (e == cudaSuccess)
        e = launch_histogram(reinterpret_cast<const float4 *>(target_xyzw), n, g, keys_out, counts, bcounts, occ,
                             tiles, nullptr, nullptr, ctl, st, false);
    if (e == cudaSuccess)
        e = launch_scan(counts, g, offsets_out, occ, tiles, desc, ctl, st, true);
    unsigned err = 0;
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&err, &ctl->err, sizeof err, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return VICP_ERR_CUDA;
    }
    if (err & DEVERR_TIMEOUT)
        return VICP_ERR_TIMEOUT;
    return err ? VICP_ERR_CUDA : VICP_OK;
}
