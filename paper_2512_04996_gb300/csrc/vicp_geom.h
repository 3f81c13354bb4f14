// vicp_geom.h -- host-side grid geometry (Sec. 2.2: the voxel grid over the
// target's bounding box, voxel edge h = extent / 2^N or given), shared by the
// single-pair context and the batched registration so that both fit the
// same grid to the same cloud.
#pragma once

#include <cmath>
#include <cstring>

#include "vicp_device.cuh"

namespace vicp {

// Inverse of the device's order-preserving float -> unsigned map.
inline float ordered_to_float_host(unsigned o)
{
    const unsigned b = (o & 0x80000000u) ? (o & 0x7fffffffu) : ~o;
    float f;
    std::memcpy(&f, &b, 4);
    return f;
}

enum GeomResult { GEOM_OK = 0, GEOM_NONFINITE = 1, GEOM_TOO_LARGE = 2 };

// Bounding-box grid from the box [lo, hi]: origin = lo, h = voxel_size when
// > 0, else extent / divisions (the largest side over the division count;
// h = 1 when every point coincides), and dims_a = floor(extent_a * inv_h) + 1
// with inv_h = (float)(1 / (double)h).  `axis` names the failing axis.
inline GeomResult fit_box(const float lo[3], const float hi[3], float voxel_size, int divisions, float *h_out,
                          int dims[3], int *axis)
{
    float ext[3], extent = 0.0f;
    for (int a = 0; a < 3; ++a) {
        if (!std::isfinite(lo[a]) || !std::isfinite(hi[a])) {
            *axis = a;
            return GEOM_NONFINITE;
        }
        ext[a] = hi[a] - lo[a];
        if (ext[a] > extent)
            extent = ext[a];
    }
    float h;
    if (voxel_size > 0.0f) {
        h = voxel_size;
    } else {
        h = extent / (float)divisions;
        if (!(h > 0.0f))
            h = 1.0f;   // all target points coincide: one voxel
    }
    const float inv_h = (float)(1.0 / (double)h);
    for (int a = 0; a < 3; ++a) {
        const float s = ext[a] * inv_h;
        if (!(s < 2147483520.0f)) {
            *axis = a;
            return GEOM_TOO_LARGE;
        }
        dims[a] = (int)std::floor(s) + 1;
    }
    *h_out = h;
    return GEOM_OK;
}

// The device geometry of a grid with the given origin, voxel edge and
// dimensions (checked by the caller: h finite > 0, dims >= 1, V < 2^31 - 1).
inline GridGeom make_geom(const float origin[3], float h, const int dims[3])
{
    GridGeom g{};
    g.ox = origin[0];
    g.oy = origin[1];
    g.oz = origin[2];
    g.h = h;
    g.inv_h = (float)(1.0 / (double)h);
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
    return g;
}

// Centre of the reduction: the grid centre, rounded to float.
inline float3 grid_center(const GridGeom &g)
{
    return make_float3((float)((double)g.ox + 0.5 * (double)g.h * g.nx), (float)((double)g.oy + 0.5 * (double)g.h * g.ny),
                       (float)((double)g.oz + 0.5 * (double)g.h * g.nz));
}

}  // namespace vicp
