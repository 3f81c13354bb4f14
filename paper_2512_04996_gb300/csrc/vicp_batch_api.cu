// vicp_batch_api.cu -- the batched-registration part of the C ABI declared
// in include/vicp.h: the pooled layout of many pairs, workspace allocation,
// the build and iteration launch sequences, the iteration graph and the
// autotuner.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "vicp.h"
#include "vicp_batch.h"
#include "vicp_geom.h"
#include "vicp_launch.h"

using namespace vicp;

namespace {

struct BBuf {
    void *p = nullptr;
    size_t bytes = 0;
};

}  // namespace

struct vicp_batch {
    vicp_batch_params params{};
    vicp_allocator alloc{};
    bool custom_alloc = false;
    cudaStream_t stream = nullptr;
    cudaStream_t capture = nullptr;   // private stream the iteration graph is captured on
    int device = 0;
    std::string last_error;
    uint64_t cur_bytes = 0, peak_bytes = 0;
    int64_t launches = 0;

    // layout of the last build
    bool built = false;
    bool off_dense = false;          // the build writes sparse offsets; vicp_batch_pair_grid completes them
    int P = 0;
    int N = 0;                       // pooled target points
    long long Vt = 0;                // pooled voxels (with alignment gaps)
    int Bt = 0;                      // pooled brick slots
    int n_titems = 0;
    int L = -1;
    const float4 *target = nullptr;
    std::vector<BatchPair> pairs;    // host copy of the descriptors
    std::vector<int> ustart_xy, ustart_z;
    std::vector<int> lab_dims;       // grids whose labels root/ring/dirty hold (empty: none)

    // iteration layout of the last register / correspond / tune
    int M = 0;
    int n_items = 0;
    int items_shape = -1;
    std::vector<int> n_src_last;
    int tuned_shape = -1;

    // iteration graph
    cudaGraphExec_t graph = nullptr;
    bool graph_broken = false;       // capture failed once: launch directly
    const void *g_src = nullptr;
    int g_shape = -1, g_iters = -1, g_M = -1, g_items = -1;
    double g_eps = 0.0;
    bool g_f64 = false;
    int last_graph = -1;             // the last registration's iterations: 1 graph replay, 0 direct

    // device buffers
    BBuf counts, off, root, ring, inter, occ, desc, tile_sum, rows, dirty;
    BBuf bcounts, boff, blist, brange, bslot, boxord, bbox, sb_box;
    BBuf keys, ids, csr, bpts, outside;
    BBuf nn, d2, fb_list, hv_list, partials, sitems;
    BBuf pairs_d, state, pose, pose_save, titems, ustart_xy_d, ustart_z_d, bb, ctl;
    BBuf hsrc, htgt;
};

namespace {

vicp_status bfail(vicp_batch *b, vicp_status s, const char *fmt, ...)
{
    if (b) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        b->last_error = buf;
    }
    return s;
}

vicp_status bcuda(vicp_batch *b, cudaError_t e, const char *what)
{
    return bfail(b, VICP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define BTRY(x)                      \
    do {                             \
        vicp_status _s = (x);        \
        if (_s != VICP_OK)           \
            return _s;               \
    } while (0)

#define BCUDA(b, call, what)                 \
    do {                                     \
        cudaError_t _e = (call);             \
        if (_e != cudaSuccess)               \
            return bcuda((b), _e, (what));   \
    } while (0)

void bfree(vicp_batch *b, BBuf &x)
{
    if (x.p) {
        if (b->custom_alloc)
            b->alloc.free(x.p, x.bytes, (void *)b->stream, b->alloc.user);
        else
            cudaFree(x.p);
        b->cur_bytes -= x.bytes;
    }
    x.p = nullptr;
    x.bytes = 0;
}

// Grows x to at least `bytes` (contents are not kept).  *fresh is set when
// a new allocation was made.
vicp_status bensure(vicp_batch *b, BBuf &x, size_t bytes, const char *what, bool *fresh = nullptr)
{
    if (bytes == 0)
        bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    if (fresh)
        *fresh = false;
    if (x.p && x.bytes >= bytes)
        return VICP_OK;
    bfree(b, x);
    void *p = nullptr;
    if (b->custom_alloc) {
        p = b->alloc.alloc(bytes, (void *)b->stream, b->alloc.user);
        if (!p)
            return bfail(b, VICP_ERR_OOM, "allocator returned NULL for %s (%zu bytes)", what, bytes);
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return bfail(b, VICP_ERR_OOM, "cudaMalloc of %zu bytes for %s: %s", bytes, what, cudaGetErrorString(e));
        }
    }
    x.p = p;
    x.bytes = bytes;
    b->cur_bytes += bytes;
    if (b->cur_bytes > b->peak_bytes)
        b->peak_bytes = b->cur_bytes;
    if (fresh)
        *fresh = true;
    return VICP_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

DevCtl *bctl(vicp_batch *b) { return static_cast<DevCtl *>(b->ctl.p); }

void drop_graph(vicp_batch *b)
{
    if (b->graph)
        cudaGraphExecDestroy(b->graph);
    b->graph = nullptr;
    b->g_shape = b->g_iters = b->g_M = b->g_items = -1;
    b->g_src = nullptr;
}

vicp_status check_counts(vicp_batch *b, const int32_t *n, int P, const char *what, long long *total)
{
    if (!n)
        return bfail(b, VICP_ERR_INVALID, "%s: NULL size array", what);
    long long t = 0;
    for (int k = 0; k < P; ++k) {
        if (n[k] < 1)
            return bfail(b, VICP_ERR_INVALID, "%s: pair %d has %d points (need >= 1)", what, k, n[k]);
        t += n[k];
    }
    if (t >= (1ll << 31) - 1)
        return bfail(b, VICP_ERR_INVALID, "%s: %lld points in all (limit 2^31 - 2)", what, t);
    *total = t;
    return VICP_OK;
}

// Reads the device status word, clears it, and maps it to a status.
vicp_status read_status(vicp_batch *b)
{
    unsigned err = 0;
    DevCtl *d = bctl(b);
    BCUDA(b, cudaMemcpyAsync(&err, &d->err, sizeof err, cudaMemcpyDeviceToHost, b->stream), "status read-back");
    BCUDA(b, cudaStreamSynchronize(b->stream), "synchronise");
    if (err) {
        cudaMemsetAsync(&d->err, 0, sizeof(unsigned), b->stream);
        if (err & DEVERR_TIMEOUT) {
            // a barrier gave up: its arrival count is no longer meaningful
            cudaMemsetAsync(&d->bar_count, 0, sizeof(unsigned), b->stream);
            return bfail(b, VICP_ERR_TIMEOUT, "a grid barrier of the iteration kernel gave up (status 0x%x)", err);
        }
        if (err & DEVERR_BOUNDS)
            return bfail(b, VICP_ERR_CUDA, "a device-side bounds check failed (device status 0x%x)", err);
        if (err & DEVERR_DEGENERATE)
            return VICP_ERR_DEGENERATE;   // per pair; the caller decides
    }
    return VICP_OK;
}

// --- build -----------------------------------------------------------------
vicp_status build(vicp_batch *b, int P, const float *tgt, const int32_t *n_tgt, const float *voxel_size,
                  const int32_t *divisions)
{
    if (P < 1 || P > VICP_BATCH_MAX_PAIRS)
        return bfail(b, VICP_ERR_INVALID, "n_pairs must be in [1, %d]", VICP_BATCH_MAX_PAIRS);
    if (!tgt || !aligned16(tgt))
        return bfail(b, VICP_ERR_INVALID, "targets: need a non-NULL 16-byte aligned pointer");
    long long N = 0;
    BTRY(check_counts(b, n_tgt, P, "targets", &N));
    for (int k = 0; k < P; ++k) {
        const bool vs = voxel_size && voxel_size[k] > 0.0f && std::isfinite(voxel_size[k]);
        if (!vs && (!divisions || divisions[k] < 1))
            return bfail(b, VICP_ERR_INVALID, "pair %d: need voxel_size > 0 or grid_divisions >= 1", k);
    }
    b->built = false;
    drop_graph(b);
    const int L = b->params.dilation_layers;
    cudaStream_t st = b->stream;

    // target tiles
    std::vector<BatchItem> titems;
    std::vector<int> tbase(P);
    {
        long long t = 0;
        for (int k = 0; k < P; ++k) {
            tbase[k] = (int)t;
            for (int l = 0; l < n_tgt[k]; l += BATCH_TILE)
                titems.push_back({k, (int)(t + l), (int)(t + std::min(l + BATCH_TILE, n_tgt[k])), l});
            t += n_tgt[k];
        }
    }
    const int n_titems = (int)titems.size();
    BTRY(bensure(b, b->titems, titems.size() * sizeof(BatchItem), "target tiles"));
    BCUDA(b, cudaMemcpyAsync(b->titems.p, titems.data(), titems.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, st),
          "tile upload");
    BTRY(bensure(b, b->bb, (size_t)6 * P * sizeof(unsigned), "bounding boxes"));

    // per-pair bounding boxes (one synchronisation)
    const float4 *t4 = reinterpret_cast<const float4 *>(tgt);
    BCUDA(b, launch_batch_bbox(t4, (const BatchItem *)b->titems.p, n_titems, P, (unsigned *)b->bb.p, st),
          "launch of the batched bounding box");
    b->launches += 1;
    std::vector<unsigned> hb((size_t)6 * P);
    BCUDA(b, cudaMemcpyAsync(hb.data(), b->bb.p, hb.size() * sizeof(unsigned), cudaMemcpyDeviceToHost, st),
          "bounding box read-back");
    BCUDA(b, cudaStreamSynchronize(st), "bounding box read-back");

    // per-pair grids and the pooled layout
    std::vector<BatchPair> pairs(P);
    std::vector<int> uxy(P + 1), uz(P + 1), dims_key;
    long long Vt = 0, Bt = 0, Uxy = 0, Uz = 0;
    for (int k = 0; k < P; ++k) {
        float lo[3], hi[3], h = 0.0f;
        for (int a = 0; a < 3; ++a) {
            lo[a] = ordered_to_float_host(hb[3 * k + a]);
            hi[a] = ordered_to_float_host(hb[3 * P + 3 * k + a]);
        }
        int dims[3], axis = 0;
        const float vs = voxel_size ? voxel_size[k] : 0.0f;
        const GeomResult r = fit_box(lo, hi, vs, divisions ? divisions[k] : 0, &h, dims, &axis);
        if (r == GEOM_NONFINITE)
            return bfail(b, VICP_ERR_INVALID, "pair %d: target has no finite coordinate on axis %d", k, axis);
        if (r == GEOM_TOO_LARGE)
            return bfail(b, VICP_ERR_GRID_TOO_LARGE, "pair %d: grid axis %d would be too long", k, axis);
        const long long V = (long long)dims[0] * dims[1] * dims[2];
        if (V >= (1ll << 31) - 1)
            return bfail(b, VICP_ERR_GRID_TOO_LARGE, "pair %d: grid of %lld voxels", k, V);
        BatchPair &bp = pairs[k];
        std::memset(&bp, 0, sizeof bp);
        bp.g = make_geom(lo, h, dims);
        bp.vbase = Vt;
        bp.tbase = tbase[k];
        bp.n_tgt = n_tgt[k];
        bp.bbase = (int)Bt;
        bp.sbbase = (int)(Bt / SUPER_BRICKS);
        bp.uxy = (int)Uxy;
        bp.uz = (int)Uz;
        const float3 c = grid_center(bp.g);
        bp.cx = c.x;
        bp.cy = c.y;
        bp.cz = c.z;
        uxy[k] = (int)Uxy;
        uz[k] = (int)Uz;
        Vt += (V + 31) / 32 * 32;
        Bt += brick_slots(bp.g);
        Uxy += dilate_units(bp.g);
        Uz += dilate_column_units(bp.g);
        if (Vt >= (1ll << 31) - 1 || Bt >= (1ll << 31) - 1 || Uxy >= (1ll << 31) - 1 || Uz >= (1ll << 31) - 1)
            return bfail(b, VICP_ERR_GRID_TOO_LARGE, "pairs 0..%d: %lld voxels in all (limit 2^31 - 2)", k, Vt);
        dims_key.insert(dims_key.end(), {dims[0], dims[1], dims[2]});
    }
    uxy[P] = (int)Uxy;
    uz[P] = (int)Uz;

    // workspace (grown, never shrunk); arrays that must start at zero are
    // cleared when new and kept at zero by the kernels (counts, brick counts
    // and tile totals by the scatter) or cleared per build (occupancy)
    bool fresh = false;
    BTRY(bensure(b, b->counts, (size_t)Vt * 4, "counts", &fresh));
    if (fresh)
        BCUDA(b, cudaMemsetAsync(b->counts.p, 0, b->counts.bytes, st), "zero counts");
    BTRY(bensure(b, b->off, (size_t)(Vt + 1) * 4, "offsets"));
    bool fresh_lab = false, f2 = false, f3 = false;
    BTRY(bensure(b, b->root, (size_t)Vt * 4, "root", &fresh_lab));
    BTRY(bensure(b, b->ring, (size_t)Vt, "ring", &f2));
    BTRY(bensure(b, b->inter, (size_t)Vt * (L <= 15 ? 2 : 4), "dilation pass-Y words"));
    BTRY(bensure(b, b->occ, (size_t)occ_words(Vt) * 4, "occupancy"));
    BTRY(bensure(b, b->desc, (size_t)scan_tiles(Vt) * 8, "scan descriptors", &fresh));
    if (fresh)
        BCUDA(b, cudaMemsetAsync(b->desc.p, 0, b->desc.bytes, st), "zero descriptors");
    BTRY(bensure(b, b->tile_sum, (size_t)scan_tiles(Vt) * 4, "scan tile sums", &fresh));
    if (fresh)
        BCUDA(b, cudaMemsetAsync(b->tile_sum.p, 0, b->tile_sum.bytes, st), "zero tile sums");
    BTRY(bensure(b, b->rows, (size_t)Uxy * 4, "dilation row masks"));
    BTRY(bensure(b, b->dirty, (size_t)Uz, "dilation label flags", &f3));
    fresh_lab = fresh_lab || f2 || f3;
    BTRY(bensure(b, b->bcounts, (size_t)Bt * 4, "brick counts", &fresh));
    if (fresh)
        BCUDA(b, cudaMemsetAsync(b->bcounts.p, 0, b->bcounts.bytes, st), "zero brick counts");
    BTRY(bensure(b, b->boff, (size_t)Bt * 4, "brick offsets"));
    BTRY(bensure(b, b->blist, (size_t)Bt * 4, "brick list"));
    BTRY(bensure(b, b->brange, (size_t)Bt * 8, "brick ranges"));
    BTRY(bensure(b, b->bslot, (size_t)Bt * 4, "brick slots"));
    BTRY(bensure(b, b->boxord, (size_t)Bt * 32, "brick box bounds"));
    BTRY(bensure(b, b->bbox, (size_t)Bt * 32, "brick boxes"));
    BTRY(bensure(b, b->sb_box, (size_t)(Bt / SUPER_BRICKS + 1) * 32, "super-brick boxes"));
    BTRY(bensure(b, b->keys, (size_t)N * 4, "keys"));
    BTRY(bensure(b, b->ids, (size_t)N * 4, "ids"));
    BTRY(bensure(b, b->csr, (size_t)N * 16, "csr points"));
    BTRY(bensure(b, b->bpts, (size_t)N * 16, "brick points"));
    BTRY(bensure(b, b->outside, (size_t)N * 4, "outside lists"));
    BTRY(bensure(b, b->pairs_d, (size_t)P * sizeof(BatchPair), "pair descriptors"));
    BTRY(bensure(b, b->state, (size_t)P * sizeof(BatchState), "pair states"));
    BTRY(bensure(b, b->ustart_xy_d, (size_t)(P + 1) * 4, "unit starts"));
    BTRY(bensure(b, b->ustart_z_d, (size_t)(P + 1) * 4, "unit starts"));

    BCUDA(b, cudaMemcpyAsync(b->pairs_d.p, pairs.data(), (size_t)P * sizeof(BatchPair), cudaMemcpyHostToDevice, st),
          "descriptor upload");
    BCUDA(b, cudaMemcpyAsync(b->ustart_xy_d.p, uxy.data(), (size_t)(P + 1) * 4, cudaMemcpyHostToDevice, st),
          "unit start upload");
    BCUDA(b, cudaMemcpyAsync(b->ustart_z_d.p, uz.data(), (size_t)(P + 1) * 4, cudaMemcpyHostToDevice, st),
          "unit start upload");
    BCUDA(b, cudaMemsetAsync(b->state.p, 0, (size_t)P * sizeof(BatchState), st), "state reset");
    BCUDA(b, cudaMemsetAsync(b->occ.p, 0, (size_t)occ_words(Vt) * 4, st), "zero occupancy");

    DevCtl *d = bctl(b);
    const BatchPair *pd = (const BatchPair *)b->pairs_d.p;
    const BatchItem *ti = (const BatchItem *)b->titems.p;
    BCUDA(b, launch_batch_histogram(t4, ti, n_titems, pd, (int *)b->keys.p, (unsigned *)b->counts.p,
                                    (unsigned *)b->bcounts.p, (unsigned *)b->occ.p, (unsigned *)b->tile_sum.p, d, st),
          "launch of the batched histogram");
    GridGeom gall{};
    gall.V = Vt;
    BCUDA(b, launch_scan((const unsigned *)b->counts.p, gall, (unsigned *)b->off.p, (const unsigned *)b->occ.p,
                         (const unsigned *)b->tile_sum.p, (unsigned long long *)b->desc.p, d, st, false),
          "launch of the scan");
    b->off_dense = false;
    BCUDA(b, launch_batch_brick_scan((const unsigned *)b->bcounts.p, pd, P, (const unsigned *)b->off.p,
                                     (unsigned *)b->boff.p, (int *)b->blist.p, (uint2 *)b->brange.p,
                                     (int *)b->bslot.p, (uint4 *)b->boxord.p, (BatchState *)b->state.p, st),
          "launch of the batched brick scan");
    BCUDA(b, launch_batch_scatter(t4, (const int *)b->keys.p, ti, n_titems, pd, (int)N, (const unsigned *)b->off.p,
                                  (unsigned *)b->counts.p, (const unsigned *)b->boff.p, (unsigned *)b->bcounts.p,
                                  (const int *)b->bslot.p, (unsigned *)b->boxord.p, (int *)b->ids.p,
                                  (float4 *)b->csr.p, (float4 *)b->bpts.p, (int *)b->outside.p,
                                  (unsigned *)b->tile_sum.p, (int)scan_tiles(Vt), (BatchState *)b->state.p, d, st),
          "launch of the batched scatter");
    BCUDA(b, launch_batch_brick_boxes((const uint4 *)b->boxord.p, (const int *)b->blist.p,
                                      (const uint2 *)b->brange.p, pd, P, (BatchState *)b->state.p,
                                      (float4 *)b->bbox.p, (float4 *)b->sb_box.p, st),
          "launch of the batched brick boxes");
    // labels: cleared in full when the arrays are new or any grid changed
    if (fresh_lab || b->lab_dims != dims_key) {
        BCUDA(b, cudaMemsetAsync(b->root.p, 0xff, (size_t)Vt * 4, st), "clear root");
        BCUDA(b, cudaMemsetAsync(b->ring.p, 0xff, (size_t)Vt, st), "clear ring");
        BCUDA(b, cudaMemsetAsync(b->dirty.p, 0, (size_t)Uz, st), "clear label flags");
        b->lab_dims = dims_key;
    }
    BCUDA(b, launch_batch_dilate((const unsigned *)b->occ.p, pd, P, (const int *)b->ustart_xy_d.p,
                                 (const int *)b->ustart_z_d.p, L, b->inter.p, (unsigned *)b->rows.p,
                                 (unsigned char *)b->dirty.p, (int *)b->root.p, (unsigned char *)b->ring.p, st),
          "launch of the batched dilation");
    b->launches += 7;

    b->P = P;
    b->N = (int)N;
    b->Vt = Vt;
    b->Bt = (int)Bt;
    b->n_titems = n_titems;
    b->L = L;
    b->target = t4;
    b->pairs = pairs;
    b->ustart_xy = uxy;
    b->ustart_z = uz;
    b->items_shape = -1;
    b->n_src_last.clear();
    b->built = true;
    return VICP_OK;
}

// --- iterations ------------------------------------------------------------
int pick_shape(vicp_batch *b)
{
    if (b->params.shape >= 0 && b->params.shape < BATCH_N_SHAPES)
        return b->params.shape;
    return b->tuned_shape >= 0 ? b->tuned_shape : 0;
}

// Source tiles of `shape` for these sizes; uploads the items and the pair
// descriptors' item ranges when they changed.
vicp_status prepare_items(vicp_batch *b, const int32_t *n_src, int shape)
{
    const int P = b->P;
    long long M = 0;
    BTRY(check_counts(b, n_src, P, "sources", &M));
    const std::vector<int> ns(n_src, n_src + P);
    if (shape == b->items_shape && ns == b->n_src_last)
        return VICP_OK;
    const int T = BATCH_SHAPES[shape].threads * BATCH_SHAPES[shape].ppt;
    std::vector<BatchItem> items;
    long long s = 0;
    for (int k = 0; k < P; ++k) {
        BatchPair &bp = b->pairs[k];
        bp.sbase = (int)s;
        bp.n_src = n_src[k];
        bp.item0 = (int)items.size();
        for (int l = 0; l < n_src[k]; l += T)
            items.push_back({k, (int)(s + l), (int)(s + std::min(l + T, n_src[k])), l});
        bp.n_items = (int)items.size() - bp.item0;
        s += n_src[k];
    }
    cudaStream_t st = b->stream;
    BTRY(bensure(b, b->sitems, items.size() * sizeof(BatchItem), "source tiles"));
    BTRY(bensure(b, b->partials, items.size() * REDUCE_VALUES * sizeof(float2), "item sums"));
    BTRY(bensure(b, b->nn, (size_t)M * 4, "nn"));
    BTRY(bensure(b, b->d2, (size_t)M * 4, "d2"));
    BTRY(bensure(b, b->fb_list, (size_t)M * sizeof(int2), "global-search list"));
    BTRY(bensure(b, b->hv_list, (size_t)M * sizeof(int4), "dense segment list"));
    BCUDA(b, cudaMemcpyAsync(b->sitems.p, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice, st),
          "tile upload");
    BCUDA(b, cudaMemcpyAsync(b->pairs_d.p, b->pairs.data(), (size_t)P * sizeof(BatchPair), cudaMemcpyHostToDevice, st),
          "descriptor upload");
    BCUDA(b, cudaStreamSynchronize(st), "tile upload");   // the host vectors go out of scope
    b->M = (int)M;
    b->n_items = (int)items.size();
    b->items_shape = shape;
    b->n_src_last = ns;
    return VICP_OK;
}

// Loop state of every pair (items_done .. last_rmse) and the search lists.
vicp_status reset_loop(vicp_batch *b)
{
    cudaStream_t st = b->stream;
    BCUDA(b,
          cudaMemset2DAsync((char *)b->state.p + offsetof(BatchState, items_done), sizeof(BatchState), 0,
                            sizeof(BatchState) - offsetof(BatchState, items_done), b->P, st),
          "loop state reset");
    DevCtl *d = bctl(b);
    BCUDA(b, cudaMemsetAsync(&d->fb_count, 0, sizeof(int), st), "list reset");
    BCUDA(b, cudaMemsetAsync(&d->hv_count, 0, sizeof(int), st), "list reset");
    BCUDA(b, cudaMemsetAsync(&d->bar_count, 0, sizeof(unsigned), st), "barrier reset");
    BCUDA(b, cudaMemsetAsync(&d->fb_next, 0, sizeof(unsigned), st), "ticket reset");
    return VICP_OK;
}

BatchIterArgs iter_args(vicp_batch *b, const float4 *src, double *pose, int *nn, float *d2, int search_only)
{
    BatchIterArgs a{};
    a.src = src;
    a.tgt = b->target;
    a.pairs = (const BatchPair *)b->pairs_d.p;
    a.state = (BatchState *)b->state.p;
    a.pose = pose;
    a.items = (const BatchItem *)b->sitems.p;
    a.n_items = b->n_items;
    a.n_pairs = b->P;
    a.n_stored = b->N;
    a.root = (const int *)b->root.p;
    a.off = (const unsigned *)b->off.p;
    a.csr = (const float4 *)b->csr.p;
    a.bpts = (const float4 *)b->bpts.p;
    a.bbox = (const float4 *)b->bbox.p;
    a.sb_box = (const float4 *)b->sb_box.p;
    a.outside = (const int *)b->outside.p;
    a.nn = nn;
    a.d2 = d2;
    a.fb_list = (int2 *)b->fb_list.p;
    a.hv_list = (int4 *)b->hv_list.p;
    a.list_cap = b->M;
    a.partials = (float2 *)b->partials.p;
    a.ctl = bctl(b);
    a.eps = b->params.rmse_eps;
    a.search_only = search_only;
    a.test_leave_early = (b->params.flags & VICP_BATCH_FLAG_TEST_BARRIER_TIMEOUT) ? 1 : 0;
    return a;
}

// FP64 sums and solve (VICP_BATCH_FLAG_FP64) for this context's iterations.
bool fp64_of(const vicp_batch *b) { return (b->params.flags & VICP_BATCH_FLAG_FP64) != 0; }

// `blocks`: batch_iter_blocks(shape, f64), queried by the caller outside any
// stream capture.
vicp_status launch_iters(vicp_batch *b, int shape, bool f64, int blocks, const BatchIterArgs &a, int iters,
                         cudaStream_t st)
{
    if (blocks < 1)
        return bfail(b, VICP_ERR_CUDA, "iteration kernel shape %d cannot be resident", shape);
    for (int k = 0; k < iters; ++k)
        BCUDA(b, launch_batch_iter(shape, f64, blocks, a, st), "launch of the batched iteration");
    b->launches += iters;
    return VICP_OK;
}

// All iterations: replayed from a captured graph (captured again whenever the
// launch parameters change), or launched one by one.
vicp_status run_iterations(vicp_batch *b, int shape, const float4 *src)
{
    const int iters = b->params.max_iters;
    if (iters == 0)
        return VICP_OK;
    const BatchIterArgs a = iter_args(b, src, (double *)b->pose.p, (int *)b->nn.p, (float *)b->d2.p, 0);
    const bool f64 = fp64_of(b);
    const int blocks = batch_iter_blocks(shape, f64);
    b->last_graph = 0;
    if ((b->params.flags & VICP_BATCH_FLAG_NO_GRAPH) || b->graph_broken)
        return launch_iters(b, shape, f64, blocks, a, iters, b->stream);
    if (!b->graph || b->g_src != src || b->g_shape != shape || b->g_iters != iters || b->g_M != b->M ||
        b->g_items != b->n_items || b->g_eps != b->params.rmse_eps || b->g_f64 != f64) {
        drop_graph(b);
        if (!b->capture)
            BCUDA(b, cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking), "capture stream");
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const int64_t before = b->launches;
            const vicp_status s = launch_iters(b, shape, f64, blocks, a, iters, b->capture);
            b->launches = before;   // counted when replayed
            e = cudaStreamEndCapture(b->capture, &g);
            if (s != VICP_OK && e == cudaSuccess)
                e = cudaErrorStreamCaptureInvalidated;
        }
        if (e == cudaSuccess)
            e = cudaGraphInstantiate(&b->graph, g, 0);
        if (g)
            cudaGraphDestroy(g);
        if (e != cudaSuccess) {
            // capture of cooperative launches unavailable: launch directly from now on
            cudaGetLastError();
            b->graph = nullptr;
            b->graph_broken = true;
            return launch_iters(b, shape, f64, blocks, a, iters, b->stream);
        }
        b->g_src = src;
        b->g_shape = shape;
        b->g_iters = iters;
        b->g_M = b->M;
        b->g_items = b->n_items;
        b->g_eps = b->params.rmse_eps;
        b->g_f64 = f64;
    }
    BCUDA(b, cudaGraphLaunch(b->graph, b->stream), "graph launch");
    b->launches += iters;
    b->last_graph = 1;
    return VICP_OK;
}

vicp_status registration(vicp_batch *b, const float *src, const int32_t *n_src, double *poses, int32_t *iters_out,
                         double *rmse_out, int32_t *status_out)
{
    if (!b->built)
        return bfail(b, VICP_ERR_STATE, "vicp_batch_register before vicp_batch_build");
    if (!src || !aligned16(src))
        return bfail(b, VICP_ERR_INVALID, "sources: need a non-NULL 16-byte aligned pointer");
    if (!poses)
        return bfail(b, VICP_ERR_INVALID, "poses: NULL");
    const int P = b->P;
    const int shape = pick_shape(b);
    BTRY(prepare_items(b, n_src, shape));
    cudaStream_t st = b->stream;
    BTRY(bensure(b, b->pose, (size_t)P * 16 * sizeof(double), "poses"));
    BCUDA(b, cudaMemcpyAsync(b->pose.p, poses, (size_t)P * 16 * sizeof(double), cudaMemcpyHostToDevice, st),
          "pose upload");
    BTRY(reset_loop(b));
    BTRY(run_iterations(b, shape, reinterpret_cast<const float4 *>(src)));
    std::vector<BatchState> hs(P);
    BCUDA(b, cudaMemcpyAsync(poses, b->pose.p, (size_t)P * 16 * sizeof(double), cudaMemcpyDeviceToHost, st),
          "pose read-back");
    BCUDA(b, cudaMemcpyAsync(hs.data(), b->state.p, (size_t)P * sizeof(BatchState), cudaMemcpyDeviceToHost, st),
          "state read-back");
    vicp_status s = read_status(b);   // synchronises
    if (s != VICP_OK && s != VICP_ERR_DEGENERATE)
        return s;
    bool degenerate = false;
    for (int k = 0; k < P; ++k) {
        const bool dg = (hs[k].err & DEVERR_DEGENERATE) != 0;
        degenerate = degenerate || dg;
        if (iters_out)
            iters_out[k] = hs[k].iters;
        if (rmse_out)
            rmse_out[k] = hs[k].last_rmse;
        if (status_out)
            status_out[k] = dg ? VICP_ERR_DEGENERATE : VICP_OK;
    }
    if (degenerate && !status_out)
        return bfail(b, VICP_ERR_DEGENERATE, "rank(H) < 2 for at least one pair");
    return VICP_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

void vicp_batch_default_params(vicp_batch_params *p)
{
    if (!p)
        return;
    std::memset(p, 0, sizeof *p);
    p->dilation_layers = 10;
    p->max_iters = 40;
    p->rmse_eps = 0.0;
    p->shape = -1;
    p->flags = 0u;
}

vicp_status vicp_batch_shape_info(int32_t shape, int32_t *threads, int32_t *points_per_thread,
                                  int32_t *resident_blocks)
{
    if (shape < 0 || shape >= BATCH_N_SHAPES)
        return VICP_ERR_INVALID;
    if (threads)
        *threads = BATCH_SHAPES[shape].threads;
    if (points_per_thread)
        *points_per_thread = BATCH_SHAPES[shape].ppt;
    if (resident_blocks)
        *resident_blocks = batch_iter_blocks(shape, false);
    return VICP_OK;
}

vicp_status vicp_batch_create(vicp_batch **out, const vicp_batch_params *params, const vicp_allocator *alloc,
                              void *cuda_stream)
{
    if (!out || !params)
        return VICP_ERR_INVALID;
    *out = nullptr;
    if (alloc && (!alloc->alloc || !alloc->free))
        return VICP_ERR_INVALID;
    if (params->dilation_layers < 0 || params->dilation_layers > DILATE_MAX_L || params->max_iters < 0 ||
        params->shape >= BATCH_N_SHAPES)
        return VICP_ERR_INVALID;
    vicp_batch *b = new vicp_batch();
    b->params = *params;
    if (alloc) {
        b->alloc = *alloc;
        b->custom_alloc = true;
    }
    b->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&b->device);
    if (bensure(b, b->ctl, sizeof(DevCtl), "control block") != VICP_OK ||
        cudaMemsetAsync(b->ctl.p, 0, sizeof(DevCtl), b->stream) != cudaSuccess ||
        cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        vicp_batch_destroy(b);
        return VICP_ERR_CUDA;
    }
    *out = b;
    return VICP_OK;
}

void vicp_batch_destroy(vicp_batch *b)
{
    if (!b)
        return;
    cudaStreamSynchronize(b->stream);
    drop_graph(b);
    if (b->capture)
        cudaStreamDestroy(b->capture);
    BBuf *all[] = {&b->counts, &b->off, &b->root, &b->ring, &b->inter, &b->occ, &b->desc, &b->tile_sum, &b->rows,
                   &b->dirty, &b->bcounts, &b->boff, &b->blist, &b->brange, &b->bslot, &b->boxord, &b->bbox,
                   &b->sb_box, &b->keys, &b->ids, &b->csr, &b->bpts, &b->outside, &b->nn, &b->d2, &b->fb_list,
                   &b->hv_list, &b->partials, &b->sitems, &b->pairs_d, &b->state, &b->pose, &b->pose_save,
                   &b->titems, &b->ustart_xy_d, &b->ustart_z_d, &b->bb, &b->ctl, &b->hsrc, &b->htgt};
    for (BBuf *x : all)
        bfree(b, *x);
    delete b;
}

vicp_status vicp_batch_build(vicp_batch *b, int32_t n_pairs, const float *tgt_xyzw, const int32_t *n_tgt,
                             const float *voxel_size, const int32_t *grid_divisions)
{
    if (!b)
        return VICP_ERR_INVALID;
    return build(b, n_pairs, tgt_xyzw, n_tgt, voxel_size, grid_divisions);
}

vicp_status vicp_batch_register(vicp_batch *b, const float *src_xyzw, const int32_t *n_src, double *poses,
                                int32_t *iters_out, double *rmse_out, int32_t *status_out)
{
    if (!b)
        return VICP_ERR_INVALID;
    return registration(b, src_xyzw, n_src, poses, iters_out, rmse_out, status_out);
}

vicp_status vicp_batch_register_host(vicp_batch *b, int32_t n_pairs, const float *src_xyzw_host,
                                     const int32_t *n_src, const float *tgt_xyzw_host, const int32_t *n_tgt,
                                     const float *voxel_size, const int32_t *grid_divisions, double *poses,
                                     int32_t *iters_out, double *rmse_out, int32_t *status_out)
{
    if (!b)
        return VICP_ERR_INVALID;
    if (!src_xyzw_host || !tgt_xyzw_host || n_pairs < 1 || n_pairs > VICP_BATCH_MAX_PAIRS)
        return bfail(b, VICP_ERR_INVALID, "vicp_batch_register_host: bad arguments");
    long long M = 0, N = 0;
    BTRY(check_counts(b, n_src, n_pairs, "sources", &M));
    BTRY(check_counts(b, n_tgt, n_pairs, "targets", &N));
    BTRY(bensure(b, b->hsrc, (size_t)M * 16, "source copy"));
    BTRY(bensure(b, b->htgt, (size_t)N * 16, "target copy"));
    BCUDA(b, cudaMemcpyAsync(b->hsrc.p, src_xyzw_host, (size_t)M * 16, cudaMemcpyHostToDevice, b->stream),
          "source upload");
    BCUDA(b, cudaMemcpyAsync(b->htgt.p, tgt_xyzw_host, (size_t)N * 16, cudaMemcpyHostToDevice, b->stream),
          "target upload");
    BTRY(build(b, n_pairs, (const float *)b->htgt.p, n_tgt, voxel_size, grid_divisions));
    return registration(b, (const float *)b->hsrc.p, n_src, poses, iters_out, rmse_out, status_out);
}

vicp_status vicp_batch_correspond(vicp_batch *b, const float *src_xyzw, const int32_t *n_src,
                                  const double *poses_dev, int32_t *nn_out, float *d2_out)
{
    if (!b)
        return VICP_ERR_INVALID;
    if (!b->built)
        return bfail(b, VICP_ERR_STATE, "vicp_batch_correspond before vicp_batch_build");
    if (!src_xyzw || !aligned16(src_xyzw) || !poses_dev || !nn_out || !d2_out)
        return bfail(b, VICP_ERR_INVALID, "vicp_batch_correspond: NULL or misaligned pointer");
    const int shape = pick_shape(b);
    BTRY(prepare_items(b, n_src, shape));
    BTRY(reset_loop(b));
    const BatchIterArgs a = iter_args(b, reinterpret_cast<const float4 *>(src_xyzw), const_cast<double *>(poses_dev),
                                      nn_out, d2_out, 1);
    BTRY(launch_iters(b, shape, false, batch_iter_blocks(shape, false), a, 1, b->stream));   // search only
    const vicp_status s = read_status(b);
    return s == VICP_ERR_DEGENERATE ? VICP_OK : s;
}

vicp_status vicp_batch_tune(vicp_batch *b, const float *src_xyzw, const int32_t *n_src, const double *poses,
                            int32_t iters, int32_t trials, int32_t *shape_out, float *ms_out)
{
    if (!b)
        return VICP_ERR_INVALID;
    if (!b->built)
        return bfail(b, VICP_ERR_STATE, "vicp_batch_tune before vicp_batch_build");
    if (!src_xyzw || !aligned16(src_xyzw) || !poses || iters < 1 || trials < 1)
        return bfail(b, VICP_ERR_INVALID, "vicp_batch_tune: bad arguments");
    const int P = b->P;
    cudaStream_t st = b->stream;
    BTRY(bensure(b, b->pose, (size_t)P * 16 * sizeof(double), "poses"));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    BCUDA(b, cudaEventCreate(&e0), "event");
    BCUDA(b, cudaEventCreate(&e1), "event");
    int best = -1;
    float best_ms = 0.0f;
    vicp_status s = VICP_OK;
    for (int shape = 0; shape < BATCH_N_SHAPES && s == VICP_OK; ++shape) {
        float ms = -1.0f;
        if (batch_iter_blocks(shape, fp64_of(b)) > 0) {
            s = prepare_items(b, n_src, shape);
            for (int t = 0; t < trials && s == VICP_OK; ++t) {
                if (cudaMemcpyAsync(b->pose.p, poses, (size_t)P * 16 * sizeof(double), cudaMemcpyHostToDevice, st) !=
                    cudaSuccess) {
                    s = bfail(b, VICP_ERR_CUDA, "pose upload");
                    break;
                }
                s = reset_loop(b);
                if (s != VICP_OK)
                    break;
                const BatchIterArgs a =
                    iter_args(b, reinterpret_cast<const float4 *>(src_xyzw), (double *)b->pose.p, (int *)b->nn.p,
                              (float *)b->d2.p, 0);
                const int blocks = batch_iter_blocks(shape, fp64_of(b));
                cudaEventRecord(e0, st);
                s = launch_iters(b, shape, fp64_of(b), blocks, a, iters, st);
                cudaEventRecord(e1, st);
                if (s != VICP_OK)
                    break;
                float t_ms = 0.0f;
                if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(&t_ms, e0, e1) != cudaSuccess) {
                    s = bfail(b, VICP_ERR_CUDA, "tuning timing");
                    break;
                }
                if (ms < 0.0f || t_ms < ms)
                    ms = t_ms;
            }
            if (s == VICP_OK) {
                s = read_status(b);
                if (s == VICP_ERR_DEGENERATE)
                    s = VICP_OK;
            }
            if (s == VICP_OK && (best < 0 || ms < best_ms)) {
                best = shape;
                best_ms = ms;
            }
        }
        if (ms_out)
            ms_out[shape] = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s != VICP_OK)
        return s;
    if (best < 0)
        return bfail(b, VICP_ERR_CUDA, "no iteration kernel shape can run on this device");
    b->tuned_shape = best;
    if (shape_out)
        *shape_out = best;
    return VICP_OK;
}

vicp_status vicp_batch_pair_grid(vicp_batch *b, int32_t pair, vicp_grid_view *out)
{
    if (!b || !out)
        return VICP_ERR_INVALID;
    if (!b->built)
        return bfail(b, VICP_ERR_STATE, "vicp_batch_pair_grid before vicp_batch_build");
    if (pair < 0 || pair >= b->P)
        return bfail(b, VICP_ERR_INVALID, "pair %d out of range", pair);
    const BatchPair &bp = b->pairs[pair];
    if (!b->off_dense) {   // complete the pooled offsets once per build
        BCUDA(b, launch_offsets_fill((unsigned *)b->off.p, (const unsigned *)b->occ.p, b->Vt, b->stream),
              "launch of the offsets fill");
        b->launches += 1;
        b->off_dense = true;
    }
    unsigned ends[2] = {0u, 0u};
    const unsigned *off = (const unsigned *)b->off.p + bp.vbase;
    BCUDA(b, cudaMemcpyAsync(&ends[0], off, 4, cudaMemcpyDeviceToHost, b->stream), "offset read-back");
    BCUDA(b, cudaMemcpyAsync(&ends[1], off + bp.g.V, 4, cudaMemcpyDeviceToHost, b->stream), "offset read-back");
    BCUDA(b, cudaStreamSynchronize(b->stream), "offset read-back");
    std::memset(out, 0, sizeof *out);
    out->origin[0] = bp.g.ox;
    out->origin[1] = bp.g.oy;
    out->origin[2] = bp.g.oz;
    out->voxel_size = bp.g.h;
    out->inv_voxel_size = bp.g.inv_h;
    out->dims[0] = bp.g.nx;
    out->dims[1] = bp.g.ny;
    out->dims[2] = bp.g.nz;
    out->n_voxels = bp.g.V;
    out->n_target = bp.n_tgt;
    out->n_stored = (int32_t)(ends[1] - ends[0]);
    out->dilation_layers = b->L;
    out->keys = (const int32_t *)b->keys.p + bp.tbase;
    out->offsets = off;
    out->ids = (const int32_t *)b->ids.p;
    out->csr_points = (const float *)b->csr.p;
    out->root = (const int32_t *)b->root.p + bp.vbase;
    out->ring = (const uint8_t *)b->ring.p + bp.vbase;
    out->occupancy = (const uint32_t *)b->occ.p + bp.vbase / 32;
    return VICP_OK;
}

vicp_status vicp_batch_report(vicp_batch *b, uint64_t *current_bytes, uint64_t *peak_bytes, vicp_stats *stats,
                              int32_t reset)
{
    if (!b)
        return VICP_ERR_INVALID;
    if (current_bytes)
        *current_bytes = b->cur_bytes;
    if (peak_bytes)
        *peak_bytes = b->peak_bytes;
    if (stats || reset) {
        DevCtl *d = bctl(b);
        unsigned long long v[4];
        BCUDA(b, cudaMemcpyAsync(v, &d->stat_queries, sizeof v, cudaMemcpyDeviceToHost, b->stream), "stats read-back");
        if (reset)
            BCUDA(b, cudaMemsetAsync(&d->stat_queries, 0, sizeof v, b->stream), "stats reset");
        BCUDA(b, cudaStreamSynchronize(b->stream), "stats read-back");
        if (stats) {
            stats->queries = v[0];
            stats->fallbacks = v[1];
            stats->local_candidates = v[2];
            stats->global_candidates = v[3];
        }
    }
    return VICP_OK;
}

vicp_status vicp_se3_exp(int32_t n, const double *xi_dev, const double *T0_dev, double *T_dev, void *cuda_stream)
{
    if (n < 1 || !xi_dev || !T0_dev || !T_dev)
        return VICP_ERR_INVALID;
    const cudaError_t e = launch_se3_exp(n, xi_dev, T0_dev, T_dev, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? VICP_OK : VICP_ERR_CUDA;
}

vicp_status vicp_se3_left_jacobian_t(int32_t n, const double *xi_dev, const double *g_dev, double *out_dev,
                                     void *cuda_stream)
{
    if (n < 1 || !xi_dev || !g_dev || !out_dev)
        return VICP_ERR_INVALID;
    const cudaError_t e = launch_se3_jlt(n, xi_dev, g_dev, out_dev, static_cast<cudaStream_t>(cuda_stream));
    return e == cudaSuccess ? VICP_OK : VICP_ERR_CUDA;
}

vicp_status vicp_batch_loss(vicp_batch *b, const float *src_xyzw, const int32_t *n_src, const double *poses_dev,
                            const int32_t *nn_dev, const double *dloss_dev, double *loss_out, double *grad_pose_out,
                            float *grad_src_out)
{
    if (!b)
        return VICP_ERR_INVALID;
    if (!b->built)
        return bfail(b, VICP_ERR_STATE, "vicp_batch_loss before vicp_batch_build");
    if (!src_xyzw || !aligned16(src_xyzw) || !poses_dev || !nn_dev || !loss_out ||
        (grad_src_out && !aligned16(grad_src_out)))
        return bfail(b, VICP_ERR_INVALID, "vicp_batch_loss: NULL or misaligned pointer");
    BTRY(prepare_items(b, n_src, pick_shape(b)));
    BCUDA(b,
          cudaMemset2DAsync((char *)b->state.p + offsetof(BatchState, items_done), sizeof(BatchState), 0,
                            sizeof(unsigned), b->P, b->stream),
          "ticket reset");
    BCUDA(b,
          launch_batch_loss(reinterpret_cast<const float4 *>(src_xyzw), b->target, (const BatchPair *)b->pairs_d.p,
                            (BatchState *)b->state.p, (const BatchItem *)b->sitems.p, b->n_items, poses_dev, nn_dev,
                            dloss_dev, (float2 *)b->partials.p, loss_out, grad_pose_out,
                            reinterpret_cast<float4 *>(grad_src_out), bctl(b), b->stream),
          "launch of the batched loss");
    b->launches += 1;
    return VICP_OK;
}

vicp_status vicp_batch_set_flags(vicp_batch *b, uint32_t flags)
{
    if (!b)
        return VICP_ERR_INVALID;
    b->params.flags = flags;
    drop_graph(b);   // the captured launches hold the old flags' arguments
    return VICP_OK;
}

int64_t vicp_batch_launch_count(const vicp_batch *b) { return b ? b->launches : 0; }

int32_t vicp_batch_graph_replayed(const vicp_batch *b) { return b ? b->last_graph : -1; }

const char *vicp_batch_last_error(const vicp_batch *b) { return b ? b->last_error.c_str() : ""; }

}  // extern "C"
