// vicp_api.cu -- the C ABI declared in include/vicp.h: context, workspace
// allocation through the caller's allocator, argument checks, the launch
// sequence of each entry point, and kernel-level event timing.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <utility>
#include <vector>

#include "vicp.h"
#include "vicp_geom.h"
#include "vicp_launch.h"

using namespace vicp;

namespace {

struct Buf {
    void *p = nullptr;
    size_t bytes = 0;
};

struct Timed {
    int kernel;
    cudaEvent_t start, stop;
};

}  // namespace

struct vicp_ctx {
    vicp_params params{};
    vicp_allocator alloc{};
    bool custom_alloc = false;
    cudaStream_t stream = nullptr;
    // The dilation needs only the histogram's occupancy bits, so it runs on a
    // second stream, concurrently with the rest of the build: `side` waits
    // for ev_hist (after the histogram) and ev_nns (after the last search,
    // which reads root/ring); the context's stream waits for ev_dil (after
    // the dilation), so everything issued later sees its results.
    cudaStream_t side = nullptr;
    cudaEvent_t ev_hist = nullptr, ev_nns = nullptr, ev_dil = nullptr;
    cudaStream_t copy = nullptr;                          // host-input source copy, beside the build
    cudaEvent_t ev_copy_go = nullptr, ev_src = nullptr;
    cudaEvent_t ev_fork = nullptr, ev_clr = nullptr;      // graph capture: the buffer resets beside the copy
    int device = 0;
    int sms = 152;
    std::string last_error;
    uint64_t cur_bytes = 0, peak_bytes = 0;

    // grid state
    bool have_geom = false;
    GridGeom geom{};
    bool built = false;
    int dilated_L = -1;
    int n_target = 0;
    const float4 *target = nullptr;   // caller's target of the last build (global search)

    // V-sized
    Buf counts, off, root, ring, desc, tile_sum, inter, uflag, zdirty;
    bool labels_clean = false;   // root/ring "unlabelled" except where zdirty marks labels
    int lab_dims[3] = {0, 0, 0};   // grid dimensions that state belongs to
    Buf occ[2];       // occupancy bits: the current build's, and the next build's (kept zeroed)
    int occ_cur = 0;
    bool after_solve = false;   // the last kernel launched on `stream` is the reduction + solve
    bool off_dense = false;   // the build writes sparse offsets; vicp_get_grid completes them
    long long cap_V = -1;
    // brick level (V / 512)
    Buf bcounts, boff, brick_list, brick_range, brick_box, bslot, sb_box, sb_left;
    Buf boxk[2];      // brick bounds by key: the current build's, and the next build's (kept all ones)
    long long cap_bricks = -1;
    // N-sized
    Buf keys, ids, csr, bpts, outside;
    long long cap_N = -1;
    // M-sized
    Buf nn, d2, fb_list, hv_list, hv_range;
    long long cap_M = -1;
    // fixed
    Buf partials, rmse, bbox;
    Buf ctl;   // laid out as RegOut: the registrations' pose, then the control block
    // host-input copies (vicp_register_host)
    Buf hsrc, htgt;
    // fixed-capacity store (vicp_fixed_build): C slots per voxel
    Buf fslots, fcount, fover;
    unsigned fixed_C = 0;
    bool fixed_built = false;
    // sparse grid (VICP_FLAG_SPARSE_GRID): hashed occupied voxels (keys of the
    // current and of the next build, counts, offsets by slot; the scan's slot
    // occupancy bits and tile state) and hashed labelled voxels (keys, root
    // keys, per-block counts of pass Z + its overflow flag), instead of the
    // V-sized counts, offsets, root and ring arrays
    Buf okeys[2], ocount, ooff, socc[2], stile, sdesc, pslot;
    Buf lkeys, lseg, lroot, lparts;   // labelled-segment table (keys, masks + first roots), roots, counts
    long long cap_o = 0, cap_l = 0;   // slots (powers of two)
    long long cap_r = 0;              // root array of the labelled voxels
    int o_cur = 0;
    long long cap_occV = -1;
    long long lab_count = 0;          // labelled voxels of the last dilation
    long long lab_segs = 0;           // ... and their row segments
    bool lab_kept = false;            // with VICP_FLAG_KEEP_GRID: the table size was checked for ...
    int lab_L = -1, lab_kept_dims[3] = {0, 0, 0};   // ... this L and these grid dimensions

    // vicp_register / vicp_register_host replayed from a captured CUDA graph:
    // the call's arguments it was captured for, the kernels of one replay,
    // the private capture / replay stream with the events that order it
    // after and before the context's stream, and page-locked staging for the
    // initial pose and the results
    struct RegKey {
        bool host = false;
        const void *src = nullptr, *tgt = nullptr;
        int32_t m = 0, n = 0, max_iters = -1, L = -1;
        uint32_t flags = 0;
        double eps = 0.0;
        GridGeom geom{};
    };
    struct RegOut {
        double pose[16];
        DevCtl ctl;   // the control block after the call (loop state, status word)
    };
    RegKey rg_key, rg_last;           // the graph's call; the last direct call
    bool rg_last_valid = false, rg_broken = false;
    bool rg_replayed = false;         // the last registration call replayed the graph
    cudaGraphExec_t rg_exec = nullptr;
    int64_t rg_launches = 0;
    cudaStream_t gstream = nullptr;
    double *h_pose = nullptr;         // page-locked, 16 doubles
    RegOut *h_out = nullptr;          // page-locked
    bool capturing = false, nns_in_capture = false;

    // accounting / timing
    int64_t launches = 0;
    bool profiling = false;
    std::vector<Timed> pending;
    std::vector<cudaEvent_t> event_pool;
    int64_t prof_launches[K_COUNT] = {};
    double prof_ms[K_COUNT] = {};
};

namespace {

vicp_status fail(vicp_ctx *c, vicp_status s, const char *fmt, ...)
{
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->last_error = buf;
    }
    return s;
}

vicp_status cuda_fail(vicp_ctx *c, cudaError_t e, const char *what)
{
    return fail(c, VICP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// --- allocation ------------------------------------------------------------
vicp_status buf_free(vicp_ctx *c, Buf &b)
{
    if (b.p) {
        if (c->custom_alloc)
            c->alloc.free(b.p, b.bytes, (void *)c->stream, c->alloc.user);
        else
            cudaFree(b.p);
        c->cur_bytes -= b.bytes;
    }
    b.p = nullptr;
    b.bytes = 0;
    return VICP_OK;
}

vicp_status buf_alloc(vicp_ctx *c, Buf &b, size_t bytes, const char *what)
{
    buf_free(c, b);
    if (bytes == 0)
        bytes = 256;
    bytes = (bytes + 255) & ~(size_t)255;
    void *p = nullptr;
    if (c->custom_alloc) {
        p = c->alloc.alloc(bytes, (void *)c->stream, c->alloc.user);
        if (!p)
            return fail(c, VICP_ERR_OOM, "allocator returned NULL for %s (%zu bytes)", what, bytes);
    } else {
        cudaError_t e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(c, VICP_ERR_OOM, "cudaMalloc of %zu bytes for %s: %s", bytes, what, cudaGetErrorString(e));
        }
    }
    b.p = p;
    b.bytes = bytes;
    c->cur_bytes += bytes;
    if (c->cur_bytes > c->peak_bytes)
        c->peak_bytes = c->cur_bytes;
    return VICP_OK;
}

vicp_status buf_zero(vicp_ctx *c, Buf &b, const char *what)
{
    cudaError_t e = cudaMemsetAsync(b.p, 0, b.bytes, c->stream);
    return e == cudaSuccess ? VICP_OK : cuda_fail(c, e, what);
}

#define TRY(x)                       \
    do {                             \
        vicp_status _s = (x);        \
        if (_s != VICP_OK)           \
            return _s;               \
    } while (0)

// --- timing ----------------------------------------------------------------
cudaEvent_t take_event(vicp_ctx *c)
{
    if (!c->event_pool.empty()) {
        cudaEvent_t e = c->event_pool.back();
        c->event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

template <typename F>
vicp_status launch_on(vicp_ctx *c, int kernel, cudaStream_t st, F &&f)
{
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (c->profiling) {
        e0 = take_event(c);
        cudaEventRecord(e0, st);
    }
    cudaError_t e = f();
    if (st == c->stream)
        c->after_solve = (kernel == K_REDUCE_SOLVE || kernel == K_REDUCE_SOLVE_F64) && e == cudaSuccess &&
                         !c->profiling;
    if (c->profiling) {
        e1 = take_event(c);
        cudaEventRecord(e1, st);
        c->pending.push_back({kernel, e0, e1});
    }
    c->launches += kernel == K_DILATE ? 2 : 1;   // the dilation is two kernels
    if (e != cudaSuccess)
        return fail(c, VICP_ERR_CUDA, "launch of %s: %s", kernel_name(kernel), cudaGetErrorString(e));
    return VICP_OK;
}

template <typename F>
vicp_status launch(vicp_ctx *c, int kernel, F &&f)
{
    return launch_on(c, kernel, c->stream, std::forward<F>(f));
}

DevCtl *ctl_of(vicp_ctx *c)
{
    return reinterpret_cast<DevCtl *>(static_cast<char *>(c->ctl.p) + offsetof(vicp_ctx::RegOut, ctl));
}
// The pose a registration iterates on (16 doubles before the control block,
// so that one copy reads both back).
double *reg_pose_of(vicp_ctx *c) { return static_cast<double *>(c->ctl.p); }

bool sparse_of(const vicp_ctx *c) { return (c->params.flags & VICP_FLAG_SPARSE_GRID) != 0; }

long long pow2_at_least(long long x)
{
    long long p = 1;
    while (p < x)
        p <<= 1;
    return p;
}

HashTable table_of(const Buf &keys, long long slots)
{
    int lg = 0;
    while ((1ll << lg) < slots)
        ++lg;
    return HashTable{static_cast<unsigned *>(keys.p), (unsigned)(slots - 1), 32 - lg};
}

// The scan over the occupied-voxel table runs on its slots as if they were
// voxels.
GridGeom slot_geom(long long slots)
{
    GridGeom g{};
    g.V = slots;
    return g;
}

// --- workspace sizing ------------------------------------------------------
vicp_status ensure_voxel_buffers(vicp_ctx *c, long long V, long long n_bricks)
{
    if (V > c->cap_occV) {   // voxel occupancy bits: both grids (the dilation reads them)
        for (Buf &o : c->occ) {
            TRY(buf_alloc(c, o, (size_t)occ_words(V) * 4, "occupancy"));
            TRY(buf_zero(c, o, "zero occupancy"));
        }
        c->cap_occV = V;
    }
    if (!sparse_of(c) && V > c->cap_V) {   // the dense grid's per-voxel arrays
        TRY(buf_alloc(c, c->counts, (size_t)V * 4, "counts"));
        TRY(buf_zero(c, c->counts, "zero counts"));   // counts are kept at zero between builds
        TRY(buf_alloc(c, c->off, (size_t)(V + 1) * 4, "offsets"));
        TRY(buf_alloc(c, c->root, (size_t)V * 4, "root"));
        TRY(buf_alloc(c, c->ring, (size_t)V, "ring"));
        c->labels_clean = false;
        TRY(buf_alloc(c, c->desc, (size_t)scan_tiles(V) * 8, "scan descriptors"));
        TRY(buf_zero(c, c->desc, "zero scan descriptors"));
        TRY(buf_alloc(c, c->tile_sum, (size_t)scan_tiles(V) * 4, "scan tile sums"));
        TRY(buf_zero(c, c->tile_sum, "zero scan tile sums"));   // kept at zero between builds
        c->cap_V = V;
    }
    if (dilate_units(c->geom) * 4 > (long long)c->uflag.bytes) {
        TRY(buf_alloc(c, c->uflag, (size_t)dilate_units(c->geom) * 4, "dilation row masks"));
    }
    if (!sparse_of(c) && dilate_column_units(c->geom) > (long long)c->zdirty.bytes) {
        TRY(buf_alloc(c, c->zdirty, (size_t)dilate_column_units(c->geom), "dilation label flags"));
        c->labels_clean = false;
    }
    if (n_bricks > c->cap_bricks) {
        TRY(buf_alloc(c, c->bcounts, (size_t)n_bricks * 4, "brick counts"));
        TRY(buf_zero(c, c->bcounts, "zero brick counts"));   // kept at zero between builds
        TRY(buf_alloc(c, c->boff, (size_t)(n_bricks + 1) * 4, "brick offsets"));
        TRY(buf_alloc(c, c->brick_list, (size_t)n_bricks * 4, "brick list"));
        TRY(buf_alloc(c, c->brick_range, (size_t)n_bricks * 8, "brick ranges"));
        TRY(buf_alloc(c, c->brick_box, (size_t)n_bricks * 32, "brick boxes"));
        TRY(buf_alloc(c, c->bslot, (size_t)n_bricks * 4, "brick slots"));
        for (Buf &b : c->boxk) {
            TRY(buf_alloc(c, b, (size_t)n_bricks * 32, "brick bounds"));
            const cudaError_t e = cudaMemsetAsync(b.p, 0xff, b.bytes, c->stream);   // all ones between builds
            if (e != cudaSuccess)
                return cuda_fail(c, e, "brick bounds");
        }
        TRY(buf_alloc(c, c->sb_box, (size_t)(n_bricks / SUPER_BRICKS + 1) * 32, "super-brick boxes"));
        TRY(buf_alloc(c, c->sb_left, (size_t)(n_bricks / SUPER_BRICKS) * 4, "super-brick counts"));
        TRY(buf_zero(c, c->sb_left, "zero super-brick counts"));   // kept at zero between builds
        c->cap_bricks = n_bricks;
    }
    return VICP_OK;
}

// The sparse grid's occupied-voxel table: at least twice as many slots as
// target points (a voxel holds at least one), so it is at most half full.
vicp_status ensure_sparse_buffers(vicp_ctx *c, long long n)
{
    const long long slots = pow2_at_least(n * 2 > 1024 ? n * 2 : 1024);
    if (slots > c->cap_o) {
        for (Buf &k : c->okeys) {
            TRY(buf_alloc(c, k, (size_t)slots * 4, "occupied-voxel table"));
            const cudaError_t e = cudaMemsetAsync(k.p, 0xff, k.bytes, c->stream);   // empty
            if (e != cudaSuccess)
                return cuda_fail(c, e, "occupied-voxel table");
        }
        TRY(buf_alloc(c, c->ocount, (size_t)slots * 4, "occupied-voxel counts"));
        TRY(buf_zero(c, c->ocount, "zero occupied-voxel counts"));   // kept at zero between builds
        TRY(buf_alloc(c, c->ooff, (size_t)(slots + 1) * 4, "occupied-voxel offsets"));
        for (Buf &o : c->socc) {
            TRY(buf_alloc(c, o, (size_t)occ_words(slots) * 4, "slot occupancy"));
            TRY(buf_zero(c, o, "zero slot occupancy"));
        }
        TRY(buf_alloc(c, c->stile, (size_t)scan_tiles(slots) * 4, "slot scan tile sums"));
        TRY(buf_zero(c, c->stile, "zero slot scan tile sums"));
        TRY(buf_alloc(c, c->sdesc, (size_t)scan_tiles(slots) * 8, "slot scan descriptors"));
        TRY(buf_zero(c, c->sdesc, "zero slot scan descriptors"));
        c->cap_o = slots;
        c->o_cur = 0;
    }
    if (n * 4 > (long long)c->pslot.bytes)
        TRY(buf_alloc(c, c->pslot, (size_t)n * 4, "point slots"));
    return VICP_OK;
}

// The labelled-segment table with `slots` slots (keys are cleared by the
// dilation itself), the root array with `roots` entries, and pass Z's
// per-block counts + overflow flag + root counter.
vicp_status ensure_label_table(vicp_ctx *c, long long slots, long long roots, int L)
{
    if (slots > c->cap_l) {
        TRY(buf_alloc(c, c->lkeys, (size_t)slots * 4, "labelled-segment table"));
        TRY(buf_alloc(c, c->lseg, (size_t)slots * 8, "labelled-segment masks"));
        c->cap_l = slots;
    }
    if (roots > c->cap_r) {
        TRY(buf_alloc(c, c->lroot, (size_t)roots * 4, "labelled roots"));
        c->cap_r = roots;
    }
    const size_t parts = (size_t)(dilate_hashed_blocks(c->geom, L) + 2) * 4;
    if (parts > c->lparts.bytes)
        TRY(buf_alloc(c, c->lparts, parts, "labelled-segment counts"));
    return VICP_OK;
}

vicp_status ensure_point_buffers(vicp_ctx *c, long long n)
{
    if (n > c->cap_N) {
        TRY(buf_alloc(c, c->keys, (size_t)n * 4, "keys"));
        TRY(buf_alloc(c, c->ids, (size_t)n * 4, "ids"));
        TRY(buf_alloc(c, c->csr, (size_t)n * 16, "csr points"));
        TRY(buf_alloc(c, c->bpts, (size_t)n * 16, "brick points"));
        TRY(buf_alloc(c, c->outside, (size_t)n * 4, "outside list"));
        c->cap_N = n;
    }
    return VICP_OK;
}

vicp_status ensure_query_buffers(vicp_ctx *c, long long m)
{
    if (m > c->cap_M) {
        TRY(buf_alloc(c, c->nn, (size_t)m * 4, "nn"));
        TRY(buf_alloc(c, c->d2, (size_t)m * 4, "d2"));
        TRY(buf_alloc(c, c->fb_list, (size_t)m * 4, "fallback list"));
        TRY(buf_alloc(c, c->hv_list, (size_t)m * 4, "dense segment list"));
        TRY(buf_alloc(c, c->hv_range, (size_t)m * 8, "dense segment ranges"));
        c->cap_M = m;
    }
    return VICP_OK;
}

// --- geometry (host side of the grid fit) ----------------------------------
vicp_status set_geometry(vicp_ctx *c, const float origin[3], float h, const int dims[3])
{
    if (!(h > 0.0f) || !std::isfinite(h))
        return fail(c, VICP_ERR_INVALID, "voxel size must be finite and > 0 (got %g)", (double)h);
    for (int a = 0; a < 3; ++a) {
        if (dims[a] < 1)
            return fail(c, VICP_ERR_INVALID, "grid dims must be >= 1");
        if (!std::isfinite(origin[a]))
            return fail(c, VICP_ERR_INVALID, "grid origin must be finite");
    }
    const long long V = (long long)dims[0] * dims[1] * dims[2];
    if (V >= (1ll << 31) - 1)
        return fail(c, VICP_ERR_GRID_TOO_LARGE, "grid of %d x %d x %d = %lld voxels (limit 2^31 - 2)", dims[0],
                    dims[1], dims[2], V);
    const GridGeom g = make_geom(origin, h, dims);
    c->geom = g;
    c->have_geom = true;
    return VICP_OK;
}

// Bounding-box grid: origin = minimum corner, h given or extent/divisions,
// dims_a = floor(extent_a * inv_h) + 1 (one synchronisation to read the box).
vicp_status fit_geometry(vicp_ctx *c, const float4 *tgt, int n)
{
    unsigned *bb = static_cast<unsigned *>(c->bbox.p);
    TRY(launch(c, K_BBOX, [&] { return launch_bbox(tgt, n, bb, c->stream); }));
    unsigned hb[6];
    cudaError_t e = cudaMemcpyAsync(hb, bb, sizeof hb, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "bounding box read-back");
    float lo[3], hi[3], h = 0.0f;
    for (int a = 0; a < 3; ++a) {
        lo[a] = ordered_to_float_host(hb[a]);
        hi[a] = ordered_to_float_host(hb[3 + a]);
    }
    int dims[3], axis = 0;
    const GeomResult r = fit_box(lo, hi, c->params.voxel_size, c->params.grid_divisions, &h, dims, &axis);
    if (r == GEOM_NONFINITE)
        return fail(c, VICP_ERR_INVALID, "target has no finite coordinate on axis %d", axis);
    if (r == GEOM_TOO_LARGE)
        return fail(c, VICP_ERR_GRID_TOO_LARGE, "grid axis %d would be too long", axis);
    return set_geometry(c, lo, h, dims);
}

vicp_status check_params(vicp_ctx *c, const vicp_params *p)
{
    if (p->dilation_layers < 0 || p->dilation_layers > DILATE_MAX_L)
        return fail(c, VICP_ERR_INVALID, "dilation_layers must be in [0, %d]", DILATE_MAX_L);
    if (p->max_iters < 0)
        return fail(c, VICP_ERR_INVALID, "max_iters must be >= 0");
    if (p->dims[0] <= 0 && !(p->voxel_size > 0.0f) && p->grid_divisions < 1)
        return fail(c, VICP_ERR_INVALID, "auto grid needs voxel_size > 0 or grid_divisions >= 1");
    if (p->dims[0] > 0 && (p->dims[1] < 1 || p->dims[2] < 1 || !(p->voxel_size > 0.0f)))
        return fail(c, VICP_ERR_INVALID, "explicit grid needs dims >= 1 and voxel_size > 0");
    return VICP_OK;
}

vicp_status check_cloud(vicp_ctx *c, const float *p, int32_t n, const char *what)
{
    if (!p || n < 1)
        return fail(c, VICP_ERR_INVALID, "%s: need a non-NULL pointer and n >= 1", what);
    if (!aligned16(p))
        return fail(c, VICP_ERR_INVALID, "%s: pointer must be 16-byte aligned", what);
    return VICP_OK;
}

vicp_status read_device_status(vicp_ctx *c)
{
    unsigned err = 0;
    DevCtl *d = ctl_of(c);
    cudaError_t e = cudaMemcpyAsync(&err, &d->err, sizeof err, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "synchronise");
    if (err) {
        cudaMemsetAsync(&d->err, 0, sizeof(unsigned), c->stream);
        if (err & DEVERR_TIMEOUT)
            return fail(c, VICP_ERR_TIMEOUT, "a device-side wait gave up (device status 0x%x)", err);
        if (err & DEVERR_BOUNDS)
            return fail(c, VICP_ERR_CUDA, "a device-side bounds check failed (device status 0x%x)", err);
        if (err & DEVERR_CAPACITY) {
            c->lab_kept = false;   // the next dilation checks its table size again
            return fail(c, VICP_ERR_STATE,
                        "a hashed voxel table of the sparse grid was too small for this cloud (the table size "
                        "found at the first build is kept under VICP_FLAG_KEEP_GRID): build and dilate again");
        }
        if (err & DEVERR_DEGENERATE)
            return fail(c, VICP_ERR_DEGENERATE, "rank(H) < 2: degenerate correspondence geometry");
    }
    return VICP_OK;
}

// The localised search (Alg. 4's root-voxel scan) on the dense or the
// sparse grid.
vicp_status run_localised(vicp_ctx *c, const float4 *src, int m, const double *pose, int *nn, float *d2,
                          int honor_stop)
{
    const GridGeom &g = c->geom;
    DevCtl *d = ctl_of(c);
    if (sparse_of(c))
        return launch(c, K_CORRESPOND, [&] {
            return launch_correspond_hashed(src, m, pose, g, table_of(c->lkeys, c->cap_l), (const uint2 *)c->lseg.p,
                                            (const int *)c->lroot.p,
                                            table_of(c->okeys[c->o_cur], c->cap_o), (const unsigned *)c->ooff.p,
                                            (const float4 *)c->csr.p, c->n_target, nn, d2, (int *)c->fb_list.p,
                                            (int *)c->hv_list.p, (uint2 *)c->hv_range.p, d, honor_stop, c->stream);
        });
    return launch(c, K_CORRESPOND, [&] {
        return launch_correspond(src, m, pose, g, (const int *)c->root.p, (const unsigned *)c->off.p,
                                 (const float4 *)c->csr.p, c->n_target, nn, d2, (int *)c->fb_list.p,
                                 (int *)c->hv_list.p, (uint2 *)c->hv_range.p, d, honor_stop, c->stream);
    });
}

// Correspond + global search into nn/d2 (shared by vicp_correspond and the step).
vicp_status run_nns(vicp_ctx *c, const float4 *src, int m, const double *pose, int *nn, float *d2, int honor_stop)
{
    DevCtl *d = ctl_of(c);
    TRY(run_localised(c, src, m, pose, nn, d2, honor_stop));
    TRY(launch(c, K_FALLBACK, [&] {
        return launch_fallback(src, pose, (const float4 *)c->bpts.p, (const float4 *)c->brick_box.p,
                               (const float4 *)c->sb_box.p, c->target, c->n_target, (const int *)c->outside.p,
                               (const int *)c->fb_list.p, (const int *)c->hv_list.p, (const uint2 *)c->hv_range.p,
                               (const float4 *)c->csr.p, d, nn, d2, m, honor_stop, c->stream);
    }));
    cudaError_t e = cudaEventRecord(c->ev_nns, c->stream);   // a later dilation waits for this search
    c->nns_in_capture = c->capturing;
    return e == cudaSuccess ? VICP_OK : cuda_fail(c, e, "event record");
}

vicp_status run_step(vicp_ctx *c, const float4 *src, int m, double *pose, double *rmse, int honor_stop)
{
    TRY(ensure_query_buffers(c, m));
    int *nn = (int *)c->nn.p;
    TRY(run_nns(c, src, m, pose, nn, (float *)c->d2.p, honor_stop));
    const float3 ctr = grid_center(c->geom);
    const int nparts = reduce_blocks(m, c->sms);
    if (c->params.flags & VICP_FLAG_FP64_SOLVE) {
        TRY(launch(c, K_REDUCE_SOLVE_F64, [&] {
            return launch_reduce_solve_f64(src, m, pose, c->target, c->n_target, nn, ctr, (double *)c->partials.p,
                                           nparts, rmse, ctl_of(c), honor_stop, c->params.rmse_eps, c->stream);
        }));
        return VICP_OK;
    }
    TRY(launch(c, K_REDUCE_SOLVE, [&] {
        return launch_reduce_solve(src, m, pose, c->target, c->n_target, nn, ctr, (float2 *)c->partials.p, nparts,
                                   rmse, ctl_of(c), honor_stop, c->params.rmse_eps, c->stream);
    }));
    return VICP_OK;
}

// load_from (may be null): the target cloud's page-locked host copy (its
// device-mapped address); the histogram then reads the points from there
// and stores them to `target` (device) for the kernels after it.
vicp_status build(vicp_ctx *c, const float *target, int32_t n, const float *load_from = nullptr)
{
    TRY(check_cloud(c, target, n, "target"));
    const float4 *tgt = reinterpret_cast<const float4 *>(target);
    const bool auto_grid = c->params.dims[0] <= 0;
    if (auto_grid) {
        if (!c->have_geom || !(c->params.flags & VICP_FLAG_KEEP_GRID))
            TRY(fit_geometry(c, tgt, n));
    } else if (!c->have_geom) {
        TRY(set_geometry(c, c->params.origin, c->params.voxel_size, c->params.dims));
    }
    const GridGeom &g = c->geom;
    const bool sparse = sparse_of(c);
    TRY(ensure_voxel_buffers(c, g.V, brick_slots(g)));
    TRY(ensure_point_buffers(c, n));
    if (sparse)
        TRY(ensure_sparse_buffers(c, n));
    DevCtl *d = ctl_of(c);
    // this build fills the zeroed occupancy buffer; its scatter clears the other
    c->occ_cur ^= 1;
    unsigned *occ = (unsigned *)c->occ[c->occ_cur].p;
    Buf &occ_next = c->occ[c->occ_cur ^ 1];
    const bool after_solve = c->after_solve;
    // the sparse grid likewise fills the empty occupied-voxel table and the
    // zeroed slot occupancy bits that the previous scatter left, and its
    // scatter resets the others for the next build
    if (sparse)
        c->o_cur ^= 1;
    const HashTable ho = sparse ? table_of(c->okeys[c->o_cur], c->cap_o) : HashTable{};
    unsigned *counts = (unsigned *)(sparse ? c->ocount.p : c->counts.p);
    unsigned *off = (unsigned *)(sparse ? c->ooff.p : c->off.p);
    unsigned *tiles = (unsigned *)(sparse ? c->stile.p : c->tile_sum.p);
    unsigned *socc = sparse ? (unsigned *)c->socc[c->o_cur].p : nullptr;
    TRY(launch(c, K_HISTOGRAM, [&] {
        return launch_histogram(load_from ? reinterpret_cast<const float4 *>(load_from) : tgt, n, g,
                                (int *)c->keys.p, counts, (unsigned *)c->bcounts.p, occ, tiles,
                                (unsigned *)c->sb_left.p, (unsigned *)c->boxk[c->occ_cur].p, d, c->stream, after_solve,
                                sparse ? &ho : nullptr, socc, (int *)c->pslot.p,
                                load_from ? const_cast<float4 *>(tgt) : nullptr);
    }));
    cudaError_t ev = cudaEventRecord(c->ev_hist, c->stream);   // the dilation may start from here
    if (ev != cudaSuccess)
        return cuda_fail(c, ev, "event record");
    TRY(launch(c, K_SCAN, [&] {
        if (sparse)
            return launch_scan(counts, slot_geom(c->cap_o), off, socc, tiles, (unsigned long long *)c->sdesc.p, d,
                               c->stream, false);
        return launch_scan(counts, g, off, occ, tiles, (unsigned long long *)c->desc.p, d, c->stream, false);
    }));
    c->off_dense = false;
    TRY(launch(c, K_BRICK_SCAN, [&] {
        return launch_brick_scan((const unsigned *)c->bcounts.p, g, (unsigned *)c->boff.p, (int *)c->brick_list.p,
                                 (uint2 *)c->brick_range.p, (int *)c->bslot.p, d, c->stream);
    }));
    TRY(launch(c, K_SCATTER, [&] {
        const int *idx = (const int *)(sparse ? c->pslot.p : c->keys.p);   // what indexes the counts
        return launch_scatter(tgt, idx, n, g, off, counts, (const unsigned *)c->boff.p, (unsigned *)c->bcounts.p,
                              (const int *)c->bslot.p, (const unsigned *)c->boxk[c->occ_cur].p,
                              (unsigned *)c->boxk[c->occ_cur ^ 1].p, (long long)(c->boxk[c->occ_cur ^ 1].bytes / 4),
                              (const uint2 *)c->brick_range.p, (float4 *)c->brick_box.p, (unsigned *)c->sb_left.p,
                              (float4 *)c->sb_box.p, (int *)c->ids.p, (float4 *)c->csr.p, (float4 *)c->bpts.p,
                              (int *)c->outside.p, tiles, (unsigned *)occ_next.p, (long long)(occ_next.bytes / 4), d,
                              c->stream, sparse ? scan_tiles(c->cap_o) : -1,
                              sparse ? (unsigned *)c->okeys[c->o_cur ^ 1].p : nullptr, sparse ? c->cap_o : 0,
                              sparse ? (unsigned *)c->socc[c->o_cur ^ 1].p : nullptr,
                              sparse ? occ_words(c->cap_o) : 0);
    }));
    c->built = true;
    c->dilated_L = -1;
    c->n_target = n;
    c->target = tgt;
    return VICP_OK;
}

// The sparse grid's dilation (on the side stream, after the waits of
// dilate()): pass Z enters the labelled row segments into the segment table
// and their roots into the root array, then the host checks that the table
// was at most half full and the roots fitted -- one synchronisation per
// dilation -- and, if not, grows them (the table to twice the segments, the
// roots to their count + 1/8) and runs the dilation again.
vicp_status dilate_sparse(vicp_ctx *c, int L)
{
    const GridGeom &g = c->geom;
    const long long n4 = (long long)c->n_target * 4 > 4096 ? (long long)c->n_target * 4 : 4096;
    long long slots = c->cap_l > 0 ? c->cap_l : pow2_at_least(n4 / 4);
    long long roots = c->cap_r > 0 ? c->cap_r : 2 * n4;
    const int blocks = dilate_hashed_blocks(g, L);
    unsigned *err = &ctl_of(c)->err;
    unsigned *parts_d = (unsigned *)c->lparts.p;
    auto run = [&]() -> vicp_status {   // (pass XY zeroes the counts, the overflow flag and the root counter)
        parts_d = (unsigned *)c->lparts.p;
        return launch_on(c, K_DILATE, c->side, [&] {
            return launch_dilate_hashed((const unsigned *)c->occ[c->occ_cur].p, g, L, c->inter.p,
                                        (unsigned *)c->uflag.p, table_of(c->lkeys, c->cap_l), (uint2 *)c->lseg.p,
                                        (int *)c->lroot.p, (unsigned)c->cap_r, parts_d, err, c->side);
        });
    };
    // VICP_FLAG_KEEP_GRID keeps the grid of the first build, and with it the
    // table sizes checked then: later dilations of the same grid run without
    // the check (a cloud that needs more room is reported by the next
    // synchronising call as VICP_ERR_STATE, and the next dilation checks).
    if ((c->params.flags & VICP_FLAG_KEEP_GRID) && c->lab_kept && c->lab_L == L && c->lab_kept_dims[0] == g.nx &&
        c->lab_kept_dims[1] == g.ny && c->lab_kept_dims[2] == g.nz) {
        TRY(run());
    } else {
        c->lab_kept = false;
        for (int attempt = 0;; ++attempt) {
            TRY(ensure_label_table(c, slots, roots, L));
            TRY(run());
            std::vector<unsigned> parts((size_t)blocks + 2);
            cudaError_t e = cudaMemcpyAsync(parts.data(), parts_d, parts.size() * 4, cudaMemcpyDeviceToHost, c->side);
            if (e == cudaSuccess)
                e = cudaStreamSynchronize(c->side);
            if (e != cudaSuccess)
                return cuda_fail(c, e, "labelled-segment count read-back");
            long long segs = 0;
            for (int b = 0; b < blocks; ++b)
                segs += parts[b];
            const bool overflow = parts[blocks] != 0;
            const long long count = parts[blocks + 1];   // roots handed out (all labelled voxels when they fitted)
            if (!overflow && 2 * segs <= c->cap_l && count <= c->cap_r) {
                c->lab_count = count;
                c->lab_segs = segs;
                c->lab_kept = true;
                c->lab_L = L;
                c->lab_kept_dims[0] = g.nx;
                c->lab_kept_dims[1] = g.ny;
                c->lab_kept_dims[2] = g.nz;
                break;
            }
            if (overflow) {   // this dilation is run again: its capacity report is withdrawn
                e = launch_clear_bits(err, DEVERR_CAPACITY, c->side);
                if (e != cudaSuccess)
                    return cuda_fail(c, e, "status update");
            }
            if (attempt >= 3)
                return fail(c, VICP_ERR_CUDA,
                            "labelled-segment table: %lld segments / %lld voxels do not fit %lld / %lld", segs, count,
                            c->cap_l, c->cap_r);
            // a root count past the array is a lower bound: grow at least twofold
            slots = pow2_at_least(2 * segs > 2 * c->cap_l ? 2 * segs : 2 * c->cap_l);
            roots = count + count / 8 > 2 * c->cap_r ? count + count / 8 : 2 * c->cap_r;
        }
    }
    cudaError_t e = cudaEventRecord(c->ev_dil, c->side);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(c->stream, c->ev_dil, 0);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "stream wait");
    c->dilated_L = L;
    return VICP_OK;
}

// Completes the build's sparse offsets (once per build) for the callers that
// hand out or scan the whole array.
vicp_status dense_offsets(vicp_ctx *c)
{
    if (c->off_dense)
        return VICP_OK;
    const GridGeom &g = c->geom;
    TRY(launch(c, K_OFFSETS_FILL, [&] {
        return launch_offsets_fill((unsigned *)c->off.p, (const unsigned *)c->occ[c->occ_cur].p, g.V, c->stream);
    }));
    c->off_dense = true;
    return VICP_OK;
}

vicp_status dilate(vicp_ctx *c, int32_t layers)
{
    if (!c->built)
        return fail(c, VICP_ERR_STATE, "vicp_dilate before vicp_build_grid");
    const int L = layers < 0 ? c->params.dilation_layers : layers;
    if (L > DILATE_MAX_L)
        return fail(c, VICP_ERR_INVALID, "dilation layers must be in [0, %d]", DILATE_MAX_L);
    const GridGeom &g = c->geom;
    // pass-Y words: 16 bits a voxel while L <= 15, else 32
    const size_t inter_bytes = (size_t)g.V * (L <= 15 ? 2 : 4);
    if (c->inter.bytes < inter_bytes)
        TRY(buf_alloc(c, c->inter, inter_bytes, "dilation pass-Y words"));
    // on the side stream, after the histogram and after the last search (in
    // a graph capture only a search of the captured call: the replay starts
    // after all earlier work of the context's stream)
    cudaError_t e = cudaStreamWaitEvent(c->side, c->ev_hist, 0);
    if (e == cudaSuccess && (!c->capturing || c->nns_in_capture))
        e = cudaStreamWaitEvent(c->side, c->ev_nns, 0);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "stream wait");
    if (sparse_of(c))
        return dilate_sparse(c, L);
    if (!c->labels_clean || c->lab_dims[0] != g.nx || c->lab_dims[1] != g.ny || c->lab_dims[2] != g.nz) {
        // new arrays or new dimensions: every voxel "unlabelled" (all bytes 0xff), no labels recorded
        e = cudaMemsetAsync(c->root.p, 0xff, (size_t)g.V * 4, c->side);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(c->ring.p, 0xff, (size_t)g.V, c->side);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(c->zdirty.p, 0, (size_t)dilate_column_units(g), c->side);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "clear root/ring");
        c->labels_clean = true;
        c->lab_dims[0] = g.nx;
        c->lab_dims[1] = g.ny;
        c->lab_dims[2] = g.nz;
    }
    TRY(launch_on(c, K_DILATE, c->side, [&] {
        return launch_dilate((const unsigned *)c->occ[c->occ_cur].p, g, L, c->inter.p, (unsigned *)c->uflag.p,
                             (unsigned char *)c->zdirty.p, (int *)c->root.p, (unsigned char *)c->ring.p, c->side);
    }));
    e = cudaEventRecord(c->ev_dil, c->side);
    if (e == cudaSuccess)
        e = cudaStreamWaitEvent(c->stream, c->ev_dil, 0);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "stream wait");
    c->dilated_L = L;
    return VICP_OK;
}

// The work of one registration: the initial pose from pose_in (host) and
// the loop state reset on the internal copy stream, where they run beside
// the build (host_copies: the caller has already queued the source cloud's
// copy there, after the context's earlier work; otherwise the copy stream is
// ordered after that work here), then on the context's stream build,
// dilate, a wait for the copy stream, the iterations, and the pose and the
// control block (loop state, status word) copied to out_pose / out_ctl
// (host).  tgt_load and src_late (host_copies only; may be null): the first
// build's histogram reads the target from its page-locked host copy
// (device-mapped address) and stores it to tgt, and the source cloud's copy
// from src_late is queued on the copy stream after that histogram, so that
// the two clouds cross the host link one after the other.
vicp_status registration_work(vicp_ctx *c, const float4 *src, int32_t m, const float *tgt, int32_t n,
                              const double *pose_in, void *out_pose, DevCtl *out_ctl, bool host_copies,
                              const float *tgt_load = nullptr, const void *src_late = nullptr)
{
    double *pose = reg_pose_of(c);
    DevCtl *d = ctl_of(c);
    cudaError_t e = cudaSuccess;
    if (!host_copies) {
        e = cudaEventRecord(c->ev_copy_go, c->stream);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(c->copy, c->ev_copy_go, 0);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(pose, pose_in, 16 * sizeof(double), cudaMemcpyHostToDevice, c->copy);
    if (e == cudaSuccess)   // stop, iters, prev_rmse, last_rmse (the build's kernels use other fields)
        e = cudaMemsetAsync(&d->stop, 0, sizeof(DevCtl) - offsetof(DevCtl, stop), c->copy);
    if (e == cudaSuccess && !src_late)
        e = cudaEventRecord(c->ev_src, c->copy);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "pose upload and loop state reset");
    TRY(build(c, tgt, n, tgt_load));
    if (src_late) {   // ev_hist: recorded by the build right after its histogram
        e = cudaStreamWaitEvent(c->copy, c->ev_hist, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync((void *)src, src_late, (size_t)m * 16, cudaMemcpyHostToDevice, c->copy);
        if (e == cudaSuccess)
            e = cudaEventRecord(c->ev_src, c->copy);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "host-to-device copy of the source cloud");
    }
    TRY(dilate(c, -1));
    e = cudaStreamWaitEvent(c->stream, c->ev_src, 0);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "stream wait");
    for (int k = 0; k < c->params.max_iters; ++k) {
        if (k > 0 && (c->params.flags & VICP_FLAG_REBUILD_EACH_ITER)) {
            TRY(build(c, tgt, n));
            TRY(dilate(c, -1));
        }
        TRY(run_step(c, src, m, pose, nullptr, 1));
    }
    if (reinterpret_cast<char *>(out_ctl) == static_cast<char *>(out_pose) + offsetof(vicp_ctx::RegOut, ctl)) {
        e = cudaMemcpyAsync(out_pose, c->ctl.p, sizeof(vicp_ctx::RegOut), cudaMemcpyDeviceToHost, c->stream);
    } else {
        e = cudaMemcpyAsync(out_pose, pose, 16 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(out_ctl, d, sizeof(DevCtl), cudaMemcpyDeviceToHost, c->stream);
    }
    if (e != cudaSuccess)
        return cuda_fail(c, e, "result read-back");
    return VICP_OK;
}

// A device status word read back by a graph replay, as read_device_status
// maps it (the word is cleared on the device when set).
vicp_status device_status_from(vicp_ctx *c, unsigned err)
{
    if (!err)
        return VICP_OK;
    DevCtl *d = ctl_of(c);
    cudaMemsetAsync(&d->err, 0, sizeof(unsigned), c->stream);
    if (err & DEVERR_TIMEOUT)
        return fail(c, VICP_ERR_TIMEOUT, "a device-side wait gave up (device status 0x%x)", err);
    if (err & DEVERR_BOUNDS)
        return fail(c, VICP_ERR_CUDA, "a device-side bounds check failed (device status 0x%x)", err);
    if (err & DEVERR_CAPACITY)
        return fail(c, VICP_ERR_STATE, "a hashed voxel table of the sparse grid was too small for this cloud");
    if (err & DEVERR_DEGENERATE)
        return fail(c, VICP_ERR_DEGENERATE, "rank(H) < 2: degenerate correspondence geometry");
    return VICP_OK;
}

bool same_call(const vicp_ctx::RegKey &a, const vicp_ctx::RegKey &b)
{
    return a.host == b.host && a.src == b.src && a.tgt == b.tgt && a.m == b.m && a.n == b.n &&
           a.max_iters == b.max_iters && a.L == b.L && a.flags == b.flags && a.eps == b.eps &&
           std::memcmp(&a.geom, &b.geom, sizeof(GridGeom)) == 0;
}

// A call can be replayed from a graph when nothing in it synchronises with
// the host or allocates: the dense grid, a grid geometry that the call does
// not refit (explicit, or kept), no kernel timing, graphs not switched off.
bool graphable(const vicp_ctx *c)
{
    const uint32_t f = c->params.flags;
    if ((f & VICP_FLAG_NO_GRAPH) || (f & VICP_FLAG_SPARSE_GRID) || c->profiling || c->rg_broken || !c->have_geom)
        return false;
    return c->params.dims[0] > 0 || (f & VICP_FLAG_KEEP_GRID);
}

// Captures the call's work (on the private stream, with the context's
// stream redirected to it) into rg_exec.  The double-buffered occupancy and
// brick-bound buffers that the first build of the call fills are reset at
// the start, so that a replay does not depend on how many builds came
// before it.
vicp_status capture_registration(vicp_ctx *c, const vicp_ctx::RegKey &key, const float4 *src, const float *tgt,
                                 const float *src_host, const float *tgt_host)
{
    if (!c->gstream) {
        if (cudaStreamCreateWithFlags(&c->gstream, cudaStreamNonBlocking) != cudaSuccess ||
            cudaMallocHost((void **)&c->h_pose, 16 * sizeof(double)) != cudaSuccess ||
            cudaMallocHost((void **)&c->h_out, sizeof(vicp_ctx::RegOut)) != cudaSuccess) {
            cudaGetLastError();
            c->rg_broken = true;
            return VICP_ERR_CUDA;
        }
    }
    if (c->rg_exec) {
        cudaGraphExecDestroy(c->rg_exec);
        c->rg_exec = nullptr;
    }
    cudaStream_t saved = c->stream;
    const bool saved_after = c->after_solve;
    const int saved_occ = c->occ_cur;
    const int64_t launches0 = c->launches;
    c->stream = c->gstream;
    c->capturing = true;
    c->nns_in_capture = false;
    c->after_solve = false;
    cudaGraph_t g = nullptr;
    vicp_status s = VICP_OK;
    // A page-locked host target is read by the first histogram itself (its
    // device-mapped address); a pageable one is copied first.
    const float *tgt_mapped = nullptr;
    if (key.host) {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, tgt_host) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
            pa.devicePointer && (reinterpret_cast<uintptr_t>(pa.devicePointer) & 15u) == 0)
            tgt_mapped = static_cast<const float *>(pa.devicePointer);
        cudaGetLastError();
    }
    cudaError_t e = cudaStreamBeginCapture(c->gstream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        // the buffers the call's first build fills are reset on the copy
        // stream (with host clouds: beside the target cloud's copy, or
        // before the histogram that reads it from host memory)
        const int first = c->occ_cur ^ 1;
        cudaStream_t rs = key.host ? c->copy : c->gstream;
        if (key.host) {
            e = cudaEventRecord(c->ev_fork, c->gstream);
            if (e == cudaSuccess)
                e = cudaStreamWaitEvent(c->copy, c->ev_fork, 0);
        }
        if (e == cudaSuccess)
            e = cudaMemsetAsync(c->occ[first].p, 0, c->occ[first].bytes, rs);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(c->boxk[first].p, 0xff, c->boxk[first].bytes, rs);
        if (e == cudaSuccess && key.host && tgt_mapped) {   // the source is copied after the histogram
            e = cudaEventRecord(c->ev_clr, c->copy);
            if (e == cudaSuccess)
                e = cudaStreamWaitEvent(c->gstream, c->ev_clr, 0);
        } else if (e == cudaSuccess && key.host) {
            const size_t sb = (size_t)key.m * 16, tb = (size_t)key.n * 16;
            e = cudaEventRecord(c->ev_clr, c->copy);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->htgt.p, tgt_host, tb, cudaMemcpyHostToDevice, c->gstream);
            if (e == cudaSuccess)
                e = cudaStreamWaitEvent(c->gstream, c->ev_clr, 0);
            if (e == cudaSuccess)
                e = cudaEventRecord(c->ev_copy_go, c->gstream);
            if (e == cudaSuccess)
                e = cudaStreamWaitEvent(c->copy, c->ev_copy_go, 0);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(c->hsrc.p, src_host, sb, cudaMemcpyHostToDevice, c->copy);
            if (e == cudaSuccess)
                e = cudaEventRecord(c->ev_src, c->copy);
        }
        if (e == cudaSuccess)
            s = registration_work(c, src, key.m, tgt, key.n, c->h_pose, c->h_out->pose, &c->h_out->ctl, key.host,
                                  tgt_mapped, tgt_mapped ? src_host : nullptr);
        const cudaError_t e2 = cudaStreamEndCapture(c->gstream, &g);
        if (e == cudaSuccess)
            e = e2;
    }
    if (e == cudaSuccess && s == VICP_OK)
        e = cudaGraphInstantiate(&c->rg_exec, g, 0);
    if (g)
        cudaGraphDestroy(g);
    c->stream = saved;
    c->capturing = false;
    // an event last recorded inside the capture names a node of the graph,
    // and a later direct launch may not wait for it: every event the work
    // records is recorded again, outside the capture, on the context's stream
    for (cudaEvent_t ev : {c->ev_hist, c->ev_nns, c->ev_dil, c->ev_copy_go, c->ev_src, c->ev_fork, c->ev_clr})
        if (cudaEventRecord(ev, saved) != cudaSuccess && e == cudaSuccess)
            e = cudaErrorUnknown;
    c->after_solve = false;
    c->rg_launches = c->launches - launches0;
    c->launches = launches0;   // counted when replayed
    if (e != cudaSuccess || s != VICP_OK) {
        // capture unavailable for this call (for example pageable host
        // clouds): launch directly from now on; the host state the capture
        // advanced is put back
        cudaGetLastError();
        c->rg_exec = nullptr;
        c->rg_broken = true;
        c->occ_cur = saved_occ;
        c->after_solve = saved_after;
        return VICP_ERR_CUDA;
    }
    c->rg_key = key;
    return VICP_OK;
}

vicp_status replay_registration(vicp_ctx *c, double pose_host[16], int32_t *iters_out, double *rmse_out)
{
    std::memcpy(c->h_pose, pose_host, 16 * sizeof(double));
    // launched into the context's stream itself: ordered after everything
    // issued there before, with no event between them
    cudaError_t e = cudaGraphLaunch(c->rg_exec, c->stream);
    if (e == cudaSuccess)
        e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "graph replay");
    c->launches += c->rg_launches;
    c->after_solve = false;
    std::memcpy(pose_host, c->h_out->pose, 16 * sizeof(double));
    if (iters_out)
        *iters_out = c->h_out->ctl.iters;
    if (rmse_out)
        *rmse_out = c->h_out->ctl.last_rmse;
    return device_status_from(c, c->h_out->ctl.err);
}

vicp_status registration(vicp_ctx *c, const float4 *src, int32_t m, const float *tgt, int32_t n,
                         double pose_host[16], int32_t *iters_out, double *rmse_out,
                         const float *src_host = nullptr, const float *tgt_host = nullptr)
{
    vicp_ctx::RegKey key;
    key.host = src_host != nullptr;
    key.src = key.host ? (const void *)src_host : (const void *)src;
    key.tgt = key.host ? (const void *)tgt_host : (const void *)tgt;
    key.m = m;
    key.n = n;
    key.max_iters = c->params.max_iters;
    key.L = c->params.dilation_layers;
    key.flags = c->params.flags;
    key.eps = c->params.rmse_eps;
    key.geom = c->geom;
    c->rg_replayed = false;
    if (graphable(c)) {
        if (c->rg_exec && same_call(key, c->rg_key)) {
            c->rg_replayed = true;
            return replay_registration(c, pose_host, iters_out, rmse_out);
        }
        // the second call in a row with the same arguments: capture it
        if (c->rg_last_valid && same_call(key, c->rg_last) &&
            capture_registration(c, key, src, tgt, src_host, tgt_host) == VICP_OK) {
            c->rg_replayed = true;
            return replay_registration(c, pose_host, iters_out, rmse_out);
        }
    }
    if (key.host) {   // the direct path issues the copies itself
        const size_t sb = (size_t)m * 16, tb = (size_t)n * 16;
        cudaError_t e = cudaMemcpyAsync(c->htgt.p, tgt_host, tb, cudaMemcpyHostToDevice, c->stream);
        c->after_solve = false;   // the build's histogram reads what this copy writes
        if (e == cudaSuccess)
            e = cudaEventRecord(c->ev_copy_go, c->stream);
        if (e == cudaSuccess)
            e = cudaStreamWaitEvent(c->copy, c->ev_copy_go, 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(c->hsrc.p, src_host, sb, cudaMemcpyHostToDevice, c->copy);
        if (e == cudaSuccess)
            e = cudaEventRecord(c->ev_src, c->copy);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "host-to-device copy of the clouds");
    }
    DevCtl ctl_h;
    TRY(registration_work(c, src, m, tgt, n, pose_host, pose_host, &ctl_h, key.host));
    const cudaError_t se = cudaStreamSynchronize(c->stream);
    if (se != cudaSuccess)
        return cuda_fail(c, se, "synchronise");
    vicp_status st = device_status_from(c, ctl_h.err);
    if (iters_out)
        *iters_out = ctl_h.iters;
    if (rmse_out)
        *rmse_out = ctl_h.last_rmse;
    key.geom = c->geom;   // as fitted by this call
    c->rg_last = key;
    c->rg_last_valid = st == VICP_OK || st == VICP_ERR_DEGENERATE;
    return st;
}

// The sparse grid's memory accounting: the same figures as the dense
// grid's, from the occupied-voxel table (its slot offsets are valid at
// occupied slots and just past them).  Synchronous.
vicp_status memory_report_sparse(vicp_ctx *c, vicp_memory *out)
{
    const GridGeom &g = c->geom;
    DevCtl *d = ctl_of(c);
    TRY(launch(c, K_MAXCOUNT, [&] {
        return launch_maxcount((const unsigned *)c->ooff.p, slot_geom(c->cap_o), d, c->stream,
                               (const unsigned *)c->okeys[c->o_cur].p);
    }));
    unsigned mc[2] = {0, 0};
    uint32_t stored = 0;
    int32_t nbricks = 0;
    cudaError_t e = cudaMemcpyAsync(mc, &d->max_count, sizeof mc, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&nbricks, &d->n_bricks, sizeof nbricks, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&stored, (const unsigned *)c->ooff.p + c->cap_o, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "memory report read-back");
    vicp_status st = read_device_status(c);
    const uint64_t V = (uint64_t)g.V, So = (uint64_t)c->cap_o, Sl = (uint64_t)c->cap_l, Sr = (uint64_t)c->cap_r;
    out->static_bytes = So * 4 * 3 + 4;   // occupied-voxel table: keys, counts, offsets
    // + ids + the labelled-segment table (keys, masks and first roots) and the roots
    out->csr_store_bytes = So * 4 * 2 + 4 + (uint64_t)stored * 4 + Sl * 12 + Sr * 4;
    out->max_voxel_count = mc[0];
    out->occupied_voxels = mc[1];
    out->nonempty_bricks = (uint32_t)nbricks;
    out->fixed_capacity_bytes = V * (uint64_t)mc[0] * 4;
    out->paper_static_layout_bytes = V * 65536ull;
    out->labelled_voxels = (uint32_t)c->lab_count;
    return st;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================
extern "C" {

int32_t vicp_abi_version(void) { return VICP_ABI_VERSION; }

const char *vicp_status_string(vicp_status s)
{
    switch (s) {
    case VICP_OK: return "ok";
    case VICP_ERR_INVALID: return "invalid argument";
    case VICP_ERR_CUDA: return "CUDA error";
    case VICP_ERR_OOM: return "out of device memory";
    case VICP_ERR_GRID_TOO_LARGE: return "grid too large";
    case VICP_ERR_TIMEOUT: return "device-side wait timed out";
    case VICP_ERR_STATE: return "call order";
    case VICP_ERR_DEGENERATE: return "degenerate geometry";
    }
    return "unknown status";
}

void vicp_default_params(vicp_params *p)
{
    if (!p)
        return;
    std::memset(p, 0, sizeof *p);
    p->voxel_size = 0.0f;
    p->grid_divisions = 16;
    p->dims[0] = p->dims[1] = p->dims[2] = 0;
    p->dilation_layers = 10;
    p->max_iters = 50;
    p->rmse_eps = 1e-5;
    p->flags = 0u;
}

vicp_status vicp_create(vicp_ctx **out, const vicp_params *params, const vicp_allocator *alloc, void *cuda_stream)
{
    if (!out || !params)
        return VICP_ERR_INVALID;
    *out = nullptr;
    if (alloc && (!alloc->alloc || !alloc->free))
        return VICP_ERR_INVALID;
    vicp_ctx *c = new vicp_ctx();
    c->params = *params;
    vicp_status s = check_params(c, params);
    if (s != VICP_OK) {
        delete c;
        return s;
    }
    if (alloc) {
        c->alloc = *alloc;
        c->custom_alloc = true;
    }
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    cudaGetDevice(&c->device);
    if (cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_hist, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_nns, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_dil, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&c->copy, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_copy_go, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_src, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_clr, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        vicp_destroy(c);
        return VICP_ERR_CUDA;
    }
    if (cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || c->sms < 1) {
        cudaGetLastError();
        c->sms = 152;
    }
    s = buf_alloc(c, c->ctl, sizeof(vicp_ctx::RegOut), "control block and registration pose");
    if (s == VICP_OK)
        s = buf_zero(c, c->ctl, "zero control block");
    if (s == VICP_OK)
        s = buf_alloc(c, c->partials, REDUCE_MAX_BLOCKS * REDUCE_VALUES * sizeof(float2), "partials");
    if (s == VICP_OK)
        s = buf_alloc(c, c->rmse, sizeof(double), "rmse");
    if (s == VICP_OK)
        s = buf_alloc(c, c->bbox, 8 * sizeof(unsigned), "bounding box");
    if (s != VICP_OK) {
        vicp_destroy(c);
        return s;
    }
    *out = c;
    return VICP_OK;
}

void vicp_destroy(vicp_ctx *c)
{
    if (!c)
        return;
    cudaStreamSynchronize(c->stream);
    if (c->side)
        cudaStreamSynchronize(c->side);
    Buf *all[] = {&c->counts,  &c->off,      &c->root,       &c->ring,       &c->occ[0],    &c->occ[1], &c->desc, &c->tile_sum,
                  &c->inter,       &c->uflag,      &c->zdirty,
                  &c->bcounts, &c->boff,     &c->brick_list, &c->brick_range, &c->brick_box, &c->bslot,
                  &c->boxk[0], &c->boxk[1], &c->sb_box,     &c->sb_left,    &c->keys,
                  &c->ids,     &c->csr,      &c->bpts,       &c->outside,    &c->nn,        &c->d2,
                  &c->fb_list, &c->hv_list, &c->hv_range, &c->partials, &c->rmse,       &c->ctl,       &c->bbox,
                  &c->hsrc,    &c->htgt,    &c->fslots,   &c->fcount,   &c->fover,
                  &c->okeys[0], &c->okeys[1], &c->ocount, &c->ooff, &c->socc[0], &c->socc[1], &c->stile, &c->sdesc,
                  &c->pslot,   &c->lkeys,   &c->lseg,     &c->lroot,    &c->lparts};
    for (Buf *b : all)
        buf_free(c, *b);
    for (auto &t : c->pending) {
        cudaEventDestroy(t.start);
        cudaEventDestroy(t.stop);
    }
    for (cudaEvent_t e : c->event_pool)
        cudaEventDestroy(e);
    if (c->copy)
        cudaStreamSynchronize(c->copy);
    if (c->gstream)
        cudaStreamSynchronize(c->gstream);
    if (c->rg_exec)
        cudaGraphExecDestroy(c->rg_exec);
    if (c->h_pose)
        cudaFreeHost(c->h_pose);
    if (c->h_out)
        cudaFreeHost(c->h_out);
    if (c->gstream)
        cudaStreamDestroy(c->gstream);
    for (cudaEvent_t e : {c->ev_hist, c->ev_nns, c->ev_dil, c->ev_copy_go, c->ev_src, c->ev_fork, c->ev_clr})
        if (e)
            cudaEventDestroy(e);
    if (c->side)
        cudaStreamDestroy(c->side);
    if (c->copy)
        cudaStreamDestroy(c->copy);
    delete c;
}

vicp_status vicp_set_stream(vicp_ctx *c, void *cuda_stream)
{
    if (!c)
        return VICP_ERR_INVALID;
    c->stream = static_cast<cudaStream_t>(cuda_stream);
    c->after_solve = false;
    return VICP_OK;   // a captured registration orders itself after this stream at each replay
}

vicp_status vicp_build_grid(vicp_ctx *c, const float *target_xyzw, int32_t n_target)
{
    if (!c)
        return VICP_ERR_INVALID;
    return build(c, target_xyzw, n_target);
}

vicp_status vicp_dilate(vicp_ctx *c, int32_t layers)
{
    if (!c)
        return VICP_ERR_INVALID;
    return dilate(c, layers);
}

vicp_status vicp_correspond(vicp_ctx *c, const float *src_xyzw, int32_t n_src, const double *pose_dev,
                            int32_t *nn_out, float *d2_out, int32_t *n_fallback_out)
{
    if (!c)
        return VICP_ERR_INVALID;
    TRY(check_cloud(c, src_xyzw, n_src, "source"));
    if (!pose_dev || !nn_out || !d2_out)
        return fail(c, VICP_ERR_INVALID, "pose, nn and d2 pointers must be non-NULL");
    if (!c->built || c->dilated_L < 0)
        return fail(c, VICP_ERR_STATE, "vicp_correspond needs vicp_build_grid and vicp_dilate first");
    TRY(ensure_query_buffers(c, n_src));
    const float4 *src = reinterpret_cast<const float4 *>(src_xyzw);
    DevCtl *d = ctl_of(c);
    if (n_fallback_out) {
        // fb_count is zero between searches; the correspond kernel counts this
        // search's global queries and the fallback kernel clears it again.
        TRY(run_localised(c, src, n_src, pose_dev, nn_out, d2_out, 0));
        cudaError_t e = cudaMemcpyAsync(n_fallback_out, &d->fb_count, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                        c->stream);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "fallback count copy");
        TRY(launch(c, K_FALLBACK, [&] {
            return launch_fallback(src, pose_dev, (const float4 *)c->bpts.p, (const float4 *)c->brick_box.p,
                                   (const float4 *)c->sb_box.p, c->target, c->n_target, (const int *)c->outside.p,
                                   (const int *)c->fb_list.p, (const int *)c->hv_list.p,
                                   (const uint2 *)c->hv_range.p, (const float4 *)c->csr.p, d, nn_out, d2_out, n_src, 0,
                                   c->stream);
        }));
        e = cudaEventRecord(c->ev_nns, c->stream);   // a later dilation waits for this search
        return e == cudaSuccess ? VICP_OK : cuda_fail(c, e, "event record");
    }
    return run_nns(c, src, n_src, pose_dev, nn_out, d2_out, 0);
}

vicp_status vicp_step(vicp_ctx *c, const float *src_xyzw, int32_t n_src, double *pose_dev, double *rmse_dev)
{
    if (!c)
        return VICP_ERR_INVALID;
    TRY(check_cloud(c, src_xyzw, n_src, "source"));
    if (!pose_dev)
        return fail(c, VICP_ERR_INVALID, "pose pointer must be non-NULL");
    if (!c->built || c->dilated_L < 0)
        return fail(c, VICP_ERR_STATE, "vicp_step needs vicp_build_grid and vicp_dilate first");
    return run_step(c, reinterpret_cast<const float4 *>(src_xyzw), n_src, pose_dev, rmse_dev, 0);
}

vicp_status vicp_register(vicp_ctx *c, const float *src_xyzw, int32_t n_src, const float *tgt_xyzw, int32_t n_tgt,
                          double pose_host[16], int32_t *iters_out, double *rmse_out)
{
    if (!c)
        return VICP_ERR_INVALID;
    TRY(check_cloud(c, src_xyzw, n_src, "source"));
    TRY(check_cloud(c, tgt_xyzw, n_tgt, "target"));
    if (!pose_host)
        return fail(c, VICP_ERR_INVALID, "pose_host must be non-NULL");
    return registration(c, reinterpret_cast<const float4 *>(src_xyzw), n_src, tgt_xyzw, n_tgt, pose_host,
                        iters_out, rmse_out);
}

vicp_status vicp_register_host(vicp_ctx *c, const float *src_host, int32_t n_src, const float *tgt_host,
                               int32_t n_tgt, double pose_host[16], int32_t *iters_out, double *rmse_out)
{
    if (!c)
        return VICP_ERR_INVALID;
    if (!src_host || !tgt_host || n_src < 1 || n_tgt < 1 || !pose_host)
        return fail(c, VICP_ERR_INVALID, "host clouds, sizes >= 1 and pose_host are required");
    const size_t sb = (size_t)n_src * 16, tb = (size_t)n_tgt * 16;
    if (c->hsrc.bytes < sb)
        TRY(buf_alloc(c, c->hsrc, sb, "source copy"));
    if (c->htgt.bytes < tb)
        TRY(buf_alloc(c, c->htgt, tb, "target copy"));
    // The target on the context's stream (the build needs it first); the
    // source on the copy stream, after everything issued so far on the
    // context's stream (earlier searches may still read the buffer), so it
    // travels while the grid is built; the first search waits for it.
    return registration(c, (const float4 *)c->hsrc.p, n_src, (const float *)c->htgt.p, n_tgt, pose_host,
                        iters_out, rmse_out, src_host, tgt_host);
}

vicp_status vicp_get_grid(vicp_ctx *c, vicp_grid_view *out)
{
    if (!c || !out)
        return VICP_ERR_INVALID;
    if (!c->built)
        return fail(c, VICP_ERR_STATE, "no grid built");
    if (sparse_of(c))
        return fail(c, VICP_ERR_STATE, "the sparse grid has no dense arrays: use vicp_get_sparse_grid");
    const GridGeom &g = c->geom;
    std::memset(out, 0, sizeof *out);
    out->origin[0] = g.ox;
    out->origin[1] = g.oy;
    out->origin[2] = g.oz;
    out->voxel_size = g.h;
    out->inv_voxel_size = g.inv_h;
    out->dims[0] = g.nx;
    out->dims[1] = g.ny;
    out->dims[2] = g.nz;
    out->n_voxels = g.V;
    out->n_target = c->n_target;
    out->dilation_layers = c->dilated_L;
    TRY(dense_offsets(c));
    uint32_t stored = 0;
    cudaError_t e = cudaMemcpyAsync(&stored, (const unsigned *)c->off.p + g.V, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "read n_stored");
    vicp_status st = read_device_status(c);
    out->n_stored = (int32_t)stored;
    out->keys = (const int32_t *)c->keys.p;
    out->offsets = (const uint32_t *)c->off.p;
    out->ids = (const int32_t *)c->ids.p;
    out->csr_points = (const float *)c->csr.p;
    out->root = (const int32_t *)c->root.p;
    out->ring = (const uint8_t *)c->ring.p;
    out->occupancy = (const uint32_t *)c->occ[c->occ_cur].p;
    return st;
}

vicp_status vicp_get_sparse_grid(vicp_ctx *c, vicp_sparse_view *out)
{
    if (!c || !out)
        return VICP_ERR_INVALID;
    if (!sparse_of(c))
        return fail(c, VICP_ERR_STATE, "not a sparse-grid context (VICP_FLAG_SPARSE_GRID)");
    if (!c->built)
        return fail(c, VICP_ERR_STATE, "no grid built");
    const GridGeom &g = c->geom;
    std::memset(out, 0, sizeof *out);
    for (int a = 0; a < 3; ++a)
        out->origin[a] = a == 0 ? g.ox : (a == 1 ? g.oy : g.oz);
    out->voxel_size = g.h;
    out->inv_voxel_size = g.inv_h;
    out->dims[0] = g.nx;
    out->dims[1] = g.ny;
    out->dims[2] = g.nz;
    out->n_voxels = g.V;
    out->n_target = c->n_target;
    out->dilation_layers = c->dilated_L;
    uint32_t stored = 0;
    cudaError_t e = cudaMemcpyAsync(&stored, (const unsigned *)c->ooff.p + c->cap_o, 4, cudaMemcpyDeviceToHost,
                                    c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "read n_stored");
    vicp_status st = read_device_status(c);
    out->n_stored = (int32_t)stored;
    out->occupied_slots = c->cap_o;
    out->occupied_keys = (const uint32_t *)c->okeys[c->o_cur].p;
    out->occupied_offsets = (const uint32_t *)c->ooff.p;
    out->labelled_slots = c->dilated_L >= 0 ? c->cap_l : 0;
    out->labelled_keys = c->dilated_L >= 0 ? (const uint32_t *)c->lkeys.p : nullptr;
    out->labelled_segments = c->dilated_L >= 0 ? (const uint32_t *)c->lseg.p : nullptr;
    out->labelled_root = c->dilated_L >= 0 ? (const int32_t *)c->lroot.p : nullptr;
    out->labelled_voxels = c->dilated_L >= 0 ? c->lab_count : 0;
    out->labelled_segment_count = c->dilated_L >= 0 ? c->lab_segs : 0;
    out->keys = (const int32_t *)c->keys.p;
    out->ids = (const int32_t *)c->ids.p;
    out->csr_points = (const float *)c->csr.p;
    out->occupancy = (const uint32_t *)c->occ[c->occ_cur].p;
    return st;
}

vicp_status vicp_sync(vicp_ctx *c)
{
    if (!c)
        return VICP_ERR_INVALID;
    return read_device_status(c);
}

vicp_status vicp_memory_report(vicp_ctx *c, vicp_memory *out)
{
    if (!c || !out)
        return VICP_ERR_INVALID;
    std::memset(out, 0, sizeof *out);
    out->current_bytes = c->cur_bytes;
    out->peak_bytes = c->peak_bytes;
    if (!c->built)
        return VICP_OK;
    const GridGeom &g = c->geom;
    DevCtl *d = ctl_of(c);
    cudaError_t e = cudaMemsetAsync(&d->max_count, 0, 2 * sizeof(unsigned), c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "memory report");
    if (sparse_of(c))
        return memory_report_sparse(c, out);
    TRY(dense_offsets(c));
    TRY(launch(c, K_MAXCOUNT, [&] { return launch_maxcount((const unsigned *)c->off.p, g, d, c->stream); }));
    unsigned mc[2] = {0, 0};
    uint32_t stored = 0;
    int32_t nbricks = 0;
    e = cudaMemcpyAsync(mc, &d->max_count, sizeof mc, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&nbricks, &d->n_bricks, sizeof nbricks, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&stored, (const unsigned *)c->off.p + g.V, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "memory report read-back");
    vicp_status st = read_device_status(c);
    const uint64_t V = (uint64_t)g.V;
    out->static_bytes = V * 4 + (V + 1) * 4;
    out->csr_store_bytes = (V + 1) * 4 + (uint64_t)stored * 4 + V * 4 + V;
    out->max_voxel_count = mc[0];
    out->occupied_voxels = mc[1];
    out->nonempty_bricks = (uint32_t)nbricks;
    out->fixed_capacity_bytes = V * (uint64_t)mc[0] * 4;
    out->paper_static_layout_bytes = V * 65536ull;
    return st;
}

vicp_status vicp_profile_enable(vicp_ctx *c, int32_t enable)
{
    if (!c)
        return VICP_ERR_INVALID;
    c->profiling = enable != 0;
    return VICP_OK;
}

vicp_status vicp_fixed_build(vicp_ctx *c, const float *target_xyzw, int32_t n, int32_t capacity,
                             uint32_t *overflow_out, uint64_t *store_bytes_out)
{
    if (!c)
        return VICP_ERR_INVALID;
    if (sparse_of(c))
        return fail(c, VICP_ERR_STATE, "the fixed-capacity store needs the dense grid's labels");
    TRY(check_cloud(c, target_xyzw, n, "target"));
    if (capacity < 1)
        return fail(c, VICP_ERR_INVALID, "capacity must be >= 1");
    if (!c->built || reinterpret_cast<const float4 *>(target_xyzw) != c->target || n != c->n_target)
        return fail(c, VICP_ERR_STATE, "vicp_fixed_build needs vicp_build_grid on the same target first");
    const GridGeom &g = c->geom;
    if ((unsigned long long)g.V * (unsigned long long)capacity >= (1ull << 32))
        return fail(c, VICP_ERR_GRID_TOO_LARGE, "%lld voxels x %d slots exceed 2^32 slots", g.V, capacity);
    const size_t slot_bytes = (size_t)g.V * (size_t)capacity * 16;
    if (c->fslots.bytes < slot_bytes)
        TRY(buf_alloc(c, c->fslots, slot_bytes, "fixed-capacity slots"));
    if (c->fcount.bytes < (size_t)g.V * 4)
        TRY(buf_alloc(c, c->fcount, (size_t)g.V * 4, "fixed-capacity counts"));
    if (!c->fover.p)
        TRY(buf_alloc(c, c->fover, 4, "overflow counter"));
    cudaError_t e = cudaMemsetAsync(c->fcount.p, 0, (size_t)g.V * 4, c->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->fover.p, 0, 4, c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "fixed-capacity reset");
    c->fixed_C = (unsigned)capacity;
    TRY(launch(c, K_FIXED_SCATTER, [&] {
        return launch_fixed_scatter(reinterpret_cast<const float4 *>(target_xyzw), n, g, c->fixed_C,
                                    (unsigned *)c->fcount.p, (float4 *)c->fslots.p, (unsigned *)c->fover.p,
                                    c->stream);
    }));
    c->fixed_built = true;
    unsigned over = 0;
    e = cudaMemcpyAsync(&over, c->fover.p, 4, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "overflow read-back");
    TRY(read_device_status(c));   // synchronises
    if (overflow_out)
        *overflow_out = over;
    if (store_bytes_out)
        *store_bytes_out = (uint64_t)slot_bytes + (uint64_t)g.V * 4;
    return VICP_OK;
}

vicp_status vicp_fixed_view(vicp_ctx *c, const float **slots_out, const uint32_t **fill_out, int32_t *capacity_out)
{
    if (!c)
        return VICP_ERR_INVALID;
    if (!c->fixed_built)
        return fail(c, VICP_ERR_STATE, "vicp_fixed_view needs vicp_fixed_build first");
    TRY(read_device_status(c));   // synchronises
    if (slots_out)
        *slots_out = static_cast<const float *>(c->fslots.p);
    if (fill_out)
        *fill_out = static_cast<const uint32_t *>(c->fcount.p);
    if (capacity_out)
        *capacity_out = (int32_t)c->fixed_C;
    return VICP_OK;
}

vicp_status vicp_fixed_correspond(vicp_ctx *c, const float *src_xyzw, int32_t n_src, const double *pose_dev,
                                  int32_t *nn_out, float *d2_out, int32_t *n_fallback_out)
{
    if (!c)
        return VICP_ERR_INVALID;
    TRY(check_cloud(c, src_xyzw, n_src, "source"));
    if (!pose_dev || !nn_out || !d2_out)
        return fail(c, VICP_ERR_INVALID, "pose, nn and d2 pointers must be non-NULL");
    if (!c->fixed_built || c->dilated_L < 0)
        return fail(c, VICP_ERR_STATE, "vicp_fixed_correspond needs vicp_fixed_build and vicp_dilate first");
    TRY(ensure_query_buffers(c, n_src));
    const float4 *src = reinterpret_cast<const float4 *>(src_xyzw);
    DevCtl *d = ctl_of(c);
    TRY(launch(c, K_FIXED_CORRESPOND, [&] {
        return launch_correspond_fixed(src, n_src, pose_dev, c->geom, (const int *)c->root.p,
                                       (const unsigned *)c->fcount.p, c->fixed_C, (const float4 *)c->fslots.p,
                                       nn_out, d2_out, (int *)c->fb_list.p, (int *)c->hv_list.p,
                                       (uint2 *)c->hv_range.p, d, c->stream);
    }));
    if (n_fallback_out) {
        cudaError_t e = cudaMemcpyAsync(n_fallback_out, &d->fb_count, sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                        c->stream);
        if (e != cudaSuccess)
            return cuda_fail(c, e, "fallback count copy");
    }
    // global searches over the brick level of the CSR build; dense segments
    // are scanned in the slots
    TRY(launch(c, K_FALLBACK, [&] {
        return launch_fallback(src, pose_dev, (const float4 *)c->bpts.p, (const float4 *)c->brick_box.p,
                               (const float4 *)c->sb_box.p, c->target, c->n_target, (const int *)c->outside.p,
                               (const int *)c->fb_list.p, (const int *)c->hv_list.p, (const uint2 *)c->hv_range.p,
                               (const float4 *)c->fslots.p, d, nn_out, d2_out, n_src, 0, c->stream);
    }));
    cudaError_t e = cudaEventRecord(c->ev_nns, c->stream);
    return e == cudaSuccess ? VICP_OK : cuda_fail(c, e, "event record");
}

int32_t vicp_kernel_count(void) { return K_COUNT; }

const char *vicp_kernel_name(int32_t k) { return kernel_name(k); }

vicp_status vicp_profile_read(vicp_ctx *c, int64_t *launches, double *total_ms)
{
    if (!c)
        return VICP_ERR_INVALID;
    vicp_status st = read_device_status(c);   // synchronises
    for (auto &t : c->pending) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, t.start, t.stop) == cudaSuccess) {
            c->prof_ms[t.kernel] += ms;
            c->prof_launches[t.kernel] += 1;
        }
        c->event_pool.push_back(t.start);
        c->event_pool.push_back(t.stop);
    }
    c->pending.clear();
    for (int k = 0; k < K_COUNT; ++k) {
        if (launches)
            launches[k] = c->prof_launches[k];
        if (total_ms)
            total_ms[k] = c->prof_ms[k];
        c->prof_launches[k] = 0;
        c->prof_ms[k] = 0.0;
    }
    return st;
}

vicp_status vicp_read_stats(vicp_ctx *c, vicp_stats *out, int32_t reset)
{
    if (!c || !out)
        return VICP_ERR_INVALID;
    DevCtl *d = ctl_of(c);
    unsigned long long v[4] = {0, 0, 0, 0};
    static_assert(offsetof(DevCtl, stat_global_cand) - offsetof(DevCtl, stat_queries) == 24, "stats layout");
    cudaError_t e = cudaMemcpyAsync(v, &d->stat_queries, sizeof v, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && reset)
        e = cudaMemsetAsync(&d->stat_queries, 0, sizeof v, c->stream);
    if (e != cudaSuccess)
        return cuda_fail(c, e, "read stats");
    vicp_status st = read_device_status(c);
    out->queries = v[0];
    out->fallbacks = v[1];
    out->local_candidates = v[2];
    out->global_candidates = v[3];
    return st;
}

int64_t vicp_launch_count(const vicp_ctx *c) { return c ? c->launches : 0; }

const char *vicp_last_error(const vicp_ctx *c) { return c ? c->last_error.c_str() : ""; }

int32_t vicp_graph_replayed(const vicp_ctx *c)
{
    if (!c)
        return -1;
    return c->rg_replayed ? 1 : 0;
}

}  // extern "C"

namespace vicp {
const char *kernel_name(int k)
{
    static const char *names[K_COUNT] = {"bbox",       "histogram", "scan",     "scatter",      "brick_scan",
                                         "dilate",   "correspond", "fallback", "reduce_solve",
                                         "maxcount",   "fixed_scatter", "fixed_correspond", "offsets_fill",
                                         "reduce_solve_f64"};
    return (k >= 0 && k < K_COUNT) ? names[k] : "?";
}
}  // namespace vicp
