/*
 * vicp_oracle.c -- plain, slow CPU oracle for the dilation-based ICP hot path
 * (VANICP with per-voxel dynamic memory assignment, arXiv 2512.04996).
 *
 * TEST INFRASTRUCTURE ONLY.  The tests, the smoke check and the benchmark's
 * CPU-baseline leg call it; the product (CUDA) path never does, and this file
 * shares no code, header, table or constant generator with it.
 *
 * Every function restates one step of the paper in the most direct form:
 * no blocking, no fusion, no reordering.  Floating-point arithmetic is plain
 * C `float`/`double` compiled with -ffp-contract=off, so each operation is
 * rounded exactly once, in source order.
 *
 * The file is compiled twice: plain (one thread), and with OpenMP, where the
 * loops whose iterations are independent of one another -- the keys of the
 * points, the voxels of one dilation round, the searches of the source
 * points -- are shared out over threads.  Every iteration computes exactly
 * what it computes in the plain build and writes only its own outputs, and
 * every loop that accumulates (histogram, CSR fill, reductions) stays
 * sequential, so both builds give bit-identical results.
 *
 * Readings of the paper where it is silent or ambiguous (each is applied
 * identically by the CUDA path, and each is pinned by a test):
 *   - Grid: origin = component-wise minimum of the target, voxel edge h
 *     given or = extent / divisions, inv_h = (float)(1.0/(double)h),
 *     dims_a = floor(ext_a * inv_h) + 1; any dims, not only powers of two
 *     (Sec. 4.1 "Parameter" fixes 2^N per axis for unit-sphere clouds).
 *   - Concat (Alg. 1/2/4): x is the fastest axis, key = x + nx*(y + ny*z),
 *     as implied by the neighbour offsets {+-1, +-2^N, +-2^2N} of Alg. 3.
 *   - A point is outside the grid when a scaled coordinate is NaN, < 0 or
 *     >= dims_a.  Outside target points are not stored; outside source
 *     points take the global search, like empty voxels (Alg. 4).
 *   - Offsets drop the two header words per voxel of Alg. 1's CPU part:
 *     off[v] = sum_{u<v} count[u]; the paper's address is off[v] + 2v.
 *   - CSR order inside a voxel segment is ascending point index (Alg. 2's
 *     lock order leaves it unspecified; any order is a valid segment).
 *   - Dilation (Alg. 3): L synchronous rounds over the six in-grid face
 *     neighbours; a newly reached voxel stores the smallest root index among
 *     its already-labelled neighbours (the label is the root voxel, Sec. 3).
 *   - NNS (Alg. 4): only the root voxel's segment is searched; squared
 *     distance ((dx*dx + dy*dy) + dz*dz) in float; strict minimum, ties to the
 *     smaller target index, a NaN distance after every number.  R, t are
 *     the float-rounded pose entries and s_a = ((R_a0*x + R_a1*y) + R_a2*z) + t_a.
 *   - Grid fit ignores NaN coordinates; a target without any finite
 *     coordinate on some axis has no grid (status 1).
 *   - Rigid update (Eq. 1): no rejection; centroids and cross-covariance in
 *     double (two passes); SVD by one-sided Jacobi; reflection fixed by
 *     diag(1,1,sign det(V U^T)); pose T <- dT * T; source points are always
 *     transformed from the original cloud by the accumulated T.
 *   - rank(H) < 2 (||cof(H)||_F <= 1e-12 ||H||_F^2) is degenerate: status 7,
 *     pose unchanged.
 *   - Early stop (Sec. 4.1): after iteration k >= 1 applied its update, stop
 *     when |rmse_k - rmse_{k-1}| < eps (eps <= 0 disables it).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OG_OK 0
#define OG_ERR_INVALID 1
#define OG_ERR_DEGENERATE 7

/* Grid geometry.  Layout is shared with the ctypes wrapper only. */
typedef struct {
    float origin[3];
    float h;       /* voxel edge                           */
    float inv_h;   /* (float)(1.0 / (double)h)             */
    int32_t dims[3];
} og_grid;

/* Threads of the OpenMP build (1 in the plain build). */
int32_t og_set_threads(int32_t n)
{
#ifdef _OPENMP
    if (n >= 1)
        omp_set_num_threads(n);
    return (int32_t)omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Grid fitting (Sec. 4.1 "Parameter"; reading: bounding-box origin)        */
/* ------------------------------------------------------------------------ */
int og_fit_grid(const float *tgt, int32_t n, float voxel_size, int32_t divisions, og_grid *g)
{
    if (n < 1)
        return OG_ERR_INVALID;
    /* NaN coordinates never compare less or greater, so they are left out. */
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    for (int32_t j = 0; j < n; ++j)
        for (int a = 0; a < 3; ++a) {
            float c = tgt[4 * (int64_t)j + a];
            if (c < lo[a]) lo[a] = c;
            if (c > hi[a]) hi[a] = c;
        }
    for (int a = 0; a < 3; ++a)
        if (!isfinite(lo[a]) || !isfinite(hi[a]))
            return OG_ERR_INVALID;
    float ext[3];
    float extent = 0.0f;
    for (int a = 0; a < 3; ++a) {
        ext[a] = hi[a] - lo[a];
        if (ext[a] > extent) extent = ext[a];
    }
    float h;
    if (voxel_size > 0.0f)
        h = voxel_size;
    else {
        if (divisions < 1)
            return OG_ERR_INVALID;
        h = extent / (float)divisions;
        if (!(h > 0.0f))
            h = 1.0f; /* all target points coincide: one voxel */
    }
    if (!isfinite(h))
        return OG_ERR_INVALID;
    g->h = h;
    g->inv_h = (float)(1.0 / (double)h);
    for (int a = 0; a < 3; ++a) {
        g->origin[a] = lo[a];
        float s = ext[a] * g->inv_h;
        if (!(s < 2147483520.0f))
            return OG_ERR_INVALID;
        g->dims[a] = (int32_t)floorf(s) + 1;
    }
    return OG_OK;
}

int64_t og_num_voxels(const og_grid *g)
{
    return (int64_t)g->dims[0] * g->dims[1] * g->dims[2];
}

/* ------------------------------------------------------------------------ */
/* Quantize + Concat (Alg. 1 / Alg. 2 first lines, Alg. 4 "Scale")          */
/* ------------------------------------------------------------------------ */
int32_t og_voxel_key(const og_grid *g, float x, float y, float z)
{
    float p[3] = {x, y, z};
    int32_t i[3];
    for (int a = 0; a < 3; ++a) {
        float d = p[a] - g->origin[a];
        float s = d * g->inv_h;
        if (!(s >= 0.0f) || s >= (float)g->dims[a])
            return -1;
        i[a] = (int32_t)floorf(s);
    }
    return i[0] + g->dims[0] * (i[1] + g->dims[1] * i[2]);
}

void og_keys(const og_grid *g, const float *pts, int32_t n, int32_t *keys)
{
#pragma omp parallel for schedule(static)
    for (int32_t j = 0; j < n; ++j) {
        const float *q = pts + 4 * (int64_t)j;
        keys[j] = og_voxel_key(g, q[0], q[1], q[2]);
    }
}

/* ------------------------------------------------------------------------ */
/* VOH: voxel occupancy histogram (Alg. 1, GPU part)                        */
/* ------------------------------------------------------------------------ */
void og_histogram(const int32_t *keys, int32_t n, int64_t V, uint32_t *counts)
{
    memset(counts, 0, (size_t)V * sizeof(uint32_t));
    for (int32_t j = 0; j < n; ++j)
        if (keys[j] >= 0)
            counts[keys[j]] += 1;
}

/* ------------------------------------------------------------------------ */
/* MOC: memory offsets (Alg. 1, CPU part) without the two header words      */
/* ------------------------------------------------------------------------ */
void og_offsets(const uint32_t *counts, int64_t V, uint32_t *off)
{
    uint32_t head = 0;
    for (int64_t v = 0; v < V; ++v) {
        off[v] = head;
        head += counts[v];
    }
    off[V] = head;
}

/* The paper's own layout: every voxel segment holds two header words
 * (lock, count-or-mask) before its point indices, so the start address of
 * voxel v advances by count+2 (Alg. 1, CPU part, written as stated there). */
void og_paper_moc(const uint32_t *counts, int64_t V, uint32_t *addr)
{
    uint32_t head = 0;
    for (int64_t v = 0; v < V; ++v) {
        uint32_t cnt = (counts[v] == 0) ? 2u : counts[v] + 2u;
        addr[v] = head;
        head += cnt;
    }
}

/* Bytes of the static part of the paper's layout: the histogram and the
 * address-offset array, one 32-bit word per voxel each (Table 1, note 1). */
int64_t og_paper_static_bytes(int64_t V)
{
    return V * 2 * (int64_t)sizeof(uint32_t);
}

/* ------------------------------------------------------------------------ */
/* VDMA: point indices into per-voxel segments (Alg. 2)                     */
/* ------------------------------------------------------------------------ */
void og_csr(const int32_t *keys, int32_t n, const uint32_t *off, int64_t V, int32_t *ids)
{
    uint32_t *fill = (uint32_t *)calloc((size_t)V, sizeof(uint32_t));
    for (int32_t j = 0; j < n; ++j) {
        int32_t v = keys[j];
        if (v < 0)
            continue;
        ids[off[v] + fill[v]] = j;
        fill[v] += 1;
    }
    free(fill);
}

/* ------------------------------------------------------------------------ */
/* DDMA: dilation of root labels into empty voxels (Alg. 3, Sec. 3 text)    */
/* ------------------------------------------------------------------------ */
void og_dilate(const og_grid *g, const uint32_t *off, int32_t L, int32_t *root, uint8_t *ring)
{
    const int64_t nx = g->dims[0], ny = g->dims[1], nz = g->dims[2];
    const int64_t V = nx * ny * nz;
    for (int64_t v = 0; v < V; ++v) {
        int occupied = off[v + 1] > off[v];
        root[v] = occupied ? (int32_t)v : -1;
        ring[v] = occupied ? 0 : 255;
    }
    int32_t *prev = (int32_t *)malloc((size_t)V * sizeof(int32_t));
    for (int32_t r = 1; r <= L; ++r) {
        memcpy(prev, root, (size_t)V * sizeof(int32_t));
#pragma omp parallel for schedule(static)
        for (int64_t z = 0; z < nz; ++z)
            for (int64_t y = 0; y < ny; ++y)
                for (int64_t x = 0; x < nx; ++x) {
                    int64_t v = x + nx * (y + ny * z);
                    if (prev[v] != -1)
                        continue;
                    int32_t best = -1;
                    int64_t nb[6];
                    int k = 0;
                    if (x > 0) nb[k++] = v - 1;
                    if (x + 1 < nx) nb[k++] = v + 1;
                    if (y > 0) nb[k++] = v - nx;
                    if (y + 1 < ny) nb[k++] = v + nx;
                    if (z > 0) nb[k++] = v - nx * ny;
                    if (z + 1 < nz) nb[k++] = v + nx * ny;
                    for (int i = 0; i < k; ++i) {
                        int32_t c = prev[nb[i]];
                        if (c != -1 && (best == -1 || c < best))
                            best = c;
                    }
                    if (best != -1) {
                        root[v] = best;
                        ring[v] = (uint8_t)r;
                    }
                }
    }
    free(prev);
}

/* ------------------------------------------------------------------------ */
/* Rigid transform of one source point with the float-rounded pose          */
/* ------------------------------------------------------------------------ */
static void og_transform(const double pose[16], const float *p, float s[3])
{
    for (int a = 0; a < 3; ++a) {
        float r0 = (float)pose[4 * a + 0];
        float r1 = (float)pose[4 * a + 1];
        float r2 = (float)pose[4 * a + 2];
        float t = (float)pose[4 * a + 3];
        float acc = r0 * p[0];
        acc = acc + r1 * p[1];
        acc = acc + r2 * p[2];
        s[a] = acc + t;
    }
}

/* Candidate order of the nearest-neighbour search: smaller squared distance
 * first, NaN after every number, equal distances to the smaller index. */
static int og_better(float d, int32_t j, float bd, int32_t bj)
{
    if (bj < 0)
        return 1;
    if (isnan(d) != isnan(bd))
        return isnan(bd);
    if (!isnan(d) && d != bd)
        return d < bd;
    return j < bj;
}

static float og_dist2(const float s[3], const float *q)
{
    float dx = s[0] - q[0];
    float dy = s[1] - q[1];
    float dz = s[2] - q[2];
    float acc = dx * dx;
    acc = acc + dy * dy;
    return acc + dz * dz;
}

/* ------------------------------------------------------------------------ */
/* NNS: localised nearest-neighbour search with global fallback (Alg. 4)    */
/* ------------------------------------------------------------------------ */
void og_correspond(const og_grid *g, const uint32_t *off, const int32_t *ids, const int32_t *root,
                   const float *tgt, int32_t n, const float *src, int32_t m, const double pose[16],
                   int32_t *nn, float *d2, uint8_t *fallback)
{
#pragma omp parallel for schedule(dynamic, 64)
    for (int32_t i = 0; i < m; ++i) {
        float s[3];
        og_transform(pose, src + 4 * (int64_t)i, s);
        int32_t v = og_voxel_key(g, s[0], s[1], s[2]);
        int32_t r = (v >= 0) ? root[v] : -1;
        int32_t best = -1;
        float bd = 0.0f;
        if (r >= 0) {
            /* Local search over the root voxel's point indices. */
            for (uint32_t k = off[r]; k < off[r + 1]; ++k) {
                int32_t j = ids[k];
                float d = og_dist2(s, tgt + 4 * (int64_t)j);
                if (og_better(d, j, bd, best)) {
                    best = j;
                    bd = d;
                }
            }
            fallback[i] = 0;
        } else {
            /* Global search over the whole target set. */
            for (int32_t j = 0; j < n; ++j) {
                float d = og_dist2(s, tgt + 4 * (int64_t)j);
                if (og_better(d, j, bd, best)) {
                    best = j;
                    bd = d;
                }
            }
            fallback[i] = 1;
        }
        nn[i] = best;
        d2[i] = bd;
    }
}

/* ------------------------------------------------------------------------ */
/* Reduction for Eq. 1: centroids, cross-covariance, RMSE (double, 2 pass)  */
/* ------------------------------------------------------------------------ */
void og_reduce(const float *tgt, const float *src, int32_t m, const double pose[16],
               const int32_t *nn, double pbar[3], double qbar[3], double H[9], double *rmse)
{
    double sp[3] = {0, 0, 0}, sq[3] = {0, 0, 0}, se = 0.0;
    for (int32_t i = 0; i < m; ++i) {
        float s[3];
        og_transform(pose, src + 4 * (int64_t)i, s);
        const float *q = tgt + 4 * (int64_t)nn[i];
        for (int a = 0; a < 3; ++a) {
            sp[a] += (double)s[a];
            sq[a] += (double)q[a];
            double e = (double)s[a] - (double)q[a];
            se += e * e;
        }
    }
    for (int a = 0; a < 3; ++a) {
        pbar[a] = sp[a] / (double)m;
        qbar[a] = sq[a] / (double)m;
    }
    for (int k = 0; k < 9; ++k)
        H[k] = 0.0;
    for (int32_t i = 0; i < m; ++i) {
        float s[3];
        og_transform(pose, src + 4 * (int64_t)i, s);
        const float *q = tgt + 4 * (int64_t)nn[i];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                H[3 * a + b] += ((double)s[a] - pbar[a]) * ((double)q[b] - qbar[b]);
    }
    *rmse = sqrt(se / (double)m);
}

/* ------------------------------------------------------------------------ */
/* Solve Eq. 1 for (dR, dt): SVD of H by one-sided Jacobi (Kabsch)          */
/* ------------------------------------------------------------------------ */
static double og_det3(const double M[9])
{
    return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
           M[2] * (M[3] * M[7] - M[4] * M[6]);
}

/* H = U diag(sig) V^T, row-major 3x3, singular values in descending order. */
void og_svd3(const double H[9], double U[9], double sig[3], double V[9])
{
    double A[9];
    memcpy(A, H, sizeof(A));
    for (int k = 0; k < 9; ++k)
        V[k] = (k % 4 == 0) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                double alpha = 0, beta = 0, gamma = 0;
                for (int i = 0; i < 3; ++i) {
                    alpha += A[3 * i + p] * A[3 * i + p];
                    beta += A[3 * i + q] * A[3 * i + q];
                    gamma += A[3 * i + p] * A[3 * i + q];
                }
                if (gamma == 0.0 || fabs(gamma) <= 1e-300)
                    continue;
                double rel = fabs(gamma) / sqrt(alpha * beta);
                if (rel > off)
                    off = rel;
                if (rel < 1e-15)
                    continue;
                double zeta = (beta - alpha) / (2.0 * gamma);
                double t = (zeta >= 0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
                double c = 1.0 / sqrt(1.0 + t * t);
                double s = c * t;
                for (int i = 0; i < 3; ++i) {
                    double ap = A[3 * i + p], aq = A[3 * i + q];
                    A[3 * i + p] = c * ap - s * aq;
                    A[3 * i + q] = s * ap + c * aq;
                    double vp = V[3 * i + p], vq = V[3 * i + q];
                    V[3 * i + p] = c * vp - s * vq;
                    V[3 * i + q] = s * vp + c * vq;
                }
            }
        if (off < 1e-15)
            break;
    }
    /* Column norms are the singular values; sort descending. */
    int order[3] = {0, 1, 2};
    double nrm[3];
    for (int k = 0; k < 3; ++k)
        nrm[k] = sqrt(A[k] * A[k] + A[3 + k] * A[3 + k] + A[6 + k] * A[6 + k]);
    for (int i = 0; i < 3; ++i)
        for (int j = i + 1; j < 3; ++j)
            if (nrm[order[j]] > nrm[order[i]]) {
                int t = order[i];
                order[i] = order[j];
                order[j] = t;
            }
    double Vs[9];
    for (int k = 0; k < 3; ++k) {
        int c = order[k];
        sig[k] = nrm[c];
        for (int i = 0; i < 3; ++i) {
            Vs[3 * i + k] = V[3 * i + c];
            U[3 * i + k] = (nrm[c] > 0.0) ? A[3 * i + c] / nrm[c] : 0.0;
        }
    }
    memcpy(V, Vs, sizeof(Vs));
    /* A zero third singular value leaves U's third column free: complete the
     * basis with the cross product of the first two. */
    if (!(sig[2] > 1e-300 * (sig[0] + 1e-300))) {
        U[2] = U[3] * U[7] - U[6] * U[4];
        U[5] = U[6] * U[1] - U[0] * U[7];
        U[8] = U[0] * U[4] - U[3] * U[1];
    }
}

/* rank(H) < 2 test: every 2x2 minor of H negligible against ||H||^2. */
int og_is_degenerate(const double H[9])
{
    double h2 = 0.0;
    for (int k = 0; k < 9; ++k)
        h2 += H[k] * H[k];
    if (h2 == 0.0)
        return 1;
    double c2 = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            int i1 = (i + 1) % 3, i2 = (i + 2) % 3, j1 = (j + 1) % 3, j2 = (j + 2) % 3;
            double c = H[3 * i1 + j1] * H[3 * i2 + j2] - H[3 * i1 + j2] * H[3 * i2 + j1];
            c2 += c * c;
        }
    return sqrt(c2) <= 1e-12 * h2;
}

/* Best rigid (dR, dt) taking the source centroid frame onto the target's:
 * dR = V diag(1, 1, sign det(V U^T)) U^T, dt = qbar - dR pbar.  dT is 4x4. */
int og_solve(const double pbar[3], const double qbar[3], const double H[9], double dT[16])
{
    if (og_is_degenerate(H))
        return OG_ERR_DEGENERATE;
    double U[9], sig[3], V[9];
    og_svd3(H, U, sig, V);
    double VUt[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k)
                acc += V[3 * i + k] * U[3 * j + k];
            VUt[3 * i + j] = acc;
        }
    double d = og_det3(VUt) < 0.0 ? -1.0 : 1.0;
    double diag[3] = {1.0, 1.0, d};
    double R[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k)
                acc += V[3 * i + k] * diag[k] * U[3 * j + k];
            R[3 * i + j] = acc;
        }
    for (int k = 0; k < 16; ++k)
        dT[k] = 0.0;
    for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
            dT[4 * i + j] = R[3 * i + j];
        dT[4 * i + 3] = qbar[i] - (R[3 * i] * pbar[0] + R[3 * i + 1] * pbar[1] + R[3 * i + 2] * pbar[2]);
    }
    dT[15] = 1.0;
    return OG_OK;
}

/* T <- dT * T (4x4 row-major). */
void og_compose(const double dT[16], double T[16])
{
    double out[16];
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 4; ++k)
                acc += dT[4 * i + k] * T[4 * k + j];
            out[4 * i + j] = acc;
        }
    memcpy(T, out, sizeof(out));
}

/* ------------------------------------------------------------------------ */
/* Grid build: keys, counts, offsets, CSR ids, dilation labels              */
/* ------------------------------------------------------------------------ */
void og_build(const og_grid *g, const float *tgt, int32_t n, int32_t L, int32_t *keys,
              uint32_t *counts, uint32_t *off, int32_t *ids, int32_t *root, uint8_t *ring)
{
    int64_t V = og_num_voxels(g);
    og_keys(g, tgt, n, keys);
    og_histogram(keys, n, V, counts);
    og_offsets(counts, V, off);
    og_csr(keys, n, off, V, ids);
    og_dilate(g, off, L, root, ring);
}

/* One ICP iteration on a built grid: correspond, reduce, solve, compose.
 * Returns the status of the solve; rmse_out gets this iteration's RMSE. */
int og_iterate(const og_grid *g, const uint32_t *off, const int32_t *ids, const int32_t *root,
               const float *tgt, int32_t n, const float *src, int32_t m, double pose[16],
               int32_t *nn, float *d2, uint8_t *fallback, double *rmse_out, int32_t *n_fallback)
{
    og_correspond(g, off, ids, root, tgt, n, src, m, pose, nn, d2, fallback);
    int32_t nf = 0;
    for (int32_t i = 0; i < m; ++i)
        nf += fallback[i];
    if (n_fallback)
        *n_fallback = nf;
    double pbar[3], qbar[3], H[9], dT[16];
    og_reduce(tgt, src, m, pose, nn, pbar, qbar, H, rmse_out);
    int st = og_solve(pbar, qbar, H, dT);
    if (st != OG_OK)
        return st;
    og_compose(dT, pose);
    return OG_OK;
}

/* Full registration (Sec. 2.1 loop, Sec. 4.1 stopping rule).  Workspace is
 * allocated here; rmse_hist (may be NULL) receives one RMSE per iteration. */
int og_register(const og_grid *g, int32_t L, const float *tgt, int32_t n, const float *src,
                int32_t m, double pose[16], int32_t max_iters, double eps, int32_t *iters_out,
                double *rmse_hist)
{
    int64_t V = og_num_voxels(g);
    int32_t *keys = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    uint32_t *counts = (uint32_t *)malloc((size_t)V * sizeof(uint32_t));
    uint32_t *off = (uint32_t *)malloc((size_t)(V + 1) * sizeof(uint32_t));
    int32_t *ids = (int32_t *)malloc((size_t)n * sizeof(int32_t));
    int32_t *root = (int32_t *)malloc((size_t)V * sizeof(int32_t));
    uint8_t *ring = (uint8_t *)malloc((size_t)V);
    int32_t *nn = (int32_t *)malloc((size_t)m * sizeof(int32_t));
    float *d2 = (float *)malloc((size_t)m * sizeof(float));
    uint8_t *fb = (uint8_t *)malloc((size_t)m);
    og_build(g, tgt, n, L, keys, counts, off, ids, root, ring);
    int st = OG_OK;
    int32_t it = 0;
    double prev = 0.0;
    for (int32_t k = 0; k < max_iters; ++k) {
        double rmse;
        st = og_iterate(g, off, ids, root, tgt, n, src, m, pose, nn, d2, fb, &rmse, NULL);
        if (rmse_hist)
            rmse_hist[k] = rmse;
        if (st != OG_OK)
            break;
        it = k + 1;
        if (eps > 0.0 && k >= 1 && fabs(rmse - prev) < eps)
            break;
        prev = rmse;
    }
    *iters_out = it;
    free(keys);
    free(counts);
    free(off);
    free(ids);
    free(root);
    free(ring);
    free(nn);
    free(d2);
    free(fb);
    return st;
}
