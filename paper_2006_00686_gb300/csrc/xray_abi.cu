// Host side of the C ABI declared in include/xray.h: validation, handle lifetime, launches.
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <new>

#include <algorithm>

#include "xray_internal.h"

using namespace xr;

static thread_local int32_t g_last_cuda = 0;

xr_status xr_fail_cuda(cudaError_t e)
{
    g_last_cuda = (int32_t)e;
    return XR_ERR_CUDA;
}

static xr_status cuda_fail(cudaError_t e) { return xr_fail_cuda(e); }

#define XR_CUDA(call)                               \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_fail(e_); \
    } while (0)

static bool kind_helical(int k) { return k == XR_HELIX || k == XR_HELIX_ARC; }
static bool kind_divergent(int k)
{
    return k == XR_FAN2D || k == XR_FAN2D_ARC || (k >= XR_CONE && k <= XR_HELIX_ARC);
}
static bool kind_flat(int k) { return k == XR_FAN2D || k == XR_CONE || k == XR_HELIX; }
static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

static xr_status validate(const xr_geometry_desc *d)
{
    if (!d) return XR_ERR_NULL;
    if (d->kind < XR_PAR2D || d->kind > XR_RAYS3D) return XR_ERR_KIND;
    const bool three = kind_is3d(d->kind), list = kind_is_list(d->kind);
    const int nz = three ? d->nz : 1, nr = (three && !list) ? d->n_rows : 1;
    if (list && (d->n_cols != 1 || (three && d->n_rows != 1))) return XR_ERR_SIZE;
    if (d->nx < 1 || d->ny < 1 || nz < 1 || d->nx > 16384 || d->ny > 16384 || nz > 16384) return XR_ERR_SIZE;
    if (d->n_views < 1 || d->n_cols < 1 || nr < 1) return XR_ERR_SIZE;
    if ((int64_t)d->n_views * nr * d->n_cols > ((int64_t)1 << 40)) return XR_ERR_SIZE;
    if ((int64_t)nr * d->n_cols >= ((int64_t)1 << 31)) return XR_ERR_SIZE;
    if (!d->angles) return XR_ERR_NULL;
    if (kind_helical(d->kind) && !d->src_z) return XR_ERR_NULL;
    if (!(d->dx > 0) || !(d->dy > 0) || (three && !(d->dz > 0))) return XR_ERR_GEOMETRY;
    if (!list && (!(d->du > 0) || (three && !(d->dv > 0)))) return XR_ERR_GEOMETRY;
    if (kind_divergent(d->kind)) {
        if (!(d->sod > 0)) return XR_ERR_GEOMETRY;
        if (kind_flat(d->kind) && !(d->sdd > 0)) return XR_ERR_GEOMETRY;
        // the source circle must stay outside the image (farthest corner in the xy-plane)
        const double ex = fabs(d->cx) + 0.5 * d->nx * d->dx, ey = fabs(d->cy) + 0.5 * d->ny * d->dy;
        if (!(d->sod > sqrt(ex * ex + ey * ey))) return XR_ERR_GEOMETRY;
    }
    // foot-point coordinates of rays that cross the image must fit the 16-bit record
    const double dz = three ? d->dz : 1.0;
    const double R = 0.5 * sqrt(pow(d->nx * d->dx, 2) + pow(d->ny * d->dy, 2) + pow(nz * dz, 2));
    if (0.5 * d->nx + R / d->dx > 32000 || 0.5 * d->ny + R / d->dy > 32000 || 0.5 * nz + R / dz > 32000)
        return XR_ERR_SIZE;
    return XR_OK;
}

static Grid make_grid(const xr_geometry *g)
{
    Grid gr;
    gr.nx = g->params.nx;
    gr.ny = g->params.ny;
    gr.nz = g->params.nz;
    gr.three = kind_is3d(g->params.kind);
    gr.sx = 1;
    gr.sy = gr.nx;
    gr.sz = (int64_t)gr.nx * gr.ny;
    return gr;
}

// Per-view data of the 2D gather's footprint test (computed in double, stored as float).
static void fill_view_table(const xr_geometry_desc *d, float *vt)
{
    for (int v = 0; v < d->n_views; ++v) {
        double e[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        if (kind_is_list(d->kind)) {  // no detector: the gathers do not take ray lists
            for (int k = 0; k < 8; ++k) vt[8 * v + k] = 0.f;
            continue;
        }
        const double a = d->angles[v];
        if (d->kind == XR_PAR2D) {
            e[0] = -sin(a);  // s = -x sin(phi) + y cos(phi)
            e[1] = cos(a);
        } else {
            e[0] = -d->sod * sin(a);  // source
            e[1] = d->sod * cos(a);
            e[2] = sin(a);  // towards the origin
            e[3] = -cos(a);
            e[4] = cos(a);  // along the detector
            e[5] = sin(a);
        }
        for (int k = 0; k < 8; ++k) vt[8 * v + k] = (float)e[k];
    }
}

// Images walked together by one thread: the handle's tuning, at most the batch.
static int pick_chunk(const xr_geometry *g, int batch)
{
    int c = g->tune.batch_chunk;
    while (c > 1 && c > batch) c >>= 1;
    return c < 1 ? 1 : c;
}

// Images per chunk of the batched fast path.
static int fast_chunk(int batch) { return batch > 8 ? 16 : (batch > 4 ? 8 : 4); }

// Units of one image in the fast path's padded interleaved layout (border of 2 in x and y).
static size_t padded_units(const xr_geometry *g)
{
    return (size_t)(g->params.nx + 4) * (size_t)(g->params.ny + 4) * (size_t)g->params.nz;
}

// Two chunks of quad planes (the forward's images, or the scatter's accumulators), then the
// gather records of the batch for any plane count the tuning may pick (at least one chunk of
// sinograms: the attenuated path keeps its attenuation planes there).
static size_t fast_ws_bytes(const xr_geometry *g, int batch)
{
    const int Bp = fast_chunk(batch);
    const size_t padded = (size_t)((batch + Bp - 1) / Bp) * Bp;
    size_t tail = padded * sizeof(float) * (size_t)g->n_rays;
    for (int nq = 1; nq <= 4; nq *= 2) tail = std::max(tail, gather_records_bytes((int)padded, nq, g->n_rays));
    return padded * sizeof(float) * 2 * padded_units(g) + tail;
}

// The batched fast path applies when the workspace holds the batch and the batch is >= 4.
// Planes (of 4 images) one thread walks: the handle's batch_chunk / 4, at most what the batch needs.
static int plane_nq(const xr_geometry *g, int batch)
{
    int nq = g->tune.batch_chunk >= 16 ? 4 : (g->tune.batch_chunk >= 8 ? 2 : 1);
    const int Q = (batch + 3) / 4;
    while (nq > 1 && nq > Q) nq >>= 1;
    return nq;
}

// Tiled path: 2D scans, batches of 4 or more (no workspace needed).
static bool use_tiled(const xr_geometry *g, int batch)
{
    return !kind_is3d(g->params.kind) && !kind_is_list(g->params.kind) && batch >= 4 && g->tune.batch_chunk != 1 && g->tune.path == XR_PATH_TILED;
}

static bool use_fast(const xr_geometry *g, int batch)
{
    // the fast kernels index one chunk of interleaved images with 32-bit offsets
    return !kind_is3d(g->params.kind) && batch >= 4 && batch <= g->ws_batch && g->tune.batch_chunk != 1 && g->tune.path != XR_PATH_RAY &&
           !use_tiled(g, batch) &&
           (int64_t)padded_units(g) * fast_chunk(batch) < ((int64_t)1 << 31) &&
           g->n_rays * fast_chunk(batch) < ((int64_t)1 << 31) && g->n_units < ((int64_t)1 << 31);
}

// Single-image fast path (3D scans, and 2D scans outside the quad-plane path) with a
// reserved workspace: the crossing-order walk over the image and its [z][x][y] copy, one
// image at a time (32-bit offsets and ray ids).
static bool use_dda(const xr_geometry *g)
{
    return g->tune.path != XR_PATH_RAY && g->d_ws &&
           g->ws_bytes >= (size_t)g->n_units * sizeof(float) && g->n_units < ((int64_t)1 << 31) &&
           g->n_rays < ((int64_t)1 << 31);
}

// Ray order of the 3D fast path (0 view, 1 row, 2 column, 3 row-blocked; see
// launch_project3d).  Automatic, measured on GB300: circular cones row-blocked in both
// directions (a warp's rays are neighbouring rows of one column, whose reductions fall on
// neighbouring words of the z-fastest copy, and the rays in flight cross one slab of z:
// cone 512^3 adjoint 341 ms vs 398 column-major and 437 row-major, forward 242 vs 246 ms);
// helices the ray order forward (the source moves through z view by view; 88 vs 93 ms) and
// column-major adjoint (148 vs 166 ms); the ray order otherwise.
static int ray_order(const xr_geometry *g, bool adjoint)
{
    if (g->tune.order == XR_ORDER_ROWBLOCK) return 3;
    if (g->tune.order == XR_ORDER_COLUMN) return 2;
    if (g->tune.order == XR_ORDER_ROW) return 1;
    if (g->tune.order == XR_ORDER_VIEW) return 0;
    const int k = g->params.kind;
    if (k == XR_CONE || k == XR_CONE_ARC) return 3;
    if (adjoint && (k == XR_HELIX || k == XR_HELIX_ARC)) return 2;
    return 0;
}

// Single-tilt-axis parallel scans: the column images as quad planes in both orders (the
// forward) and the gather records (the adjoint).  Planes are padded to a multiple of 4 (the
// forward walks up to 4 planes per thread).
static int64_t slice_n2(const xr_geometry *g) { return (int64_t)g->params.n_views * g->params.n_rows; }
static int64_t slice_np(const xr_geometry *g)
{
    return (int64_t)(g->params.nx + 2 * XR_IL_PAD) * (g->params.nz + 2 * XR_IL_PAD);
}
static int64_t slice_planes(const xr_geometry *g) { return (int64_t)((g->params.n_cols + 15) / 16) * 4; }
// Two sets of column-image planes (the forward), then the gather records of one volume's
// columns for any plane count the tuning may pick.
static size_t slice_ws_bytes(const xr_geometry *g)
{
    size_t tail = 0;
    for (int nq = 1; nq <= 4; nq *= 2) tail = std::max(tail, gather_records_bytes(g->params.n_cols, nq, slice_n2(g)));
    return (size_t)slice_planes(g) * sizeof(float4) * (size_t)(2 * slice_np(g)) + tail;
}

// The batch-of-columns path of single-tilt-axis parallel scans (32-bit offsets in a plane,
// 32-bit ray ids of the 2D problem).
static bool use_slices(const xr_geometry *g)
{
    return g->slices.ok && g->tune.path != XR_PATH_RAY && g->d_ws && g->ws_bytes >= slice_ws_bytes(g) &&
           slice_np(g) * 4 < ((int64_t)1 << 31) && slice_n2(g) < ((int64_t)1 << 31) &&
           (g->params.n_cols + 3) / 4 <= 65535;  // planes index gridDim.y
}

// Single images of 2D scans in the ray order (neighbouring rays of a view in a warp) that
// fill the GPU, 1024 rays per SM or more (slab2d.cu): the adjoint walks 32 rays per warp in
// lockstep into padded accumulator planes in the workspace, the forward one ray per thread on
// pair planes there.  Smaller scans, where the longest warp and the extra launch decide the
// time, keep the crossing-order walk one ray per thread (parallel 64^2: 23 vs 25 us).
static bool use_slab2d(const xr_geometry *g, bool adjoint)
{
    if (kind_is3d(g->params.kind) || g->tune.path == XR_PATH_RAY || !g->d_ws) return false;
    const int64_t floats = adjoint ? slab2d_acc_floats(g->params.nx, g->params.ny)
                                   : slab2d_pair_floats(g->params.nx, g->params.ny);
    if (g->ws_bytes < (size_t)floats * sizeof(float) || floats >= ((int64_t)1 << 31) ||
        g->n_rays >= ((int64_t)1 << 31) || ray_order(g, true) > 1)
        return false;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, g->device) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return g->n_rays >= 1024 * (int64_t)sms;
}

static BatchItem slab_item(const xr_geometry *g, const float *img, float *sino)
{
    BatchItem P{};
    P.src = g->d_src;
    P.img = img;
    P.sino = sino;
    P.aux = g->d_ws;
    P.nx = g->params.nx;
    P.ny = g->params.ny;
    P.nz = 1;
    P.n_rays = g->n_rays;
    return P;
}

// The column-trace walk of cone and helical scans (workspace: the padded z-fastest copy).
static bool use_trace(const xr_geometry *g)
{
    return g->trace_ok && g->tune.path != XR_PATH_RAY && g->d_ws && g->ws_bytes >= trace_ws_bytes(g->params) &&
           (g->tune.order == XR_ORDER_AUTO || g->tune.order == XR_ORDER_TRACE);
}

static size_t reserve_bytes(const xr_geometry *g, int batch)
{
    if (kind_is3d(g->params.kind) || batch < 4) {
        size_t one = (size_t)g->n_units * sizeof(float);
        if (!kind_is3d(g->params.kind))  // the single-image planes (adjoint and forward)
            one = std::max(one, (size_t)std::max(slab2d_acc_floats(g->params.nx, g->params.ny),
                                                 slab2d_pair_floats(g->params.nx, g->params.ny)) *
                                    sizeof(float));
        if (g->trace_ok) one = std::max(one, trace_ws_bytes(g->params));
        return g->slices.ok ? std::max(one, slice_ws_bytes(g)) : one;
    }
    return fast_ws_bytes(g, batch);  // >= n_units floats: serves the single-image path too
}

// Cone and helical scans: the column-trace walk's tables (per column: cos / sin of the fan
// angle; per detector sample: the row's rise per unit horizontal distance) and whether the
// walk applies: every row crosses at most one z plane per xy slab (a slab is at most the
// (dx, dy) cell's diagonal long) and offsets of the padded z-fastest copy fit 32 bits.  Flat detectors: tan(alpha) = u / sdd and
// t_z = v / sqrt(sdd^2 + u^2) (eq. equispaced_cone_beam with t = u sod/sdd, h = v sod/sdd);
// equiangular detectors: alpha = u, t_z = tan(v) (eq. equiangular_cone_beam).
static bool kind_cone(int k) { return k >= XR_CONE && k <= XR_HELIX_ARC; }


static bool trace_tables(const GeoParams &p, std::vector<float4> &cols, std::vector<float2> &tz, TraceGeo &T)
{
    if (!kind_cone(p.kind)) return false;
    const bool flat = (p.kind == XR_CONE || p.kind == XR_HELIX);
    cols.resize((size_t)p.n_cols);
    tz.resize((size_t)p.n_rows * p.n_cols);
    double tzmax = 0.0;
    for (int c = 0; c < p.n_cols; ++c) {
        const double u = (c - 0.5 * (p.n_cols - 1)) * p.du + p.u0;
        const double h = sqrt(p.sdd * p.sdd + u * u);
        const DF ca = df_from_double(flat ? p.sdd / h : cos(u)), sa = df_from_double(flat ? u / h : sin(u));
        cols[(size_t)c] = make_float4(ca.hi, ca.lo, sa.hi, sa.lo);
        for (int r = 0; r < p.n_rows; ++r) {
            const double v = (r - 0.5 * (p.n_rows - 1)) * p.dv + p.v0;
            const double t = flat ? v / h : tan(v);
            const DF d = df_from_double(t);
            tz[(size_t)r * p.n_cols + c] = make_float2(d.hi, d.lo);
            tzmax = std::max(tzmax, fabs(t));
        }
    }
    const double slab_z = tzmax * sqrt(p.dx * p.dx + p.dy * p.dy) / p.dz;
    if (!(slab_z < 0.99)) return false;
    if ((int64_t)p.nx * p.ny * (p.nz + 2) >= ((int64_t)1 << 31)) return false;
    T.nx = p.nx;
    T.ny = p.ny;
    T.nz = p.nz;
    T.n_views = p.n_views;
    T.n_rows = p.n_rows;
    T.n_cols = p.n_cols;
    T.n_rb = (p.n_rows + 31) / 32;
    T.ncg = (p.n_cols + 3) / 4;
    if ((int64_t)T.ncg * p.n_views * T.n_rb >= ((int64_t)1 << 31)) return false;
    T.x0 = df_from_double(p.cx - 0.5 * p.nx * p.dx);
    T.y1 = df_from_double(p.cy + 0.5 * p.ny * p.dy);
    T.z1 = df_from_double(p.cz + 0.5 * p.nz * p.dz);
    T.idx = df_from_double(p.inv_dx);
    T.idy = df_from_double(p.inv_dy);
    T.idz = df_from_double(p.inv_dz);
    T.cx = df_from_double(p.cx);
    T.cy = df_from_double(p.cy);
    T.D = df_from_double(p.sod);
    const double rxy = 0.5 * sqrt(pow(p.nx * p.dx, 2) + pow(p.ny * p.dy, 2)) * (1.0 + 1e-5) + 1e-3 * (p.dx + p.dy);
    T.rxy2 = (float)(rxy * rxy);
    return true;
}

// Rebuild the 2D column problem's ray records from the 3D ray table.
static cudaError_t slice_setup(xr_geometry *g, cudaStream_t s)
{
    if (!g->slices.ok) return cudaSuccess;
    cudaError_t e = launch_slice_rays(g->src, slice_n2(g), g->params.n_cols, g->slices.c_rep, g->d_rays2, s);
    if (e == cudaSuccess) e = launch_gather_prep(g->d_rays2, slice_n2(g), g->d_grec2, s);
    return e;
}

extern "C" {

xr_status xr_geometry_create(const xr_geometry_desc *desc, xr_geometry **out)
{
    if (!out) return XR_ERR_NULL;
    *out = nullptr;
    xr_status st = validate(desc);
    if (st != XR_OK) return st;
    xr_geometry *g = new (std::nothrow) xr_geometry();
    if (!g) return XR_ERR_ALLOC;
    g->desc = *desc;
    const bool three = kind_is3d(desc->kind);
    if (kind_is_list(desc->kind)) {
        g->desc.n_rows = 1;
        g->desc.n_cols = 1;
        g->desc.du = g->desc.dv = 1.0;
        g->desc.u0 = g->desc.v0 = 0.0;
    }
    if (!three) {
        g->desc.nz = 1;
        g->desc.n_rows = 1;
        g->desc.dz = g->desc.dz > 0 ? g->desc.dz : 1.0;
        g->desc.dv = g->desc.dv > 0 ? g->desc.dv : 1.0;
    }
    g->desc.angles = nullptr;
    g->desc.src_z = nullptr;
    GeoParams &p = g->params;
    p.kind = desc->kind;
    p.nx = desc->nx;
    p.ny = desc->ny;
    p.nz = g->desc.nz;
    p.n_views = desc->n_views;
    p.n_rows = g->desc.n_rows;
    p.n_cols = g->desc.n_cols;
    p.dx = desc->dx;
    p.dy = desc->dy;
    p.dz = g->desc.dz;
    p.cx = desc->cx;
    p.cy = desc->cy;
    p.cz = desc->cz;
    p.du = g->desc.du;
    p.dv = g->desc.dv;
    p.u0 = g->desc.u0;
    p.v0 = three ? g->desc.v0 : 0.0;
    p.sod = desc->sod;
    p.sdd = desc->sdd;
    p.inv_dx = 1.0 / p.dx;
    p.inv_dy = 1.0 / p.dy;
    p.inv_dz = 1.0 / p.dz;
    g->n_rays = (int64_t)p.n_views * p.n_rows * p.n_cols;
    g->n_units = (int64_t)p.nx * p.ny * p.nz;
    g->tune.block = 128;
    g->tune.batch_chunk = 16;
    // automatic: the gather on the batched quad-plane path (fan beam 512^2 x 16 on GB300:
    // gather 1.97 ms, vector-atomic scatter 2.94 ms) and for single-tilt-axis parallel scans
    // run as 2D column problems, the scatter elsewhere (one image: the per-pixel gather loops
    // over every view and is many times slower; 3D: the tiled gather loses to the scatter).
    // The tuner may fix either per scan.
    g->tune.adjoint = XR_ADJ_AUTO;
    g->tune.path = XR_PATH_INTERLEAVED;
    g->tune.order = XR_ORDER_AUTO;

    cudaError_t e = cudaGetDevice(&g->device);
    const size_t n_det = (size_t)p.n_rows * p.n_cols;
    if (e == cudaSuccess) e = cudaMalloc(&g->d_views, (size_t)p.n_views * sizeof(ViewRec));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_views_df, (size_t)p.n_views * sizeof(ViewDF));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_det, n_det * sizeof(DetRec));
    // 3D parallel, cone and helical scans keep no ray table: their kernels rebuild each record
    // from the per-view and per-detector tables (RaySrc); 2D scans and ray lists keep one (the
    // 2D batched kernels and the ray lists' per-ray parameters read it)
    const bool table = !kind_cone(p.kind) && p.kind != XR_PAR3D;
    if (e == cudaSuccess && table) e = cudaMalloc(&g->d_rays, (size_t)g->n_rays * sizeof(RayRec));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_src, sizeof(RaySrc));
    if (e == cudaSuccess) e = cudaMalloc(&g->d_err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(g->d_err, 0, sizeof(int));
    if (e == cudaSuccess && !three) e = cudaMalloc(&g->d_view_tab, (size_t)p.n_views * 8 * sizeof(float));
    if (e == cudaSuccess && !three) e = cudaMalloc(&g->d_grec, (size_t)g->n_rays * gather_rec_bytes());
    if (e == cudaSuccess && three && slice_plan(desc, &g->slices)) {
        const size_t n2 = (size_t)slice_n2(g);
        e = cudaMalloc(&g->d_rays2, n2 * sizeof(RayRec));
        if (e == cudaSuccess) e = cudaMalloc(&g->d_grec2, n2 * gather_rec_bytes());
        if (e == cudaSuccess) e = cudaMalloc(&g->d_vt2, g->slices.vt.size() * sizeof(float));
        if (e == cudaSuccess) e = cudaMalloc(&g->d_slice_of, g->slices.slice_of.size() * sizeof(int));
        if (e == cudaSuccess)
            e = cudaMemcpy(g->d_vt2, g->slices.vt.data(), g->slices.vt.size() * sizeof(float), cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(g->d_slice_of, g->slices.slice_of.data(), g->slices.slice_of.size() * sizeof(int),
                           cudaMemcpyHostToDevice);
    }
    if (e == cudaSuccess && three) {
        std::vector<float4> cols;
        std::vector<float2> tz;
        g->trace_ok = trace_tables(p, cols, tz, g->trace);
        if (g->trace_ok) {
            e = cudaMalloc(&g->d_tcols, cols.size() * sizeof(float4));
            if (e == cudaSuccess) e = cudaMalloc(&g->d_tz, tz.size() * sizeof(float2));
            if (e == cudaSuccess)
                e = cudaMemcpy(g->d_tcols, cols.data(), cols.size() * sizeof(float4), cudaMemcpyHostToDevice);
            if (e == cudaSuccess) e = cudaMemcpy(g->d_tz, tz.data(), tz.size() * sizeof(float2), cudaMemcpyHostToDevice);
            g->trace.views = g->d_views_df;
            g->trace.cols = g->d_tcols;
            g->trace.tz = g->d_tz;
        }
    }
    if (e != cudaSuccess) {
        const bool oom = (e == cudaErrorMemoryAllocation);
        cudaGetLastError();
        xr_geometry_destroy(g);
        if (oom) return XR_ERR_ALLOC;
        return cuda_fail(e);
    }
    {
        // per view: cos/sin of the view angle(s) and the source height, in double
        ViewRec *vr = (ViewRec *)calloc((size_t)p.n_views, sizeof(ViewRec));
        if (!vr) {
            xr_geometry_destroy(g);
            return XR_ERR_ALLOC;
        }
        for (int v = 0; v < p.n_views; ++v) {
            if (desc->kind == XR_RAYS2D) {  // (s, phi)
                vr[v].c1 = cos(desc->angles[2 * v + 1]);
                vr[v].s1 = sin(desc->angles[2 * v + 1]);
                vr[v].H = desc->angles[2 * v];
                continue;
            }
            if (desc->kind == XR_RAYS3D) {  // (s1, s2, phi1, phi2)
                const double *q = desc->angles + 4 * (size_t)v;
                vr[v].c1 = cos(q[2]);
                vr[v].s1 = sin(q[2]);
                vr[v].c2 = cos(q[3]);
                vr[v].s2 = sin(q[3]);
                vr[v].H = q[0];
                vr[v].pad0 = q[1];
                continue;
            }
            const double a = desc->kind == XR_PAR3D ? desc->angles[2 * v] : desc->angles[v];
            vr[v].c1 = cos(a);
            vr[v].s1 = sin(a);
            if (desc->kind == XR_PAR3D) {
                vr[v].c2 = cos(desc->angles[2 * v + 1]);
                vr[v].s2 = sin(desc->angles[2 * v + 1]);
            }
            vr[v].H = kind_helical(desc->kind) ? desc->src_z[v] : 0.0;
        }
        e = cudaMemcpy(g->d_views, vr, (size_t)p.n_views * sizeof(ViewRec), cudaMemcpyHostToDevice);
        ViewDF *vd = (ViewDF *)calloc((size_t)p.n_views, sizeof(ViewDF));
        if (!vd) {
            free(vr);
            xr_geometry_destroy(g);
            return XR_ERR_ALLOC;
        }
        for (int v = 0; v < p.n_views; ++v) {
            vd[v].c1 = df_from_double(vr[v].c1);
            vd[v].s1 = df_from_double(vr[v].s1);
            vd[v].c2 = df_from_double(vr[v].c2);
            vd[v].s2 = df_from_double(vr[v].s2);
            vd[v].H = df_from_double(vr[v].H);
            vd[v].pad = df_from_double(vr[v].pad0);
        }
        if (e == cudaSuccess)
            e = cudaMemcpy(g->d_views_df, vd, (size_t)p.n_views * sizeof(ViewDF), cudaMemcpyHostToDevice);
        free(vd);
        free(vr);
    }
    if (e == cudaSuccess && !three) {
        float *vt = (float *)malloc((size_t)p.n_views * 8 * sizeof(float));
        if (!vt) {
            xr_geometry_destroy(g);
            return XR_ERR_ALLOC;
        }
        fill_view_table(desc, vt);
        e = cudaMemcpy(g->d_view_tab, vt, (size_t)p.n_views * 8 * sizeof(float), cudaMemcpyHostToDevice);
        free(vt);
    }
    if (e == cudaSuccess) e = launch_det_setup(p, g->d_det, nullptr);
    g->setup_df = make_setup_df(p);
    g->src.tab = g->d_rays;
    g->src.views = g->d_views_df;
    g->src.det = g->d_det;
    g->src.ndet = (int64_t)p.n_rows * p.n_cols;
    g->src.g = p;
    g->src.K = g->setup_df;
    if (e == cudaSuccess) e = cudaMemcpy(g->d_src, &g->src, sizeof(RaySrc), cudaMemcpyHostToDevice);
    if (e == cudaSuccess && g->d_rays)
        e = launch_ray_setup(p, g->setup_df, g->d_views_df, g->d_det, g->d_rays, g->n_rays, nullptr);
    // the quad-plane gather's per-ray constants are built when a workspace for batches of four
    // or more is reserved (the only path that reads them), and rebuilt by later ray setups
    if (e == cudaSuccess) e = slice_setup(g, nullptr);
    if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    if (e != cudaSuccess) {
        xr_geometry_destroy(g);
        return cuda_fail(e);
    }
    *out = g;
    return XR_OK;
}

void xr_geometry_destroy(xr_geometry *g)
{
    if (!g) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(g->device);
    cudaDeviceSynchronize();
    cudaFree(g->d_views);
    cudaFree(g->d_views_df);
    cudaFree(g->d_det);
    cudaFree(g->d_rays);
    cudaFree(g->d_src);
    cudaFree(g->d_view_tab);
    cudaFree(g->d_grec);
    cudaFree(g->d_ws);
    cudaFree(g->d_err);
    cudaFree(g->d_rays2);
    cudaFree(g->d_grec2);
    cudaFree(g->d_vt2);
    cudaFree(g->d_slice_of);
    cudaFree(g->d_tcols);
    cudaFree(g->d_tz);
    cudaSetDevice(prev);
    delete g;
}

xr_status xr_ray_setup(xr_geometry *g, xr_stream stream)
{
    if (!g) return XR_ERR_NULL;
    if (g->d_rays && ray_setup_inline_ok(g->params)) {
        XR_CUDA(launch_ray_setup_inline(g->params, g->setup_df, g->d_views_df, g->d_det, g->d_rays,
                                        (cudaStream_t)stream));
    } else {
        XR_CUDA(launch_det_setup(g->params, g->d_det, (cudaStream_t)stream));
        if (g->d_rays)
            XR_CUDA(launch_ray_setup(g->params, g->setup_df, g->d_views_df, g->d_det, g->d_rays, g->n_rays,
                                     (cudaStream_t)stream));
    }
    if (g->d_grec && g->ws_batch >= 4)
        XR_CUDA(launch_gather_prep(g->d_rays, g->n_rays, g->d_grec, (cudaStream_t)stream));
    XR_CUDA(slice_setup(g, (cudaStream_t)stream));
    return XR_OK;
}

xr_status xr_reserve(xr_geometry *g, int32_t max_batch)
{
    if (!g) return XR_ERR_NULL;
    if (max_batch < 1) return XR_ERR_BATCH;
    if (max_batch <= g->ws_batch) return XR_OK;
    const size_t bytes = reserve_bytes(g, max_batch);
    int prev = 0;
    XR_CUDA(cudaGetDevice(&prev));
    XR_CUDA(cudaSetDevice(g->device));
    XR_CUDA(cudaDeviceSynchronize());  // the old workspace may still be in use
    cudaFree(g->d_ws);
    g->d_ws = nullptr;
    g->ws_bytes = 0;
    g->ws_batch = 0;
    size_t got = bytes;
    cudaError_t e = cudaMalloc(&g->d_ws, got);
    const size_t one = (size_t)g->n_units * sizeof(float);
    if (e == cudaErrorMemoryAllocation && kind_is3d(g->params.kind) && bytes > one) {
        // the column batch's planes do not fit: keep the single-image copy (the 3D walk)
        cudaGetLastError();
        got = one;
        e = cudaMalloc(&g->d_ws, got);
    }
    // the borders of the interleaved copies stay zero: only interiors are ever written
    if (e == cudaSuccess) e = cudaMemset(g->d_ws, 0, got);
    if (e == cudaSuccess && g->d_grec && max_batch >= 4) {  // the quad-plane gather's constants
        e = launch_gather_prep(g->d_rays, g->n_rays, g->d_grec, nullptr);
        if (e == cudaSuccess) e = cudaStreamSynchronize(nullptr);
    }
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        cudaGetLastError();
        g->d_ws = nullptr;
        return e == cudaErrorMemoryAllocation ? XR_ERR_ALLOC : cuda_fail(e);
    }
    g->ws_bytes = got;
    g->ws_batch = max_batch;
    return XR_OK;
}

xr_status xr_geometry_get_info(const xr_geometry *g, xr_geometry_info *info)
{
    if (!g || !info) return XR_ERR_NULL;
    info->n_rays = g->n_rays;
    info->n_units = g->n_units;
    info->table_bytes = (g->d_rays ? g->n_rays * (int64_t)sizeof(RayRec) : 0) + (int64_t)g->params.n_views * (8 * 4 + sizeof(ViewRec) + sizeof(ViewDF)) +
                        (int64_t)g->params.n_rows * g->params.n_cols * (int64_t)sizeof(DetRec) +
                        (g->d_grec ? g->n_rays * (int64_t)gather_rec_bytes() : 0) + (int64_t)g->ws_bytes +
                        (g->slices.ok ? slice_n2(g) * (int64_t)(sizeof(RayRec) + gather_rec_bytes()) : 0) +
                        (g->trace_ok ? (int64_t)g->params.n_cols * (int64_t)(sizeof(float4) + g->params.n_rows * sizeof(float2)) : 0);
    info->is3d = kind_is3d(g->params.kind);
    info->device = g->device;
    info->column_batch = g->slices.ok ? 1 : 0;
    info->trace_walk = g->trace_ok ? 1 : 0;
    return XR_OK;
}

xr_status xr_column_batch_plan(const xr_geometry_desc *desc, int32_t *slice_of, int32_t *eligible)
{
    if (!desc || !eligible) return XR_ERR_NULL;
    const xr_status st = validate(desc);
    if (st != XR_OK) return st;
    SlicePlan sp;
    const bool ok = kind_is3d(desc->kind) && slice_plan(desc, &sp);
    *eligible = ok ? 1 : 0;
    if (slice_of)
        for (int c = 0; c < desc->n_cols; ++c) slice_of[c] = ok ? sp.slice_of[(size_t)c] : -1;
    return XR_OK;
}

xr_status xr_set_tuning(xr_geometry *g, const xr_tuning *t)
{
    if (!g || !t) return XR_ERR_NULL;
    if (t->block && (t->block < 64 || t->block > 256 || (t->block & 31))) return XR_ERR_ARG;
    if (t->batch_chunk && t->batch_chunk != 1 && t->batch_chunk != 2 && t->batch_chunk != 4 &&
        t->batch_chunk != 8 && t->batch_chunk != 16)
        return XR_ERR_ARG;
    if (t->adjoint && t->adjoint != XR_ADJ_SCATTER && t->adjoint != XR_ADJ_GATHER) return XR_ERR_ARG;
    if (t->path < 0 || t->path > XR_PATH_RAY) return XR_ERR_ARG;
    if (t->order < 0 || t->order > XR_ORDER_TRACE) return XR_ERR_ARG;
    if (t->order) g->tune.order = t->order;
    if (t->path) g->tune.path = t->path;
    if (t->block) g->tune.block = t->block;
    if (t->batch_chunk) g->tune.batch_chunk = t->batch_chunk;
    if (t->adjoint) g->tune.adjoint = t->adjoint;
    return XR_OK;
}

xr_status xr_get_tuning(const xr_geometry *g, xr_tuning *t)
{
    if (!g || !t) return XR_ERR_NULL;
    *t = g->tune;
    return XR_OK;
}

xr_status xr_project(const xr_geometry *g, const float *d_img, float *d_sino, int32_t batch, xr_stream stream)
{
    if (!g || !d_img || !d_sino) return XR_ERR_NULL;
    if (batch < 1) return XR_ERR_BATCH;
    if (!aligned16(d_img) || !aligned16(d_sino)) return XR_ERR_ALIGN;
    if (use_tiled(g, batch)) {
        if ((batch + 3) / 4 > 65535) return XR_ERR_SIZE;
        XR_CUDA(launch_tile2d(g->d_rays, g->params, g->d_view_tab, d_img, d_sino, batch, 0, (cudaStream_t)stream));
        return XR_OK;
    }
    if (use_slices(g)) {
        // one 2D problem per detector column: the volume's y-slices as quad planes
        const cudaStream_t s = (cudaStream_t)stream;
        const GeoParams &p = g->params;
        float *il0 = g->d_ws, *il1 = g->d_ws + 4 * slice_planes(g) * slice_np(g);
        for (int b = 0; b < batch; ++b) {
            XR_CUDA(launch_slice_planes(d_img + (size_t)b * g->n_units, p.nx, p.ny, p.nz, g->d_slice_of, p.n_cols,
                                        il0, il1, s));
            XR_CUDA(launch_project_plane(g->d_rays2, slice_n2(g), p.nx, p.nz, 1, il0, il1,
                                         d_sino + (size_t)b * g->n_rays, p.n_cols, plane_nq(g, p.n_cols), s, 1,
                                         p.n_cols, true));
        }
        return XR_OK;
    }
    if (use_trace(g)) {
        const cudaStream_t s = (cudaStream_t)stream;
        for (int b = 0; b < batch; ++b)
            XR_CUDA(launch_trace_project(g->trace, d_img + (size_t)b * g->n_units, g->d_ws,
                                         d_sino + (size_t)b * g->n_rays, s));
        return XR_OK;
    }
    if (!use_fast(g, batch) && use_slab2d(g, false)) {
        for (int b = 0; b < batch; ++b)
            XR_CUDA(launch_slab2d_project_one(slab_item(g, d_img + (size_t)b * g->n_units,
                                                        d_sino + (size_t)b * g->n_rays),
                                              (cudaStream_t)stream));
        return XR_OK;
    }
    if (!use_fast(g, batch) && use_dda(g)) {
        const cudaStream_t s = (cudaStream_t)stream;
        for (int b = 0; b < batch; ++b) {
            const float *img = d_img + (size_t)b * g->n_units;
            XR_CUDA(launch_project3d(g->src, g->params, g->n_rays, ray_order(g, false), img, g->d_ws,
                                     d_sino + (size_t)b * g->n_rays, g->tune.block, g->d_err, s));
        }
        return XR_OK;
    }
    if (use_fast(g, batch)) {
        // quad planes, one thread per ray for plane_nq(g) * 4 images
        const int Q = (batch + 3) / 4;
        if (Q > 65535) return XR_ERR_SIZE;
        const size_t padded = (size_t)((batch + fast_chunk(batch) - 1) / fast_chunk(batch)) * fast_chunk(batch);
        float *il0 = g->d_ws, *il1 = g->d_ws + padded * padded_units(g);
        const cudaStream_t s = (cudaStream_t)stream;
        XR_CUDA(launch_interleave_planes(d_img, batch, g->params.nx, g->params.ny, g->params.nz, il0, il1, s));
        XR_CUDA(launch_project_plane(g->d_rays, g->n_rays, g->params.nx, g->params.ny, g->params.nz, il0, il1, d_sino,
                                     batch, plane_nq(g, batch), s));
        return XR_OK;
    }
    const int chunk = pick_chunk(g, batch);
    if ((batch + chunk - 1) / chunk > 65535) return XR_ERR_SIZE;
    XR_CUDA(launch_project(g->src, g->n_rays, make_grid(g), d_img, g->n_units, d_sino, g->n_rays, batch,
                           chunk, g->tune.block, (cudaStream_t)stream));
    return XR_OK;
}

xr_status xr_backproject_method(const xr_geometry *g, const float *d_sino, float *d_img, int32_t batch,
                                int32_t method, xr_stream stream)
{
    if (!g || !d_img || !d_sino) return XR_ERR_NULL;
    if (batch < 1) return XR_ERR_BATCH;
    if (!aligned16(d_img) || !aligned16(d_sino)) return XR_ERR_ALIGN;
    if (method == XR_ADJ_AUTO) method = g->tune.adjoint;
    if (kind_is_list(g->params.kind)) {
        if (method == XR_ADJ_GATHER) return XR_ERR_ARG;
        method = XR_ADJ_SCATTER;
    }
    if (method == XR_ADJ_AUTO) {
        // measured on GB300: 3D scatter 438 ms vs tiled gather 682 ms (circular cone 512^3);
        // single-tilt-axis scans as 2D column problems: the staged gather (C3 1.19 ms vs the 3D
        // scatter 2.76 ms); 2D: the staged gather beats the vector-atomic scatter (1.44 vs
        // 2.94 ms, fan beam 512^2 x 16), one image: the scatter
        if (kind_is3d(g->params.kind))
            method = use_slices(g) ? XR_ADJ_GATHER : XR_ADJ_SCATTER;
        else
            method = (!use_tiled(g, batch) && use_fast(g, batch)) ? XR_ADJ_GATHER : XR_ADJ_SCATTER;
    }
    const int chunk = pick_chunk(g, batch);
    if ((batch + chunk - 1) / chunk > 65535) return XR_ERR_SIZE;
    const cudaStream_t s = (cudaStream_t)stream;
    if (method == XR_ADJ_GATHER) {
        if (use_slices(g)) {
            // one 2D gather per detector column, written into the column's y-slice
            const GeoParams &p = g->params;
            float *recs = g->d_ws + 8 * slice_planes(g) * slice_np(g);
            for (int b = 0; b < batch; ++b) {
                float *img = d_img + (size_t)b * g->n_units;
                if (!g->slices.surjective) XR_CUDA(cudaMemsetAsync(img, 0, (size_t)g->n_units * sizeof(float), s));
                // column c of 2D ray r2 at sino[r2 * n_cols + c]
                XR_CUDA(launch_gather_staged(g->d_rays2, g->d_grec2, g->slices.g2, g->d_vt2, d_sino + (size_t)b * g->n_rays,
                                             slice_n2(g), img, p.n_cols, plane_nq(g, p.n_cols), recs, s, g->d_err, 1,
                                             p.n_cols, g->d_slice_of, p.nx, (int64_t)p.ny * p.nx));
            }
            return XR_OK;
        }
        if (kind_is3d(g->params.kind)) {
            if (batch > 65535) return XR_ERR_SIZE;
            XR_CUDA(launch_tile3d_adj(g->src, g->d_views, g->params, d_sino, g->n_rays, d_img, batch, s));
            return XR_OK;
        }
        if (use_fast(g, batch)) {
            // the staged gather on records built after the forward's planes in the workspace
            const size_t padded = (size_t)((batch + fast_chunk(batch) - 1) / fast_chunk(batch)) * fast_chunk(batch);
            float *recs = g->d_ws + 2 * padded * padded_units(g);
            XR_CUDA(launch_gather_staged(g->d_rays, g->d_grec, g->params, g->d_view_tab, d_sino, g->n_rays, d_img,
                                         batch, plane_nq(g, batch), recs, s, g->d_err));
            return XR_OK;
        }
        XR_CUDA(launch_backproject_gather2d(g->d_rays, g->params, make_grid(g), g->d_view_tab, d_sino, g->n_rays,
                                            d_img, g->n_units, batch, chunk, g->tune.block, s));
        return XR_OK;
    }
    if (method != XR_ADJ_SCATTER) return XR_ERR_ARG;
    if (use_trace(g)) {
        for (int b = 0; b < batch; ++b)
            XR_CUDA(launch_trace_backproject(g->trace, d_sino + (size_t)b * g->n_rays, d_img + (size_t)b * g->n_units,
                                             g->d_ws, s));
        return XR_OK;
    }
    if (!use_tiled(g, batch) && !use_fast(g, batch) && use_slab2d(g, true)) {
        for (int b = 0; b < batch; ++b)
            XR_CUDA(launch_slab2d_adjoint_one(slab_item(g, d_img + (size_t)b * g->n_units,
                                                        const_cast<float *>(d_sino) + (size_t)b * g->n_rays),
                                              s));
        return XR_OK;
    }
    if (!use_tiled(g, batch) && !use_fast(g, batch) && use_dda(g)) {
        for (int b = 0; b < batch; ++b)
            XR_CUDA(launch_scatter3d(g->src, g->params, g->n_rays, ray_order(g, true), d_sino + (size_t)b * g->n_rays,
                                     d_img + (size_t)b * g->n_units, g->d_ws, g->tune.block, g->d_err, s));
        return XR_OK;
    }
    if (use_tiled(g, batch)) {
        if ((batch + 3) / 4 > 65535) return XR_ERR_SIZE;
        XR_CUDA(launch_tile2d(g->d_rays, g->params, g->d_view_tab, d_sino, d_img, batch, 1, s));
        return XR_OK;
    }
    if (use_fast(g, batch)) {
        // ray-driven scatter into two zeroed interleaved accumulators, then summed back
        const int Bp = fast_chunk(batch);
        const size_t padded = (size_t)((batch + Bp - 1) / Bp) * Bp;
        float *acc0 = g->d_ws, *acc1 = g->d_ws + padded * padded_units(g);
        XR_CUDA(launch_scatter_fast2(g->d_rays, g->n_rays, g->params.nx, g->params.ny, g->params.nz, acc0, acc1,
                                     padded * padded_units(g) * sizeof(float), Bp, d_sino, d_img, batch, 256, s));
        return XR_OK;
    }
    XR_CUDA(cudaMemsetAsync(d_img, 0, (size_t)g->n_units * batch * sizeof(float), s));
    XR_CUDA(launch_backproject_scatter(g->src, g->n_rays, make_grid(g), d_sino, g->n_rays, d_img, g->n_units,
                                       batch, chunk, g->tune.block, s));
    return XR_OK;
}

xr_status xr_backproject(const xr_geometry *g, const float *d_sino, float *d_img, int32_t batch,
                         xr_stream stream)
{
    return xr_backproject_method(g, d_sino, d_img, batch, XR_ADJ_AUTO, stream);
}

xr_status xr_project_backproject(const xr_geometry *g, const float *d_img, float *d_sino, float *d_out,
                                 int32_t batch, xr_stream stream)
{
    if (!g || !d_img || !d_sino || !d_out) return XR_ERR_NULL;
    if (batch < 1) return XR_ERR_BATCH;
    if (!aligned16(d_img) || !aligned16(d_sino) || !aligned16(d_out)) return XR_ERR_ALIGN;
    // out is written while other threads still read img and sino: the three must not overlap
    const uintptr_t i0 = (uintptr_t)d_img, i1 = i0 + (uintptr_t)g->n_units * batch * sizeof(float);
    const uintptr_t s0 = (uintptr_t)d_sino, s1 = s0 + (uintptr_t)g->n_rays * batch * sizeof(float);
    const uintptr_t o0 = (uintptr_t)d_out, o1 = o0 + (uintptr_t)g->n_units * batch * sizeof(float);
    if ((o0 < i1 && i0 < o1) || (o0 < s1 && s0 < o1) || (i0 < s1 && s0 < i1)) return XR_ERR_ARG;
    const cudaStream_t s = (cudaStream_t)stream;
    XR_CUDA(cudaMemsetAsync(d_out, 0, (size_t)g->n_units * batch * sizeof(float), s));
    if (g->n_rays < ((int64_t)1 << 31) && batch <= 65535) {
        // the single-image walks (units generated ahead of their loads and reductions)
        XR_CUDA(launch_fwd_adj(g->src, g->params, g->n_rays, d_img, d_sino, d_out, batch, 128, g->d_err, s));
        return XR_OK;
    }
    const int chunk = pick_chunk(g, batch);
    if ((batch + chunk - 1) / chunk > 65535) return XR_ERR_SIZE;
    XR_CUDA(launch_project_backproject(g->src, g->n_rays, make_grid(g), d_img, g->n_units, d_sino, g->n_rays, d_out,
                                       g->n_units, batch, chunk, g->tune.block, s));
    return XR_OK;
}

// Attenuated transform of a 2D batch on the interleaved layouts: the batched fast path's
// workspace, with room after the two image copies for the map's two padded copies.
static bool use_atten_planes(const xr_geometry *g, int batch)
{
    if (kind_is3d(g->params.kind) || !use_fast(g, batch)) return false;
    const size_t padded = (size_t)((batch + fast_chunk(batch) - 1) / fast_chunk(batch)) * fast_chunk(batch);
    return 2 * padded_units(g) <= padded * (size_t)g->n_rays && g->n_rays < ((int64_t)1 << 31);
}

xr_status xr_project_attenuated(const xr_geometry *g, const float *d_mu, const float *d_img, float *d_sino,
                                int32_t batch, xr_stream stream)
{
    if (!g || !d_mu || !d_img || !d_sino) return XR_ERR_NULL;
    if (batch < 1) return XR_ERR_BATCH;
    if (!aligned16(d_mu) || !aligned16(d_img) || !aligned16(d_sino)) return XR_ERR_ALIGN;
    const cudaStream_t s = (cudaStream_t)stream;
    if (use_atten_planes(g, batch)) {
        const size_t padded = (size_t)((batch + fast_chunk(batch) - 1) / fast_chunk(batch)) * fast_chunk(batch);
        float *il0 = g->d_ws, *il1 = g->d_ws + padded * padded_units(g);
        float *mu0 = g->d_ws + 2 * padded * padded_units(g), *mu1 = mu0 + padded_units(g);
        XR_CUDA(launch_interleave_planes(d_img, batch, g->params.nx, g->params.ny, 1, il0, il1, s));
        XR_CUDA(launch_mu_layouts(d_mu, g->params.nx, g->params.ny, mu0, mu1, s));
        XR_CUDA(launch_atten_plane_fwd(g->d_rays, g->n_rays, g->params.nx, g->params.ny, il0, il1, mu0, mu1, d_sino,
                                       batch, plane_nq(g, batch), s));
        return XR_OK;
    }
    const int chunk = pick_chunk(g, batch);
    if ((batch + chunk - 1) / chunk > 65535) return XR_ERR_SIZE;
    XR_CUDA(launch_attenuated(false, g->src, g->n_rays, make_grid(g), d_mu, d_img, d_sino, g->n_units, batch,
                              chunk, g->tune.block, s));
    return XR_OK;
}

xr_status xr_backproject_attenuated(const xr_geometry *g, const float *d_mu, const float *d_sino, float *d_img,
                                    int32_t batch, xr_stream stream)
{
    if (!g || !d_mu || !d_img || !d_sino) return XR_ERR_NULL;
    if (batch < 1) return XR_ERR_BATCH;
    if (!aligned16(d_mu) || !aligned16(d_img) || !aligned16(d_sino)) return XR_ERR_ALIGN;
    const int chunk = pick_chunk(g, batch);
    if ((batch + chunk - 1) / chunk > 65535) return XR_ERR_SIZE;
    const cudaStream_t s = (cudaStream_t)stream;
    if (use_atten_planes(g, batch)) {
        const int Bp = fast_chunk(batch);
        const size_t padded = (size_t)((batch + Bp - 1) / Bp) * Bp;
        float *acc0 = g->d_ws, *acc1 = g->d_ws + padded * padded_units(g);
        float *mu0 = g->d_ws + 2 * padded * padded_units(g), *mu1 = mu0 + padded_units(g);
        XR_CUDA(launch_mu_layouts(d_mu, g->params.nx, g->params.ny, mu0, mu1, s));
        XR_CUDA(launch_atten_plane_adj(g->d_rays, g->n_rays, g->params.nx, g->params.ny, acc0, acc1,
                                       padded * padded_units(g) * sizeof(float), mu0, mu1, d_sino, d_img, batch, Bp,
                                       s));
        return XR_OK;
    }
    XR_CUDA(cudaMemsetAsync(d_img, 0, (size_t)g->n_units * batch * sizeof(float), s));
    XR_CUDA(launch_attenuated(true, g->src, g->n_rays, make_grid(g), d_mu, d_sino, d_img, g->n_units, batch,
                              chunk, g->tune.block, s));
    return XR_OK;
}

xr_status xr_get_device_error(const xr_geometry *g, int32_t *code)
{
    if (!g || !code) return XR_ERR_NULL;
    int prev = 0, h = 0;
    XR_CUDA(cudaGetDevice(&prev));
    XR_CUDA(cudaSetDevice(g->device));
    cudaError_t e = cudaMemcpy(&h, g->d_err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemset(g->d_err, 0, sizeof(int));
    cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(e);
    *code = h;
    return XR_OK;
}

xr_status xr_ray_units(const xr_geometry *g, const int64_t *d_rays, int32_t n, int32_t cap, int64_t *d_idx,
                       float *d_len, int32_t *d_count, xr_stream stream)
{
    if (!g || !d_rays || !d_idx || !d_len || !d_count) return XR_ERR_NULL;
    if (n < 1 || cap < 1) return XR_ERR_SIZE;
    XR_CUDA(launch_ray_units(g->src, g->n_rays, make_grid(g), d_rays, n, cap, d_idx, d_len, d_count,
                             (cudaStream_t)stream));
    return XR_OK;
}

static xr_status csr_args(const xr_geometry *g, int64_t ray0, int32_t n, const void *ptr)
{
    if (!g || !ptr) return XR_ERR_NULL;
    if (n < 1 || ray0 < 0 || ray0 + n > g->n_rays) return XR_ERR_SIZE;
    if ((uintptr_t)ptr & 7u) return XR_ERR_ALIGN;
    return XR_OK;
}

xr_status xr_system_rows_count(const xr_geometry *g, int64_t ray0, int32_t n, int64_t *d_row_ptr, xr_stream stream)
{
    const xr_status st = csr_args(g, ray0, n, d_row_ptr);
    if (st != XR_OK) return st;
    XR_CUDA(launch_csr_count(g->src, ray0, n, make_grid(g), d_row_ptr, (cudaStream_t)stream));
    return XR_OK;
}

xr_status xr_system_rows_fill(const xr_geometry *g, int64_t ray0, int32_t n, const int64_t *d_row_ptr, int64_t *d_col,
                              float *d_val, xr_stream stream)
{
    const xr_status st = csr_args(g, ray0, n, d_row_ptr);
    if (st != XR_OK) return st;
    if (!d_col || !d_val) return XR_ERR_NULL;
    if (((uintptr_t)d_col & 7u) || ((uintptr_t)d_val & 3u)) return XR_ERR_ALIGN;
    XR_CUDA(launch_csr_fill(g->src, ray0, n, make_grid(g), d_row_ptr, d_col, d_val, (cudaStream_t)stream));
    return XR_OK;
}

}  // extern "C"

struct xr_batch {
    int device;
    int n;
    bool lock2d;  // every problem is 2D: the adjoint is the lockstep slab walk (slab2d.cu)
    int sms;
    SetupItem *d_setup;          // per problem: the ray setup's work (xr_batch_ray_setup)
    int64_t setup_det, setup_rays;  // detector samples and table rays over all problems
    int tile, block, ctas_fwd, ctas_adj;
    int64_t n_tiles;
    BatchItem *d_items;
    unsigned long long *d_counter;
    float *d_aux;  // every problem's [nz][nx][ny] copy / accumulator (2D: also the adjoint's planes), back to back
};

extern "C" {

xr_status xr_batch_create(const xr_problem *probs, int32_t n, int32_t tile, int32_t block, xr_batch **out)
{
    if (!out) return XR_ERR_NULL;
    *out = nullptr;
    if (!probs) return XR_ERR_NULL;
    if (n < 1) return XR_ERR_SIZE;
    if (tile == 0) tile = 256;
    if (block == 0) block = 256;
    if (tile < 32 || tile > 65536 || (tile & 31) || block < 64 || block > 256 || (block & 31)) return XR_ERR_ARG;
    int dev = 0;
    XR_CUDA(cudaGetDevice(&dev));
    BatchItem *items = (BatchItem *)malloc(sizeof(BatchItem) * (size_t)n);
    if (!items) return XR_ERR_ALLOC;
    bool all2d = true;
    for (int i = 0; i < n; ++i) all2d = all2d && probs[i].geom && !kind_is3d(probs[i].geom->params.kind);
    // floats of problem g's aux buffer, a multiple of 4 (every buffer 16-byte aligned)
    auto aux_floats = [all2d](const xr_geometry *g) -> int64_t {
        const int64_t f = all2d ? std::max(slab2d_acc_floats(g->params.nx, g->params.ny),
                                           slab2d_pair_floats(g->params.nx, g->params.ny))
                                : g->n_units;
        return (f + 3) & ~(int64_t)3;
    };
    int64_t tiles = 0, aux_units = 0;
    for (int i = 0; i < n; ++i) {
        const xr_geometry *g = probs[i].geom;
        if (!g || !probs[i].img || !probs[i].sino) {
            free(items);
            return XR_ERR_NULL;
        }
        if (g->device != dev) {  // the plan's launches run on the current device
            free(items);
            return XR_ERR_ARG;
        }
        if (!aligned16(probs[i].img) || !aligned16(probs[i].sino)) {
            free(items);
            return XR_ERR_ALIGN;
        }
        if (g->n_units >= ((int64_t)1 << 31) ||  // the walks index one problem with 32 bits
            (all2d && slab2d_pair_floats(g->params.nx, g->params.ny) >= ((int64_t)1 << 31))) {
            free(items);
            return XR_ERR_SIZE;
        }
        items[i].src = g->d_src;
        items[i].img = probs[i].img;
        items[i].sino = probs[i].sino;
        items[i].aux = nullptr;
        items[i].nx = g->params.nx;
        items[i].ny = g->params.ny;
        items[i].nz = g->params.nz;
        items[i].three = kind_is3d(g->params.kind);
        items[i].n_rays = g->n_rays;
        items[i].tile_begin = tiles;
        tiles += (g->n_rays + tile - 1) / tile;
        aux_units += aux_floats(g);
    }
    if (n > 65535) {
        free(items);
        return XR_ERR_SIZE;
    }
    xr_batch *b = new (std::nothrow) xr_batch();
    if (!b) {
        free(items);
        return XR_ERR_ALLOC;
    }
    b->n = n;
    b->lock2d = all2d;
    b->tile = tile;
    b->block = block;
    b->n_tiles = tiles;
    int sms = 0;
    cudaError_t e = cudaGetDevice(&b->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    b->sms = sms;
    if (e == cudaSuccess) e = cudaMalloc(&b->d_items, sizeof(BatchItem) * (size_t)n);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_counter, 256);
    if (e == cudaSuccess) e = cudaMalloc(&b->d_aux, (size_t)aux_units * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_setup, sizeof(SetupItem) * (size_t)n);
    if (e == cudaSuccess) {
        // the ray setup of every problem: detector tables, and ray tables where kept
        SetupItem *si = (SetupItem *)malloc(sizeof(SetupItem) * (size_t)n);
        if (!si) e = cudaErrorMemoryAllocation;
        int64_t nd = 0, nr = 0;
        for (int i = 0; e == cudaSuccess && i < n; ++i) {
            const xr_geometry *g = probs[i].geom;
            si[i].g = g->params;
            si[i].K = g->setup_df;
            si[i].views = g->d_views_df;
            si[i].det = g->d_det;
            si[i].rays = g->d_rays;
            si[i].det_begin = nd;
            si[i].ray_begin = nr;
            nd += (int64_t)g->params.n_rows * g->params.n_cols;
            if (g->d_rays) nr += g->n_rays;
        }
        b->setup_det = nd;
        b->setup_rays = nr;
        if (e == cudaSuccess)
            e = cudaMemcpy(b->d_setup, si, sizeof(SetupItem) * (size_t)n, cudaMemcpyHostToDevice);
        free(si);
    }
    if (e == cudaSuccess) {
        int64_t at = 0;
        for (int i = 0; i < n; ++i) {
            items[i].aux = b->d_aux + at;
            at += aux_floats(probs[i].geom);
        }
        e = cudaMemcpy(b->d_items, items, sizeof(BatchItem) * (size_t)n, cudaMemcpyHostToDevice);
    }
    free(items);
    if (e != cudaSuccess) {
        const bool oom = (e == cudaErrorMemoryAllocation);
        cudaGetLastError();
        xr_batch_destroy(b);
        return oom ? XR_ERR_ALLOC : cuda_fail(e);
    }
    b->ctas_fwd = sms * (b->lock2d ? slab2d_ctas_per_sm(block, false) : batched_ctas_per_sm(block, 0));
    b->ctas_adj = sms * (b->lock2d ? slab2d_ctas_per_sm(block, true) : batched_ctas_per_sm(block, 1));
    *out = b;
    return XR_OK;
}

void xr_batch_destroy(xr_batch *b)
{
    if (!b) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    cudaFree(b->d_items);
    cudaFree(b->d_counter);
    cudaFree(b->d_aux);
    cudaFree(b->d_setup);
    cudaSetDevice(prev);
    delete b;
}

xr_status xr_batch_ray_setup(const xr_batch *b, xr_stream stream)
{
    if (!b) return XR_ERR_NULL;
    XR_CUDA(launch_batch_setup(b->d_setup, b->n, b->setup_det, b->setup_rays, (cudaStream_t)stream));
    return XR_OK;
}

xr_status xr_batch_project(const xr_batch *b, xr_stream stream)
{
    if (!b) return XR_ERR_NULL;
    if (b->lock2d)
        XR_CUDA(launch_slab2d_project(b->d_items, b->n, b->n_tiles, b->tile, b->d_counter, b->ctas_fwd, b->block,
                                      b->sms, (cudaStream_t)stream));
    else
        XR_CUDA(launch_batched(b->d_items, b->n, b->n_tiles, b->tile, b->d_counter, 0, 1, b->ctas_fwd, b->block,
                               (cudaStream_t)stream));
    return XR_OK;
}

xr_status xr_batch_backproject(const xr_batch *b, xr_stream stream)
{
    if (!b) return XR_ERR_NULL;
    if (b->lock2d)
        XR_CUDA(launch_slab2d_adjoint(b->d_items, b->n, b->n_tiles, b->tile, b->d_counter, b->ctas_adj, b->block,
                                      b->sms, (cudaStream_t)stream));
    else
        XR_CUDA(launch_batched(b->d_items, b->n, b->n_tiles, b->tile, b->d_counter, 1, 1, b->ctas_adj, b->block,
                               (cudaStream_t)stream));
    return XR_OK;
}

const char *xr_status_string(xr_status s)
{
    switch (s) {
    case XR_OK: return "ok";
    case XR_ERR_NULL: return "a required pointer is NULL";
    case XR_ERR_SIZE: return "a size is non-positive or too large";
    case XR_ERR_KIND: return "unknown scan kind";
    case XR_ERR_GEOMETRY: return "inconsistent scan geometry";
    case XR_ERR_ALIGN: return "device pointer not 16-byte aligned";
    case XR_ERR_CUDA: return "CUDA call failed";
    case XR_ERR_ALLOC: return "device allocation failed";
    case XR_ERR_BATCH: return "batch must be >= 1";
    case XR_ERR_ARG: return "argument out of range";
    case XR_ERR_TUNE: return "tuning cache could not be read or written";
    case XR_ERR_CAPACITY: return "more problems than the fixed no-allocation scratch holds";
    }
    return "unknown status";
}

int32_t xr_last_cuda_error(void) { return g_last_cuda; }

int32_t xr_version(void) { return 1; }

}  // extern "C"
