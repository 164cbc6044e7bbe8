// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "xray.h"
#include "xray_core.cuh"

// Zero border (units) around the interleaved images of the 2D quad-plane layouts.
#define XR_IL_PAD 2

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

namespace xr {

// Scan description passed by value to the ray-setup kernel.
struct GeoParams {
    int kind, nx, ny, nz, n_views, n_rows, n_cols;
    double dx, dy, dz, cx, cy, cz, du, dv, u0, v0, sod, sdd;
    double inv_dx, inv_dy, inv_dz;  // 1/dx, 1/dy, 1/dz
};

// Image extents and layout strides passed to the ray kernels.
struct Grid {
    int nx, ny, nz;
    int three;           // 1: a 3D scan (crossing-order walk), 0: 2D (slab walk)
    int64_t sx, sy, sz;  // element strides of i, j, k
};

inline bool kind_is3d(int k) { return k >= XR_PAR3D && k != XR_RAYS2D; }
inline bool kind_is_list(int k) { return k == XR_RAYS2D || k == XR_RAYS3D; }

// A float pair hi + lo with |lo| <= ulp(hi) / 2: about 48 significant bits, computed on the
// FP32 pipes (GB300's FP64 rate is a small fraction of its FP32 rate).
struct DF {
    float hi, lo;
};

inline DF df_from_double(double x)
{
    DF r;
    r.hi = (float)x;
    r.lo = (float)(x - (double)r.hi);
    return r;
}

// Per detector sample: the parts of the ray parameters that depend on the detector only
// (2D: s and cos/sin of gamma; 3D: s1, the detector part of s2, cos/sin of alpha and beta).
struct DetRec {
    DF s1, s2, ca, sa, cb, sb;
};

// Per view: cos/sin of the view angle (PAR3D: of phi1 and phi2) and the source height.
// Ray lists (one ray per view): cos/sin of phi (phi1, phi2) and, in H and pad0, s (s1, s2).
struct ViewRec {
    double c1, s1, c2, s2, H, pad0, pad1, pad2;
};

// The same per view, as float pairs, for the ray setup (ray lists: s or s1 in H, s2 in pad).
struct ViewDF {
    DF c1, s1, c2, s2, H, pad;
};

// Scan constants of the ray setup, as float pairs: the image centre, the planes i = 0,
// j = 0, k = 0 (x0 = cx - nx dx / 2, y1 = cy + ny dy / 2, z1 = cz + nz dz / 2) and 1/d.
struct SetupDF {
    DF cx, cy, cz, x0, y1, z1, idx, idy, idz;
};

SetupDF make_setup_df(const GeoParams &g);

// Where kernels get ray records: the handle's table (tab), or -- for scans without a table --
// rebuilt in the kernel from the per-view and per-detector tables (operator[] is defined in
// xray_rays.cuh, which kernels that use it include).
struct RaySrc {
    const RayRec *tab;
    const ViewDF *views;
    const DetRec *det;
    int64_t ndet;  // detector samples per view
    GeoParams g;
    SetupDF K;
    __device__ __forceinline__ RayRec operator[](int64_t r) const;
};

cudaError_t launch_det_setup(const GeoParams &g, DetRec *d_det, cudaStream_t s);

// One problem of a plan's ray setup (device copy): its detector table, and its ray table when
// it keeps one (rays == NULL: the detector table only), at offsets det_begin / ray_begin of the
// concatenated index ranges.
struct SetupItem {
    GeoParams g;
    SetupDF K;
    const ViewDF *views;
    DetRec *det;
    RayRec *rays;
    int64_t det_begin, ray_begin;
};
// Every item's detector samples (n_det in total) in one launch, then every item's rays (n_rays
// in total, items with a ray table only) in one launch.
cudaError_t launch_batch_setup(const SetupItem *items, int n, int64_t n_det, int64_t n_rays, cudaStream_t s);
cudaError_t launch_ray_setup(const GeoParams &g, const SetupDF &c, const ViewDF *d_views, const DetRec *d_det,
                             RayRec *d_rays, int64_t n_rays, cudaStream_t s);
// Parallel beams and ray lists (whose detector part needs no transcendentals), up to 65535
// views: the detector table and the ray table in one launch, the same records as the two.
bool ray_setup_inline_ok(const GeoParams &g);
cudaError_t launch_ray_setup_inline(const GeoParams &g, const SetupDF &c, const ViewDF *d_views, DetRec *d_det,
                                    RayRec *d_rays, cudaStream_t s);

cudaError_t launch_project(const RaySrc &rays, int64_t n_rays, const Grid &grid, const float *img,
                           int64_t img_bs, float *sino, int64_t sino_bs, int batch, int chunk,
                           int block, cudaStream_t s);

// Both operators in one pass per ray: sino = A img, then out += A^T sino (out zeroed by the
// caller), `chunk` images per thread.
cudaError_t launch_project_backproject(const RaySrc &rays, int64_t n_rays, const Grid &grid, const float *img,
                                       int64_t img_bs, float *sino, int64_t sino_bs, float *out, int64_t out_bs,
                                       int batch, int chunk, int block, cudaStream_t s);

cudaError_t launch_backproject_scatter(const RaySrc &rays, int64_t n_rays, const Grid &grid,
                                       const float *sino, int64_t sino_bs, float *img,
                                       int64_t img_bs, int batch, int chunk, int block,
                                       cudaStream_t s);

cudaError_t launch_backproject_gather2d(const RayRec *rays, const GeoParams &g, const Grid &grid,
                                        const float *d_view_tab, const float *sino,
                                        int64_t sino_bs, float *img, int64_t img_bs, int batch,
                                        int chunk, int block, cudaStream_t s);

cudaError_t launch_ray_units(const RaySrc &rays, int64_t n_rays, const Grid &grid, const int64_t *ray_ids,
                             int n, int cap, int64_t *idx, float *len, int32_t *count, cudaStream_t s);

// CSR rows of rays [ray0, ray0 + n): count (ptr[0..n], scanned in place) and fill.
cudaError_t launch_csr_count(const RaySrc &rays, int64_t ray0, int n, const Grid &grid, int64_t *ptr, cudaStream_t s);
cudaError_t launch_csr_fill(const RaySrc &rays, int64_t ray0, int n, const Grid &grid, const int64_t *ptr,
                            int64_t *col, float *val, cudaStream_t s);

// One problem of a persistent batched launch (device copy).
struct BatchItem {
    const RaySrc *src;  // device copy of the problem's ray source
    const float *img;
    float *sino;
    float *aux;  // n_units floats: the [nz][nx][ny] copy / accumulator, or NULL (read img only)
    int nx, ny, nz;
    int three;  // 1: a 3D scan
    int64_t n_rays;
    int64_t tile_begin;  // first global tile index of this problem
};

// The problem owning global tile t (items sorted by tile_begin).
__device__ __forceinline__ int find_item(const BatchItem *items, int n, int64_t t)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (items[mid].tile_begin <= t) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Persistent launch over the work list (fast3d.cu): the crossing-order walk for every
// problem.  Forward: the [nz][nx][ny] copies are written first when the items carry aux
// buffers; adjoint: images (and aux) are zeroed, scattered into, and aux added back.
// The tile counter is zeroed here.
// lock2d: every problem is 2D -- the adjoint's walk is batch2d_adj_kernel straight into the
// images (grid_ctas sized for it; the no-allocation entry points, which hold no planes).
// The forward keeps the crossing-order walk: for one image per problem the lockstep slab walk
// measured slower (64 uneven fans: 40.6 vs 22.2 ms), its adjoint faster (39.7 vs 71.9 ms).
cudaError_t launch_batched(const BatchItem *items, int n_items, int64_t n_tiles, int tile,
                           unsigned long long *counter, int adjoint, int with_aux, int grid_ctas, int block,
                           cudaStream_t s, bool lock2d = false);

// Forward persistent launch over a work list already in device memory, items without aux;
// the tile counter must be zero (no memset here).  The last argument is unused (the forward is
// the crossing-order walk for every work list).
cudaError_t launch_batched_items(const BatchItem *items, int n_items, int64_t n_tiles, int tile,
                                 unsigned long long *counter, int grid_ctas, int block, cudaStream_t s,
                                 bool lock2d = false);

int batched_ctas_per_sm(int block, int adjoint);

// The adjoint of a work list whose problems are all 2D (batch2d.cu): the slab walk in warp
// lockstep, 32 neighbouring rays of one problem per warp, reduced straight into the images
// (and aux copies, where given).  No copies or zero fills here.
int batch2d_ctas_per_sm(int block);
cudaError_t launch_batch2d_adjoint(const BatchItem *items, int n_items, int64_t n_tiles, int tile,
                                   unsigned long long *counter, int grid_ctas, int block, cudaStream_t s);

// The lockstep slab-walk adjoint of 2D problems (slab2d.cu): floats of one problem's
// accumulator planes (one per driving axis, every column padded with rows -2 .. N_B + 1).
__host__ __device__ inline int64_t slab2d_acc_floats(int nx, int ny)
{
    return (int64_t)nx * (ny + 4) + (int64_t)ny * (nx + 4);
}
// One problem, its planes at P.aux (slab2d_acc_floats, 16-byte aligned): zeroes them, walks
// 32 neighbouring rays per warp, then writes their sum into P.img.
cudaError_t launch_slab2d_adjoint_one(const BatchItem &P, cudaStream_t s);
// The same for a work list of 2D problems (persistent launch over an atomic tile counter,
// zeroed here), each item's planes at its aux.
int slab2d_ctas_per_sm(int block, bool adjoint);
cudaError_t launch_slab2d_adjoint(const BatchItem *items, int n_items, int64_t n_tiles, int tile,
                                  unsigned long long *counter, int grid_ctas, int block, int sms, cudaStream_t s);
// The forward of 2D problems with one image each: pair planes of every column (floats:
// slab2d_pair_floats) built from P.img at P.aux, then one ray per thread slab by slab.
__host__ __device__ inline int64_t slab2d_pair_floats(int nx, int ny)
{
    return 2 * ((int64_t)nx * (ny + 6) + (int64_t)ny * (nx + 6));
}
cudaError_t launch_slab2d_project_one(const BatchItem &P, cudaStream_t s);
cudaError_t launch_slab2d_project(const BatchItem *items, int n_items, int64_t n_tiles, int tile,
                                  unsigned long long *counter, int grid_ctas, int block, int sms, cudaStream_t s);

// Batched fast path for rays with at most two active axes (fast2d.cu).
cudaError_t launch_scatter_fast2(const RayRec *rays, int64_t n_rays, int nx, int ny, int nz, float *acc0,
                                 float *acc1, size_t acc_bytes, int Bp, const float *sino, float *img, int batch,
                                 int block, cudaStream_t s);
cudaError_t launch_gather_prep(const RayRec *rays, int64_t n_rays, void *grec, cudaStream_t s);

// Quad-plane layout kernels (fast2d.cu): one thread per ray / pixel for 4*nq images.
cudaError_t launch_interleave_planes(const float *img, int batch, int nx, int ny, int nz, float *il0, float *il1,
                                     cudaStream_t s);
// The forward writes image b, ray r at sino[b * sb + r * sr] (sb < 0: the user layout).
// only_cross: a slab that stays in one row reads it once (see fwd_plane_kernel).
cudaError_t launch_project_plane(const RayRec *rays, int64_t n_rays, int nx, int ny, int nz, const float *il0,
                                 const float *il1, float *sino, int batch, int nq, cudaStream_t s, int64_t sb = -1,
                                 int64_t sr = 1, bool only_cross = false);
// The gather adjoint of a batch of sinograms (image b, ray r at sino[b * sb + r * sr]; sb < 0:
// the user layout [batch][n_rays]): builds the gather records (gather_records_bytes(batch, nq,
// n_rays) bytes at recs, 16-byte aligned) and reads them through shared-memory stages.  Image b
// goes to the user layout, or (slice_of != NULL) to y-slice slice_of[b] of a volume (pixel
// (i, j) of the image at slice * slice_stride + j * row_stride + i).  err: the handle's device
// error word.
size_t gather_records_bytes(int batch, int nq, int64_t n_rays);
// One warp waits on an mbarrier that nothing completes with the staged gather's bounded wait
// (bound `limit` SM cycles); *d_out = 1 when the wait gave up.
cudaError_t launch_wait_selftest(long long limit, int *d_out, cudaStream_t s);
cudaError_t launch_gather_staged(const RayRec *rays, const void *grec, const GeoParams &g, const float *vt,
                                 const float *sino, int64_t n_rays, float *img, int batch, int nq, void *recs,
                                 cudaStream_t s, int *err, int64_t sb = -1, int64_t sr = 1,
                                 const int *slice_of = nullptr, int64_t slice_stride = 0, int64_t row_stride = 0);

// Single-tilt-axis parallel scans as batches of 2D problems, one per detector column
// (slices.cu).  slice_of[c]: the y-slice of column c's ray plane, or -1 outside the volume;
// c_rep: a column inside the volume (its rays give the 2D ray records); g2 and vt: the 2D
// parallel problem in (x, z) with the rows as its detector, and its gather view table.
struct SlicePlan {
    bool ok = false;
    bool surjective = false;  // every slice has a column
    int c_rep = -1;
    std::vector<int> slice_of;
    std::vector<float> vt;
    GeoParams g2{};
};
bool slice_plan(const xr_geometry_desc *d, SlicePlan *sp);
cudaError_t launch_slice_rays(const RaySrc &rays3, int64_t n2, int n_cols, int c_rep, RayRec *rays2, cudaStream_t s);
cudaError_t launch_slice_planes(const float *vol, int nx, int ny, int nz, const int *slice_of, int n_img, float *il0,
                                float *il1, cudaStream_t s);
// Tiled forward / adjoint for 2D scans and batches (tile2d.cu); in: user-layout input,
// out: user-layout output (cleared inside).
cudaError_t launch_tile2d(const RayRec *rays, const GeoParams &g, const float *vt, const float *in, float *out,
                          int batch, int adjoint, cudaStream_t s);
size_t gather_rec_bytes();
// Fast path for 3D scans (fast3d.cu): one thread per ray with the crossing-order walk,
// reading the caller's image or its [z][x][y] copy by the ray's direction.
cudaError_t launch_transpose_xy(const float *in, float *out, int nx, int ny, int nz, cudaStream_t s);
// order: 0 the ray order, 1 threads over (row, view, col), 2 threads over (view, col, row)
// on a z-fastest copy.  ws: one volume of workspace (the [z][x][y] copy, or for order 2 the
// [y][x][z] copy), written here.  err: the handle's device error word (XR_DEVERR_* bits are
// or-ed in), or NULL.
cudaError_t launch_project3d(const RaySrc &rays, const GeoParams &g, int64_t n_rays, int order, const float *img,
                             float *ws, float *sino, int block, int *err, cudaStream_t s);
// Forward, then the adjoint of its result, per (ray, image) with the single-image walks on the
// caller's layout: sino = A img, out += A^T sino (out zeroed by the caller).  n_rays < 2^31,
// batch <= 65535.
cudaError_t launch_fwd_adj(const RaySrc &rays, const GeoParams &g, int64_t n_rays, const float *img, float *sino,
                           float *out, int batch, int block, int *err, cudaStream_t s);
// Orders 0 and 1: zeroes `out` and `accT`, scatters, then adds accT (transposed) into out.
// Order 2: zeroes the z-fastest accumulator accT, scatters, then writes it transposed to out.
cudaError_t launch_scatter3d(const RaySrc &rays, const GeoParams &g, int64_t n_rays, int order,
                             const float *sino, float *out, float *accT, int block, int *err, cudaStream_t s);
// Unit-driven adjoint for 3D scans (tile3d.cu): one CTA per 16^3 tile of voxels gathers
// every ray of its detector footprint in shared memory and writes the tile once.
cudaError_t launch_tile3d_adj(const RaySrc &rays, const ViewRec *views, const GeoParams &g, const float *sino,
                              int64_t n_rays, float *img, int batch, cudaStream_t s);
cudaError_t launch_deinterleave_sum(const float *acc0, const float *acc1, int batch, int nx, int ny, int nz, int Bp,
                                    float *img, cudaStream_t s);

// Attenuated transform of 2D batches on the interleaved layouts (atten2d.cu).
cudaError_t launch_mu_layouts(const float *mu, int nx, int ny, float *mu0, float *mu1, cudaStream_t s);
cudaError_t launch_atten_plane_fwd(const RayRec *rays, int64_t n_rays, int nx, int ny, const float *il0,
                                   const float *il1, const float *mu0, const float *mu1, float *sino, int batch,
                                   int nq, cudaStream_t s);
cudaError_t launch_atten_plane_adj(const RayRec *rays, int64_t n_rays, int nx, int ny, float *acc0, float *acc1,
                                   size_t acc_bytes, const float *mu0, const float *mu1, const float *sino,
                                   float *img, int batch, int Bp, cudaStream_t s);

// Cone and helical scans walked by detector column (trace3d.cu): the vertical plane of a
// (view, column) shares its xy crossings among the column's rows.  Built at geometry creation
// for the cone and helix kinds when every row crosses at most one z plane per xy slab.
struct TraceGeo {
    int nx, ny, nz, n_views, n_rows, n_cols;
    int n_rb;          // blocks of 32 detector rows (a warp: one view, one column, one block)
    int ncg;           // groups of neighbouring columns, one CTA each (set at launch)
    int split;         // parts of the columns taken in turn within a row block (set at launch)
    DF x0, y1, z1, idx, idy, idz, cx, cy, D;  // planes i = 0, j = 0, k = 0; 1/d; centre; sod
    float rxy2;            // squared xy half-diagonal of the image (with a small margin)
    const ViewDF *views;   // cos / sin of the view angle, source height H
    const float4 *cols;    // per detector column: cos / sin of its fan angle alpha (float pairs)
    const float2 *tz;      // per detector sample [row][col]: rise per unit horizontal distance
};
size_t trace_ws_bytes(const GeoParams &g);  // the z-fastest copy with a zero voxel above and below
cudaError_t launch_trace_project(const TraceGeo &T, const float *img, float *ws, float *sino, cudaStream_t s);
cudaError_t launch_trace_backproject(const TraceGeo &T, const float *sino, float *img, float *ws, cudaStream_t s);

// Attenuated transform (atten.cu): one thread per ray, `chunk` images per thread; in/out
// in the caller's layout ([batch][units] / [batch][rays]); the adjoint adds into out.
cudaError_t launch_attenuated(bool adjoint, const RaySrc &rays, int64_t n_rays, const Grid &grid, const float *mu,
                              const float *in, float *out, int64_t n_units, int batch, int chunk, int block,
                              cudaStream_t s);

}  // namespace xr

// Record a CUDA error for xr_last_cuda_error() and return XR_ERR_CUDA.
xr_status xr_fail_cuda(cudaError_t e);

// The handle behind the opaque xr_geometry.
struct xr_geometry {
    xr_geometry_desc desc;  // copy; the array pointers are not kept
    xr::GeoParams params;
    int device;
    int64_t n_rays, n_units;
    xr::ViewRec *d_views;    // per view (host-computed cos/sin of the view angles)
    xr::ViewDF *d_views_df;  // the same as float pairs
    xr::SetupDF setup_df;    // scan constants of the ray setup
    xr::DetRec *d_det;       // per detector sample (det_setup_kernel)
    xr::RayRec *d_rays;      // the ray table (NULL for cone and helical scans)
    xr::RaySrc src;          // where kernels get ray records (the table, or rebuilt in the kernel)
    xr::RaySrc *d_src;       // its device copy, for batch work lists
    float *d_view_tab;   // per view: 2D gather footprint data (8 floats)
    void *d_grec;        // per ray: plane constants of the 2D gather
    float *d_ws;         // workspace of the batched fast path (interleaved copies)
    int *d_err;          // device error word (XR_DEVERR_* bits)
    size_t ws_bytes;
    int ws_batch;        // largest batch the workspace holds (0: none reserved)
    xr_tuning tune;
    // single-tilt-axis parallel scans: the batch of 2D column problems (slices.cu)
    xr::SlicePlan slices;
    xr::RayRec *d_rays2;  // 2D ray records, n_views * n_rows
    void *d_grec2;        // their gather records
    float *d_vt2;         // the 2D gather's view table
    int *d_slice_of;      // column -> slice
    // cone and helical scans: the column-trace walk (trace3d.cu)
    bool trace_ok;
    xr::TraceGeo trace;
    float4 *d_tcols;      // per detector column (cos, sin) of the fan angle, float pairs
    float2 *d_tz;         // per detector sample, the row's rise per unit horizontal distance
};
