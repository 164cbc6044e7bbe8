/*
 * xray.h -- C ABI of the GB300 (sm_103a) X-ray transform library (libxray.so).
 *
 * The library computes the X-ray transform of a pixel/voxel image (eq. Xray_transform_image
 * of Chen, Wang, Bajaj, Oktem, "A Fast and Adaptive Algorithm to Compute the X-ray
 * Transform") and its adjoint, ray by ray: for every ray only the units that satisfy the
 * non-vanishing-intersectability condition (eq. conditions_2D_1 / conditions_3D_1) are
 * visited, and each contributes its analytic length C_up - C_low (eq. range_length /
 * range_length_3D).  Nothing is stored per (ray, unit): lengths are recomputed on the fly.
 *
 * Conventions (Section 2.1 and Section 3.1):
 *   image    float32 [batch][nz][ny][nx] (2D: nz = 1), i along +x, j = row from the top
 *            (y decreasing), k = slice from the top (z decreasing); unit (k,j,i) has support
 *            [cx+(i-nx/2)dx, cx+(i-nx/2+1)dx] x [cy+(ny/2-j-1)dy, cy+(ny/2-j)dy] x (same in z).
 *   sinogram float32 [batch][n_views][n_rows][n_cols] (2D: n_rows = 1); detector sample
 *            coordinates u_c = (c-(n_cols-1)/2)du + u0, v_r = (r-(n_rows-1)/2)dv + v0.
 *
 * Ownership: every device pointer passed in is CUDA global memory owned by the caller;
 * the library never frees it.  A geometry handle owns its own device tables (one record
 * per ray, built by the ray-setup kernel) and frees them in xr_geometry_destroy.
 *
 * Streams: every launching call is asynchronous and ordered on the given stream
 * (NULL = the legacy default stream); it performs no host synchronisation and no device
 * allocation, so it may be captured in a CUDA graph.
 *
 * Errors: every call returns an xr_status and never aborts or exits.  After XR_ERR_CUDA,
 * xr_last_cuda_error() returns the CUDA error code seen by the calling thread.
 * Thread safety: calls on different handles may run concurrently; calls on one handle
 * must not, and work launched through one handle on different streams must not overlap in
 * time (the handle's workspace holds the interleaved copies and accumulators of the call).
 */
#ifndef XRAY_H
#define XRAY_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* A CUDA stream (cudaStream_t); NULL selects the legacy default stream. */
typedef struct CUstream_st *xr_stream;

typedef enum {
    XR_OK = 0,
    XR_ERR_NULL = 1,      /* a required pointer is NULL */
    XR_ERR_SIZE = 2,      /* a size is non-positive or too large */
    XR_ERR_KIND = 3,      /* unknown scan kind */
    XR_ERR_GEOMETRY = 4,  /* inconsistent scan (spacing <= 0, sdd <= sod, source inside the image) */
    XR_ERR_ALIGN = 5,     /* a device pointer is not 16-byte aligned */
    XR_ERR_CUDA = 6,      /* a CUDA call failed; see xr_last_cuda_error() */
    XR_ERR_ALLOC = 7,     /* device memory for the handle's tables could not be allocated */
    XR_ERR_BATCH = 8,     /* batch < 1 */
    XR_ERR_ARG = 9,       /* an argument is out of its documented range */
    XR_ERR_TUNE = 10,     /* the tuning cache could not be read or written */
    XR_ERR_CAPACITY = 11, /* more problems than XR_NOALLOC_MAX_PROBLEMS */
} xr_status;

/* Scan kinds (Section 2.2 and Section 3.2). */
typedef enum {
    XR_PAR2D = 0,      /* parallel beam: angles[v] = phi, u = s                          (Sec. 2.2.1) */
    XR_FAN2D = 1,      /* equispaced fan, flat detector: angles[v] = alpha (eq. 2Dparalleltofan_2) */
    XR_FAN2D_ARC = 2,  /* equiangular fan: angles[v] = alpha, u is the angle gamma (eq. 2Dparalleltofan) */
    XR_PAR3D = 3,      /* parallel beam: angles[2v], angles[2v+1] = phi1, phi2; u = s1, v = s2 (Sec. 3.2.1) */
    XR_CONE = 4,       /* equispaced circular cone, flat detector: angles[v] = phi'_1 (eq. equispaced_cone_beam) */
    XR_CONE_ARC = 5,   /* equiangular circular cone: u, v are the angles alpha, beta (eq. equiangular_cone_beam) */
    XR_HELIX = 6,      /* equispaced helical cone: src_z[v] = H (eq. Helical_cone_beam_equispaced) */
    XR_HELIX_ARC = 7,  /* equiangular helical cone (eq. Helical_cone_beam_equiangular) */
    XR_RAYS2D = 8,     /* a list of rays given by their parameters: angles[2r], angles[2r+1] = s, phi
                          (Section 4.3, Adaptability); n_views = number of rays */
    XR_RAYS3D = 9,     /* a list of rays: angles[4r .. 4r+3] = s1, s2, phi1, phi2 (Section 4.3) */
} xr_kind;

/* Scan description.  Host memory; the library copies what it needs during
 * xr_geometry_create, so the caller may free it (and the arrays) afterwards.
 * Flat detectors lie at distance sdd from the source; their samples map to the paper's
 * (t, h) on the plane through the rotation axis by t = u*sod/sdd, h = v*sod/sdd.
 * For *_ARC kinds du, u0 (and dv, v0) are angles in radians. */
typedef struct {
    int32_t kind;                  /* xr_kind */
    int32_t nx, ny, nz;            /* image size (2D: nz = 1); each in [1, 16384] */
    double dx, dy, dz;             /* unit spacing (> 0) */
    double cx, cy, cz;             /* image centre (Section 4.2) */
    int32_t n_views, n_rows, n_cols; /* detector (2D: n_rows = 1; ray lists: n_rows = n_cols = 1) */
    const double *angles;          /* [n_views] (XR_PAR3D: [n_views][2]; XR_RAYS2D: [n_rays][2];
                                      XR_RAYS3D: [n_rays][4]) */
    const double *src_z;           /* [n_views] source heights H for helical kinds, else NULL */
    double du, dv, u0, v0;         /* detector sampling */
    double sod, sdd;               /* source-origin and source-detector distances (fan/cone) */
} xr_geometry_desc;

typedef struct xr_geometry xr_geometry;

/* Geometry facts reported by xr_geometry_get_info. */
typedef struct {
    int64_t n_rays;        /* n_views * n_rows * n_cols */
    int64_t n_units;       /* nx * ny * nz */
    int64_t table_bytes;   /* device bytes held by the handle (tables and workspace); 3D parallel,
                              cone and helical scans hold no per-ray table */
    int32_t is3d;
    int32_t device;        /* CUDA device the handle's tables live on */
    int32_t column_batch;  /* 1: a 3D parallel scan whose views all have phi_1 = 0 (or all pi):
                              every ray lies in the y-plane of its detector column (the
                              in-plane case, Section 3.2 Case 2), and with a workspace
                              (xr_reserve) the forward and the gather adjoint run it as a
                              batch of 2D problems, one per column, on the 2D batched kernels.
                              Requires distinct columns in distinct y-slices and no column
                              plane within 1e-6 dy of a slice boundary; 0 otherwise */
    int32_t trace_walk;    /* 1: a cone or helical scan the column-trace walk (XR_ORDER_TRACE)
                              applies to; 0 otherwise */
} xr_geometry_info;

/* Launch tuning of a handle.  Zero fields keep the current value. */
typedef struct {
    int32_t block;         /* threads per block of the ray kernels (64..256, multiple of 32) */
    int32_t batch_chunk;   /* images walked together by one thread (1, 2, 4, 8 or 16);
                              1 also disables the batched paths */
    int32_t adjoint;       /* XR_ADJ_SCATTER or XR_ADJ_GATHER; XR_ADJ_AUTO (the default): the
                              gather on the 2D quad-plane path and for single-tilt-axis
                              parallel scans run as 2D column problems (column_batch), the
                              scatter elsewhere */
    int32_t path;          /* 2D scans, batches >= 4: XR_PATH_TILED, XR_PATH_INTERLEAVED or
                              XR_PATH_RAY (one thread per ray, several images per thread).
                              3D scans: XR_PATH_RAY keeps the one-thread-per-ray kernels on
                              the caller's layout; any other value takes the 3D fast path
                              when a workspace is reserved */
    int32_t order;         /* 3D fast path: the order threads take rays in.  XR_ORDER_VIEW:
                              [view][row][col]; XR_ORDER_ROW: (row, view, col), so the rays in
                              flight share detector rows across views; XR_ORDER_COLUMN: (view,
                              col, row) on a z-fastest copy; XR_ORDER_ROWBLOCK: the same in
                              blocks of 32 rows; XR_ORDER_TRACE: the column-trace walk of cone
                              and helical scans; XR_ORDER_AUTO (the default): TRACE where it
                              applies, else ROWBLOCK for circular cones, for helices VIEW forward
                              and COLUMN adjoint, VIEW otherwise */
} xr_tuning;

enum { XR_ADJ_AUTO = 0, XR_ADJ_SCATTER = 1, XR_ADJ_GATHER = 2 };

/* XR_ORDER_COLUMN (3D fast path): threads run over (view, col, row), so a warp holds 32
 * neighbouring rows of one detector column, and the rays read a z-fastest [y][x][z] copy of
 * the volume (the adjoint adds into a z-fastest accumulator): in a cone or helical scan a
 * column's rays share one vertical plane at neighbouring heights. */
/* XR_ORDER_ROWBLOCK: as XR_ORDER_COLUMN, with the rows taken in blocks of 32 across every
 * view and column before the next block, so that the rays in flight in a circular cone scan
 * cross one slab of z. */
/* XR_ORDER_TRACE (cone and helical scans): the column-trace walk.  The rays of one detector
 * column in one view lie in one vertical plane; a warp computes that plane's xy crossings once
 * (the (i, j) columns of voxels it crosses, in order) and its lanes, one per row of a block of
 * 32, walk them in lockstep with only their own z crossings, on a z-fastest copy of the volume
 * with a zero voxel above and below every column (workspace 4 * nx * ny * (nz + 2) bytes).  Ray
 * records are not used: the rays are rebuilt in the kernel from per-view, per-column and
 * per-sample tables.  Applies when every row crosses at most one z plane while the plane's
 * trace crosses one (x, y) cell (max |rise per horizontal distance| x cell diagonal < 0.99 dz)
 * and nx * ny * (nz + 2) < 2^31; XR_ORDER_AUTO takes it whenever it applies.  The adjoint is a
 * ray-driven scatter (one reduction per row and voxel). */
enum { XR_ORDER_AUTO = 0, XR_ORDER_VIEW = 1, XR_ORDER_ROW = 2, XR_ORDER_COLUMN = 3, XR_ORDER_ROWBLOCK = 4,
       XR_ORDER_TRACE = 5 };

/* Batched paths.  TILED: a CTA stages a 32x32 tile of up to 16 images in shared memory and
 * walks every ray of a group of views through it (2D scans).  INTERLEAVED (the default): the
 * images are copied into device workspace (xr_reserve) as planes of 4 images (one float4 per
 * unit); one thread walks each ray for up to 16 images (forward), one thread gathers a pair
 * of neighbouring pixels (XR_ADJ_GATHER), or 4 lanes per ray add with 128-bit reductions
 * (XR_ADJ_SCATTER); for 3D scans, the single-image path with a y-fastest copy, or the column
 * batch of single-tilt-axis scans.  RAY: one thread per ray on the caller's layout. */
enum { XR_PATH_AUTO = 0, XR_PATH_TILED = 1, XR_PATH_INTERLEAVED = 2, XR_PATH_RAY = 3 };

/* Validate `desc`, allocate the handle and its tables (a per-ray table for 2D scans and ray
 * lists; 3D scans rebuild each ray's record in the kernels) on the current CUDA device and run
 * the ray-setup kernel once (ray parameters from eq. 2Dparalleltofan(_2),
 * equiangular/equispaced_cone_beam, Helical_cone_beam_*, in double precision), then
 * synchronise that device.  On error *out is set to NULL.
 * Errors: XR_ERR_NULL, XR_ERR_KIND, XR_ERR_SIZE, XR_ERR_GEOMETRY, XR_ERR_ALLOC, XR_ERR_CUDA. */
xr_status xr_geometry_create(const xr_geometry_desc *desc, xr_geometry **out);

/* Free the handle and its device tables (synchronises its device).  NULL is accepted. */
void xr_geometry_destroy(xr_geometry *g);

/* Re-run the per-geometry ray setup on `stream`: the detector-sample kernel (the
 * transcendental part of the transformation formulas) and, for handles with a ray table, the
 * per-ray kernel (rebuilds the table in place).  2D parallel beams and 2D ray lists of up to
 * 65535 views, whose detector part needs no transcendentals, build both tables in one launch
 * with the same records. */
xr_status xr_ray_setup(xr_geometry *g, xr_stream stream);

/* Reserve the handle's workspace for batches of up to max_batch images (allocates on the
 * handle's device and synchronises it; do this outside stream capture).
 * 2D scans: with a workspace, xr_project and the adjoint take the batched fast path for
 * batches of 4 or more: the forward interleaves the images of each chunk of 16 so that one
 * unit's values sit in one 64-byte line, in two spatial orders (x fastest and y fastest), and
 * one thread walks each ray for up to 16 images; the gather adjoint builds per-ray records of
 * the sinograms (16 values and the ray's plane constants) after those planes.
 * Workspace bytes: 4 * padded_batch * 2 * (nx+4)(ny+4)nz + 12 * padded_batch * n_rays.
 * For fewer than 4 images the 2D workspace is 8 * (nx (ny+6) + ny (nx+6)) bytes.  When the
 * scan has 1024 rays per SM or more, the forward writes pair planes there (for each driving
 * axis, every column's pairs of neighbouring pixels, three rows of padding on each side) and
 * walks one ray per thread slab by slab on them, one 64-bit load per slab; the adjoint
 * zeroes two accumulator planes there (rows padded by two on each side), into which 32
 * neighbouring rays per warp reduce slab by slab in lockstep, and sums them into the image.
 * 3D scans: the workspace is one [nz][nx][ny] copy of a volume (4 * n_units bytes, any
 * batch); each image is copied into it and every ray reads whichever of the two layouts
 * has its warp's neighbouring rays in neighbouring words; the scatter adjoint uses it as a
 * second accumulator.  Single-tilt-axis parallel scans (xr_geometry_info.column_batch)
 * reserve the larger of that and 16 * P * 2 (nx+4)(nz+4) + 48 * P * n_views * n_rows bytes
 * (P = 4 * ceil(n_cols / 16)): the column images as quad planes, then the gather records of the
 * columns (the largest record set any tuning needs); when that allocation fails the
 * single-image copy is reserved and the 3D walk runs.
 * Without a workspace, or for larger batches, the calls use the one-thread-per-ray kernels
 * on the caller's layout (same lengths).
 * Errors: XR_ERR_NULL, XR_ERR_BATCH, XR_ERR_ALLOC, XR_ERR_CUDA. */
xr_status xr_reserve(xr_geometry *g, int32_t max_batch);

xr_status xr_geometry_get_info(const xr_geometry *g, xr_geometry_info *info);

/* Host-only query (no CUDA call, no allocation on the device): whether a scan description is
 * a single-tilt-axis parallel scan that the forward and the gather adjoint run as 2D column
 * problems (xr_geometry_info.column_batch of a handle made from it), and the y-slice of each
 * detector column's ray plane (Section 3.2, Case 2: with phi_1 = 0 the rays of a column lie in
 * the plane y = s_1 = u).  slice_of: n_cols int32 values written when not NULL: the slice
 * index j (counting down in y), or -1 for a column whose plane misses the volume, and -1 for
 * every column when the scan is not eligible.  *eligible: 1 or 0.
 * Errors: XR_ERR_NULL (desc or eligible NULL), and the codes xr_geometry_create returns for an
 * invalid description (XR_ERR_KIND, XR_ERR_SIZE, XR_ERR_GEOMETRY, XR_ERR_NULL). */
xr_status xr_column_batch_plan(const xr_geometry_desc *desc, int32_t *slice_of, int32_t *eligible);
xr_status xr_set_tuning(xr_geometry *g, const xr_tuning *t);
xr_status xr_get_tuning(const xr_geometry *g, xr_tuning *t);

/* Autotuning (the paper has no counterpart).  Times every candidate tuning of the handle --
 * batched path, images per thread, adjoint method, ray order -- on forward + adjoint of
 * images and sinograms of ones, for the batch size the workspace is reserved for (1 without
 * a reservation; the call reserves it), on a stream of its own, and keeps the fastest.
 * cache_path (may be NULL): a text file with one line per scan and GPU; a scan found there
 * is set without timing anything, a new result is appended.  Allocates and synchronises the
 * handle's device: not for stream capture.
 * Errors: XR_ERR_NULL, XR_ERR_TUNE (no candidate ran, or the cache could not be written),
 * XR_ERR_ALLOC, XR_ERR_CUDA. */
xr_status xr_tune(xr_geometry *g, const char *cache_path);

/* Forward projection (eq. Xray_transform_image): for b < batch and every ray r,
 * sino[b][r] = sum over units I crossed by r of img[b][I] * l_I(r).
 * d_img: [batch][n_units] float32, d_sino: [batch][n_rays] float32 (overwritten).
 * Both 16-byte aligned.  Errors: XR_ERR_NULL, XR_ERR_BATCH, XR_ERR_ALIGN, XR_ERR_CUDA. */
xr_status xr_project(const xr_geometry *g, const float *d_img, float *d_sino, int32_t batch,
                     xr_stream stream);

/* Adjoint (backprojection; the transpose of the forward operator, Section 1):
 * img[b][I] = sum over rays r crossing I of l_I(r) * sino[b][r].  d_img is overwritten.
 * The method is the handle's tuning (ray-driven scatter with atomics, or unit-driven gather
 * over the same condition); both visit the same (ray, unit) pairs with the same lengths. */
xr_status xr_backproject(const xr_geometry *g, const float *d_sino, float *d_img, int32_t batch,
                         xr_stream stream);

/* As xr_backproject with an explicit method (ray lists have no detector to gather over: the
 * scatter only, XR_ADJ_GATHER returns XR_ERR_ARG).  XR_ADJ_SCATTER: ray-driven, each ray adds
 * l * g to every unit it crosses (atomics).  XR_ADJ_GATHER: unit-driven; 2D scans: one thread
 * per pixel (on the batched fast path: per pair of horizontally adjacent pixels, with the
 * views split into chunks whose sums are added in a fixed order) sums the rays whose
 * detector footprint covers it; deterministic, no atomics; 3D scans: one CTA per 16^3
 * tile of voxels walks every ray of the tile's detector footprint through the tile and sums
 * in shared memory.  All give the same (ray, unit) lengths. */
xr_status xr_backproject_method(const xr_geometry *g, const float *d_sino, float *d_img,
                                int32_t batch, int32_t method, xr_stream stream);

/* Forward projection and the adjoint of its result in one launch (the operators of
 * xr_project and xr_backproject, composed; the paper has no counterpart): sino = A img and
 * out = A^T sino, i.e. out = A^T A img.  One thread per ray sums its units (eq.
 * Xray_transform_image), writes sino[b][r], then walks the same units again adding
 * l_I(r) * sino[b][r] into out (atomics, so the order of the additions, and the last bits of
 * out, may differ from run to run).  Meant for problems too small to fill the GPU, whose
 * separate calls are bound by their launches; any scan and batch.  Up to 256 rays per SM
 * (rays x batch), two threads share each ray, one per half of the grid along the ray's
 * driving axis, and add their halves' sums before spreading them.  d_img: [batch][n_units],
 * d_sino: [batch][n_rays] (overwritten), d_out: [batch][n_units] (overwritten), float32,
 * device, 16-byte aligned, none overlapping another.
 * Errors: XR_ERR_NULL, XR_ERR_BATCH, XR_ERR_ALIGN, XR_ERR_ARG (overlapping buffers),
 * XR_ERR_SIZE, XR_ERR_CUDA. */
xr_status xr_project_backproject(const xr_geometry *g, const float *d_img, float *d_sino, float *d_out,
                                 int32_t batch, xr_stream stream);

/* Attenuated transform: the generalized Radon transform of eq. generalizedRadontransform
 * with the exponential attenuation weight of the SPECT case (Section 1),
 * Phi(theta, x, t) = exp(-int_t^inf mu(x + s theta) ds), for an attenuation image d_mu
 * ([n_units] float32, device, one map for the whole batch).  With f and mu constant on each
 * unit, ray r gives sino[b][r] = sum over its units k (in the order the ray crosses them) of
 * img[b][I_k] * exp(-A_k) * E_k, where A_k is the attenuation between unit k and the ray's far
 * end (towards +theta, the ray's own direction) and E_k = (1 - exp(-mu_k l_k)) / mu_k (l_k when
 * mu_k = 0).  Same layouts, alignment and errors as xr_project; one thread per ray on the
 * caller's layout (two walks per ray: the total attenuation, then the weights).
 * xr_backproject_attenuated is its exact transpose (overwrites d_img). */
xr_status xr_project_attenuated(const xr_geometry *g, const float *d_mu, const float *d_img, float *d_sino,
                                int32_t batch, xr_stream stream);
xr_status xr_backproject_attenuated(const xr_geometry *g, const float *d_mu, const float *d_sino, float *d_img,
                                    int32_t batch, xr_stream stream);

/* Device error word of the handle (the paper has no counterpart): bits or-ed in by the
 * handle's kernels since the last call, then cleared.  XR_DEVERR_WALK_BOUND: a ray's walk on
 * the single-image fast path reached its step bound (nx + ny + nz + 2 units) before the
 * image box's exit -- a ray record inconsistent with the grid; its sum is then incomplete.
 * XR_DEVERR_WAIT_BOUND: a kernel's wait for its own asynchronous copies into shared memory
 * (the staged gather adjoint of 2D batches) ran out of its bound (about 2 s); the pixels of
 * the waiting warp are then NaN.
 * Synchronises the handle's device.  Errors: XR_ERR_NULL, XR_ERR_CUDA. */
enum { XR_DEVERR_WALK_BOUND = 1, XR_DEVERR_WAIT_BOUND = 2 };
xr_status xr_get_device_error(const xr_geometry *g, int32_t *code);

/* Sparse rows of the projection matrix (Algorithm 1/2 "Output", Section 4.2): for each of
 * the n rays listed in d_rays (device int64 ray ids), the units it crosses with positive
 * length, written in visiting order to d_idx[q*cap ...] (1D index I, int64) and
 * d_len[q*cap ...] (float32); d_count[q] receives the number of units (int32), which may
 * exceed cap (then only the first cap are written), or -1 for an id outside [0, n_rays).
 * Same walk as xr_project. */
xr_status xr_ray_units(const xr_geometry *g, const int64_t *d_rays, int32_t n, int32_t cap,
                       int64_t *d_idx, float *d_len, int32_t *d_count, xr_stream stream);

/* Compressed sparse rows (CSR) of the projection matrix for the rays [ray0, ray0 + n)
 * (Algorithm 1/2 "Output": each ray's units I with their lengths l; Section 4.2: the matrix
 * stored in sparse pattern).  Two passes over the same walk as xr_ray_units and the
 * crossing-order kernels:
 *   xr_system_rows_count writes d_row_ptr[0 .. n] (device int64, 8-byte aligned): row q (ray
 *   ray0 + q) holds entries d_row_ptr[q] .. d_row_ptr[q + 1] - 1, d_row_ptr[0] = 0 and
 *   d_row_ptr[n] = the number of entries (a counting kernel, then an in-place scan by one CTA;
 *   meant for validation-sized problems);
 *   xr_system_rows_fill then writes d_col[k] (device int64: the 1D unit index I) and d_val[k]
 *   (device float32: the length) for every entry, each row in the order the ray crosses its
 *   units.  The caller allocates d_col and d_val with d_row_ptr[n] elements.
 * Stream-ordered; no allocation.  Errors: XR_ERR_NULL, XR_ERR_SIZE (n < 1, ray0 < 0 or
 * ray0 + n > n_rays), XR_ERR_ALIGN, XR_ERR_CUDA. */
xr_status xr_system_rows_count(const xr_geometry *g, int64_t ray0, int32_t n, int64_t *d_row_ptr, xr_stream stream);
xr_status xr_system_rows_fill(const xr_geometry *g, int64_t ray0, int32_t n, const int64_t *d_row_ptr,
                              int64_t *d_col, float *d_val, xr_stream stream);

/* One problem of a batched launch: a geometry with its own image and sinogram. */
typedef struct {
    const xr_geometry *geom;
    const float *img;   /* device, [n_units], 16-byte aligned */
    float *sino;        /* device, [n_rays], 16-byte aligned */
} xr_problem;

/* A plan for one persistent launch over n independent problems (uneven sizes allowed).
 * The work list -- every problem's rays cut into tiles of `tile` consecutive rays -- is
 * uploaded once here (synchronously); the launches below then do stream work only, so
 * they may be captured in a CUDA graph and replayed while the problems' buffers stay put.
 * tile: rays per work item (32..65536, multiple of 32; 0 = 256); block: threads per CTA
 * (64..256, multiple of 32; 0 = 256).  All geometries must live on the current device.
 * Errors: XR_ERR_NULL, XR_ERR_SIZE, XR_ERR_ALIGN, XR_ERR_ARG, XR_ERR_ALLOC, XR_ERR_CUDA. */
typedef struct xr_batch xr_batch;
xr_status xr_batch_create(const xr_problem *probs, int32_t n, int32_t tile, int32_t block,
                          xr_batch **out);
void xr_batch_destroy(xr_batch *b);

/* The ray setup of every problem of the plan (what xr_ray_setup does for one handle, for the
 * tables the plan's kernels read: each problem's detector-sample table and, where the problem
 * keeps one, its ray table) in two launches over all problems: one thread per detector sample,
 * then one per ray.  Stream-ordered, no allocation.  Errors: XR_ERR_NULL, XR_ERR_CUDA. */
xr_status xr_batch_ray_setup(const xr_batch *b, xr_stream stream);

/* Forward projection of every problem of the plan: one persistent launch whose CTAs (one
 * set per SM, as many as fit) take tiles from one atomic counter until none is left.  When
 * every problem is 2D, one launch first writes each problem's pair planes (every column's
 * pairs of neighbouring pixels) and the rays walk slab by slab on them, one 64-bit load per
 * slab; otherwise the rays walk in crossing order. */
xr_status xr_batch_project(const xr_batch *b, xr_stream stream);

/* Adjoint of every problem of the plan (ray-driven scatter after one zeroing launch):
 * overwrites every problem's img with the adjoint of its sino.  When every problem is 2D,
 * 32 neighbouring rays per warp reduce slab by slab in lockstep into padded accumulator planes,
 * which one more launch sums into the images. */
xr_status xr_batch_backproject(const xr_batch *b, xr_stream stream);

/* Batched forward projection that allocates nothing (the paper has no counterpart; this
 * serves callers that cannot call cudaMalloc where they project: code running during a
 * global-mode stream capture, hosts whose allocator owns the whole device pool, loops that
 * cannot afford the synchronisation of an allocation).  Each ray is walked in crossing order on
 * the caller's layout, as xr_project walks one problem without pair planes: its sums are those
 * of that walk bit for bit, and those of xr_batch_project within rounding (a plan of 2D
 * problems sums the same lengths slab by slab).  The work list and tile counter live in one fixed array in device
 * memory that the library reserves on every device that loads it, until the process exits
 * (XR_NOALLOC_MAX_PROBLEMS work-list entries, about 16 KiB).  The caller still passes and
 * owns every image and sinogram.
 * The first call on a device looks up the array's device address (once, with that device
 * current); make that first call before any stream capture.  Each call rewrites the work
 * list and zeroes the counter, stream-ordered; calls that overlap on the GPU race on the
 * shared array, so order them (one stream, or events).
 * Every problem's geometry must have been created on the current device.
 * tile: rays per work item (32..65536, multiple of 32; 0 = 256).
 * Errors: XR_ERR_NULL, XR_ERR_SIZE (n < 1), XR_ERR_CAPACITY (n > XR_NOALLOC_MAX_PROBLEMS),
 * XR_ERR_ARG (tile out of range, or a geometry of another device), XR_ERR_ALIGN, XR_ERR_CUDA. */
#define XR_NOALLOC_MAX_PROBLEMS 256
xr_status xr_project_batched_noalloc(const xr_problem *probs, int32_t n, int32_t tile,
                                     xr_stream stream);

/* One-call batched forward and adjoint over uneven problems (the paper has no counterpart:
 * batching is a systems form of its per-ray method).  Same work list, capacity
 * (XR_NOALLOC_MAX_PROBLEMS), no-allocation property and concurrency rule as
 * xr_project_batched_noalloc, with work items of 256 rays.  xr_project_batched writes every
 * problem's sino from its img; xr_backproject_batched overwrites every problem's img with
 * the adjoint of its sino (a zero fill, then one persistent scatter launch; the problems'
 * images are the only accumulators, so it is slower than a plan's backproject, which keeps
 * a second layout).  Errors: as xr_project_batched_noalloc. */
xr_status xr_project_batched(const xr_problem *probs, int32_t n, xr_stream stream);
xr_status xr_backproject_batched(const xr_problem *probs, int32_t n, xr_stream stream);

/* Read-bandwidth probe (measurement only; the paper has no counterpart).  Reads the device
 * buffer d_buf of n_floats floats (a multiple of 4, 16-byte aligned) `reps` times with 128-bit
 * loads that are cached in L2 only, on a grid of every SM's resident CTAs, and writes one float
 * per thread to d_sink (device, sink_floats >= SMs x resident CTAs x 256).  Timed with events on
 * `stream`, bytes / time is the L2 read bandwidth when the buffer fits L2.
 * Errors: XR_ERR_NULL, XR_ERR_SIZE, XR_ERR_ALIGN, XR_ERR_CUDA. */
xr_status xr_read_probe(const float *d_buf, int64_t n_floats, int32_t reps, float *d_sink,
                        int32_t sink_floats, xr_stream stream);

/* FP32 FMA probe (measurement only; the paper has no counterpart): every SM's resident CTAs
 * run 8 independent fused multiply-add chains per thread for `iters` steps and write one
 * float per thread to d_sink (sink_floats >= SMs x resident CTAs x 256); *flop receives the
 * FLOP count (2 per FMA) of the launch, to be divided by its event-timed duration.
 * Errors: XR_ERR_NULL, XR_ERR_SIZE, XR_ERR_CUDA. */
xr_status xr_fma_probe(int32_t iters, float *d_sink, int32_t sink_floats, int64_t *flop, xr_stream stream);

/* Self-test of the bounded waits (the paper has no counterpart): one warp of the current device
 * waits, with the wait the staged gather uses for its asynchronous copies, on an mbarrier
 * that nothing completes, giving up after `cycles` SM clock cycles (1 .. 2e10); *timed_out
 * (host) receives 1 when the wait gave up -- the expected result -- and 0 otherwise.  The
 * device stays usable.  Synchronises the current device.
 * Errors: XR_ERR_NULL, XR_ERR_SIZE, XR_ERR_CUDA. */
xr_status xr_wait_bound_selftest(int64_t cycles, int32_t *timed_out);

/* Text of a status code (static storage). */
const char *xr_status_string(xr_status s);

/* CUDA error code of the last XR_ERR_CUDA returned on the calling thread (0 if none). */
int32_t xr_last_cuda_error(void);

/* Library version, e.g. 1 for 0.1. */
int32_t xr_version(void);

#ifdef __cplusplus
}
#endif

#endif /* XRAY_H */
