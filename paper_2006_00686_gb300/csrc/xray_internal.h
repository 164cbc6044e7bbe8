// Internal declarations shared by the library's translation units.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "xray.h"
#include "xray_core.cuh"

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

namespace xr {

// Scan description passed by value to the ray-setup kernel.
struct GeoParams {
    int kind, nx, ny, nz, n_views, n_rows, n_cols;
    double dx, dy, dz, cx, cy, cz, du, dv, u0, v0, sod, sdd;
};

// Image extents and layout strides passed to the ray kernels.
struct Grid {
    int nx, ny, nz;
    int64_t sx, sy, sz;  // element strides of i, j, k
};

cudaError_t launch_ray_setup(const GeoParams &g, const double *d_angles, const double *d_src_z,
                             RayRec *d_rays, int64_t n_rays, cudaStream_t s);

cudaError_t launch_project(const RayRec *rays, int64_t n_rays, const Grid &grid, const float *img,
                           int64_t img_bs, float *sino, int64_t sino_bs, int batch, int chunk,
                           int block, cudaStream_t s);

cudaError_t launch_backproject_scatter(const RayRec *rays, int64_t n_rays, const Grid &grid,
                                       const float *sino, int64_t sino_bs, float *img,
                                       int64_t img_bs, int batch, int chunk, int block,
                                       cudaStream_t s);

cudaError_t launch_backproject_gather2d(const RayRec *rays, const GeoParams &g, const Grid &grid,
                                        const double *d_view_tab, const float *sino,
                                        int64_t sino_bs, float *img, int64_t img_bs, int batch,
                                        int chunk, int block, cudaStream_t s);

cudaError_t launch_ray_units(const RayRec *rays, int64_t n_rays, const Grid &grid, const int64_t *ray_ids,
                             int n, int cap, int64_t *idx, float *len, int32_t *count, cudaStream_t s);

// One problem of a persistent batched launch (device copy).
struct BatchItem {
    const RayRec *rays;
    const float *img;
    float *sino;
    int nx, ny, nz;
    int pad;
    int64_t n_rays;
    int64_t tile_begin;  // first global tile index of this problem
};

cudaError_t launch_batched(const BatchItem *items, int n_items, int64_t n_tiles, int tile,
                           unsigned long long *counter, int adjoint, int grid_ctas, int block,
                           cudaStream_t s);

// Forward persistent launch over a work list already in device memory; the tile counter
// must be zero (no memset here).
cudaError_t launch_batched_items(const BatchItem *items, int n_items, int64_t n_tiles, int tile,
                                 unsigned long long *counter, int grid_ctas, int block, cudaStream_t s);

int batched_ctas_per_sm(int block, int adjoint);

}  // namespace xr

// Record a CUDA error for xr_last_cuda_error() and return XR_ERR_CUDA.
xr_status xr_fail_cuda(cudaError_t e);

// The handle behind the opaque xr_geometry.
struct xr_geometry {
    xr_geometry_desc desc;  // copy; the array pointers are not kept
    xr::GeoParams params;
    int device;
    int64_t n_rays, n_units;
    double *d_angles;
    double *d_src_z;
    xr::RayRec *d_rays;
    double *d_view_tab;  // per view: 2D gather footprint data
    xr_tuning tune;
};
