// Single-tilt-axis parallel scans as batches of 2D problems.
//
// A 3D parallel beam whose views all have phi_1 = 0 (or all phi_1 = pi) has direction
// theta = (c1 cos phi_2, 0, sin phi_2) and foot point (-c1 s_2 sin phi_2, c1 s_1, s_2 cos phi_2)
// (eq. 3Dparallel_direction and the foot point s_1 theta_1 + s_2 theta_2, c1 = cos phi_1 = +-1,
// with s_1 = u the column and s_2 = w the row coordinate).  Every ray lies in the plane
// y = c1 u of its detector column: the in-plane case of Section 3.2 (Case 2, eq.
// condition_nonzero_t_case2_3D_1), where the condition is the 2D one in (x, z) plus the ray's
// plane lying in slice j.  A column is therefore a 2D parallel-beam problem on one y-slice,
// with the rows as its detector, and the whole scan is a batch of such problems, one per
// column, all with the same rays in (x, z).
//
// The batch runs on the 2D quad-plane kernels (fast2d.cu): image b = column b, holding the
// y-slice slice_of[b] of the volume as an (x, z) image; 2D ray r2 = view * n_rows + row;
// the 3D sinogram [view][row][col] is the 2D batch with image stride 1 and ray stride n_cols.
// The 2D ray records are the 3D records of one column with the z components in the y slots:
// the index-space walk in (i, k) is the 3D walk of that column's rays, so every (ray, voxel)
// length is the 3D one.
#include <cmath>
#include <vector>

#include "xray_rays.cuh"

namespace xr {

// 2D ray r2 = the 3D ray (r2, column c_rep) with (w, f, o) of z moved to the y slots.
__global__ void slice_rays_kernel(RaySrc rays3, int64_t n2, int n_cols, int c_rep, RayRec *__restrict__ rays2)
{
    const int64_t r2 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r2 >= n2) return;
    const RayRec R = rays3[r2 * n_cols + c_rep];
    RayRec Q;
    Q.w0 = R.w0;
    Q.w1 = R.w2;
    Q.w2 = 0.f;
    Q.f0 = R.f0;
    Q.f1 = R.f2;
    Q.f2 = 0.f;
    Q.o0 = R.o0;
    Q.o1 = R.o2;
    Q.o2 = 0;
    Q.flags = R.flags;
    rays2[r2] = Q;
}

// Volume [nz][ny][nx] -> quad planes of the column images in both bordered orders (IL0:
// [Q][nz+2P][nx+2P] x fastest, IL1: [Q][nx+2P][nz+2P] z fastest).  Plane q holds columns
// 4q..4q+3; a column without a slice (or past the last column) holds zeros.  The grid covers
// the padded units, so the borders are rewritten on every call.
__global__ void slice_planes_kernel(const float *__restrict__ vol, int nx, int ny, int nz,
                                    const int *__restrict__ slice_of, int n_img, float4 *__restrict__ il0,
                                    float4 *__restrict__ il1)
{
    const int px = nx + 2 * XR_IL_PAD, pz = nz + 2 * XR_IL_PAD;
    const int64_t np = (int64_t)px * pz;
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // padded unit, IL0 order
    if (u >= np) return;
    const int q = blockIdx.y;
    const int ip = (int)(u % px), kp = (int)(u / px);
    const int i = ip - XR_IL_PAD, k = kp - XR_IL_PAD;
    float e[4] = {0.f, 0.f, 0.f, 0.f};
    if (i >= 0 && i < nx && k >= 0 && k < nz) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const int c = 4 * q + b;
            const int sl = c < n_img ? __ldg(slice_of + c) : -1;
            if (sl >= 0) e[b] = __ldg(vol + ((int64_t)k * ny + sl) * nx + i);
        }
    }
    const float4 v = make_float4(e[0], e[1], e[2], e[3]);
    il0[(int64_t)q * np + u] = v;
    il1[(int64_t)q * np + (int64_t)ip * pz + kp] = v;
}

// ---------------------------------------------------------------------------------------
// Host side
// ---------------------------------------------------------------------------------------

// Whether the scan is a batch of 2D problems, and the column -> slice map.  All views must
// have sin(phi_1) = 0 (|sin| < 1e-12, which the ray setup snaps to 0) with one sign of
// cos(phi_1); the column planes y = c1 u_c must keep 1e-6 (in units of dy) away from every
// slice boundary, so that no tie (the bigger-index rule) can round differently here and in
// the 3D setup, and distinct columns must lie in distinct slices.
bool slice_plan(const xr_geometry_desc *d, SlicePlan *sp)
{
    sp->ok = false;
    if (d->kind != XR_PAR3D || d->n_views < 1 || d->n_cols < 1 || !d->angles) return false;
    const double c1 = cos(d->angles[0]);
    if (!(fabs(c1) > 0.5)) return false;
    for (int v = 0; v < d->n_views; ++v) {
        const double a = d->angles[2 * (size_t)v];
        if (!(fabs(sin(a)) < 1e-12) || (cos(a) > 0) != (c1 > 0)) return false;
    }
    const double sgn = c1 > 0 ? 1.0 : -1.0;
    sp->slice_of.assign((size_t)d->n_cols, -1);
    std::vector<char> used((size_t)d->ny, 0);
    sp->c_rep = -1;
    sp->surjective = true;
    for (int c = 0; c < d->n_cols; ++c) {
        const double y = sgn * ((c - 0.5 * (d->n_cols - 1)) * d->du + d->u0);
        const double yh = (d->cy + 0.5 * d->ny * d->dy - y) / d->dy;  // index coordinate, j counts down
        if (fabs(yh - std::nearbyint(yh)) < 1e-6) return false;
        if (yh < 0.0 || yh > d->ny) continue;
        const int j = (int)std::floor(yh);
        if (used[(size_t)j]) return false;
        used[(size_t)j] = 1;
        sp->slice_of[(size_t)c] = j;
        if (sp->c_rep < 0) sp->c_rep = c;
    }
    for (int j = 0; j < d->ny; ++j) sp->surjective = sp->surjective && used[(size_t)j];
    // the 2D problem: x stays x, the 2D y axis is z; the rows are its detector
    GeoParams &p = sp->g2;
    p.kind = XR_PAR2D;
    p.nx = d->nx;
    p.ny = d->nz;
    p.nz = 1;
    p.n_views = d->n_views;
    p.n_rows = 1;
    p.n_cols = d->n_rows;
    p.dx = d->dx;
    p.dy = d->dz;
    p.dz = 1.0;
    p.cx = d->cx;
    p.cy = d->cz;
    p.cz = 0.0;
    p.du = d->dv;
    p.dv = 1.0;
    p.u0 = d->v0;
    p.v0 = 0.0;
    p.sod = p.sdd = 0.0;
    p.inv_dx = 1.0 / p.dx;
    p.inv_dy = 1.0 / p.dy;
    p.inv_dz = 1.0;
    // per view, the row coordinate of a point: w = -c1 sin(phi_2) x + cos(phi_2) z
    sp->vt.assign((size_t)d->n_views * 8, 0.f);
    for (int v = 0; v < d->n_views; ++v) {
        const double a2 = d->angles[2 * (size_t)v + 1];
        sp->vt[8 * (size_t)v + 0] = (float)(-sgn * sin(a2));
        sp->vt[8 * (size_t)v + 1] = (float)cos(a2);
    }
    sp->ok = sp->c_rep >= 0;
    return sp->ok;
}

cudaError_t launch_slice_rays(const RaySrc &rays3, int64_t n2, int n_cols, int c_rep, RayRec *rays2, cudaStream_t s)
{
    slice_rays_kernel<<<(unsigned)((n2 + 255) / 256), 256, 0, s>>>(rays3, n2, n_cols, c_rep, rays2);
    return cudaGetLastError();
}

cudaError_t launch_slice_planes(const float *vol, int nx, int ny, int nz, const int *slice_of, int n_img, float *il0,
                                float *il1, cudaStream_t s)
{
    const int64_t np = (int64_t)(nx + 2 * XR_IL_PAD) * (nz + 2 * XR_IL_PAD);
    const int Q = (n_img + 3) / 4;
    slice_planes_kernel<<<dim3((unsigned)((np + 255) / 256), (unsigned)Q), 256, 0, s>>>(
        vol, nx, ny, nz, slice_of, n_img, reinterpret_cast<float4 *>(il0), reinterpret_cast<float4 *>(il1));
    return cudaGetLastError();
}

}  // namespace xr
