// Per-geometry ray setup in two kernels.
//
// The paper maps every scan to parallel-beam ray parameters by its transformation formulas
// (eq. 2Dparalleltofan, eq. 2Dparalleltofan_2, eq. equiangular_cone_beam,
// eq. equispaced_cone_beam, eq. Helical_cone_beam_equiangular,
// eq. Helical_cone_beam_equispaced).  Their angles split into a part that depends only on
// the detector sample (gamma; alpha and beta) and the view angle, which enters as a sum
// (phi = gamma + alpha_v - pi/2, phi1 = phi'_1 + alpha):
//   * det_setup_kernel: per detector sample, in double precision, the transcendental part
//     (atan, sqrt, sin, cos) -- s, s1, the detector part of s2, and cos/sin of gamma, alpha,
//     beta -- stored as float pairs;
//   * ray_setup_kernel: per ray, cos/sin of the summed angle by the angle-sum identities,
//     the ray point and direction (eq. direction_normal; eq. 3Dparallel_direction,
//     theta_1, theta_2), the foot point closest to the image centre and the index-space
//     record the walk uses (see xray_core.cuh).  A ray list carries each ray's parameters
//     in its per-view record (Section 4.3: the method needs nothing but them).
// The per-ray arithmetic runs on float pairs (hi + lo) with the error-free transformations
// of Dekker (1971) and Knuth (TAOCP vol. 2, 4.2.2): a product's rounding error is recovered
// with one FMA, a sum's with the two-sum sequence.  That keeps about 48 significant bits --
// the foot point's fraction needs about 37 -- on the FP32 pipes.  Products and sums of exact
// values (axis-parallel rays, integer detector offsets) stay exact, so the fixed indices of
// on-grid rays are found as with exact arithmetic.
// The view part (cos/sin of the view angle, source height H) comes from the host.
#include "xray_rays.cuh"

namespace xr {

// The detector part of detector sample d (row d / n_cols, column d % n_cols).
__device__ DetRec det_record(const GeoParams &g, int64_t d)
{
    const int c = (int)(d % g.n_cols), row = (int)(d / g.n_cols);
    const double u = (c - 0.5 * (g.n_cols - 1)) * g.du + g.u0;
    const double w = (row - 0.5 * (g.n_rows - 1)) * g.dv + g.v0;
    const double D = g.sod;
    double s1 = u, s2 = w, ca = 1.0, sa = 0.0, cb = 1.0, sb = 0.0;
    switch (g.kind) {
    case XR_FAN2D: {  // eq. 2Dparalleltofan_2: t on the line through the origin
        const double t = u * g.sod / g.sdd;
        const double gam = atan(t / D);
        s1 = D * t / sqrt(D * D + t * t);
        sincos(gam, &sa, &ca);
        break;
    }
    case XR_FAN2D_ARC:  // eq. 2Dparalleltofan: u is gamma
        s1 = D * sin(u);
        sincos(u, &sa, &ca);
        break;
    case XR_CONE:
    case XR_HELIX: {  // eq. equispaced_cone_beam (+ Helical_cone_beam_equispaced, H added per view)
        const double t = u * g.sod / g.sdd, h = w * g.sod / g.sdd;
        const double alpha = atan(t / D);
        const double beta = atan(h / sqrt(D * D + t * t));
        sincos(alpha, &sa, &ca);
        sincos(beta, &sb, &cb);
        s1 = D * sa;
        s2 = h * ca * ca * cb;
        break;
    }
    case XR_CONE_ARC:
    case XR_HELIX_ARC:  // eq. equiangular_cone_beam (+ Helical_cone_beam_equiangular)
        sincos(u, &sa, &ca);
        sincos(w, &sb, &cb);
        s1 = D * sa;
        s2 = D * ca * sb;
        break;
    default:  // parallel beams: s = u (2D); s1 = u, s2 = w (3D)
        break;
    }
    DetRec R;
    R.s1 = to_df(s1);
    R.s2 = to_df(s2);
    R.ca = to_df(ca);
    R.sa = to_df(sa);
    R.cb = to_df(cb);
    R.sb = to_df(sb);
    return R;
}

__global__ void det_setup_kernel(GeoParams g, DetRec *__restrict__ out)
{
    const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= (int64_t)g.n_rows * g.n_cols) return;
    out[d] = det_record(g, d);
}

// Ray setup of every problem of a batch plan in two launches (detector samples, then rays):
// thread k works on global index k of the concatenated per-problem index ranges.
__device__ __forceinline__ int setup_item(const SetupItem *items, int n, int64_t k, bool rays)
{
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((rays ? items[mid].ray_begin : items[mid].det_begin) <= k) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void batch_det_setup_kernel(const SetupItem *__restrict__ items, int n, int64_t total)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    const SetupItem &S = items[setup_item(items, n, k, false)];
    const int64_t d = k - S.det_begin;
    S.det[d] = det_record(S.g, d);
}

__global__ void batch_ray_setup_kernel(const SetupItem *__restrict__ items, int n, int64_t total)
{
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= total) return;
    const SetupItem &S = items[setup_item(items, n, k, true)];
    const int64_t r = k - S.ray_begin;
    const int64_t ndet = (int64_t)S.g.n_rows * S.g.n_cols;
    const int64_t v = r / ndet;
    S.rays[r] = ray_record(S.g, S.K, S.views[v], S.det[r - v * ndet]);
}

// blockIdx.y = view (when the views fit the grid's y extent), x: detector samples.
__global__ void ray_setup_kernel(GeoParams g, SetupDF K, const ViewDF *__restrict__ views,
                                 const DetRec *__restrict__ det, RayRec *__restrict__ out)
{
    const int ndet = g.n_rows * g.n_cols;
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= ndet) return;
    const int v = blockIdx.y;
    out[(int64_t)v * ndet + d] = ray_record(g, K, views[v], det[d]);
}

// Parallel beams and ray lists: the detector part has no transcendentals (s = u), so each ray
// computes its detector record itself, and view 0's threads also store it -- the ray setup in
// one launch instead of two, the same records bit for bit (a launch-bound step, parallel beam
// 64^2: one dependent launch fewer per step).
__global__ void ray_setup_inline_kernel(GeoParams g, SetupDF K, const ViewDF *__restrict__ views,
                                        DetRec *__restrict__ det, RayRec *__restrict__ out)
{
    const int ndet = g.n_rows * g.n_cols;
    const int d = blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= ndet) return;
    const int v = blockIdx.y;
    const DetRec R = det_record(g, d);
    if (v == 0) det[d] = R;
    out[(int64_t)v * ndet + d] = ray_record(g, K, views[v], R);
}

// The same over a 1D grid, for scans with more views than the grid's y extent.
__global__ void ray_setup_flat_kernel(GeoParams g, SetupDF K, const ViewDF *__restrict__ views,
                                      const DetRec *__restrict__ det, RayRec *__restrict__ out, int64_t n_rays)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const int64_t ndet = (int64_t)g.n_rows * g.n_cols;
    const int64_t v = r / ndet;
    out[r] = ray_record(g, K, views[v], det[r - v * ndet]);
}

cudaError_t launch_batch_setup(const SetupItem *items, int n, int64_t n_det, int64_t n_rays, cudaStream_t s)
{
    const int block = 128;
    if (n_det > 0) batch_det_setup_kernel<<<(unsigned)((n_det + block - 1) / block), block, 0, s>>>(items, n, n_det);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || n_rays <= 0) return e;
    batch_ray_setup_kernel<<<(unsigned)((n_rays + block - 1) / block), block, 0, s>>>(items, n, n_rays);
    return cudaGetLastError();
}

cudaError_t launch_det_setup(const GeoParams &g, DetRec *d_det, cudaStream_t s)
{
    const int64_t n = (int64_t)g.n_rows * g.n_cols;
    det_setup_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g, d_det);
    return cudaGetLastError();
}

cudaError_t launch_ray_setup(const GeoParams &g, const SetupDF &c, const ViewDF *d_views, const DetRec *d_det,
                             RayRec *d_rays, int64_t n_rays, cudaStream_t s)
{
    const int block = 128;
    const int64_t ndet = (int64_t)g.n_rows * g.n_cols;
    if (g.n_views <= 65535) {
        const dim3 grid((unsigned)((ndet + block - 1) / block), (unsigned)g.n_views);
        ray_setup_kernel<<<grid, block, 0, s>>>(g, c, d_views, d_det, d_rays);
    } else {
        ray_setup_flat_kernel<<<(unsigned)((n_rays + block - 1) / block), block, 0, s>>>(g, c, d_views, d_det, d_rays,
                                                                                        n_rays);
    }
    return cudaGetLastError();
}

bool ray_setup_inline_ok(const GeoParams &g)
{
    return (g.kind == XR_PAR2D || g.kind == XR_RAYS2D) && g.n_views <= 65535;
}

cudaError_t launch_ray_setup_inline(const GeoParams &g, const SetupDF &c, const ViewDF *d_views, DetRec *d_det,
                                    RayRec *d_rays, cudaStream_t s)
{
    const int block = 128;
    const int64_t ndet = (int64_t)g.n_rows * g.n_cols;
    const dim3 grid((unsigned)((ndet + block - 1) / block), (unsigned)g.n_views);
    ray_setup_inline_kernel<<<grid, block, 0, s>>>(g, c, d_views, d_det, d_rays);
    return cudaGetLastError();
}

SetupDF make_setup_df(const GeoParams &g)
{
    SetupDF K;
    K.cx = df_from_double(g.cx);
    K.cy = df_from_double(g.cy);
    K.cz = df_from_double(g.cz);
    K.x0 = df_from_double(g.cx - 0.5 * g.nx * g.dx);
    K.y1 = df_from_double(g.cy + 0.5 * g.ny * g.dy);
    K.z1 = df_from_double(g.cz + 0.5 * g.nz * g.dz);
    K.idx = df_from_double(g.inv_dx);
    K.idy = df_from_double(g.inv_dy);
    K.idz = df_from_double(g.inv_dz);
    return K;
}

}  // namespace xr
