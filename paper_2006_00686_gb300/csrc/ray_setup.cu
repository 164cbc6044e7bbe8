// Per-geometry ray setup, double precision, in two kernels.
//
// The paper maps every scan to parallel-beam ray parameters by its transformation formulas
// (eq. 2Dparalleltofan, eq. 2Dparalleltofan_2, eq. equiangular_cone_beam,
// eq. equispaced_cone_beam, eq. Helical_cone_beam_equiangular,
// eq. Helical_cone_beam_equispaced).  Their angles split into a part that depends only on
// the detector sample (gamma; alpha and beta) and the view angle, which enters as a sum
// (phi = gamma + alpha_v - pi/2, phi1 = phi'_1 + alpha):
//   * det_setup_kernel: per detector sample, the transcendental part (atan, sqrt, sin,
//     cos) -- s, s1, the detector part of s2, and cos/sin of gamma, alpha, beta;
//   * ray_setup_kernel: per ray, cos/sin of the summed angle by the angle-sum identities,
//     the ray point and direction (eq. direction_normal; eq. 3Dparallel_direction,
//     theta_1, theta_2), the foot point closest to the image centre and the index-space
//     record the walk uses (see xray_core.cuh).  Multiply-adds only.
// The view part (cos/sin of the view angle, source height H) comes from the host.
#include "xray_internal.h"

namespace xr {

// Snap cos/sin pairs within 1e-12 of a multiple of pi/2 to exact 0 and +-1, so that
// axis-parallel and in-plane rays are recognised as such.
__device__ __forceinline__ void snap(double &c, double &s)
{
    if (fabs(c) < 1e-12) {
        c = 0.0;
        s = s > 0.0 ? 1.0 : -1.0;
    } else if (fabs(s) < 1e-12) {
        s = 0.0;
        c = c > 0.0 ? 1.0 : -1.0;
    }
}

__global__ void det_setup_kernel(GeoParams g, DetRec *__restrict__ out)
{
    const int64_t d = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (d >= (int64_t)g.n_rows * g.n_cols) return;
    const int c = (int)(d % g.n_cols), row = (int)(d / g.n_cols);
    const double u = (c - 0.5 * (g.n_cols - 1)) * g.du + g.u0;
    const double w = (row - 0.5 * (g.n_rows - 1)) * g.dv + g.v0;
    const double D = g.sod;
    DetRec R;
    R.s1 = u;
    R.s2 = w;
    R.ca = 1.0;
    R.sa = 0.0;
    R.cb = 1.0;
    R.sb = 0.0;
    switch (g.kind) {
    case XR_FAN2D: {  // eq. 2Dparalleltofan_2: t on the line through the origin
        const double t = u * g.sod / g.sdd;
        const double gam = atan(t / D);
        R.s1 = D * t / sqrt(D * D + t * t);
        sincos(gam, &R.sa, &R.ca);
        break;
    }
    case XR_FAN2D_ARC:  // eq. 2Dparalleltofan: u is gamma
        R.s1 = D * sin(u);
        sincos(u, &R.sa, &R.ca);
        break;
    case XR_CONE:
    case XR_HELIX: {  // eq. equispaced_cone_beam (+ Helical_cone_beam_equispaced, H added per view)
        const double t = u * g.sod / g.sdd, h = w * g.sod / g.sdd;
        const double alpha = atan(t / D);
        const double beta = atan(h / sqrt(D * D + t * t));
        sincos(alpha, &R.sa, &R.ca);
        sincos(beta, &R.sb, &R.cb);
        R.s1 = D * R.sa;
        R.s2 = h * R.ca * R.ca * R.cb;
        break;
    }
    case XR_CONE_ARC:
    case XR_HELIX_ARC:  // eq. equiangular_cone_beam (+ Helical_cone_beam_equiangular)
        sincos(u, &R.sa, &R.ca);
        sincos(w, &R.sb, &R.cb);
        R.s1 = D * R.sa;
        R.s2 = D * R.ca * R.sb;
        break;
    default:  // parallel beams: s = u (2D); s1 = u, s2 = w (3D)
        break;
    }
    out[d] = R;
}

__global__ void ray_setup_kernel(GeoParams g, const ViewRec *__restrict__ views,
                                 const DetRec *__restrict__ det, RayRec *__restrict__ out, int64_t n_rays)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const int64_t ndet = (int64_t)g.n_rows * g.n_cols;
    const int v = (int)(r / ndet);
    const DetRec R = det[r - (int64_t)v * ndet];
    const ViewRec V = views[v];

    double P[3], T[3];
    if (g.kind <= XR_FAN2D_ARC) {
        double cp, sp;
        if (g.kind == XR_PAR2D) {
            cp = V.c1;  // phi = angles[v]
            sp = V.s1;
        } else {
            // phi = gamma + alpha - pi/2: cos(phi) = sin(gamma + alpha), sin(phi) = -cos(gamma + alpha)
            cp = R.sa * V.c1 + R.ca * V.s1;
            sp = R.sa * V.s1 - R.ca * V.c1;
        }
        snap(cp, sp);
        T[0] = cp;
        T[1] = sp;
        T[2] = 0.0;
        P[0] = -R.s1 * sp;
        P[1] = R.s1 * cp;
        P[2] = g.cz;
    } else {
        double c1, sn1, c2, sn2, s1 = R.s1, s2 = R.s2;
        if (g.kind == XR_PAR3D) {
            c1 = V.c1;
            sn1 = V.s1;
            c2 = V.c2;
            sn2 = V.s2;
        } else {
            // phi1 = phi'_1 + alpha, phi2 = beta
            c1 = V.c1 * R.ca - V.s1 * R.sa;
            sn1 = V.s1 * R.ca + V.c1 * R.sa;
            c2 = R.cb;
            sn2 = R.sb;
            s2 += V.H * R.cb;
        }
        snap(c1, sn1);
        snap(c2, sn2);
        T[0] = c2 * c1;
        T[1] = c2 * sn1;
        T[2] = sn2;
        P[0] = -s1 * sn1 - s2 * sn2 * c1;
        P[1] = s1 * c1 - s2 * sn2 * sn1;
        P[2] = s2 * c2;
    }
    // Foot point: the point of the line closest to the image centre.
    const double tf = (g.cx - P[0]) * T[0] + (g.cy - P[1]) * T[1] + (g.cz - P[2]) * T[2];
    for (int a = 0; a < 3; ++a) P[a] += (T[a] == 0.0 ? 0.0 : tf * T[a]);

    // Index space: u_x grows with i, u_y with j (y falls), u_z with k (z falls).  The
    // reciprocal spacings come from the host; whether the ray enters the image is decided by
    // the walk's own box test.
    const int N[3] = {g.nx, g.ny, g.nz};
    const double o[3] = {(P[0] - (g.cx - 0.5 * g.nx * g.dx)) * g.inv_dx,
                         ((g.cy + 0.5 * g.ny * g.dy) - P[1]) * g.inv_dy,
                         ((g.cz + 0.5 * g.nz * g.dz) - P[2]) * g.inv_dz};
    const double wd[3] = {T[0] * g.inv_dx, -T[1] * g.inv_dy, -T[2] * g.inv_dz};

    RayRec rec;
    int flags = 0;
    float wf[3], ff[3];
    int oi[3];
    for (int a = 0; a < 3; ++a) {
        if (wd[a] == 0.0) {
            // Fixed index: unit n holds u in [n, n+1]; a ray on the plane u = n (two
            // candidates) takes the bigger index (Section 4.1), the far edge u = N the last.
            wf[a] = 0.f;
            ff[a] = 0.f;
            if (o[a] >= 0.0 && o[a] <= N[a]) {
                oi[a] = min((int)floor(o[a]), N[a] - 1);
            } else {
                oi[a] = -1;
                flags |= RAY_MISS;
            }
        } else {
            double fl = floor(o[a]);
            float fr = (float)(o[a] - fl);
            if (fr >= 1.0f) {
                fr = 0.0f;
                fl += 1.0;
            }
            wf[a] = (float)wd[a];
            ff[a] = fr;
            if (fabs(fl) > 32000.0) {
                flags |= RAY_MISS;
                fl = 0.0;
            }
            oi[a] = (int)fl;
        }
    }
    rec.w0 = wf[0];
    rec.w1 = wf[1];
    rec.w2 = wf[2];
    rec.f0 = ff[0];
    rec.f1 = ff[1];
    rec.f2 = ff[2];
    rec.o0 = (int16_t)oi[0];
    rec.o1 = (int16_t)oi[1];
    rec.o2 = (int16_t)oi[2];
    rec.flags = (int16_t)flags;
    out[r] = rec;
}

cudaError_t launch_det_setup(const GeoParams &g, DetRec *d_det, cudaStream_t s)
{
    const int64_t n = (int64_t)g.n_rows * g.n_cols;
    det_setup_kernel<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(g, d_det);
    return cudaGetLastError();
}

cudaError_t launch_ray_setup(const GeoParams &g, const ViewRec *d_views, const DetRec *d_det, RayRec *d_rays,
                             int64_t n_rays, cudaStream_t s)
{
    const int block = 128;
    const int64_t grid = (n_rays + block - 1) / block;
    ray_setup_kernel<<<(unsigned)grid, block, 0, s>>>(g, d_views, d_det, d_rays, n_rays);
    return cudaGetLastError();
}

}  // namespace xr
