// Per-geometry ray-setup kernel: one thread per ray, double precision.
//
// Scan parameters -> parallel-beam ray parameters by the paper's transformation formulas
// (eq. 2Dparalleltofan, eq. 2Dparalleltofan_2, eq. equiangular_cone_beam,
// eq. equispaced_cone_beam, eq. Helical_cone_beam_equiangular,
// eq. Helical_cone_beam_equispaced), then the ray point and direction
// (eq. direction_normal; eq. 3Dparallel_direction, theta_1, theta_2), then the index-space
// record the walk uses (see xray_core.cuh).
#include "xray_internal.h"

namespace xr {

// cos and sin of an angle; within 1e-12 of a multiple of pi/2 they are exactly 0 and +-1,
// so that axis-parallel and in-plane rays are recognised as such.
__device__ __forceinline__ void cos_sin_snap(double a, double &c, double &s)
{
    sincos(a, &s, &c);
    if (fabs(c) < 1e-12) {
        c = 0.0;
        s = s > 0.0 ? 1.0 : -1.0;
    } else if (fabs(s) < 1e-12) {
        s = 0.0;
        c = c > 0.0 ? 1.0 : -1.0;
    }
}

__global__ void ray_setup_kernel(GeoParams g, const double *__restrict__ angles,
                                 const double *__restrict__ src_z, RayRec *__restrict__ out,
                                 int64_t n_rays)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const int c = (int)(r % g.n_cols);
    const int64_t vr = r / g.n_cols;
    const int row = (int)(vr % g.n_rows);
    const int v = (int)(vr / g.n_rows);
    const double u = (c - 0.5 * (g.n_cols - 1)) * g.du + g.u0;
    const double w = (row - 0.5 * (g.n_rows - 1)) * g.dv + g.v0;
    const double D = g.sod;

    double P[3], T[3];
    if (g.kind <= XR_FAN2D_ARC) {
        double s, phi;
        if (g.kind == XR_PAR2D) {
            s = u;
            phi = angles[v];
        } else if (g.kind == XR_FAN2D) {
            const double t = u * g.sod / g.sdd;  // flat detector -> line through the origin
            s = D * t / sqrt(D * D + t * t);
            phi = atan(t / D) + angles[v] - 0.5 * M_PI;
        } else {
            s = D * sin(u);
            phi = u + angles[v] - 0.5 * M_PI;
        }
        double cp, sp;
        cos_sin_snap(phi, cp, sp);
        T[0] = cp;
        T[1] = sp;
        T[2] = 0.0;
        P[0] = -s * sp;
        P[1] = s * cp;
        P[2] = g.cz;
    } else {
        double s1, s2, phi1, phi2;
        if (g.kind == XR_PAR3D) {
            phi1 = angles[2 * v];
            phi2 = angles[2 * v + 1];
            s1 = u;
            s2 = w;
        } else {
            const double H = (g.kind == XR_HELIX || g.kind == XR_HELIX_ARC) ? src_z[v] : 0.0;
            double alpha, beta;
            if (g.kind == XR_CONE || g.kind == XR_HELIX) {
                const double t = u * g.sod / g.sdd, h = w * g.sod / g.sdd;
                alpha = atan(t / D);
                beta = atan(h / sqrt(D * D + t * t));
                const double ca = cos(alpha), cb = cos(beta);
                s2 = h * ca * ca * cb + H * cb;
            } else {
                alpha = u;
                beta = w;
                s2 = D * cos(alpha) * sin(beta) + H * cos(beta);
            }
            phi1 = angles[v] + alpha;
            phi2 = beta;
            s1 = D * sin(alpha);
        }
        double c1, sn1, c2, sn2;
        cos_sin_snap(phi1, c1, sn1);
        cos_sin_snap(phi2, c2, sn2);
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

    // Index space: u_x grows with i, u_y with j (y falls), u_z with k (z falls).
    const int N[3] = {g.nx, g.ny, g.nz};
    const double o[3] = {(P[0] - (g.cx - 0.5 * g.nx * g.dx)) / g.dx,
                         ((g.cy + 0.5 * g.ny * g.dy) - P[1]) / g.dy,
                         ((g.cz + 0.5 * g.nz * g.dz) - P[2]) / g.dz};
    const double wd[3] = {T[0] / g.dx, -T[1] / g.dy, -T[2] / g.dz};

    RayRec rec;
    int flags = 0;
    float wf[3], ff[3];
    int oi[3];
    double tin = -1e300, tout = 1e300;
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
            const double t0 = (0.0 - o[a]) / wd[a], t1 = (N[a] - o[a]) / wd[a];
            tin = fmax(tin, fmin(t0, t1));
            tout = fmin(tout, fmax(t0, t1));
        }
    }
    if (!(tin < tout)) flags |= RAY_MISS;
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

cudaError_t launch_ray_setup(const GeoParams &g, const double *d_angles, const double *d_src_z,
                             RayRec *d_rays, int64_t n_rays, cudaStream_t s)
{
    const int block = 128;
    const int64_t grid = (n_rays + block - 1) / block;
    ray_setup_kernel<<<(unsigned)grid, block, 0, s>>>(g, d_angles, d_src_z, d_rays, n_rays);
    return cudaGetLastError();
}

}  // namespace xr
