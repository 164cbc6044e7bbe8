// Unit-driven adjoint for 3D scans: one CTA per tile of 16 x 16 x 16 voxels.
//
// For every view the CTA projects the tile's corners onto the detector, takes every ray of
// that detector rectangle, walks it through the tile only (the crossing-order walk of
// xray_core.cuh on the tile's box, with the grid's own planes, so each (ray, voxel) length
// is the float the forward computes) and adds l * g into a shared-memory copy of the tile.
// Each voxel is written to global memory once, by the CTA that owns it: no global atomics,
// no zero fill, and the result is the exact transpose of the forward projection.
//
// The rays of all views form one stream of candidates that the CTA's 256 threads take in
// turn (thread t takes every candidate whose running index is t mod 256), so the work
// stays balanced whatever the footprint sizes.
#include "xray_rays.cuh"

namespace xr {

namespace {

constexpr int TX = 16, TY = 16, TZ = 16;
// shared-memory strides of j and k, padded so that 32 lanes at neighbouring j (or k) fall
// in distinct banks
constexpr int PY = TX + 1, PZ = PY * TY + 1;
constexpr int kBlock = 256;  // threads per CTA; also the views whose footprints are computed per pass

// Detector rectangle of one view: first column / row, columns, candidates (0: none).
struct Foot {
    int c0, r0, wc, n;
};

// What the footprint needs, in float.
struct Geo3 {
    int kind, nx, ny, nz, n_views, n_rows, n_cols;
    float x0, y1, z1;  // world x of index plane i = 0, y of plane j = 0, z of plane k = 0
    float dx, dy, dz;
    float sod, sdd, du, dv, u0, v0, half_c, half_r;
};

__device__ __forceinline__ void grow(float v, float &lo, float &hi)
{
    lo = fminf(lo, v);
    hi = fmaxf(hi, v);
}

// Detector coordinates (u, w) of the rays that can meet the box [xa, xb] x [ya, yb] x
// [za, zb] in view V, as a range per coordinate.  Parallel beams: u = p . theta_1,
// w = p . theta_2 (linear, so the corners bound it).  Cones: source S = -sod (cos phi,
// sin phi, 0) + H e_z; a flat detector at sdd has u = sdd lat / depth, w = sdd dz / depth
// (linear-fractional with depth > 0: the corners bound it); an arc detector has angles
// u = atan2(lat, depth), w = atan2(dz, rho), whose elevation is bounded through the ranges
// of dz and of the horizontal distance rho.
__device__ Foot footprint(const Geo3 &G, const ViewRec &V, float xa, float xb, float ya, float yb, float za, float zb)
{
    float ulo = INFINITY, uhi = -INFINITY, wlo = INFINITY, whi = -INFINITY;
    if (G.kind == XR_PAR3D) {
        const float c1 = (float)V.c1, s1 = (float)V.s1, c2 = (float)V.c2, s2 = (float)V.s2;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
            const float x = (q & 1) ? xb : xa, y = (q & 2) ? yb : ya, z = (q & 4) ? zb : za;
            grow(-s1 * x + c1 * y, ulo, uhi);
            grow(-s2 * c1 * x - s2 * s1 * y + c2 * z, wlo, whi);
        }
    } else {
        const float c = (float)V.c1, s = (float)V.s1, H = (float)V.H;
        const float Sx = -G.sod * c, Sy = -G.sod * s;
        const bool flat = (G.kind == XR_CONE || G.kind == XR_HELIX);
        float rlo = INFINITY, rhi = -INFINITY;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float ex = ((q & 1) ? xb : xa) - Sx, ey = ((q & 2) ? yb : ya) - Sy;
            const float depth = ex * c + ey * s, lat = -ex * s + ey * c;
            if (flat) {
                grow(G.sdd * lat / depth, ulo, uhi);
                grow(G.sdd * (za - H) / depth, wlo, whi);
                grow(G.sdd * (zb - H) / depth, wlo, whi);
            } else {
                grow(atan2f(lat, depth), ulo, uhi);
                grow(sqrtf(depth * depth + lat * lat), rlo, rhi);
            }
        }
        if (!flat) {
            // nearest horizontal distance: the source to the box's xy rectangle
            const float px = fminf(fmaxf(Sx, xa), xb) - Sx, py = fminf(fmaxf(Sy, ya), yb) - Sy;
            rlo = fminf(rlo, sqrtf(px * px + py * py));
            const float dza = za - H, dzb = zb - H;
            wlo = atan2f(dza, dza >= 0.f ? rhi : rlo);
            whi = atan2f(dzb, dzb >= 0.f ? rlo : rhi);
        }
    }
    // a ray at detector index c has coordinate (c - half) * du + u0; one index of margin
    const float cl = (ulo - G.u0) / G.du + G.half_c, ch = (uhi - G.u0) / G.du + G.half_c;
    const float rl = (wlo - G.v0) / G.dv + G.half_r, rh = (whi - G.v0) / G.dv + G.half_r;
    Foot F{0, 0, 0, 0};
    if (!(cl <= ch) || !(rl <= rh)) return F;  // also catches NaN
    const int c0 = max((int)floorf(fmaxf(cl, -1e9f)) - 1, 0), c1 = min((int)ceilf(fminf(ch, 1e9f)) + 1, G.n_cols - 1);
    const int r0 = max((int)floorf(fmaxf(rl, -1e9f)) - 1, 0), r1 = min((int)ceilf(fminf(rh, 1e9f)) + 1, G.n_rows - 1);
    if (c0 > c1 || r0 > r1) return F;
    F.c0 = c0;
    F.r0 = r0;
    F.wc = c1 - c0 + 1;
    F.n = F.wc * (r1 - r0 + 1);
    return F;
}

__global__ void __launch_bounds__(kBlock) tile3d_adj_kernel(RaySrc rays,
                                                            const ViewRec *__restrict__ views, Geo3 G, int ntx,
                                                            int nty, const float *__restrict__ sino, int64_t n_rays,
                                                            float *__restrict__ img, int64_t n_units)
{
    __shared__ float acc[PZ * TZ];
    __shared__ Foot fp[kBlock];
    const int tid = threadIdx.x;
    const int tile = blockIdx.x;
    const int tx = tile % ntx, ty = (tile / ntx) % nty, tz = tile / (ntx * nty);
    const int i0 = tx * TX, i1 = min(i0 + TX, G.nx);
    const int j0 = ty * TY, j1 = min(j0 + TY, G.ny);
    const int k0 = tz * TZ, k1 = min(k0 + TZ, G.nz);
    sino += (int64_t)blockIdx.y * n_rays;
    img += (int64_t)blockIdx.y * n_units;
    for (int e = tid; e < PZ * TZ; e += kBlock) acc[e] = 0.f;
    // the tile's world box (y and z fall as j and k grow)
    const float xa = G.x0 + i0 * G.dx, xb = G.x0 + i1 * G.dx;
    const float ya = G.y1 - j1 * G.dy, yb = G.y1 - j0 * G.dy;
    const float za = G.z1 - k1 * G.dz, zb = G.z1 - k0 * G.dz;
    const int max_steps = dda_max_steps(TX, TY, TZ);
    int base = 0;  // running candidate index mod kBlock at the start of the current view
    for (int v0 = 0; v0 < G.n_views; v0 += kBlock) {
        __syncthreads();  // the previous pass's footprints are no longer read
        {
            Foot F{0, 0, 0, 0};
            if (v0 + tid < G.n_views) F = footprint(G, views[v0 + tid], xa, xb, ya, yb, za, zb);
            fp[tid] = F;
        }
        __syncthreads();
        const int nb = min(kBlock, G.n_views - v0);
        for (int q = 0; q < nb; ++q) {
            const Foot F = fp[q];
            if (F.n == 0) continue;
            const int64_t vbase = (int64_t)(v0 + q) * G.n_rows;
            for (int e = (tid - base) & (kBlock - 1); e < F.n; e += kBlock) {
                const int row = F.r0 + e / F.wc, col = F.c0 + e % F.wc;
                const int64_t r = (vbase + row) * G.n_cols + col;
                const float g = __ldg(sino + r);
                if (g == 0.f) continue;
                const RayRec rr = rays[r];
                Dda<int> D;
                if (!dda_setup_box<int>(rr, i0, i1, j0, j1, k0, k1, 1, PY, PZ, D)) continue;
                for (int k = max_steps; k > 0 && D.tcur < D.tout; --k) {
                    int off;
                    float l;
                    dda_step(D, off, l);
                    if (l > 0.f) atomicAdd(&acc[off], __fmul_rn(g, l));
                }
            }
            base = (base + F.n) & (kBlock - 1);
        }
    }
    __syncthreads();
    const int wx = i1 - i0, wy = j1 - j0, wz = k1 - k0;
    for (int e = tid; e < TX * TY * TZ; e += kBlock) {
        const int li = e % TX, lj = (e / TX) % TY, lk = e / (TX * TY);
        if (li < wx && lj < wy && lk < wz)
            img[((int64_t)(k0 + lk) * G.ny + (j0 + lj)) * G.nx + (i0 + li)] = acc[li + PY * lj + PZ * lk];
    }
}

}  // namespace

cudaError_t launch_tile3d_adj(const RaySrc &rays, const ViewRec *views, const GeoParams &g, const float *sino,
                              int64_t n_rays, float *img, int batch, cudaStream_t s)
{
    Geo3 G;
    G.kind = g.kind;
    G.nx = g.nx;
    G.ny = g.ny;
    G.nz = g.nz;
    G.n_views = g.n_views;
    G.n_rows = g.n_rows;
    G.n_cols = g.n_cols;
    G.x0 = (float)(g.cx - 0.5 * g.nx * g.dx);
    G.y1 = (float)(g.cy + 0.5 * g.ny * g.dy);
    G.z1 = (float)(g.cz + 0.5 * g.nz * g.dz);
    G.dx = (float)g.dx;
    G.dy = (float)g.dy;
    G.dz = (float)g.dz;
    G.sod = (float)g.sod;
    G.sdd = (float)g.sdd;
    G.du = (float)g.du;
    G.dv = (float)g.dv;
    G.u0 = (float)g.u0;
    G.v0 = (float)g.v0;
    G.half_c = 0.5f * (float)(g.n_cols - 1);
    G.half_r = 0.5f * (float)(g.n_rows - 1);
    const int ntx = (g.nx + TX - 1) / TX, nty = (g.ny + TY - 1) / TY, ntz = (g.nz + TZ - 1) / TZ;
    const int64_t tiles = (int64_t)ntx * nty * ntz;
    if (tiles > 0x7fffffff || batch > 65535) return cudaErrorInvalidValue;
    const int64_t n_units = (int64_t)g.nx * g.ny * g.nz;
    tile3d_adj_kernel<<<dim3((unsigned)tiles, (unsigned)batch), kBlock, 0, s>>>(rays, views, G, ntx, nty, sino, n_rays,
                                                                               img, n_units);
    return cudaGetLastError();
}

}  // namespace xr
