// Ray kernels on the caller's layout: forward projection, ray-driven scatter adjoint,
// unit-driven gather adjoint (2D) and sparse-row export.  All FP32 with FP32
// accumulation; no tensor cores (the work is a gather along rays, not a contraction).
#include "xray_rays.cuh"

namespace xr {

// ---------------------------------------------------------------------------------------
// Visitors
// ---------------------------------------------------------------------------------------

// Forward: acc[b] += f_b[I] * l for the `nb` images of this thread's chunk.
template <int BC>
struct FwdVisitor {
    const float *__restrict__ img;
    int64_t bs;
    int nb;
    float acc[BC];
    __device__ __forceinline__ void operator()(int64_t off, float l)
    {
#pragma unroll
        for (int b = 0; b < BC; ++b)
            if (b < nb) acc[b] = __fmaf_rn(__ldg(img + b * bs + off), l, acc[b]);
    }
};

// Adjoint, ray-driven: img_b[I] += g_b * l (fire-and-forget atomic adds).
template <int BC>
struct ScatterVisitor {
    float *__restrict__ img;
    int64_t bs;
    int nb;
    float g[BC];
    __device__ __forceinline__ void operator()(int64_t off, float l)
    {
#pragma unroll
        for (int b = 0; b < BC; ++b)
            if (b < nb && g[b] != 0.f) red_add(img + b * bs + off, __fmul_rn(g[b], l));
    }
};

// Sparse-row export: (I, l) in visiting order, up to cap entries.
struct ExportVisitor {
    int64_t *idx;
    float *len;
    int cap;
    int n;
    __device__ __forceinline__ void operator()(int64_t off, float l)
    {
        if (n < cap) {
            idx[n] = off;
            len[n] = l;
        }
        ++n;
    }
};

// ---------------------------------------------------------------------------------------
// Forward projection: one thread per ray, `BC` images per thread (blockIdx.y = image chunk)
// ---------------------------------------------------------------------------------------

template <int BC>
__global__ void __launch_bounds__(256) project_kernel(RaySrc rays, int64_t n_rays,
                                                      Grid grid, const float *__restrict__ img,
                                                      int64_t img_bs, float *__restrict__ sino,
                                                      int64_t sino_bs, int batch)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const int b0 = blockIdx.y * BC;
    FwdVisitor<BC> vis;
    vis.img = img + b0 * img_bs;
    vis.bs = img_bs;
    vis.nb = min(BC, batch - b0);
#pragma unroll
    for (int b = 0; b < BC; ++b) vis.acc[b] = 0.f;
    walk_ray(rays[r], grid.nx, grid.ny, grid.nz, grid.sx, grid.sy, grid.sz, grid.three, vis);
#pragma unroll
    for (int b = 0; b < BC; ++b)
        if (b < vis.nb) sino[(b0 + b) * sino_bs + r] = vis.acc[b];
}

template <int BC>
__global__ void __launch_bounds__(256) scatter_kernel(RaySrc rays, int64_t n_rays,
                                                      Grid grid, const float *__restrict__ sino,
                                                      int64_t sino_bs, float *__restrict__ img,
                                                      int64_t img_bs, int batch)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const int b0 = blockIdx.y * BC;
    ScatterVisitor<BC> vis;
    vis.img = img + b0 * img_bs;
    vis.bs = img_bs;
    vis.nb = min(BC, batch - b0);
    bool any = false;
#pragma unroll
    for (int b = 0; b < BC; ++b) {
        vis.g[b] = (b < vis.nb) ? __ldg(sino + (b0 + b) * sino_bs + r) : 0.f;
        any |= vis.g[b] != 0.f;
    }
    if (!any) return;
    walk_ray(rays[r], grid.nx, grid.ny, grid.nz, grid.sx, grid.sy, grid.sz, grid.three, vis);
}

// Forward, then the adjoint of the forward's result, in one pass per ray: the thread sums its
// ray (y = A x, written to sino) and walks the same units again spreading y * l into out
// (zeroed by the caller): out = A^T A x.  The two walks are the kernels' above.
template <int BC>
__global__ void __launch_bounds__(256) project_backproject_kernel(RaySrc rays, int64_t n_rays, Grid grid,
                                                                  const float *__restrict__ img, int64_t img_bs,
                                                                  float *__restrict__ sino, int64_t sino_bs,
                                                                  float *__restrict__ out, int64_t out_bs, int batch)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const int b0 = blockIdx.y * BC;
    const RayRec rr = rays[r];
    FwdVisitor<BC> f;
    f.img = img + b0 * img_bs;
    f.bs = img_bs;
    f.nb = min(BC, batch - b0);
#pragma unroll
    for (int b = 0; b < BC; ++b) f.acc[b] = 0.f;
    walk_ray(rr, grid.nx, grid.ny, grid.nz, grid.sx, grid.sy, grid.sz, grid.three, f);
    ScatterVisitor<BC> sv;
    sv.img = out + b0 * out_bs;
    sv.bs = out_bs;
    sv.nb = f.nb;
    bool any = false;
#pragma unroll
    for (int b = 0; b < BC; ++b) {
        sv.g[b] = b < f.nb ? f.acc[b] : 0.f;
        if (b < f.nb) sino[(b0 + b) * sino_bs + r] = f.acc[b];
        any |= sv.g[b] != 0.f;
    }
    if (any) walk_ray(rr, grid.nx, grid.ny, grid.nz, grid.sx, grid.sy, grid.sz, grid.three, sv);
}

template <int BC>
static cudaError_t launch_project_t(const RaySrc &rays, int64_t n_rays, const Grid &grid,
                                    const float *img, int64_t img_bs, float *sino, int64_t sino_bs,
                                    int batch, int block, cudaStream_t s)
{
    const dim3 g((unsigned)((n_rays + block - 1) / block), (unsigned)((batch + BC - 1) / BC));
    project_kernel<BC><<<g, block, 0, s>>>(rays, n_rays, grid, img, img_bs, sino, sino_bs, batch);
    return cudaGetLastError();
}

template <int BC>
static cudaError_t launch_scatter_t(const RaySrc &rays, int64_t n_rays, const Grid &grid,
                                    const float *sino, int64_t sino_bs, float *img, int64_t img_bs,
                                    int batch, int block, cudaStream_t s)
{
    const dim3 g((unsigned)((n_rays + block - 1) / block), (unsigned)((batch + BC - 1) / BC));
    scatter_kernel<BC><<<g, block, 0, s>>>(rays, n_rays, grid, sino, sino_bs, img, img_bs, batch);
    return cudaGetLastError();
}

cudaError_t launch_project(const RaySrc &rays, int64_t n_rays, const Grid &grid, const float *img,
                           int64_t img_bs, float *sino, int64_t sino_bs, int batch, int chunk,
                           int block, cudaStream_t s)
{
    switch (chunk) {
    case 16: return launch_project_t<16>(rays, n_rays, grid, img, img_bs, sino, sino_bs, batch, block, s);
    case 8: return launch_project_t<8>(rays, n_rays, grid, img, img_bs, sino, sino_bs, batch, block, s);
    case 4: return launch_project_t<4>(rays, n_rays, grid, img, img_bs, sino, sino_bs, batch, block, s);
    case 2: return launch_project_t<2>(rays, n_rays, grid, img, img_bs, sino, sino_bs, batch, block, s);
    default: return launch_project_t<1>(rays, n_rays, grid, img, img_bs, sino, sino_bs, batch, block, s);
    }
}

template <int BC>
static cudaError_t launch_project_backproject_t(const RaySrc &rays, int64_t n_rays, const Grid &grid,
                                                const float *img, int64_t img_bs, float *sino, int64_t sino_bs,
                                                float *out, int64_t out_bs, int batch, int block, cudaStream_t s)
{
    const dim3 g((unsigned)((n_rays + block - 1) / block), (unsigned)((batch + BC - 1) / BC));
    project_backproject_kernel<BC><<<g, block, 0, s>>>(rays, n_rays, grid, img, img_bs, sino, sino_bs, out, out_bs,
                                                       batch);
    return cudaGetLastError();
}

cudaError_t launch_project_backproject(const RaySrc &rays, int64_t n_rays, const Grid &grid, const float *img,
                                       int64_t img_bs, float *sino, int64_t sino_bs, float *out, int64_t out_bs,
                                       int batch, int chunk, int block, cudaStream_t s)
{
    switch (chunk) {
    case 16: return launch_project_backproject_t<16>(rays, n_rays, grid, img, img_bs, sino, sino_bs, out, out_bs, batch, block, s);
    case 8: return launch_project_backproject_t<8>(rays, n_rays, grid, img, img_bs, sino, sino_bs, out, out_bs, batch, block, s);
    case 4: return launch_project_backproject_t<4>(rays, n_rays, grid, img, img_bs, sino, sino_bs, out, out_bs, batch, block, s);
    case 2: return launch_project_backproject_t<2>(rays, n_rays, grid, img, img_bs, sino, sino_bs, out, out_bs, batch, block, s);
    default: return launch_project_backproject_t<1>(rays, n_rays, grid, img, img_bs, sino, sino_bs, out, out_bs, batch, block, s);
    }
}

cudaError_t launch_backproject_scatter(const RaySrc &rays, int64_t n_rays, const Grid &grid,
                                       const float *sino, int64_t sino_bs, float *img,
                                       int64_t img_bs, int batch, int chunk, int block,
                                       cudaStream_t s)
{
    switch (chunk) {
    case 16: return launch_scatter_t<16>(rays, n_rays, grid, sino, sino_bs, img, img_bs, batch, block, s);
    case 8: return launch_scatter_t<8>(rays, n_rays, grid, sino, sino_bs, img, img_bs, batch, block, s);
    case 4: return launch_scatter_t<4>(rays, n_rays, grid, sino, sino_bs, img, img_bs, batch, block, s);
    case 2: return launch_scatter_t<2>(rays, n_rays, grid, sino, sino_bs, img, img_bs, batch, block, s);
    default: return launch_scatter_t<1>(rays, n_rays, grid, sino, sino_bs, img, img_bs, batch, block, s);
    }
}

// ---------------------------------------------------------------------------------------
// Adjoint, unit-driven gather (2D): one thread per pixel; for every view, the detector bins
// whose rays can cross the pixel (projection of its corners, one bin of margin), and for
// each the length the forward walk gives that (ray, pixel) pair.
// View table (8 floats per view): parallel: (-sin phi, cos phi); fan: source (Sx, Sy),
// central direction (ex, ey), detector direction (tx, ty).
// ---------------------------------------------------------------------------------------

template <int BC>
__global__ void __launch_bounds__(256) gather2d_kernel(const RayRec *__restrict__ rays, GeoParams g,
                                                       Grid grid, const float *__restrict__ vt,
                                                       const float *__restrict__ sino, int64_t sino_bs,
                                                       float *__restrict__ img, int64_t img_bs, int batch)
{
    const int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t n_pix = (int64_t)g.nx * g.ny;
    if (p >= n_pix) return;
    const int i = (int)(p % g.nx), j = (int)(p / g.nx);
    const int b0 = blockIdx.y * BC;
    const int nb = min(BC, batch - b0);
    float acc[BC];
#pragma unroll
    for (int b = 0; b < BC; ++b) acc[b] = 0.f;
    // pixel corners (world coordinates)
    const float x0 = (float)(g.cx + (i - 0.5 * g.nx) * g.dx), x1 = x0 + (float)g.dx;
    const float y1 = (float)(g.cy + (0.5 * g.ny - j) * g.dy), y0 = y1 - (float)g.dy;
    const float half = 0.5f * (float)(g.n_cols - 1);
    const float inv_du = (float)(1.0 / g.du), u0 = (float)g.u0;
    for (int v = 0; v < g.n_views; ++v) {
        const float *e = vt + 8 * v;
        float cmin = 1e30f, cmax = -1e30f;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float X = (q & 1) ? x1 : x0, Y = (q & 2) ? y1 : y0;
            float uc;
            if (g.kind == XR_PAR2D) {
                uc = e[0] * X + e[1] * Y;
            } else {
                const float rx = X - e[0], ry = Y - e[1];
                const float depth = rx * e[2] + ry * e[3];
                const float lat = rx * e[4] + ry * e[5];
                uc = (g.kind == XR_FAN2D) ? (float)g.sdd * lat / depth : atan2f(lat, depth);
            }
            const float c = (uc - u0) * inv_du + half;
            cmin = fminf(cmin, c);
            cmax = fmaxf(cmax, c);
        }
        const int c0 = max((int)floorf(cmin) - 1, 0), c1 = min((int)ceilf(cmax) + 1, g.n_cols - 1);
        for (int c = c0; c <= c1; ++c) {
            const int64_t r = (int64_t)v * g.n_cols + c;
            Walk W;
            if (!walk_setup(rays[r], grid.nx, grid.ny, grid.nz, grid.sx, grid.sy, grid.sz, W)) continue;
            const float l = walk_unit_length(W, i, j, 0);
            if (l > 0.f) {
#pragma unroll
                for (int b = 0; b < BC; ++b)
                    if (b < nb) acc[b] = __fmaf_rn(__ldg(sino + (b0 + b) * sino_bs + r), l, acc[b]);
            }
        }
    }
#pragma unroll
    for (int b = 0; b < BC; ++b)
        if (b < nb) img[(b0 + b) * img_bs + (int64_t)j * grid.sy + (int64_t)i * grid.sx] = acc[b];
}

template <int BC>
static cudaError_t launch_gather_t(const RayRec *rays, const GeoParams &g, const Grid &grid,
                                   const float *vt, const float *sino, int64_t sino_bs, float *img,
                                   int64_t img_bs, int batch, int block, cudaStream_t s)
{
    const int64_t n_pix = (int64_t)g.nx * g.ny;
    const dim3 gr((unsigned)((n_pix + block - 1) / block), (unsigned)((batch + BC - 1) / BC));
    gather2d_kernel<BC><<<gr, block, 0, s>>>(rays, g, grid, vt, sino, sino_bs, img, img_bs, batch);
    return cudaGetLastError();
}

cudaError_t launch_backproject_gather2d(const RayRec *rays, const GeoParams &g, const Grid &grid,
                                        const float *vt, const float *sino, int64_t sino_bs,
                                        float *img, int64_t img_bs, int batch, int chunk, int block,
                                        cudaStream_t s)
{
    switch (chunk) {
    case 16: return launch_gather_t<16>(rays, g, grid, vt, sino, sino_bs, img, img_bs, batch, block, s);
    case 8: return launch_gather_t<8>(rays, g, grid, vt, sino, sino_bs, img, img_bs, batch, block, s);
    case 4: return launch_gather_t<4>(rays, g, grid, vt, sino, sino_bs, img, img_bs, batch, block, s);
    case 2: return launch_gather_t<2>(rays, g, grid, vt, sino, sino_bs, img, img_bs, batch, block, s);
    default: return launch_gather_t<1>(rays, g, grid, vt, sino, sino_bs, img, img_bs, batch, block, s);
    }
}

// ---------------------------------------------------------------------------------------
// Sparse rows (projection-matrix export): one thread per listed ray.
// ---------------------------------------------------------------------------------------

__global__ void ray_units_kernel(RaySrc rays, int64_t n_rays, Grid grid,
                                 const int64_t *__restrict__ ids, int n, int cap,
                                 int64_t *__restrict__ idx, float *__restrict__ len,
                                 int32_t *__restrict__ count)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int64_t id = ids[q];
    if (id < 0 || id >= n_rays) {  // not a ray of this scan: empty row, count -1
        count[q] = -1;
        return;
    }
    ExportVisitor vis{idx + (int64_t)q * cap, len + (int64_t)q * cap, cap, 0};
    walk_ray(rays[id], grid.nx, grid.ny, grid.nz, grid.sx, grid.sy, grid.sz, grid.three, vis);
    count[q] = vis.n;
}

cudaError_t launch_ray_units(const RaySrc &rays, int64_t n_rays, const Grid &grid, const int64_t *ids, int n,
                             int cap, int64_t *idx, float *len, int32_t *count, cudaStream_t s)
{
    const int block = 128;
    ray_units_kernel<<<(n + block - 1) / block, block, 0, s>>>(rays, n_rays, grid, ids, n, cap, idx, len,
                                                               count);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------------------
// Compressed sparse rows of the projection matrix: a counting pass, a scan of the counts into
// row pointers, a filling pass.  Both passes walk each ray the same way, so the fill writes
// exactly the counted entries.
// ---------------------------------------------------------------------------------------

struct CountVisitor {
    int64_t n;
    __device__ __forceinline__ void operator()(int64_t, float) { ++n; }
};

struct CsrVisitor {
    int64_t *col;
    float *val;
    int64_t k, end;  // next slot, end of the row
    __device__ __forceinline__ void operator()(int64_t off, float l)
    {
        if (k < end) {  // never false: the counting pass walked the same units
            col[k] = off;
            val[k] = l;
        }
        ++k;
    }
};

// ptr[q + 1] = number of units ray ray0 + q crosses; ptr[0] = 0
__global__ void csr_count_kernel(RaySrc rays, int64_t ray0, int n, Grid grid, int64_t *__restrict__ ptr)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q == 0) ptr[0] = 0;
    if (q >= n) return;
    CountVisitor vis{0};
    walk_ray(rays[ray0 + q], grid.nx, grid.ny, grid.nz, grid.sx, grid.sy, grid.sz, grid.three, vis);
    ptr[q + 1] = vis.n;
}

// In-place inclusive scan of a[0 .. n) by one CTA of 1024 threads, 4096 elements per round with
// the running total carried between rounds (no scratch memory).
__global__ void __launch_bounds__(1024) csr_scan_kernel(int64_t *__restrict__ a, int64_t n)
{
    __shared__ int64_t warp_tot[32];
    __shared__ int64_t carry_s;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int64_t base = 0; base < n; base += 4096) {
        const int64_t i0 = base + (int64_t)threadIdx.x * 4;
        int64_t v[4], t = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            v[k] = (i0 + k < n) ? a[i0 + k] : 0;
            t += v[k];
            v[k] = t;  // inclusive within the thread
        }
        // inclusive scan of the thread totals across the warp, then across the warps
        int64_t x = t;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int64_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane == 31) warp_tot[w] = x;
        __syncthreads();
        if (w == 0) {
            int64_t z = warp_tot[lane];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, z, d);
                if (lane >= d) z += y;
            }
            warp_tot[lane] = z;  // inclusive over warps
        }
        __syncthreads();
        const int64_t before = carry_s + (w > 0 ? warp_tot[w - 1] : 0) + (x - t);
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (i0 + k < n) a[i0 + k] = before + v[k];
        __syncthreads();
        if (threadIdx.x == 0) carry_s += warp_tot[31];
        __syncthreads();
    }
}

__global__ void csr_fill_kernel(RaySrc rays, int64_t ray0, int n, Grid grid, const int64_t *__restrict__ ptr,
                                int64_t *__restrict__ col, float *__restrict__ val)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    CsrVisitor vis{col, val, ptr[q], ptr[q + 1]};
    walk_ray(rays[ray0 + q], grid.nx, grid.ny, grid.nz, grid.sx, grid.sy, grid.sz, grid.three, vis);
}

cudaError_t launch_csr_count(const RaySrc &rays, int64_t ray0, int n, const Grid &grid, int64_t *ptr, cudaStream_t s)
{
    const int block = 128;
    csr_count_kernel<<<(unsigned)((n + block - 1) / block), block, 0, s>>>(rays, ray0, n, grid, ptr);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    csr_scan_kernel<<<1, 1024, 0, s>>>(ptr + 1, n);
    return cudaGetLastError();
}

cudaError_t launch_csr_fill(const RaySrc &rays, int64_t ray0, int n, const Grid &grid, const int64_t *ptr,
                            int64_t *col, float *val, cudaStream_t s)
{
    const int block = 128;
    csr_fill_kernel<<<(unsigned)((n + block - 1) / block), block, 0, s>>>(rays, ray0, n, grid, ptr, col, val);
    return cudaGetLastError();
}

}  // namespace xr
