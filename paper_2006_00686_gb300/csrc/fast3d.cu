// Fast path for 3D scans: one thread per ray, the crossing-order walk, and a second copy
// of the volume with y fastest.
//
// A warp holds 32 neighbouring detector columns of one row; their rays run side by side,
// spread across the horizontal direction perpendicular to the beam.  When the beam runs
// mostly along x (|w_x| > |w_y|) that spread is along y, so in the [z][y][x] layout the 32
// lanes touch 32 different rows of the volume at every step; in a [z][x][y] copy they
// touch neighbouring words.  Each ray therefore reads the copy whose fastest axis is the
// one its warp is spread along:  x-leaning rays read the [z][x][y] copy, the others the
// caller's image.  The adjoint scatters the same way into two accumulators and adds the
// transposed one back.
//
// The forward walk generates U voxels (offset, length) ahead, then issues their U loads
// together, so every thread keeps U independent loads in flight instead of one.
#include "xray_internal.h"

namespace xr {

namespace {

constexpr int TT = 32;  // transpose tile

// out[z][x][y] = in[z][y][x]
__global__ void __launch_bounds__(256) transpose_xy_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                           int nx, int ny)
{
    __shared__ float tile[TT][TT + 1];
    const int x0 = blockIdx.x * TT, y0 = blockIdx.y * TT;
    const size_t zoff = (size_t)blockIdx.z * (size_t)nx * (size_t)ny;
    for (int dy = threadIdx.y; dy < TT; dy += blockDim.y) {
        const int x = x0 + threadIdx.x, y = y0 + dy;
        if (x < nx && y < ny) tile[dy][threadIdx.x] = in[zoff + (size_t)y * nx + x];
    }
    __syncthreads();
    for (int dx = threadIdx.y; dx < TT; dx += blockDim.y) {
        const int y = y0 + threadIdx.x, x = x0 + dx;
        if (x < nx && y < ny) out[zoff + (size_t)x * ny + y] = tile[threadIdx.x][dx];
    }
}

// out[z][y][x] += accT[z][x][y]
__global__ void __launch_bounds__(256) add_transposed_kernel(const float *__restrict__ accT, float *__restrict__ out,
                                                             int nx, int ny)
{
    __shared__ float tile[TT][TT + 1];
    const int x0 = blockIdx.x * TT, y0 = blockIdx.y * TT;
    const size_t zoff = (size_t)blockIdx.z * (size_t)nx * (size_t)ny;
    for (int dx = threadIdx.y; dx < TT; dx += blockDim.y) {
        const int y = y0 + threadIdx.x, x = x0 + dx;
        if (x < nx && y < ny) tile[dx][threadIdx.x] = accT[zoff + (size_t)x * ny + y];
    }
    __syncthreads();
    for (int dy = threadIdx.y; dy < TT; dy += blockDim.y) {
        const int x = x0 + threadIdx.x, y = y0 + dy;
        if (x < nx && y < ny) out[zoff + (size_t)y * nx + x] += tile[threadIdx.x][dy];
    }
}

// The layout a ray reads: the [z][x][y] copy when it leans along x.
__device__ __forceinline__ bool leans_x(const RayRec &r) { return fabsf(r.w0) > fabsf(r.w1); }

// Thread -> ray.  View-major: thread t is ray t ([view][row][col]).  Row-major: threads run
// over (row, view, col), so the rays in flight at one time are one detector row in many
// views; in a circular cone scan those rays cross one slab of z, which stays in L2 while
// every view passes through it.
struct RayOrder {
    int row_major;
    int n_cols, n_views, n_rows;
    __device__ __forceinline__ int ray(int t) const
    {
        if (!row_major) return t;
        const int col = t % n_cols, rest = t / n_cols;
        const int view = rest % n_views, row = rest / n_views;
        return (view * n_rows + row) * n_cols + col;
    }
};

template <int U>
__global__ void __launch_bounds__(256) fwd3d_kernel(const RayRec *__restrict__ rays, int n_rays, RayOrder ord,
                                                    int nx, int ny, int nz, const float *__restrict__ img,
                                                    const float *__restrict__ imgT, float *__restrict__ sino)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_rays) return;
    const int r = ord.ray(t);
    const RayRec rr = rays[r];
    const bool tr = leans_x(rr);
    const float *__restrict__ base = tr ? imgT : img;
    Dda<int> D;
    float acc = 0.f;
    if (dda_setup<int>(rr, nx, ny, nz, tr ? ny : 1, tr ? 1 : nx, nx * ny, D)) {
        // U voxels generated ahead, then their U loads issued together
        for (int g = dda_max_steps(nx, ny, nz) / U + 1; g > 0 && D.tcur < D.tout; --g) {
            int off[U];
            float l[U];
#pragma unroll
            for (int u = 0; u < U; ++u) dda_step(D, off[u], l[u]);
            float v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = l[u] > 0.f ? __ldg(base + off[u]) : 0.f;
#pragma unroll
            for (int u = 0; u < U; ++u) acc = __fmaf_rn(v[u], l[u], acc);  // + 0 where l == 0
        }
    }
    sino[r] = acc;
}

// Adjoint: one RED per (ray, voxel).  As in the forward, U voxels are generated ahead and
// their U REDs issued back to back from separate registers, so a warp does not wait for
// one RED's operands to be taken before building the next.
template <int U>
__global__ void __launch_bounds__(256) scatter3d_kernel(const RayRec *__restrict__ rays, int n_rays, RayOrder ord,
                                                        int nx, int ny, int nz, const float *__restrict__ sino,
                                                        float *__restrict__ out, float *__restrict__ accT)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_rays) return;
    const int r = ord.ray(t);
    const float g = __ldg(sino + r);
    if (g == 0.f) return;
    const RayRec rr = rays[r];
    const bool tr = leans_x(rr);
    float *__restrict__ base = tr ? accT : out;
    Dda<int> D;
    if (!dda_setup<int>(rr, nx, ny, nz, tr ? ny : 1, tr ? 1 : nx, nx * ny, D)) return;
    for (int k = dda_max_steps(nx, ny, nz) / U + 1; k > 0 && D.tcur < D.tout; --k) {
        int off[U];
        float l[U];
#pragma unroll
        for (int u = 0; u < U; ++u) dda_step(D, off[u], l[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (l[u] > 0.f) atomicAdd(base + off[u], __fmul_rn(g, l[u]));
    }
}

// voxels generated ahead of their loads (forward) and REDs (adjoint)
#ifndef XR_FWD3D_AHEAD
#define XR_FWD3D_AHEAD 16
#endif
#ifndef XR_ADJ3D_AHEAD
#define XR_ADJ3D_AHEAD 4
#endif
constexpr int kFwdAhead = XR_FWD3D_AHEAD;
constexpr int kAdjAhead = XR_ADJ3D_AHEAD;

}  // namespace

cudaError_t launch_transpose_xy(const float *in, float *out, int nx, int ny, int nz, cudaStream_t s)
{
    const dim3 grid((unsigned)((nx + TT - 1) / TT), (unsigned)((ny + TT - 1) / TT), (unsigned)nz);
    transpose_xy_kernel<<<grid, dim3(TT, 8), 0, s>>>(in, out, nx, ny);
    return cudaGetLastError();
}

static RayOrder make_order(const GeoParams &g, int row_major)
{
    return RayOrder{row_major, g.n_cols, g.n_views, g.n_rows};
}

cudaError_t launch_project3d(const RayRec *rays, const GeoParams &g, int64_t n_rays, int row_major,
                             const float *img, const float *imgT, float *sino, int block, cudaStream_t s)
{
    const unsigned blocks = (unsigned)((n_rays + block - 1) / block);
    fwd3d_kernel<kFwdAhead><<<blocks, block, 0, s>>>(rays, (int)n_rays, make_order(g, row_major), g.nx, g.ny, g.nz,
                                                     img, imgT, sino);
    return cudaGetLastError();
}

cudaError_t launch_scatter3d(const RayRec *rays, const GeoParams &g, int64_t n_rays, int row_major,
                             const float *sino, float *out, float *accT, int block, cudaStream_t s)
{
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const size_t bytes = (size_t)nx * ny * nz * sizeof(float);
    cudaError_t e = cudaMemsetAsync(out, 0, bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(accT, 0, bytes, s);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((n_rays + block - 1) / block);
    scatter3d_kernel<kAdjAhead><<<blocks, block, 0, s>>>(rays, (int)n_rays, make_order(g, row_major), nx, ny, nz, sino, out,
                                              accT);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((nx + TT - 1) / TT), (unsigned)((ny + TT - 1) / TT), (unsigned)nz);
    add_transposed_kernel<<<grid, dim3(TT, 8), 0, s>>>(accT, out, nx, ny);
    return cudaGetLastError();
}

}  // namespace xr
