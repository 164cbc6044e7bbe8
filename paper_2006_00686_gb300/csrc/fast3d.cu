// Fast path for single images (3D scans, and 2D scans outside the batched quad-plane
// path) and for persistent launches over uneven problems: one thread per ray, the
// crossing-order walk, and a second copy of the image with y fastest.
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
#include <algorithm>

#include "xray_rays.cuh"

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

// Thread -> ray.  View-major (mode 0): thread t is ray t ([view][row][col]).  Row-major
// (mode 1): threads run over (row, view, col), so the rays in flight at one time are one
// detector row in many views; in a circular cone scan those rays cross one slab of z, which
// stays in L2 while every view passes through it.  Column-major (mode 2): threads run over
// (view, col, row), so a warp holds 32 neighbouring rows of one detector column; in a cone
// or helical scan those rays share the vertical plane through the source and the column and
// sit at neighbouring heights, so with the volume stored z fastest they touch neighbouring
// words.  Row-blocked (mode 3): threads run over (block of 32 rows, view, col, row in the
// block): warps as in mode 2, and the rays in flight are one block of rows in every view,
// which in a circular cone cross one slab of z (the L2 locality of mode 1).  Threads past the
// last row of a partial block get -1.
constexpr int kRowBlock = 32;

struct RayOrder {
    int mode;
    int n_cols, n_views, n_rows;
    __device__ __forceinline__ int ray(int t) const
    {
        if (mode == 0) return t;
        if (mode == 1) {
            const int col = t % n_cols, rest = t / n_cols;
            const int view = rest % n_views, row = rest / n_views;
            return (view * n_rows + row) * n_cols + col;
        }
        if (mode == 2) {
            const int row = t % n_rows, rest = t / n_rows;
            const int col = rest % n_cols, view = rest / n_cols;
            return (view * n_rows + row) * n_cols + col;
        }
        const int rib = t % kRowBlock, rest = t / kRowBlock;
        const int col = rest % n_cols, rest2 = rest / n_cols;
        const int view = rest2 % n_views, row = (rest2 / n_views) * kRowBlock + rib;
        return row < n_rows ? (view * n_rows + row) * n_cols + col : -1;
    }
};

// Forward sum of one ray; imgT may be NULL (then every ray reads img).  SKIP: an axis the
// ray does not cross (w = 0), left out of every step, or 0.
template <int U, int SKIP>
__device__ __forceinline__ float fwd_ray_s(const RayRec &rr, int nx, int ny, int nz, const float *__restrict__ base,
                                           int sx, int sy, int sz, int *err)
{
    Dda<int> D;
    float acc = 0.f;
    if (dda_setup<int>(rr, nx, ny, nz, sx, sy, sz, D)) {
        // U voxels generated ahead, then their U loads issued together
        for (int g = dda_max_steps(nx, ny, nz) / U + 1; g > 0 && D.tcur < D.tout; --g) {
            int off[U];
            float l[U];
#pragma unroll
            for (int u = 0; u < U; ++u) dda_step_t<SKIP>(D, off[u], l[u]);
            float v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = l[u] > 0.f ? __ldg(base + off[u]) : 0.f;
#pragma unroll
            for (int u = 0; u < U; ++u) acc = __fmaf_rn(v[u], l[u], acc);  // + 0 where l == 0
        }
        if (err && D.tcur < D.tout) atomicOr(err, XR_DEVERR_WALK_BOUND);
    }
    return acc;
}

template <int U, int SKIP>
__device__ __forceinline__ float fwd_ray_t(const RayRec &rr, int nx, int ny, int nz, const float *__restrict__ img,
                                           const float *__restrict__ imgT, int *err)
{
    const bool tr = imgT != nullptr && leans_x(rr);
    return fwd_ray_s<U, SKIP>(rr, nx, ny, nz, tr ? imgT : img, tr ? ny : 1, tr ? 1 : nx, nx * ny, err);
}

// Rays of 2D scans and of single-tilt-axis scans keep one index fixed: their walk leaves
// that axis out (the same voxels and lengths, fewer instructions per step).
template <int U>
__device__ __forceinline__ float fwd_ray(const RayRec &rr, int nx, int ny, int nz, const float *__restrict__ img,
                                         const float *__restrict__ imgT, int *err = nullptr)
{
    if (rr.w2 == 0.f) return fwd_ray_t<U, 2>(rr, nx, ny, nz, img, imgT, err);
    if (rr.w1 == 0.f) return fwd_ray_t<U, 1>(rr, nx, ny, nz, img, imgT, err);
    return fwd_ray_t<U, 0>(rr, nx, ny, nz, img, imgT, err);
}

// Adjoint of one ray: one RED per voxel.  As in the forward, U voxels are generated ahead
// and their U REDs issued back to back from separate registers.  accT may be NULL.
template <int U, int SKIP>
__device__ __forceinline__ void scatter_ray_s(const RayRec &rr, float g, int nx, int ny, int nz,
                                              float *__restrict__ base, int sx, int sy, int sz, int *err)
{
    Dda<int> D;
    if (!dda_setup<int>(rr, nx, ny, nz, sx, sy, sz, D)) return;
    for (int k = dda_max_steps(nx, ny, nz) / U + 1; k > 0 && D.tcur < D.tout; --k) {
        int off[U];
        float l[U];
#pragma unroll
        for (int u = 0; u < U; ++u) dda_step_t<SKIP>(D, off[u], l[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (l[u] > 0.f) red_add(base + off[u], __fmul_rn(g, l[u]));
    }
    if (err && D.tcur < D.tout) atomicOr(err, XR_DEVERR_WALK_BOUND);
}

template <int U, int SKIP>
__device__ __forceinline__ void scatter_ray_t(const RayRec &rr, float g, int nx, int ny, int nz,
                                              float *__restrict__ out, float *__restrict__ accT, int *err)
{
    const bool tr = accT != nullptr && leans_x(rr);
    scatter_ray_s<U, SKIP>(rr, g, nx, ny, nz, tr ? accT : out, tr ? ny : 1, tr ? 1 : nx, nx * ny, err);
}

template <int U>
__device__ __forceinline__ void scatter_ray(const RayRec &rr, float g, int nx, int ny, int nz, float *__restrict__ out,
                                            float *__restrict__ accT, int *err = nullptr)
{
    if (rr.w2 == 0.f) scatter_ray_t<U, 2>(rr, g, nx, ny, nz, out, accT, err);
    else if (rr.w1 == 0.f) scatter_ray_t<U, 1>(rr, g, nx, ny, nz, out, accT, err);
    else scatter_ray_t<U, 0>(rr, g, nx, ny, nz, out, accT, err);
}

template <int U>
__global__ void __launch_bounds__(256) fwd3d_kernel(RaySrc rays, int n_rays, RayOrder ord,
                                                    int nx, int ny, int nz, const float *__restrict__ img,
                                                    const float *__restrict__ imgT, float *__restrict__ sino, int *err)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // no wrap near 2^31
    if (t >= n_rays) return;
    const int r = ord.ray((int)t);  // t < n_rays < 2^31
    sino[r] = fwd_ray<U>(rays[r], nx, ny, nz, img, imgT, err);
}

template <int U>
__global__ void __launch_bounds__(256) scatter3d_kernel(RaySrc rays, int n_rays, RayOrder ord,
                                                        int nx, int ny, int nz, const float *__restrict__ sino,
                                                        float *__restrict__ out, float *__restrict__ accT, int *err)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // no wrap near 2^31
    if (t >= n_rays) return;
    const int r = ord.ray((int)t);  // t < n_rays < 2^31
    const float g = __ldg(sino + r);
    if (g != 0.f) scatter_ray<U>(rays[r], g, nx, ny, nz, out, accT, err);
}

// The same walks on a z-fastest copy [y][x][z] (strides nz, nx * nz, 1): the column-major
// ray order's layout.
template <int U>
__global__ void __launch_bounds__(256) fwd3dz_kernel(RaySrc rays, int n_threads, RayOrder ord,
                                                     int nx, int ny, int nz, const float *__restrict__ imgZ,
                                                     float *__restrict__ sino, int *err)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // no wrap near 2^31
    if (t >= n_threads) return;
    const int r = ord.ray((int)t);  // t < n_threads < 2^31
    if (r < 0) return;
    const RayRec rr = rays[r];
    const int sx = nz, sy = nx * nz;
    float v;
    if (rr.w2 == 0.f) v = fwd_ray_s<U, 2>(rr, nx, ny, nz, imgZ, sx, sy, 1, err);
    else if (rr.w1 == 0.f) v = fwd_ray_s<U, 1>(rr, nx, ny, nz, imgZ, sx, sy, 1, err);
    else v = fwd_ray_s<U, 0>(rr, nx, ny, nz, imgZ, sx, sy, 1, err);
    sino[r] = v;
}

template <int U>
__global__ void __launch_bounds__(256) scatter3dz_kernel(RaySrc rays, int n_threads,
                                                         RayOrder ord, int nx, int ny, int nz,
                                                         const float *__restrict__ sino, float *__restrict__ accZ,
                                                         int *err)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // no wrap near 2^31
    if (t >= n_threads) return;
    const int r = ord.ray((int)t);  // t < n_threads < 2^31
    if (r < 0) return;
    const float g = __ldg(sino + r);
    if (g == 0.f) return;
    const RayRec rr = rays[r];
    const int sx = nz, sy = nx * nz;
    if (rr.w2 == 0.f) scatter_ray_s<U, 2>(rr, g, nx, ny, nz, accZ, sx, sy, 1, err);
    else if (rr.w1 == 0.f) scatter_ray_s<U, 1>(rr, g, nx, ny, nz, accZ, sx, sy, 1, err);
    else scatter_ray_s<U, 0>(rr, g, nx, ny, nz, accZ, sx, sy, 1, err);
}

// out[p][k] = in[k][p] for a [rows][cols] matrix (tiles of 32 x 32 through shared memory):
// [z][y x] -> [y x][z] with rows = nz, and back with rows = nx * ny.
__global__ void __launch_bounds__(256) transpose_rc_kernel(const float *__restrict__ in, float *__restrict__ out,
                                                           int64_t rows, int64_t cols)
{
    __shared__ float tile[TT][TT + 1];
    const int64_t c0 = (int64_t)blockIdx.x * TT;
    const int64_t row_tiles = (rows + TT - 1) / TT;
    for (int64_t ty = blockIdx.y; ty < row_tiles; ty += gridDim.y) {  // gridDim.y is capped
        const int64_t r0 = ty * TT;
        for (int dr = threadIdx.y; dr < TT; dr += blockDim.y) {
            const int64_t r = r0 + dr, c = c0 + threadIdx.x;
            if (r < rows && c < cols) tile[dr][threadIdx.x] = in[r * cols + c];
        }
        __syncthreads();
        for (int dc = threadIdx.y; dc < TT; dc += blockDim.y) {
            const int64_t c = c0 + dc, r = r0 + threadIdx.x;
            if (r < rows && c < cols) out[c * rows + r] = tile[threadIdx.x][dc];
        }
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------------------
// Work lists of uneven problems: every warp takes work items of `tile` consecutive rays from
// one atomic counter until none is left.  A warp never waits for another warp (no CTA
// barrier), so a long ray holds up only its own warp.  The per-problem copies and
// accumulators are prepared and folded back by the item kernels below, one launch each for
// the whole list (blockIdx.y = problem, grid-stride over its 32 x 32 tiles).
// ---------------------------------------------------------------------------------------

// CTAs per SM the adjoint's registers must allow: its REDs are issued and not waited for,
// so more resident warps keep more of them in flight
#ifndef XR_BATCH_ADJ_MIN_BLOCKS
#define XR_BATCH_ADJ_MIN_BLOCKS 6
#endif

template <int U, bool ADJ>
__global__ void __launch_bounds__(256, ADJ ? XR_BATCH_ADJ_MIN_BLOCKS : 1) batched_dda_kernel(const BatchItem *__restrict__ items, int n_items,
                                                          int64_t n_tiles, int tile,
                                                          unsigned long long *__restrict__ counter)
{
    const int lane = threadIdx.x & 31;
    for (;;) {
        unsigned long long t = 0;
        if (lane == 0) t = atomicAdd(counter, 1ull);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= (unsigned long long)n_tiles) break;
        const BatchItem &P = items[find_item(items, n_items, (int64_t)t)];
        const int64_t first = ((int64_t)t - P.tile_begin) * tile;
        for (int q = lane; q < tile; q += 32) {
            const int64_t r = first + q;
            if (r >= P.n_rays) break;
            if (!ADJ) {
                P.sino[r] = fwd_ray<U>((*P.src)[r], P.nx, P.ny, P.nz, P.img, P.aux);
            } else {
                const float g = __ldg(P.sino + r);
                if (g != 0.f) scatter_ray<U>((*P.src)[r], g, P.nx, P.ny, P.nz, const_cast<float *>(P.img), P.aux);
            }
        }
    }
}

// The same work list as one ordinary launch: CTA b takes work item b (tile = CTA threads).
template <int U, bool ADJ>
__global__ void __launch_bounds__(1024) flat_dda_kernel(const BatchItem *__restrict__ items, int n_items, int tile)
{
    const int64_t t = blockIdx.x;
    const BatchItem &P = items[find_item(items, n_items, t)];
    const int64_t r = (t - P.tile_begin) * tile + threadIdx.x;
    if (r >= P.n_rays) return;
    if (!ADJ) {
        P.sino[r] = fwd_ray<U>((*P.src)[r], P.nx, P.ny, P.nz, P.img, P.aux);
    } else {
        const float g = __ldg(P.sino + r);
        if (g != 0.f) scatter_ray<U>((*P.src)[r], g, P.nx, P.ny, P.nz, const_cast<float *>(P.img), P.aux);
    }
}

__device__ __forceinline__ int item_tiles(const BatchItem &P) { return ((P.nx + TT - 1) / TT) * ((P.ny + TT - 1) / TT) * P.nz; }

// aux = [z][x][y] copy of img, per item
__global__ void __launch_bounds__(256) transpose_items_kernel(const BatchItem *__restrict__ items)
{
    __shared__ float tile[TT][TT + 1];
    const BatchItem &P = items[blockIdx.y];
    if (!P.aux) return;
    const int ntx = (P.nx + TT - 1) / TT, nty = (P.ny + TT - 1) / TT;
    for (int b = blockIdx.x; b < item_tiles(P); b += gridDim.x) {
        const int x0 = (b % ntx) * TT, y0 = ((b / ntx) % nty) * TT, z = b / (ntx * nty);
        const size_t zoff = (size_t)z * P.nx * P.ny;
        __syncthreads();
        for (int dy = threadIdx.y; dy < TT; dy += blockDim.y) {
            const int x = x0 + threadIdx.x, y = y0 + dy;
            if (x < P.nx && y < P.ny) tile[dy][threadIdx.x] = P.img[zoff + (size_t)y * P.nx + x];
        }
        __syncthreads();
        for (int dx = threadIdx.y; dx < TT; dx += blockDim.y) {
            const int y = y0 + threadIdx.x, x = x0 + dx;
            if (x < P.nx && y < P.ny) P.aux[zoff + (size_t)x * P.ny + y] = tile[threadIdx.x][dx];
        }
    }
}

// img = 0 and aux = 0, per item
__global__ void __launch_bounds__(256) zero_items_kernel(const BatchItem *__restrict__ items)
{
    const BatchItem &P = items[blockIdx.y];
    const int64_t n = (int64_t)P.nx * P.ny * P.nz;
    float *img = const_cast<float *>(P.img);
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x) {
        img[u] = 0.f;
        if (P.aux) P.aux[u] = 0.f;
    }
}

// img += [z][y][x] view of aux, per item
__global__ void __launch_bounds__(256) add_transposed_items_kernel(const BatchItem *__restrict__ items)
{
    __shared__ float tile[TT][TT + 1];
    const BatchItem &P = items[blockIdx.y];
    if (!P.aux) return;
    float *img = const_cast<float *>(P.img);
    const int ntx = (P.nx + TT - 1) / TT, nty = (P.ny + TT - 1) / TT;
    for (int b = blockIdx.x; b < item_tiles(P); b += gridDim.x) {
        const int x0 = (b % ntx) * TT, y0 = ((b / ntx) % nty) * TT, z = b / (ntx * nty);
        const size_t zoff = (size_t)z * P.nx * P.ny;
        __syncthreads();
        for (int dx = threadIdx.y; dx < TT; dx += blockDim.y) {
            const int y = y0 + threadIdx.x, x = x0 + dx;
            if (x < P.nx && y < P.ny) tile[dx][threadIdx.x] = P.aux[zoff + (size_t)x * P.ny + y];
        }
        __syncthreads();
        for (int dy = threadIdx.y; dy < TT; dy += blockDim.y) {
            const int x = x0 + threadIdx.x, y = y0 + dy;
            if (x < P.nx && y < P.ny) img[zoff + (size_t)y * P.nx + x] += tile[threadIdx.x][dy];
        }
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

// Forward and the adjoint of its result in one pass per (ray, image): the single-image walks
// on the caller's layout (no copies), y written to sino, then y * l spread into out (zeroed
// by the caller).  blockIdx.y: the image.
__global__ void __launch_bounds__(256) fwd_adj_kernel(RaySrc rays, int n_rays, int nx, int ny, int nz,
                                                      const float *__restrict__ img, float *__restrict__ sino,
                                                      float *__restrict__ out, int64_t n_units, int *err)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // no wrap near 2^31
    if (t >= n_rays) return;
    const int r = (int)t;
    const int64_t b = blockIdx.y;
    const RayRec rr = rays[r];
    const float v = fwd_ray<kFwdAhead>(rr, nx, ny, nz, img + b * n_units, nullptr, err);
    sino[b * n_rays + r] = v;
    if (v != 0.f) scatter_ray<kAdjAhead>(rr, v, nx, ny, nz, out + b * n_units, nullptr, err);
}

// The walks of fwd_ray_s / scatter_ray_s restricted to the box [lo, hi) of the grid (the grid's
// own planes, so every voxel keeps its length); base points at the box's first voxel.
template <int U, int SKIP>
__device__ __forceinline__ float fwd_box_s(const RayRec &rr, const int3 lo, const int3 hi, int nx, int ny, int nz,
                                           const float *__restrict__ base, int sx, int sy, int sz)
{
    Dda<int> D;
    float acc = 0.f;
    if (dda_setup_box<int>(rr, lo.x, hi.x, lo.y, hi.y, lo.z, hi.z, sx, sy, sz, D)) {
        for (int g = dda_max_steps(nx, ny, nz) / U + 1; g > 0 && D.tcur < D.tout; --g) {
            int off[U];
            float l[U];
#pragma unroll
            for (int u = 0; u < U; ++u) dda_step_t<SKIP>(D, off[u], l[u]);
            float v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = l[u] > 0.f ? __ldg(base + off[u]) : 0.f;
#pragma unroll
            for (int u = 0; u < U; ++u) acc = __fmaf_rn(v[u], l[u], acc);
        }
    }
    return acc;
}

template <int U, int SKIP>
__device__ __forceinline__ void scatter_box_s(const RayRec &rr, float g, const int3 lo, const int3 hi, int nx, int ny,
                                              int nz, float *__restrict__ base, int sx, int sy, int sz)
{
    Dda<int> D;
    if (!dda_setup_box<int>(rr, lo.x, hi.x, lo.y, hi.y, lo.z, hi.z, sx, sy, sz, D)) return;
    for (int k = dda_max_steps(nx, ny, nz) / U + 1; k > 0 && D.tcur < D.tout; --k) {
        int off[U];
        float l[U];
#pragma unroll
        for (int u = 0; u < U; ++u) dda_step_t<SKIP>(D, off[u], l[u]);
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (l[u] > 0.f) red_add(base + off[u], __fmul_rn(g, l[u]));
    }
}

// fwd_adj_kernel with two threads per (ray, image) for problems that leave most of the GPU idle:
// the threads of a pair (neighbouring lanes) take the two halves of the grid on either side of
// the middle plane of the ray's driving axis (its largest |w|); their sums add up to the ray's
// (one shuffle, reached by every lane of the warp outside the walks' branches), and each spreads
// that sum over its own half.
__global__ void __launch_bounds__(256) fwd_adj_split_kernel(RaySrc rays, int n_rays, int nx, int ny, int nz,
                                                            const float *__restrict__ img, float *__restrict__ sino,
                                                            float *__restrict__ out, int64_t n_units)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t r = t >> 1;
    const int h = (int)(t & 1);
    const bool valid = r < n_rays;  // the same for both threads of a pair
    if (!__any_sync(0xffffffffu, valid)) return;  // the whole warp
    const int64_t b = blockIdx.y;
    RayRec rr{};  // an invalid lane's zero record crosses nothing
    if (valid) rr = rays[r];
    const float a0 = fabsf(rr.w0), a1 = fabsf(rr.w1), a2 = fabsf(rr.w2);
    const int ax = (a0 >= a1 && a0 >= a2) ? 0 : (a1 >= a2 ? 1 : 2);
    int3 lo = make_int3(0, 0, 0), hi = make_int3(nx, ny, nz);
    const int mid = (ax == 0 ? nx : (ax == 1 ? ny : nz)) / 2;
    if (ax == 0) (h ? lo.x : hi.x) = mid;
    else if (ax == 1) (h ? lo.y : hi.y) = mid;
    else (h ? lo.z : hi.z) = mid;
    const int64_t corner = lo.x + (int64_t)lo.y * nx + (int64_t)lo.z * nx * ny;
    const float *im = img + b * n_units + corner;
    float *o = out + b * n_units + corner;
    const int sy = nx, sz = nx * ny;
    float part;
    if (rr.w2 == 0.f) part = fwd_box_s<kFwdAhead, 2>(rr, lo, hi, nx, ny, nz, im, 1, sy, sz);
    else if (rr.w1 == 0.f) part = fwd_box_s<kFwdAhead, 1>(rr, lo, hi, nx, ny, nz, im, 1, sy, sz);
    else part = fwd_box_s<kFwdAhead, 0>(rr, lo, hi, nx, ny, nz, im, 1, sy, sz);
    const float v = part + __shfl_xor_sync(0xffffffffu, part, 1);
    if (!valid) return;
    if (h == 0) sino[b * n_rays + r] = v;
    if (v == 0.f) return;
    if (rr.w2 == 0.f) scatter_box_s<kAdjAhead, 2>(rr, v, lo, hi, nx, ny, nz, o, 1, sy, sz);
    else if (rr.w1 == 0.f) scatter_box_s<kAdjAhead, 1>(rr, v, lo, hi, nx, ny, nz, o, 1, sy, sz);
    else scatter_box_s<kAdjAhead, 0>(rr, v, lo, hi, nx, ny, nz, o, 1, sy, sz);
}

}  // namespace

cudaError_t launch_fwd_adj(const RaySrc &rays, const GeoParams &g, int64_t n_rays, const float *img, float *sino,
                           float *out, int batch, int block, int *err, cudaStream_t s)
{
    const int64_t n_units = (int64_t)g.nx * g.ny * g.nz;
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (n_rays * batch <= 256 * (int64_t)sms && 2 * n_rays < ((int64_t)1 << 31)) {
        // a problem this small leaves the GPU mostly idle: two threads per ray halve each
        // thread's walk
        const dim3 grid((unsigned)((2 * n_rays + block - 1) / block), (unsigned)batch);
        fwd_adj_split_kernel<<<grid, block, 0, s>>>(rays, (int)n_rays, g.nx, g.ny, g.nz, img, sino, out, n_units);
        return cudaGetLastError();
    }
    const dim3 grid((unsigned)((n_rays + block - 1) / block), (unsigned)batch);
    fwd_adj_kernel<<<grid, block, 0, s>>>(rays, (int)n_rays, g.nx, g.ny, g.nz, img, sino, out, n_units, err);
    return cudaGetLastError();
}

int batched_ctas_per_sm(int block, int adjoint)
{
    int n = 0;
    if (adjoint)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batched_dda_kernel<kAdjAhead, true>, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batched_dda_kernel<kFwdAhead, false>, block, 0);
    return n > 0 ? n : 1;
}

cudaError_t launch_batched(const BatchItem *items, int n_items, int64_t n_tiles, int tile,
                           unsigned long long *counter, int adjoint, int with_aux, int grid_ctas, int block,
                           cudaStream_t s, bool lock2d)
{
    const dim3 per_item(256, (unsigned)n_items);
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
#ifndef XR_BATCH_FLAT
#define XR_BATCH_FLAT 0
#endif
    const bool flat = !lock2d && (XR_BATCH_FLAT & (adjoint ? 2 : 1)) && tile <= 1024;
    if (!adjoint) {
        if (with_aux) transpose_items_kernel<<<per_item, dim3(TT, 8), 0, s>>>(items);
        if (flat)
            flat_dda_kernel<kFwdAhead, false><<<(unsigned)n_tiles, tile, 0, s>>>(items, n_items, tile);
        else
            batched_dda_kernel<kFwdAhead, false><<<grid_ctas, block, 0, s>>>(items, n_items, n_tiles, tile, counter);
        return cudaGetLastError();
    }
    zero_items_kernel<<<per_item, 256, 0, s>>>(items);
    if (lock2d) {
        e = launch_batch2d_adjoint(items, n_items, n_tiles, tile, counter, grid_ctas, block, s);
        if (e != cudaSuccess) return e;
    } else if (flat)
        flat_dda_kernel<kAdjAhead, true><<<(unsigned)n_tiles, tile, 0, s>>>(items, n_items, tile);
    else
        batched_dda_kernel<kAdjAhead, true><<<grid_ctas, block, 0, s>>>(items, n_items, n_tiles, tile, counter);
    if (with_aux) add_transposed_items_kernel<<<per_item, dim3(TT, 8), 0, s>>>(items);
    return cudaGetLastError();
}

cudaError_t launch_batched_items(const BatchItem *items, int n_items, int64_t n_tiles, int tile,
                                 unsigned long long *counter, int grid_ctas, int block, cudaStream_t s,
                                 bool)
{
    batched_dda_kernel<kFwdAhead, false><<<grid_ctas, block, 0, s>>>(items, n_items, n_tiles, tile, counter);
    return cudaGetLastError();
}

cudaError_t launch_transpose_xy(const float *in, float *out, int nx, int ny, int nz, cudaStream_t s)
{
    const dim3 grid((unsigned)((nx + TT - 1) / TT), (unsigned)((ny + TT - 1) / TT), (unsigned)nz);
    transpose_xy_kernel<<<grid, dim3(TT, 8), 0, s>>>(in, out, nx, ny);
    return cudaGetLastError();
}

static RayOrder make_order(const GeoParams &g, int mode)
{
    return RayOrder{mode, g.n_cols, g.n_views, g.n_rows};
}

// Threads of a launch in the given order (mode 3 pads the rows to whole blocks).
static int64_t order_threads(const GeoParams &g, int64_t n_rays, int mode)
{
    if (mode != 3) return n_rays;
    return (int64_t)((g.n_rows + kRowBlock - 1) / kRowBlock) * kRowBlock * g.n_cols * g.n_views;
}

// Thread ids are 32-bit: a row-blocked launch whose padding would pass 2^31 threads takes the
// plain column-major order (the same rays, the same z-fastest layout).
static int fit_order(const GeoParams &g, int64_t n_rays, int mode)
{
    return (mode == 3 && order_threads(g, n_rays, 3) >= ((int64_t)1 << 31)) ? 2 : mode;
}

static cudaError_t launch_transpose_rc(const float *in, float *out, int64_t rows, int64_t cols, cudaStream_t s)
{
    const dim3 grid((unsigned)((cols + TT - 1) / TT), (unsigned)std::min<int64_t>((rows + TT - 1) / TT, 65535));
    transpose_rc_kernel<<<grid, dim3(TT, 8), 0, s>>>(in, out, rows, cols);
    return cudaGetLastError();
}

cudaError_t launch_project3d(const RaySrc &rays, const GeoParams &g, int64_t n_rays, int order, const float *img,
                             float *ws, float *sino, int block, int *err, cudaStream_t s)
{
    order = fit_order(g, n_rays, order);
    const unsigned blocks = (unsigned)((n_rays + block - 1) / block);
    cudaError_t e;
    if (order >= 2) {
        // z-fastest copy, then the column-major (or row-blocked) walk
        e = launch_transpose_rc(img, ws, g.nz, (int64_t)g.nx * g.ny, s);
        if (e != cudaSuccess) return e;
        const int64_t nt = order_threads(g, n_rays, order);
        fwd3dz_kernel<kFwdAhead><<<(unsigned)((nt + block - 1) / block), block, 0, s>>>(
            rays, (int)nt, make_order(g, order), g.nx, g.ny, g.nz, ws, sino, err);
        return cudaGetLastError();
    }
    e = launch_transpose_xy(img, ws, g.nx, g.ny, g.nz, s);
    if (e != cudaSuccess) return e;
    fwd3d_kernel<kFwdAhead><<<blocks, block, 0, s>>>(rays, (int)n_rays, make_order(g, order), g.nx, g.ny, g.nz,
                                                     img, ws, sino, err);
    return cudaGetLastError();
}

cudaError_t launch_scatter3d(const RaySrc &rays, const GeoParams &g, int64_t n_rays, int order,
                             const float *sino, float *out, float *accT, int block, int *err, cudaStream_t s)
{
    order = fit_order(g, n_rays, order);
    const int nx = g.nx, ny = g.ny, nz = g.nz;
    const size_t bytes = (size_t)nx * ny * nz * sizeof(float);
    if (order >= 2) {
        // one z-fastest accumulator, transposed into out (every element written)
        cudaError_t e = cudaMemsetAsync(accT, 0, bytes, s);
        if (e != cudaSuccess) return e;
        const int64_t nt = order_threads(g, n_rays, order);
        scatter3dz_kernel<kAdjAhead><<<(unsigned)((nt + block - 1) / block), block, 0, s>>>(
            rays, (int)nt, make_order(g, order), nx, ny, nz, sino, accT, err);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return launch_transpose_rc(accT, out, (int64_t)nx * ny, nz, s);
    }
    cudaError_t e = cudaMemsetAsync(out, 0, bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(accT, 0, bytes, s);
    if (e != cudaSuccess) return e;
    const unsigned blocks = (unsigned)((n_rays + block - 1) / block);
    scatter3d_kernel<kAdjAhead><<<blocks, block, 0, s>>>(rays, (int)n_rays, make_order(g, order), nx, ny, nz, sino, out,
                                              accT, err);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((nx + TT - 1) / TT), (unsigned)((ny + TT - 1) / TT), (unsigned)nz);
    add_transposed_kernel<<<grid, dim3(TT, 8), 0, s>>>(accT, out, nx, ny);
    return cudaGetLastError();
}

}  // namespace xr
