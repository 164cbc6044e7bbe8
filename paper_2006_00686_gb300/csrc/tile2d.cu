// Tiled forward and adjoint for 2D scans and batches of images (the batched fast path).
//
// A CTA owns a T x T tile of pixels for NB images, staged in shared memory, and walks
// every ray of a group of views through that tile only:
//   * forward: the tile is loaded once; each ray's walk inside the tile reads the NB
//     values of every unit it crosses from shared memory and accumulates f * l in
//     registers; the per-(ray, tile) partial sums are added into the sinogram with one
//     coalesced atomic per image (the sinogram is zeroed first);
//   * adjoint: the tile starts at zero; every unit a ray crosses receives g * l by shared-
//     memory atomics; the tile is then added into the image (zeroed first) once per view
//     group.
// Walk and lengths are those of xray_core.cuh (driving axis, minor rows per slab from the
// floor of the minor coordinate at the slab's planes, C_up - C_low of each unit), clipped
// to the tile's slabs and rows.
//
// Shared layout: tile[b][row][col] with a row pitch of T+1 floats, so that a warp's rays --
// neighbouring bins of one view, at neighbouring rows (x-driven) or columns (y-driven) of
// the same slab -- hit distinct banks in both cases.
//
// Work split: the four 64-thread quarters of a CTA take four views at a time; a quarter's
// threads take the bins whose rays can cross the tile (projection of the tile's corners).
#include "xray_internal.h"

namespace xr {

namespace {

constexpr int T = 32;         // tile side (pixels)
constexpr int PITCH = T + 1;  // shared row pitch (floats)
constexpr int TILE = T * PITCH;
constexpr float kMagicT = 12582912.0f;  // 1.5 * 2^23: one round-down add gives floor
constexpr int kMagicBitsT = 0x4B400000;

// Bins whose rays can cross the box [x0, x1] x [y0, y1] in view v (conservative).
template <int KIND>
__device__ __forceinline__ void footprint(const float *__restrict__ vt, int v, float x0, float x1, float y0,
                                          float y1, float u0, float inv_du, float half, float sdd, int ncols,
                                          int &c0, int &c1)
{
    const float4 e0 = __ldg(reinterpret_cast<const float4 *>(vt) + 2 * v);
    const float4 e1 = __ldg(reinterpret_cast<const float4 *>(vt) + 2 * v + 1);
    const float xc = 0.5f * (x0 + x1), yc = 0.5f * (y0 + y1), hx = 0.5f * (x1 - x0), hy = 0.5f * (y1 - y0);
    float umin, umax;
    if (KIND == XR_PAR2D) {
        const float uc = e0.x * xc + e0.y * yc, hw = fabsf(e0.x) * hx + fabsf(e0.y) * hy;
        umin = uc - hw;
        umax = uc + hw;
    } else {
        const float rx = xc - e0.x, ry = yc - e0.y;
        const float depth = rx * e0.z + ry * e0.w, lat = rx * e1.x + ry * e1.y;
        const float dd = fabsf(e0.z) * hx + fabsf(e0.w) * hy, dl = fabsf(e1.x) * hx + fabsf(e1.y) * hy;
        const float r1 = __fdividef(1.0f, depth - dd), r2 = __fdividef(1.0f, depth + dd);
        const float lo = lat - dl, hi = lat + dl;
        const float a = fminf(lo * r1, lo * r2), b = fmaxf(hi * r1, hi * r2);
        if (KIND == XR_FAN2D) {
            umin = sdd * a;
            umax = sdd * b;
        } else {
            umin = atanf(a);
            umax = atanf(b);
        }
    }
    // one bin of margin: the walk decides which rays really cross
    const float c0f = fminf(fmaxf((umin - u0) * inv_du + half - 1.0f, -1.0f), 4.0e6f);
    const float c1f = fminf(fmaxf((umax - u0) * inv_du + half + 1.0f, -1.0f), 4.0e6f);
    c0 = max(__float_as_int(__fadd_ru(c0f, kMagicT)) - kMagicBitsT, 0);
    c1 = min(__float_as_int(__fadd_rd(c1f, kMagicT)) - kMagicBitsT, ncols - 1);
}

// The walk of one ray clipped to the tile.  Calls op(shared_index, length) for every unit
// of the tile the ray crosses.
template <class OP>
__device__ __forceinline__ void walk_in_tile(const Walk &W, int i0, int j0, int ni, int nj, OP &op)
{
    // tile origin and extent along the walk's axes
    const int A0 = W.axA == 0 ? i0 : j0, nA = W.axA == 0 ? ni : nj;
    const int B0 = W.axB == 0 ? i0 : j0, nB = W.axB == 0 ? ni : nj;
    const int sA = W.axA == 0 ? 1 : PITCH, sB = W.axA == 0 ? PITCH : 1;
    const bool bact = W.nact >= 2;
    // rows relative to the tile: absolute row = oB + r (active B) or the fixed oB
    const int rowoff = W.oB - B0;
    const int mlo = max(W.mlo, A0), mhi = min(W.mhi, A0 + nA - 1);
    if (mlo > mhi) return;
    if (!bact && (unsigned)rowoff >= (unsigned)nB) return;
    const float invA = W.invA, bA = W.bA, wB = W.wB, fB = W.fB, invB = W.invB, bB = W.bB;
    float p = (float)(mlo - W.oA);
    float tcur = __fmaf_rn(p, invA, bA);
    float sc = __fadd_rd(__fmaf_rn(wB, tcur, fB), kMagicT);
    float jc = __fadd_rn(sc, -kMagicT);
    int mloc = (mlo - A0) * sA;
    for (int m = mlo; m <= mhi; ++m, mloc += sA) {
        p += 1.0f;
        const float tn = __fmaf_rn(p, invA, bA);
        const float sn = __fadd_rd(__fmaf_rn(wB, tn, fB), kMagicT);
        const float jn = __fadd_rn(sn, -kMagicT);
        const int rc = __float_as_int(sc) - kMagicBitsT + rowoff;
        const int rn = __float_as_int(sn) - kMagicBitsT + rowoff;
        if (fabsf(jn - jc) < 1.5f) {
            const bool cross = rn != rc;
            const float tc = __fmaf_rn(fmaxf(jc, jn), invB, bB);
            const float tcc = cross ? fminf(fmaxf(tc, fminf(tcur, tn)), fmaxf(tcur, tn)) : tn;
            const float lc = fabsf(__fsub_rn(tcc, tcur));
            const float ln = fabsf(__fsub_rn(tn, tcc));
            if ((unsigned)rc < (unsigned)nB && lc > 0.f) op(mloc + rc * sB, lc);
            if (cross && (unsigned)rn < (unsigned)nB && ln > 0.f) op(mloc + rn * sB, ln);
        } else {
            // crossing two rows in one slab (within rounding of a diagonal): per-candidate formula
            const float tlo = W.sgA ? tn : tcur, thi = W.sgA ? tcur : tn;
            const int jlo = (int)fminf(jc, jn), jhi = (int)fmaxf(jc, jn);
            for (int j = jlo; j <= jhi; ++j) {
                const float q = (float)j;
                const float tb0 = __fmaf_rn(q + (float)W.sgB, invB, bB);
                const float tb1 = __fmaf_rn(q + (float)(1 - W.sgB), invB, bB);
                const float l = __fsub_rn(fminf(thi, tb1), fmaxf(tlo, tb0));
                const int rl = j + rowoff;
                if ((unsigned)rl < (unsigned)nB && l > 0.f) op(mloc + rl * sB, l);
            }
        }
        tcur = tn;
        sc = sn;
        jc = jn;
    }
}

template <int NB>
struct TileGather {
    const float *tile;
    float acc[NB];
    __device__ __forceinline__ void operator()(int idx, float l)
    {
#pragma unroll
        for (int b = 0; b < NB; ++b) acc[b] = __fmaf_rn(tile[b * TILE + idx], l, acc[b]);
    }
};

template <int NB>
struct TileScatter {
    float *tile;
    float g[NB];
    __device__ __forceinline__ void operator()(int idx, float l)
    {
#pragma unroll
        for (int b = 0; b < NB; ++b) atomicAdd(tile + b * TILE + idx, g[b] * l);
    }
};

}  // namespace

// grid: (tiles_x * tiles_y, view groups, image chunks of NB); block 256; dynamic shared
// NB * TILE floats.  ADJ: adjoint (sino -> img) else forward (img -> sino).
template <int NB, int KIND, bool ADJ>
__global__ void __launch_bounds__(256, 3) tile2d_kernel(const RayRec *__restrict__ rays, GeoParams g,
                                                     const float *__restrict__ vt, int views_per_group,
                                                     const float *__restrict__ in, float *__restrict__ out,
                                                     int batch)
{
    extern __shared__ float tile[];
    const int tiles_x = (g.nx + T - 1) / T;
    const int ti = blockIdx.x % tiles_x, tj = blockIdx.x / tiles_x;
    const int i0 = ti * T, j0 = tj * T;
    const int ni = min(T, g.nx - i0), nj = min(T, g.ny - j0);
    const int b0 = blockIdx.z * NB;
    const int64_t n_pix = (int64_t)g.nx * g.ny;
    const int64_t n_rays = (int64_t)g.n_views * g.n_cols;

    // stage (forward) or clear (adjoint) the tile
    for (int e = threadIdx.x; e < NB * T * T; e += blockDim.x) {
        const int b = e / (T * T), rc = e % (T * T), r = rc / T, c = rc % T;
        float v = 0.f;
        if (!ADJ && r < nj && c < ni && b0 + b < batch)
            v = __ldg(in + (int64_t)(b0 + b) * n_pix + (int64_t)(j0 + r) * g.nx + i0 + c);
        tile[b * TILE + r * PITCH + c] = v;
    }
    __syncthreads();

    // tile box in world coordinates
    const float x0 = (float)(g.cx + (i0 - 0.5 * g.nx) * g.dx), x1 = x0 + (float)(ni * g.dx);
    const float y1 = (float)(g.cy + (0.5 * g.ny - j0) * g.dy), y0 = y1 - (float)(nj * g.dy);
    const float half = 0.5f * (float)(g.n_cols - 1);
    const float inv_du = (float)(1.0 / g.du), u0 = (float)g.u0, sdd = (float)g.sdd;
    const int quarter = threadIdx.x >> 6, qt = threadIdx.x & 63;
    const int vbeg = blockIdx.y * views_per_group;
    const int vend = min(g.n_views, vbeg + views_per_group);
    for (int v = vbeg + quarter; v < vend; v += 4) {
        int c0, c1;
        footprint<KIND>(vt, v, x0, x1, y0, y1, u0, inv_du, half, sdd, g.n_cols, c0, c1);
        for (int c = c0 + qt; c <= c1; c += 64) {
            const int64_t r = (int64_t)v * g.n_cols + c;
            Walk W;
            if (!walk_setup(rays[r], g.nx, g.ny, 1, 1, g.nx, n_pix, W)) continue;
            if (ADJ) {
                TileScatter<NB> op;
                op.tile = tile;
                bool any = false;
#pragma unroll
                for (int b = 0; b < NB; ++b) {
                    op.g[b] = (b0 + b < batch) ? __ldg(in + (int64_t)(b0 + b) * n_rays + r) : 0.f;
                    any |= op.g[b] != 0.f;
                }
                if (any) walk_in_tile(W, i0, j0, ni, nj, op);
            } else {
                TileGather<NB> op;
                op.tile = tile;
#pragma unroll
                for (int b = 0; b < NB; ++b) op.acc[b] = 0.f;
                walk_in_tile(W, i0, j0, ni, nj, op);
#pragma unroll
                for (int b = 0; b < NB; ++b)
                    if (b0 + b < batch && op.acc[b] != 0.f) atomicAdd(out + (int64_t)(b0 + b) * n_rays + r, op.acc[b]);
            }
        }
    }
    if (ADJ) {
        __syncthreads();
        for (int e = threadIdx.x; e < NB * T * T; e += blockDim.x) {
            const int b = e / (T * T), rc = e % (T * T), r = rc / T, c = rc % T;
            const float v = tile[b * TILE + r * PITCH + c];
            if (r < nj && c < ni && b0 + b < batch && v != 0.f)
                atomicAdd(out + (int64_t)(b0 + b) * n_pix + (int64_t)(j0 + r) * g.nx + i0 + c, v);
        }
    }
}

size_t tile2d_smem_bytes(int nb) { return (size_t)nb * TILE * sizeof(float); }

template <int NB, int KIND, bool ADJ>
static cudaError_t launch_tile_t(const RayRec *rays, const GeoParams &g, const float *vt, int groups,
                                 const float *in, float *out, int batch, cudaStream_t s)
{
    const size_t smem = tile2d_smem_bytes(NB);
    // opt in to more than 48 KiB of dynamic shared memory (cheap; done on every launch so
    // that it holds on whichever device is current)
    cudaError_t e = cudaFuncSetAttribute(tile2d_kernel<NB, KIND, ADJ>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    const int tiles = ((g.nx + T - 1) / T) * ((g.ny + T - 1) / T);
    const int vpg = (g.n_views + groups - 1) / groups;
    const dim3 grid((unsigned)tiles, (unsigned)groups, (unsigned)((batch + NB - 1) / NB));
    tile2d_kernel<NB, KIND, ADJ><<<grid, 256, smem, s>>>(rays, g, vt, vpg, in, out, batch);
    return cudaGetLastError();
}

template <int NB, bool ADJ>
static cudaError_t launch_tile_k(const RayRec *rays, const GeoParams &g, const float *vt, int groups,
                                 const float *in, float *out, int batch, cudaStream_t s)
{
    if (g.kind == XR_PAR2D) return launch_tile_t<NB, XR_PAR2D, ADJ>(rays, g, vt, groups, in, out, batch, s);
    if (g.kind == XR_FAN2D) return launch_tile_t<NB, XR_FAN2D, ADJ>(rays, g, vt, groups, in, out, batch, s);
    return launch_tile_t<NB, XR_FAN2D_ARC, ADJ>(rays, g, vt, groups, in, out, batch, s);
}

// Number of view groups: enough CTAs for about four waves of resident CTAs.
static int tile2d_groups(const GeoParams &g, int batch, int nb)
{
    int dev = 0, sms = 152;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int per_sm = nb >= 16 ? 3 : 6;
    const int tiles = ((g.nx + T - 1) / T) * ((g.ny + T - 1) / T) * ((batch + nb - 1) / nb);
    int groups = (4 * sms * per_sm + tiles - 1) / tiles;
    groups = max(1, min(groups, g.n_views / 4 > 0 ? g.n_views / 4 : 1));
    return groups;
}

cudaError_t launch_tile2d(const RayRec *rays, const GeoParams &g, const float *vt, const float *in, float *out,
                          int batch, int adjoint, cudaStream_t s)
{
    const int nb = batch >= 9 ? 16 : (batch >= 5 ? 8 : 4);
    // outputs are accumulated with atomics: clear them first
    const size_t out_elems = adjoint ? (size_t)g.nx * g.ny * batch : (size_t)g.n_views * g.n_cols * batch;
    cudaError_t e = cudaMemsetAsync(out, 0, out_elems * sizeof(float), s);
    if (e != cudaSuccess) return e;
    const int groups = tile2d_groups(g, batch, nb);
    if (adjoint) {
        if (nb == 16) return launch_tile_k<16, true>(rays, g, vt, groups, in, out, batch, s);
        if (nb == 8) return launch_tile_k<8, true>(rays, g, vt, groups, in, out, batch, s);
        return launch_tile_k<4, true>(rays, g, vt, groups, in, out, batch, s);
    }
    if (nb == 16) return launch_tile_k<16, false>(rays, g, vt, groups, in, out, batch, s);
    if (nb == 8) return launch_tile_k<8, false>(rays, g, vt, groups, in, out, batch, s);
    return launch_tile_k<4, false>(rays, g, vt, groups, in, out, batch, s);
}

}  // namespace xr
