// The forward and the adjoint of 2D problems with one image each (a single image of a 2D scan,
// or the problems of a batch plan), walked slab by slab.  The adjoint: 32 neighbouring rays per
// warp in lockstep, reduced into padded accumulator planes, one plane per driving axis (this
// part of the file).  The forward: one ray per thread on pair planes (the part further below).
//
// A ray driven along axis A (the axis with the largest index-space slope, Section 4.3) crosses
// at most one plane of the other axis B inside a slab [m, m + 1] of A: the pixels it meets
// there are rows j and j + 1 of column m, j = min of floor(u_B) at the slab's two planes (the
// open range of eq. restriction_j evaluated at the planes), split by the B plane j + 1, and
// their lengths are C_up - C_low with the slab's planes and that plane (eq. conditions_2D_1).
// With no crossing, plane j + 1 lies outside the slab and one of the two lengths is zero.
// Each length > 0 gives one `red.global.add.f32` at the row's entry; a slab costs no test of
// which rows it met beyond the two length signs.
//
// Layout (per problem, the x-driving plane first, then the y-driving one):
//   plane X: column m = x (nx columns), entry e = y + 2 for rows y = -2 .. ny + 1
//   plane Y: column m = y (ny columns), entry e = x + 2 for rows x = -2 .. nx + 1
// Each slab clamps the minor coordinate u_B into [-1.5, N_B + 0.5] before its floor, so rows j
// and j + 1 are within -2 .. N_B + 1.  A lane whose ray is outside the image over a slab (the
// warp steps over the union of its lanes' driving ranges) then reduces only into the padding
// rows, which the final sum never reads: no lane needs a bounds test.  The image is the sum
// v(x, y) = X[x][y + 2] + Y[y][x + 2].
//
// At a slab the lanes of a warp sit at neighbouring rows of one column, so their reductions
// fall on a few neighbouring sectors.  Lanes whose ray is parallel to an axis, or driven along
// the other axis than the warp's first lane, walk their ray alone with the crossing-order walk
// into plane Y (entry x + 2 of column y is pixel (x, y)).
//
// Every plane position is the same multiply-add of (plane index, 1/w, -frac/w) as in the
// other walks, so the lengths are theirs; each lane measures t as s = +-t, the sign making s
// grow with the driving index.
//
// Measured on GB300 (64 uneven fans, one plan): 29.0 ms, against 32.4 ms with one 64-bit
// reduction of the pair (row j, row j + 1) per slab into pair planes (half of whose bytes are
// zeros where the slab crosses no row) and 35.7 ms for the earlier lockstep walk into the
// image and its transposed copy.  A forward in this lockstep form, on pair planes (coalesced
// 64-bit loads, a row selection per slab), was slower than the crossing-order walk one ray per
// thread for one image (32.3 vs 25.1 ms for the 64 plain forwards; the ALU pipe bounds its
// per-slab bookkeeping); the per-thread pair-plane forward below takes 16.6 ms.  A warp whose lanes all
// see u_B move the same way along m could walk m in the direction that makes it grow and drop
// the row selection from every slab: 28.98 vs 29.12 ms, not kept.
#include <algorithm>

#include "xray_rays.cuh"

namespace xr {

namespace {

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: x + kMagic rounded down holds floor(x) in its low bits
constexpr int kMagicBits = 0x4B400000;

constexpr int kPadRows = 4;  // rows -2, -1 and N_B, N_B + 1 around every column

// One ray alone (crossing-order walk) on a layout with strides (sx, sy): its sum.
__device__ __forceinline__ float fwd_alone(const RayRec &rr, int nx, int ny, const float *__restrict__ img, int sx,
                                           int sy)
{
    Dda<int> D;
    float acc = 0.f;
    if (!dda_setup<int>(rr, nx, ny, 1, sx, sy, nx * ny, D)) return 0.f;
    for (int k = dda_max_steps(nx, ny, 1); k > 0 && D.tcur < D.tout; --k) {
        int off;
        float l;
        dda_step(D, off, l);
        if (l > 0.f) acc = __fmaf_rn(__ldg(img + off), l, acc);
    }
    return acc;
}

// One ray alone: g * l added into a layout with strides (sx, sy).
__device__ __forceinline__ void adj_alone(const RayRec &rr, int nx, int ny, float *acc, int sx, int sy, float g)
{
    Dda<int> D;
    if (!dda_setup<int>(rr, nx, ny, 1, sx, sy, nx * ny, D)) return;
    for (int k = dda_max_steps(nx, ny, 1); k > 0 && D.tcur < D.tout; --k) {
        int off;
        float l;
        dda_step(D, off, l);
        if (l > 0.f) red_add(acc + off, __fmul_rn(g, l));
    }
}

// The slab step of one lane in the s measure: the entry of row j (relative to the walk's
// column offset) and the lengths of rows j and j + 1.
struct SlabLane {
    float invA, bA, wB, fB, invB, bB, ulo, uhi;
    bool up;  // u_B grows with s: row j is met first
};

// Slab ending at plane p (s = sn): ebits (bits of row j's magic float) and the lengths
// (lx, ly) of rows j and j + 1; sc / mc: the slab's start and its row's magic float.
__device__ __forceinline__ void slab_rows(const SlabLane &L, float p, float sc, float mc, float &sn, float &mn,
                                          int &ebits, float &lx, float &ly)
{
    sn = __fmaf_rn(p, L.invA, L.bA);
    mn = __fadd_rd(fminf(fmaxf(__fmaf_rn(L.wB, sn, L.fB), L.ulo), L.uhi), kMagic);
    const float jm = fminf(mc, mn);
    const float ts = fminf(fmaxf(__fmaf_rn(jm - (kMagic - 1.0f), L.invB, L.bB), sc), sn);
    const float a = __fsub_rn(ts, sc), b = __fsub_rn(sn, ts);
    lx = L.up ? a : b;
    ly = L.up ? b : a;
    ebits = __float_as_int(jm);
}

// Entries per column of the accumulator plane of driving axis A (rows -2 .. N_B + 1)
__device__ __forceinline__ int plane_ld(int nb) { return nb + kPadRows; }

// 32 rays of one 2D problem, lane = ray (valid: the lane has a ray, g its sinogram value):
// g * l added into the problem's planes at P.aux.
__device__ __forceinline__ void slab_rays(const BatchItem &P, int64_t r, bool valid, float g)
{
    const int nx = P.nx, ny = P.ny;
    RayRec rr{};
    Walk W;
    bool ok = false;
    if (valid) {
        rr = (*P.src)[r];
        ok = walk_setup(rr, nx, ny, 1, 1, nx, (int64_t)nx * ny, W) && W.nact == 2;
    }
    // the warp's driving axis: that of the first lane with a ray the lockstep takes
    const unsigned okm = __ballot_sync(0xffffffffu, ok);
    const int lead = okm ? __ffs(okm) - 1 : 0;
    const int axA = __shfl_sync(0xffffffffu, ok ? W.axA : 0, lead);
    const bool lock = ok && W.axA == axA;
    const int64_t x_entries = (int64_t)nx * plane_ld(ny);
    float *plane = P.aux + (axA == 0 ? 0 : x_entries);
    const int ld = plane_ld(axA == 0 ? ny : nx);
    const int wlo = __reduce_min_sync(0xffffffffu, lock ? W.mlo : INT_MAX);
    const int whi = __reduce_max_sync(0xffffffffu, lock ? W.mhi : INT_MIN);
    if (lock) {
        SlabLane L;
        const float sgn = W.sgA ? -1.0f : 1.0f;  // s = sgn * t grows with m
        L.invA = sgn * W.invA;
        L.bA = sgn * W.bA;
        L.wB = sgn * W.wB;
        L.fB = W.fB;
        L.invB = sgn * W.invB;
        L.bB = sgn * W.bB;
        L.up = L.wB > 0.f;
        // floor(u_B) + oB clamped into -2 .. N_B
        L.ulo = -1.5f - (float)W.oB;
        L.uhi = (float)W.NB + 0.5f - (float)W.oB;
        // entry of row j from its magic float: column offset + bits - kMagicBits + oB + 2
        int moff = wlo * ld + (W.oB + 2 - kMagicBits);
        float p = (float)(wlo - W.oA);
        float sc = __fmaf_rn(p, L.invA, L.bA);
        float mc = __fadd_rd(fminf(fmaxf(__fmaf_rn(L.wB, sc, L.fB), L.ulo), L.uhi), kMagic);
#pragma unroll 2
        for (int m = wlo; m <= whi; ++m, moff += ld) {
            p += 1.0f;
            float sn, mn, lx, ly;
            int eb;
            slab_rows(L, p, sc, mc, sn, mn, eb, lx, ly);
            float *q = plane + (moff + eb);
            red_add_if_pos(q, __fmul_rn(g, lx), lx);
            red_add_if_pos(q + 1, __fmul_rn(g, ly), ly);
            sc = sn;
            mc = mn;
        }
    } else if (valid) {
        // pixel (x, y) is entry x + 2 of column y in plane Y
        adj_alone(rr, nx, ny, P.aux + x_entries + 2, 1, plane_ld(nx), g);
    }
}

// Work items of `tile` consecutive rays of one problem from one atomic counter (the batch
// plan's persistent launch); each work item walked 32 rays at a time.
__global__ void __launch_bounds__(256) slab_batch_kernel(const BatchItem *__restrict__ items, int n_items,
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
        for (int q0 = 0; q0 < tile; q0 += 32) {
            if (first + q0 >= P.n_rays) break;  // uniform over the warp
            const int64_t r = first + q0 + lane;
            const bool valid = r < P.n_rays;
            const float g = valid ? __ldg(P.sino + r) : 0.f;
            if (__all_sync(0xffffffffu, g == 0.f)) continue;  // nothing to spread
            slab_rays(P, r, valid, g);
        }
    }
}

// One problem on its own: warp w takes rays 32w .. 32w + 31.
__global__ void __launch_bounds__(256) slab_one_kernel(BatchItem P)
{
    const int lane = threadIdx.x & 31;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x - lane;
    if (first >= P.n_rays) return;  // the whole warp
    const int64_t r = first + lane;
    const bool valid = r < P.n_rays;
    const float g = valid ? __ldg(P.sino + r) : 0.f;
    if (__all_sync(0xffffffffu, g == 0.f)) return;  // nothing to spread
    slab_rays(P, r, valid, g);
}

// ---- the image from the accumulated planes ------------------------------------------------

constexpr int PT = 32;  // tile side

// Image tile b (x0 .. x0 + 31, y0 .. y0 + 31) of v(x, y) = X[x][y + 2] + Y[y][x + 2]; X's
// entries staged through shared memory so that its reads run along its columns and the
// image's writes along x.
__device__ __forceinline__ void sum_tile(const float *__restrict__ acc, int nx, int ny, float *__restrict__ img, int b,
                                         float (*s)[PT + 1])
{
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int ntx = (nx + PT - 1) / PT;
    const int x0 = (b % ntx) * PT, y0 = (b / ntx) * PT;
    const int ldx = plane_ld(ny), ldy = plane_ld(nx);
    // s[c][k] = X[x0 + c][y0 + 2 + k]
    for (int c = ty; c < PT; c += blockDim.y) {
        const int x = x0 + c, e = y0 + 2 + tx;
        s[c][tx] = (x < nx && e < ldx) ? acc[(int64_t)x * ldx + e] : 0.f;
    }
    __syncthreads();
    const float *Y = acc + (int64_t)nx * ldx;
    const int x = x0 + tx;
    for (int c = ty; c < PT; c += blockDim.y) {
        const int y = y0 + c;
        if (x < nx && y < ny) img[(int64_t)y * nx + x] = __fadd_rn(s[tx][c], Y[(int64_t)y * ldy + x + 2]);
    }
}

__global__ void __launch_bounds__(256) sum_items_kernel(const BatchItem *__restrict__ items)
{
    __shared__ float s[PT][PT + 1];
    const BatchItem &P = items[blockIdx.y];
    const int n = ((P.nx + PT - 1) / PT) * ((P.ny + PT - 1) / PT);
    for (int b = blockIdx.x; b < n; b += gridDim.x) {
        __syncthreads();
        sum_tile(P.aux, P.nx, P.ny, const_cast<float *>(P.img), b, s);
    }
}

__global__ void __launch_bounds__(256) sum_one_kernel(const float *__restrict__ acc, int nx, int ny,
                                                      float *__restrict__ img)
{
    __shared__ float s[PT][PT + 1];
    sum_tile(acc, nx, ny, img, blockIdx.x, s);
}

// Zero every problem's planes
__global__ void __launch_bounds__(256) zero_items_kernel(const BatchItem *__restrict__ items)
{
    const BatchItem &P = items[blockIdx.y];
    const int64_t n = slab2d_acc_floats(P.nx, P.ny);
    float *a = P.aux;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += (int64_t)gridDim.x * blockDim.x)
        a[u] = 0.f;
}

// ---- the forward: one ray per thread on pair planes -----------------------------------------
//
// Pair planes (per problem, the x-driving plane first): column m of the plane of axis A holds,
// at entry e = j + kPairPad, the pair (v(m, j), v(m, j + 1)) of pixels of rows j and j + 1
// along B, for j = -kPairPad .. N_B + kPairPad - 1, with v = 0 outside the image.  A thread
// walks its ray's own driving range in the direction in which u_B grows, so that at every slab
// the lower row j = floor(u_B) at the slab's start is the pair's first pixel and the B plane
// j + 1 splits the slab into the two pixels' lengths: one 64-bit load and no selection per
// slab.  Over a ray's driving range (its box interval and one slab on either side, |slope| <= 1)
// u_B stays within 2 of [0, N_B], inside the padding; the entry is also clamped to the plane,
// so no load leaves it.

constexpr int kPairPad = 3;
#ifndef XR_SLAB_FWD_AHEAD
#define XR_SLAB_FWD_AHEAD 8  // 4: 2-3% slower (64 uneven fans: 13.97 vs 13.74 ms)
#endif
constexpr int kFwdAhead = XR_SLAB_FWD_AHEAD;  // slabs split ahead of their loads

__host__ __device__ __forceinline__ int pair_ld(int nb) { return nb + 2 * kPairPad; }

// One ray's sum over the image (img: [ny][nx], for rays parallel to an axis; pairs: its planes).
__device__ __forceinline__ float slab_fwd_ray(const RayRec &rr, int nx, int ny, const float *__restrict__ img,
                                              const float2 *__restrict__ pairs)
{
    Walk W;
    if (!walk_setup(rr, nx, ny, 1, 1, nx, (int64_t)nx * ny, W)) return 0.f;
    if (W.nact != 2) return fwd_alone(rr, nx, ny, img, 1, nx);
    const int ld = pair_ld(W.NB);
    const float2 *plane = pairs + (W.axA == 0 ? 0 : (int64_t)nx * pair_ld(ny));
    const unsigned emax = (unsigned)(W.NA * ld - 1);
    // walk m up when u_B grows with it (w_A and w_B of one sign), else down; s = sign(w_B) t
    // grows along the walk and u_B = |w_B| s + f_B grows with s
    const bool upm = (W.wB > 0.f) == (W.sgA == 0);
    const float sg = W.wB > 0.f ? 1.0f : -1.0f;
    const float invA = sg * W.invA, bA = sg * W.bA, wB = sg * W.wB, fB = W.fB;
    const float invB = sg * W.invB, bB = sg * W.bB;
    const float dp = upm ? 1.0f : -1.0f;
    const int dld = upm ? ld : -ld;
    const int n = W.mhi - W.mlo + 1;
    float p = (float)((upm ? W.mlo : W.mhi + 1) - W.oA);  // the first slab's starting plane
    // entry of row j from its magic float: column offset + bits - kMagicBits + oB + kPairPad
    int moff = (upm ? W.mlo : W.mhi) * ld + (W.oB + kPairPad - kMagicBits);
    float sc = __fmaf_rn(p, invA, bA);
    float mc = __fadd_rd(__fmaf_rn(wB, sc, fB), kMagic);
    float acc0 = 0.f, acc1 = 0.f;
    int k = 0;
    for (; k + kFwdAhead <= n; k += kFwdAhead) {
        unsigned e[kFwdAhead];
        float lx[kFwdAhead], ly[kFwdAhead];
#pragma unroll
        for (int u = 0; u < kFwdAhead; ++u) {
            p += dp;
            const float sn = __fmaf_rn(p, invA, bA);
            const float mn = __fadd_rd(__fmaf_rn(wB, sn, fB), kMagic);
            const float ts = fminf(fmaxf(__fmaf_rn(mc - (kMagic - 1.0f), invB, bB), sc), sn);
            lx[u] = __fsub_rn(ts, sc);
            ly[u] = __fsub_rn(sn, ts);
            e[u] = min((unsigned)(moff + __float_as_int(mc)), emax);
            moff += dld;
            sc = sn;
            mc = mn;
        }
        float2 v[kFwdAhead];
#pragma unroll
        for (int u = 0; u < kFwdAhead; ++u) v[u] = __ldg(plane + e[u]);
#pragma unroll
        for (int u = 0; u < kFwdAhead; ++u) {
            acc0 = __fmaf_rn(v[u].x, lx[u], acc0);
            acc1 = __fmaf_rn(v[u].y, ly[u], acc1);
        }
    }
    for (; k < n; ++k) {
        p += dp;
        const float sn = __fmaf_rn(p, invA, bA);
        const float mn = __fadd_rd(__fmaf_rn(wB, sn, fB), kMagic);
        const float ts = fminf(fmaxf(__fmaf_rn(mc - (kMagic - 1.0f), invB, bB), sc), sn);
        const float2 v = __ldg(plane + min((unsigned)(moff + __float_as_int(mc)), emax));
        acc0 = __fmaf_rn(v.x, __fsub_rn(ts, sc), acc0);
        acc1 = __fmaf_rn(v.y, __fsub_rn(sn, ts), acc1);
        moff += dld;
        sc = sn;
        mc = mn;
    }
    return __fadd_rn(acc0, acc1);
}

__global__ void __launch_bounds__(256) slab_fwd_one_kernel(BatchItem P, const float2 *__restrict__ pairs)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= P.n_rays) return;
    P.sino[r] = slab_fwd_ray((*P.src)[r], P.nx, P.ny, P.img, pairs);
}

// The batch plan's persistent forward: work items of `tile` consecutive rays of one problem,
// one ray per thread; each item's pair planes at its aux.
// (62 registers; capped at 48 for 5 CTAs per SM: 13.97 vs 13.81 ms on the 64 uneven fans)
__global__ void __launch_bounds__(256) slab_fwd_batch_kernel(const BatchItem *__restrict__ items, int n_items,
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
            P.sino[r] = slab_fwd_ray((*P.src)[r], P.nx, P.ny, P.img, reinterpret_cast<const float2 *>(P.aux));
        }
    }
}

// Tiles of one problem's pair planes: the x-driving plane's (columns x, entries e), then the
// y-driving plane's.
__host__ __device__ __forceinline__ int pair_tiles_x(int nx, int ny) { return ((nx + PT - 1) / PT) * ((pair_ld(ny) + PT - 1) / PT); }
__host__ __device__ __forceinline__ int pair_tiles_y(int nx, int ny) { return ((ny + PT - 1) / PT) * ((pair_ld(nx) + PT - 1) / PT); }

// v(x, y) of an [ny][nx] image, 0 outside
__device__ __forceinline__ float pix(const float *__restrict__ img, int nx, int ny, int x, int y)
{
    return (x >= 0 && x < nx && y >= 0 && y < ny) ? __ldg(img + (int64_t)y * nx + x) : 0.f;
}

// Tile b of one problem's pair planes (blocks of 32 x 8 threads).
__device__ __forceinline__ void build_tile(const float *__restrict__ img, int nx, int ny, float2 *__restrict__ pairs,
                                           int b, float (*s)[PT + 1])
{
    const int tx = threadIdx.x, ty = threadIdx.y;
    const int tX = pair_tiles_x(nx, ny);
    if (b < tX) {
        // plane X: columns x0 .. x0 + 31, entries e0 .. e0 + 31 (rows j = e - kPairPad); the
        // image's rows e0 - kPairPad .. e0 - kPairPad + 32 staged so that reads run along x and
        // writes along e
        const int ldx = pair_ld(ny);
        const int ntx = (nx + PT - 1) / PT;
        const int x0 = (b % ntx) * PT, e0 = (b / ntx) * PT;
        for (int rr = ty; rr < PT + 1; rr += blockDim.y) s[rr][tx] = pix(img, nx, ny, x0 + tx, e0 - kPairPad + rr);
        __syncthreads();
        const int e = e0 + tx;
        for (int c = ty; c < PT; c += blockDim.y) {
            const int x = x0 + c;
            if (x < nx && e < ldx) pairs[(int64_t)x * ldx + e] = make_float2(s[tx][c], s[tx + 1][c]);
        }
    } else {
        // plane Y: columns y, entries e (rows i = e - kPairPad), both read along x
        const int ldy = pair_ld(nx);
        const int bb = b - tX;
        const int nte = (ldy + PT - 1) / PT;
        const int e = (bb % nte) * PT + tx, y0 = (bb / nte) * PT;
        float2 *py = pairs + (int64_t)nx * pair_ld(ny);
        if (e < ldy)
            for (int c = ty; c < PT; c += blockDim.y) {
                const int y = y0 + c;
                if (y < ny)
                    py[(int64_t)y * ldy + e] = make_float2(pix(img, nx, ny, e - kPairPad, y),
                                                           pix(img, nx, ny, e - kPairPad + 1, y));
            }
    }
}

__global__ void __launch_bounds__(256) build_items_kernel(const BatchItem *__restrict__ items)
{
    __shared__ float s[PT + 1][PT + 1];
    const BatchItem &P = items[blockIdx.y];
    const int n = pair_tiles_x(P.nx, P.ny) + pair_tiles_y(P.nx, P.ny);
    for (int b = blockIdx.x; b < n; b += gridDim.x) {
        __syncthreads();
        build_tile(P.img, P.nx, P.ny, reinterpret_cast<float2 *>(P.aux), b, s);
    }
}

__global__ void __launch_bounds__(256) build_one_kernel(const float *__restrict__ img, int nx, int ny,
                                                        float2 *__restrict__ pairs)
{
    __shared__ float s[PT + 1][PT + 1];
    build_tile(img, nx, ny, pairs, blockIdx.x, s);
}

}  // namespace

cudaError_t launch_slab2d_adjoint_one(const BatchItem &P, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(P.aux, 0, (size_t)slab2d_acc_floats(P.nx, P.ny) * sizeof(float), s);
    if (e != cudaSuccess) return e;
    slab_one_kernel<<<(unsigned)((P.n_rays + 255) / 256), 256, 0, s>>>(P);
    const unsigned img_tiles = (unsigned)(((P.nx + PT - 1) / PT) * ((P.ny + PT - 1) / PT));
    sum_one_kernel<<<img_tiles, dim3(PT, 8), 0, s>>>(P.aux, P.nx, P.ny, const_cast<float *>(P.img));
    return cudaGetLastError();
}

int slab2d_ctas_per_sm(int block, bool adjoint)
{
    int n = 0;
    if (adjoint)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, slab_batch_kernel, block, 0);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, slab_fwd_batch_kernel, block, 0);
    return n > 0 ? n : 1;
}

cudaError_t launch_slab2d_project_one(const BatchItem &P, cudaStream_t s)
{
    float2 *pairs = reinterpret_cast<float2 *>(P.aux);
    build_one_kernel<<<(unsigned)(pair_tiles_x(P.nx, P.ny) + pair_tiles_y(P.nx, P.ny)), dim3(PT, 8), 0, s>>>(
        P.img, P.nx, P.ny, pairs);
    slab_fwd_one_kernel<<<(unsigned)((P.n_rays + 255) / 256), 256, 0, s>>>(P, pairs);
    return cudaGetLastError();
}

cudaError_t launch_slab2d_project(const BatchItem *items, int n_items, int64_t n_tiles, int tile,
                                  unsigned long long *counter, int grid_ctas, int block, int sms, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    const dim3 per_item((unsigned)std::max(1, 4 * sms / std::max(1, n_items)), (unsigned)n_items);
    build_items_kernel<<<per_item, dim3(PT, 8), 0, s>>>(items);
    slab_fwd_batch_kernel<<<grid_ctas, block, 0, s>>>(items, n_items, n_tiles, tile, counter);
    return cudaGetLastError();
}

cudaError_t launch_slab2d_adjoint(const BatchItem *items, int n_items, int64_t n_tiles, int tile,
                                  unsigned long long *counter, int grid_ctas, int block, int sms, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(counter, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess) return e;
    // per-problem passes: a few waves of CTAs per problem, grid-strided over its tiles
    const dim3 per_item((unsigned)std::max(1, 4 * sms / std::max(1, n_items)), (unsigned)n_items);
    zero_items_kernel<<<per_item, 256, 0, s>>>(items);
    slab_batch_kernel<<<grid_ctas, block, 0, s>>>(items, n_items, n_tiles, tile, counter);
    sum_items_kernel<<<per_item, dim3(PT, 8), 0, s>>>(items);
    return cudaGetLastError();
}

}  // namespace xr
