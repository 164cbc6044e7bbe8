// The adjoint of 2D problems with one image each (a single image of a 2D scan, or the problems
// of a batch plan): 32 neighbouring rays per warp walked slab by slab in lockstep, reduced into
// padded accumulator planes, one plane per driving axis.
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
// Measured on GB300 (64 uneven fans, one plan): 29.2 ms, against 32.4 ms with one 64-bit
// reduction of the pair (row j, row j + 1) per slab into pair planes (half of whose bytes are
// zeros where the slab crosses no row) and 35.7 ms for the earlier lockstep walk into the
// image and its transposed copy.  A forward on pair planes (one 64-bit load per slab) was
// slower than the crossing-order walk one ray per thread for one image (32.3 vs 25.1 ms for
// the 64 plain forwards): the ALU pipe bounds its per-slab bookkeeping.
#include <algorithm>

#include "xray_rays.cuh"

namespace xr {

namespace {

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: x + kMagic rounded down holds floor(x) in its low bits
constexpr int kMagicBits = 0x4B400000;

constexpr int kPadRows = 4;  // rows -2, -1 and N_B, N_B + 1 around every column

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

int slab2d_ctas_per_sm(int block)
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, slab_batch_kernel, block, 0);
    return n > 0 ? n : 1;
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
