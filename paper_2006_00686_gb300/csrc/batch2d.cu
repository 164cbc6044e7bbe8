// Adjoint of 2D problems (one image each) with the slab walk in warp lockstep, reduced
// straight into the caller's images: the one-call batched adjoint (xr_backproject_batched),
// which holds no per-problem planes, takes it when every problem is 2D (64 uneven fans: 38 ms
// against 72 ms for rays walked one by one).  Batch plans and single images, which hold
// padded accumulator planes, take the leaner form of this walk in slab2d.cu.  The forward
// stays the crossing-order walk one ray at a time: the same lockstep walk as a forward
// measured 40.6 ms, and 48 ms with eight slabs' loads issued together, against 22.1 ms -- for
// one image per problem the lockstep's per-slab bookkeeping and its union of the lanes' slab
// ranges cost more than its coalesced loads save, while for reductions the coalescing decides.
//
// Warps take work items of consecutive rays of one problem from one atomic counter; a work
// item is walked 32 rays at a time, one lane per ray.  The 32 rays are neighbouring detector
// bins of one view, so they share the driving axis A (the axis with the largest index-space
// slope, Section 4.3) and run side by side.  The lanes step the driving index m together; per
// slab a lane's minor index at the slab's two planes is floor(u_B) there (the open range of
// eq. restriction_j evaluated at the planes), the minor plane crossed inside the slab splits
// it into the two pixels (c, n), and their lengths are C_up - C_low with the slab's planes and
// the minor plane (eq. conditions_2D_1).  Every plane is the same multiply-add of (plane index,
// 1/w, -frac/w) as in the crossing-order walk, so the lengths are that walk's.
//
// At a given slab the 32 lanes sit at neighbouring rows of the minor axis; the kernel reduces
// into the layout whose fastest axis is the minor one -- the problem's y-fastest copy for rays
// driven along x, the image itself for rays driven along y -- so a warp's reductions fall on a
// few neighbouring sectors, where rays walked one by one drift apart and touch a sector each.
// Lanes whose ray is axis-parallel, or driven along the other axis than the warp's first lane,
// walk their ray alone with the crossing-order walk.
#include "xray_rays.cuh"

namespace xr {

namespace {

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: x + kMagic rounded down holds floor(x) in its low bits
constexpr int kMagicBits = 0x4B400000;

// One lane's ray alone (crossing-order walk) on the caller's layout.
__device__ __forceinline__ void scatter_alone(const RayRec &rr, int nx, int ny, float *acc, float g)
{
    Dda<int> D;
    if (!dda_setup<int>(rr, nx, ny, 1, 1, nx, nx * ny, D)) return;
    for (int k = dda_max_steps(nx, ny, 1); k > 0 && D.tcur < D.tout; --k) {
        int off;
        float l;
        dda_step(D, off, l);
        if (l > 0.f) red_add(acc + off, __fmul_rn(g, l));
    }
}

// 32 rays of one 2D problem, lane = ray (valid: the lane has a ray): adds g * l into the
// problem's accumulators (img for rays driven along y, aux -- the y-fastest [x][y] layout -- for
// rays driven along x; aux may be NULL, then img).
//
// Each lane measures its ray in s = +-t, the sign chosen so that s grows with the driving index
// (plane positions and the minor slope negated together for a ray whose index u_A falls along
// t): lengths are differences of s, and a slab [s(m), s(m + 1)] always runs forward.  The minor
// plane between the rows at the slab's two ends is max(j_c, j_n) (relative to the foot point);
// clamped into the slab it gives pixel c the part before it and pixel n the part after it --
// with no crossing (j_c = j_n) one of the two parts is the whole slab and the other empty.  The
// warp steps over the union of its lanes' driving ranges: at a slab outside a lane's own range
// (within the grid) the lane's ray is outside the image in the minor direction, so its rows fail
// the row bounds check.
__device__ __forceinline__ void slab2d_adjoint(const BatchItem &P, int64_t r, bool valid, float g)
{
    const int nx = P.nx, ny = P.ny;
    RayRec rr{};
    Walk W;
    bool ok = false;
    if (valid) {
        rr = (*P.src)[r];
        ok = walk_setup(rr, nx, ny, 1, 1, nx, (int64_t)nx * ny, W) && W.nact == 2;
    }
    // the warp's driving axis: the first lane with a lockstep-able ray
    const unsigned okm = __ballot_sync(0xffffffffu, ok);
    const int lead = okm ? __ffs(okm) - 1 : 0;
    const int axA = __shfl_sync(0xffffffffu, ok ? W.axA : 0, lead);
    const bool lock = ok && W.axA == axA;
    const bool y_fast = axA == 0 && P.aux != nullptr;  // minor axis y: reduce into the [x][y] copy
    const int sA = axA == 0 ? (y_fast ? ny : 1) : nx;   // stride of the driving index
    const int sB = axA == 0 ? (y_fast ? 1 : nx) : 1;    // stride of the minor index
    float *base = y_fast ? P.aux : const_cast<float *>(P.img);
    const int wlo = __reduce_min_sync(0xffffffffu, lock ? W.mlo : INT_MAX);
    const int whi = __reduce_max_sync(0xffffffffu, lock ? W.mhi : INT_MIN);
    if (lock) {
        const float sgn = W.sgA ? -1.0f : 1.0f;  // s = sgn * t grows with m
        const float invA = sgn * W.invA, bA = sgn * W.bA, wB = sgn * W.wB, fB = W.fB;
        const float invB = sgn * W.invB, bB = sgn * W.bB;
        const int oB = W.oB, NB = W.NB;
        float p = (float)(wlo - W.oA);
        float tcur = __fmaf_rn(p, invA, bA);
        float sc = __fadd_rd(__fmaf_rn(wB, tcur, fB), kMagic);
        float jc = __fadd_rn(sc, -kMagic);
        int moff = wlo * sA;
        for (int m = wlo; m <= whi; ++m, moff += sA) {
            p += 1.0f;
            const float tn = __fmaf_rn(p, invA, bA);
            const float sn = __fadd_rd(__fmaf_rn(wB, tn, fB), kMagic);
            const float jn = __fadd_rn(sn, -kMagic);
            const int rc = __float_as_int(sc) - kMagicBits + oB, rn = __float_as_int(sn) - kMagicBits + oB;
            if (fabsf(jn - jc) < 1.5f) {
                // at most one minor plane inside the slab
                const float tx = fminf(fmaxf(__fmaf_rn(fmaxf(jc, jn), invB, bB), tcur), tn);
                const float lc = __fsub_rn(tx, tcur), ln = __fsub_rn(tn, tx);
                if ((unsigned)rc < (unsigned)NB && lc > 0.f) red_add(base + moff + rc * sB, __fmul_rn(g, lc));
                if ((unsigned)rn < (unsigned)NB && ln > 0.f) red_add(base + moff + rn * sB, __fmul_rn(g, ln));
            } else if (m >= W.mlo && m <= W.mhi) {
                // crossing two minor planes (within rounding of a diagonal): each candidate row
                const int jlo = (int)fminf(jc, jn), jhi = (int)fmaxf(jc, jn);
                for (int j = jlo; j <= jhi; ++j) {
                    const int jg = j + oB;
                    if ((unsigned)jg >= (unsigned)NB) continue;
                    const float t0 = __fmaf_rn((float)j, invB, bB), t1 = __fmaf_rn((float)(j + 1), invB, bB);
                    const float l = __fsub_rn(fminf(tn, fmaxf(t0, t1)), fmaxf(tcur, fminf(t0, t1)));
                    if (l > 0.f) red_add(base + moff + jg * sB, __fmul_rn(g, l));
                }
            }
            tcur = tn;
            sc = sn;
            jc = jn;
        }
    } else if (valid) {
        scatter_alone(rr, nx, ny, const_cast<float *>(P.img), g);
    }
}

// The work list as in batched_dda_kernel (2D problems only: the host sends this kernel lists
// whose problems are all 2D).
__global__ void __launch_bounds__(256) batch2d_adj_kernel(const BatchItem *__restrict__ items, int n_items,
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
            slab2d_adjoint(P, r, valid, g);
        }
    }
}

}  // namespace

int batch2d_ctas_per_sm(int block)
{
    int n = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch2d_adj_kernel, block, 0);
    return n > 0 ? n : 1;
}

cudaError_t launch_batch2d_adjoint(const BatchItem *items, int n_items, int64_t n_tiles, int tile,
                                   unsigned long long *counter, int grid_ctas, int block, cudaStream_t s)
{
    batch2d_adj_kernel<<<grid_ctas, block, 0, s>>>(items, n_items, n_tiles, tile, counter);
    return cudaGetLastError();
}

}  // namespace xr
