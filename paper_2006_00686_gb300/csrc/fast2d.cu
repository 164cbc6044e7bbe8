// Batched fast path for 2D scans (rays with at most two active axes), batches of 4 or more.
//
// Two layouts of the batch, both in two bordered spatial orders (IL0: x fastest, IL1:
// y fastest), so that the rays of a warp -- neighbouring detector bins, which sit on
// neighbouring units of the minor axis at every driving step -- touch neighbouring memory:
//   * quad planes [Q][ny+2P][nx+2P][4] (second half of this file): plane q holds images
//     4q..4q+3 as one float4 per unit; the forward (one thread per ray) and the gather adjoint
//     (one thread per pair of pixels) run on it;
//   * Bp-interleaved [chunk][...][Bp] (Bp = 4 * LPR images of one chunk contiguous, 64 bytes
//     for Bp = 16): the accumulators of the ray-driven scatter adjoint, which adds with
//     128-bit vector reductions.
// A border of P = 2 zero units surrounds the image in x and y: the walk visits driving
// slabs one beyond the image's extent, where the minor index can leave the image by at
// most two, so every row the kernel can touch is valid memory and holds zero outside the
// image -- no per-unit range test is needed.
//
// Slab step (2D form of the walk in xray_core.cuh).  Between driving planes m and m+1 the
// ray moves from row jc = floor(u_B(m)) to row jn = floor(u_B(m+1)); if they differ it
// crosses the plane max(jc, jn) at tc, and the slab splits into |tc - t_m| in row jc and
// |t_{m+1} - tc| in row jn.  These are C_up - C_low of the two units with the same plane
// values the walk uses; the rare step that crosses two rows falls back to the general
// per-candidate formula.
#include <algorithm>
#include <atomic>
#include <cmath>

#include "xray_internal.h"


// Resident blocks per SM the forward kernel is compiled for (a register budget).
#ifndef XR_FWD_MIN_BLOCKS
#define XR_FWD_MIN_BLOCKS 4
#endif


namespace xr {

// ---------------------------------------------------------------------------------------
// Layout conversions
// ---------------------------------------------------------------------------------------

// Adjoint accumulators -> user images: img[b][u] = IL0 + IL1 at unit u (interiors only).
__global__ void deinterleave_sum_kernel(const float *__restrict__ il0, const float *__restrict__ il1, int batch,
                                        int nx, int ny, int nz, int Bp, float *__restrict__ img)
{
    const int64_t n = (int64_t)nx * ny * nz;
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= n) return;
    const int chunk = blockIdx.y;
    const int i = (int)(u % nx);
    const int64_t rest = u / nx;
    const int j = (int)(rest % ny);
    const int k = (int)(rest / ny);
    const int px = nx + 2 * XR_IL_PAD, py = ny + 2 * XR_IL_PAD;
    const int64_t np = (int64_t)px * py * nz;
    const int64_t o0 = ((int64_t)chunk * np + ((int64_t)k * py + j + XR_IL_PAD) * px + i + XR_IL_PAD) * Bp;
    const int64_t o1 = ((int64_t)chunk * np + ((int64_t)k * px + i + XR_IL_PAD) * py + j + XR_IL_PAD) * Bp;
    for (int b4 = 0; b4 < Bp; b4 += 4) {
        const float4 a = *reinterpret_cast<const float4 *>(il0 + o0 + b4);
        const float4 c = *reinterpret_cast<const float4 *>(il1 + o1 + b4);
        const int b = chunk * Bp + b4;
        if (b + 0 < batch) img[(int64_t)(b + 0) * n + u] = a.x + c.x;
        if (b + 1 < batch) img[(int64_t)(b + 1) * n + u] = a.y + c.y;
        if (b + 2 < batch) img[(int64_t)(b + 2) * n + u] = a.z + c.z;
        if (b + 3 < batch) img[(int64_t)(b + 3) * n + u] = a.w + c.w;
    }
}

__device__ __forceinline__ void fma4(float4 &acc, const float4 v, float l)
{
    acc.x = __fmaf_rn(v.x, l, acc.x);
    acc.y = __fmaf_rn(v.y, l, acc.y);
    acc.z = __fmaf_rn(v.z, l, acc.z);
    acc.w = __fmaf_rn(v.w, l, acc.w);
}

// Rows jlo..jhi of the current slab with the per-candidate formula (a step that crosses
// two rows: rare, only for rays within rounding of a diagonal).  Returns the contribution.
__device__ __noinline__ float4 slab_rows_general(int oB, int NB, int sgB, float invB, float bB, float tlo,
                                                 float thi, int jlo, int jhi, const float *__restrict__ base,
                                                 int64_t sB)
{
    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    for (int j = jlo; j <= jhi; ++j) {
        const int jg = j + oB;
        if ((unsigned)jg >= (unsigned)NB) continue;
        const float q = (float)j;
        const float tb0 = __fmaf_rn(q + (float)sgB, invB, bB);
        const float tb1 = __fmaf_rn(q + (float)(1 - sgB), invB, bB);
        const float l = __fsub_rn(fminf(thi, tb1), fmaxf(tlo, tb0));
        if (l > 0.f) fma4(acc, __ldg(reinterpret_cast<const float4 *>(base + (int64_t)jg * sB)), l);
    }
    return acc;
}

// Scatter counterpart of slab_rows_general: adds g * l into rows jlo..jhi of the slab.
__device__ __noinline__ void scatter_rows_general(int oB, int NB, int sgB, float invB, float bB, float tlo,
                                                  float thi, int jlo, int jhi, const float *__restrict__ base,
                                                  int64_t sB, float4 g)
{
    for (int j = jlo; j <= jhi; ++j) {
        const int jg = j + oB;
        if ((unsigned)jg >= (unsigned)NB) continue;
        const float q = (float)j;
        const float tb0 = __fmaf_rn(q + (float)sgB, invB, bB);
        const float tb1 = __fmaf_rn(q + (float)(1 - sgB), invB, bB);
        const float l = __fsub_rn(fminf(thi, tb1), fmaxf(tlo, tb0));
        if (l > 0.f) red_add4(const_cast<float *>(base + (int64_t)jg * sB), g.x * l, g.y * l, g.z * l, g.w * l);
    }
}

// Scatter visitor for rays with three active axes on the interleaved layout.
struct Il4ScatterVisitor {
    float *il;
    float4 g;
    __device__ __forceinline__ void operator()(int64_t off, float l)
    {
        red_add4(il + off, g.x * l, g.y * l, g.z * l, g.w * l);
    }
};

// Visitor for rays with three active axes (general walk on the interleaved layout).
struct Il4Visitor {
    const float *il;
    float4 acc;
    __device__ __forceinline__ void operator()(int64_t off, float l)
    {
        fma4(acc, __ldg(reinterpret_cast<const float4 *>(il + off)), l);
    }
};

// ---------------------------------------------------------------------------------------
// Forward, LPR lanes per ray, 4 images per lane
// ---------------------------------------------------------------------------------------

// floor of |x| < 2^22 with one round-down add: the float floor and the integer floor
constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23
constexpr int kMagicBits = 0x4B400000;

// One unit of the walk: the forward gathers the unit's 4 images, the adjoint adds the ray's
// 4 sinogram values times the length into them (one 128-bit vector atomic).
template <bool ADJ>
__device__ __forceinline__ void unit_op(const float *p, bool on, float l, float4 &acc)
{
    if (ADJ) {
        if (on && l > 0.f) red_add4(const_cast<float *>(p), acc.x * l, acc.y * l, acc.z * l, acc.w * l);
    } else {
        const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
        fma4(acc, on ? __ldg(reinterpret_cast<const float4 *>(p)) : z, l);
    }
}

// LPR lanes cooperate on one ray, each owning 4 images.  ADJ = true (the one launched): the
// scatter adjoint, sino the input and il0/il1 the zeroed Bp-interleaved accumulators.
// ADJ = false walks the same way as a forward on Bp-interleaved images.
template <int LPR, bool ADJ>
__global__ void __launch_bounds__(256, XR_FWD_MIN_BLOCKS) fwd_fast2_kernel(const RayRec *__restrict__ rays, int64_t n_rays,
                                                           int nx, int ny, int nz, const float *__restrict__ il0,
                                                           const float *__restrict__ il1, int Bp,
                                                           float *__restrict__ sino, int batch)
{
    constexpr int RPW = 32 / LPR;  // rays per warp
    const int lane = threadIdx.x & 31;
    const int q = lane % LPR;  // image quad owned by this lane
    const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int64_t r = warp * RPW + lane / LPR;
    const int chunk = blockIdx.y;
    const int px = nx + 2 * XR_IL_PAD, py = ny + 2 * XR_IL_PAD;
    const int64_t np = (int64_t)px * py * nz;

    Walk W;
    bool ok = false;
    // this kernel's slab step covers rays with at most two active axes whose minor axis has
    // a border (x or y); the rest take the general walk, which tests every index
    if (r < n_rays)
        ok = walk_setup(rays[r], nx, ny, nz, 1, nx, (int64_t)nx * ny, W) && W.nact <= 2 &&
             !(W.nact == 2 && W.axB == 2);
    const bool general = (r < n_rays) && !ok;
    // layout of the warp: the driving axis of its first ray
    const int axA0 = __shfl_sync(0xffffffffu, ok ? W.axA : 1, 0);
    const bool y_fast = (axA0 == 0);
    // element strides (floats) of i, j, k in that layout; one padded chunk holds np*Bp < 2^31
    const int si = y_fast ? py * Bp : Bp;
    const int sj = y_fast ? Bp : px * Bp;
    const int sk = px * py * Bp;
    // unit (0, 0, 0) of the image inside the border
    const float *il = (y_fast ? il1 : il0) + (int64_t)chunk * np * Bp + 4 * q + XR_IL_PAD * (si + sj);

    float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
    if (ADJ && r < n_rays) {
        // the adjoint scatters g * l: acc holds this lane's 4 sinogram values
        const int b0 = chunk * Bp + 4 * q;
        acc.x = (b0 + 0 < batch) ? __ldg(sino + (int64_t)(b0 + 0) * n_rays + r) : 0.f;
        acc.y = (b0 + 1 < batch) ? __ldg(sino + (int64_t)(b0 + 1) * n_rays + r) : 0.f;
        acc.z = (b0 + 2 < batch) ? __ldg(sino + (int64_t)(b0 + 2) * n_rays + r) : 0.f;
        acc.w = (b0 + 3 < batch) ? __ldg(sino + (int64_t)(b0 + 3) * n_rays + r) : 0.f;
    }
    const int wlo = __reduce_min_sync(0xffffffffu, ok ? W.mlo : INT_MAX);
    const int whi = __reduce_max_sync(0xffffffffu, ok ? W.mhi : INT_MIN);
    if (ok) {
        const int sA = sel3(W.axA, si, sj, sk), sB = sel3(W.axB, si, sj, sk), sC = sel3(W.axC, si, sj, sk);
        const bool bact = W.nact >= 2;
        // offset of the fixed axes in this layout (walk_setup folded them with its own strides)
        const int base = W.oC * sC + (bact ? 0 : W.oB * sB) + (bact ? W.oB * sB : 0);
        const float *pA = il + base;
        const float invA = W.invA, bA = W.bA, wB = W.wB, fB = W.fB, invB = W.invB, bB = W.bB;
        const int mlo = W.mlo, mhi = W.mhi;
        float p = (float)(wlo - W.oA);
        float tcur = __fmaf_rn(p, invA, bA);
        float sm = __fadd_rd(__fmaf_rn(wB, tcur, fB), kMagic);
        float j0 = __fadd_rn(sm, -kMagic);
        int moff = wlo * sA;
        for (int m = wlo; m <= whi; m += 2, moff += 2 * sA) {
            // slab m: planes m, m+1; slab m+1: planes m+1, m+2
            const float t1 = __fmaf_rn(p + 1.0f, invA, bA);
            const float t2 = __fmaf_rn(p + 2.0f, invA, bA);
            const float s1 = __fadd_rd(__fmaf_rn(wB, t1, fB), kMagic);
            const float s2 = __fadd_rd(__fmaf_rn(wB, t2, fB), kMagic);
            const float j1 = __fadd_rn(s1, -kMagic), j2 = __fadd_rn(s2, -kMagic);
            // rows relative to the ray's foot row; the border makes every reachable row valid
            const int r0 = __float_as_int(sm) - kMagicBits;
            const int r1 = __float_as_int(s1) - kMagicBits;
            const int r2 = __float_as_int(s2) - kMagicBits;
            const bool act0 = m >= mlo && m <= mhi, act1 = m + 1 >= mlo && m + 1 <= mhi;
            if (fabsf(j1 - j0) < 1.5f && fabsf(j2 - j1) < 1.5f) {
                const bool x01 = r1 != r0, x12 = r2 != r1;
                // crossing planes of the two slabs (plane max(jc, jn) of the minor axis)
                const float tc0 = __fmaf_rn(fmaxf(j0, j1), invB, bB);
                const float tc1 = __fmaf_rn(fmaxf(j1, j2), invB, bB);
                const float tcc0 = x01 ? fminf(fmaxf(tc0, fminf(tcur, t1)), fmaxf(tcur, t1)) : t1;
                const float tcc1 = x12 ? fminf(fmaxf(tc1, fminf(t1, t2)), fmaxf(t1, t2)) : t2;
                const float la = fabsf(__fsub_rn(tcc0, tcur)), lb = fabsf(__fsub_rn(t1, tcc0));
                const float lc = fabsf(__fsub_rn(tcc1, t1)), ld = fabsf(__fsub_rn(t2, tcc1));
                const float *p0 = pA + moff, *p1 = pA + moff + sA;
                if (ADJ) {
                    // only units inside the image receive anything (the border stays clean)
                    const unsigned NBu = bact ? (unsigned)W.NB : 1u;
                    const int rb = bact ? W.oB : 0;
                    const bool in0 = (unsigned)(rb + r0) < NBu, in1 = (unsigned)(rb + r1) < NBu,
                               in2 = (unsigned)(rb + r2) < NBu;
                    unit_op<true>(p0 + r0 * sB, act0 && in0, la, acc);
                    unit_op<true>(p0 + r1 * sB, act0 && x01 && in1, lb, acc);
                    unit_op<true>(p1 + r1 * sB, act1 && in1, lc, acc);
                    unit_op<true>(p1 + r2 * sB, act1 && x12 && in2, ld, acc);
                } else {
                    const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
                    const float4 va = act0 ? __ldg(reinterpret_cast<const float4 *>(p0 + r0 * sB)) : z;
                    const float4 vb = (act0 && x01) ? __ldg(reinterpret_cast<const float4 *>(p0 + r1 * sB)) : z;
                    const float4 vc = act1 ? __ldg(reinterpret_cast<const float4 *>(p1 + r1 * sB)) : z;
                    const float4 vd = (act1 && x12) ? __ldg(reinterpret_cast<const float4 *>(p1 + r2 * sB)) : z;
                    fma4(acc, va, la);
                    fma4(acc, vb, lb);
                    fma4(acc, vc, lc);
                    fma4(acc, vd, ld);
                }
            } else {
                // a step that crosses two rows (within rounding of a diagonal): per-candidate formula
                if (ADJ) {
                    if (act0)
                        scatter_rows_general(W.oB, W.NB, W.sgB, invB, bB, W.sgA ? t1 : tcur, W.sgA ? tcur : t1,
                                             (int)fminf(j0, j1), (int)fmaxf(j0, j1), pA - W.oB * sB + moff, sB, acc);
                    if (act1)
                        scatter_rows_general(W.oB, W.NB, W.sgB, invB, bB, W.sgA ? t2 : t1, W.sgA ? t1 : t2,
                                             (int)fminf(j1, j2), (int)fmaxf(j1, j2), pA - W.oB * sB + moff + sA, sB,
                                             acc);
                } else {
                if (act0) {
                    const float tlo = W.sgA ? t1 : tcur, thi = W.sgA ? tcur : t1;
                    const float4 a = slab_rows_general(W.oB, W.NB, W.sgB, invB, bB, tlo, thi, (int)fminf(j0, j1),
                                                       (int)fmaxf(j0, j1), pA - W.oB * sB + moff, sB);
                    acc.x += a.x; acc.y += a.y; acc.z += a.z; acc.w += a.w;
                }
                if (act1) {
                    const float tlo = W.sgA ? t2 : t1, thi = W.sgA ? t1 : t2;
                    const float4 a = slab_rows_general(W.oB, W.NB, W.sgB, invB, bB, tlo, thi, (int)fminf(j1, j2),
                                                       (int)fmaxf(j1, j2), pA - W.oB * sB + moff + sA, sB);
                    acc.x += a.x; acc.y += a.y; acc.z += a.z; acc.w += a.w;
                }
                }
            }
            p += 2.0f;
            tcur = t2;
            sm = s2;
            j0 = j2;
        }
    } else if (general) {
        Walk W2;
        if (ADJ) {
            Il4ScatterVisitor vis{const_cast<float *>(il), acc};
            if (walk_setup(rays[r], nx, ny, nz, si, sj, sk, W2)) walk(W2, vis);
        } else {
            Il4Visitor vis{il, make_float4(0.f, 0.f, 0.f, 0.f)};
            if (walk_setup(rays[r], nx, ny, nz, si, sj, sk, W2)) walk(W2, vis);
            acc = vis.acc;
        }
    }
    if (!ADJ && r < n_rays) {
        const int b0 = chunk * Bp + 4 * q;
        if (b0 + 0 < batch) sino[(int64_t)(b0 + 0) * n_rays + r] = acc.x;
        if (b0 + 1 < batch) sino[(int64_t)(b0 + 1) * n_rays + r] = acc.y;
        if (b0 + 2 < batch) sino[(int64_t)(b0 + 2) * n_rays + r] = acc.z;
        if (b0 + 3 < batch) sino[(int64_t)(b0 + 3) * n_rays + r] = acc.w;
    }
}

// ---------------------------------------------------------------------------------------
// Per-ray plane constants of the gather adjoint (gather_stage_kernel below)
// ---------------------------------------------------------------------------------------

// Per-ray plane constants of both in-plane axes, t(plane q of axis a) = fma(q - o_a, inv_a, b_a),
// stored as two arrays so that a warp's loads of neighbouring rays are contiguous:
//     GA[r] = (inv_x, b_x, inv_y, b_y)   16 B
//     GB[r] = (o_x, o_y)                 8 B, the integer parts of the foot point (exact floats)
// A ray that misses the image, or is parallel to an axis, has inv_x == 0 or inv_y == 0 (a
// missing ray all zeros); those take the walk's own unit length.
constexpr size_t kGatherRecBytes = sizeof(float4) + sizeof(float2);

__global__ void gather_prep_kernel(const RayRec *__restrict__ rays, int64_t n_rays, float4 *__restrict__ ga,
                                   float2 *__restrict__ gb)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const RayRec R = rays[r];
    float4 a = make_float4(0.f, 0.f, 0.f, 0.f);
    if (!(R.flags & RAY_MISS)) {
        a.x = R.w0 != 0.f ? __frcp_rn(R.w0) : 0.f;
        a.y = __fmul_rn(-R.f0, a.x);
        a.z = R.w1 != 0.f ? __frcp_rn(R.w1) : 0.f;
        a.w = __fmul_rn(-R.f1, a.z);
    }
    ga[r] = a;
    gb[r] = make_float2((float)R.o0, (float)R.o1);
}

// ---------------------------------------------------------------------------------------
// Launchers
// ---------------------------------------------------------------------------------------

cudaError_t launch_scatter_fast2(const RayRec *rays, int64_t n_rays, int nx, int ny, int nz, float *acc0,
                                 float *acc1, size_t acc_bytes, int Bp, const float *sino, float *img, int batch,
                                 int block, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(acc0, 0, acc_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(acc1, 0, acc_bytes, s);
    if (e != cudaSuccess) return e;
    const int lpr = Bp / 4;
    const int64_t threads = n_rays * lpr;
    const int64_t warps = (threads + 31) / 32;
    const dim3 grid((unsigned)((warps * 32 + block - 1) / block), (unsigned)((batch + Bp - 1) / Bp));
    float *sv = const_cast<float *>(sino);
    if (lpr == 4) fwd_fast2_kernel<4, true><<<grid, block, 0, s>>>(rays, n_rays, nx, ny, nz, acc0, acc1, Bp, sv, batch);
    else if (lpr == 2) fwd_fast2_kernel<2, true><<<grid, block, 0, s>>>(rays, n_rays, nx, ny, nz, acc0, acc1, Bp, sv, batch);
    else fwd_fast2_kernel<1, true><<<grid, block, 0, s>>>(rays, n_rays, nx, ny, nz, acc0, acc1, Bp, sv, batch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int64_t n = (int64_t)nx * ny * nz;
    deinterleave_sum_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)((batch + Bp - 1) / Bp)), 256, 0, s>>>(
        acc0, acc1, batch, nx, ny, nz, Bp, img);
    return cudaGetLastError();
}

cudaError_t launch_deinterleave_sum(const float *acc0, const float *acc1, int batch, int nx, int ny, int nz, int Bp,
                                    float *img, cudaStream_t s)
{
    const int64_t n = (int64_t)nx * ny * nz;
    deinterleave_sum_kernel<<<dim3((unsigned)((n + 255) / 256), (unsigned)((batch + Bp - 1) / Bp)), 256, 0, s>>>(
        acc0, acc1, batch, nx, ny, nz, Bp, img);
    return cudaGetLastError();
}

cudaError_t launch_gather_prep(const RayRec *rays, int64_t n_rays, void *grec, cudaStream_t s)
{
    float4 *ga = reinterpret_cast<float4 *>(grec);
    gather_prep_kernel<<<(unsigned)((n_rays + 255) / 256), 256, 0, s>>>(rays, n_rays, ga,
                                                                        reinterpret_cast<float2 *>(ga + n_rays));
    return cudaGetLastError();
}

size_t gather_rec_bytes() { return kGatherRecBytes; }

}  // namespace xr

// =======================================================================================
// Quad-plane layout: one thread per ray (forward) or per pair of pixels (gather) for all images.
//
// The images of the batch (padded to a multiple of 4) are stored as planes of 4 images:
// plane q holds images 4q..4q+3 as one float4 per unit, in the same two bordered spatial
// orders as above (IL0: x fastest, IL1: y fastest).  A thread walking a ray loads one float4
// per plane for every unit; the neighbouring rays of a warp load neighbouring float4s of
// the same plane, so every 128-bit load instruction is coalesced across the warp.  The walk
// geometry is computed once per ray for all images.
// =======================================================================================

namespace xr {

// user images [B][nz][ny][nx] -> planes [Q][padded units][4] in both orders.  The grid
// covers the padded units, so the zero border is rewritten on every call (the workspace is
// shared with the scatter adjoint's accumulators).
__global__ void interleave_planes_kernel(const float *__restrict__ img, int batch, int nx, int ny, int nz,
                                         float *__restrict__ il0, float *__restrict__ il1)
{
    const int px = nx + 2 * XR_IL_PAD, py = ny + 2 * XR_IL_PAD;
    const int64_t np = (int64_t)px * py * nz;
    const int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // padded unit in IL0 order
    if (u >= np) return;
    const int q = blockIdx.y;  // plane
    const int ip = (int)(u % px);
    const int64_t rest = u / px;
    const int jp = (int)(rest % py);
    const int k = (int)(rest / py);
    const int i = ip - XR_IL_PAD, j = jp - XR_IL_PAD;
    const int64_t n = (int64_t)nx * ny * nz;
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (i >= 0 && i < nx && j >= 0 && j < ny) {
        const int64_t uu = ((int64_t)k * ny + j) * nx + i;
        const int b = 4 * q;
        v.x = (b + 0 < batch) ? __ldg(img + (int64_t)(b + 0) * n + uu) : 0.f;
        v.y = (b + 1 < batch) ? __ldg(img + (int64_t)(b + 1) * n + uu) : 0.f;
        v.z = (b + 2 < batch) ? __ldg(img + (int64_t)(b + 2) * n + uu) : 0.f;
        v.w = (b + 3 < batch) ? __ldg(img + (int64_t)(b + 3) * n + uu) : 0.f;
    }
    const int64_t o0 = (int64_t)q * np + u;
    const int64_t o1 = (int64_t)q * np + ((int64_t)k * px + ip) * py + jp;
    reinterpret_cast<float4 *>(il0)[o0] = v;
    reinterpret_cast<float4 *>(il1)[o1] = v;
}

// Forward: one thread per ray, NQ planes (4*NQ images) per thread; blockIdx.y = group of
// NQ planes.  il0/il1: plane layout; sino: image b, ray r at sino[b * sb + r * sr] (the
// user layout: sb = n_rays, sr = 1).  ONLY_CROSS: a slab that stays in one row reads that row
// once (the second row's loads sit in a branch taken by the lanes that cross into it): the
// L1 data path, which bounds this kernel, then carries fewer bytes, at the cost of the branch
// -- faster for the single-tilt-axis column problems (C3 1.04 vs 1.12 ms), slower for the fan
// batch (1.20 vs 1.16 ms).
template <int NQ, bool ONLY_CROSS>
__global__ void __launch_bounds__(256, NQ >= 4 ? 3 : XR_FWD_MIN_BLOCKS) fwd_plane_kernel(const RayRec *__restrict__ rays,
                                                                           int64_t n_rays, int nx, int ny, int nz,
                                                                           const float4 *__restrict__ il0,
                                                                           const float4 *__restrict__ il1,
                                                                           int n_planes, float *__restrict__ sino,
                                                                           int batch, int sb, int sr)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int q0 = blockIdx.y * NQ;
    const int px = nx + 2 * XR_IL_PAD, py = ny + 2 * XR_IL_PAD;
    const int np = px * py * nz;  // padded units per plane (< 2^31 / 4, checked by the host)

    Walk W;
    bool ok = false;
    if (r < n_rays)
        ok = walk_setup(rays[r], nx, ny, nz, 1, nx, (int64_t)nx * ny, W) && W.nact <= 2 &&
             !(W.nact == 2 && W.axB == 2);
    const bool general = (r < n_rays) && !ok;
    const int axA0 = __shfl_sync(0xffffffffu, ok ? W.axA : 1, 0);
    const bool y_fast = (axA0 == 0);
    const int si = y_fast ? py : 1, sj = y_fast ? 1 : px, sk = px * py;
    const float4 *il = (y_fast ? il1 : il0) + (int64_t)q0 * np + XR_IL_PAD * (si + sj);
    const float4 *zero_unit = il - XR_IL_PAD * (si + sj);  // padded origin of each plane: zero

    float4 acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    const int wlo = __reduce_min_sync(0xffffffffu, ok ? W.mlo : INT_MAX);
    const int whi = __reduce_max_sync(0xffffffffu, ok ? W.mhi : INT_MIN);
    if (ok) {
        const int sA = sel3(W.axA, si, sj, sk), sB = sel3(W.axB, si, sj, sk), sC = sel3(W.axC, si, sj, sk);
        const float4 *pA = il + (W.oC * sC + W.oB * sB);
        const float invA = W.invA, bA = W.bA, wB = W.wB, fB = W.fB, invB = W.invB, bB = W.bB;
        const int mlo = W.mlo, mhi = W.mhi;
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
            const int rc = __float_as_int(sc) - kMagicBits, rn = __float_as_int(sn) - kMagicBits;
            const bool act = m >= mlo && m <= mhi;
            if (fabsf(jn - jc) < 1.5f) {
                const bool cross = rn != rc;
                const float tc = __fmaf_rn(fmaxf(jc, jn), invB, bB);
                const float tcc = cross ? fminf(fmaxf(tc, fminf(tcur, tn)), fmaxf(tcur, tn)) : tn;
                const float lc = fabsf(__fsub_rn(tcc, tcur)), ln = fabsf(__fsub_rn(tn, tcc));
                // Unpredicated loads: a lane outside its slab range reads the zero border unit
                // at the padded origin, and a slab that stays in one row reads that row twice
                // with ln == 0.  (Predicated loads with zeroed destinations: 34% more
                // instructions and register spills, 1.255 vs 1.157 ms at fan beam 512^2 x 16.)
                const float4 *pc = act ? pA + moff + rc * sB : zero_unit;
                const float4 *pn = act ? pA + moff + rn * sB : zero_unit;
                if (ONLY_CROSS) {
                // the second row only where the lane's slab crosses into it (ln > 0 only there)
                float4 vc[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) vc[q] = __ldg(pc + (int64_t)q * np);
#pragma unroll
                for (int q = 0; q < NQ; ++q) fma4(acc[q], vc[q], lc);
                if (cross && act) {
                    float4 vn[NQ];
#pragma unroll
                    for (int q = 0; q < NQ; ++q) vn[q] = __ldg(pn + (int64_t)q * np);
#pragma unroll
                    for (int q = 0; q < NQ; ++q) fma4(acc[q], vn[q], ln);
                }
                } else {
                float4 vc[NQ], vn[NQ];
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    vc[q] = __ldg(pc + (int64_t)q * np);
                    vn[q] = __ldg(pn + (int64_t)q * np);
                }
#pragma unroll
                for (int q = 0; q < NQ; ++q) {
                    fma4(acc[q], vc[q], lc);
                    fma4(acc[q], vn[q], ln);
                }
                }
            } else if (act) {
                // crossing two rows (within rounding of a diagonal): per-candidate formula
                const float tlo = W.sgA ? tn : tcur, thi = W.sgA ? tcur : tn;
                const int jlo = (int)fminf(jc, jn), jhi = (int)fmaxf(jc, jn);
                for (int j = jlo; j <= jhi; ++j) {
                    const int jg = j + W.oB;
                    if ((unsigned)jg >= (unsigned)W.NB) continue;
                    const float qq = (float)j;
                    const float tb0 = __fmaf_rn(qq + (float)W.sgB, invB, bB);
                    const float tb1 = __fmaf_rn(qq + (float)(1 - W.sgB), invB, bB);
                    const float l = __fsub_rn(fminf(thi, tb1), fmaxf(tlo, tb0));
                    if (l > 0.f) {
#pragma unroll
                        for (int q = 0; q < NQ; ++q) fma4(acc[q], __ldg(pA + moff + j * sB + (int64_t)q * np), l);
                    }
                }
            }
            tcur = tn;
            sc = sn;
            jc = jn;
        }
    } else if (general) {
        Walk W2;
        if (walk_setup(rays[r], nx, ny, nz, si, sj, sk, W2)) {
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                Il4Visitor vis{reinterpret_cast<const float *>(il + (int64_t)q * np), make_float4(0.f, 0.f, 0.f, 0.f)};
                // the visitor indexes floats: scale the unit strides by 4
                Walk W4 = W2;
                W4.sA *= 4;
                W4.sB *= 4;
                W4.sC *= 4;
                W4.base *= 4;
                walk(W4, vis);
                acc[q] = vis.acc;
            }
        }
    }
    if (r < n_rays) {
        float *out = sino + r * (int64_t)sr;
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
            const int b = 4 * (q0 + q);
            if (b + 0 < batch) out[(int64_t)(b + 0) * sb] = acc[q].x;
            if (b + 1 < batch) out[(int64_t)(b + 1) * sb] = acc[q].y;
            if (b + 2 < batch) out[(int64_t)(b + 2) * sb] = acc[q].z;
            if (b + 3 < batch) out[(int64_t)(b + 3) * sb] = acc[q].w;
        }
    }
}

// Gather adjoint: one thread per pair of horizontally adjacent pixels (i, j), (i+1, j) of one
// row (the last pixel of an odd row alone), all 4*NQ images of a group.  Per view the thread
// projects the pair's box (its four corners) onto the detector; for every bin whose centre lies
// in that footprint it reads the ray's plane constants and the bin's NQ sinogram quads once and
// adds l * g to both pixels.  The lengths are C_up - C_low of each pixel from the same plane
// crossings the forward uses (x planes i, i+1, i+2 and y planes j, j+1, each one FMA); a bin
// that misses a pixel gives C_up <= C_low there and adds nothing.
//
// The views are split into nch chunks inside each CTA of 256 threads, each warp on one chunk.
// The chunks' sums are added in chunk order through shared memory by the chunk-0 threads, so
// the result does not depend on scheduling.  nch multiplies the threads of the launch; the
// host picks it so that the CTAs fill whole waves of the GPU (512^2 pairs on 152 SMs: 1.68
// waves of one-chunk CTAs).
constexpr int kGatherThreads = 256;

// Where image b of the gather goes: the user layout ([b][rows][nx]) when slice_of is NULL;
// otherwise the y-slice slice_of[b] of a volume [rows][ny][nx] (slice stride nx, row stride
// ny * nx), nothing for slice_of[b] < 0.
struct ImgMap {
    const int *slice_of;
    int64_t slice_stride, row_stride;
    __device__ __forceinline__ int64_t image(int b, int n_pix) const
    {
        if (!slice_of) return (int64_t)b * n_pix;
        const int sl = __ldg(slice_of + b);
        return sl < 0 ? -1 : (int64_t)sl * slice_stride;
    }
    __device__ __forceinline__ int64_t row(int nx) const { return slice_of ? row_stride : nx; }
};

// ---------------------------------------------------------------------------------------
// Staged gather: the per-view data of a warp's pixel tile in shared memory
// ---------------------------------------------------------------------------------------
//
// The bins' data come from gather records: record r of group y holds the group's NQ quads of
// sinogram values of ray r, then GA[r] and GB[r], padded to an odd number of 16-byte words
// (rec_words), so that the
// records of neighbouring bins start in different bank groups of shared memory.  A warp owns an
// 8 x 8 pixel tile (4 pairs x 8 rows, lane = pair (lane & 3) of row (lane >> 2)) and walks its
// chunk of views; for each view the union of the lanes' candidate bins is one range [cA, cA +
// nb) of that view's records, which one bulk asynchronous copy (cp.async.bulk, completion
// counted in bytes on an mbarrier) brings into a shared-memory stage.  kGStages stages per warp
// keep the next view's copy in flight while the lanes read the current one, so the inner loop
// waits on shared memory, not on L2.  A view whose range exceeds kGStageBins bins (steep
// magnification, fine detector) is read from the records in global memory directly.  Waits are
// bounded (kWaitCycles); a wait that runs out sets XR_DEVERR_WAIT_BOUND in the error word, and
// the warp stops, waits (bounded) for the copies it still has in flight and writes NaN sums for
// its pixels.
//
// Measured on the fan beam 512^2 x 16 images: 1.53 ms, against 1.95 ms for the same sums with
// every bin's data loaded from L2 (one pair per thread, 32 pairs of a row per warp: 4.7
// long-scoreboard stalls per issued instruction at 25% occupancy) and 1.81 ms with six copies
// per view (sinogram planes and constants as separate arrays).  Two stages per warp measured
// as fast as three or four; two bins per loop step (128 registers) and an interval footprint
// (two reciprocals instead of four corner divisions, 30% more candidate bins) were slower.
constexpr int kGStageBins = 32;  // bins per staged view: 8 x 8 pixels of C2 project onto <= 25
#ifndef XR_GATHER_STAGES
#define XR_GATHER_STAGES 2
#endif
constexpr int kGStages = XR_GATHER_STAGES;  // views per warp in flight or being read
constexpr long long kWaitCycles = 4000000000ll;  // about 2 s at 2 GHz

// 16-byte words of one gather record: NQ quads, GA, GB (+ padding to an odd count)
template <int NQ>
__host__ __device__ constexpr int rec_words()
{
    return (NQ + 2) | 1;
}

template <int NQ>
struct GStage {
    // per warp and stage: kGStageBins records; header: the mbarriers, (cA, nb) and the lanes' bin
    // ranges
    static constexpr int kBytes = kGStageBins * rec_words<NQ>() * 16;
    static constexpr int kWarps = kGatherThreads / 32;
    static constexpr int kMeta = kWarps * kGStages * 8;
    static constexpr int kRange = kMeta + kWarps * kGStages * 16;
    static constexpr int kHeader = kRange + kWarps * kGStages * 32 * 8;
    static constexpr int kSmem = kHeader + kWarps * kGStages * kBytes;
};

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// The waiting thread is suspended until the phase completes or the hint (1 ms) runs out, so a
// warp that waits for its copies issues nothing meanwhile.
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, unsigned parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity), "r"(1000000u)
        : "memory");
    return done != 0;
}

// true when the phase with this parity completed; false after `limit` SM clock cycles
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, unsigned parity, long long limit = kWaitCycles)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait(bar, parity))
        if (clock64() - t0 > limit) return false;
    return true;
}

// Called by the whole warp with the same operands in every lane; one lane, the one elect.sync
// picks, arrives on the stage's mbarrier expecting `bytes` and issues the copy of `bytes`
// (> 0, a multiple of 16) from global src to shared dst (both 16-byte aligned).
__device__ __forceinline__ void stage_copy_elect(void *dst, const void *src, unsigned bytes, uint64_t *bar)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "elect.sync _|p, 0xffffffff;\n\t"
        "@p mbarrier.arrive.expect_tx.shared::cta.b64 _, [%3], %2;\n\t"
        "@p cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n\t}" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

// The same without a copy: the stage's phase completes at once.
__device__ __forceinline__ void stage_arrive_elect(uint64_t *bar)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "elect.sync _|p, 0xffffffff;\n\t"
        "@p mbarrier.arrive.shared::cta.b64 _, [%0];\n\t}" ::"r"(smem_addr(bar))
        : "memory");
}

// Detector bins [c0, c1] (clamped to the detector) that the box (centre (xc, yc), half sizes
// (hx, hy)) projects onto in a view, widened by margin bins on each side.  The constants are
// FP32 copies made on the host (FP64 arithmetic in a kernel's prologue costs ~16 cycles per
// warp instruction on this GPU).
struct BinMap {
    float x_left, y_top, dx, dy;  // the image's left and top edges, unit sizes
    float sdd, u0, inv_du, half;  // detector: source distance, offset, 1 / spacing, (n_cols - 1) / 2
    int ncols;
};

static BinMap bin_map(const GeoParams &g)
{
    return BinMap{(float)(g.cx - 0.5 * g.nx * g.dx), (float)(g.cy + 0.5 * g.ny * g.dy), (float)g.dx, (float)g.dy,
                  (float)g.sdd, (float)g.u0, (float)(1.0 / g.du), 0.5f * (float)(g.n_cols - 1), g.n_cols};
}

template <int KIND>
__device__ __forceinline__ void box_bins(const float4 e0, const float4 e1, float xc, float yc, float hx, float hy,
                                         const BinMap &bm, float margin, int &c0, int &c1)
{
    float umin, umax;
    if (KIND == XR_PAR2D) {
        const float uc = e0.x * xc + e0.y * yc, hw = fabsf(e0.x) * hx + fabsf(e0.y) * hy;
        umin = uc - hw;
        umax = uc + hw;
    } else {
        // the projections of the box's four corners from the source (exact footprint)
        const float rx = xc - e0.x, ry = yc - e0.y;
        const float depth = rx * e0.z + ry * e0.w, lat = rx * e1.x + ry * e1.y;
        const float dpx = hx * e0.z, dpy = hy * e0.w, dlx = hx * e1.x, dly = hy * e1.y;
        const float a0 = __fdividef(lat - dlx - dly, depth - dpx - dpy);
        const float a1 = __fdividef(lat + dlx - dly, depth + dpx - dpy);
        const float a2 = __fdividef(lat - dlx + dly, depth - dpx + dpy);
        const float a3 = __fdividef(lat + dlx + dly, depth + dpx + dpy);
        const float a = fminf(fminf(a0, a1), fminf(a2, a3)), b = fmaxf(fmaxf(a0, a1), fmaxf(a2, a3));
        if (KIND == XR_FAN2D) {
            umin = bm.sdd * a;
            umax = bm.sdd * b;
        } else {
            umin = atanf(a);
            umax = atanf(b);
        }
    }
    const float c0f = fminf(fmaxf((umin - bm.u0) * bm.inv_du + bm.half - margin, -1.0f), 4.0e6f);
    const float c1f = fminf(fmaxf((umax - bm.u0) * bm.inv_du + bm.half + margin, -1.0f), 4.0e6f);
    c0 = max(__float_as_int(__fadd_ru(c0f, kMagic)) - kMagicBits, 0);
    c1 = min(__float_as_int(__fadd_rd(c1f, kMagic)) - kMagicBits, bm.ncols - 1);
}

// One candidate bin of a pixel pair: the lengths of ray r in pixels (i, j) and (i + 1, j) from
// the ray's plane constants (ga, gb), spread with the bin's NQ quads of sinogram values.
template <int NQ>
__device__ __forceinline__ void pair_bin(const float4 ga, const float2 gb, const float4 (&sv)[NQ], float fi, float fj,
                                         int i, int j, bool hasB, const RayRec *__restrict__ rays, int r, int nx, int ny,
                                         float4 (&accA)[NQ], float4 (&accB)[NQ])
{
    float la, lb;
    if (ga.x != 0.f && ga.z != 0.f) {
        // plane crossings t = fma(q - o, 1/w, -f/w): x planes i, i+1, i+2; y planes j, j+1
        const float qx = fi - gb.x, qy = fj - gb.y;
        const float tx0 = __fmaf_rn(qx, ga.x, ga.y), tx1 = __fmaf_rn(qx + 1.0f, ga.x, ga.y);
        const float tx2 = __fmaf_rn(qx + 2.0f, ga.x, ga.y);
        const float ty0 = __fmaf_rn(qy, ga.z, ga.w), ty1 = __fmaf_rn(qy + 1.0f, ga.z, ga.w);
        const float ylo = fminf(ty0, ty1), yhi = fmaxf(ty0, ty1);
        la = __fsub_rn(fminf(fmaxf(tx0, tx1), yhi), fmaxf(fminf(tx0, tx1), ylo));
        lb = __fsub_rn(fminf(fmaxf(tx1, tx2), yhi), fmaxf(fminf(tx1, tx2), ylo));
    } else {
        // a ray parallel to an axis: the walk's own unit lengths (rare)
        la = lb = 0.f;
        Walk W;
        if (walk_setup(rays[r], nx, ny, 1, 1, nx, (int64_t)nx * ny, W)) {
            la = walk_unit_length(W, i, j, 0);
            if (hasB) lb = walk_unit_length(W, i + 1, j, 0);
        }
    }
    la = la > 0.f ? la : 0.f;
    lb = (hasB && lb > 0.f) ? lb : 0.f;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        fma4(accA[q], sv[q], la);
        fma4(accB[q], sv[q], lb);
    }
}

// pair_bin for a ray that is not parallel to an axis (a missing ray gives 0): the plane
// crossings only.  x2: 2 for a pair, 1 for a lone last pixel (then pixel B's length is 0).
template <int NQ>
__device__ __forceinline__ void pair_bin_planes(const float4 ga, const float4 gb, const float4 *sv, float fi, float fj,
                                                float x2, float4 (&accA)[NQ], float4 (&accB)[NQ])
{
    const float qx = fi - gb.x, qy = fj - gb.y;
    const float tx0 = __fmaf_rn(qx, ga.x, ga.y), tx1 = __fmaf_rn(qx + 1.0f, ga.x, ga.y);
    const float tx2 = __fmaf_rn(qx + x2, ga.x, ga.y);
    const float ty0 = __fmaf_rn(qy, ga.z, ga.w), ty1 = __fmaf_rn(qy + 1.0f, ga.z, ga.w);
    const float ylo = fminf(ty0, ty1), yhi = fmaxf(ty0, ty1);
    const float la = fmaxf(__fsub_rn(fminf(fmaxf(tx0, tx1), yhi), fmaxf(fminf(tx0, tx1), ylo)), 0.f);
    const float lb = fmaxf(__fsub_rn(fminf(fmaxf(tx1, tx2), yhi), fmaxf(fminf(tx1, tx2), ylo)), 0.f);
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        fma4(accA[q], sv[q], la);
        fma4(accB[q], sv[q], lb);
    }
}

// The chunks' sums of one pair go to its chunk-0 thread in chunk order (red: [nch - 1][8 NQ]
// [ppc] floats), which writes the pair's pixels of every image of the group.
template <int NQ>
__device__ __forceinline__ void gather_finish(float4 (&accA)[NQ], float4 (&accB)[NQ], float *red, int nch, int chunk,
                                              int pl, int ppc, bool live, bool hasB, int i, int j, int q0, int batch,
                                              int nx, int n_pix, const ImgMap &om, float *__restrict__ img)
{
    if (nch > 1) {
        if (chunk > 0) {
            float *r = red + (size_t)(chunk - 1) * 8 * NQ * ppc + pl;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                r[(8 * q + 0) * ppc] = accA[q].x;
                r[(8 * q + 1) * ppc] = accA[q].y;
                r[(8 * q + 2) * ppc] = accA[q].z;
                r[(8 * q + 3) * ppc] = accA[q].w;
                r[(8 * q + 4) * ppc] = accB[q].x;
                r[(8 * q + 5) * ppc] = accB[q].y;
                r[(8 * q + 6) * ppc] = accB[q].z;
                r[(8 * q + 7) * ppc] = accB[q].w;
            }
        }
        __syncthreads();
        if (chunk > 0) return;
        for (int c = 1; c < nch; ++c) {
            const float *r = red + (size_t)(c - 1) * 8 * NQ * ppc + pl;
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                accA[q].x += r[(8 * q + 0) * ppc];
                accA[q].y += r[(8 * q + 1) * ppc];
                accA[q].z += r[(8 * q + 2) * ppc];
                accA[q].w += r[(8 * q + 3) * ppc];
                accB[q].x += r[(8 * q + 4) * ppc];
                accB[q].y += r[(8 * q + 5) * ppc];
                accB[q].z += r[(8 * q + 6) * ppc];
                accB[q].w += r[(8 * q + 7) * ppc];
            }
        }
    }
    if (!live) return;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int b = 4 * (q0 + q);
        const float a4[4] = {accA[q].x, accA[q].y, accA[q].z, accA[q].w};
        const float b4[4] = {accB[q].x, accB[q].y, accB[q].z, accB[q].w};
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (b + k < batch) {
                const int64_t base = om.image(b + k, n_pix);
                if (base < 0) continue;
                float *o = img + base + (int64_t)j * om.row(nx) + i;
                o[0] = a4[k];
                if (hasB) o[1] = b4[k];
            }
        }
    }
}

// Gather records of group y = blockIdx.y (see the staged gather below) from the sinograms --
// value of image b, ray r at sino[b * sb + r * sr] -- and the plane constants; images past the
// batch read as zero.
template <int NQ>
__global__ void gather_records_kernel(const float *__restrict__ sino, int64_t sb, int64_t sr, int batch,
                                      int64_t n_rays, const RayRec *__restrict__ rays, const float4 *__restrict__ grec,
                                      float4 *__restrict__ rec)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    constexpr int W = rec_words<NQ>();
    float4 *o = rec + ((int64_t)blockIdx.y * n_rays + r) * W;
    const int b0 = 4 * NQ * (int)blockIdx.y;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        float v[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int b = b0 + 4 * q + k;
            v[k] = b < batch ? __ldg(sino + b * sb + r * sr) : 0.f;
        }
        o[q] = make_float4(v[0], v[1], v[2], v[3]);
    }
    const float4 ga = __ldg(grec + r);
    o[NQ] = ga;
    const float2 gb = __ldg(reinterpret_cast<const float2 *>(grec + n_rays) + r);
    // z = 1: a ray parallel to an axis, whose lengths only the walk gives (the plane-crossing
    // form gives 0 for it, as for a ray that misses the image)
    const bool walk = (ga.x == 0.f || ga.z == 0.f) && !(__ldg(&rays[r].flags) & RAY_MISS);
    o[NQ + 1] = make_float4(gb.x, gb.y, walk ? 1.f : 0.f, 0.f);
#pragma unroll
    for (int w = NQ + 2; w < W; ++w) o[w] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// CTA of 256 threads = tpc warp tiles x nch view chunks (tpc * nch = 8); warp w takes tile
// blockIdx.x * tpc + w % tpc (tiles row-major over the image, 8 x 8 pixels) and views
// [chunk * n_views / nch, (chunk + 1) * n_views / nch) of chunk w / tpc.  A view's staged bin
// range is the union of the lanes' own candidate ranges, which each lane computes once, when
// the view's copy is issued, and keeps in shared memory until it reads the stage.
template <int NQ, int KIND>
__global__ void __launch_bounds__(kGatherThreads, NQ >= 2 ? 2 : 3) gather_stage_kernel(
    const RayRec *__restrict__ rays, GeoParams g, BinMap bm, const float *__restrict__ vt,
    const float4 *__restrict__ rec, int64_t n_rays, float *__restrict__ img, int batch, int nch, ImgMap om,
    int *__restrict__ err)
{
    using L = GStage<NQ>;
    constexpr int W = rec_words<NQ>();
    extern __shared__ __align__(128) unsigned char gsm[];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tpc = (kGatherThreads / 32) / nch;
    const int chunk = warp / tpc, wt = warp - chunk * tpc;
    const int ppc = 32 * tpc, pl = wt * 32 + lane;
    const int tpr = (g.nx + 1) >> 1;  // pairs per row
    const int tiles_x = (tpr + 3) >> 2;
    const int tile = (int)blockIdx.x * tpc + wt;
    const int ty = tile / tiles_x, tx = tile - ty * tiles_x;
    const int pi = 4 * tx + (lane & 3), j = 8 * ty + (lane >> 2);
    const bool live = pi < tpr && j < g.ny;
    const int i = 2 * pi;
    const bool hasB = live && i + 1 < g.nx;
    const bool tile_live = 8 * ty < g.ny;  // warp-uniform
    const int n_pix = g.nx * g.ny;
    const int q0 = blockIdx.y * NQ;
    const float4 *R = rec + (int64_t)blockIdx.y * n_rays * W;
    const float4 *V4 = reinterpret_cast<const float4 *>(vt);
    const int ncols = bm.ncols;
    // the pair's box: centre and half sizes
    const float w = hasB ? 2.0f : 1.0f;
    const float fi = (float)i, fj = (float)j;
    const float xc = __fmaf_rn(fi + 0.5f * w, bm.dx, bm.x_left), yc = __fmaf_rn(-(fj + 0.5f), bm.dy, bm.y_top);
    const float hx = 0.5f * w * bm.dx, hy = 0.5f * bm.dy;
    const float x2 = w;  // the pair's right edge, in x planes from i
    float4 accA[NQ], accB[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) accA[q] = accB[q] = make_float4(0.f, 0.f, 0.f, 0.f);

    uint64_t *bar = reinterpret_cast<uint64_t *>(gsm) + warp * kGStages;
    int2 *meta = reinterpret_cast<int2 *>(gsm + L::kMeta) + warp * kGStages;
    int2 *rng = reinterpret_cast<int2 *>(gsm + L::kRange) + warp * kGStages * 32;
    unsigned char *stage0 = gsm + L::kHeader + (size_t)warp * kGStages * L::kBytes;
    const int v0 = (int)((int64_t)chunk * g.n_views / nch), v1 = (int)((int64_t)(chunk + 1) * g.n_views / nch);

    // stage s <- view v: the lanes' bin ranges and the records of their union [cA, cA + nb)
    auto issue = [&](int v, int s) {
        int c0 = INT_MAX, c1 = INT_MIN;
        if (live) {
            const float4 e0 = __ldg(V4 + 2 * v), e1 = __ldg(V4 + 2 * v + 1);
            box_bins<KIND>(e0, e1, xc, yc, hx, hy, bm, 1e-3f, c0, c1);
            if (c0 > c1) {
                c0 = INT_MAX;
                c1 = INT_MIN;
            }
        }
        rng[s * 32 + lane] = make_int2(c0, c1);
        const int cA = __reduce_min_sync(0xffffffffu, c0), cB = __reduce_max_sync(0xffffffffu, c1);
        const int nb = cB >= cA ? cB - cA + 1 : 0;
        const int code = nb > kGStageBins ? -1 : nb;  // bins staged; -1: read directly
        if (lane == 0) meta[s] = make_int2(cA, code);
        if (code > 0)
            stage_copy_elect(stage0 + s * L::kBytes, R + ((int64_t)v * ncols + cA) * W, (unsigned)(nb * W * 16),
                             bar + s);
        else
            stage_arrive_elect(bar + s);
    };

    if (tile_live) {
        if (lane == 0) {
            for (int s = 0; s < kGStages; ++s) mbar_init(bar + s, 1);
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
        __syncwarp();
        unsigned phase = 0, pending = 0;  // per stage: parity of its next completion; copies in flight
        bool dead = false;
        for (int s = 0; s < kGStages - 1 && v0 + s < v1; ++s) {
            issue(v0 + s, s);
            pending |= 1u << s;
        }
        int s = 0;
        for (int v = v0; v < v1; ++v) {
            __syncwarp();  // every lane is done with stage s - 1 (view v - 1)
            const int sn = s == 0 ? kGStages - 1 : s - 1;
            if (v + kGStages - 1 < v1) {
                issue(v + kGStages - 1, sn);
                pending |= 1u << sn;
            }
            const bool ok = mbar_wait_bounded(bar + s, (phase >> s) & 1u);
            if (!__all_sync(0xffffffffu, ok)) {
                dead = true;
                break;
            }
            phase ^= 1u << s;
            pending &= ~(1u << s);
            const int2 m = meta[s];
            const int2 cr = rng[s * 32 + lane];
            const int vb = v * ncols;
            // records of bins cr.x .. cr.y: in the stage (m.y > 0) or in global memory (m.y < 0)
            if (m.y > 0) {
                const float4 *st = reinterpret_cast<const float4 *>(stage0 + s * L::kBytes);
                // a ray of the staged range that needs the walk (lane k looks at record k)
                const bool walk = __any_sync(0xffffffffu, lane < m.y && st[lane * W + NQ + 1].z != 0.f);
                if (!walk) {
                    for (int c = cr.x; c <= cr.y; ++c) {
                        const float4 *o = st + (c - m.x) * W;
                        pair_bin_planes<NQ>(o[NQ], o[NQ + 1], o, fi, fj, x2, accA, accB);
                    }
                } else {
                    for (int c = cr.x; c <= cr.y; ++c) {
                        const float4 *o = st + (c - m.x) * W;
                        float4 sv[NQ];
#pragma unroll
                        for (int q = 0; q < NQ; ++q) sv[q] = o[q];
                        const float4 gb = o[NQ + 1];
                        pair_bin<NQ>(o[NQ], make_float2(gb.x, gb.y), sv, fi, fj, i, j, hasB, rays, vb + c, g.nx,
                                     g.ny, accA, accB);
                    }
                }
            } else if (m.y < 0) {
                for (int c = cr.x; c <= cr.y; ++c) {
                    const float4 *o = R + (int64_t)(vb + c) * W;
                    float4 sv[NQ];
#pragma unroll
                    for (int q = 0; q < NQ; ++q) sv[q] = __ldg(o + q);
                    const float4 gb = __ldg(o + NQ + 1);
                    pair_bin<NQ>(__ldg(o + NQ), make_float2(gb.x, gb.y), sv, fi, fj, i, j, hasB, rays, vb + c, g.nx,
                                 g.ny, accA, accB);
                }
            }
            s = s + 1 == kGStages ? 0 : s + 1;
        }
        if (dead) {
            // stop: wait (bounded) for this warp's copies still in flight
            if (lane == 0 && err) atomicOr(err, XR_DEVERR_WAIT_BOUND);
            for (int q = 0; q < kGStages; ++q)
                if ((pending >> q) & 1u) mbar_wait_bounded(bar + q, (phase >> q) & 1u);
            accA[0].x = __int_as_float(0x7fc00000);  // NaN in the sums of the warp's pixels
        }
    }
    __syncthreads();  // every warp is done with its stages: the chunk sums reuse them
    gather_finish<NQ>(accA, accB, reinterpret_cast<float *>(gsm + L::kHeader), nch, chunk, pl, ppc, live, hasB, i, j,
                      q0, batch, g.nx, n_pix, om, img);
}

cudaError_t launch_interleave_planes(const float *img, int batch, int nx, int ny, int nz, float *il0, float *il1,
                                     cudaStream_t s)
{
    const int64_t np = (int64_t)(nx + 2 * XR_IL_PAD) * (ny + 2 * XR_IL_PAD) * nz;
    const int Q = (batch + 3) / 4;
    interleave_planes_kernel<<<dim3((unsigned)((np + 255) / 256), Q), 256, 0, s>>>(img, batch, nx, ny, nz, il0, il1);
    return cudaGetLastError();
}

cudaError_t launch_project_plane(const RayRec *rays, int64_t n_rays, int nx, int ny, int nz, const float *il0,
                                 const float *il1, float *sino, int batch, int nq, cudaStream_t s, int64_t sb,
                                 int64_t sr, bool only_cross)
{
    const int Q = (batch + 3) / 4;
    const int groups = (Q + nq - 1) / nq;
    const dim3 grid((unsigned)((n_rays + 255) / 256), (unsigned)groups);
    const float4 *a = reinterpret_cast<const float4 *>(il0), *b = reinterpret_cast<const float4 *>(il1);
    if (sb < 0) {
        sb = n_rays;
        sr = 1;
    }
    // both strides fit 32 bits: n_rays < 2^31 and n_cols on the batched paths
    const int isb = (int)sb, isr = (int)sr;
#define XR_FP(NQV, OC) fwd_plane_kernel<NQV, OC><<<grid, 256, 0, s>>>(rays, n_rays, nx, ny, nz, a, b, Q, sino, batch, isb, isr)
    if (only_cross) {
        if (nq == 4) XR_FP(4, true);
        else if (nq == 2) XR_FP(2, true);
        else XR_FP(1, true);
    } else {
        if (nq == 4) XR_FP(4, false);
        else if (nq == 2) XR_FP(2, false);
        else XR_FP(1, false);
    }
#undef XR_FP
    return cudaGetLastError();
}

// View chunks per CTA of the gather: the CTAs of nch chunks take ceil(ctas / slots) waves of
// 1/nch of the per-pair work each; take the smallest nch within 5% of the best estimate
// (fewer chunks keep fewer views' sinogram rows in flight per SM).
static int gather_chunks(int64_t pairs, int groups, int blocks_per_sm, int n_views)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms <= 0)
        return 1;
    const double slots = (double)sms * blocks_per_sm;
    double cost[4];
    const int cand[4] = {1, 2, 4, 8};
    double best = 1e300;
    for (int k = 0; k < 4; ++k) {
        cost[k] = 1e300;
        if (cand[k] > n_views) continue;  // every chunk keeps at least one view
        const int ppc = kGatherThreads / cand[k];
        const double ctas = (double)((pairs + ppc - 1) / ppc) * groups;
        cost[k] = std::ceil(ctas / slots) / cand[k];
        best = std::min(best, cost[k]);
    }
    for (int k = 0; k < 4; ++k)
        if (cost[k] <= 1.05 * best) return cand[k];
    return 1;
}

// The bounded wait of the staged gather on an mbarrier that nothing completes (a test of its
// way out): one warp; out[0] = 1 when every lane gave up after `limit` cycles, 0 otherwise.
__global__ void wait_selftest_kernel(long long limit, int *__restrict__ out)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncwarp();
    const bool ok = mbar_wait_bounded(&bar, 0u, limit);
    const bool gave_up = __all_sync(0xffffffffu, !ok);
    if (threadIdx.x == 0) out[0] = gave_up ? 1 : 0;
}

cudaError_t launch_wait_selftest(long long limit, int *d_out, cudaStream_t s)
{
    wait_selftest_kernel<<<1, 32, 0, s>>>(limit, d_out);
    return cudaGetLastError();
}

// The staged kernel takes more than 48 KB of dynamic shared memory: opt in once per device.
template <int NQ, int KIND>
static cudaError_t stage_smem_optin()
{
    static std::atomic<unsigned long long> done{0};
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    const unsigned long long bit = 1ull << (dev & 63);
    if (done.load() & bit) return cudaSuccess;
    e = cudaFuncSetAttribute(gather_stage_kernel<NQ, KIND>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             GStage<NQ>::kSmem);
    if (e == cudaSuccess) done.fetch_or(bit);
    return e;
}

size_t gather_records_bytes(int batch, int nq, int64_t n_rays)
{
    const int Q = (batch + 3) / 4;
    const int groups = (Q + nq - 1) / nq;
    const int words = nq == 4 ? rec_words<4>() : (nq == 2 ? rec_words<2>() : rec_words<1>());
    return (size_t)groups * (size_t)n_rays * (size_t)words * 16;
}

cudaError_t launch_gather_staged(const RayRec *rays, const void *grec, const GeoParams &g, const float *vt,
                                 const float *sino, int64_t n_rays, float *img, int batch, int nq, void *recs,
                                 cudaStream_t s, int *err, int64_t sb, int64_t sr, const int *slice_of,
                                 int64_t slice_stride, int64_t row_stride)
{
    const ImgMap om{slice_of, slice_stride, row_stride};
    if (sb < 0) {
        sb = n_rays;
        sr = 1;
    }
    const int Q = (batch + 3) / 4;
    const int groups = (Q + nq - 1) / nq;
    const float4 *G = reinterpret_cast<const float4 *>(grec);
    float4 *Rw = reinterpret_cast<float4 *>(recs);
    const int64_t tiles = (int64_t)(((g.nx + 1) / 2 + 3) / 4) * ((g.ny + 7) / 8);
    const int nch = gather_chunks(32 * tiles, groups, nq >= 2 ? 2 : 3, g.n_views);  // 1, 2, 4 or 8
    const int tpc = (kGatherThreads / 32) / nch;
    const dim3 grid((unsigned)((tiles + tpc - 1) / tpc), (unsigned)groups);
    const dim3 rgrid((unsigned)((n_rays + 255) / 256), (unsigned)groups);
    const BinMap bm = bin_map(g);
    cudaError_t e = cudaSuccess;
#define XR_GS(NQV, K)                                                                                               \
    do {                                                                                                            \
        e = stage_smem_optin<NQV, K>();                                                                             \
        if (e != cudaSuccess) break;                                                                                \
        gather_records_kernel<NQV><<<rgrid, 256, 0, s>>>(sino, sb, sr, batch, n_rays, rays, G, Rw);                \
        gather_stage_kernel<NQV, K><<<grid, kGatherThreads, GStage<NQV>::kSmem, s>>>(rays, g, bm, vt, Rw, n_rays,  \
                                                                                     img, batch, nch, om, err);     \
    } while (0)
#define XR_GS_K(K)                     \
    do {                               \
        if (nq == 4) XR_GS(4, K);      \
        else if (nq == 2) XR_GS(2, K); \
        else XR_GS(1, K);              \
    } while (0)
    if (g.kind == XR_PAR2D) XR_GS_K(XR_PAR2D);
    else if (g.kind == XR_FAN2D) XR_GS_K(XR_FAN2D);
    else XR_GS_K(XR_FAN2D_ARC);
#undef XR_GS_K
#undef XR_GS
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

}  // namespace xr
