// Device core of the X-ray transform: ray records and the per-ray walk.
//
// A ray is kept in "index space": along axis a the continuous coordinate u_a runs over
// [0, N_a] and unit n covers [n, n+1] (x grows with i; y and z are flipped so that they
// grow with j and k, the orientation of Section 2.1 / Section 3.1).  Along the ray,
// u_a(t) = o_a + w_a t with t the physical length.  The integer part of the foot point o_a
// is kept apart from its fraction so that a plane crossing t = (q - o_a)/w_a keeps the
// full float precision even for a ray almost parallel to that axis's planes.
//
// The walk is the paper's method laid out for a GPU thread:
//   * the driving axis A is the one with the largest |w_a| (the paper drives with i;
//     Section 4.3 allows any index to drive), so each step of the driving index m moves
//     every other index by at most one;
//   * for each m, the valid indices of a minor axis are those whose open interval meets
//     the minor coordinate's range across the slab -- eq. restriction_j(_3D) and
//     eq. restriction_k_3D_1 -- evaluated as floor(u_B) at the slab's two planes;
//   * every candidate unit gets C_low = max of the three entering planes' t and
//     C_up = min of the three leaving planes' t (eq. conditions_3D_1) and is kept iff
//     C_low < C_up, with length C_up - C_low (eq. range_length_3D);
//   * an axis with w_a = 0 holds the ray in one family of grid planes: its index is the
//     one fixed by the ray-setup kernel with the ambiguity rule of Section 4.1, which
//     reduces the walk to the 2D case (Case 2) or to a run along one axis (Cases 3, 4).
//
// Every plane crossing is a single fused multiply-add of (plane index, 1/w, -frac/w), so
// the same (ray, unit) pair always yields the same float length, whichever kernel
// evaluates it (forward walk, scatter adjoint, gather adjoint, sparse-row export).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace xr {

// One ray in index space, 32 bytes.  Built in double precision by the ray-setup kernel.
struct __align__(16) RayRec {
    float w0, w1, w2;  // du_a/dt (0: the ray lies in one family of planes of axis a)
    float f0;          // fractional part of the foot-point coordinate along x
    float f1, f2;      // ... along y, z
    int16_t o0, o1, o2;  // integer part of the foot-point coordinate, or the fixed index (w == 0)
    int16_t flags;       // bit 0: the ray does not enter the image
};
static_assert(sizeof(RayRec) == 32, "RayRec layout");

enum { RAY_MISS = 1 };

// Fire-and-forget float add to global memory.  Written out because a pointer read from a
// struct or a work list is generic to the compiler, which then emits an atomic that returns
// the old value (and waits for it) instead of a reduction.
__device__ __forceinline__ void red_add(float *p, float v)
{
    asm volatile("red.global.add.f32 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "f"(v) : "memory");
}

// red_add(p, v) when len > 0, predicated inside the instruction: a C++ `if` around the asm
// becomes a divergent branch (with its reconvergence bookkeeping) where only some lanes add.
// Which is faster depends on how often the lanes add: the column-trace adjoint gained 1.6 %
// (cone 512^3: 217 vs 221 ms); the lockstep 2D adjoint, whose second reduction is rare, lost
// (64 uneven fans: 45.6 vs 38.1 ms) and keeps the branch.
__device__ __forceinline__ void red_add_if_pos(float *p, float v, float len)
{
    asm volatile(
        "{\n\t.reg .pred q;\n\tsetp.gt.f32 q, %2, 0f00000000;\n\t@q red.global.add.f32 [%0], %1;\n\t}" ::"l"(
            __cvta_generic_to_global(p)),
        "f"(v), "f"(len)
        : "memory");
}

// The same for four consecutive floats (16-byte aligned): one 128-bit vector reduction.
__device__ __forceinline__ void red_add4(float *p, float a, float b, float c, float d)
{
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(__cvta_generic_to_global(p)), "f"(a), "f"(b),
                 "f"(c), "f"(d)
                 : "memory");
}

template <class T>
__device__ __forceinline__ T sel3(int a, T x, T y, T z)
{
    return a == 0 ? x : (a == 1 ? y : z);
}

// The walk state of one ray, axes permuted to (A driving, B, C minor).
struct Walk {
    int nact;             // number of axes the ray is not parallel to (1..3)
    int axA, axB, axC;    // original axis (0 = x/i, 1 = y/j, 2 = z/k) of A, B, C
    int NA, NB, NC;
    int oA, oB, oC;
    int sgA, sgB, sgC;    // 1 when w < 0: the entering plane of unit n is n + 1
    float invA, bA;       // t(plane q) = fma(q - o, inv, b), b = -frac * inv
    float invB, bB, wB, fB;
    float invC, bC, wC, fC;
    int64_t sA, sB, sC;   // element strides of the axes in the image layout
    int64_t base;         // offset of the fixed indices
    int mlo, mhi;         // driving indices to visit
};

// Prepare the walk; false when the ray crosses no unit (then W.nact == 0 and walk() does
// nothing).  Strides sx, sy, sz give the image layout (1, nx, nx*ny for [nz][ny][nx]).
__device__ __forceinline__ bool walk_setup(const RayRec &r, int nx, int ny, int nz, int64_t sx,
                                           int64_t sy, int64_t sz, Walk &W)
{
    W.nact = 0;
    if (r.flags & RAY_MISS) return false;
    const bool a0 = r.w0 != 0.f, a1 = r.w1 != 0.f, a2 = r.w2 != 0.f;
    const int nact = (int)a0 + (int)a1 + (int)a2;
    if (nact == 0) return false;
    const float m0 = a0 ? fabsf(r.w0) : -1.f, m1 = a1 ? fabsf(r.w1) : -1.f, m2 = a2 ? fabsf(r.w2) : -1.f;
    const int A = (m0 >= m1 && m0 >= m2) ? 0 : (m1 >= m2 ? 1 : 2);
    int B = (A == 0) ? 1 : 0;
    int C = (A == 2) ? 1 : 2;
    if (!sel3(B, a0, a1, a2) && sel3(C, a0, a1, a2)) {
        const int t = B;
        B = C;
        C = t;
    }
    W.axA = A;
    W.axB = B;
    W.axC = C;
    W.NA = sel3(A, nx, ny, nz);
    W.NB = sel3(B, nx, ny, nz);
    W.NC = sel3(C, nx, ny, nz);
    W.oA = sel3(A, (int)r.o0, (int)r.o1, (int)r.o2);
    W.oB = sel3(B, (int)r.o0, (int)r.o1, (int)r.o2);
    W.oC = sel3(C, (int)r.o0, (int)r.o1, (int)r.o2);
    W.sA = sel3(A, sx, sy, sz);
    W.sB = sel3(B, sx, sy, sz);
    W.sC = sel3(C, sx, sy, sz);

    const float wA = sel3(A, r.w0, r.w1, r.w2), fA = sel3(A, r.f0, r.f1, r.f2);
    W.invA = __frcp_rn(wA);
    W.bA = __fmul_rn(-fA, W.invA);
    W.sgA = wA < 0.f;
    W.base = 0;
    W.invB = W.bB = W.wB = W.fB = 0.f;
    W.invC = W.bC = W.wC = W.fC = 0.f;
    W.sgB = W.sgC = 0;

    float tin = -INFINITY, tout = INFINITY;
    {
        const float t0 = __fmaf_rn((float)(0 - W.oA), W.invA, W.bA);
        const float t1 = __fmaf_rn((float)(W.NA - W.oA), W.invA, W.bA);
        tin = fmaxf(tin, fminf(t0, t1));
        tout = fminf(tout, fmaxf(t0, t1));
    }
    if (nact >= 2) {
        W.wB = sel3(B, r.w0, r.w1, r.w2);
        W.fB = sel3(B, r.f0, r.f1, r.f2);
        W.invB = __frcp_rn(W.wB);
        W.bB = __fmul_rn(-W.fB, W.invB);
        W.sgB = W.wB < 0.f;
        const float t0 = __fmaf_rn((float)(0 - W.oB), W.invB, W.bB);
        const float t1 = __fmaf_rn((float)(W.NB - W.oB), W.invB, W.bB);
        tin = fmaxf(tin, fminf(t0, t1));
        tout = fminf(tout, fmaxf(t0, t1));
    } else {
        if ((unsigned)W.oB >= (unsigned)W.NB) return false;
        W.base += (int64_t)W.oB * W.sB;
    }
    if (nact == 3) {
        W.wC = sel3(C, r.w0, r.w1, r.w2);
        W.fC = sel3(C, r.f0, r.f1, r.f2);
        W.invC = __frcp_rn(W.wC);
        W.bC = __fmul_rn(-W.fC, W.invC);
        W.sgC = W.wC < 0.f;
        const float t0 = __fmaf_rn((float)(0 - W.oC), W.invC, W.bC);
        const float t1 = __fmaf_rn((float)(W.NC - W.oC), W.invC, W.bC);
        tin = fmaxf(tin, fminf(t0, t1));
        tout = fminf(tout, fmaxf(t0, t1));
    } else {
        if ((unsigned)W.oC >= (unsigned)W.NC) return false;
        W.base += (int64_t)W.oC * W.sC;
    }
    if (!(tin < tout)) return false;
    // Driving indices spanned inside the image, with one slab of margin on each side.
    const float uin = __fmaf_rn(wA, tin, fA), uout = __fmaf_rn(wA, tout, fA);
    const int lo = (int)floorf(fminf(uin, uout)) + W.oA - 1;
    const int hi = (int)floorf(fmaxf(uin, uout)) + W.oA + 1;
    W.mlo = max(lo, 0);
    W.mhi = min(hi, W.NA - 1);
    if (W.mlo > W.mhi) return false;
    // only a complete setup makes the walk non-empty: on every early return nact stays 0
    W.nact = nact;
    return true;
}

// t of the entering / leaving planes of driving slab m.
__device__ __forceinline__ void slab_planes(const Walk &W, int m, float &tlo, float &thi)
{
    const float p = (float)(m - W.oA);
    const float t0 = __fmaf_rn(p, W.invA, W.bA);
    const float t1 = __fmaf_rn(p + 1.0f, W.invA, W.bA);
    tlo = W.sgA ? t1 : t0;
    thi = W.sgA ? t0 : t1;
}

// Walk the ray: vis(offset, length) for every unit with C_low < C_up.
template <int NACT, class V>
__device__ __forceinline__ void walk_run(const Walk &W, V &vis)
{
    float p = (float)(W.mlo - W.oA);
    float tcur = __fmaf_rn(p, W.invA, W.bA);
    float uB = 0.f, uC = 0.f;
    if (NACT >= 2) uB = __fmaf_rn(W.wB, tcur, W.fB);
    if (NACT == 3) uC = __fmaf_rn(W.wC, tcur, W.fC);
    int64_t offA = W.base + (int64_t)W.mlo * W.sA;
    for (int m = W.mlo; m <= W.mhi; ++m, offA += W.sA) {
        p += 1.0f;
        const float tnext = __fmaf_rn(p, W.invA, W.bA);
        const float tlo = W.sgA ? tnext : tcur;
        const float thi = W.sgA ? tcur : tnext;
        if (NACT == 1) {
            vis(offA, __fsub_rn(thi, tlo));
        } else {
            const float uBn = __fmaf_rn(W.wB, tnext, W.fB);
            const int j0 = (int)floorf(fminf(uB, uBn)), j1 = (int)floorf(fmaxf(uB, uBn));
            int k0 = 0, k1 = 0;
            float uCn = 0.f;
            if (NACT == 3) {
                uCn = __fmaf_rn(W.wC, tnext, W.fC);
                k0 = (int)floorf(fminf(uC, uCn));
                k1 = (int)floorf(fmaxf(uC, uCn));
            }
            for (int j = j0; j <= j1; ++j) {
                const int jg = j + W.oB;
                if ((unsigned)jg >= (unsigned)W.NB) continue;
                const float q = (float)j;
                const float tb0 = __fmaf_rn(q + (float)W.sgB, W.invB, W.bB);
                const float tb1 = __fmaf_rn(q + (float)(1 - W.sgB), W.invB, W.bB);
                const float lo = fmaxf(tlo, tb0), hi = fminf(thi, tb1);
                const int64_t offB = offA + (int64_t)jg * W.sB;
                if (NACT == 2) {
                    const float l = __fsub_rn(hi, lo);
                    if (l > 0.f) vis(offB, l);
                } else {
                    for (int k = k0; k <= k1; ++k) {
                        const int kg = k + W.oC;
                        if ((unsigned)kg >= (unsigned)W.NC) continue;
                        const float r = (float)k;
                        const float tc0 = __fmaf_rn(r + (float)W.sgC, W.invC, W.bC);
                        const float tc1 = __fmaf_rn(r + (float)(1 - W.sgC), W.invC, W.bC);
                        const float l = __fsub_rn(fminf(hi, tc1), fmaxf(lo, tc0));
                        if (l > 0.f) vis(offB + (int64_t)kg * W.sC, l);
                    }
                }
            }
            uB = uBn;
            if (NACT == 3) uC = uCn;
        }
        tcur = tnext;
    }
}

template <class V>
__device__ __forceinline__ void walk(const Walk &W, V &vis)
{
    if (W.nact == 3) walk_run<3>(W, vis);
    else if (W.nact == 2) walk_run<2>(W, vis);
    else if (W.nact == 1) walk_run<1>(W, vis);
}

// ---------------------------------------------------------------------------------------
// The 3D walk in crossing order.
//
// For a voxel, C_low is the largest of its three entering planes' t and C_up the smallest
// of its three leaving planes' t (eq. conditions_3D_1).  Visiting the voxels in the order
// the ray crosses planes gives both directly: C_low is the last plane crossed and C_up
// the nearest plane ahead, one per axis.  So the walk keeps, per axis, the t of the
// current voxel's leaving plane, takes the smallest, emits C_up - C_low when positive
// (the condition C_low < C_up: a tie of two planes gives a voxel of zero length, which is
// skipped), and steps that axis.  Every plane t is the same fused multiply-add
// (plane index - o) * (1/w) + (-frac/w) as in the slab walk, so each (ray, voxel) length
// is one well-defined float and the set of voxels is exactly those with C_low < C_up.
// An axis with w = 0 keeps its fixed index and never crosses a plane (t = +inf).
//
// The walk ends at tout, the box's exit (the nearest of the three exit planes, computed
// by the same expression as that plane's t in the walk).  Every voxel entered before tout
// lies inside the grid: an index leaves its range only by crossing its axis's exit plane,
// at a t >= tout.  From then on the clamped C_up = min(..., tout) equals C_low and every
// length is 0, so nothing outside the grid is ever read or written.
// ---------------------------------------------------------------------------------------

template <class Off>
struct Dda {
    float t0, t1, t2;     // t of the current voxel's leaving plane per axis (+inf: inactive)
    float q0, q1, q2;     // that plane's index minus the integer foot point, per axis
    float s0, s1, s2;     // +1 or -1: direction of travel per axis
    float i0, b0, i1, b1, i2, b2;  // plane t = fma(q, i, b)
    Off d0, d1, d2;       // signed offset step per axis
    Off off;              // offset of the current voxel
    float tcur;           // C_low of the current voxel
    float tout;           // exit from the grid
};

// Axis setup: plane constants and entry/exit of the index range [lo, hi) of this axis;
// false when the ray misses it (inactive axis with its fixed index outside the range).
__device__ __forceinline__ bool dda_axis(float w, float f, int o, int lo, int hi, float &inv, float &b, float &tin,
                                         float &tout)
{
    if (w == 0.f) {
        inv = 0.f;
        b = 0.f;
        return o >= lo && o < hi;
    }
    inv = __frcp_rn(w);
    b = __fmul_rn(-f, inv);
    const float ta = __fmaf_rn((float)(lo - o), inv, b);
    const float tb = __fmaf_rn((float)(hi - o), inv, b);
    tin = fmaxf(tin, fminf(ta, tb));
    tout = fminf(tout, fmaxf(ta, tb));
    return true;
}

// The voxel of this axis containing the start of the walk (just after tin) and its
// leaving plane.  Unit n of the axis spans planes n and n + 1; offsets count from lo.
template <class Off>
__device__ __forceinline__ void dda_start(float w, float f, int o, int lo, int hi, float inv, float b, float tin,
                                          Off stride, float &t, float &q, float &s, Off &d, Off &off)
{
    if (w == 0.f) {
        t = INFINITY;
        q = 0.f;
        s = 0.f;
        d = 0;
        off += (Off)(o - lo) * stride;
        return;
    }
    int n = (int)floorf(__fmaf_rn(w, tin, f)) + o;
    if (w > 0.f) {
        // want t(n) <= tin < t(n + 1)
#pragma unroll
        for (int it = 0; it < 2; ++it)
            if (__fmaf_rn((float)(n + 1 - o), inv, b) <= tin) ++n;
#pragma unroll
        for (int it = 0; it < 2; ++it)
            if (__fmaf_rn((float)(n - o), inv, b) > tin) --n;
        n = min(max(n, lo), hi - 1);
        q = (float)(n + 1 - o);
        s = 1.f;
        d = stride;
    } else {
        // planes ordered the other way: want t(n + 1) <= tin < t(n)
#pragma unroll
        for (int it = 0; it < 2; ++it)
            if (__fmaf_rn((float)(n - o), inv, b) <= tin) --n;
#pragma unroll
        for (int it = 0; it < 2; ++it)
            if (__fmaf_rn((float)(n + 1 - o), inv, b) > tin) ++n;
        n = min(max(n, lo), hi - 1);
        q = (float)(n - o);
        s = -1.f;
        d = -stride;
    }
    t = __fmaf_rn(q, inv, b);
    off += (Off)(n - lo) * stride;
}

// Prepare the walk through the box [lo0, hi0) x [lo1, hi1) x [lo2, hi2) of the grid (index
// planes are the grid's, so every voxel gets the same length as in a walk of the whole
// grid); offsets count from the box's first voxel with the given strides.  False when the
// ray crosses no voxel of the box.
template <class Off>
__device__ __forceinline__ bool dda_setup_box(const RayRec &r, int lo0, int hi0, int lo1, int hi1, int lo2, int hi2,
                                              Off sx, Off sy, Off sz, Dda<Off> &D)
{
    if (r.flags & RAY_MISS) return false;
    if (r.w0 == 0.f && r.w1 == 0.f && r.w2 == 0.f) return false;
    float tin = -INFINITY, tout = INFINITY;
    if (!dda_axis(r.w0, r.f0, r.o0, lo0, hi0, D.i0, D.b0, tin, tout)) return false;
    if (!dda_axis(r.w1, r.f1, r.o1, lo1, hi1, D.i1, D.b1, tin, tout)) return false;
    if (!dda_axis(r.w2, r.f2, r.o2, lo2, hi2, D.i2, D.b2, tin, tout)) return false;
    if (!(tin < tout)) return false;
    D.off = 0;
    dda_start(r.w0, r.f0, r.o0, lo0, hi0, D.i0, D.b0, tin, sx, D.t0, D.q0, D.s0, D.d0, D.off);
    dda_start(r.w1, r.f1, r.o1, lo1, hi1, D.i1, D.b1, tin, sy, D.t1, D.q1, D.s1, D.d1, D.off);
    dda_start(r.w2, r.f2, r.o2, lo2, hi2, D.i2, D.b2, tin, sz, D.t2, D.q2, D.s2, D.d2, D.off);
    D.tcur = tin;
    D.tout = tout;
    return true;
}

// The walk through the whole grid.
template <class Off>
__device__ __forceinline__ bool dda_setup(const RayRec &r, int nx, int ny, int nz, Off sx, Off sy, Off sz,
                                          Dda<Off> &D)
{
    return dda_setup_box<Off>(r, 0, nx, 0, ny, 0, nz, sx, sy, sz, D);
}

// Upper bound on the steps of one ray: one per voxel, at most nx + ny + nz + 1.
__device__ __forceinline__ int dda_max_steps(int nx, int ny, int nz) { return nx + ny + nz + 2; }

// One voxel: its length (0 once past the exit) and offset; then step to the next voxel.
// Returns the axis stepped (0, 1, 2; 3 once past the exit).
template <class Off>
__device__ __forceinline__ int dda_step(Dda<Off> &D, Off &off, float &l)
{
    const float tn = fminf(fminf(D.t0, D.t1), fminf(D.t2, D.tout));
    l = __fsub_rn(tn, D.tcur);
    off = D.off;
    D.tcur = fmaxf(D.tcur, tn);
    const bool c0 = D.t0 == tn, c1 = !c0 && D.t1 == tn, c2 = !c0 && !c1 && D.t2 == tn;
    D.off += c0 ? D.d0 : (c1 ? D.d1 : (c2 ? D.d2 : (Off)0));
    if (c0) {
        D.q0 += D.s0;
        D.t0 = __fmaf_rn(D.q0, D.i0, D.b0);
    }
    if (c1) {
        D.q1 += D.s1;
        D.t1 = __fmaf_rn(D.q1, D.i1, D.b1);
    }
    if (c2) {
        D.q2 += D.s2;
        D.t2 = __fmaf_rn(D.q2, D.i2, D.b2);
    }
    return c0 ? 0 : (c1 ? 1 : (c2 ? 2 : 3));
}

// The same step for a ray whose axis SKIP (1 or 2) has w = 0: that axis's leaving t is +inf
// and never the smallest, so leaving it out of the minimum and the selects changes nothing in
// the (offset, length) sequence -- it only saves the instructions.
template <int SKIP, class Off>
__device__ __forceinline__ void dda_step_skip(Dda<Off> &D, Off &off, float &l)
{
    static_assert(SKIP == 1 || SKIP == 2, "axis left out");
    const float ta = D.t0, tb = SKIP == 2 ? D.t1 : D.t2;
    const float tn = fminf(fminf(ta, tb), D.tout);
    l = __fsub_rn(tn, D.tcur);
    off = D.off;
    D.tcur = fmaxf(D.tcur, tn);
    const bool c0 = ta == tn, cb = !c0 && tb == tn;
    D.off += c0 ? D.d0 : (cb ? (SKIP == 2 ? D.d1 : D.d2) : (Off)0);
    if (c0) {
        D.q0 += D.s0;
        D.t0 = __fmaf_rn(D.q0, D.i0, D.b0);
    }
    if (cb) {
        if (SKIP == 2) {
            D.q1 += D.s1;
            D.t1 = __fmaf_rn(D.q1, D.i1, D.b1);
        } else {
            D.q2 += D.s2;
            D.t2 = __fmaf_rn(D.q2, D.i2, D.b2);
        }
    }
}

// dda_step with the axes the ray may cross fixed at compile time: SKIP = 0 keeps all three.
template <int SKIP, class Off>
__device__ __forceinline__ void dda_step_t(Dda<Off> &D, Off &off, float &l)
{
    if (SKIP == 0) dda_step(D, off, l);
    else dda_step_skip<SKIP == 0 ? 1 : SKIP>(D, off, l);
}

// Walk the ray: vis(offset, length) for every voxel with C_low < C_up, in crossing order.
template <class Off, class V>
__device__ __forceinline__ void dda_run(Dda<Off> &D, int max_steps, V &vis)
{
    for (int k = 0; k < max_steps && D.tcur < D.tout; ++k) {
        Off off;
        float l;
        dda_step(D, off, l);
        if (l > 0.f) vis(off, l);
    }
}

// Either walk, by the scan's dimension: the slab walk for 2D scans, the crossing-order
// walk for 3D scans.
template <class V>
__device__ __forceinline__ void walk_ray(const RayRec &r, int nx, int ny, int nz, int64_t sx, int64_t sy,
                                         int64_t sz, bool three, V &vis)
{
    if (three) {
        Dda<int64_t> D;
        if (dda_setup<int64_t>(r, nx, ny, nz, sx, sy, sz, D)) dda_run(D, dda_max_steps(nx, ny, nz), vis);
    } else {
        Walk W;
        if (walk_setup(r, nx, ny, nz, sx, sy, sz, W)) walk(W, vis);
    }
}

// Length of unit (i, j, k) exactly as walk_run computes it, or 0 when the walk does not
// visit it.  Used by the unit-driven (gather) adjoint.
__device__ __forceinline__ float walk_unit_length(const Walk &W, int i, int j, int k)
{
    const int m = sel3(W.axA, i, j, k), jg = sel3(W.axB, i, j, k), kg = sel3(W.axC, i, j, k);
    if (m < W.mlo || m > W.mhi) return 0.f;
    if (W.nact < 3 && kg != W.oC) return 0.f;
    if (W.nact < 2 && jg != W.oB) return 0.f;
    // identical to walk_run: plane m from p, plane m+1 from p + 1
    const float p = (float)(m - W.oA);
    const float tcur = __fmaf_rn(p, W.invA, W.bA);
    const float tnext = __fmaf_rn(p + 1.0f, W.invA, W.bA);
    const float tlo = W.sgA ? tnext : tcur;
    const float thi = W.sgA ? tcur : tnext;
    if (W.nact == 1) return __fsub_rn(thi, tlo);
    const float uB = __fmaf_rn(W.wB, tcur, W.fB), uBn = __fmaf_rn(W.wB, tnext, W.fB);
    const int jr = jg - W.oB;
    if (jr < (int)floorf(fminf(uB, uBn)) || jr > (int)floorf(fmaxf(uB, uBn))) return 0.f;
    const float q = (float)jr;
    const float tb0 = __fmaf_rn(q + (float)W.sgB, W.invB, W.bB);
    const float tb1 = __fmaf_rn(q + (float)(1 - W.sgB), W.invB, W.bB);
    const float lo = fmaxf(tlo, tb0), hi = fminf(thi, tb1);
    float l;
    if (W.nact == 3) {
        const float uC = __fmaf_rn(W.wC, tcur, W.fC), uCn = __fmaf_rn(W.wC, tnext, W.fC);
        const int kr = kg - W.oC;
        if (kr < (int)floorf(fminf(uC, uCn)) || kr > (int)floorf(fmaxf(uC, uCn))) return 0.f;
        const float r = (float)kr;
        const float tc0 = __fmaf_rn(r + (float)W.sgC, W.invC, W.bC);
        const float tc1 = __fmaf_rn(r + (float)(1 - W.sgC), W.invC, W.bC);
        l = __fsub_rn(fminf(hi, tc1), fmaxf(lo, tc0));
    } else {
        l = __fsub_rn(hi, lo);
    }
    return l > 0.f ? l : 0.f;
}

}  // namespace xr
