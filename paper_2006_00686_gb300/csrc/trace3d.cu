// Cone and helical scans walked column by column (circular and helical cone beams, flat and
// equiangular detectors; eq. equispaced_cone_beam, eq. equiangular_cone_beam,
// eq. Helical_cone_beam_equispaced, eq. Helical_cone_beam_equiangular).
//
// Every ray of one detector column in one view starts at the source S and ends on a vertical
// line of the detector, so all of them lie in one vertical plane.  Measured by the horizontal
// distance tau along that plane's trace, the rays share the x and y plane crossings: the
// sequence of (i, j) columns of voxels the trace crosses, with the tau of each crossing, is
// the same for every row.  Only the z crossings differ per row, and along tau each row's z
// is linear: z(tau) = z_F + t_z tau, with t_z the row's rise per unit horizontal distance.
// The physical length inside a voxel is the tau-length times sec = sqrt(1 + t_z^2).
//
// A warp takes one (view, column) and a block of 32 rows (one lane per row):
//   1. the trace: the xy-plane crossings of the vertical plane inside the image box, merged
//      in tau order into slabs (tau at the slab's end, column offset), laid out in chunks of
//      256 slots in the warp's shared memory.  Each lane places the crossings of its own
//      share of a chunk's tau range: a crossing's slot is its index plus the number of
//      crossings of the other family before it, counted exactly, so the lanes need no
//      communication beyond the chunk's first rank;
//   2. every lane walks the chunk's slabs in lockstep with the others: per slab, the voxel
//      index at the slab's two ends is floor(u_z) at those tau (a row crosses at most one
//      z plane per slab -- the host admits a scan only when max |t_z| x the longest slab
//      stays below one voxel), the z plane crossed inside the slab splits it into two
//      voxels A (entered) and B (left), and their lengths are C_up - C_low of eq.
//      conditions_3D_1 with the slab's xy planes and the z plane as the entering and leaving
//      planes.  A voxel with a zero length contributes nothing (the condition C_low < C_up).
// Warps run in the order (row block, part of the columns, view, column), so the rays in flight
// are one block of 32 rows in a few views: a thin slab of the volume that L2 holds (a band of
// 128 rows kept ~40 % of a 512^3 cone volume in flight and read it from DRAM ~27 times per
// launch).
// The lanes of a warp are neighbouring rows: at every slab they touch one (i, j) column of
// the z-fastest volume copy, at neighbouring heights, so their loads (forward) or
// reductions (adjoint) fall on a few neighbouring sectors.  The copy has one zero voxel above
// and below each column: a row outside the volume in z is clamped onto them, so rows that
// enter or leave through the top or bottom face need no extra test.  The forward reads the
// copy as pair columns (entry e holds voxels e and e + 1), so a slab's two voxels come in one
// 64-bit load: circular cone 512^3 174 vs 182 ms, helix 512^2 x 256 60 vs 69 ms.
//
// The adjoint adds g * sec * length into a z-fastest accumulator with one reduction per
// (row, voxel).  XR_TRACE_AGG=1 builds the warp-aggregated form instead: lanes whose B voxels
// coincide (rows closer than one voxel) first sum their values with a segmented shuffle
// reduction, and only the first lane of each run reduces (the rows are ordered, so equal
// voxels are neighbouring lanes).  Measured on GB300 it lost: the shuffles doubled the
// kernel's instructions while the reductions of a warp already fall on a few neighbouring
// sectors (circular cone 512^3: 494 vs 241 ms; helix 512^2 x 256: 219 vs 82 ms).
//
// Every geometric quantity of the trace and of a row is computed here from per-view,
// per-column and per-detector-sample tables (no per-ray table): the trace and the rows' foot
// points in float pairs (no FP64: its rate on GB300 is a small fraction of FP32), the walk in
// float with the integer parts of the foot point kept apart.
#include <algorithm>

#include "xray_df.cuh"
#include "xray_internal.h"

namespace xr {

namespace {

constexpr float kMagic = 12582912.0f;  // 1.5 * 2^23: x + kMagic (rounded down) holds floor(x) in its low bits
constexpr int kMagicBits = 0x4B400000;

// floor(w) for |w| < 2^22: the float kMagic + floor(w) (exact), whose bit pattern is
// kMagicBits + floor(w).
__device__ __forceinline__ float magic_floor(float w) { return __fadd_rd(w, kMagic); }

// Number of crossings of one family (plane tau = fma(q0 + a s, inv, b), a = 0, 1, ...)
// strictly before T (or_equal: at or before T), within [0, n]: an estimate from the family's
// rate (crossings per unit tau, |w|), then exact comparisons of the same expressions the slab
// list is built from.  Counts stay in float (exact below 2^24) and the estimate is truncated
// with the magic-number add, so no int/float conversion is needed.
__device__ __forceinline__ float count_before(float T, float q0, float s, float inv, float b, float rate, float n,
                                              bool or_equal)
{
    if (n <= 0.f) return 0.f;
    const float e = (T - __fmaf_rn(q0, inv, b)) * rate;
    // estimate: trunc(e) + 1 within [0, n]
    float k = !(e >= 0.f) ? 0.f : (e >= n ? n : __fadd_rz(__fadd_rz(e, 8388608.0f), -8388608.0f) + 1.0f);
    // exact: crossing k - 1 before T, crossing k not
#pragma unroll 1
    for (int it = 0; it < 8 && k < n; ++it) {
        const float tk = __fmaf_rn(__fmaf_rn(k, s, q0), inv, b);
        if (or_equal ? (tk <= T) : (tk < T)) k += 1.f;
        else break;
    }
#pragma unroll 1
    for (int it = 0; it < 8 && k > 0.f; ++it) {
        const float tk = __fmaf_rn(__fmaf_rn(k - 1.f, s, q0), inv, b);
        if (or_equal ? (tk > T) : (tk >= T)) k -= 1.f;
        else break;
    }
    return k;
}

// The xy trace of (view, column) in index space as a ray record with a fixed z (w2 = 0):
// u_x(tau) = o0 + f0 + w0 tau, u_y(tau) = o1 + f1 + w1 tau, tau = horizontal distance from
// the foot point F (the trace's point closest to the image centre).  Returns false when the
// trace misses the image.  tauF: distance of F from the source.  Float pairs throughout (the
// foot point's fraction needs about 37 bits).
__device__ __forceinline__ bool trace_record(const TraceGeo &T, const ViewDF &V, float4 cs, RayRec &r, DF &tauF)
{
    // horizontal direction at angle phi + alpha (angle-sum identities), source S
    const DF ca{cs.x, cs.y}, sa{cs.z, cs.w};
    DF hx = df_sub(df_mul(V.c1, ca), df_mul(V.s1, sa));
    DF hy = df_add(df_mul(V.s1, ca), df_mul(V.c1, sa));
    snap(hx, hy);
    const DF Sx = df_neg(df_mul(T.D, V.c1)), Sy = df_neg(df_mul(T.D, V.s1));
    tauF = df_add(df_mul(df_sub(T.cx, Sx), hx), df_mul(df_sub(T.cy, Sy), hy));
    const DF Fx = df_add(Sx, df_mul(tauF, hx)), Fy = df_add(Sy, df_mul(tauF, hy));
    // a trace farther from the centre than the image's half-diagonal misses it
    const float dxF = df_sub(Fx, T.cx).hi, dyF = df_sub(Fy, T.cy).hi;
    if (dxF * dxF + dyF * dyF > T.rxy2) return false;
    const DF u[2] = {df_mul(df_sub(Fx, T.x0), T.idx), df_mul(df_sub(T.y1, Fy), T.idy)};
    const DF w[2] = {df_mul(hx, T.idx), df_neg(df_mul(hy, T.idy))};
    const int N[2] = {T.nx, T.ny};
    float wf[2], ff[2];
    int oi[2];
    int flags = 0;
#pragma unroll
    for (int a = 0; a < 2; ++a) {
        if (df_is_zero(w[a])) {
            // the trace lies in one family of planes: the unit holding it, the bigger index on a
            // plane, the last unit on the far edge (Section 4.1)
            wf[a] = 0.f;
            ff[a] = 0.f;
            const bool below = u[a].hi < 0.f || (u[a].hi == 0.f && u[a].lo < 0.f);
            const bool above = u[a].hi > (float)N[a] || (u[a].hi == (float)N[a] && u[a].lo > 0.f);
            int fl;
            float fr;
            df_floor_frac(u[a], fl, fr);
            oi[a] = (below || above) ? 0 : min(fl, N[a] - 1);
            if (below || above) flags |= RAY_MISS;
        } else {
            wf[a] = __fadd_rn(w[a].hi, w[a].lo);
            df_floor_frac(u[a], oi[a], ff[a]);
        }
    }
    r.w0 = wf[0];
    r.w1 = wf[1];
    r.w2 = 0.f;
    r.f0 = ff[0];
    r.f1 = ff[1];
    r.f2 = 0.f;
    r.o0 = (int16_t)oi[0];
    r.o1 = (int16_t)oi[1];
    r.o2 = 0;
    r.flags = (int16_t)flags;
    return !(flags & RAY_MISS);
}

// The xy crossings of one trace: the families x and y of plane crossings strictly inside
// (tin, tout), crossing a of family x at fma(qx + a sx, ix, bx) (likewise y), and the start
// column (i0, j0).  One warp walks one trace; it lays the slabs out in chunks of kChunk slots
// in its shared memory, each chunk covering `span` of tau, which holds at most kChunk - 4
// crossings (the two families cross |w0| + |w1| planes per unit tau).
#ifndef XR_TRACE_CHUNK
#define XR_TRACE_CHUNK 256
#endif
#ifndef XR_TRACE_MINB
#define XR_TRACE_MINB 1
#endif
#ifndef XR_TRACE_ADJ_UNROLL
#define XR_TRACE_ADJ_UNROLL 2
#endif
#ifndef XR_TRACE_B_ALWAYS
#define XR_TRACE_B_ALWAYS 1
#endif
constexpr int kAdjUnroll = XR_TRACE_ADJ_UNROLL;
#ifndef XR_TRACE_FWD_MINB
#define XR_TRACE_FWD_MINB 8  // 64 registers: 32 warps per SM to hide the loads' latency
#endif
constexpr int kChunk = XR_TRACE_CHUNK;
#ifndef XR_TRACE_WPC
#define XR_TRACE_WPC 4
#endif
constexpr int kWarpsPerCta = XR_TRACE_WPC;  // a CTA takes kWarpsPerCta neighbouring columns

struct WTrace {
    float tin, tout;
    float qx, sx, ix, bx, rx;  // rx, ry: crossings per unit tau
    float qy, sy, iy, by, ry;
    int nxc, nyc, i0, j0, di, dj;
    float fnx, fny;  // nxc, nyc as floats
    float dl;    // tau covered by one lane's share of a chunk (span / 32)
    int nchunk;
};

__device__ __forceinline__ bool trace_setup(const TraceGeo &T, const RayRec &r, WTrace &W)
{
    Dda<int> D;
    if (!dda_setup_box<int>(r, 0, T.nx, 0, T.ny, 0, 1, 1, T.nx, 0, D)) return false;
    W.tin = D.tcur;
    W.tout = D.tout;
    W.qx = D.q0;
    W.sx = D.s0;
    W.ix = D.i0;
    W.bx = D.b0;
    W.rx = fabsf(r.w0);
    W.qy = D.q1;
    W.sy = D.s1;
    W.iy = D.i1;
    W.by = D.b1;
    W.ry = fabsf(r.w1);
    W.fnx = W.sx != 0.f ? count_before(D.tout, W.qx, W.sx, W.ix, W.bx, W.rx, (float)T.nx, false) : 0.f;
    W.fny = W.sy != 0.f ? count_before(D.tout, W.qy, W.sy, W.iy, W.by, W.ry, (float)T.ny, false) : 0.f;
    W.nxc = (int)W.fnx;
    W.nyc = (int)W.fny;
    W.i0 = D.off % T.nx;  // D.off = i0 + j0 nx
    W.j0 = D.off / T.nx;
    W.di = W.sx > 0.f ? 1 : (W.sx < 0.f ? -1 : 0);
    W.dj = W.sy > 0.f ? 1 : (W.sy < 0.f ? -1 : 0);
    const float span = (float)(kChunk - 4) / (W.rx + W.ry);  // rx + ry > 0: the trace is a line
    W.dl = span * (1.0f / 32.0f);
    const float n = ceilf((W.tout - W.tin) / span);
    W.nchunk = n >= 1.f ? (n < 1048576.f ? (int)n : 1048576) : 1;
    return true;
}

// z-fastest offset of the column before the crossing with cx x- and cy y-crossings behind it
__device__ __forceinline__ int col_offset(const TraceGeo &T, const WTrace &W, int cx, int cy)
{
    const int i = min(max(W.i0 + W.di * cx, 0), T.nx - 1), j = min(max(W.j0 + W.dj * cy, 0), T.ny - 1);
    return i * (T.nz + 2) + j * (T.nx * (T.nz + 2));
}

// Chunk c of the warp's slab list into slot[] (0 .. return value - 1): x = tau at the slab's
// end, y = the bits of its column offset.  Lane L places
// the crossings in its share [la, lb) of the chunk's tau: its starting counts are those
// strictly before la, and it steps through its crossings in order (x first on a tie).  Each
// slab ends at one crossing and is stored at that crossing's rank in the merged order minus the
// chunk's first rank; the last chunk adds the slab that ends at the exit.
__device__ __forceinline__ int build_chunk(const TraceGeo &T, const WTrace &W, int c, int lane, float2 *slot)
{
    const bool last = c == W.nchunk - 1;
    const int k = c * 32 + lane;
    const float la = __fmaf_rn((float)k, W.dl, W.tin);
    const float lb = (last && lane == 31) ? INFINITY : __fmaf_rn((float)(k + 1), W.dl, W.tin);
    float fx = count_before(la, W.qx, W.sx, W.ix, W.bx, W.rx, W.fnx, false);
    float fy = count_before(la, W.qy, W.sy, W.iy, W.by, W.ry, W.fny, false);
    // the next plane of each family: q + count * s (exact small integers in float)
    float qxc = __fmaf_rn(fx, W.sx, W.qx), qyc = __fmaf_rn(fy, W.sy, W.qy);
    int cx = (int)fx, cy = (int)fy;
    const int base = __shfl_sync(0xffffffffu, cx + cy, 0);
#pragma unroll 1
    for (int it = 0; it < kChunk; ++it) {
        const float tx = cx < W.nxc ? __fmaf_rn(qxc, W.ix, W.bx) : INFINITY;
        const float ty = cy < W.nyc ? __fmaf_rn(qyc, W.iy, W.by) : INFINITY;
        const float t = fminf(tx, ty);
        if (!(t < lb)) break;
        const int k2 = cx + cy - base;
        if (k2 >= 0 && k2 < kChunk) slot[k2] = make_float2(t, __int_as_float(col_offset(T, W, cx, cy)));
        if (tx <= ty) {
            ++cx;
            qxc += W.sx;
        } else {
            ++cy;
            qyc += W.sy;
        }
    }
    int n = __shfl_sync(0xffffffffu, cx + cy, 31) - base;
    if (last) {
        if (lane == 0 && n >= 0 && n < kChunk)
            slot[n] = make_float2(W.tout, __int_as_float(col_offset(T, W, W.nxc, W.nyc)));
        ++n;
    }
    __syncwarp();
    return min(max(n, 0), kChunk);
}

// One row, in a z index u that grows along the walk: u(tau) = oz + fz + ez tau with ez >= 0.
// For a row whose index u_z (counting down in z) falls along tau, u = nz - u_z: the column is
// read from its other end.  Voxel m of u (unit [m, m + 1]) is at offset
//   zs * (kMagicBits + m - oz) + C   (mod 2^32)
// of its padded column, zs = 1 (C = oz - kMagicBits + 1) or zs = -1 (C = nz - oz + kMagicBits),
// so that the magic float of floor(w) gives the offset with one multiply-add.  Clamped to
// [-0.5, nz + 0.5], rows outside the volume fall on the zero voxels m = -1 and m = nz.
// inside: w stays in [-1 - oz, nz + 1 - oz) over the whole trace, so no clamp is needed.
struct Row {
    float ez, fz, iez, bz, lo, hi, sec;
    unsigned zs, C;
    bool live, inside;
};

__device__ __forceinline__ Row make_row(const TraceGeo &T, const ViewDF &V, int col, int row, DF tauF,
                                        float tin, float tout)
{
    Row R;
    R.live = row < T.n_rows;
    const float2 tzp = R.live ? T.tz[(size_t)row * T.n_cols + col] : make_float2(0.f, 0.f);
    const DF tz{tzp.x, tzp.y};
    DF uz = df_mul(df_sub(T.z1, df_add(V.H, df_mul(tz, tauF))), T.idz);
    // a row this far from the volume (2^20 voxels) cannot reach it within the trace (|u_z|
    // changes by less than nx + ny along it); bounding u_z keeps every w below 2^22, the range
    // of magic_floor
    if (fabsf(uz.hi) > 1048576.f) uz = DF{copysignf(1048576.f, uz.hi), 0.f};
    const DF ezd = df_neg(df_mul(tz, T.idz));
    float ez = __fadd_rn(ezd.hi, ezd.lo);
    if (fabsf(ez) < 1e-20f) ez = 0.f;
    int oz;
    float fz;
    bool flip = false;
    if (!R.live || ez == 0.f) {
        // a horizontal row keeps one voxel: the bigger index on a plane, the last voxel on the
        // bottom face (Section 4.1); outside the volume, the zero voxel above the column
        const bool below = uz.hi < 0.f || (uz.hi == 0.f && uz.lo < 0.f);
        const bool above = uz.hi > (float)T.nz || (uz.hi == (float)T.nz && uz.lo > 0.f);
        int fl;
        float fr;
        df_floor_frac(uz, fl, fr);
        oz = (!R.live || below || above) ? -1 : min(fl, T.nz - 1);
        fz = 0.5f;
        ez = 0.f;
    } else {
        flip = ez < 0.f;
        if (flip) {
            uz = df_sub(DF{(float)T.nz, 0.f}, uz);
            ez = -ez;
        }
        df_floor_frac(uz, oz, fz);
    }
    R.ez = ez;
    R.fz = fz;
    R.iez = ez != 0.f ? __frcp_rn(ez) : 0.f;
    R.bz = ez != 0.f ? __fmul_rn(-fz, R.iez) : -INFINITY;
    R.lo = -0.5f - (float)oz;
    R.hi = (float)(T.nz - oz) + 0.5f;
    R.sec = R.live ? __fsqrt_rn(__fmaf_rn(tz.hi, tz.hi, 1.0f)) : 0.f;
    R.zs = flip ? 0xffffffffu : 1u;
    R.C = flip ? (unsigned)(T.nz - oz) + (unsigned)kMagicBits : (unsigned)(oz + 1) - (unsigned)kMagicBits;
    const float w0 = __fmaf_rn(ez, tin, fz), w1 = __fmaf_rn(ez, tout, fz);  // w is monotone in tau
    R.inside = ez == 0.f || (w0 >= -1.0f - (float)oz && w1 < (float)(T.nz + 1 - oz));
    return R;
}

// The voxel of the row at tau: the magic float of floor(w), w = u - oz (clamped if CLAMP).
template <bool CLAMP>
__device__ __forceinline__ float row_floor(const Row &R, float tau)
{
    float w = __fmaf_rn(R.ez, tau, R.fz);
    if (CLAMP) w = fminf(fmaxf(w, R.lo), R.hi);
    return magic_floor(w);
}

// One slab [ta, tb] of column offset oxy: voxels A (at ta) and B (at tb), their offsets and
// lengths (in tau).  ma / mb: the magic floats of the voxel index at ta / tb (mb - ma is 0 or
// 1).  The z plane crossed inside the slab is u = mb; with no crossing, that plane lies behind
// ta and A gets no length.  Rounding can leave lB a few ulp below zero at a crossing on tb.
__device__ __forceinline__ void slab_split(const Row &R, float ta, float tb, float ma, float mb, int oxy,
                                           unsigned &oA, unsigned &oB, float &lA, float &lB)
{
    const float tx = fmaxf(__fmaf_rn(mb - kMagic, R.iez, R.bz), ta);
    lA = __fsub_rn(tx, ta);
    lB = __fsub_rn(tb, tx);
    const unsigned ob = (unsigned)oxy + R.C;
    oA = R.zs * (unsigned)__float_as_int(ma) + ob;
    oB = R.zs * (unsigned)__float_as_int(mb) + ob;
}

// Warp w of CTA b: column (b % ncg) * kWarpsPerCta + w, view (b / ncg) % n_views, row block
// b / (ncg n_views) (32 rows; lane = row in the block).  The row blocks are the slowest index,
// so the rays in flight are one block of 32 rows in a few views: a thin slab of the volume,
// which stays in L2.  False for a warp past the last column.
struct WarpJob {
    int col, view, row;
};

// Parts of the detector columns taken in turn within a row block, each through all views
// (T.split): the columns of one side of the central ray cover about half of the xy plane in a
// view, so a part's rows in flight touch about half the volume slab that all columns would.
// Measured on GB300: the forward reads pair columns (twice the float copy's bytes), and two
// parts keep more of its slab in L2 (circular cone 512^3: 156.5 vs 173.8 ms; 4 parts 156.2 ms;
// helix 512^2 x 256: 58.9 vs 59.7 ms); the adjoint's float accumulator keeps one part (two
// parts: 218.7 vs 215.4 ms).
constexpr int kFwdSplit = 2, kAdjSplit = 1;

__host__ __device__ __forceinline__ int col_groups_per_part(int ncg, int split) { return (ncg + split - 1) / split; }

__device__ __forceinline__ bool warp_job(const TraceGeo &T, WarpJob &J)
{
    const int64_t b = blockIdx.x;
    const int ncgp = col_groups_per_part(T.ncg, T.split);
    const int cgl = (int)(b % ncgp);
    const int64_t rest = b / ncgp;
    J.view = (int)(rest % T.n_views);
    const int64_t rest2 = rest / T.n_views;
    const int cg = (int)(rest2 % T.split) * ncgp + cgl;
    J.col = cg * kWarpsPerCta + (int)(threadIdx.x >> 5);
    J.row = (int)(rest2 / T.split) * 32 + (int)(threadIdx.x & 31);
    return J.col < T.n_cols;
}

// The forward walk on pair columns: entry e of a padded column holds (z(e), z(e + 1)), so
// voxel m of a row and voxel m + 1 come in one 64-bit load, at the entry of m (the entry of
// m + 1 for a row read from the column's far end, whose pair then holds (m + 1, m)).  The z
// plane m + 1 splits the slab: voxel m gets the part before it, voxel m + 1 the rest -- with
// no crossing the plane lies past the slab's end and voxel m gets it all (a horizontal row:
// plane at +infinity).  FLIP: 0 no row of the warp is read from the far end, 1 every row, 2
// some (a per-row select).
template <int U, bool CLAMP, int FLIP>
__device__ __forceinline__ float fwd_walk_pairs(const TraceGeo &T, const WTrace &W, const Row &R, int lane,
                                                float2 *slot, const float2 *__restrict__ volP)
{
    float acc0 = 0.f, acc1 = 0.f;  // two chains: the pairs' first and second voxels
    const bool flip = R.zs != 1u;
    const float bz = R.ez != 0.f ? R.bz : INFINITY;
    const unsigned C = R.C - (flip ? 1u : 0u);  // the pair's entry: that of m, or of m + 1
    float ta = W.tin, ma = row_floor<CLAMP>(R, ta);
    for (int c = 0; c < W.nchunk; ++c) {
        const int n = build_chunk(T, W, c, lane, slot);
        int s = 0;
        for (; s + U <= n; s += U) {
            int e[U];
            float l0[U], l1[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float2 sl = slot[s + u];
                const float mb = row_floor<CLAMP>(R, sl.x);
                const float tx = fminf(fmaxf(__fmaf_rn(ma - (kMagic - 1.0f), R.iez, bz), ta), sl.x);
                const float a = __fsub_rn(tx, ta), b = __fsub_rn(sl.x, tx);
                l0[u] = FLIP == 0 ? a : (FLIP == 1 ? b : (flip ? b : a));
                l1[u] = FLIP == 0 ? b : (FLIP == 1 ? a : (flip ? a : b));
                e[u] = (int)(R.zs * (unsigned)__float_as_int(ma) + ((unsigned)__float_as_int(sl.y) + C));
                ta = sl.x;
                ma = mb;
            }
            float2 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = __ldg(volP + e[u]);
#pragma unroll
            for (int u = 0; u < U; ++u) {
                acc0 = __fmaf_rn(v[u].x, l0[u], acc0);
                acc1 = __fmaf_rn(v[u].y, l1[u], acc1);
            }
        }
        for (; s < n; ++s) {
            const float2 sl = slot[s];
            const float mb = row_floor<CLAMP>(R, sl.x);
            const float tx = fminf(fmaxf(__fmaf_rn(ma - (kMagic - 1.0f), R.iez, bz), ta), sl.x);
            const float a = __fsub_rn(tx, ta), b = __fsub_rn(sl.x, tx);
            const float2 v = __ldg(volP + (int)(R.zs * (unsigned)__float_as_int(ma) +
                                                ((unsigned)__float_as_int(sl.y) + C)));
            acc0 = __fmaf_rn(v.x, FLIP == 0 ? a : (FLIP == 1 ? b : (flip ? b : a)), acc0);
            acc1 = __fmaf_rn(v.y, FLIP == 0 ? b : (FLIP == 1 ? a : (flip ? a : b)), acc1);
            ta = sl.x;
            ma = mb;
        }
        __syncwarp();  // the next chunk overwrites the slots
    }
    return __fadd_rn(acc0, acc1);
}

template <int U, bool CLAMP>
__device__ __forceinline__ float fwd_walk_pairs_any(const TraceGeo &T, const WTrace &W, const Row &R, int lane,
                                                    float2 *slot, const float2 *__restrict__ volP)
{
    const unsigned fm = __ballot_sync(0xffffffffu, R.zs != 1u);
    if (fm == 0u) return fwd_walk_pairs<U, CLAMP, 0>(T, W, R, lane, slot, volP);
    if (fm == 0xffffffffu) return fwd_walk_pairs<U, CLAMP, 1>(T, W, R, lane, slot, volP);
    return fwd_walk_pairs<U, CLAMP, 2>(T, W, R, lane, slot, volP);
}

template <int U>
__global__ void __launch_bounds__(32 * kWarpsPerCta, XR_TRACE_FWD_MINB) trace_fwd_kernel(TraceGeo T, const float2 *__restrict__ volP,
                                                                     float *__restrict__ sino)
// volP: the pair columns of the padded z-fastest copy
{
    __shared__ float2 slot_s[kWarpsPerCta][kChunk];
    WarpJob J;
    if (!warp_job(T, J)) return;  // the whole warp
    const int lane = threadIdx.x & 31;
    float2 *slot = slot_s[threadIdx.x >> 5];
    const ViewDF V = T.views[J.view];
    RayRec r;
    DF tauF{0.f, 0.f};
    WTrace W;
    float acc = 0.f;
    if (trace_record(T, V, T.cols[J.col], r, tauF) && trace_setup(T, r, W)) {  // uniform over the warp
        const Row R = make_row(T, V, J.col, J.row, tauF, W.tin, W.tout);
        if (__all_sync(0xffffffffu, R.inside))
            acc = fwd_walk_pairs_any<U, false>(T, W, R, lane, slot, volP);
        else
            acc = fwd_walk_pairs_any<U, true>(T, W, R, lane, slot, volP);
        acc = __fmul_rn(acc, R.sec);
    }
    if (J.row < T.n_rows) sino[((int64_t)J.view * T.n_rows + J.row) * T.n_cols + J.col] = acc;
}

// Segmented sum over runs of equal keys in neighbouring lanes (keys are ordered by lane):
// the first lane of each run ends with the run's sum.  runs: an upper bound on a run's length
// for the whole warp.
__device__ __forceinline__ float run_sum(float v, int key, int lane, int runs)
{
    for (int d = 1; d < runs; d <<= 1) {
        const float o = __shfl_down_sync(0xffffffffu, v, d);
        const int k = __shfl_down_sync(0xffffffffu, key, d);
        if (lane + d < 32 && k == key) v += o;
    }
    return v;
}

// Longest run of lanes in one voxel over the whole trace: neighbouring rows are at least
// `pitch` apart in u_z (their gap is linear in tau, so its ends bound it).
__device__ __forceinline__ int longest_run(const TraceGeo &T, const Row &R, const WTrace &W, int row, int lane)
{
    const float w0 = __fmaf_rn(R.ez, W.tin, R.fz) - R.lo, w1 = __fmaf_rn(R.ez, W.tout, R.fz) - R.lo;
    const float n0 = __shfl_down_sync(0xffffffffu, w0, 1), n1 = __shfl_down_sync(0xffffffffu, w1, 1);
    const bool pair = lane < 31 && row + 1 < T.n_rows;
    float pitch = pair ? fminf(fabsf(n0 - w0), fabsf(n1 - w1)) : INFINITY;
    if (pair && (n0 - w0) * (n1 - w1) <= 0.f) pitch = 0.f;
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) pitch = fminf(pitch, __shfl_xor_sync(0xffffffffu, pitch, d));
    return pitch > 0.04f ? min(32, 2 + (int)(1.0f / pitch)) : 32;
}

// The adjoint walk of one row: g * sec * length added to voxels A (at a crossing) and B.
template <bool AGG, bool CLAMP>
__device__ __forceinline__ void adj_walk(const TraceGeo &T, const WTrace &W, const Row &R, int lane, int runs,
                                         float gs, float2 *slot, float *__restrict__ accZ)
{
    float ta = W.tin, ma = row_floor<CLAMP>(R, ta);
    for (int c = 0; c < W.nchunk; ++c) {
        const int n = build_chunk(T, W, c, lane, slot);
#pragma unroll(kAdjUnroll)
        for (int s = 0; s < n; ++s) {
            const float2 sl = slot[s];
            const float mb = row_floor<CLAMP>(R, sl.x);
            unsigned oA, oB;
            float lA, lB;
            slab_split(R, ta, sl.x, ma, mb, __float_as_int(sl.y), oA, oB, lA, lB);
            red_add_if_pos(accZ + oA, __fmul_rn(gs, lA), lA);
            if (AGG) {
                float vB = lB > 0.f ? __fmul_rn(gs, lB) : 0.f;
                vB = run_sum(vB, (int)oB, lane, runs);
                const unsigned kp = __shfl_up_sync(0xffffffffu, oB, 1);
                if ((lane == 0 || kp != oB) && vB != 0.f) red_add(accZ + oB, vB);
            } else if (XR_TRACE_B_ALWAYS) {
                // B gets a length on all but grazing slabs: an unpredicated reduction (a length a
                // few ulp below zero at a crossing on the slab's end adds a rounding-sized term)
                red_add(accZ + oB, __fmul_rn(gs, lB));
            } else {
                red_add_if_pos(accZ + oB, __fmul_rn(gs, lB), lB);
            }
            ta = sl.x;
            ma = mb;
        }
        __syncwarp();
    }
}

template <bool AGG>
__global__ void __launch_bounds__(32 * kWarpsPerCta, XR_TRACE_MINB) trace_adj_kernel(TraceGeo T, const float *__restrict__ sino,
                                                                     float *__restrict__ accZ)
{
    __shared__ float2 slot_s[kWarpsPerCta][kChunk];
    WarpJob J;
    if (!warp_job(T, J)) return;
    const int lane = threadIdx.x & 31;
    float2 *slot = slot_s[threadIdx.x >> 5];
    const ViewDF V = T.views[J.view];
    RayRec r;
    DF tauF{0.f, 0.f};
    WTrace W;
    if (!trace_record(T, V, T.cols[J.col], r, tauF) || !trace_setup(T, r, W)) return;  // uniform
    const Row R = make_row(T, V, J.col, J.row, tauF, W.tin, W.tout);
    const float g = R.live ? __ldg(sino + ((int64_t)J.view * T.n_rows + J.row) * T.n_cols + J.col) : 0.f;
    if (__all_sync(0xffffffffu, g == 0.f)) return;  // nothing to spread
    const float gs = __fmul_rn(g, R.sec);
    const int runs = AGG ? longest_run(T, R, W, J.row, lane) : 1;
    if (__all_sync(0xffffffffu, R.inside))
        adj_walk<AGG, false>(T, W, R, lane, runs, gs, slot, accZ);
    else
        adj_walk<AGG, true>(T, W, R, lane, runs, gs, slot, accZ);
}

// Pair columns of a [rows = nz][cols = nx ny] volume: out[p * ld + e] = (z(e), z(e + 1)) for
// e = 0 .. ld - 1 (ld = nz + 2), z(0) = 0, z(1 + k) = in[k * cols + p], z(nz + 1) = z(nz + 2) = 0;
// out[-1] (a leading pair the caller allocates) = (0, 0).  Rows e0 - 1 .. e0 + 31 of a tile are
// staged so that reads run along p and writes along e.
__global__ void __launch_bounds__(256) to_zpairs_kernel(const float *__restrict__ in, float2 *__restrict__ out,
                                                        int64_t rows, int64_t cols)
{
    __shared__ float tile[33][33];
    const int64_t ld = rows + 2;
    const int64_t c0 = (int64_t)blockIdx.x * 32;
    const int64_t e_tiles = (ld + 31) / 32;
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0 && threadIdx.y == 0) out[-1] = make_float2(0.f, 0.f);
    for (int64_t ty = blockIdx.y; ty < e_tiles; ty += gridDim.y) {
        const int64_t e0 = ty * 32;
        for (int rr = threadIdx.y; rr < 33; rr += blockDim.y) {
            const int64_t k = e0 + rr - 1, c = c0 + threadIdx.x;  // z(e0 + rr) = in[k] for 0 <= k < rows
            tile[rr][threadIdx.x] = (k >= 0 && k < rows && c < cols) ? in[k * cols + c] : 0.f;
        }
        __syncthreads();
        for (int dc = threadIdx.y; dc < 32; dc += blockDim.y) {
            const int64_t c = c0 + dc, e = e0 + threadIdx.x;
            if (c < cols && e < ld) out[c * ld + e] = make_float2(tile[threadIdx.x][dc], tile[threadIdx.x + 1][dc]);
        }
        __syncthreads();
    }
}

// out[k * cols + p] = acc[p * ld + 1 + k] (the padding voxels are dropped)
__global__ void __launch_bounds__(256) from_zpad_kernel(const float *__restrict__ acc, float *__restrict__ out,
                                                        int64_t rows, int64_t cols)
{
    __shared__ float tile[32][33];
    const int64_t ld = rows + 2;
    const int64_t c0 = (int64_t)blockIdx.x * 32;
    const int64_t row_tiles = (rows + 31) / 32;
    for (int64_t ty = blockIdx.y; ty < row_tiles; ty += gridDim.y) {
        const int64_t r0 = ty * 32;
        for (int dc = threadIdx.y; dc < 32; dc += blockDim.y) {
            const int64_t c = c0 + dc, r = r0 + threadIdx.x;
            if (r < rows && c < cols) tile[dc][threadIdx.x] = acc[c * ld + 1 + r];
        }
        __syncthreads();
        for (int dr = threadIdx.y; dr < 32; dr += blockDim.y) {
            const int64_t r = r0 + dr, c = c0 + threadIdx.x;
            if (r < rows && c < cols) out[r * cols + c] = tile[threadIdx.x][dr];
        }
        __syncthreads();
    }
}

#ifndef XR_TRACE_AHEAD
#define XR_TRACE_AHEAD 8
#endif
#ifndef XR_TRACE_AGG
#define XR_TRACE_AGG 0
#endif

dim3 zpad_grid(int64_t rows, int64_t cols)
{
    return dim3((unsigned)((cols + 31) / 32), (unsigned)std::min<int64_t>((rows + 31) / 32, 65535));
}


}  // namespace

// The adjoint's padded z-fastest accumulator (floats), or the forward's pair columns after one
// leading pair
size_t trace_ws_bytes(const GeoParams &g)
{
    const size_t units = (size_t)g.nx * g.ny * (size_t)(g.nz + 2);
    return (units + 1) * sizeof(float2);
}

cudaError_t launch_trace_project(const TraceGeo &T, const float *img, float *ws, float *sino, cudaStream_t s)
{
    const int64_t cols = (int64_t)T.nx * T.ny;
    float2 *pairs = reinterpret_cast<float2 *>(ws) + 1;
    to_zpairs_kernel<<<zpad_grid(T.nz + 2, cols), dim3(32, 8), 0, s>>>(img, pairs, T.nz, cols);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    TraceGeo G = T;
    G.ncg = (T.n_cols + kWarpsPerCta - 1) / kWarpsPerCta;
    G.split = kFwdSplit;
    const int64_t ctas = (int64_t)col_groups_per_part(G.ncg, G.split) * G.split * G.n_views * G.n_rb;
    trace_fwd_kernel<XR_TRACE_AHEAD><<<(unsigned)ctas, 32 * kWarpsPerCta, 0, s>>>(G, pairs, sino);
    return cudaGetLastError();
}

cudaError_t launch_trace_backproject(const TraceGeo &T, const float *sino, float *img, float *ws, cudaStream_t s)
{
    const int64_t cols = (int64_t)T.nx * T.ny;
    cudaError_t e = cudaMemsetAsync(ws, 0, (size_t)cols * (T.nz + 2) * sizeof(float), s);
    if (e != cudaSuccess) return e;
    TraceGeo G = T;
    G.ncg = (T.n_cols + kWarpsPerCta - 1) / kWarpsPerCta;
    G.split = kAdjSplit;
    const int64_t ctas = (int64_t)col_groups_per_part(G.ncg, G.split) * G.split * G.n_views * G.n_rb;
    if (XR_TRACE_AGG)
        trace_adj_kernel<true><<<(unsigned)ctas, 32 * kWarpsPerCta, 0, s>>>(G, sino, ws);
    else
        trace_adj_kernel<false><<<(unsigned)ctas, 32 * kWarpsPerCta, 0, s>>>(G, sino, ws);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    from_zpad_kernel<<<zpad_grid(T.nz, cols), dim3(32, 8), 0, s>>>(ws, img, T.nz, cols);
    return cudaGetLastError();
}

}  // namespace xr
