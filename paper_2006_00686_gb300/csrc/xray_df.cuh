// Float-pair arithmetic on the FP32 pipes: a value hi + lo with |lo| <= ulp(hi) / 2 (about 48
// significant bits), with the error-free transformations of Dekker (1971) and Knuth (TAOCP
// vol. 2, 4.2.2): a product's rounding error is recovered with one FMA, a sum's with the
// two-sum sequence.  GB300's FP64 rate is a small fraction of its FP32 rate, so per-ray and
// per-CTA geometry that needs more than float precision is computed this way.
#pragma once

#include "xray_internal.h"

namespace xr {

// round-to-nearest intrinsics throughout: no contraction or reordering

__device__ __forceinline__ DF two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    const float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return DF{s, e};
}

// requires |a| >= |b| (or a == 0)
__device__ __forceinline__ DF quick_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return DF{s, __fsub_rn(b, __fsub_rn(s, a))};
}

__device__ __forceinline__ DF df_add(DF a, DF b)
{
    DF s = two_sum(a.hi, b.hi);
    const DF t = two_sum(a.lo, b.lo);
    s.lo = __fadd_rn(s.lo, t.hi);
    s = quick_two_sum(s.hi, s.lo);
    s.lo = __fadd_rn(s.lo, t.lo);
    return quick_two_sum(s.hi, s.lo);
}

__device__ __forceinline__ DF df_neg(DF a) { return DF{-a.hi, -a.lo}; }
__device__ __forceinline__ DF df_sub(DF a, DF b) { return df_add(a, df_neg(b)); }

__device__ __forceinline__ DF df_mul(DF a, DF b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return quick_two_sum(p, e);
}

__device__ __forceinline__ bool df_is_zero(DF a) { return a.hi == 0.f && a.lo == 0.f; }

// Snap cos/sin pairs within 1e-12 of a multiple of pi/2 to exact 0 and +-1, so that
// axis-parallel and in-plane rays are recognised as such.
__device__ __forceinline__ void snap(DF &c, DF &s)
{
    if (fabsf(c.hi) < 1e-12f) {
        c = DF{0.f, 0.f};
        s = DF{s.hi > 0.f ? 1.f : -1.f, 0.f};
    } else if (fabsf(s.hi) < 1e-12f) {
        s = DF{0.f, 0.f};
        c = DF{c.hi > 0.f ? 1.f : -1.f, 0.f};
    }
}

__device__ __forceinline__ DF to_df(double x)
{
    const float hi = __double2float_rn(x);
    return DF{hi, __double2float_rn(x - (double)hi)};
}

// floor of hi + lo as an int and the fraction left (in [0, 1)), as a float
__device__ __forceinline__ void df_floor_frac(DF x, int &fl, float &fr)
{
    float f = floorf(x.hi);
    if (x.hi == f && x.lo < 0.f) f -= 1.f;
    float r = __fadd_rn(__fsub_rn(x.hi, f), x.lo);
    if (r >= 1.0f) {
        r = 0.0f;
        f += 1.f;
    }
    fl = (int)f;
    fr = r;
}

}  // namespace xr
