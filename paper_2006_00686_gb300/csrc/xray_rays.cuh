// A ray's index-space record (see xray_core.cuh), built from the per-view and per-detector
// tables by the float-pair arithmetic of the ray setup -- and RaySrc, which hands kernels a
// ray's record either from the handle's table or rebuilt on the spot from those tables.
// Cone and helical scans keep no table (at 32 B per ray a 512^3 cone scan with a 1024 x 768
// detector and 720 views would hold 18 GB): every kernel that needs a record calls
// ray_record with the same inputs, so the record is bit for bit the one a table would hold.
#pragma once

#include "xray_df.cuh"
#include "xray_internal.h"

namespace xr {

// One ray: view v, detector sample d.
__device__ __forceinline__ RayRec ray_record(const GeoParams &g, const SetupDF &K, const ViewDF &V, const DetRec &R)
{
    DF P[3], T[3];
    const DF zero{0.f, 0.f};
    if (g.kind <= XR_FAN2D_ARC || g.kind == XR_RAYS2D) {
        DF cp, sp, sv = R.s1;
        if (g.kind == XR_PAR2D || g.kind == XR_RAYS2D) {
            cp = V.c1;  // phi = angles[v]
            sp = V.s1;
            if (g.kind == XR_RAYS2D) sv = V.H;  // the ray's own s
        } else {
            // phi = gamma + alpha - pi/2: cos(phi) = sin(gamma + alpha), sin(phi) = -cos(gamma + alpha)
            cp = df_add(df_mul(R.sa, V.c1), df_mul(R.ca, V.s1));
            sp = df_sub(df_mul(R.sa, V.s1), df_mul(R.ca, V.c1));
        }
        snap(cp, sp);
        T[0] = cp;
        T[1] = sp;
        T[2] = zero;
        P[0] = df_neg(df_mul(sv, sp));
        P[1] = df_mul(sv, cp);
        P[2] = K.cz;
    } else {
        DF c1, sn1, c2, sn2, s1 = R.s1, s2 = R.s2;
        if (g.kind == XR_PAR3D || g.kind == XR_RAYS3D) {
            c1 = V.c1;
            sn1 = V.s1;
            c2 = V.c2;
            sn2 = V.s2;
            if (g.kind == XR_RAYS3D) {  // the ray's own s1, s2
                s1 = V.H;
                s2 = V.pad;
            }
        } else {
            // phi1 = phi'_1 + alpha, phi2 = beta
            c1 = df_sub(df_mul(V.c1, R.ca), df_mul(V.s1, R.sa));
            sn1 = df_add(df_mul(V.s1, R.ca), df_mul(V.c1, R.sa));
            c2 = R.cb;
            sn2 = R.sb;
            s2 = df_add(s2, df_mul(V.H, R.cb));
        }
        snap(c1, sn1);
        snap(c2, sn2);
        T[0] = df_mul(c2, c1);
        T[1] = df_mul(c2, sn1);
        T[2] = sn2;
        const DF s2sn2 = df_mul(s2, sn2);
        P[0] = df_neg(df_add(df_mul(s1, sn1), df_mul(s2sn2, c1)));
        P[1] = df_sub(df_mul(s1, c1), df_mul(s2sn2, sn1));
        P[2] = df_mul(s2, c2);
    }
    // Foot point: the point of the line closest to the image centre.
    const DF tf = df_add(df_add(df_mul(df_sub(K.cx, P[0]), T[0]), df_mul(df_sub(K.cy, P[1]), T[1])),
                         df_mul(df_sub(K.cz, P[2]), T[2]));
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (!df_is_zero(T[a])) P[a] = df_add(P[a], df_mul(tf, T[a]));

    // Index space: u_x grows with i, u_y with j (y falls), u_z with k (z falls).  Whether
    // the ray enters the image is decided by the walk's own box test.
    const int N[3] = {g.nx, g.ny, g.nz};
    const DF o[3] = {df_mul(df_sub(P[0], K.x0), K.idx), df_mul(df_sub(K.y1, P[1]), K.idy),
                     df_mul(df_sub(K.z1, P[2]), K.idz)};
    const DF wd[3] = {df_mul(T[0], K.idx), df_neg(df_mul(T[1], K.idy)), df_neg(df_mul(T[2], K.idz))};

    RayRec rec;
    int flags = 0;
    float wf[3], ff[3];
    int oi[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        // floor of hi + lo, and the fraction left
        float fl = floorf(o[a].hi);
        if (o[a].hi == fl && o[a].lo < 0.f) fl -= 1.f;
        const bool below = o[a].hi < 0.f || (o[a].hi == 0.f && o[a].lo < 0.f);
        if (df_is_zero(wd[a])) {
            // Fixed index: unit n holds u in [n, n+1]; a ray on the plane u = n (two
            // candidates) takes the bigger index (Section 4.1), the far edge u = N the last.
            wf[a] = 0.f;
            ff[a] = 0.f;
            const bool above = o[a].hi > (float)N[a] || (o[a].hi == (float)N[a] && o[a].lo > 0.f);
            if (!below && !above) {
                oi[a] = min((int)fl, N[a] - 1);
            } else {
                oi[a] = -1;
                flags |= RAY_MISS;
            }
        } else {
            float fr = __fadd_rn(__fsub_rn(o[a].hi, fl), o[a].lo);
            if (fr >= 1.0f) {
                fr = 0.0f;
                fl += 1.f;
            }
            wf[a] = __fadd_rn(wd[a].hi, wd[a].lo);
            ff[a] = fr;
            if (fabsf(fl) > 32000.f) {
                flags |= RAY_MISS;
                fl = 0.f;
            }
            oi[a] = (int)fl;
        }
    }
    rec.w0 = wf[0];
    rec.w1 = wf[1];
    rec.w2 = wf[2];
    rec.f0 = ff[0];
    rec.f1 = ff[1];
    rec.f2 = ff[2];
    rec.o0 = (int16_t)oi[0];
    rec.o1 = (int16_t)oi[1];
    rec.o2 = (int16_t)oi[2];
    rec.flags = (int16_t)flags;
    return rec;
}

// The record of ray r: from the table when there is one, else rebuilt from view r / ndet and
// detector sample r % ndet.
__device__ __forceinline__ RayRec RaySrc::operator[](int64_t r) const
{
    if (tab) return tab[r];
    const int64_t v = r / ndet;
    return ray_record(g, K, views[v], det[r - v * ndet]);
}

}  // namespace xr
