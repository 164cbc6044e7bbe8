// Attenuated transform for batches of 2D images on the interleaved layouts of the batched
// fast path: the same weights as atten.cu (two crossing-order walks per ray: the total
// attenuation, then exp(-A_k) E_k per unit), with the images read as planes of 4 (a float4
// per unit and plane) and the adjoint added with 128-bit reductions into the Bp-interleaved
// accumulators, in the layout (x fastest or y fastest) whose fastest axis the ray's warp is
// spread along.  The attenuation map is copied into both padded layouts first, so one
// offset serves the map and the images.
#include "xray_internal.h"

namespace xr {

constexpr int kPad = 2;  // the interleaved layouts' zero border (fast2d.cu)

namespace {

// mu0[jp][ip] and mu1[ip][jp] over the padded grid (zero on the border)
__global__ void mu_layouts_kernel(const float *__restrict__ mu, int nx, int ny, float *__restrict__ mu0,
                                  float *__restrict__ mu1)
{
    const int px = nx + 2 * kPad, py = ny + 2 * kPad;
    const int u = blockIdx.x * blockDim.x + threadIdx.x;
    if (u >= px * py) return;
    const int ip = u % px, jp = u / px;
    const int i = ip - kPad, j = jp - kPad;
    const float v = (i >= 0 && i < nx && j >= 0 && j < ny) ? __ldg(mu + (int64_t)j * nx + i) : 0.f;
    mu0[u] = v;
    mu1[ip * py + jp] = v;
}

struct Kahan2 {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
};

__device__ __forceinline__ float weight2(const Kahan2 &T, const Kahan2 &P, float m, float l)
{
    const float A = fmaxf(__fadd_rn(__fsub_rn(T.s, P.s), __fsub_rn(P.c, T.c)), 0.f);
    const float a = __fmul_rn(m, l);
    const float E = a > 0.f ? -expm1f(-a) / m : l;
    return __fmul_rn(expf(-A), E);
}

// Walk setup in the padded layout chosen for the ray; false when it crosses no pixel.
__device__ __forceinline__ bool setup2(const RayRec &rr, int nx, int ny, bool &tr, Dda<int> &D)
{
    const int px = nx + 2 * kPad, py = ny + 2 * kPad;
    tr = fabsf(rr.w0) > fabsf(rr.w1);
    const int si = tr ? py : 1, sj = tr ? 1 : px;
    if (!dda_setup<int>(rr, nx, ny, 1, si, sj, 0, D)) return false;
    D.off += kPad * (si + sj);
    return true;
}

template <int NQ>
__global__ void __launch_bounds__(256) atten_plane_fwd_kernel(const RayRec *__restrict__ rays, int n_rays, int nx,
                                                              int ny, const float4 *__restrict__ il0,
                                                              const float4 *__restrict__ il1,
                                                              const float *__restrict__ mu0,
                                                              const float *__restrict__ mu1, float *__restrict__ sino,
                                                              int batch)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const int np = (nx + 2 * kPad) * (ny + 2 * kPad);
    const int q0 = blockIdx.y * NQ;
    float4 acc[NQ];
#pragma unroll
    for (int q = 0; q < NQ; ++q) acc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
    bool tr;
    Dda<int> D;
    if (setup2(rays[r], nx, ny, tr, D)) {
        const float *__restrict__ mu = tr ? mu1 : mu0;
        const float4 *__restrict__ il = (tr ? il1 : il0) + (int64_t)q0 * np;
        const int max_steps = dda_max_steps(nx, ny, 1);
        Kahan2 T;
        {
            Dda<int> E = D;
            for (int k = 0; k < max_steps && E.tcur < E.tout; ++k) {
                int off;
                float l;
                dda_step(E, off, l);
                if (l > 0.f) T.add(__fmul_rn(__ldg(mu + off), l));
            }
        }
        Kahan2 P;
        for (int k = 0; k < max_steps && D.tcur < D.tout; ++k) {
            int off;
            float l;
            dda_step(D, off, l);
            if (!(l > 0.f)) continue;
            const float m = __ldg(mu + off);
            P.add(__fmul_rn(m, l));
            const float w = weight2(T, P, m, l);
#pragma unroll
            for (int q = 0; q < NQ; ++q) {
                const float4 v = __ldg(il + (int64_t)q * np + off);
                acc[q].x = __fmaf_rn(v.x, w, acc[q].x);
                acc[q].y = __fmaf_rn(v.y, w, acc[q].y);
                acc[q].z = __fmaf_rn(v.z, w, acc[q].z);
                acc[q].w = __fmaf_rn(v.w, w, acc[q].w);
            }
        }
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
        const int b = 4 * (q0 + q);
        if (b + 0 < batch) sino[(int64_t)(b + 0) * n_rays + r] = acc[q].x;
        if (b + 1 < batch) sino[(int64_t)(b + 1) * n_rays + r] = acc[q].y;
        if (b + 2 < batch) sino[(int64_t)(b + 2) * n_rays + r] = acc[q].z;
        if (b + 3 < batch) sino[(int64_t)(b + 3) * n_rays + r] = acc[q].w;
    }
}

// acc0/acc1: [chunk][np][Bp], Bp = 4 * NB4 images per chunk; blockIdx.y = chunk
template <int NB4>
__global__ void __launch_bounds__(256) atten_plane_adj_kernel(const RayRec *__restrict__ rays, int n_rays, int nx,
                                                              int ny, float *__restrict__ acc0,
                                                              float *__restrict__ acc1,
                                                              const float *__restrict__ mu0,
                                                              const float *__restrict__ mu1,
                                                              const float *__restrict__ sino, int batch)
{
    const int r = blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    constexpr int Bp = 4 * NB4;
    const int np = (nx + 2 * kPad) * (ny + 2 * kPad);
    const int b0 = blockIdx.y * Bp;
    float g[Bp];
    bool any = false;
#pragma unroll
    for (int b = 0; b < Bp; ++b) {
        g[b] = (b0 + b < batch) ? __ldg(sino + (int64_t)(b0 + b) * n_rays + r) : 0.f;
        any |= g[b] != 0.f;
    }
    if (!any) return;
    bool tr;
    Dda<int> D;
    if (!setup2(rays[r], nx, ny, tr, D)) return;
    const float *__restrict__ mu = tr ? mu1 : mu0;
    float *__restrict__ acc = (tr ? acc1 : acc0) + (int64_t)blockIdx.y * np * Bp;
    const int max_steps = dda_max_steps(nx, ny, 1);
    Kahan2 T;
    {
        Dda<int> E = D;
        for (int k = 0; k < max_steps && E.tcur < E.tout; ++k) {
            int off;
            float l;
            dda_step(E, off, l);
            if (l > 0.f) T.add(__fmul_rn(__ldg(mu + off), l));
        }
    }
    Kahan2 P;
    for (int k = 0; k < max_steps && D.tcur < D.tout; ++k) {
        int off;
        float l;
        dda_step(D, off, l);
        if (!(l > 0.f)) continue;
        const float m = __ldg(mu + off);
        P.add(__fmul_rn(m, l));
        const float w = weight2(T, P, m, l);
        float *p = acc + (int64_t)off * Bp;
#pragma unroll
        for (int q = 0; q < NB4; ++q)
            red_add4(p + 4 * q, __fmul_rn(g[4 * q], w), __fmul_rn(g[4 * q + 1], w), __fmul_rn(g[4 * q + 2], w),
                     __fmul_rn(g[4 * q + 3], w));
    }
}

}  // namespace

cudaError_t launch_mu_layouts(const float *mu, int nx, int ny, float *mu0, float *mu1, cudaStream_t s)
{
    const int n = (nx + 2 * kPad) * (ny + 2 * kPad);
    mu_layouts_kernel<<<(n + 255) / 256, 256, 0, s>>>(mu, nx, ny, mu0, mu1);
    return cudaGetLastError();
}

cudaError_t launch_atten_plane_fwd(const RayRec *rays, int64_t n_rays, int nx, int ny, const float *il0,
                                   const float *il1, const float *mu0, const float *mu1, float *sino, int batch,
                                   int nq, cudaStream_t s)
{
    const int Q = (batch + 3) / 4, groups = (Q + nq - 1) / nq;
    const dim3 grid((unsigned)((n_rays + 255) / 256), (unsigned)groups);
    const float4 *a = reinterpret_cast<const float4 *>(il0), *b = reinterpret_cast<const float4 *>(il1);
    if (nq == 4)
        atten_plane_fwd_kernel<4><<<grid, 256, 0, s>>>(rays, (int)n_rays, nx, ny, a, b, mu0, mu1, sino, batch);
    else if (nq == 2)
        atten_plane_fwd_kernel<2><<<grid, 256, 0, s>>>(rays, (int)n_rays, nx, ny, a, b, mu0, mu1, sino, batch);
    else
        atten_plane_fwd_kernel<1><<<grid, 256, 0, s>>>(rays, (int)n_rays, nx, ny, a, b, mu0, mu1, sino, batch);
    return cudaGetLastError();
}

cudaError_t launch_atten_plane_adj(const RayRec *rays, int64_t n_rays, int nx, int ny, float *acc0, float *acc1,
                                   size_t acc_bytes, const float *mu0, const float *mu1, const float *sino,
                                   float *img, int batch, int Bp, cudaStream_t s)
{
    cudaError_t e = cudaMemsetAsync(acc0, 0, acc_bytes, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(acc1, 0, acc_bytes, s);
    if (e != cudaSuccess) return e;
    const dim3 grid((unsigned)((n_rays + 255) / 256), (unsigned)((batch + Bp - 1) / Bp));
    if (Bp == 16)
        atten_plane_adj_kernel<4><<<grid, 256, 0, s>>>(rays, (int)n_rays, nx, ny, acc0, acc1, mu0, mu1, sino, batch);
    else if (Bp == 8)
        atten_plane_adj_kernel<2><<<grid, 256, 0, s>>>(rays, (int)n_rays, nx, ny, acc0, acc1, mu0, mu1, sino, batch);
    else
        atten_plane_adj_kernel<1><<<grid, 256, 0, s>>>(rays, (int)n_rays, nx, ny, acc0, acc1, mu0, mu1, sino, batch);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return launch_deinterleave_sum(acc0, acc1, batch, nx, ny, 1, Bp, img, s);
}

}  // namespace xr
