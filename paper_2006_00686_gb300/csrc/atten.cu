// Attenuated transform: the generalized Radon transform (eq. generalizedRadontransform) with
// the exponential attenuation weight of the SPECT case,
//     Phi(theta, x, t) = exp(-int_t^inf mu(x + s theta) ds),
// mu an attenuation image on the same grid.  With f and mu constant on each unit, a ray's
// units k in the order of increasing t (the crossing-order walk's order), lengths l_k and
// A_k = sum_{m > k} mu_m l_m (the attenuation between unit k and the ray's far end):
//     g = sum_k f_k exp(-A_k) E_k,   E_k = int_0^{l_k} exp(-mu_k (l_k - t)) dt
//                                        = -expm1(-mu_k l_k) / mu_k   (l_k when mu_k l_k = 0).
// One thread per ray walks it twice: the first walk sums the total attenuation T, the second
// forms A_k = T - (attenuation up to and including unit k) and applies the weights to BC
// images at once (forward) or spreads g * weight (adjoint, the exact transpose).  Both sums
// are compensated (Kahan), so A_k keeps the precision of its own size, not of T.
// The direction theta is the ray's own (the record's w), so attenuation is taken towards
// the side the ray runs to.
#include "xray_rays.cuh"

namespace xr {
namespace {

struct Kahan {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float x)
    {
        const float y = __fsub_rn(x, c);
        const float t = __fadd_rn(s, y);
        c = __fsub_rn(__fsub_rn(t, s), y);
        s = t;
    }
};

// Total attenuation along the ray.
__device__ __forceinline__ Kahan total_attenuation(Dda<int64_t> D, int max_steps, const float *__restrict__ mu)
{
    Kahan T;
    for (int k = 0; k < max_steps && D.tcur < D.tout; ++k) {
        int64_t off;
        float l;
        dda_step(D, off, l);
        if (l > 0.f) T.add(__fmul_rn(__ldg(mu + off), l));
    }
    return T;
}

// exp(-A_k) E_k of the unit with attenuation m and length l, given P = attenuation up to and
// including it (compensated) and the total T.
__device__ __forceinline__ float unit_weight(const Kahan &T, const Kahan &P, float m, float l)
{
    const float A = fmaxf(__fadd_rn(__fsub_rn(T.s, P.s), __fsub_rn(P.c, T.c)), 0.f);
    const float a = __fmul_rn(m, l);
    const float E = a > 0.f ? -expm1f(-a) / m : l;
    return __fmul_rn(expf(-A), E);
}

template <int BC>
__global__ void __launch_bounds__(256) atten_fwd_kernel(RaySrc rays, int64_t n_rays, Grid grid,
                                                        const float *__restrict__ mu, const float *__restrict__ img,
                                                        int64_t img_bs, float *__restrict__ sino, int64_t sino_bs,
                                                        int batch)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const int b0 = blockIdx.y * BC, nb = min(BC, batch - b0);
    float acc[BC];
#pragma unroll
    for (int b = 0; b < BC; ++b) acc[b] = 0.f;
    Dda<int64_t> D;
    const int max_steps = dda_max_steps(grid.nx, grid.ny, grid.nz);
    if (dda_setup<int64_t>(rays[r], grid.nx, grid.ny, grid.nz, grid.sx, grid.sy, grid.sz, D)) {
        const Kahan T = total_attenuation(D, max_steps, mu);
        Kahan P;
        for (int k = 0; k < max_steps && D.tcur < D.tout; ++k) {
            int64_t off;
            float l;
            dda_step(D, off, l);
            if (!(l > 0.f)) continue;
            const float m = __ldg(mu + off);
            P.add(__fmul_rn(m, l));
            const float w = unit_weight(T, P, m, l);
#pragma unroll
            for (int b = 0; b < BC; ++b)
                if (b < nb) acc[b] = __fmaf_rn(__ldg(img + (b0 + b) * img_bs + off), w, acc[b]);
        }
    }
#pragma unroll
    for (int b = 0; b < BC; ++b)
        if (b < nb) sino[(b0 + b) * sino_bs + r] = acc[b];
}

template <int BC>
__global__ void __launch_bounds__(256) atten_adj_kernel(RaySrc rays, int64_t n_rays, Grid grid,
                                                        const float *__restrict__ mu, const float *__restrict__ sino,
                                                        int64_t sino_bs, float *__restrict__ img, int64_t img_bs,
                                                        int batch)
{
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n_rays) return;
    const int b0 = blockIdx.y * BC, nb = min(BC, batch - b0);
    float gv[BC];
    bool any = false;
#pragma unroll
    for (int b = 0; b < BC; ++b) {
        gv[b] = b < nb ? __ldg(sino + (b0 + b) * sino_bs + r) : 0.f;
        any |= gv[b] != 0.f;
    }
    if (!any) return;
    Dda<int64_t> D;
    const int max_steps = dda_max_steps(grid.nx, grid.ny, grid.nz);
    if (!dda_setup<int64_t>(rays[r], grid.nx, grid.ny, grid.nz, grid.sx, grid.sy, grid.sz, D)) return;
    const Kahan T = total_attenuation(D, max_steps, mu);
    Kahan P;
    for (int k = 0; k < max_steps && D.tcur < D.tout; ++k) {
        int64_t off;
        float l;
        dda_step(D, off, l);
        if (!(l > 0.f)) continue;
        const float m = __ldg(mu + off);
        P.add(__fmul_rn(m, l));
        const float w = unit_weight(T, P, m, l);
#pragma unroll
        for (int b = 0; b < BC; ++b)
            if (b < nb && gv[b] != 0.f) red_add(img + (b0 + b) * img_bs + off, __fmul_rn(gv[b], w));
    }
}

template <int BC>
cudaError_t launch_atten_t(bool adjoint, const RaySrc &rays, int64_t n_rays, const Grid &grid, const float *mu,
                           const float *in, float *out, int64_t n_units, int batch, int block, cudaStream_t s)
{
    const dim3 g((unsigned)((n_rays + block - 1) / block), (unsigned)((batch + BC - 1) / BC));
    if (adjoint)
        atten_adj_kernel<BC><<<g, block, 0, s>>>(rays, n_rays, grid, mu, in, n_rays, out, n_units, batch);
    else
        atten_fwd_kernel<BC><<<g, block, 0, s>>>(rays, n_rays, grid, mu, in, n_units, out, n_rays, batch);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_attenuated(bool adjoint, const RaySrc &rays, int64_t n_rays, const Grid &grid, const float *mu,
                              const float *in, float *out, int64_t n_units, int batch, int chunk, int block,
                              cudaStream_t s)
{
    switch (chunk) {
    case 16: return launch_atten_t<16>(adjoint, rays, n_rays, grid, mu, in, out, n_units, batch, block, s);
    case 8: return launch_atten_t<8>(adjoint, rays, n_rays, grid, mu, in, out, n_units, batch, block, s);
    case 4: return launch_atten_t<4>(adjoint, rays, n_rays, grid, mu, in, out, n_units, batch, block, s);
    case 2: return launch_atten_t<2>(adjoint, rays, n_rays, grid, mu, in, out, n_units, batch, block, s);
    default: return launch_atten_t<1>(adjoint, rays, n_rays, grid, mu, in, out, n_units, batch, block, s);
    }
}

}  // namespace xr
