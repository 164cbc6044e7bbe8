// Read-bandwidth probe: the denominator of the L2 roofline the benchmark reports next to the
// FP32 one.  A buffer small enough to stay in L2 is read `reps` times with 128-bit loads by a
// grid of (SMs x resident CTAs); one float per thread is written so the loads are not dropped.
#include "xray_internal.h"

namespace xr {
namespace {

__global__ void __launch_bounds__(256) read_probe_kernel(const float4 *__restrict__ buf, int64_t n4, int reps,
                                                         float *__restrict__ sink)
{
    float acc = 0.f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int r = 0; r < reps; ++r) {
        for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n4; k += stride) {
            const float4 v = __ldcg(buf + k);  // cached in L2 only: every pass is an L2 read
            acc += (v.x + v.y) + (v.z + v.w);
        }
    }
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

// FP32 FMA throughput: 8 independent chains per thread, `iters` steps each, written once.
__global__ void __launch_bounds__(256) fma_probe_kernel(int iters, float *__restrict__ sink)
{
    float a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = (float)(threadIdx.x + k) * 1e-3f;
    const float m = 0.999999f, c = 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = __fmaf_rn(a[k], m, c);
    }
    float t = 0.f;
#pragma unroll
    for (int k = 0; k < 8; ++k) t += a[k];
    sink[(int64_t)blockIdx.x * blockDim.x + threadIdx.x] = t;
}

}  // namespace
}  // namespace xr

#define PROBE_CUDA(call)                              \
    do {                                              \
        cudaError_t e_ = (call);                      \
        if (e_ != cudaSuccess) return xr_fail_cuda(e_); \
    } while (0)

extern "C" xr_status xr_read_probe(const float *d_buf, int64_t n_floats, int32_t reps, float *d_sink,
                                   int32_t sink_floats, xr_stream stream)
{
    using namespace xr;
    if (!d_buf || !d_sink) return XR_ERR_NULL;
    if (n_floats < 4 || reps < 1 || (n_floats & 3)) return XR_ERR_SIZE;
    if (((uintptr_t)d_buf & 15u) != 0) return XR_ERR_ALIGN;
    int dev = 0, sms = 0, per_sm = 0;
    PROBE_CUDA(cudaGetDevice(&dev));
    PROBE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PROBE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, read_probe_kernel, 256, 0));
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    if ((int64_t)grid * 256 > sink_floats) return XR_ERR_SIZE;
    read_probe_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(reinterpret_cast<const float4 *>(d_buf), n_floats / 4,
                                                              reps, d_sink);
    PROBE_CUDA(cudaGetLastError());
    return XR_OK;
}

extern "C" xr_status xr_fma_probe(int32_t iters, float *d_sink, int32_t sink_floats, int64_t *flop, xr_stream stream)
{
    using namespace xr;
    if (!d_sink || !flop) return XR_ERR_NULL;
    if (iters < 1) return XR_ERR_SIZE;
    int dev = 0, sms = 0, per_sm = 0;
    PROBE_CUDA(cudaGetDevice(&dev));
    PROBE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    PROBE_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_probe_kernel, 256, 0));
    const int grid = sms * (per_sm > 0 ? per_sm : 1);
    if ((int64_t)grid * 256 > sink_floats) return XR_ERR_SIZE;
    fma_probe_kernel<<<grid, 256, 0, (cudaStream_t)stream>>>(iters, d_sink);
    PROBE_CUDA(cudaGetLastError());
    *flop = (int64_t)grid * 256 * 8 * 2 * (int64_t)iters;
    return XR_OK;
}

extern "C" xr_status xr_wait_bound_selftest(int64_t cycles, int32_t *timed_out)
{
    if (!timed_out) return XR_ERR_NULL;
    if (cycles < 1 || cycles > 20000000000ll) return XR_ERR_SIZE;
    int *d = nullptr;
    PROBE_CUDA(cudaMalloc(&d, sizeof(int)));
    cudaError_t e = cudaMemset(d, 0xff, sizeof(int));
    if (e == cudaSuccess) e = xr::launch_wait_selftest((long long)cycles, d, nullptr);
    int h = -1;
    if (e == cudaSuccess) e = cudaMemcpy(&h, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return xr_fail_cuda(e);
    *timed_out = h;
    return XR_OK;
}
