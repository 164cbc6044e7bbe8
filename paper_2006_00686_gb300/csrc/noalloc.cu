// xr_project_batched_noalloc: the batched forward projection for callers that cannot
// allocate device memory (and xr_project_batched / xr_backproject_batched, the one-call
// forward and adjoint over the same fixed work-list array).
//
// Some callers cannot call cudaMalloc at the point where they need a projection: code
// running while a stream is captured in global mode (where cudaMalloc is refused), hosts
// whose own allocator owns the whole device pool and forbids allocations behind its back,
// and tight loops that cannot afford the implicit synchronisation of cudaMalloc/cudaFree.
// xr_batch_create allocates its work list and counter; this entry point instead keeps
// them in one fixed-size array in device memory, reserved when the library's module is
// loaded on a device and held by every device that loads it until the process exits.
//
// Set-up: the first call on a device (with that device current) looks up the array's
// device address with cudaGetSymbolAddress and remembers it; in host code the array's
// name is only a host-side stand-in and must never be handed to a kernel.  That first call
// should come before any stream capture.  Every later call reuses the remembered address.
//
// Every call shares the array: each call first overwrites the work list and zeroes the
// tile counter (stream-ordered), so nothing from the previous call leaks in, but calls
// whose launches overlap on the GPU (different streams, no ordering) race on it.
#include <mutex>

#include "xray_internal.h"

using namespace xr;

namespace {

constexpr int kMaxProblems = XR_NOALLOC_MAX_PROBLEMS;
constexpr size_t kCounterBytes = 256;  // tile counter, padded to keep the list aligned
constexpr size_t kScratchBytes = kCounterBytes + kMaxProblems * sizeof(BatchItem);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// The work list travels as a kernel parameter (by value), so no host staging buffer or
// copy engine transfer is involved.
struct WorkList {
    BatchItem items[kMaxProblems];
    int n;
};
static_assert(sizeof(WorkList) < 32000, "work list must fit the kernel parameter space");

__global__ void noalloc_upload_kernel(WorkList w, unsigned char *scratch)
{
    BatchItem *dst = reinterpret_cast<BatchItem *>(scratch + kCounterBytes);
    for (int i = threadIdx.x; i < w.n; i += blockDim.x) dst[i] = w.items[i];
    if (threadIdx.x == 0) *reinterpret_cast<unsigned long long *>(scratch) = 0ull;
}

std::mutex g_mu;
unsigned char *g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once per device).
cudaError_t scratch_on_current_device(unsigned char **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
    }
    *out = g_scratch_ptr[dev];
    return cudaSuccess;
}

}  // namespace

// Uploads the work list into the scratch array and launches the forward (adjoint = 0) or
// the zero fill and the adjoint (adjoint = 1) over it.
static xr_status noalloc_launch(const xr_problem *probs, int32_t n, int32_t tile, int adjoint, xr_stream stream);

extern "C" xr_status xr_project_batched_noalloc(const xr_problem *probs, int32_t n, int32_t tile,
                                                xr_stream stream)
{
    return noalloc_launch(probs, n, tile, 0, stream);
}

extern "C" xr_status xr_project_batched(const xr_problem *probs, int32_t n, xr_stream stream)
{
    return noalloc_launch(probs, n, 0, 0, stream);
}

extern "C" xr_status xr_backproject_batched(const xr_problem *probs, int32_t n, xr_stream stream)
{
    return noalloc_launch(probs, n, 0, 1, stream);
}

static xr_status noalloc_launch(const xr_problem *probs, int32_t n, int32_t tile, int adjoint, xr_stream stream)
{
    if (!probs) return XR_ERR_NULL;
    if (n < 1) return XR_ERR_SIZE;
    if (n > kMaxProblems) return XR_ERR_CAPACITY;
    if (tile == 0) tile = 256;
    if (tile < 32 || tile > 65536 || (tile & 31)) return XR_ERR_ARG;
    WorkList w;
    w.n = n;
    int64_t tiles = 0;
    for (int i = 0; i < n; ++i) {
        const xr_geometry *g = probs[i].geom;
        if (!g || !probs[i].img || !probs[i].sino) return XR_ERR_NULL;
        if (((uintptr_t)probs[i].img & 15u) || ((uintptr_t)probs[i].sino & 15u)) return XR_ERR_ALIGN;
        if (g->n_units >= ((int64_t)1 << 31)) return XR_ERR_SIZE;  // 32-bit walk offsets
        BatchItem &it = w.items[i];
        it.rays = g->d_rays;
        it.img = probs[i].img;
        it.sino = probs[i].sino;
        it.aux = nullptr;  // no copies: every ray reads the caller's layout
        it.nx = g->params.nx;
        it.ny = g->params.ny;
        it.nz = g->params.nz;
        it.three = kind_is3d(g->params.kind);
        it.n_rays = g->n_rays;
        it.tile_begin = tiles;
        tiles += (g->n_rays + tile - 1) / tile;
    }
    unsigned char *scratch = nullptr;
    cudaError_t e = scratch_on_current_device(&scratch);
    int dev = 0, sms = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return xr_fail_cuda(e);
    const cudaStream_t s = (cudaStream_t)stream;
    const int block = 256;
    noalloc_upload_kernel<<<1, 256, 0, s>>>(w, scratch);
    e = cudaGetLastError();
    const BatchItem *items = reinterpret_cast<const BatchItem *>(scratch + kCounterBytes);
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(scratch);
    if (e == cudaSuccess && !adjoint)
        e = launch_batched_items(items, n, tiles, tile, counter, sms * batched_ctas_per_sm(block, 0), block, s);
    if (e == cudaSuccess && adjoint)  // zero fill, then the scatter straight into the images
        e = launch_batched(items, n, tiles, tile, counter, 1, 0, sms * batched_ctas_per_sm(block, 1), block, s);
    if (e != cudaSuccess) return xr_fail_cuda(e);
    return XR_OK;
}
