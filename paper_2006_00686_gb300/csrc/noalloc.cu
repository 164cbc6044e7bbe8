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
// device address with cudaGetSymbolAddress and remembers it, with the persistent launch's
// grid size; in host code the array's
// name is only a host-side stand-in and must never be handed to a kernel.  That first call
// should come before any stream capture.  Every later call reuses the remembered address.
//
// Every call shares the array: each call first overwrites the work list and zeroes the
// tile counter (stream-ordered), so nothing from the previous call leaks in, but calls
// whose launches overlap on the GPU (different streams, no ordering) race on it.  Every
// problem's geometry must live on the current device (XR_ERR_ARG otherwise).
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
// copy engine transfer is involved.  Two capacities: calls of up to kSmallList problems
// send a parameter block of about 1 KiB instead of the full list's 16 KiB.
constexpr int kSmallList = 16;

template <int CAP>
struct WorkList {
    BatchItem items[CAP];
    int n;
};
static_assert(sizeof(WorkList<kMaxProblems>) < 32000, "work list must fit the kernel parameter space");

template <int CAP>
__global__ void noalloc_upload_kernel(WorkList<CAP> w, unsigned char *scratch)
{
    BatchItem *dst = reinterpret_cast<BatchItem *>(scratch + kCounterBytes);
    for (int i = threadIdx.x; i < w.n; i += blockDim.x) dst[i] = w.items[i];
    if (threadIdx.x == 0) *reinterpret_cast<unsigned long long *>(scratch) = 0ull;
}

// Per device, looked up once with that device current: the scratch array's device address
// and the persistent launch's grid (SMs x resident CTAs of the forward and the adjoint).
struct DeviceFacts {
    unsigned char *scratch = nullptr;
    int ctas_fwd = 0, ctas_adj = 0;      // crossing-order walk over any problems
    int ctas2d_adj = 0;                  // lockstep slab walk (adjoint) when every problem is 2D
};

std::mutex g_mu;
DeviceFacts g_facts[kMaxDevices];

constexpr int kBlock = 256;

cudaError_t facts_of_current_device(int *dev_out, DeviceFacts *out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_mu);
    DeviceFacts &f = g_facts[dev];
    if (!f.scratch) {
        void *p = nullptr;
        int sms = 0;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return e;
        f.ctas_fwd = sms * batched_ctas_per_sm(kBlock, 0);
        f.ctas_adj = sms * batched_ctas_per_sm(kBlock, 1);
        f.ctas2d_adj = sms * batch2d_ctas_per_sm(kBlock);
        f.scratch = static_cast<unsigned char *>(p);
    }
    *dev_out = dev;
    *out = f;
    return cudaSuccess;
}

// Fill the work list; XR_OK or the validation error.  Every geometry must live on `dev`.
template <int CAP>
xr_status fill_list(const xr_problem *probs, int32_t n, int32_t tile, int dev, WorkList<CAP> &w, int64_t &tiles)
{
    w.n = n;
    tiles = 0;
    for (int i = 0; i < n; ++i) {
        const xr_geometry *g = probs[i].geom;
        if (!g || !probs[i].img || !probs[i].sino) return XR_ERR_NULL;
        if (g->device != dev) return XR_ERR_ARG;  // its tables live on another device
        if (((uintptr_t)probs[i].img & 15u) || ((uintptr_t)probs[i].sino & 15u)) return XR_ERR_ALIGN;
        if (g->n_units >= ((int64_t)1 << 31)) return XR_ERR_SIZE;  // 32-bit walk offsets
        BatchItem &it = w.items[i];
        it.src = g->d_src;
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
    return XR_OK;
}

template <int CAP>
xr_status upload_and_launch(const xr_problem *probs, int32_t n, int32_t tile, int adjoint, int dev,
                            const DeviceFacts &f, cudaStream_t s)
{
    WorkList<CAP> w;
    int64_t tiles = 0;
    const xr_status st = fill_list<CAP>(probs, n, tile, dev, w, tiles);
    if (st != XR_OK) return st;
    bool lock2d = true;  // the same kernel a plan of these problems runs
    for (int i = 0; i < n; ++i) lock2d = lock2d && !w.items[i].three;
    noalloc_upload_kernel<CAP><<<1, 256, 0, s>>>(w, f.scratch);
    cudaError_t e = cudaGetLastError();
    const BatchItem *items = reinterpret_cast<const BatchItem *>(f.scratch + kCounterBytes);
    unsigned long long *counter = reinterpret_cast<unsigned long long *>(f.scratch);
    if (e == cudaSuccess && !adjoint)
        e = launch_batched_items(items, n, tiles, tile, counter, f.ctas_fwd, kBlock, s);
    if (e == cudaSuccess && adjoint)  // zero fill, then the scatter straight into the images
        e = launch_batched(items, n, tiles, tile, counter, 1, 0, lock2d ? f.ctas2d_adj : f.ctas_adj, kBlock, s,
                           lock2d);
    if (e != cudaSuccess) return xr_fail_cuda(e);
    return XR_OK;
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
    int dev = 0;
    DeviceFacts f;
    const cudaError_t e = facts_of_current_device(&dev, &f);
    if (e != cudaSuccess) return xr_fail_cuda(e);
    const cudaStream_t s = (cudaStream_t)stream;
    if (n <= kSmallList) return upload_and_launch<kSmallList>(probs, n, tile, adjoint, dev, f, s);
    return upload_and_launch<kMaxProblems>(probs, n, tile, adjoint, dev, f, s);
}
