// xr_tune: chooses a handle's launch tuning by timing the candidates on the current GPU and
// keeps the choice in a text cache, one line per scan:
//     <key> <block> <batch_chunk> <adjoint> <path> <order> <forward+adjoint ms>
// key = GPU name | kind | nx,ny,nz | dx,dy,dz | views | rows,cols | batch (spaces in the GPU
// name become '_').  Only the public entry points are used: the tuner reserves the
// workspace, sets each candidate with xr_set_tuning and times xr_project + xr_backproject
// with CUDA events on a stream of its own, over images and sinograms of ones.
#include <stdio.h>
#include <string.h>

#include <string>
#include <vector>

#include "xray_internal.h"

namespace {

__global__ void fill_ones_kernel(float *p, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = 1.f;
}

std::string scan_key(const xr_geometry *g, int batch)
{
    cudaDeviceProp prop;
    std::string name = "gpu";
    if (cudaGetDeviceProperties(&prop, g->device) == cudaSuccess) name = prop.name;
    for (char &c : name)
        if (c == ' ') c = '_';
    char buf[512];
    const xr::GeoParams &p = g->params;
    snprintf(buf, sizeof(buf), "%s|%d|%d,%d,%d|%g,%g,%g|%d|%d,%d|%d", name.c_str(), p.kind, p.nx, p.ny, p.nz, p.dx,
             p.dy, p.dz, p.n_views, p.n_rows, p.n_cols, batch);
    return buf;
}

// The cached tuning for key, if any.  false also when the file does not exist.
bool cache_lookup(const char *path, const std::string &key, xr_tuning *t)
{
    FILE *f = fopen(path, "r");
    if (!f) return false;
    char line[1024];
    bool found = false;
    while (fgets(line, sizeof(line), f)) {
        char k[600];
        xr_tuning c{};
        float ms = 0.f;
        if (sscanf(line, "%599s %d %d %d %d %d %f", k, &c.block, &c.batch_chunk, &c.adjoint, &c.path, &c.order,
                   &ms) == 7 &&
            key == k) {
            *t = c;  // the last matching line wins
            found = true;
        }
    }
    fclose(f);
    return found;
}

std::vector<xr_tuning> candidates(const xr_geometry *g, int batch)
{
    const int kind = g->params.kind;
    const bool three = xr::kind_is3d(kind), list = xr::kind_is_list(kind);
    std::vector<xr_tuning> out;
    const int adjs[2] = {XR_ADJ_SCATTER, XR_ADJ_GATHER};
    const int n_adj = list ? 1 : 2;
    if (three) {
        if (g->trace_ok)  // the column-trace walk (scatter adjoint)
            out.push_back(xr_tuning{128, 16, XR_ADJ_SCATTER, XR_PATH_INTERLEAVED, XR_ORDER_TRACE});
        for (int order : {XR_ORDER_VIEW, XR_ORDER_ROW, XR_ORDER_COLUMN, XR_ORDER_ROWBLOCK})
            for (int a = 0; a < n_adj; ++a) out.push_back(xr_tuning{128, 16, adjs[a], XR_PATH_INTERLEAVED, order});
        out.push_back(xr_tuning{128, batch < 16 ? (batch < 2 ? 1 : 2) : 16, XR_ADJ_SCATTER, XR_PATH_RAY,
                                XR_ORDER_VIEW});
        return out;
    }
    if (batch >= 4) {
        for (int chunk : {16, 8, 4})
            for (int a = 0; a < n_adj; ++a)
                out.push_back(xr_tuning{128, chunk, adjs[a], XR_PATH_INTERLEAVED, XR_ORDER_VIEW});
        if (!list) out.push_back(xr_tuning{128, 16, XR_ADJ_SCATTER, XR_PATH_TILED, XR_ORDER_VIEW});
    } else {
        for (int a = 0; a < n_adj; ++a) out.push_back(xr_tuning{128, 1, adjs[a], XR_PATH_INTERLEAVED, XR_ORDER_VIEW});
    }
    for (int a = 0; a < n_adj; ++a) out.push_back(xr_tuning{128, batch >= 4 ? 16 : 1, adjs[a], XR_PATH_RAY,
                                                             XR_ORDER_VIEW});
    return out;
}

}  // namespace

extern "C" xr_status xr_tune(xr_geometry *g, const char *cache_path)
{
    if (!g) return XR_ERR_NULL;
    const int batch = g->ws_batch > 0 ? g->ws_batch : 1;
    const std::string key = scan_key(g, batch);
    xr_tuning best{};
    if (cache_path && cache_lookup(cache_path, key, &best)) return xr_set_tuning(g, &best);

    xr_status st = xr_reserve(g, batch);
    if (st != XR_OK) return st;
    int prev = 0;
    if (cudaGetDevice(&prev) != cudaSuccess) return XR_ERR_CUDA;
    if (cudaSetDevice(g->device) != cudaSuccess) return XR_ERR_CUDA;
    float *img = nullptr, *sino = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const size_t n_img = (size_t)g->n_units * batch, n_sino = (size_t)g->n_rays * batch;
    cudaError_t e = cudaMalloc(&img, n_img * sizeof(float));
    if (e == cudaSuccess) e = cudaMalloc(&sino, n_sino * sizeof(float));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        fill_ones_kernel<<<1024, 256, 0, s>>>(img, (int64_t)n_img);
        fill_ones_kernel<<<1024, 256, 0, s>>>(sino, (int64_t)n_sino);
        e = cudaGetLastError();
    }
    float best_ms = 1e30f;
    const xr_tuning saved = g->tune;
    for (const xr_tuning &c : candidates(g, batch)) {
        if (e != cudaSuccess) break;
        st = xr_set_tuning(g, &c);
        if (st != XR_OK) continue;
        float ms = 1e30f;
        for (int rep = 0; rep < 4 && st == XR_OK; ++rep) {  // the first pass warms up
            cudaEventRecord(e0, s);
            st = xr_project(g, img, sino, batch, (xr_stream)s);
            if (st == XR_OK) st = xr_backproject(g, sino, img, batch, (xr_stream)s);
            cudaEventRecord(e1, s);
            e = cudaEventSynchronize(e1);
            float t = 0.f;
            if (e == cudaSuccess && st == XR_OK && cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && rep > 0)
                ms = t < ms ? t : ms;
            if (st == XR_OK) {  // keep the inputs ones (the adjoint overwrote the image)
                fill_ones_kernel<<<1024, 256, 0, s>>>(img, (int64_t)n_img);
                fill_ones_kernel<<<1024, 256, 0, s>>>(sino, (int64_t)n_sino);
            }
        }
        if (st == XR_OK && e == cudaSuccess && ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) cudaStreamDestroy(s);
    cudaFree(img);
    cudaFree(sino);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        g->tune = saved;
        return xr_fail_cuda(e);
    }
    if (best_ms >= 1e30f) {
        g->tune = saved;
        return XR_ERR_TUNE;
    }
    st = xr_set_tuning(g, &best);
    if (st != XR_OK) return st;
    if (cache_path) {
        FILE *f = fopen(cache_path, "a");
        if (!f) return XR_ERR_TUNE;
        fprintf(f, "%s %d %d %d %d %d %.4f\n", key.c_str(), best.block, best.batch_chunk, best.adjoint, best.path,
                best.order, best_ms);
        if (fclose(f) != 0) return XR_ERR_TUNE;
    }
    return XR_OK;
}
