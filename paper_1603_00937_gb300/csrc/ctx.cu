// Context, errors and small helpers of libgbe.
#include <cstdarg>
#include <cstring>

#include "gbe_internal.h"

static thread_local char g_errmsg[1024] = "";

void gbe_set_error(const char* fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_errmsg, sizeof(g_errmsg), fmt, ap);
    va_end(ap);
}

extern "C" const char* gbe_last_error_message(void) { return g_errmsg; }

extern "C" const char* gbe_strerror(int code) {
    switch (code) {
        case GBE_OK: return "ok";
        case GBE_EINVAL: return "invalid argument";
        case GBE_ENOMEM: return "out of memory";
        case GBE_ECUDA: return "CUDA error";
        case GBE_ETIMEOUT: return "device wait timed out";
        case GBE_ENOCONV: return "SP2 did not converge within n_max";
        case GBE_ENUMERIC: return "NaN or Inf encountered";
        case GBE_ECAPACITY: return "capacity exceeded";
        case GBE_ENODEV: return "no usable sm_103 device";
        default: return "unknown error";
    }
}

int gbe_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        gbe_set_error("cudaMalloc(%zu bytes): %s", bytes, cudaGetErrorString(e));
        (void)cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? GBE_ENOMEM : GBE_ECUDA;
    }
    return GBE_OK;
}

int gbe_sync(gbe_ctx* ctx) {
    GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GBE_OK;
}

extern "C" int gbe_create(gbe_ctx** out, int device, void* cuda_stream) {
    GBE_CHECK_ARG(out != nullptr, "ctx out pointer is NULL");
    *out = nullptr;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev <= device || device < 0) {
        (void)cudaGetLastError();
        gbe_set_error("CUDA device %d not available (%d devices)", device, ndev);
        return GBE_ENODEV;
    }
    cudaDeviceProp prop;
    GBE_CUDA_TRY(cudaGetDeviceProperties(&prop, device));
    if (prop.major != 10 || prop.minor != 3) {
        gbe_set_error("device %d is sm_%d%d; libgbe is built for sm_103a only", device, prop.major, prop.minor);
        return GBE_ENODEV;
    }
    GBE_CUDA_TRY(cudaSetDevice(device));
    gbe_ctx* c = new gbe_ctx();
    c->device = device;
    c->stream = (cudaStream_t)cuda_stream;
    c->sm_count = prop.multiProcessorCount;
    c->smem_optin = (int)prop.sharedMemPerBlockOptin;
    int r = gbe_alloc(&c->d_scratch, 4096);
    if (r != GBE_OK) { delete c; return r; }
    if (cudaMallocHost(&c->h_scratch, 4096) != cudaSuccess) {
        cudaFree(c->d_scratch);
        delete c;
        gbe_set_error("cudaMallocHost failed");
        return GBE_ENOMEM;
    }
    r = gbe_tc_prepare(c);
    if (r != GBE_OK) { cudaFree(c->d_scratch); cudaFreeHost(c->h_scratch); delete c; return r; }
    *out = c;
    return GBE_OK;
}

extern "C" int gbe_destroy(gbe_ctx* ctx) {
    if (!ctx) return GBE_OK;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    cudaFree(ctx->d_scratch);
    cudaFreeHost(ctx->h_scratch);
    delete ctx;
    return GBE_OK;
}

extern "C" int gbe_set_stream(gbe_ctx* ctx, void* cuda_stream) {
    GBE_CHECK_ARG(ctx != nullptr, "ctx is NULL");
    ctx->stream = (cudaStream_t)cuda_stream;
    return GBE_OK;
}

extern "C" int gbe_set_profiling(gbe_ctx* ctx, int on) {
    GBE_CHECK_ARG(ctx != nullptr, "ctx is NULL");
    ctx->profile = on ? 1 : 0;
    return GBE_OK;
}

extern "C" int gbe_device_sm_count(const gbe_ctx* ctx) { return ctx ? ctx->sm_count : 0; }
