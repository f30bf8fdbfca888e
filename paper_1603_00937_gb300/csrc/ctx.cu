// Context, errors and small helpers of libgbe.
#include <cstdarg>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "devmem.h"
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
        case GBE_EPEER: return "another rank reported an error";
        default: return "unknown error";
    }
}

// ------------------------------------------------------------------ device memory
bool gbe_device_memory_of(const void* p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

int gbe_check_device(const gbe_ctx* ctx, const void* p, size_t bytes, const char* what) {
    if (bytes == 0 || gbe_device_memory_of(p, ctx->device)) return GBE_OK;
    gbe_set_error("%s is flagged as device memory but is not device memory of GPU %d", what, ctx->device);
    return GBE_EINVAL;
}

int gbe_check_device_csr(const gbe_ctx* ctx, const gbe_csr* H, const char* what) {
    if (!H->on_device) return GBE_OK;
    if (gbe_check_device(ctx, H->rowptr, (size_t)(H->n + 1) * 8, "CSR rowptr") != GBE_OK ||
        gbe_check_device(ctx, H->col, (size_t)H->nnz * 4, "CSR col") != GBE_OK ||
        gbe_check_device(ctx, H->val, (size_t)H->nnz * 8, "CSR val") != GBE_OK) {
        gbe_set_error("%s: arrays flagged on_device = 1 are not device memory of GPU %d", what, ctx->device);
        return GBE_EINVAL;
    }
    return GBE_OK;
}

int gbe_check_device_ell(const gbe_ctx* ctx, const gbe_ell* D, const char* what) {
    if (!D->on_device) return GBE_OK;
    const size_t total = (size_t)D->n * (size_t)D->width;
    if (gbe_check_device(ctx, D->col, total * 4, "ELL col") != GBE_OK ||
        gbe_check_device(ctx, D->val, total * 8, "ELL val") != GBE_OK) {
        gbe_set_error("%s: arrays flagged on_device = 1 are not device memory of GPU %d", what, ctx->device);
        return GBE_EINVAL;
    }
    return GBE_OK;
}

namespace {
thread_local cudaStream_t t_stream = nullptr;
thread_local cudaMemPool_t t_pool = nullptr;
std::mutex g_alloc_mu;
struct PooledBlock {
    cudaStream_t stream;   // stream the block was allocated on (and is freed on)
    cudaMemPool_t pool;
};
std::unordered_map<void*, PooledBlock> g_pooled;
// Live blocks per pool, and whether the pool's context was destroyed: a pool outlives its
// context until its last block is freed (objects may be released after their context).
struct PoolState {
    int64_t live = 0;
    bool closed = false;
};
std::unordered_map<cudaMemPool_t, PoolState> g_pools;
}  // namespace

AllocScope::AllocScope(const gbe_ctx* ctx) : prev_stream(t_stream), prev_pool(t_pool) {
    if (ctx && ctx->pool) {
        t_stream = ctx->stream;
        t_pool = ctx->pool;
    }
}

AllocScope::~AllocScope() {
    t_stream = prev_stream;
    t_pool = prev_pool;
}

int gbe_alloc(void** p, size_t bytes) {
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    const bool pooled = t_pool != nullptr;
    cudaError_t e = pooled ? cudaMallocFromPoolAsync(p, bytes, t_pool, t_stream) : cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        gbe_set_error("device allocation of %zu bytes: %s", bytes, cudaGetErrorString(e));
        (void)cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? GBE_ENOMEM : GBE_ECUDA;
    }
    if (pooled) {
        std::lock_guard<std::mutex> lock(g_alloc_mu);
        g_pooled[*p] = PooledBlock{t_stream, t_pool};
        g_pools[t_pool].live += 1;
    }
    return GBE_OK;
}

void gbe_free(void* p) {
    if (!p) return;
    bool pooled = false, destroy = false;
    PooledBlock b{nullptr, nullptr};
    {
        std::lock_guard<std::mutex> lock(g_alloc_mu);
        auto it = g_pooled.find(p);
        if (it != g_pooled.end()) {
            pooled = true;
            b = it->second;
            g_pooled.erase(it);
            PoolState& ps = g_pools[b.pool];
            ps.live -= 1;
            if (ps.live == 0 && ps.closed) {
                destroy = true;
                g_pools.erase(b.pool);
            }
        }
    }
    if (!pooled) {
        cudaFree(p);
        return;
    }
    cudaFreeAsync(p, b.stream);
    if (destroy) {   // the last block of a destroyed context's pool
        cudaStreamSynchronize(b.stream);
        cudaMemPoolDestroy(b.pool);
    }
}

// Destroy a context's pool now, or, while blocks of it are still held by live objects,
// when the last of them is freed.
static void release_pool(cudaMemPool_t pool) {
    bool now = false;
    {
        std::lock_guard<std::mutex> lock(g_alloc_mu);
        auto it = g_pools.find(pool);
        if (it == g_pools.end() || it->second.live == 0) {
            now = true;
            if (it != g_pools.end()) g_pools.erase(it);
        } else {
            it->second.closed = true;
        }
    }
    if (now) cudaMemPoolDestroy(pool);
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
    cudaMemPoolProps props;
    memset(&props, 0, sizeof(props));
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    if (cudaMemPoolCreate(&c->pool, &props) != cudaSuccess) {
        (void)cudaGetLastError();
        delete c;
        gbe_set_error("cudaMemPoolCreate failed on device %d", device);
        return GBE_ECUDA;
    }
    uint64_t keep = UINT64_MAX;   // keep freed blocks for reuse instead of returning them at every sync
    cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    AllocScope scope(c);
    int r = gbe_alloc(&c->d_scratch, 4096);
    if (r != GBE_OK) { release_pool(c->pool); delete c; return r; }
    if (cudaMallocHost(&c->h_scratch, 4096) != cudaSuccess) {
        gbe_free(c->d_scratch);
        cudaStreamSynchronize(c->stream);
        release_pool(c->pool);
        delete c;
        gbe_set_error("cudaMallocHost failed");
        return GBE_ENOMEM;
    }
    r = gbe_tc_prepare(c);
    if (r != GBE_OK) {
        gbe_free(c->d_scratch);
        cudaStreamSynchronize(c->stream);
        cudaFreeHost(c->h_scratch);
        release_pool(c->pool);
        delete c;
        return r;
    }
    *out = c;
    return GBE_OK;
}

extern "C" int gbe_destroy(gbe_ctx* ctx) {
    if (!ctx) return GBE_OK;
    cudaSetDevice(ctx->device);
    gbe_free(ctx->d_scratch);
    cudaStreamSynchronize(ctx->stream);
    cudaFreeHost(ctx->h_scratch);
    // blocks still held by live objects keep the pool alive until they are freed
    release_pool(ctx->pool);
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

extern "C" int gbe_set_graph_launch(gbe_ctx* ctx, int on) {
    GBE_CHECK_ARG(ctx != nullptr, "ctx is NULL");
    ctx->graphs = on ? 1 : 0;
    return GBE_OK;
}

extern "C" int gbe_device_sm_count(const gbe_ctx* ctx) { return ctx ? ctx->sm_count : 0; }
