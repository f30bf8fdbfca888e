// Gershgorin spectral bounds without any device allocation.
//
// Same bounds as the Gershgorin step of gbe_sp2_run (e_min = min_i H_ii - sum_{j!=i}|H_ij|,
// e_max = max_i H_ii + sum_{j!=i}|H_ij|, one warp per row summing in the same order), but
// the per-block partial results live in a fixed file-scope device array instead of
// memory obtained from cudaMalloc, so the call works for callers that may not allocate.
#include <cuda.h>

#include <cmath>
#include <mutex>

#include "devmem.h"
#include "gbe_internal.h"

namespace {

constexpr int kRowsPerBlock = 256;    // 8 warps x 32 rows
constexpr int kMaxBlocks = 16384;     // => at most 4,194,304 rows

// [0, 2*kMaxBlocks): per-block (min, max) order-preserving keys; [2*kMaxBlocks]: non-finite flag.
// Held by every device that loads the library, for the life of the process (about 256 KB).
static __device__ __align__(256) unsigned long long g_gersh_scratch[2 * kMaxBlocks + 32];

__device__ __forceinline__ unsigned long long okey(double x) {
    unsigned long long b = (unsigned long long)__double_as_longlong(x);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__device__ __forceinline__ double okey_inv(unsigned long long k) {
    unsigned long long b = (k >> 63) ? (k & 0x7fffffffffffffffull) : ~k;
    return __longlong_as_double((long long)b);
}

__global__ void __launch_bounds__(256) gersh_partial_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                                            const double* __restrict__ val, int64_t n,
                                                            unsigned long long* scratch) {
    __shared__ unsigned long long smin[8], smax[8];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long kmin = ~0ull, kmax = 0ull;
    bool bad = false;
    const int64_t r0 = (int64_t)blockIdx.x * kRowsPerBlock + w * 32;
    for (int t = 0; t < 32; ++t) {
        const int64_t i = r0 + t;
        if (i >= n) break;
        double off = 0.0, d = 0.0;
        for (int64_t p = rowptr[i] + lane; p < rowptr[i + 1]; p += 32) {
            const double v = val[p];
            if (!isfinite(v)) bad = true;
            if (col[p] == i) d = v; else off += fabs(v);
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_xor_sync(0xffffffffu, off, o);
            d += __shfl_xor_sync(0xffffffffu, d, o);
        }
        kmin = min(kmin, okey(d - off));
        kmax = max(kmax, okey(d + off));
    }
    if (__any_sync(0xffffffffu, bad) && lane == 0) scratch[2 * kMaxBlocks] = 1ull;
    if (lane == 0) { smin[w] = kmin; smax[w] = kmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < 8; ++k) { kmin = min(kmin, smin[k]); kmax = max(kmax, smax[k]); }
        kmin = min(kmin, smin[0]);
        kmax = max(kmax, smax[0]);
        scratch[2 * blockIdx.x] = kmin;
        scratch[2 * blockIdx.x + 1] = kmax;
    }
}

__global__ void __launch_bounds__(1024) gersh_reduce_kernel(const unsigned long long* scratch, int nblocks, double* bounds) {
    __shared__ unsigned long long smin[32], smax[32];
    unsigned long long kmin = ~0ull, kmax = 0ull;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) {
        kmin = min(kmin, scratch[2 * b]);
        kmax = max(kmax, scratch[2 * b + 1]);
    }
    for (int o = 16; o > 0; o >>= 1) {
        kmin = min(kmin, __shfl_xor_sync(0xffffffffu, kmin, o));
        kmax = max(kmax, __shfl_xor_sync(0xffffffffu, kmax, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (lane == 0) { smin[w] = kmin; smax[w] = kmax; }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int k = 1; k < (int)(blockDim.x >> 5); ++k) { kmin = min(kmin, smin[k]); kmax = max(kmax, smax[k]); }
        kmin = min(kmin, smin[0]);
        kmax = max(kmax, smax[0]);
        if (scratch[2 * kMaxBlocks] != 0ull) {
            bounds[0] = NAN;
            bounds[1] = NAN;
        } else {
            bounds[0] = okey_inv(kmin);
            bounds[1] = okey_inv(kmax);
        }
    }
}

// Device address of the scratch array, looked up once per device with that device current,
// and again whenever the device's current context is another one than at the lookup (after
// cudaDeviceReset the primary context is new and the array has a new address).
std::mutex g_mu;
unsigned long long* g_scratch_addr[64] = {nullptr};
CUcontext g_scratch_ctx[64] = {nullptr};
typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
CtxGetCurrentFn g_ctx_get = nullptr;

int scratch_for(int device, unsigned long long** out) {
    std::lock_guard<std::mutex> lock(g_mu);
    if (device < 0 || device >= 64) {
        gbe_set_error("device index %d out of range for the no-allocation scratch table", device);
        return GBE_EINVAL;
    }
    if (!g_ctx_get) {
        void* fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        const cudaError_t e = cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &fn, 12000, cudaEnableDefault, &q);
        if (e != cudaSuccess || q != cudaDriverEntryPointSuccess || !fn) {
            gbe_set_error("cuCtxGetCurrent not available: %s", cudaGetErrorString(e));
            return GBE_ECUDA;
        }
        g_ctx_get = (CtxGetCurrentFn)fn;
    }
    CUcontext cur = nullptr;
    if (g_ctx_get(&cur) != CUDA_SUCCESS || cur == nullptr) {
        gbe_set_error("no current CUDA context on device %d", device);
        return GBE_ECUDA;
    }
    if (!g_scratch_addr[device] || g_scratch_ctx[device] != cur) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_gersh_scratch);
        if (e != cudaSuccess || p == nullptr) {
            gbe_set_error("cudaGetSymbolAddress(g_gersh_scratch) on device %d: %s", device, cudaGetErrorString(e));
            return GBE_ECUDA;
        }
        g_scratch_addr[device] = (unsigned long long*)p;
        g_scratch_ctx[device] = cur;
    }
    *out = g_scratch_addr[device];
    return GBE_OK;
}

}  // namespace

extern "C" int gbe_gershgorin_noalloc(gbe_ctx* ctx, const gbe_csr* H, double* bounds) {
    AllocScope alloc_scope_(ctx);
    GBE_CHECK_ARG(ctx && H && bounds, "NULL argument");
    GBE_CHECK_ARG(H->on_device == 1, "gbe_gershgorin_noalloc needs a device CSR (copying host data would allocate)");
    GBE_CHECK_ARG(H->rowptr && H->col && H->val, "CSR arrays are NULL");
    const int64_t max_rows = (int64_t)kMaxBlocks * kRowsPerBlock;
    if (H->n <= 0 || H->n > max_rows) {
        gbe_set_error("gbe_gershgorin_noalloc: n = %lld rows, supported range is 1..%lld (fixed scratch of %d blocks)",
                      (long long)H->n, (long long)max_rows, kMaxBlocks);
        return GBE_EINVAL;
    }
    GBE_CUDA_TRY(cudaSetDevice(ctx->device));
    // the pointers are checked before anything is enqueued (no allocation, no synchronisation)
    GBE_CHECK_ARG(gbe_device_memory_of(bounds, ctx->device), "bounds is not device memory of the context's GPU");
    GBE_CHECK_ARG(gbe_device_memory_of(H->rowptr, ctx->device) && gbe_device_memory_of(H->col, ctx->device) &&
                      gbe_device_memory_of(H->val, ctx->device),
                  "H arrays are not device memory of the context's GPU (on_device = 1 needs device pointers)");
    unsigned long long* scratch = nullptr;
    GBE_TRY(scratch_for(ctx->device, &scratch));
    const int nblocks = (int)((H->n + kRowsPerBlock - 1) / kRowsPerBlock);
    // the non-finite flag must start at zero; the partials are fully rewritten each call
    GBE_CUDA_TRY(cudaMemsetAsync(scratch + 2 * kMaxBlocks, 0, sizeof(unsigned long long), ctx->stream));
    gersh_partial_kernel<<<nblocks, 256, 0, ctx->stream>>>(H->rowptr, H->col, H->val, H->n, scratch);
    gersh_reduce_kernel<<<1, 1024, 0, ctx->stream>>>(scratch, nblocks, bounds);
    GBE_CUDA_TRY(cudaGetLastError());
    return GBE_OK;
}
