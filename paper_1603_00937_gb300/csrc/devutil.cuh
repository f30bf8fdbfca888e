// Device utilities shared by the graph / partition / Hamiltonian and edge-classifier
// translation units: exclusive scan, spatial cell grid, minimum-image distance,
// deterministic sparse row dot product, and small host helpers.
#pragma once
#include <algorithm>
#include <cmath>

#include "devmem.h"
#include "gbe_internal.h"

namespace gbe_dev {

// ------------------------------------------------------------------ scan (exclusive, int32 -> int64)
constexpr int kScanThreads = 1024, kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

static __device__ int64_t block_exclusive_scan(int64_t v, int64_t* sh, int64_t* total) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        int64_t s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int64_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    const int64_t base = (w > 0) ? sh[w - 1] : 0;
    if (total) *total = sh[(blockDim.x >> 5) - 1];
    const int64_t r = base + x - v;
    __syncthreads();
    return r;
}

static __global__ void __launch_bounds__(kScanThreads) scan_local_kernel(const int32_t* __restrict__ in, int64_t* out,
                                                                  int64_t n, int64_t* bsum) {
    __shared__ int64_t sh[32];
    const int64_t base = (int64_t)blockIdx.x * kScanBlock + (int64_t)threadIdx.x * kScanItems;
    int64_t v[kScanItems], s = 0;
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = (base + i < n) ? in[base + i] : 0;
        s += v[i];
    }
    int64_t tot;
    int64_t ex = block_exclusive_scan(s, sh, &tot);
    for (int i = 0; i < kScanItems; ++i) {
        if (base + i < n) out[base + i] = ex;
        ex += v[i];
    }
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

static __global__ void __launch_bounds__(kScanThreads) scan_top_kernel(int64_t* bsum, int nb, int64_t* total) {
    __shared__ int64_t sh[32];
    int64_t carry = 0;
    for (int b0 = 0; b0 < nb; b0 += kScanThreads) {
        const int i = b0 + threadIdx.x;
        const int64_t v = (i < nb) ? bsum[i] : 0;
        int64_t tot;
        const int64_t ex = block_exclusive_scan(v, sh, &tot);
        if (i < nb) bsum[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *total = carry;
}

static __global__ void scan_add_kernel(int64_t* out, int64_t n, const int64_t* bsum, const int64_t* total) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] += bsum[i / kScanBlock];
    if (i == n) out[n] = *total;
}

struct CellGrid {
    int nc[3];
    double box[3];
    double inv[3];   // 1 / box
};

__device__ __forceinline__ int cell_of(const double* p, const CellGrid& g) {
    int c[3];
    for (int d = 0; d < 3; ++d) {
        int v = (int)floor(p[d] / g.box[d] * g.nc[d]);
        c[d] = min(max(v, 0), g.nc[d] - 1);
    }
    return (c[0] * g.nc[1] + c[1]) * g.nc[2] + c[2];
}

static __global__ void cell_count_kernel(const double* __restrict__ pos, int64_t n, CellGrid g, int32_t* cell, int32_t* cnt) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell_of(pos + 3 * i, g);
    cell[i] = c;
    atomicAdd(&cnt[c], 1);
}

static __global__ void cell_fill_kernel(const int32_t* __restrict__ cell, int64_t n, const int64_t* __restrict__ start,
                                 int32_t* cursor, int32_t* members) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int c = cell[i];
    members[start[c] + atomicAdd(&cursor[c], 1)] = (int32_t)i;
}

// Minimum image d - L rint(d / L), with the quotient taken as d * (1/L): the two can round to
// different integers only when d / L lies within an ulp of a half-integer, i.e. for pairs about
// L/2 apart, which every caller rejects (its cutoff is below L/2), so accepted pairs get the
// same separation as with a true division (an FP64 division is many times the cost of a
// multiplication on this part's FP64 pipe).
__device__ __forceinline__ double min_image(double d, double L, double invL) {
    return __dsub_rn(d, __dmul_rn(L, rint(__dmul_rn(d, invL))));
}
__device__ __forceinline__ double dist2(double x, double y, double z) {
    return __dadd_rn(__dadd_rn(__dmul_rn(x, x), __dmul_rn(y, y)), __dmul_rn(z, z));
}
// FP32 copies of the positions, one float4 per site (a 16-byte load per candidate).
static __global__ void pos_f32_kernel(const double* __restrict__ pos, int64_t n, float4* out) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = make_float4((float)pos[3 * i], (float)pos[3 * i + 1], (float)pos[3 * i + 2], 0.f);
}

// Cheap pre-filter of a candidate pair in FP32: rejects only pairs whose FP32 minimum-image
// distance exceeds the cutoff plus a margin larger than the FP32 error of the positions and
// of the box (see filter_lim2), so every pair the exact FP64 test accepts passes.
__device__ __forceinline__ float dist2_f32(float4 a, float4 b, float bx, float by, float bz, float ix, float iy,
                                           float iz) {
    float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
    dx -= bx * rintf(dx * ix);
    dy -= by * rintf(dy * iy);
    dz -= bz * rintf(dz * iz);
    return dx * dx + dy * dy + dz * dz;
}
__device__ __forceinline__ bool near_f32(float4 a, float4 b, float bx, float by, float bz, float ix, float iy, float iz,
                                         float lim2) {
    return dist2_f32(a, b, bx, by, bz, ix, iy, iz) < lim2;
}
// (cutoff + margin)^2 with margin = 1e-3 + 2^-16 * box: FP32 positions and box lengths are
// off by at most 2^-24 * box each, so the FP32 separation is within ~2^-21 * box of the exact one
static inline float filter_lim2(double cutoff, const double box[3]) {
    const double bmax = std::max(box[0], std::max(box[1], box[2]));
    const double lim = cutoff + 1e-3 + bmax * (1.0 / 65536.0);
    return (float)(lim * lim);
}
// The inner bound: (cutoff - margin)^2, rounded down, or 0.  A pair whose FP32 squared
// separation is below it lies inside the cutoff in exact arithmetic too (the margin is ~100
// times the FP32 error), so the exact FP64 test is needed only between the two bounds.
static inline float filter_lim2_in(double cutoff, const double box[3]) {
    const double bmax = std::max(box[0], std::max(box[1], box[2]));
    const double lim = cutoff - 1e-3 - bmax * (1.0 / 65536.0);
    if (lim <= 0.0) return 0.0f;
    const float l2 = (float)(lim * lim);
    return (double)l2 > lim * lim ? std::nextafter(l2, 0.0f) : l2;
}

// squared minimum-image distance between sites i and j of a [n][3] position array
__device__ __forceinline__ double pair_dist2(const double* pos, double xi, double yi, double zi, int j, const CellGrid& g) {
    return dist2(min_image(xi - pos[3 * j], g.box[0], g.inv[0]), min_image(yi - pos[3 * j + 1], g.box[1], g.inv[1]),
                 min_image(zi - pos[3 * j + 2], g.box[2], g.inv[2]));
}

// Deterministic sparse dot product of two sorted CSR rows (ascending column order,
// separate multiply and add).
static __device__ double row_dot(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, const double* __restrict__ va,
                          int i, int j) {
    int64_t p = rp[i], pe = rp[i + 1], q = rp[j], qe = rp[j + 1];
    double s = 0.0;
    while (p < pe && q < qe) {
        const int a = ci[p], b = ci[q];
        if (a == b) { s = __dadd_rn(s, __dmul_rn(va[p], va[q])); ++p; ++q; }
        else if (a < b) ++p;
        else ++q;
    }
    return s;
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) gbe_free(p); }
    template <class T> T* as() { return (T*)p; }
};

static inline int read_flag(gbe_ctx* ctx, const int* d, int* h) {
    GBE_CUDA_TRY(cudaMemcpyAsync(h, d, 4, cudaMemcpyDeviceToHost, ctx->stream));
    GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    return GBE_OK;
}


static inline int scan_exclusive(gbe_ctx* ctx, const int32_t* in, int64_t* out, int64_t n, int64_t* total_host) {
    const int nb = (int)((n + kScanBlock - 1) / kScanBlock);
    DevBuf bs;
    GBE_TRY(gbe_alloc(&bs.p, (size_t)(nb + 1) * 8));
    int64_t* tot = bs.as<int64_t>() + nb;
    if (n > 0) scan_local_kernel<<<nb, kScanThreads, 0, ctx->stream>>>(in, out, n, bs.as<int64_t>());
    scan_top_kernel<<<1, kScanThreads, 0, ctx->stream>>>(bs.as<int64_t>(), nb, tot);
    scan_add_kernel<<<(unsigned)((n + 1 + 255) / 256), 256, 0, ctx->stream>>>(out, n, bs.as<int64_t>(), tot);
    GBE_CUDA_TRY(cudaGetLastError());
    if (total_host) {
        GBE_CUDA_TRY(cudaMemcpyAsync(total_host, tot, 8, cudaMemcpyDeviceToHost, ctx->stream));
        GBE_CUDA_TRY(cudaStreamSynchronize(ctx->stream));
    }
    return GBE_OK;
}

// Copy an array to the device when it is on the host.
static inline int to_device(gbe_ctx* ctx, const void* src, size_t bytes, int on_device, DevBuf& hold, const void** out) {
    if (on_device) {
        GBE_TRY(gbe_check_device(ctx, src, bytes, "an input array"));
        *out = src;
        return GBE_OK;
    }
    GBE_TRY(gbe_alloc(&hold.p, bytes));
    GBE_CUDA_TRY(cudaMemcpyAsync(hold.p, src, bytes, cudaMemcpyHostToDevice, ctx->stream));
    *out = hold.p;
    return GBE_OK;
}


}  // namespace gbe_dev
