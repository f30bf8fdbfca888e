// Split formats of a submatrix element for the tensor-core squarings.
//
// FP16X6 (planes s0, s1, s2, s1s):
//   s0  = x rounded to the fixed-point grid 2^-10 (|x| <= ~1, so |s0| <= 1024 * 2^-10 is exact
//         in fp16); products of two s0 values are multiples of 2^-20 and every partial sum
//         of a row-by-column product is bounded by ||x_i|| ||x_j|| <= 1 (the spectrum of
//         every SP2 iterate lies in [0, 1]), so FP32 accumulation of s0 * s0 is exact.
//   r1  = x - s0 (|r1| <= 2^-11),  t = r1 * 2^11,
//   s1  = fp16(t),  s2 = fp16(t - s1),  s1s = fp16(r1)  (unscaled residual for s1 * s1).
//   x  ~= s0 + 2^-11 (s1 + s2), absolute representation error ~2^-34.
//   X^2 ~= s0 s0^T + 2^-11 (s0 s1^T + s1 s0^T + s1 s1s^T + s0 s2^T + s2 s0^T)
//         (the first product in one accumulator, the five others in a second one).
// BF16X3 (planes hi, lo): hi = bf16(x), lo = bf16(x - hi);  X^2 ~= hi hi + hi lo + lo hi.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

#define GBE_OZ_S0_SCALE 1024.0f          // 2^10
#define GBE_OZ_R_SCALE 2048.0f           // 2^11
#define GBE_OZ_R_INV (1.0f / 2048.0f)

struct OzSplit {
    uint16_t s0, s1, s2, s1s;
};

__device__ __forceinline__ uint16_t h_bits(__half h) { return __half_as_ushort(h); }
__device__ __forceinline__ float h_val(uint16_t b) { return __half2float(__ushort_as_half(b)); }
__device__ __forceinline__ uint16_t b_bits(__nv_bfloat16 h) { return __bfloat16_as_ushort(h); }
__device__ __forceinline__ float b_val(uint16_t b) { return __bfloat162float(__ushort_as_bfloat16(b)); }

// Split of x = P + Q where P is an exact fp32 multiple of 2^-20 and Q a small fp32 correction.
__device__ __forceinline__ OzSplit oz_split_pq(float P, float Q) {
    float y = P + Q;
    float s0 = rintf(y * GBE_OZ_S0_SCALE) * (1.0f / GBE_OZ_S0_SCALE);
    float r1 = (P - s0) + Q;
    float t = r1 * GBE_OZ_R_SCALE;
    __half h1 = __float2half_rn(t);
    float rest = t - __half2float(h1);
    OzSplit o;
    o.s0 = h_bits(__float2half_rn(s0));
    o.s1 = h_bits(h1);
    o.s2 = h_bits(__float2half_rn(rest));
    o.s1s = h_bits(__float2half_rn(r1));
    return o;
}

// Split of an FP64 value (gather of X_0).
__device__ __forceinline__ OzSplit oz_split_d(double x) {
    double s0 = rint(x * 1024.0) * (1.0 / 1024.0);
    double r1 = x - s0;
    double t = r1 * 2048.0;
    __half h1 = __double2half(t);
    double rest = t - (double)__half2float(h1);
    OzSplit o;
    o.s0 = h_bits(__double2half(s0));
    o.s1 = h_bits(h1);
    o.s2 = h_bits(__double2half(rest));
    o.s1s = h_bits(__double2half(r1));
    return o;
}

__device__ __forceinline__ double oz_value(uint16_t s0, uint16_t s1, uint16_t s2) {
    return (double)h_val(s0) + ((double)h_val(s1) + (double)h_val(s2)) * (1.0 / 2048.0);
}

__device__ __forceinline__ double bf_value(uint16_t hi, uint16_t lo) {
    return (double)b_val(hi) + (double)b_val(lo);
}
