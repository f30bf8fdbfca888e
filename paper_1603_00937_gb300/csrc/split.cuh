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
#include <cstring>

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

// x = hi + lo with hi = x truncated to a 24-bit significand (exact) and lo the remaining
// 29 bits rounded to FP32 (|lo - (x - hi)| <= 2^-47 |x|), using integer operations only:
// on this part FP64<->FP32 conversions run on the narrow FP64 pipe.  Values below 2^-60
// in magnitude (irrelevant at the 2^-35 resolution of the splits) become 0.
__device__ __forceinline__ void f64_to_f32_pair(double x, float& hi, float& lo) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const uint32_t sign = (uint32_t)(u >> 63) << 31;
    const int e = (int)((u >> 52) & 0x7FF) - 1023;
    if (e < -60) { hi = 0.0f; lo = 0.0f; return; }
    const unsigned long long mant = u & 0xFFFFFFFFFFFFFull;
    hi = __uint_as_float(sign | ((uint32_t)(e + 127) << 23) | (uint32_t)(mant >> 29));
    const float l = (float)(uint32_t)(mant & 0x1FFFFFFFull);                  // units of 2^(e-52)
    lo = l * __uint_as_float((uint32_t)(e - 52 + 127) << 23);
    lo = sign ? -lo : lo;
}

// Two adjacent elements at once (the first in the low 16 bits of every word): the same
// rounding as oz_split_pq, with packed conversions.
struct OzSplit2 {
    uint32_t s0, s1, s2, s1s;
};

__device__ __forceinline__ uint32_t h2_bits(__half2 h) {
    uint32_t u;
    memcpy(&u, &h, 4);
    return u;
}
__device__ __forceinline__ float2 h2_val(uint32_t u) {
    __half2 h;
    memcpy(&h, &u, 4);
    return __half22float2(h);
}

__device__ __forceinline__ OzSplit2 oz_split_pq2(float P0, float Q0, float P1, float Q1) {
    const float y0 = P0 + Q0, y1 = P1 + Q1;
    const float s00 = rintf(y0 * GBE_OZ_S0_SCALE) * (1.0f / GBE_OZ_S0_SCALE);
    const float s01 = rintf(y1 * GBE_OZ_S0_SCALE) * (1.0f / GBE_OZ_S0_SCALE);
    const float r10 = (P0 - s00) + Q0, r11 = (P1 - s01) + Q1;
    const float t0 = r10 * GBE_OZ_R_SCALE, t1 = r11 * GBE_OZ_R_SCALE;
    const __half2 h1 = __floats2half2_rn(t0, t1);
    const float2 f1 = __half22float2(h1);
    OzSplit2 o;
    o.s0 = h2_bits(__floats2half2_rn(s00, s01));
    o.s1 = h2_bits(h1);
    o.s2 = h2_bits(__floats2half2_rn(t0 - f1.x, t1 - f1.y));
    o.s1s = h2_bits(__floats2half2_rn(r10, r11));
    return o;
}

__device__ __forceinline__ double oz_value(uint16_t s0, uint16_t s1, uint16_t s2) {
    return (double)h_val(s0) + ((double)h_val(s1) + (double)h_val(s2)) * (1.0 / 2048.0);
}

__device__ __forceinline__ double bf_value(uint16_t hi, uint16_t lo) {
    return (double)b_val(hi) + (double)b_val(lo);
}

// Double-float (FP32 pair) accumulation: (sh, sl) += (bh, bl).
__device__ __forceinline__ void df_add(float& sh, float& sl, float bh, float bl) {
    const float s = sh + bh;
    const float bp = s - sh;
    const float err = (sh - (s - bp)) + (bh - bp);
    sh = s;
    sl += err + bl;
}

// Double-float accumulation of w * (P + Q)^2 (FP64-grade traces from FP32 parts).
__device__ __forceinline__ void df_add_sq(float& sh, float& sl, float P, float Q, float w) {
    const float p2 = P * P;
    const float e2 = fmaf(P, P, -p2);
    const float th = w * p2;
    const float tl = w * (e2 + Q * (2.0f * P + Q));
    const float s = sh + th;
    const float bp = s - sh;
    const float err = (sh - (s - bp)) + (th - bp);
    sh = s;
    sl += err + tl;
}

// -(ah + al) * (bh + bl) as an FP32 pair (P, Q): the product of the leading parts with its
// exact rounding error (FMA) plus both cross terms; relative error ~2^-47.
__device__ __forceinline__ void neg_mul_pair(float ah, float al, float bh, float bl, float& P, float& Q) {
    const float p = ah * bh;
    float e = fmaf(ah, bh, -p);
    e = fmaf(ah, bl, e);
    e = fmaf(al, bh, e);
    P = -p;
    Q = -e;
}
