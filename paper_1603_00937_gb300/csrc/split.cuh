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
// FP64TC (ten planes): x rounded to the fixed-point grid 2^-50, V = x 2^50 (int64, |V| <= 2^50),
//   cut into digits k0..k4 by rounding to nearest at 2^40, 2^30, 2^20, 2^10:
//   x = t0 + 2^-10 t1 + 2^-20 t2 + 2^-30 t3 + 2^-40 t4,  t_p = k_p 2^-10 (|k0| <= 1024,
//   |k1..k4| <= 512: every t_p exact in fp16), and t1 = u + v with u = round(32 t1) / 32,
//   v = t1 - u (|v| <= 2^-6).  Stored planes (this order, so that the A operand takes planes
//   0-8 and the B operand planes 1-9 in one box each):
//     0 u' = u 2^-10, 1 t0, 2 t1, 3 t2, 4 t3, 5 u, 6 v, 7 t3' = t3 2^-10, 8 t4' = t4 2^-10,
//     9 t2' = t2 2^-10 (every scaled value a multiple of 2^-20 below 2^-9 in magnitude:
//     exact in fp16, subnormals included).
//   X^2 = ACC0 + 2^-10 ACC1 + 2^-20 ACC2 + 2^-30 ACC3 with
//     ACC0 = t0 t0                                  (grid 2^-20, |partial sums| <= 1)
//     ACC1 = t0 t1 + t1 t0 + u' u                   (grid 2^-20)
//     ACC2 = t0 t2 + t2 t0 + u v + v u + v v        (grid 2^-20)
//     ACC3 = t0 t3 + t3 t0 + t1 t2 + t2 t1 + t0 t4' + t4' t0 + t1 t3' + t3' t1 + t2 t2'
//   ACC0..ACC2 are exact in FP32 while every partial sum stays below 16 (2^24 units of
//   2^-20); t1 t1 is taken as u u + u v + v u + v v because its diagonal (a row's sum of
//   squares, ~K/12) would not be.  ACC3 carries the 2^-30 and (pre-scaled) 2^-40 levels and
//   needs no exactness; the levels from 2^-50 on are dropped.  The rounding of ACC3 (one
//   FP32 rounding per MMA at |ACC3| ~ 4, i.e. ~2^-52 of x per addition) and the dropped
//   2^-50 level (~2^-49 of x) leave each squaring within a few 1e-15 of the exact one.
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

// ---------------------------------------------------------------------------- FP64TC digits
#define GBE_F64TC_PLANES 10
struct F64Digits {
    int k0, k1, k2, k3, k4;
};
// Digits of V = x 2^50 (round to nearest at each level; |V| <= 2^50).
__device__ __forceinline__ F64Digits f64tc_digits(long long V) {
    F64Digits d;
    const long long q0 = (V + (1LL << 39)) >> 40;
    long long r = V - (q0 << 40);
    const long long q1 = (r + (1LL << 29)) >> 30;
    int r1 = (int)(r - (q1 << 30));
    d.k0 = (int)q0;
    d.k1 = (int)q1;
    d.k2 = (r1 + (1 << 19)) >> 20;
    r1 -= d.k2 << 20;
    d.k3 = (r1 + (1 << 9)) >> 10;
    d.k4 = r1 - (d.k3 << 10);
    return d;
}
__device__ __forceinline__ long long f64tc_value(int k0, int k1, int k2, int k3, int k4) {
    return ((long long)k0 << 40) + ((long long)k1 << 30) + ((long long)k2 << 20) + ((long long)k3 << 10) + (long long)k4;
}
// plane halves of a pair of digit sets (first element in the low 16 bits of each word)
__device__ __forceinline__ void f64tc_planes2(const F64Digits& a, const F64Digits& b, uint32_t (&w)[GBE_F64TC_PLANES]) {
    const int ua = (a.k1 + 16) >> 5, ub = (b.k1 + 16) >> 5;
    const int va = a.k1 - 32 * ua, vb = b.k1 - 32 * ub;
    const float s10 = 1.0f / 1024.0f, s20 = 1.0f / 1048576.0f;
    w[0] = h2_bits(__floats2half2_rn((float)ua * (1.0f / 32768.0f), (float)ub * (1.0f / 32768.0f)));
    w[1] = h2_bits(__floats2half2_rn((float)a.k0 * s10, (float)b.k0 * s10));
    w[2] = h2_bits(__floats2half2_rn((float)a.k1 * s10, (float)b.k1 * s10));
    w[3] = h2_bits(__floats2half2_rn((float)a.k2 * s10, (float)b.k2 * s10));
    w[4] = h2_bits(__floats2half2_rn((float)a.k3 * s10, (float)b.k3 * s10));
    w[5] = h2_bits(__floats2half2_rn((float)ua * (1.0f / 32.0f), (float)ub * (1.0f / 32.0f)));
    w[6] = h2_bits(__floats2half2_rn((float)va * s10, (float)vb * s10));
    w[7] = h2_bits(__floats2half2_rn((float)a.k3 * s20, (float)b.k3 * s20));
    w[8] = h2_bits(__floats2half2_rn((float)a.k4 * s20, (float)b.k4 * s20));
    w[9] = h2_bits(__floats2half2_rn((float)a.k2 * s20, (float)b.k2 * s20));
}
// V of an element from its stored planes t0 (1), t1 (2), t2 (3), t3 (4), t4' (8)
__device__ __forceinline__ long long f64tc_from_planes(uint16_t t0, uint16_t t1, uint16_t t2, uint16_t t3, uint16_t t4s) {
    return f64tc_value(__float2int_rn(h_val(t0) * 1024.0f), __float2int_rn(h_val(t1) * 1024.0f),
                       __float2int_rn(h_val(t2) * 1024.0f), __float2int_rn(h_val(t3) * 1024.0f),
                       __float2int_rn(h_val(t4s) * 1048576.0f));
}
// x as an FP32 pair (P exact: the 2^-10 and 2^-20 digits; Q the rest, rounded)
__device__ __forceinline__ void f64tc_pair(const F64Digits& d, float& P, float& Q) {
    P = (float)d.k0 * (1.0f / 1024.0f) + (float)d.k1 * (1.0f / 1048576.0f);
    Q = (float)d.k2 * 9.313225746154785e-10f + ((float)d.k3 * 9.094947017729282e-13f + (float)d.k4 * 8.881784197001252e-16f);
}
