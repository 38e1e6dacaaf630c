// Shared device helpers of the Léja log-determinant library (sm_103a).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "leja.h"

namespace ll {

// ------------------------------------------------------------------------------------------------
// Counter-based probe generator: the SplitMix64 output function (Steele, Lea & Flood 2014)
// applied to z + 0x9E3779B97F4A7C15, used as a hash of (seed, stream, column, row).
// ------------------------------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
    z += 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__host__ __device__ __forceinline__ uint64_t probe_bits(uint64_t seed, uint32_t stream, uint32_t col, uint32_t row) {
    const uint64_t ctr = ((uint64_t)stream << 56) | ((uint64_t)col << 32) | (uint64_t)row;
    return splitmix_mix(seed ^ splitmix_mix(ctr));
}

__device__ __forceinline__ double probe_value(int kind, uint64_t seed, uint32_t stream, uint32_t col, uint32_t row) {
    const uint64_t x = probe_bits(seed, stream, col, row);
    if (kind == LL_PROBE_RADEMACHER) return (x >> 63) ? -1.0 : 1.0;
    // Box-Muller: u1 in (0, 1], u2 in [0, 1)
    const double u1 = (double)((x >> 11) + 1ull) * 0x1.0p-53;
    const double u2 = (double)(splitmix_mix(x) >> 11) * 0x1.0p-53;
    return sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
}

// ------------------------------------------------------------------------------------------------
// Double-float ("df64") arithmetic: a value is an unevaluated sum hi + lo of two floats with
// |lo| <= ulp(hi)/2 after normalisation. Error-free transformations after Dekker (1971) and
// Knuth (TAOCP vol. 2): TwoSum, and TwoProd via FMA. The __f*_rn intrinsics keep the compiler
// from contracting the steps into FMAs, which would break the error-free transformations.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ void df_mac(float& sh, float& sl, float xh, float xl, float yh, float yl) {
    // (sh, sl) += (xh + xl) * (yh + yl), dropping xl*yl; sl collects every rounding error
    const float p = __fmul_rn(xh, yh);
    float e = __fmaf_rn(xh, yh, -p);
    e = __fmaf_rn(xh, yl, e);
    e = __fmaf_rn(xl, yh, e);
    const float s = __fadd_rn(sh, p);
    const float bb = __fsub_rn(s, sh);
    const float err = __fadd_rn(__fsub_rn(sh, __fsub_rn(s, bb)), __fsub_rn(p, bb));
    sh = s;
    sl = __fadd_rn(sl, __fadd_rn(err, e));
}

__device__ __forceinline__ float2 df_norm(float sh, float sl) {
    const float s = __fadd_rn(sh, sl);
    const float e = __fsub_rn(sl, __fsub_rn(s, sh));
    return make_float2(s, e);
}

__host__ __device__ __forceinline__ float2 df_split(double x) {
    const float hi = (float)x;
    const float lo = (float)(x - (double)hi);
    return make_float2(hi, lo);
}

__device__ __forceinline__ double df_to_double(float2 v) { return (double)v.x + (double)v.y; }

// A double as an unevaluated float pair hi + lo, from its bit fields with integer operations and
// one integer-to-float conversion (GB300 runs FP64 instructions, conversions from double among
// them, at a small fraction of the FP32 rate): hi takes the sign, the exponent and the leading 23
// stored mantissa bits (truncated), lo the remaining 29 bits rounded to 24, scaled by
// 2^(e - 52). |x - hi - lo| <= 2^-47 |x|. Values outside the float pair's exponent range (zero,
// subnormals, |x| >= 2^128, inf, nan) take the plain conversion and lo = 0.
__device__ __forceinline__ void split_bits(double x, float& h, float& l) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x);
    const unsigned int hw = (unsigned int)(u >> 32);
    const int e = (int)((hw >> 20) & 0x7ffu) - 1023;
    if (e < -126 || e > 127) {
        h = (e < -126) ? __uint_as_float(hw & 0x80000000u) : __double2float_rn(x);
        l = 0.f;
        return;
    }
    const unsigned int sign = hw & 0x80000000u;
    const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
    h = __uint_as_float(sign | ((unsigned int)(e + 127) << 23) | (unsigned int)(m >> 29));
    const float lf = __uint2float_rn((unsigned int)(m & 0x1FFFFFFFull));
    l = ldexpf(sign ? -lf : lf, e - 52);
}

// ------------------------------------------------------------------------------------------------
// Packed FP32 pairs (Blackwell f32x2 instructions): two floats in one 64-bit register, the first
// in the low word. One instruction performs the operation on both lanes with IEEE RN rounding.
// ------------------------------------------------------------------------------------------------
typedef unsigned long long f2x;

__device__ __forceinline__ f2x f2_pack(float a, float b) {
    f2x r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void f2_unpack(f2x v, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v));
}
__device__ __forceinline__ f2x f2_fma(f2x a, f2x b, f2x c) {
    f2x d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2x f2_mul(f2x a, f2x b) {
    f2x d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x f2_add(f2x a, f2x b) {
    f2x d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2x f2_sub(f2x a, f2x b) {
    f2x d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// (sh, sl) += a * (xh + xl) on both lanes, a = ah + al a double-float scalar broadcast to both
// lanes as ah2 = (ah, ah), al2 = (al, al), nah2 = (-ah, -ah). Same operations, in the same order,
// as df_mac on each lane: q = -round(ah*xh) so fma(ah, xh, q) is the exact product error.
__device__ __forceinline__ void df2_mac(f2x& sh, f2x& sl, f2x ah2, f2x al2, f2x nah2, f2x xh2, f2x xl2) {
    const f2x q = f2_mul(nah2, xh2);
    f2x e = f2_fma(ah2, xh2, q);
    e = f2_fma(ah2, xl2, e);
    e = f2_fma(al2, xh2, e);
    const f2x s = f2_sub(sh, q);
    const f2x bb = f2_sub(s, sh);
    const f2x t2 = f2_sub(sh, f2_sub(s, bb));
    const f2x t3 = f2_add(q, bb);
    sl = f2_add(sl, f2_add(f2_sub(t2, t3), e));
    sh = s;
}
// (sh, sl) += a * x on both lanes for a double-float scalar a and plain float pairs x (lo = 0).
__device__ __forceinline__ void df2_mac_f(f2x& sh, f2x& sl, f2x ah2, f2x al2, f2x nah2, f2x x2) {
    const f2x q = f2_mul(nah2, x2);
    f2x e = f2_fma(ah2, x2, q);
    e = f2_fma(al2, x2, e);
    const f2x s = f2_sub(sh, q);
    const f2x bb = f2_sub(s, sh);
    const f2x t2 = f2_sub(sh, f2_sub(s, bb));
    const f2x t3 = f2_add(q, bb);
    sl = f2_add(sl, f2_add(f2_sub(t2, t3), e));
    sh = s;
}
// (sh, sl) += (xh + xl) * (yh + yl) lane-wise for two double-float pairs; nxh2 = -xh2.
__device__ __forceinline__ void df2_mac_pp(f2x& sh, f2x& sl, f2x xh2, f2x xl2, f2x nxh2, f2x yh2, f2x yl2) {
    const f2x q = f2_mul(nxh2, yh2);
    f2x e = f2_fma(xh2, yh2, q);
    e = f2_fma(xh2, yl2, e);
    e = f2_fma(xl2, yh2, e);
    const f2x s = f2_sub(sh, q);
    const f2x bb = f2_sub(s, sh);
    const f2x t2 = f2_sub(sh, f2_sub(s, bb));
    const f2x t3 = f2_add(q, bb);
    sl = f2_add(sl, f2_add(f2_sub(t2, t3), e));
    sh = s;
}
// (ah, al) += (bh, bl) on both lanes of double-float pairs: TwoSum (Knuth) of the leading parts,
// the trailing parts added to the error, then a renormalisation (FastTwoSum)
__device__ __forceinline__ void df2_add(f2x& ah, f2x& al, f2x bh, f2x bl) {
    const f2x s = f2_add(ah, bh);
    const f2x bb = f2_sub(s, ah);
    f2x e = f2_add(f2_sub(ah, f2_sub(s, bb)), f2_sub(bh, bb));
    e = f2_add(e, f2_add(al, bl));
    ah = f2_add(s, e);
    al = f2_sub(e, f2_sub(ah, s));
}
__device__ __forceinline__ void df2_norm(f2x sh, f2x sl, f2x& h, f2x& l) {
    const f2x s = f2_add(sh, sl);
    l = f2_sub(sl, f2_sub(s, sh));
    h = s;
}

// ------------------------------------------------------------------------------------------------
// Double-float blocks are stored in column pairs: the 16 bytes of pair (2q, 2q+1) of a row hold
// (hi_2q, hi_2q+1, lo_2q, lo_2q+1), so one 16-byte load yields the hi pair and the lo pair of two
// columns, ready for the f32x2 instructions. Leading dimensions (in columns) of such blocks are
// even, so a flat element index i = row * ld + col keeps the parity of col. `dfp` is the element
// tag of these blocks (a float array of 2 * n * ld entries).
// ------------------------------------------------------------------------------------------------
struct dfp {
    float f;
};
__host__ __device__ __forceinline__ size_t dfp_hi(size_t i) { return (i >> 1) * 4 + (i & 1); }

// Typed load/store of block elements as FP64.
template <typename T> __device__ __forceinline__ double load_f64(const T* p, size_t i);
template <> __device__ __forceinline__ double load_f64<double>(const double* p, size_t i) { return p[i]; }
template <> __device__ __forceinline__ double load_f64<float>(const float* p, size_t i) { return (double)p[i]; }
template <> __device__ __forceinline__ double load_f64<float2>(const float2* p, size_t i) { return df_to_double(p[i]); }

template <typename T> __device__ __forceinline__ void store_f64(T* p, size_t i, double v);
template <> __device__ __forceinline__ void store_f64<double>(double* p, size_t i, double v) { p[i] = v; }
template <> __device__ __forceinline__ void store_f64<float>(float* p, size_t i, double v) { p[i] = (float)v; }
template <> __device__ __forceinline__ void store_f64<float2>(float2* p, size_t i, double v) { p[i] = df_split(v); }
template <> __device__ __forceinline__ double load_f64<dfp>(const dfp* p, size_t i) {
    const float* f = reinterpret_cast<const float*>(p) + dfp_hi(i);
    return (double)f[0] + (double)f[2];
}
template <> __device__ __forceinline__ void store_f64<dfp>(dfp* p, size_t i, double v) {
    float* f = reinterpret_cast<float*>(p) + dfp_hi(i);
    const float2 s = df_split(v);
    f[0] = s.x;
    f[2] = s.y;
}

}  // namespace ll
