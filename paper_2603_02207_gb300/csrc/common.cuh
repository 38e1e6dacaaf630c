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

// Typed load/store of block elements as FP64.
template <typename T> __device__ __forceinline__ double load_f64(const T* p, size_t i);
template <> __device__ __forceinline__ double load_f64<double>(const double* p, size_t i) { return p[i]; }
template <> __device__ __forceinline__ double load_f64<float>(const float* p, size_t i) { return (double)p[i]; }
template <> __device__ __forceinline__ double load_f64<float2>(const float2* p, size_t i) { return df_to_double(p[i]); }

template <typename T> __device__ __forceinline__ void store_f64(T* p, size_t i, double v);
template <> __device__ __forceinline__ void store_f64<double>(double* p, size_t i, double v) { p[i] = v; }
template <> __device__ __forceinline__ void store_f64<float>(float* p, size_t i, double v) { p[i] = (float)v; }
template <> __device__ __forceinline__ void store_f64<float2>(float2* p, size_t i, double v) { p[i] = df_split(v); }

}  // namespace ll
