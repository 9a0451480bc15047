// Shared device-side definitions of the GB300 box-spline filter library.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <string.h>

#include "../../include/bsf.h"

typedef unsigned __int128 u128;
typedef __int128 i128;

// Arithmetic forms of the pre-integrated buffer.
//   MODE_U64  : uint8 image, exact integer running sums modulo 2^64
//   MODE_U128 : float32 image in fixed point (32 fractional bits), sums modulo 2^128
//   MODE_F64  : all-FP64 form (Algorithm 1 computed literally in double)
enum { MODE_U64 = 0, MODE_U128 = 1, MODE_F64 = 2 };

template <int MODE> struct mode_traits;
template <> struct mode_traits<MODE_U64> {
    typedef unsigned long long T;
    static constexpr int ACC_BITS = 64;
    static constexpr int VAL_BITS = 8;    // |f| < 2^8
    static constexpr int FRAC_BITS = 0;
};
template <> struct mode_traits<MODE_U128> {
    typedef u128 T;
    static constexpr int ACC_BITS = 128;
    static constexpr int VAL_BITS = 63;   // |f * 2^32| < 2^63
    static constexpr int FRAC_BITS = 32;
};
template <> struct mode_traits<MODE_F64> {
    typedef double T;
    static constexpr int ACC_BITS = 0;
    static constexpr int VAL_BITS = 0;
    static constexpr int FRAC_BITS = 0;
};

// Round-to-nearest-even of a float to a 64-bit integer (as __float2ll_rn, saturating at
// 2^63; NaN saturates too) with FP32 additions and integer operations only: below 2^23
// adding and subtracting 2^23 with the sign of x rounds to an integer (the sum lies where
// the spacing of floats is 1), above it every float is one; the integer is then read from
// the exponent and mantissa bits
__device__ __forceinline__ long long f32_to_i64_rn(float x) {
    const float t = copysignf(8388608.0f, x);
    const float r = fabsf(x) < 8388608.0f ? (x + t) - t : x;
    const unsigned b = __float_as_uint(r);
    const int ef = (int)((b >> 23) & 0xFFu);
    const long long m = (long long)((b & 0x7FFFFFu) | 0x800000u);
    const int e = ef - 150;  // |r| = m 2^e for a normal r
    long long v = e >= 0 ? (e < 40 ? m << e : 0x7FFFFFFFFFFFFFFFLL) : (e > -24 ? m >> (-e) : 0LL);
    if (ef == 0) v = 0;  // zero (subnormals round to zero above)
    return (b >> 31) ? -v : v;
}
// (64-bit integer <-> float conversions run on the FP64 pipe, 1/64 of the FP32 rate on GB300.)

// Image sample -> accumulator element.
__device__ __forceinline__ unsigned long long to_acc_u64(uint8_t v) { return (unsigned long long)v; }
__device__ __forceinline__ u128 to_acc_u128(float v) {
    // round(v * 2^32) as a signed 64-bit integer (the scaling is exact in FP32), sign-extended to 128 bits
    return (u128)(i128)f32_to_i64_rn(v * 4294967296.0f);
}

template <int MODE, class InT> __device__ __forceinline__ typename mode_traits<MODE>::T load_sample(InT v);
template <> __device__ __forceinline__ unsigned long long load_sample<MODE_U64, uint8_t>(uint8_t v) {
    return to_acc_u64(v);
}
template <> __device__ __forceinline__ u128 load_sample<MODE_U128, float>(float v) { return to_acc_u128(v); }
template <> __device__ __forceinline__ double load_sample<MODE_F64, uint8_t>(uint8_t v) { return (double)v; }
template <> __device__ __forceinline__ double load_sample<MODE_F64, float>(float v) { return (double)v; }

// Warp shuffles of 64/128-bit (and small aggregate) values, split into 32-bit words.
#define BSF_SHFL_T(NAME, CALL)                                                   \
    template <class T> __device__ __forceinline__ T NAME(T v, int d) {           \
        static_assert(sizeof(T) % 4 == 0, "word size");                          \
        unsigned w[sizeof(T) / 4];                                               \
        memcpy(w, &v, sizeof(T));                                                \
        _Pragma("unroll") for (int i = 0; i < (int)(sizeof(T) / 4); ++i) w[i] = CALL; \
        T r;                                                                     \
        memcpy(&r, w, sizeof(T));                                                \
        return r;                                                                \
    }
BSF_SHFL_T(shfl_up_T, __shfl_up_sync(0xffffffffu, w[i], d))
BSF_SHFL_T(shfl_down_T, __shfl_down_sync(0xffffffffu, w[i], d))
BSF_SHFL_T(shfl_idx_T, __shfl_sync(0xffffffffu, w[i], d))
#undef BSF_SHFL_T

// Device status word bits (1 << BSF_E*).
__device__ __forceinline__ void raise_status(unsigned* status, int code) {
    if (status) atomicOr(status, 1u << code);
}

// 128-bit two's-complement integer -> float (round to nearest of the top 64 bits).
__device__ __forceinline__ float i128_to_float(u128 v) {
    bool neg = (long long)(unsigned long long)(v >> 64) < 0;
    u128 m = neg ? (u128)(-(i128)v) : v;
    unsigned long long hi = (unsigned long long)(m >> 64), lo = (unsigned long long)m;
    float r;
    if (hi == 0) {
        r = __ull2float_rn(lo);
    } else {
        int lz = __clzll(hi);               // 0..63
        int sh = 64 - lz;                   // bits to drop so the value fits 64 bits
        u128 t = m >> sh;
        // sticky bit keeps round-to-nearest honest for the dropped part
        unsigned long long top = (unsigned long long)t | (((m & ((((u128)1) << sh) - 1)) != 0) ? 1ull : 0ull);
        r = ldexpf(__ull2float_rn(top), sh);
    }
    return neg ? -r : r;
}

__host__ __device__ __forceinline__ int ceil_div_i(int a, int b) { return (a + b - 1) / b; }
