// One DP cell of Eq. 1 (paper Section 2) for the two arithmetic modes.
//
//   D(i,j) = (x_i - y_j)^2 + min{ D(i-1,j), D(i,j-1), D(i-1,j-1) }
//
// FP32: one subtract, one three-input minimum (sm_100+ min.f32 with three
// sources) and one fused multiply-add.
// INT:  int8 samples widened to int32; costs are non-negative int32.  A
// non-negative int32 read as an IEEE float sorts exactly like the integer
// (the bit patterns 0 .. 0x7F7FFFFF are the finite non-negative floats in
// increasing order, subnormals included, and min.f32 without .ftz keeps
// subnormals), so the same three-input float minimum picks the integer
// minimum; d*d + m is one integer multiply-add.
#pragma once

#include <cstdint>

namespace sdtw {

__device__ __forceinline__ float min3_f32(float a, float b, float c)
{
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

template <typename Tin>
struct Mode;

template <>
struct Mode<float> {
    using V = float;  // x, y and D
    // FP32 D values are kept relative to a per-thread base (see sdtw_forward.cu)
    static constexpr bool kRebase = true;
    static __device__ __forceinline__ V inf() { return __int_as_float(0x7f800000); }
    static __device__ __forceinline__ V empty_cost() { return inf(); }  // empty query
    static __device__ __forceinline__ V zero() { return 0.0f; }
    static __device__ __forceinline__ V widen(float v) { return v; }
    static __device__ __forceinline__ V cell(V x, V y, V up, V diag, V left)
    {
        const float d = x - y;
        return fmaf(d, d, min3_f32(up, diag, left));
    }
};

template <>
struct Mode<int8_t> {
    using V = int32_t;
    static constexpr bool kRebase = false;  // integer sums are exact
    // Largest finite float pattern: above every reachable cost (N <= 33,000
    // samples of at most 254^2 each), and never NaN or infinity.
    static __device__ __forceinline__ V inf() { return 0x7f7fffff; }
    static __device__ __forceinline__ V empty_cost() { return 0x7fffffff; }  // empty query: INT32_MAX
    static __device__ __forceinline__ V zero() { return 0; }
    static __device__ __forceinline__ V widen(int8_t v) { return static_cast<V>(v); }
    static __device__ __forceinline__ V cell(V x, V y, V up, V diag, V left)
    {
        const int32_t d = x - y;
        const int32_t m = __float_as_int(
            min3_f32(__int_as_float(up), __int_as_float(diag), __int_as_float(left)));
        return d * d + m;
    }
};

}  // namespace sdtw
