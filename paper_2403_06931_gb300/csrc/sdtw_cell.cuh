// One DP cell of Eq. 1 (paper Section 2) for the two arithmetic modes.
//
//   D(i,j) = (x_i - y_j)^2 + min{ D(i-1,j), D(i,j-1), D(i-1,j-1) }
//
// FP32: one subtract, one three-input minimum (sm_100+ min.f32 with three
// sources) and one fused multiply-add; two independent cells share one packed
// f32x2 multiply-add (sm_100+).
// INT:  int8 samples or uint8 codes widened to int32; costs are non-negative int32.  A
// non-negative int32 read as an IEEE float sorts exactly like the integer
// (the bit patterns 0 .. 0x7F7FFFFF are the finite non-negative floats in
// increasing order, subnormals included, and min.f32 without .ftz keeps
// subnormals), so the same three-input float minimum picks the integer
// minimum; d*d + m is one integer multiply-add.
// F16:  the paper's precision (Section 5.2 packs float16 pairs as __half2):
// two queries share a thread as the low and high halves of __half2, against
// the same reference sample in both halves; a packed subtract (rounded, never
// contracted), two packed minimums and a packed fused multiply-add -- four
// instructions for two cells.  Values are absolute (no rebasing), as in the
// paper, and a sum beyond the largest binary16 value becomes +inf.
#pragma once

#include <cuda_fp16.h>

#include <climits>
#include <cstdint>
#include <cstring>

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
    using Col = int;  // a column of the running bottom-row minimum
    static constexpr bool kPair = false;
    // FP32 D values are kept relative to a per-thread base (see sdtw_fill.cuh)
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
    // two independent cells at once: the multiply-adds as one packed
    // f32x2 fused multiply-add (each lane rounded once, exactly as fmaf), so
    // the pair costs five instructions instead of six and every value is
    // the one cell() gives
    static constexpr bool kPack2 = true;
    static __device__ __forceinline__ float2 cell2(V x0, V y0, V up0, V dg0, V lf0, V x1, V y1, V up1, V dg1, V lf1)
    {
        const float2 d = make_float2(x0 - y0, x1 - y1);
        const float2 m = make_float2(min3_f32(up0, dg0, lf0), min3_f32(up1, dg1, lf1));
        return __ffma2_rn(d, d, m);
    }
};

// The integer modes (int8 samples, or uint8 codebook codes): int32 costs.
template <typename T>
struct ModeInt {
    using V = int32_t;
    using Col = int;
    static constexpr bool kPair = false;
    static constexpr bool kPack2 = false;
    static constexpr bool kRebase = false;  // integer sums are exact
    // Largest finite float pattern: above every reachable cost (N <= 32,896
    // samples of at most 255^2 each), and never NaN or infinity.
    static __device__ __forceinline__ V inf() { return 0x7f7fffff; }
    static __device__ __forceinline__ V empty_cost() { return 0x7fffffff; }  // empty query: INT32_MAX
    static __device__ __forceinline__ V zero() { return 0; }
    static __device__ __forceinline__ V widen(T v) { return static_cast<V>(v); }
    static __device__ __forceinline__ V cell(V x, V y, V up, V diag, V left)
    {
        const int32_t d = x - y;
        const int32_t m = __float_as_int(
            min3_f32(__int_as_float(up), __int_as_float(diag), __int_as_float(left)));
        return d * d + m;
    }
    // early-INF pruning (paper Section 8): a cell whose samples differ by more
    // than gap is +inf, and +inf absorbs (d*d + inf stays below 2^31 and is
    // clamped back to inf)
    static __device__ __forceinline__ V cell_pruned(V x, V y, V up, V diag, V left, int gap)
    {
        const int32_t d = x - y;
        const int32_t m = __float_as_int(
            min3_f32(__int_as_float(up), __int_as_float(diag), __int_as_float(left)));
        const int32_t t = min(d * d + m, inf());
        return abs(d) > gap ? inf() : t;
    }
};

template <>
struct Mode<int8_t> : ModeInt<int8_t> {};
template <>
struct Mode<uint8_t> : ModeInt<uint8_t> {};

// Binary16 pairs: two queries per thread (see the F16 note above).
template <>
struct Mode<__half> {
    using V = __half2;
    using Col = int2;  // the two queries' bottom-row minimum columns
    static constexpr bool kRebase = false;
    static constexpr bool kPair = true;
    static constexpr bool kPack2 = false;
    static __device__ __forceinline__ V inf() { return __halves2half2(__ushort_as_half(0x7c00), __ushort_as_half(0x7c00)); }
    static __device__ __forceinline__ V zero() { return __halves2half2(__ushort_as_half(0), __ushort_as_half(0)); }
    static __device__ __forceinline__ V widen(__half v) { return __halves2half2(v, v); }  // a reference sample, both halves
    static __device__ __forceinline__ V pack(__half a, __half b) { return __halves2half2(a, b); }
    static __device__ __forceinline__ V cell(V x, V y, V up, V diag, V left)
    {
        const V d = __hsub2_rn(x, y);
        return __hfma2(d, d, __hmin2(__hmin2(up, diag), left));
    }
    // the running bottom-row minimum of each half: strict '<' keeps the
    // smallest column of exact ties when columns arrive in increasing order
    static __device__ __forceinline__ void bot_update(V v, int col, V& best, int2& bc)
    {
        const __half lo = __low2half(v), hi = __high2half(v);
        __half blo = __low2half(best), bhi = __high2half(best);
        if (__hlt(lo, blo)) {
            blo = lo;
            bc.x = col;
        }
        if (__hlt(hi, bhi)) {
            bhi = hi;
            bc.y = col;
        }
        best = __halves2half2(blo, bhi);
    }
    static __device__ __forceinline__ uint32_t bits(V v)
    {
        uint32_t u;
        memcpy(&u, &v, 4);
        return u;
    }
    static __device__ __forceinline__ V from_bits(uint32_t u)
    {
        V v;
        memcpy(&v, &u, 4);
        return v;
    }
};

}  // namespace sdtw
