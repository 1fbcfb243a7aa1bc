// Batch z-normalisation (paper Section 5.1, Eq. 2): every series of a batch
// becomes (x - mean) / S with its own mean and population standard deviation
// S; a series with S == 0 is only centred.
//
// The paper's normaliser runs one block per query, each thread summing a few
// elements and a shared-memory tree reducing the partial sums and sums of
// squares, then applies Eq. 2 from the variance sumSq/n - mean^2.  Here one
// warp (short series) or one CTA (long series) per series makes two
// reduction passes, the mean and then the centred second moment: the one-pass
// difference cancels digits when the mean is large against the spread.  FP64
// runs at a small fraction of the FP32 rate on this part (a version with
// double reductions spent most of its time in them), so everything is FP32,
// with compensated float pairs (hi + lo) where one float is not enough:
//   * each lane sums x - x[0] (shifting by the series' first sample removes a
//     large common offset) with Kahan compensation, and the lanes' partial
//     sums are combined as float pairs (error-free TwoSum);
//   * the mean is the float pair x[0] + S/n (a pair division by n), and every
//     sample is centred as (x - hi) - lo, accurate to about one float rounding;
//     the centred squares are again Kahan-summed and pair-reduced; the scale is
//     1 / sqrt(variance) in float.
// Series of up to 2,048 samples stay in the warp's registers between the
// passes; longer ones are read three times (the second and third reads hit
// L2 for query-sized series).  HBM sees one read and one write per sample.
//
// For queries the library normalises itself, the derivative of Eq. 2
// (znorm_vjp_kernel) carries a gradient with respect to the normalised series
// back to the raw one.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstdint>

#include "sdtw_internal.h"

namespace {

constexpr int kNormThreads = 256;
constexpr int kWarpMaxN = 16384;  // uniform series up to this length take one warp each

// A value carried as an unevaluated sum of two floats, hi + lo.
struct FF {
    float hi, lo;
};

// error-free sums (TwoSum; FastTwoSum when |a| >= |b|)
__device__ __forceinline__ FF two_sum(float a, float b)
{
    const float s = a + b;
    const float bb = s - a;
    return {s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ FF fast_two_sum(float a, float b)
{
    const float s = a + b;
    return {s, b - (s - a)};
}

__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const FF s = two_sum(a.hi, b.hi);
    return fast_two_sum(s.hi, s.lo + (a.lo + b.lo));
}

// a / n for a count n (the remainder of the first quotient is exact by FMA)
__device__ __forceinline__ FF ff_div(FF a, float n)
{
    const float q1 = a.hi / n;
    const float r = fmaf(-q1, n, a.hi) + a.lo;
    return fast_two_sum(q1, r / n);
}

// Kahan-compensated running sum; its value is the pair (s, -c)
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ FF value() const { return {s, -c}; }
};

__device__ __forceinline__ FF warp_sum(FF v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1)
        v = ff_add(v, FF{__shfl_xor_sync(0xffffffffu, v.hi, off), __shfl_xor_sync(0xffffffffu, v.lo, off)});
    return v;
}

// sum over the CTA of one pair per thread, returned to every thread
__device__ __forceinline__ FF block_sum(FF v, FF* red)
{
    v = warp_sum(v);
    __syncthreads();  // red[] may still be read by the previous reduction
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    FF t = red[0];
#pragma unroll
    for (int w = 1; w < kNormThreads / 32; ++w) t = ff_add(t, red[w]);
    return t;
}

// the scale 1 / S from the sum of squares (1 when the spread is zero)
__device__ __forceinline__ float inv_spread(FF sq, float n)
{
    const float var = ff_div(sq, n).hi;
    return var > 0.f ? 1.f / sqrtf(var) : 1.f;
}

// Eq. 2 on one series of n samples at x (written to z), by `count` threads
// with index `idx`; REDUCE sums a pair over those threads.
template <typename Reduce>
__device__ __forceinline__ void znorm_series(const float* x, float* z, int64_t n, int idx, int count, Reduce reduce)
{
    const float x0 = x[0];
    const float nf = static_cast<float>(n);
    KSum s1;
    for (int64_t i = idx; i < n; i += count) s1.add(x[i] - x0);
    const FF mean = ff_add(FF{x0, 0.f}, ff_div(reduce(s1.value()), nf));
    KSum s2;
    for (int64_t i = idx; i < n; i += count) {
        const float c = (x[i] - mean.hi) - mean.lo;
        s2.add(c * c);
    }
    const float inv = inv_spread(reduce(s2.value()), nf);
    // each thread rewrites only elements it read itself: safe in place
    for (int64_t i = idx; i < n; i += count) z[i] = ((x[i] - mean.hi) - mean.lo) * inv;
}

// The series q of a batch: [a, a + n) of the buffers; false for an empty or
// malformed series, or one reaching past `limit` elements (limit < 0: none),
// which is then reported in *status (if given) and left untouched.
__device__ __forceinline__ bool series_of(const int64_t* offsets, int32_t N, int q, int64_t limit, int* status,
                                          int64_t& a, int64_t& n)
{
    if (offsets) {
        a = offsets[q];
        n = offsets[q + 1] - a;
        if (a < 0 || n <= 0) return false;
    } else {
        a = static_cast<int64_t>(q) * N;
        n = N;
    }
    if (limit >= 0 && a + n > limit) {
        if (status && threadIdx.x == 0) atomicOr(status, sdtw::kStatusBadLength);
        return false;
    }
    return true;
}

// one CTA per series: long series, and ragged batches (lengths on the device)
__global__ void __launch_bounds__(kNormThreads)
znorm_kernel(const float* in, float* out, const int64_t* offsets, int32_t N, int64_t limit, int* status)
{
    __shared__ FF red[kNormThreads / 32];
    int64_t a, n;
    if (!series_of(offsets, N, blockIdx.x, limit, status, a, n)) return;
    znorm_series(in + a, out + a, n, threadIdx.x, kNormThreads, [&](FF v) { return block_sum(v, red); });
}

// The derivative of Eq. 2 applied to a gradient: for z = (x - mean) * inv
// (inv = 1/S, or 1 for a series with S == 0),
//   dcost/dx_k = inv * (g_k - mean(g) - z_k * mean(g z))
// with g = dcost/dz, rewritten in place.  z and inv are recomputed from x with
// the normaliser's own arithmetic; the two sums are compensated.  One CTA per
// series.
__global__ void __launch_bounds__(kNormThreads)
znorm_vjp_kernel(const float* x, float* g, const int64_t* offsets, int32_t N, int64_t limit)
{
    __shared__ FF red[kNormThreads / 32];
    int64_t a, n;
    if (!series_of(offsets, N, blockIdx.x, limit, nullptr, a, n)) return;
    const float* xs = x + a;
    float* gs = g + a;
    const int idx = threadIdx.x;
    const float x0 = xs[0];
    const float nf = static_cast<float>(n);
    KSum s1;
    for (int64_t i = idx; i < n; i += kNormThreads) s1.add(xs[i] - x0);
    const FF mean = ff_add(FF{x0, 0.f}, ff_div(block_sum(s1.value(), red), nf));
    KSum s2;
    for (int64_t i = idx; i < n; i += kNormThreads) {
        const float c = (xs[i] - mean.hi) - mean.lo;
        s2.add(c * c);
    }
    const float inv = inv_spread(block_sum(s2.value(), red), nf);
    KSum sg, sgz;
    for (int64_t i = idx; i < n; i += kNormThreads) {
        const float z = ((xs[i] - mean.hi) - mean.lo) * inv;
        sg.add(gs[i]);
        sgz.add(gs[i] * z);
    }
    const FF tg = block_sum(sg.value(), red);
    const FF tgz = block_sum(sgz.value(), red);
    const float mg = ff_div(tg, nf).hi, mgz = ff_div(tgz, nf).hi;
    for (int64_t i = idx; i < n; i += kNormThreads) {
        const float z = ((xs[i] - mean.hi) - mean.lo) * inv;
        gs[i] = inv * (gs[i] - mg - z * mgz);
    }
}

// The same with 16-byte loads and stores: series of a multiple of 4 samples
// starting on a 16-byte boundary.
__device__ __forceinline__ void znorm_series_v4(const float4* x, float4* z, int n4, int lane)
{
    const float x0 = reinterpret_cast<const float*>(x)[0];
    const float nf = 4.f * n4;
    KSum s1;
    for (int i = lane; i < n4; i += 32) {
        const float4 v = x[i];
        s1.add(v.x - x0);
        s1.add(v.y - x0);
        s1.add(v.z - x0);
        s1.add(v.w - x0);
    }
    const FF mean = ff_add(FF{x0, 0.f}, ff_div(warp_sum(s1.value()), nf));
    const float hi = mean.hi, lo = mean.lo;
    KSum s2;
    for (int i = lane; i < n4; i += 32) {
        const float4 v = x[i];
        const float c0 = (v.x - hi) - lo, c1 = (v.y - hi) - lo, c2 = (v.z - hi) - lo, c3 = (v.w - hi) - lo;
        s2.add(c0 * c0);
        s2.add(c1 * c1);
        s2.add(c2 * c2);
        s2.add(c3 * c3);
    }
    const float inv = inv_spread(warp_sum(s2.value()), nf);
    for (int i = lane; i < n4; i += 32) {
        const float4 v = x[i];
        z[i] = make_float4(((v.x - hi) - lo) * inv, ((v.y - hi) - lo) * inv, ((v.z - hi) - lo) * inv,
                           ((v.w - hi) - lo) * inv);
    }
}

// The same for a series of up to 32 * 4 * kRegVec4 samples held in the warp's
// registers: one read and one write per sample, no second or third pass over
// memory.
constexpr int kRegVec4 = 16;  // float4 per lane: series of up to 2,048 samples

__device__ __forceinline__ void znorm_series_regs(const float4* x, float4* z, int n4, int lane)
{
    float4 v[kRegVec4];
#pragma unroll
    for (int k = 0; k < kRegVec4; ++k)
        v[k] = lane + 32 * k < n4 ? x[lane + 32 * k] : make_float4(0.f, 0.f, 0.f, 0.f);
    const float x0 = __shfl_sync(0xffffffffu, v[0].x, 0);
    const float nf = 4.f * n4;
    KSum s1;
#pragma unroll
    for (int k = 0; k < kRegVec4; ++k) {
        if (lane + 32 * k < n4) {
            s1.add(v[k].x - x0);
            s1.add(v[k].y - x0);
            s1.add(v[k].z - x0);
            s1.add(v[k].w - x0);
        }
    }
    const FF mean = ff_add(FF{x0, 0.f}, ff_div(warp_sum(s1.value()), nf));
    const float hi = mean.hi, lo = mean.lo;
    KSum s2;
#pragma unroll
    for (int k = 0; k < kRegVec4; ++k) {
        v[k] = make_float4((v[k].x - hi) - lo, (v[k].y - hi) - lo, (v[k].z - hi) - lo, (v[k].w - hi) - lo);
        if (lane + 32 * k < n4) {
            s2.add(v[k].x * v[k].x);
            s2.add(v[k].y * v[k].y);
            s2.add(v[k].z * v[k].z);
            s2.add(v[k].w * v[k].w);
        }
    }
    const float inv = inv_spread(warp_sum(s2.value()), nf);
#pragma unroll
    for (int k = 0; k < kRegVec4; ++k)
        if (lane + 32 * k < n4) z[lane + 32 * k] = make_float4(v[k].x * inv, v[k].y * inv, v[k].z * inv, v[k].w * inv);
}

__global__ void __launch_bounds__(kNormThreads)
znorm_warp_regs_kernel(const float* in, float* out, int32_t B, int32_t N)
{
    const int q = blockIdx.x * (kNormThreads / 32) + (threadIdx.x >> 5);
    if (q >= B) return;
    const int64_t a = static_cast<int64_t>(q) * N;
    znorm_series_regs(reinterpret_cast<const float4*>(in + a), reinterpret_cast<float4*>(out + a), N / 4,
                      threadIdx.x & 31);
}

// one warp per series (eight series per CTA): no CTA barrier
__global__ void __launch_bounds__(kNormThreads)
znorm_warp_kernel(const float* in, float* out, int32_t B, int32_t N, bool vec4)
{
    const int q = blockIdx.x * (kNormThreads / 32) + (threadIdx.x >> 5);
    if (q >= B) return;
    const int64_t a = static_cast<int64_t>(q) * N;
    if (vec4)
        znorm_series_v4(reinterpret_cast<const float4*>(in + a), reinterpret_cast<float4*>(out + a), N / 4,
                        threadIdx.x & 31);
    else
        znorm_series(in + a, out + a, N, threadIdx.x & 31, 32, [](FF v) { return warp_sum(v); });
}

}  // namespace

namespace sdtw {

cudaError_t launch_znormalize(const float* in, float* out, const int64_t* offsets, int32_t B, int32_t N, int64_t limit,
                              int* status, cudaStream_t st)
{
    if (B <= 0) return cudaSuccess;
    // uniform series up to kWarpMaxN samples: a warp each; otherwise (long
    // series, or ragged batches whose lengths live on the device) a CTA each
    if (!offsets && N <= kWarpMaxN && (limit < 0 || static_cast<int64_t>(B) * N <= limit)) {
        const int per = kNormThreads / 32;
        const bool vec4 = N % 4 == 0 && reinterpret_cast<uintptr_t>(in) % 16 == 0 &&
                          reinterpret_cast<uintptr_t>(out) % 16 == 0;
        if (vec4 && N <= 32 * 4 * kRegVec4)
            znorm_warp_regs_kernel<<<(B + per - 1) / per, kNormThreads, 0, st>>>(in, out, B, N);
        else
            znorm_warp_kernel<<<(B + per - 1) / per, kNormThreads, 0, st>>>(in, out, B, N, vec4);
    } else {
        znorm_kernel<<<B, kNormThreads, 0, st>>>(in, out, offsets, N, limit, status);
    }
    return cudaGetLastError();
}

cudaError_t launch_znorm_vjp(const float* x, float* g, const int64_t* offsets, int32_t B, int32_t N, int64_t limit,
                             cudaStream_t st)
{
    if (B <= 0) return cudaSuccess;
    znorm_vjp_kernel<<<B, kNormThreads, 0, st>>>(x, g, offsets, N, limit);
    return cudaGetLastError();
}

sdtw_status znormalize_call(const float* in, float* out, const int64_t* offsets, int32_t B, int32_t N, cudaStream_t st)
{
    if (B < 0 || (!offsets && N < 1)) return SDTW_E_INVALID;
    if (B == 0) return SDTW_OK;
    if (!in || !out) return SDTW_E_INVALID;
    return launch_znormalize(in, out, offsets, B, N, -1, nullptr, st) == cudaSuccess ? SDTW_OK : SDTW_E_CUDA;
}

}  // namespace sdtw

extern "C" sdtw_status sdtw_znormalize(const float* in, float* out, const int64_t* offsets, int32_t B, int32_t N,
                                       void* stream)
{
    nvtxRangePushA("sdtw_znormalize");
    const sdtw_status st = sdtw::znormalize_call(in, out, offsets, B, N, static_cast<cudaStream_t>(stream));
    nvtxRangePop();
    return st;
}
