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
// throughput is a small fraction of FP32 on this part, so the per-sample work
// stays in FP32 without losing accuracy:
//   * each lane sums x - x[0] (shifting by the series' first sample removes a
//     large common offset) with Kahan compensation, and only the lanes'
//     (sum, compensation) pairs are combined in double;
//   * the mean is carried as a pair of floats (hi + lo), and every sample is
//     centred as (x - hi) - lo, so the centred values are accurate to about
//     one float rounding; their squares are again Kahan-summed per lane.
// The series is read three times (the second and third reads hit L2 for
// query-sized series), so HBM sees one read and one write per sample.
#include <cuda_runtime.h>

#include <cstdint>

#include "sdtw.h"

namespace {

constexpr int kNormThreads = 256;
constexpr int kWarpMaxN = 16384;  // uniform series up to this length take one warp each

// Kahan-compensated running sum
struct KSum {
    float s = 0.f, c = 0.f;
    __device__ __forceinline__ void add(float v)
    {
        const float y = v - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return static_cast<double>(s) - static_cast<double>(c); }
};

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

// sum over the CTA of one double per thread, returned to every thread
__device__ __forceinline__ double block_sum(double v, double* red)
{
    v = warp_sum(v);
    __syncthreads();  // red[] may still be read by the previous reduction
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kNormThreads / 32; ++w) t += red[w];
    return t;
}

// Eq. 2 on one series of n samples at x (written to z), by `count` threads
// with index `idx`; REDUCE sums a double over those threads.
template <typename Reduce>
__device__ __forceinline__ void znorm_series(const float* x, float* z, int64_t n, int idx, int count, Reduce reduce)
{
    const float x0 = x[0];
    KSum s1;
    for (int64_t i = idx; i < n; i += count) s1.add(x[i] - x0);
    const double mean = static_cast<double>(x0) + reduce(s1.value()) / static_cast<double>(n);
    const float hi = static_cast<float>(mean);
    const float lo = static_cast<float>(mean - static_cast<double>(hi));
    KSum s2;
    for (int64_t i = idx; i < n; i += count) {
        const float c = (x[i] - hi) - lo;
        s2.add(c * c);
    }
    double sd = sqrt(reduce(s2.value()) / static_cast<double>(n));
    if (!(sd > 0.0)) sd = 1.0;
    const float inv = static_cast<float>(1.0 / sd);
    // each thread rewrites only elements it read itself: safe in place
    for (int64_t i = idx; i < n; i += count) z[i] = ((x[i] - hi) - lo) * inv;
}

// one CTA per series: long series, and ragged batches (lengths on the device)
__global__ void __launch_bounds__(kNormThreads)
znorm_kernel(const float* in, float* out, const int64_t* offsets, int32_t N)
{
    __shared__ double red[kNormThreads / 32];
    const int q = blockIdx.x;
    int64_t a, n;
    if (offsets) {
        a = offsets[q];
        n = offsets[q + 1] - a;
        if (a < 0 || n <= 0) return;  // empty (or malformed) series: nothing to write
    } else {
        a = static_cast<int64_t>(q) * N;
        n = N;
    }
    znorm_series(in + a, out + a, n, threadIdx.x, kNormThreads, [&](double v) { return block_sum(v, red); });
}

// The same with 16-byte loads and stores: series of a multiple of 4 samples
// starting on a 16-byte boundary.
__device__ __forceinline__ void znorm_series_v4(const float4* x, float4* z, int n4, int lane)
{
    const float x0 = reinterpret_cast<const float*>(x)[0];
    KSum s1;
    for (int i = lane; i < n4; i += 32) {
        const float4 v = x[i];
        s1.add(v.x - x0);
        s1.add(v.y - x0);
        s1.add(v.z - x0);
        s1.add(v.w - x0);
    }
    const double n = 4.0 * n4;
    const double mean = static_cast<double>(x0) + warp_sum(s1.value()) / n;
    const float hi = static_cast<float>(mean);
    const float lo = static_cast<float>(mean - static_cast<double>(hi));
    KSum s2;
    for (int i = lane; i < n4; i += 32) {
        const float4 v = x[i];
        const float c0 = (v.x - hi) - lo, c1 = (v.y - hi) - lo, c2 = (v.z - hi) - lo, c3 = (v.w - hi) - lo;
        s2.add(c0 * c0);
        s2.add(c1 * c1);
        s2.add(c2 * c2);
        s2.add(c3 * c3);
    }
    double sd = sqrt(warp_sum(s2.value()) / n);
    if (!(sd > 0.0)) sd = 1.0;
    const float inv = static_cast<float>(1.0 / sd);
    for (int i = lane; i < n4; i += 32) {
        const float4 v = x[i];
        z[i] = make_float4(((v.x - hi) - lo) * inv, ((v.y - hi) - lo) * inv, ((v.z - hi) - lo) * inv,
                           ((v.w - hi) - lo) * inv);
    }
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
        znorm_series(in + a, out + a, N, threadIdx.x & 31, 32, [](double v) { return warp_sum(v); });
}

}  // namespace

extern "C" sdtw_status sdtw_znormalize(const float* in, float* out, const int64_t* offsets, int32_t B, int32_t N,
                                       void* stream)
{
    if (B < 0 || (!offsets && N < 1)) return SDTW_E_INVALID;
    if (B == 0) return SDTW_OK;
    if (!in || !out) return SDTW_E_INVALID;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // uniform series up to kWarpMaxN samples: a warp each; otherwise (long
    // series, or ragged batches whose lengths live on the device) a CTA each
    if (!offsets && N <= kWarpMaxN) {
        const int per = kNormThreads / 32;
        const bool vec4 = N % 4 == 0 && reinterpret_cast<uintptr_t>(in) % 16 == 0 &&
                          reinterpret_cast<uintptr_t>(out) % 16 == 0;
        znorm_warp_kernel<<<(B + per - 1) / per, kNormThreads, 0, st>>>(in, out, B, N, vec4);
    } else {
        znorm_kernel<<<B, kNormThreads, 0, st>>>(in, out, offsets, N);
    }
    return cudaGetLastError() == cudaSuccess ? SDTW_OK : SDTW_E_CUDA;
}
