// Batch z-normalisation (paper Section 5.1, Eq. 2): every series of a batch
// becomes (x - mean) / S with its own mean and population standard deviation
// S; a series with S == 0 is only centred.
//
// The paper's normaliser runs one block per query, each thread summing a few
// elements and a shared-memory tree reducing the partial sums and sums of
// squares, then applies Eq. 2 from the variance sumSq/n - mean^2.  Here one
// CTA per series makes two reduction passes in double (the mean, then the
// centred second moment): the one-pass difference cancels digits when the mean
// is large against the spread.  The series is read three times (the second
// and third reads hit L2 for query-sized series), so HBM sees one read and one
// write per sample.  Warp partial sums are combined with shuffles and one
// shared-memory slot per warp.
#include <cuda_runtime.h>

#include <cstdint>

#include "sdtw.h"

namespace {

constexpr int kNormThreads = 256;

// sum of v over the CTA, returned to every thread
__device__ __forceinline__ double block_sum(double v, double* red)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    __syncthreads();  // red[] may still be read by the previous reduction
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
    __syncthreads();
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < kNormThreads / 32; ++w) t += red[w];
    return t;
}

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
    const float* x = in + a;
    float* z = out + a;

    double s = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kNormThreads) s += x[i];
    const double mean = block_sum(s, red) / static_cast<double>(n);
    double ss = 0.0;
    for (int64_t i = threadIdx.x; i < n; i += kNormThreads) {
        const double c = static_cast<double>(x[i]) - mean;
        ss += c * c;
    }
    double sd = sqrt(block_sum(ss, red) / static_cast<double>(n));
    if (!(sd > 0.0)) sd = 1.0;
    const double inv = 1.0 / sd;
    // each thread rewrites only elements it read itself: safe in place
    for (int64_t i = threadIdx.x; i < n; i += kNormThreads)
        z[i] = static_cast<float>((static_cast<double>(x[i]) - mean) * inv);
}

// The same for series of up to kWarpMaxN samples, one warp per series (eight
// series per CTA): the reductions are warp shuffles, with no CTA barrier.
constexpr int kWarpMaxN = 16384;

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

__global__ void __launch_bounds__(kNormThreads)
znorm_warp_kernel(const float* in, float* out, const int64_t* offsets, int32_t B, int32_t N)
{
    const int q = blockIdx.x * (kNormThreads / 32) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (q >= B) return;
    int64_t a, n;
    if (offsets) {
        a = offsets[q];
        n = offsets[q + 1] - a;
        if (a < 0 || n <= 0) return;
    } else {
        a = static_cast<int64_t>(q) * N;
        n = N;
    }
    const float* x = in + a;
    float* z = out + a;
    double s = 0.0;
    for (int64_t i = lane; i < n; i += 32) s += x[i];
    const double mean = warp_sum(s) / static_cast<double>(n);
    double ss = 0.0;
    for (int64_t i = lane; i < n; i += 32) {
        const double c = static_cast<double>(x[i]) - mean;
        ss += c * c;
    }
    double sd = sqrt(warp_sum(ss) / static_cast<double>(n));
    if (!(sd > 0.0)) sd = 1.0;
    const double inv = 1.0 / sd;
    for (int64_t i = lane; i < n; i += 32) z[i] = static_cast<float>((static_cast<double>(x[i]) - mean) * inv);
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
        znorm_warp_kernel<<<(B + per - 1) / per, kNormThreads, 0, st>>>(in, out, offsets, B, N);
    } else {
        znorm_kernel<<<B, kNormThreads, 0, st>>>(in, out, offsets, N);
    }
    return cudaGetLastError() == cudaSuccess ? SDTW_OK : SDTW_E_CUDA;
}
