// Reference codebook: uint8 codes for the integer DP (the paper's Section 8
// proposes quantising below fp16 to uint8 with a codebook built from the
// reference: the bulk of the reference's value distribution divided evenly
// over the 256 codes, outliers clamped to the extreme codes).
//
// The bulk is mean +- sigmas * S of the reference (population spread S), so
// code k covers [lo + k step, lo + (k + 1) step) with step = 2 sigmas S / 256.
// The fit runs in double on one CTA (set-up work, once per reference); the
// encoding decides every code in float32 -- (x - lo) rounded, times 1/step
// rounded, floored and clamped -- so that a checker working in float32 takes
// the same decisions.  The DP then runs on the codes (SDTW_U8): exact int32
// sums of squared code differences, a cost in units of step^2.
#include <cuda_runtime.h>

#include <cstdint>

#include "sdtw.h"
#include "sdtw_internal.h"

namespace {

constexpr int kFitThreads = 1024;

__device__ double block_sum(double v, double* red)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) red[w] = v;
    __syncthreads();
    v = l < (blockDim.x >> 5) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;  // in every thread of warp 0 (and, after the shuffles, every warp)
}

__global__ void __launch_bounds__(kFitThreads) codebook_fit_kernel(const float* __restrict__ ref, int64_t M,
                                                                   float sigmas, float* __restrict__ params)
{
    __shared__ double red[32];
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < M; i += blockDim.x) s += ref[i];
    const double mean = block_sum(s, red) / static_cast<double>(M);
    double v = 0.0;
    for (int64_t i = threadIdx.x; i < M; i += blockDim.x) {
        const double d = static_cast<double>(ref[i]) - mean;
        v += d * d;
    }
    const double sd = sqrt(block_sum(v, red) / static_cast<double>(M));
    if (threadIdx.x == 0) {
        double lo = mean - 128.0, step = 1.0;  // zero spread: the constant lands mid-range
        if (sd > 0.0) {
            lo = mean - static_cast<double>(sigmas) * sd;
            step = 2.0 * static_cast<double>(sigmas) * sd / 256.0;
        }
        params[0] = static_cast<float>(lo);
        params[1] = static_cast<float>(1.0 / step);
        params[2] = static_cast<float>(step);
        params[3] = 0.f;
    }
}

__device__ __forceinline__ uint8_t encode_one(float x, float lo, float inv)
{
    // the explicit roundings keep the compiler from fusing the two operations
    float t = floorf(__fmul_rn(__fsub_rn(x, lo), inv));
    t = fminf(fmaxf(t, 0.f), 255.f);
    return static_cast<uint8_t>(t);
}

__global__ void codebook_encode_kernel(const float* __restrict__ in, int64_t n, const float* __restrict__ params,
                                       uint8_t* __restrict__ out, bool vec)
{
    const float lo = params[0], inv = params[1];
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    const int64_t t0 = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (vec) {
        // 16-byte loads, 4-byte stores (both buffers aligned, n a multiple of 4)
        const float4* in4 = reinterpret_cast<const float4*>(in);
        uchar4* out4 = reinterpret_cast<uchar4*>(out);
        for (int64_t i = t0; i < n / 4; i += stride) {
            const float4 v = in4[i];
            out4[i] = make_uchar4(encode_one(v.x, lo, inv), encode_one(v.y, lo, inv), encode_one(v.z, lo, inv),
                                  encode_one(v.w, lo, inv));
        }
    } else {
        for (int64_t i = t0; i < n; i += stride) out[i] = encode_one(in[i], lo, inv);
    }
}

}  // namespace

extern "C" {

sdtw_status sdtw_codebook_fit(const float* ref, int64_t M, float sigmas, float* params, void* stream)
{
    if (!ref || !params || M < 1 || !(sigmas > 0.f) || !(sigmas < 1e30f)) return SDTW_E_INVALID;
    codebook_fit_kernel<<<1, kFitThreads, 0, static_cast<cudaStream_t>(stream)>>>(ref, M, sigmas, params);
    return cudaGetLastError() == cudaSuccess ? SDTW_OK : SDTW_E_CUDA;
}

sdtw_status sdtw_codebook_encode(const float* in, int64_t n, const float* params, uint8_t* out, void* stream)
{
    if (n < 0 || (n > 0 && (!in || !params || !out))) return SDTW_E_INVALID;
    if (n == 0) return SDTW_OK;
    const bool vec = n % 4 == 0 && reinterpret_cast<uintptr_t>(in) % 16 == 0 && reinterpret_cast<uintptr_t>(out) % 4 == 0;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SDTW_E_CUDA;
    const int threads = 256;
    const int64_t work = vec ? n / 4 : n;
    const int64_t want = (work + threads - 1) / threads;
    const int blocks = static_cast<int>(want < static_cast<int64_t>(sms) * 8 ? want : static_cast<int64_t>(sms) * 8);
    codebook_encode_kernel<<<blocks, threads, 0, static_cast<cudaStream_t>(stream)>>>(in, n, params, out, vec);
    return cudaGetLastError() == cudaSuccess ? SDTW_OK : SDTW_E_CUDA;
}

}  // extern "C"
