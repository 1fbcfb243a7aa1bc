// sdtw_forward_noalloc: the forward pass for callers that cannot allocate.
//
// Some callers cannot call cudaMalloc at all: code running inside a CUDA
// graph capture that may not allocate, plug-ins loaded into a host process
// that owns every device allocation through its own pool or budget, and
// real-time loops that must not touch the allocator after start-up.  For
// them this entry point runs the same persistent forward kernel as
// sdtw_forward with no context: the only scratch the kernel needs -- the work
// counter that hands out queries, the device status word and the
// longest-first query order -- lives in one file-scope __device__ array of
// fixed size, which every GPU that loads the library holds until the process
// exits.  The caller still passes inputs and outputs.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <mutex>

#include "sdtw.h"
#include "sdtw_internal.h"

namespace {

constexpr int kNoAllocMaxDevices = 64;
constexpr int kCounter = 0;  // scratch layout: [0] work counter, [1] status word,
constexpr int kStatus = 1;   // [2 .. 2 + SDTW_NOALLOC_MAX_BATCH) query order
constexpr int kOrder = 2;

static __device__ __align__(256) int32_t g_noalloc_scratch[kOrder + SDTW_NOALLOC_MAX_BATCH];

// Device address of g_noalloc_scratch, looked up once per device.  In host
// code the symbol names a host-side stand-in, not device memory, so it must
// never be passed to a kernel directly.
std::mutex g_setup_mutex;
int32_t* g_scratch_addr[kNoAllocMaxDevices] = {};

cudaError_t scratch_for_current_device(int32_t** out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kNoAllocMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_scratch_addr[dev] = static_cast<int32_t*>(p);
    }
    *out = g_scratch_addr[dev];
    return cudaSuccess;
}

}  // namespace

extern "C" sdtw_status sdtw_forward_noalloc(sdtw_dtype dtype, const void* ref, int64_t M, const void* queries,
                                            const int64_t* offsets, int32_t B, int32_t N, void* cost,
                                            int64_t* end, void* stream)
{
    if (dtype != SDTW_F32 && dtype != SDTW_I8 && dtype != SDTW_U8 && dtype != SDTW_F16) return SDTW_E_INVALID;
    if (dtype == SDTW_F16 && offsets) return SDTW_E_UNSUPPORTED;  // binary16 pairs: uniform batches only
    if (B < 0 || M < 1 || N < 1 || M > INT_MAX / 2) return SDTW_E_INVALID;
    if (B > SDTW_NOALLOC_MAX_BATCH) return SDTW_E_INVALID;  // the order array holds at most this many queries
    if ((dtype == SDTW_I8 || dtype == SDTW_U8) && N > sdtw::kIntMaxN) return SDTW_E_INVALID;  // costs below the +inf pattern
    if (B == 0) return SDTW_OK;
    if (!ref || !queries || !cost || !end) return SDTW_E_INVALID;

    sdtw::FwdPlan plan;
    plan.W = 32;
    plan.P = 4;
    plan.RT = 4;
    while (plan.P > 1 && static_cast<int64_t>(32) * (plan.P / 2) * plan.W >= M) plan.P /= 2;
    plan.block = 32 * plan.P;
    plan.smem = sdtw::fwd_smem_bytes(dtype, N, plan.P, plan.W, plan.RT);
    plan.persistent = true;
    if (plan.smem > sdtw::kMaxSmemBytes) return SDTW_E_UNSUPPORTED;  // 64-bit size: no wrap for any N
    if (sdtw::fwd_total_steps(M, N, plan.W, plan.P, plan.RT) > INT_MAX - 4 * sdtw::kChunk) return SDTW_E_UNSUPPORTED;

    int32_t* scratch = nullptr;
    if (scratch_for_current_device(&scratch) != cudaSuccess) return SDTW_E_CUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return SDTW_E_CUDA;
    const int per_sm = sdtw::fwd_max_ctas_per_sm(dtype, plan.W, plan.P, plan.smem, plan.RT, false);
    if (per_sm <= 0) return SDTW_E_UNSUPPORTED;
    plan.grid = std::max(1, std::min(B, per_sm * sms));

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // the counter and the status word keep the previous call's values: clear them
    if (cudaMemsetAsync(scratch + kCounter, 0, 2 * sizeof(int32_t), st) != cudaSuccess) return SDTW_E_CUDA;
    sdtw::FwdArgs a{};
    a.ref = ref;
    a.M = M;
    a.queries = queries;
    a.offsets = offsets;
    a.B = B;
    a.N = N;
    a.q0 = 0;
    a.B_total = B;
    a.cost = cost;
    a.end = end;
    a.fr = nullptr;  // no checkpoints
    a.K = 1;
    a.ck_stride = sdtw::kChunk;
    a.rebase_period = sdtw::kChunk;
    a.status = scratch + kStatus;
    a.queue = scratch + kCounter;
    a.order = nullptr;
    if (offsets) {
        if (sdtw::launch_order_by_length(offsets, B, scratch + kOrder, st) != cudaSuccess) return SDTW_E_CUDA;
        a.order = scratch + kOrder;
    }
    if (sdtw::launch_forward(dtype, plan, a, st) != cudaSuccess) return SDTW_E_CUDA;
    return SDTW_OK;
}
