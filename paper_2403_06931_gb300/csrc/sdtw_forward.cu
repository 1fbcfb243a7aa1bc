// Forward fill launches: the FP32 and binary16 instantiations of the fill
// kernel (sdtw_fill.cuh), the ordering kernel of the ragged persistent form,
// and the public launch and sizing functions; the integer modes are
// instantiated in sdtw_forward_int.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "sdtw_fill.cuh"
#include "sdtw_internal.h"

namespace sdtw {
namespace {

// rank of each query by length, longest first (ties by index): order[rank] = q.
// Every thread counts the queries ranked before its own; the lengths are
// staged in shared memory a tile at a time, so each is read from global memory
// once per CTA rather than once per thread (B^2 comparisons, on-chip).
constexpr int kOrderThreads = 256;
constexpr int kOrderTile = 2048;

__global__ void __launch_bounds__(kOrderThreads) order_by_length_kernel(const int64_t* __restrict__ offsets, int32_t B,
                                                                        int32_t* __restrict__ order)
{
    __shared__ int64_t lens[kOrderTile];
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t lq = q < B ? offsets[q + 1] - offsets[q] : 0;
    int rank = 0;
    for (int p0 = 0; p0 < B; p0 += kOrderTile) {
        const int np = min(kOrderTile, B - p0);
        __syncthreads();
        for (int k = threadIdx.x; k < np; k += blockDim.x) lens[k] = offsets[p0 + k + 1] - offsets[p0 + k];
        __syncthreads();
        if (q < B) {
            for (int k = 0; k < np; ++k) {
                const int64_t lp = lens[k];
                rank += (lp > lq) || (lp == lq && p0 + k < q);
            }
        }
    }
    if (q < B) order[rank] = q;
}

// dispatch (dtype, W, RT, checkpoints) to an FP32 or binary16 instantiation;
// checkpoints exist only in FP32 mode (the backward is FP32 only)
template <typename F>
cudaError_t dispatch(sdtw_dtype dt, int W, int RT, bool ckpt, F&& f)
{
#define SDTW_W(Tin, RTv, CK)                                              \
    switch (W) {                                                          \
    case 8: return f(Inst<Tin, 8, RTv, CK>{});                            \
    case 16: return f(Inst<Tin, 16, RTv, CK>{});                          \
    case 20: return f(Inst<Tin, 20, RTv, CK>{});                          \
    case 24: return f(Inst<Tin, 24, RTv, CK>{});                          \
    case 28: return f(Inst<Tin, 28, RTv, CK>{});                          \
    case 32: return f(Inst<Tin, 32, RTv, CK>{});                          \
    default: return cudaErrorInvalidValue;                                \
    }
#define SDTW_W8(Tin, CK)                                                  \
    switch (W) {                                                          \
    case 16: return f(Inst<Tin, 16, 8, CK>{});                            \
    case 20: return f(Inst<Tin, 20, 8, CK>{});                            \
    case 24: return f(Inst<Tin, 24, 8, CK>{});                            \
    case 28: return f(Inst<Tin, 28, 8, CK>{});                            \
    default: return cudaErrorInvalidValue;                                \
    }
    if (RT == 8) {
        // 8-row tiles (the per-step work of shuffles, conversions and loop
        // control spread over 8 rows), W 16 to 28; with checkpoints FP32 only
        if (dt == SDTW_F32 && ckpt) { SDTW_W8(float, true) }
        if (ckpt) return cudaErrorInvalidValue;
        if (dt == SDTW_F16) { SDTW_W8(__half, false) }
        if (dt == SDTW_F32) { SDTW_W8(float, false) }
        return cudaErrorInvalidValue;
    }
    if (RT != 2 && RT != 4) return cudaErrorInvalidValue;
    if (dt == SDTW_F16) {
        if (ckpt) return cudaErrorInvalidValue;
        if (RT == 2) { SDTW_W(__half, 2, false) } else { SDTW_W(__half, 4, false) }
    }
    if (dt != SDTW_F32) return cudaErrorInvalidValue;
    if (ckpt) {
        if (RT == 2) { SDTW_W(float, 2, true) } else { SDTW_W(float, 4, true) }
    }
    if (RT == 2) { SDTW_W(float, 2, false) } else { SDTW_W(float, 4, false) }
#undef SDTW_W8
#undef SDTW_W
}

}  // namespace

bool fwd_width_supported(sdtw_dtype, int W) { return W == 8 || W == 16 || W == 20 || W == 24 || W == 28 || W == 32; }

bool fwd_plan_supported(sdtw_dtype dt, int W, int RT, bool ckpt)
{
    if (!fwd_width_supported(dt, W)) return false;
    if (RT == 2 || RT == 4) return true;
    return RT == 8 && W >= 16 && W <= 28 && (!ckpt || dt == SDTW_F32);
}

int64_t fwd_smem_bytes(sdtw_dtype dt, int64_t N, int P, int W, int RT)
{
    // ring [P][kRing] and column buffer [Npad/RT] of edges (16 bytes for RT = 2,
    // 32 for RT = 4, 48 for RT = 8), query samples [Npad] and the reduction (value, index)[P],
    // 4-byte elements; 64-bit, so that no query length wraps to a small size
    (void)W;
    if (N < 0) N = 0;
    const int64_t npad = (N + RT - 1) / RT * RT;
    const int64_t esz = RT == 2 ? 16 : RT == 4 ? 32 : 48;
    const int64_t red = dt == SDTW_F16 ? 4 : 2;  // binary16 pairs reduce two (value, column) pairs per warp
    return esz * (static_cast<int64_t>(P) * kRing + npad / RT) + 4 * (npad + red * static_cast<int64_t>(P));
}

int64_t fwd_total_steps(int64_t M, int N, int W, int P, int RT)
{
    const int64_t S = static_cast<int64_t>(32) * P * W;
    const int64_t nsw = (M + S - 1) / S;
    const int64_t lag_last = static_cast<int64_t>(P - 1) * (32 + kChunk) + 31;
    const int64_t nt = (N + RT - 1) / RT;
    const int64_t Pp = std::max<int64_t>(nt, lag_last + kChunk);
    return (nsw - 1) * Pp + nt + lag_last;
}

int64_t fwd_ckpts(int64_t M, int n, int W, int P, int RT, int KS)
{
    return (fwd_total_steps(M, n, W, P, RT) + KS - 1) / KS;
}

int64_t fr_slot_floats(int64_t M, int N, int W, int P, int RT, int KS)
{
    // the checkpoint count grows with the query length, so N bounds every
    // query of a ragged batch
    return fwd_ckpts(M, N, W, P, RT, KS) * 32 * P * (W + fwd_record_floats(RT));
}

int64_t ck_slot_floats(int64_t M, int N, int K)
{
    const int64_t windows = (M + K - 1) / K;
    return (windows - 1) * static_cast<int64_t>(ck_rows(N));
}

int fwd_max_ctas_per_sm(sdtw_dtype dt, int W, int P, int64_t smem, int RT, bool ckpt, bool prune)
{
    if (dt == SDTW_I8 || dt == SDTW_U8) return fwd_max_ctas_per_sm_int(dt, W, P, smem, RT, prune);
    int n = 0;
    dispatch(dt, W, RT, ckpt, [&](auto inst) {
        n = decltype(inst)::occupancy(32 * P, smem);
        return cudaSuccess;
    });
    return n;
}

cudaError_t launch_forward(sdtw_dtype dt, const FwdPlan& plan, const FwdArgs& a, cudaStream_t s)
{
    if (plan.grid <= 0) return cudaSuccess;
    if (dt == SDTW_I8 || dt == SDTW_U8) return launch_forward_int(dt, plan, a, s);
    return dispatch(dt, plan.W, plan.RT, a.fr != nullptr,
                    [&](auto inst) { return decltype(inst)::launch(plan, a, s); });
}

cudaError_t launch_order_by_length(const int64_t* offsets, int32_t B, int32_t* order, cudaStream_t s)
{
    if (B <= 0) return cudaSuccess;
    order_by_length_kernel<<<(B + kOrderThreads - 1) / kOrderThreads, kOrderThreads, 0, s>>>(offsets, B, order);
    return cudaGetLastError();
}

}  // namespace sdtw
