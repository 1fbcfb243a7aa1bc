// The integer modes of the forward fill (sdtw_fill.cuh): int8 samples and
// uint8 codebook codes, each with and without the early-INF pruning of the
// paper's Section 8 (a cell whose samples differ by more than the pruning gap
// costs +inf).  Kept in a translation unit of its own so that the library's
// sources compile in parallel.
#include <cuda_runtime.h>

#include "sdtw_fill.cuh"
#include "sdtw_internal.h"

namespace sdtw {
namespace {

template <typename F>
cudaError_t dispatch_int(sdtw_dtype dt, int W, int RT, bool prune, F&& f)
{
#define SDTW_W(Tin, RTv, PR)                                              \
    switch (W) {                                                          \
    case 8: return f(Inst<Tin, 8, RTv, false, PR>{});                     \
    case 16: return f(Inst<Tin, 16, RTv, false, PR>{});                   \
    case 20: return f(Inst<Tin, 20, RTv, false, PR>{});                   \
    case 24: return f(Inst<Tin, 24, RTv, false, PR>{});                   \
    case 28: return f(Inst<Tin, 28, RTv, false, PR>{});                   \
    case 32: return f(Inst<Tin, 32, RTv, false, PR>{});                   \
    default: return cudaErrorInvalidValue;                                \
    }
#define SDTW_W8(Tin, PR)                                                  \
    switch (W) {                                                          \
    case 16: return f(Inst<Tin, 16, 8, false, PR>{});                     \
    case 20: return f(Inst<Tin, 20, 8, false, PR>{});                     \
    case 24: return f(Inst<Tin, 24, 8, false, PR>{});                     \
    case 28: return f(Inst<Tin, 28, 8, false, PR>{});                     \
    default: return cudaErrorInvalidValue;                                \
    }
#define SDTW_RT(Tin, PR)                                                  \
    if (RT == 2) { SDTW_W(Tin, 2, PR) } else if (RT == 4) { SDTW_W(Tin, 4, PR) } else { SDTW_W8(Tin, PR) }
    if (RT != 2 && RT != 4 && RT != 8) return cudaErrorInvalidValue;
    if (dt == SDTW_I8) {
        if (prune) { SDTW_RT(int8_t, true) } else { SDTW_RT(int8_t, false) }
    }
    if (dt == SDTW_U8) {
        if (prune) { SDTW_RT(uint8_t, true) } else { SDTW_RT(uint8_t, false) }
    }
    return cudaErrorInvalidValue;
#undef SDTW_RT
#undef SDTW_W8
#undef SDTW_W
}

}  // namespace

int fwd_max_ctas_per_sm_int(sdtw_dtype dt, int W, int P, int64_t smem, int RT, bool prune)
{
    int n = 0;
    dispatch_int(dt, W, RT, prune, [&](auto inst) {
        n = decltype(inst)::occupancy(32 * P, smem);
        return cudaSuccess;
    });
    return n;
}

cudaError_t launch_forward_int(sdtw_dtype dt, const FwdPlan& plan, const FwdArgs& a, cudaStream_t s)
{
    if (plan.grid <= 0) return cudaSuccess;
    if (a.fr != nullptr) return cudaErrorInvalidValue;  // checkpoints are FP32 only
    return dispatch_int(dt, plan.W, plan.RT, a.prune_gap > 0,
                        [&](auto inst) { return decltype(inst)::launch(plan, a, s); });
}

}  // namespace sdtw
