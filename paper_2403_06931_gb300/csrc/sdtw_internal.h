// Internal declarations shared by the library's CUDA translation units.
// Nothing here is part of the public ABI (include/sdtw.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "sdtw.h"

namespace sdtw {

// Steps between CTA barriers in the forward chain, and ring slots between two
// consecutive warps of the chain.  A value crosses from warp w-1 to warp w
// kChunk+1 steps after it was written, so a barrier always lies between the
// write and the read; the ring must hold more than 2*kChunk values.
#ifndef SDTW_CHUNK_STEPS
#define SDTW_CHUNK_STEPS 32
#endif
constexpr int kChunk = SDTW_CHUNK_STEPS;
constexpr int kRing = 4 * kChunk;
static_assert(kRing >= 2 * kChunk + 2, "ring too small for the chunk");
static_assert((kRing & (kRing - 1)) == 0, "ring size must be a power of two");

constexpr int kMaxWarpsPerQuery = 16;

// Integer modes: the longest query.  Costs are compared as float bit patterns
// (non-negative int32 patterns order like the floats they encode), so every
// reachable cost -- at most N * 255^2 along the vertical path -- must stay
// below 0x7f7fffff, the pattern that stands for +inf:
// 32,896 * 65,025 = 2,139,062,400 < 2,139,095,039.
constexpr int kIntMaxN = 32896;

// FP32 mode: a strip whose left input at the first row of a tile lies more
// than this far below the strip's integer base is rebased to that input before
// the tile (see sdtw_fill.cuh).  The backward replays the same decision.
constexpr float kRebaseBelow = 256.f;

// Dynamic shared memory one CTA may use on sm_103a.  Shared-memory sizes are
// computed in 64-bit arithmetic and checked against this before any launch,
// so a huge query length cannot wrap to a small size.
constexpr int64_t kMaxSmemBytes = 227 * 1024;

// Device status bits (OR-ed into the context's status word).
constexpr int kStatusBadLength = 1;  // a ragged query longer than N
constexpr int kStatusBadEnd = 2;     // an end index outside [0, M)
constexpr int kStatusTimeout = 4;    // a bounded wait ran out
constexpr int kStatusReplay = 8;     // the backward's recompute missed the forward's cost at the end cell

struct FwdArgs {
    const void* ref;
    int64_t M;
    const void* queries;
    const int64_t* offsets;  // nullptr: uniform [B][N]
    int32_t B;    // queries in this launch
    int32_t N;
    int32_t q0;   // first query of this launch (cost/end/order are indexed by q0 + local index)
    int32_t B_total;  // queries in the whole batch (offsets has B_total + 1 entries)
    void* cost;
    int64_t* end;
    // Checkpoints for the backward pass (fr == nullptr: none).  Query q of the
    // launch uses slot q - q0 of every array below.
    //   fr     the wavefront at the start of step c * ck_stride for every
    //          c >= 1, before a rebase due at that step: for thread tau, its
    //          strip's latest row (W values relative to its base) as float4
    //          [W/4][L], then its record float4 [E/4][L] = {right-hand cells of
    //          its tile's other RT-1 rows, diag, base}; checkpoint c at
    //          c * L * (W + E); fr_slot floats per query (E = fwd_record_floats(RT))
    //   colck  the left inputs of the strip whose first column is bK (b >= 1),
    //          in that strip's base: window b at (b - 1) * ck_rows(N), one per
    //          row (tiles past the query's end included);
    //          ck_slot floats per query
    //   ck_cost, ck_end  the query's cost and end column
    float* fr;
    int64_t fr_slot;
    float* colck;
    int64_t ck_slot;
    int32_t K;    // window width: column checkpoint stride (8 W)
    int32_t ck_stride;      // steps between wavefront checkpoints: 8, 16, 32 or 64
    int32_t rebase_period;  // steps between FP32 rebases: ckpt_rebase_period(stride) of the context's checkpointing plan, else kChunk
    float* ck_cost;
    int64_t* ck_end;
    int* status;
    int64_t q_limit;     // > 0: queries end within this many samples (a ragged query past it is flagged)
    int32_t prune_gap;   // integer modes: > 0 prunes cells whose samples differ by more (Section 8); 0: off
    int* queue;          // persistent mode: device work counter (reset to 0 before the launch)
    const int32_t* order;// persistent mode: query order (longest first), or nullptr
};

struct FwdPlan {
    int W = 16;          // segment width: reference columns per thread
    int P = 8;           // warps per query chain
    int RT = 2;          // query rows per thread per step (tile height: 2, 4, or 8 for the plain FP32 fill)
    int KS = kChunk;     // with checkpoints: steps between wavefront checkpoints (8, 16, 32 or 64)
    bool persistent = false;
    int grid = 0;
    int block = 0;
    int64_t smem = 0;    // dynamic shared memory per CTA (launchable only if <= kMaxSmemBytes)
};

// Forward launch (sdtw_forward.cu).
bool fwd_width_supported(sdtw_dtype dt, int W);
// a (W, RT) the fill has an instantiation for: RT 2 or 4 for every mode, RT 8
// at W 16..28 for the plain fills and the FP32 fill with checkpoints
bool fwd_plan_supported(sdtw_dtype dt, int W, int RT, bool ckpt);
int64_t fwd_smem_bytes(sdtw_dtype dt, int64_t N, int P, int W, int RT);
// 0 when smem exceeds kMaxSmemBytes or the plan cannot be resident
int fwd_max_ctas_per_sm(sdtw_dtype dt, int W, int P, int64_t smem, int RT, bool ckpt, bool prune = false);
int64_t fwd_total_steps(int64_t M, int N, int W, int P, int RT);
cudaError_t launch_forward(sdtw_dtype dt, const FwdPlan& plan, const FwdArgs& a, cudaStream_t s);
cudaError_t launch_order_by_length(const int64_t* offsets, int32_t B, int32_t* order, cudaStream_t s);
// the integer modes (sdtw_forward_int.cu), with or without pruning
int fwd_max_ctas_per_sm_int(sdtw_dtype dt, int W, int P, int64_t smem, int RT, bool prune);
cudaError_t launch_forward_int(sdtw_dtype dt, const FwdPlan& plan, const FwdArgs& a, cudaStream_t s);

struct BwdArgs {
    const float* ref;
    int64_t M;
    const float* queries;
    const int64_t* offsets;
    int32_t B;   // queries in this launch
    int32_t N;
    int32_t q0;  // first query of this launch (chunked backward)
    int32_t B_total;  // queries in the whole batch (offsets has B_total + 1 entries)
    const int64_t* end;
    const float* grad_cost;
    float* grad_queries;
    int32_t* path;
    // checkpoints of queries q0 .. q0+B-1 (layout as FwdArgs) and the plan of
    // the forward that wrote them
    const float* fr;
    int64_t fr_slot;
    const float* colck;
    int64_t ck_slot;
    int32_t K;
    const float* ck_cost;
    const int64_t* ck_end;
    int32_t W, P, RT;
    int32_t KS;             // steps between the forward's wavefront checkpoints: a band's height in steps
    int32_t rebase_period;  // the forward's steps between rebases
    int32_t warps;          // warps per query: 1 = the walker alone, 2..4 with helpers, 0 = the library's choice
    int32_t idle_helpers;   // tests only: the helpers take no work (the walker's wait runs out)
    float* gyq;      // [B][M] per-query reference gradient rows (only the path span is written)
    int64_t* span;   // [B][2] first and last column of each query's path
    int* status;
    int64_t q_limit; // > 0: queries end within this many samples (a ragged query past it is flagged)
};

// Checkpoint geometry of a forward plan (sdtw_forward.cu, sdtw_fill.cuh): floats of one
// thread's record, wavefront checkpoints (one every KS steps) of the schedule
// for a query of n rows, and the per-query slot sizes of the two checkpoint
// arrays.  Checkpoint strides are 8, 16, 32 or 64 steps; the checkpointing fill
// rebases every max(kChunk, KS) steps, so that no band of KS steps spans a
// rebase.
__host__ __device__ constexpr int fwd_record_floats(int RT) { return RT == 2 ? 4 : RT == 4 ? 8 : 12; }
__host__ __device__ constexpr int ck_rows(int N) { return (N + 7) / 8 * 8; }
constexpr bool ckpt_stride_supported(int KS) { return KS == 8 || KS == 16 || KS == 32 || KS == 64; }
constexpr int ckpt_rebase_period(int KS) { return KS > kChunk ? KS : kChunk; }
int64_t fwd_ckpts(int64_t M, int n, int W, int P, int RT, int KS);
int64_t fr_slot_floats(int64_t M, int N, int W, int P, int RT, int KS);
int64_t ck_slot_floats(int64_t M, int N, int K);

// Backward launches (sdtw_backward.cu).
bool bwd_width_supported(int W);
// Shared memory of a backward CTA with `warps` warps (one band slot each), and
// the warps a launch uses: `requested` (1 = the walker alone, up to 4), or the
// library's choice for 0, reduced until the CTA fits; 0 if none fits or the
// request is out of range.
int64_t bwd_smem_bytes(int64_t N, int W, int RT, int KS, int warps = 1);
int bwd_warps(int64_t N, int W, int RT, int KS, int requested);
int bwd_dir_rows(int RT, int KS);
cudaError_t launch_backward_walk(const BwdArgs& a, cudaStream_t s);
cudaError_t launch_grad_ref_reduce(const float* gyq, const int64_t* span, int32_t B, int64_t M,
                                   bool accumulate, float* grad_ref, cudaStream_t s);

// Batch z-normalisation (sdtw_norm.cu): Eq. 2 on B series ([B][N] or by
// offsets) from `in` to `out`; a ragged series reaching past `limit` elements
// (limit < 0: no bound) is skipped and reported in *status.  The derivative:
// g (dcost/dz, same layout) becomes dcost/dx in place.
cudaError_t launch_znormalize(const float* in, float* out, const int64_t* offsets, int32_t B, int32_t N, int64_t limit,
                              int* status, cudaStream_t st);
cudaError_t launch_znorm_vjp(const float* x, float* g, const int64_t* offsets, int32_t B, int32_t N, int64_t limit,
                             cudaStream_t st);

}  // namespace sdtw
