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

// Device status bits (OR-ed into the context's status word).
constexpr int kStatusBadLength = 1;  // a ragged query longer than N
constexpr int kStatusBadEnd = 2;     // an end index outside [0, M)
constexpr int kStatusTimeout = 4;    // a bounded wait ran out

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
    // Checkpoints for the backward pass (nullptr: none), absolute D values:
    //   ckpt   every K-th column: query q at (start_q - start_q0) * nblk, block b
    //          (column (b+1)K-1) at b * n_q, one value per row;
    //   rowck  every R-th row: query q at floor((start_q - start_q0) / R) * M,
    //          stored row m (row (m+1)R-1) at m * M, one value per column.
    float* ckpt;
    float* rowck;
    int32_t K;    // column checkpoint stride; a multiple of the segment width
    int32_t R;    // row checkpoint stride; a power of two
    int64_t nblk; // floor(M / K)
    int64_t ckpt_rows;  // checkpoint capacity in query samples (from start_q0)
    int* status;
    int* queue;          // persistent mode: device work counter (reset to 0 before the launch)
    const int32_t* order;// persistent mode: query order (longest first), or nullptr
};

struct FwdPlan {
    int W = 16;          // segment width: reference columns per thread
    int P = 8;           // warps per query chain
    int RT = 2;          // query rows per thread per step (tile height)
    bool persistent = false;
    int grid = 0;
    int block = 0;
    int smem = 0;
};

// Forward launch (sdtw_forward.cu).
bool fwd_width_supported(sdtw_dtype dt, int W);
int fwd_smem_bytes(sdtw_dtype dt, int N, int P, int W, int K, int RT);
int fwd_max_ctas_per_sm(sdtw_dtype dt, int W, int P, int smem, int RT, bool ckpt);
int64_t fwd_total_steps(int64_t M, int N, int W, int P, int RT);
cudaError_t launch_forward(sdtw_dtype dt, const FwdPlan& plan, const FwdArgs& a, cudaStream_t s);
cudaError_t launch_order_by_length(const int64_t* offsets, int32_t B, int32_t* order, cudaStream_t s);

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
    const float* ckpt;   // column checkpoints of queries q0 .. q0+B-1 (layout as FwdArgs)
    const float* rowck;  // row checkpoints (layout as FwdArgs)
    int32_t K;           // tile columns: the column checkpoint stride
    int32_t R;           // tile rows: the row checkpoint stride
    int64_t nblk;
    int64_t ckpt_rows;  // checkpoint capacity in query samples (from start_q0)
    float* gyq;      // [B][M] per-query reference gradient rows (only the path span is written)
    int64_t* span;   // [B][2] first and last column of each query's path
    int* status;
};

// Backward launches (sdtw_backward.cu).
bool bwd_stride_supported(int K);
int bwd_smem_bytes(int N, int K, int R);
size_t ckpt_floats_per_query(int64_t N, int64_t M, int K, int R);
bool bwd_row_stride_supported(int R);
cudaError_t launch_backward_walk(const BwdArgs& a, cudaStream_t s);
cudaError_t launch_grad_ref_reduce(const float* gyq, const int64_t* span, int32_t B, int64_t M,
                                   bool accumulate, float* grad_ref, cudaStream_t s);

}  // namespace sdtw
