// Forward sDTW fill: minimum cost and end column of every query of a batch.
//
// The recurrence is Eq. 1 of the paper (Section 2) with a free start and free
// end in the reference; one CTA owns one query (Section 5.2 gives each query
// its own block).
//
// Schedule.  The CTA's L = 32*P threads form a chain; thread l owns a strip of
// W consecutive reference columns (the paper's "segment", Section 5.2) and
// keeps the strip's current DP row and reference samples in registers.  At
// every step a thread advances its strip by one query row, and thread l runs
// one row behind thread l-1, so one step fills an anti-diagonal of strips.
// The strip's right-hand cell travels to the next thread by __shfl_up_sync
// inside a warp; between warps it goes through a small shared-memory ring,
// and warp w runs kChunk+1 steps further behind warp w-1 so that one CTA
// barrier every kChunk steps orders every ring write before its read.
//
// The chain covers S = L*W columns per sweep.  Sweeps are continuous: when a
// thread finishes the last query row of sweep s it starts row 0 of sweep s+1
// (columns shifted by S) on the next step, and the chain's last thread leaves
// the sweep's right-hand column in a shared-memory column buffer that the
// first thread reads one sweep later (the paper's double-buffered column
// between wavefronts, Section 5.2, kept as a single buffer indexed by row).
// Threads therefore never idle between sweeps; only the chain's start and end
// are ragged.
//
// The bottom-row minimum (Section 5.2 aggregates it while the last row is
// produced) is kept per thread as a running (value, column) pair updated with
// a strict '<' in increasing column order, then reduced over the CTA
// lexicographically, so the smallest end column wins exact ties.
//
// FP32 accuracy.  D grows along the query (to ~10^3 for N = 2,000), so one
// rounding of an FP32 cell costs ~10^-4 absolute, and the minimum over near-tied
// neighbours systematically keeps the one that rounded low: over a 2,000-row
// path plain FP32 drifts 3e-6 low on average and up to ~1.4e-5 (relative).  In
// FP32 mode each thread therefore stores its strip relative to a base B of its
// own (D = B + D'), and every kChunk steps all threads rebase to the integer
// part of their strip's first column, so the stored D' stay small; integer
// bases make every base difference exact, so exact costs (e.g. 0 for an exact
// cut of the reference) stay exact.
// Values crossing threads travel with their sender's base and are converted
// on receipt; a sweep starts from base 0.  The drift falls below 1e-7 and the
// worst error to ~1.5e-6, for one shuffle and two adds per step (W cells).
//
// Optional checkpoints for the backward pass: a thread whose strip ends at a
// multiple of K stores that column's absolute D value for every row.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "sdtw_cell.cuh"
#include "sdtw_internal.h"

namespace sdtw {
namespace {

template <typename Tin, int W>
__global__ void __launch_bounds__(kMaxWarpsPerQuery * 32)
fwd_chain_kernel(const FwdArgs a)
{
    using Md = Mode<Tin>;
    using V = typename Md::V;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_query;

    const int P = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int L = blockDim.x;
    const int N = a.N;
    const int M = static_cast<int>(a.M);
    const int S = L * W;
    const int nsw = (M + S - 1) / S;

    V* xs = reinterpret_cast<V*>(smem_raw);               // [N]   query samples
    V* colv = xs + N;                                      // [N]   sweep boundary column (values)
    float* colb = reinterpret_cast<float*>(colv + N);      // [N]   ... and their bases
    V* ringv = reinterpret_cast<V*>(colb + N);             // [P][kRing] warp-to-warp ring (values)
    float* ringb = reinterpret_cast<float*>(ringv + P * kRing);  // [P][kRing] ... and bases
    V* red_v = reinterpret_cast<V*>(ringb + P * kRing);    // [P]   reduction scratch
    int* red_i = reinterpret_cast<int*>(red_v + P);        // [P]

    const Tin* ref = static_cast<const Tin*>(a.ref);
    const Tin* queries = static_cast<const Tin*>(a.queries);

    const int64_t first_start = a.offsets ? a.offsets[a.q0] : static_cast<int64_t>(a.q0) * a.N;
    const int lag = warp * (32 + kChunk) + lane;
    const int lag_last = (P - 1) * (32 + kChunk) + 31;
    const V* ringv_in = ringv + warp * kRing;
    const float* ringb_in = ringb + warp * kRing;
    V* ringv_out = ringv + (warp + 1) * kRing;
    float* ringb_out = ringb + (warp + 1) * kRing;

    for (int it = 0;; ++it) {
        int q;
        if (a.queue) {
            if (threadIdx.x == 0) s_query = atomicAdd(a.queue, 1);
            __syncthreads();
            q = s_query;
            if (q >= a.B) break;
            q = a.order ? a.order[q] : a.q0 + q;
        } else {
            if (it > 0) break;
            q = a.q0 + blockIdx.x;
        }

        int64_t start;
        int n;
        if (a.offsets) {
            // 0 <= offsets[q] <= offsets[q+1] <= offsets[B]: the query lies inside the batch
            start = a.offsets[q];
            const int64_t stop = a.offsets[q + 1];
            const int64_t len = stop - start;
            bool bad = start < 0 || len < 0 || len > N || stop > a.offsets[a.B_total];
            if (a.ckpt) bad = bad || start < first_start || (stop - first_start) > a.ckpt_rows;
            if (bad) {
                if (threadIdx.x == 0) atomicOr(a.status, kStatusBadLength);
                __syncthreads();
                continue;
            }
            n = static_cast<int>(len);
        } else {
            start = static_cast<int64_t>(q) * N;
            n = N;
        }
        if (n == 0) {
            if (threadIdx.x == 0) {
                static_cast<V*>(a.cost)[q] = Md::empty_cost();
                a.end[q] = -1;
            }
            __syncthreads();
            continue;
        }

        for (int i = threadIdx.x; i < n; i += blockDim.x) xs[i] = Md::widen(queries[start + i]);
        __syncthreads();

        const int Np = max(n, lag_last + kChunk);
        const int total = (nsw - 1) * Np + n + lag_last;

        V y[W], D[W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
            y[k] = Md::zero();
            D[k] = Md::zero();
        }
        V diag = Md::zero();
        float B = 0.f;  // FP32 mode: this thread's base (absolute D = B + D')
        V best = Md::inf();
        int best_col = INT_MAX;
        int r = -lag;  // query row of this thread's strip (negative: not started)
        int s = 0;     // sweep
        int base = threadIdx.x * W;  // first column of the strip in sweep s
        float* ck = nullptr;

        for (int t0 = 0; t0 < total; t0 += kChunk) {
            if constexpr (Md::kRebase) {
                // new base: the integer part of the strip's first column; bases
                // are integers (exact below 2^24), so base differences, the
                // shift and every conversion between threads add no rounding
                const float bn = floorf(B + D[0]);
                const float dl = bn - B;
#pragma unroll
                for (int k = 0; k < W; ++k) D[k] -= dl;
                diag -= dl;
                B = bn;
            }
#pragma unroll 1
            for (int u = 0; u < kChunk; ++u) {
                const int t = t0 + u;
                V recv = __shfl_up_sync(0xffffffffu, D[W - 1], 1);
                float rb = 0.f;
                if constexpr (Md::kRebase) rb = __shfl_up_sync(0xffffffffu, B, 1);
                const bool act = static_cast<unsigned>(r) < static_cast<unsigned>(n) && s < nsw;
                if (lane == 0) {
                    if (warp > 0) {
                        const int slot = (t - kChunk - 1) & (kRing - 1);
                        recv = ringv_in[slot];
                        if constexpr (Md::kRebase) rb = ringb_in[slot];
                    } else if (act && s > 0) {
                        recv = colv[r];
                        if constexpr (Md::kRebase) rb = colb[r];
                    } else {
                        recv = Md::inf();
                        rb = 0.f;
                    }
                }
                if (act) {
                    if (r == 0) {
                        // new sweep: load the strip's reference samples; the
                        // previous row is the virtual all-zero row -1
                        base = s * S + threadIdx.x * W;
#pragma unroll
                        for (int k = 0; k < W; ++k) {
                            const int col = base + k;
                            y[k] = col < M ? Md::widen(ref[col]) : Md::zero();
                            D[k] = Md::zero();
                        }
                        diag = Md::zero();
                        B = 0.f;
                        ck = nullptr;
                        if (a.ckpt) {
                            const int edge = base + W;
                            if (edge % a.K == 0 && edge / a.K <= a.nblk)
                                ck = a.ckpt + (start - first_start) * a.nblk + static_cast<int64_t>(edge / a.K - 1) * n;
                        }
                    }
                    V left = recv;
                    if constexpr (Md::kRebase) left = recv + (rb - B);  // into this thread's base
                    const V conv = left;
                    const V xv = xs[r];
#pragma unroll
                    for (int k = 0; k < W; ++k) {
                        const V up = D[k];
                        const V nv = Md::cell(xv, y[k], up, diag, left);
                        diag = up;
                        left = nv;
                        D[k] = nv;
                    }
                    diag = conv;
                    if (r == n - 1) {
#pragma unroll
                        for (int k = 0; k < W; ++k) {
                            V v = D[k];
                            if constexpr (Md::kRebase) v = B + D[k];
                            if (base + k < M && v < best) {
                                best = v;
                                best_col = base + k;
                            }
                        }
                    }
                    if (lane == 31) {
                        if (warp < P - 1) {
                            ringv_out[t & (kRing - 1)] = D[W - 1];
                            if constexpr (Md::kRebase) ringb_out[t & (kRing - 1)] = B;
                        } else {
                            colv[r] = D[W - 1];
                            if constexpr (Md::kRebase) colb[r] = B;
                        }
                    }
                    if (ck) ck[r] = static_cast<float>(D[W - 1]) + B;
                }
                if (++r == Np) {
                    r = 0;
                    ++s;
                }
            }
            __syncthreads();
        }

        // lexicographic (value, column) minimum over the CTA
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const V ov = __shfl_down_sync(0xffffffffu, best, off);
            const int oc = __shfl_down_sync(0xffffffffu, best_col, off);
            if (ov < best || (ov == best && oc < best_col)) {
                best = ov;
                best_col = oc;
            }
        }
        if (lane == 0) {
            red_v[warp] = best;
            red_i[warp] = best_col;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            V bv = red_v[0];
            int bc = red_i[0];
            for (int w = 1; w < P; ++w) {
                if (red_v[w] < bv || (red_v[w] == bv && red_i[w] < bc)) {
                    bv = red_v[w];
                    bc = red_i[w];
                }
            }
            static_cast<V*>(a.cost)[q] = bv;
            a.end[q] = bc;
        }
        __syncthreads();
    }
}

// rank of each query by length, longest first (ties by index): order[rank] = q
__global__ void order_by_length_kernel(const int64_t* __restrict__ offsets, int32_t B,
                                       int32_t* __restrict__ order)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= B) return;
    const int64_t lq = offsets[q + 1] - offsets[q];
    int rank = 0;
    for (int p = 0; p < B; ++p) {
        const int64_t lp = offsets[p + 1] - offsets[p];
        rank += (lp > lq) || (lp == lq && p < q);
    }
    order[rank] = q;
}

template <typename Tin, int W>
cudaError_t launch_w(const FwdPlan& plan, const FwdArgs& a, cudaStream_t s)
{
    auto k = fwd_chain_kernel<Tin, W>;
    if (plan.smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, plan.smem);
        if (e != cudaSuccess) return e;
    }
    k<<<plan.grid, plan.block, plan.smem, s>>>(a);
    return cudaGetLastError();
}

template <typename Tin>
cudaError_t launch_t(const FwdPlan& plan, const FwdArgs& a, cudaStream_t s)
{
    switch (plan.W) {
    case 8: return launch_w<Tin, 8>(plan, a, s);
    case 16: return launch_w<Tin, 16>(plan, a, s);
    case 32: return launch_w<Tin, 32>(plan, a, s);
    default: return cudaErrorInvalidValue;
    }
}

template <typename Tin, int W>
int occupancy_w(int block, int smem)
{
    int n = 0;
    auto k = fwd_chain_kernel<Tin, W>;
    if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, smem) != cudaSuccess) return 0;
    return n;
}

template <typename Tin>
int occupancy_t(int W, int block, int smem)
{
    switch (W) {
    case 8: return occupancy_w<Tin, 8>(block, smem);
    case 16: return occupancy_w<Tin, 16>(block, smem);
    case 32: return occupancy_w<Tin, 32>(block, smem);
    default: return 0;
    }
}

}  // namespace

bool fwd_width_supported(sdtw_dtype, int W) { return W == 8 || W == 16 || W == 32; }

int fwd_smem_bytes(sdtw_dtype, int N, int P)
{
    // xs[N] + column values and bases [2N] + ring values and bases [2P*kRing]
    // + reduction (value, index)[P]; 4-byte elements
    return 4 * (3 * N + 2 * P * kRing + 2 * P);
}

int64_t fwd_total_steps(int64_t M, int N, int W, int P)
{
    const int64_t S = static_cast<int64_t>(32) * P * W;
    const int64_t nsw = (M + S - 1) / S;
    const int64_t lag_last = static_cast<int64_t>(P - 1) * (32 + kChunk) + 31;
    const int64_t Np = std::max<int64_t>(N, lag_last + kChunk);
    return (nsw - 1) * Np + N + lag_last;
}

int fwd_max_ctas_per_sm(sdtw_dtype dt, int W, int P, int smem)
{
    return dt == SDTW_I8 ? occupancy_t<int8_t>(W, P * 32, smem) : occupancy_t<float>(W, P * 32, smem);
}

cudaError_t launch_forward(sdtw_dtype dt, const FwdPlan& plan, const FwdArgs& a, cudaStream_t s)
{
    if (plan.grid <= 0) return cudaSuccess;
    return dt == SDTW_I8 ? launch_t<int8_t>(plan, a, s) : launch_t<float>(plan, a, s);
}

cudaError_t launch_order_by_length(const int64_t* offsets, int32_t B, int32_t* order, cudaStream_t s)
{
    if (B <= 0) return cudaSuccess;
    order_by_length_kernel<<<(B + 255) / 256, 256, 0, s>>>(offsets, B, order);
    return cudaGetLastError();
}

}  // namespace sdtw
