// Forward sDTW fill: minimum cost and end column of every query of a batch.
//
// The recurrence is Eq. 1 of the paper (Section 2) with a free start and free
// end in the reference; one CTA owns one query (Section 5.2 gives each query
// its own block).
//
// Schedule.  The CTA's L = 32*P threads form a chain; thread l owns a strip of
// W consecutive reference columns (the paper's "segment", Section 5.2) and
// keeps the strip's reference samples and its latest DP row in registers.  At
// every step a thread advances its strip by a pair of query rows (a 2 x W
// register tile), and thread l runs one step behind thread l-1, so one step
// fills an anti-diagonal of tiles.  Inside the tile, cells (r, k) and
// (r+1, k-1) are independent, so each thread runs two dependency chains; row r
// goes to a scratch strip and row r+1 overwrites the previous row one column
// behind it, so no register has to be moved between steps.  The tile's two
// right-hand cells travel to the next thread by __shfl_up_sync inside a warp;
// between warps they go through a small shared-memory ring, and warp w runs
// kChunk+1 steps further behind warp w-1 so that one CTA barrier every kChunk
// steps orders every ring write before its read.
//
// The chain covers S = L*W columns per sweep.  Sweeps are continuous: when a
// thread finishes the last row pair of sweep s it starts row pair 0 of sweep
// s+1 (columns shifted by S) on the next step, and the chain's last thread
// leaves the sweep's right-hand column in a shared-memory column buffer that
// the first thread reads one sweep later (the paper's double-buffered column
// between wavefronts, Section 5.2, kept as one buffer indexed by row pair).
// Threads never idle between sweeps; only the chain's start and end are
// ragged.  Chunks in which no thread of a warp starts a sweep or reaches the
// bottom row run a fast path without per-step bookkeeping.
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
// cut of the reference) stay exact.  Values crossing threads travel with their
// sender's base and are converted on receipt; a sweep starts from base 0.  The
// drift falls below 1e-7 and the worst error to ~1.5e-6.
//
// Optional checkpoints for the backward pass, taken as the wavefront passes:
// a thread whose strip ends at a multiple of K stores that column's absolute D
// value for every row, and every thread stores its strip of every R-th row
// (coalesced across the chain).  The backward recomputes R x K tiles from them.
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "sdtw_cell.cuh"
#include "sdtw_internal.h"

namespace sdtw {
namespace {

// The two right-hand cells of one row pair of a strip, with their base.
template <typename V>
struct alignas(16) Edge {
    V v0, v1;
    float b;
    int pad;
};

template <typename V>
struct Pair2;
template <>
struct Pair2<float> { using T = float2; };
template <>
struct Pair2<int32_t> { using T = int2; };

// One 2 x W tile: rows r (into A) and r+1 (over prev), walking the
// anti-diagonals of the tile so that the two rows form independent chains.
//   prev   in: row r-1 of the strip; out: row r+1
//   A      out: row r (A[W-1] is kept for the next step's send)
//   diag   D(r-1, c-1);  left0 = D(r, c-1);  left1 = D(r+1, c-1)
template <typename Md, int W>
__device__ __forceinline__ void tile_step(typename Md::V (&prev)[W], typename Md::V (&A)[W],
                                          const typename Md::V (&y)[W], typename Md::V x0,
                                          typename Md::V x1, typename Md::V diag,
                                          typename Md::V left0, typename Md::V left1)
{
    using V = typename Md::V;
#pragma unroll
    for (int k = 0; k <= W; ++k) {
        if (k < W) {
            const V up = prev[k];
            const V dg = k == 0 ? diag : prev[k - 1];
            const V lf = k == 0 ? left0 : A[k - 1];
            A[k] = Md::cell(x0, y[k], up, dg, lf);
        }
        if (k >= 1) {
            const int j = k - 1;
            const V up = A[j];
            const V dg = j == 0 ? left0 : A[j - 1];
            const V lf = j == 0 ? left1 : prev[j - 1];
            prev[j] = Md::cell(x1, y[j], up, dg, lf);
        }
    }
}

// Stage a strip of a checkpoint row: the lane's W values relative to its base,
// with 16-byte stores, and the base (the flush adds it back).  Runs on one
// lane at a time, so it is kept short.
template <int W, typename V>
__device__ __forceinline__ void stage_row(float* slot, const V (&prev)[W], float* base_slot, float B)
{
    static_assert(W % 4 == 0, "segment widths are multiples of 4");
    float4* s4 = reinterpret_cast<float4*>(slot);
#pragma unroll
    for (int k = 0; k < W / 4; ++k)
        s4[k] = make_float4(static_cast<float>(prev[4 * k]), static_cast<float>(prev[4 * k + 1]),
                            static_cast<float>(prev[4 * k + 2]), static_cast<float>(prev[4 * k + 3]));
    *base_slot = B;
}

// Register cap per segment width: the strip's samples and previous row (2W)
// plus the tile's short-lived values and bookkeeping, leaving room for several
// CTAs per SM.
template <int W>
constexpr int fwd_reg_cap() { return W <= 8 ? 72 : W <= 12 ? 80 : W <= 16 ? 88 : W <= 24 ? 112 : 128; }

template <typename Tin, int W>
__global__ void __maxnreg__(fwd_reg_cap<W>())
fwd_chain_kernel(const FwdArgs a)
{
    using Md = Mode<Tin>;
    using V = typename Md::V;
    using E = Edge<V>;
    using V2 = typename Pair2<V>::T;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_query;

    const int P = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int N = a.N;
    const int Npad = (N + 1) & ~1;
    const int M = static_cast<int>(a.M);
    const int S = blockDim.x * W;
    const int nsw = (M + S - 1) / S;

    // shared memory: ring [P][kRing] and column buffer [Npad/2] of 16-byte edges;
    // with checkpoints, the staging areas (16-byte aligned); query samples
    // [Npad] (zero padded); reduction scratch (value, index)[P]
    const int nslot = a.ckpt ? 32 * W / a.K : 0;           // checkpoint lanes per warp
    const int nstage = a.ckpt ? 1 : 0;
    E* ring = reinterpret_cast<E*>(smem_raw);
    E* colbuf = ring + P * kRing;
    // checkpoint staging: each warp gathers its 32 strips of a checkpoint row
    // (values relative to each lane's base, and the bases) and its checkpoint
    // lanes' column values of a chunk, so both leave as contiguous 128-byte lines
    float* rstage_all = reinterpret_cast<float*>(colbuf + Npad / 2);        // [P][32][W]
    float* rbase_all = rstage_all + nstage * P * 32 * W;                    // [P][32]
    float* cstage_all = rbase_all + nstage * P * 32;                        // [P][nslot][2*kChunk]
    V* xs = reinterpret_cast<V*>(cstage_all + P * nslot * 2 * kChunk);      // [Npad]
    V* red_v = xs + Npad;                                                   // [P]
    int* red_i = reinterpret_cast<int*>(red_v + P);                         // [P]
    float* rstage = rstage_all + warp * 32 * W;
    float* rbase = rbase_all + warp * 32;
    float* cstage = cstage_all + warp * nslot * 2 * kChunk;

    const Tin* ref = static_cast<const Tin*>(a.ref);
    const Tin* queries = static_cast<const Tin*>(a.queries);

    const int64_t first_start = a.offsets ? a.offsets[a.q0] : static_cast<int64_t>(a.q0) * a.N;
    const int wlag = warp * (32 + kChunk);
    const int lag = wlag + lane;
    const int lag_last = (P - 1) * (32 + kChunk) + 31;
    const E* ring_in = ring + warp * kRing;
    E* ring_out = ring + (warp + 1) * kRing;
    const V INF = Md::inf();

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
        if (threadIdx.x == 0 && (n & 1)) xs[n] = Md::zero();  // a dummy row completes the last pair
        __syncthreads();

        const int npairs = (n + 1) >> 1;
        const int lastp = npairs - 1;                      // the pair holding row n-1
        const int Pp = max(npairs, lag_last + kChunk);     // sweep period in steps
        const int total = (nsw - 1) * Pp + npairs + lag_last;
        const V2* xs2 = reinterpret_cast<const V2*>(xs);

        V y[W], prev[W], A[W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
            y[k] = Md::zero();
            prev[k] = Md::zero();
            A[k] = Md::zero();
        }
        V diag = Md::zero();
        float B = 0.f;  // FP32 mode: this thread's base (absolute D = B + D')
        float* rck = a.rowck ? a.rowck + ((start - first_start) / a.R) * a.M : nullptr;
        V best = INF;
        int best_col = INT_MAX;
        int p = -lag;   // row pair of this thread's tile in sweep s (negative: not started)
        int s = 0;      // sweep
        int base = threadIdx.x * W;  // first column of the strip in sweep s
        float* ck = nullptr;

        for (int t0 = 0; t0 < total; t0 += kChunk) {
            if constexpr (Md::kRebase) {
                // new base: the integer part of the strip's first column; bases
                // are integers (exact below 2^24), so base differences, the
                // shift and every conversion between threads add no rounding
                const float bn = floorf(B + prev[0]);
                const float dl = bn - B;
#pragma unroll
                for (int k = 0; k < W; ++k) prev[k] -= dl;
                A[W - 1] -= dl;
                diag -= dl;
                B = bn;
            }
            // fast path: no thread of this warp starts a sweep, idles or meets the
            // bottom row during the chunk (the test is uniform over the warp)
            const int gmin = t0 - wlag - 31;
            const int gmax = t0 - wlag + kChunk - 1;
            bool fast = gmin >= 0;
            if (fast) {
                const int sw = gmin / Pp;
                fast = gmax / Pp == sw && sw < nsw && gmin - sw * Pp >= 1 && gmax - sw * Pp <= lastp - 1;
            }
            if (fast) {
                float dconv = 0.f;  // base difference to the left neighbour, fixed for the chunk
                if constexpr (Md::kRebase) dconv = __shfl_up_sync(0xffffffffu, B, 1) - B;
                const int p_start = p;
                float* cslot = ck ? cstage + (((lane + 1) * W) / a.K - 1) * 2 * kChunk : nullptr;
#pragma unroll 1
                for (int u = 0; u < kChunk; ++u) {
                    const int t = t0 + u;
                    V v0 = __shfl_up_sync(0xffffffffu, A[W - 1], 1);
                    V v1 = __shfl_up_sync(0xffffffffu, prev[W - 1], 1);
                    float dd = dconv;
                    if (lane == 0) {
                        if (warp > 0) {
                            const E e = ring_in[(t - kChunk - 1) & (kRing - 1)];
                            v0 = e.v0;
                            v1 = e.v1;
                            dd = e.b - B;
                        } else if (s > 0) {
                            const E e = colbuf[p];
                            v0 = e.v0;
                            v1 = e.v1;
                            dd = e.b - B;
                        } else {
                            v0 = INF;
                            v1 = INF;
                            dd = 0.f;
                        }
                    }
                    V left0 = v0, left1 = v1;
                    if constexpr (Md::kRebase) {
                        left0 = v0 + dd;
                        left1 = v1 + dd;
                    }
                    const V2 xp = xs2[p];
                    tile_step<Md, W>(prev, A, y, xp.x, xp.y, diag, left0, left1);
                    diag = left1;
                    if (lane == 31) {
                        E e;
                        e.v0 = A[W - 1];
                        e.v1 = prev[W - 1];
                        e.b = B;
                        e.pad = 0;
                        if (warp < P - 1)
                            ring_out[t & (kRing - 1)] = e;
                        else
                            colbuf[p] = e;
                    }
                    if (cslot) {
                        cslot[2 * u] = static_cast<float>(A[W - 1]) + B;
                        cslot[2 * u + 1] = static_cast<float>(prev[W - 1]) + B;
                    }
                    if (rck) {
                        if (((2 * p + 2) & (a.R - 1)) == 0) stage_row<W>(rstage + lane * W, prev, rbase + lane, B);
                        // the warp's lanes reach a checkpoint row on consecutive
                        // steps; once lane 31 has staged it, write the whole row
                        const int p31 = p + lane - 31;
                        if (((2 * p31 + 2) & (a.R - 1)) == 0) {
                            __syncwarp();
                            const int col0 = s * S + warp * 32 * W;
                            float* dst = rck + static_cast<int64_t>((2 * p31 + 2) / a.R - 1) * a.M + col0;
                            for (int e = lane; e < 32 * W; e += 32)
                                if (col0 + e < M) dst[e] = rstage[e] + rbase[e / W];
                            __syncwarp();
                        }
                    }
                    ++p;
                    // a one-warp chain reads and rewrites the column buffer less than
                    // a chunk apart: order those accesses within the warp
                    if (P == 1) __syncwarp();
                }
                if (nslot) {
                    // the chunk's column checkpoints: 2*kChunk consecutive rows per
                    // checkpoint lane, written as whole 128-byte lines
                    __syncwarp();
                    float* dstl = ck ? ck + 2 * p_start : nullptr;
                    for (int j = 0; j < nslot; ++j) {
                        const int src = ((j + 1) * a.K) / W - 1;
                        float* d = reinterpret_cast<float*>(__shfl_sync(
                            0xffffffffu, reinterpret_cast<unsigned long long>(dstl), src));
                        if (d) {
#pragma unroll
                            for (int e = lane; e < 2 * kChunk; e += 32) d[e] = cstage[j * 2 * kChunk + e];
                        }
                    }
                    __syncwarp();
                }
            } else {
#pragma unroll 1
                for (int u = 0; u < kChunk; ++u) {
                    const int t = t0 + u;
                    V v0 = __shfl_up_sync(0xffffffffu, A[W - 1], 1);
                    V v1 = __shfl_up_sync(0xffffffffu, prev[W - 1], 1);
                    float rb = 0.f;
                    if constexpr (Md::kRebase) rb = __shfl_up_sync(0xffffffffu, B, 1);
                    const bool act = static_cast<unsigned>(p) < static_cast<unsigned>(npairs) && s < nsw;
                    bool rhit = false;
                    if (lane == 0) {
                        if (warp > 0) {
                            const E e = ring_in[(t - kChunk - 1) & (kRing - 1)];
                            v0 = e.v0;
                            v1 = e.v1;
                            rb = e.b;
                        } else if (act && s > 0) {
                            const E e = colbuf[p];
                            v0 = e.v0;
                            v1 = e.v1;
                            rb = e.b;
                        } else {
                            v0 = INF;
                            v1 = INF;
                            rb = 0.f;
                        }
                    }
                    if (act) {
                        if (p == 0) {
                            // new sweep: load the strip's reference samples; the
                            // previous row is the virtual all-zero row -1
                            base = s * S + threadIdx.x * W;
#pragma unroll
                            for (int k = 0; k < W; ++k) {
                                const int col = base + k;
                                y[k] = col < M ? Md::widen(ref[col]) : Md::zero();
                                prev[k] = Md::zero();
                            }
                            diag = Md::zero();
                            B = 0.f;
                            ck = nullptr;
                            if (a.ckpt) {
                                const int edge = base + W;
                                if (edge % a.K == 0 && edge / a.K <= a.nblk)
                                    ck = a.ckpt + (start - first_start) * a.nblk +
                                         static_cast<int64_t>(edge / a.K - 1) * n;
                            }
                        }
                        V left0 = v0, left1 = v1;
                        if constexpr (Md::kRebase) {
                            const float dd = rb - B;  // into this thread's base
                            left0 = v0 + dd;
                            left1 = v1 + dd;
                        }
                        const V2 xp = xs2[p];
                        tile_step<Md, W>(prev, A, y, xp.x, xp.y, diag, left0, left1);
                        diag = left1;
                        if (p == lastp) {
                            // row n-1 is the pair's first row (odd n) or its second
#pragma unroll
                            for (int k = 0; k < W; ++k) {
                                V v = (n & 1) ? A[k] : prev[k];
                                if constexpr (Md::kRebase) v = v + B;
                                if (base + k < M && v < best) {
                                    best = v;
                                    best_col = base + k;
                                }
                            }
                        }
                        if (lane == 31) {
                            E e;
                            e.v0 = A[W - 1];
                            e.v1 = prev[W - 1];
                            e.b = B;
                            e.pad = 0;
                            if (warp < P - 1)
                                ring_out[t & (kRing - 1)] = e;
                            else
                                colbuf[p] = e;
                        }
                        if (ck) {
                            ck[2 * p] = static_cast<float>(A[W - 1]) + B;
                            if (2 * p + 1 < n) ck[2 * p + 1] = static_cast<float>(prev[W - 1]) + B;
                        }
                        if (rck && ((2 * p + 2) & (a.R - 1)) == 0 && 2 * p + 1 < n) {
                            rhit = true;
                            stage_row<W>(rstage + lane * W, prev, rbase + lane, B);
                        }
                    }
                    if (rck) {
                        // write a staged checkpoint row once lane 31 has staged it
                        // (lanes may straddle a sweep here: use lane 31's sweep and row)
                        if (__ballot_sync(0xffffffffu, rhit) & 0x80000000u) {
                            __syncwarp();
                            const int s31 = __shfl_sync(0xffffffffu, s, 31);
                            const int p31 = __shfl_sync(0xffffffffu, p, 31);
                            const int col0 = s31 * S + warp * 32 * W;
                            float* dst = rck + static_cast<int64_t>((2 * p31 + 2) / a.R - 1) * a.M + col0;
                            for (int e = lane; e < 32 * W; e += 32)
                                if (col0 + e < M) dst[e] = rstage[e] + rbase[e / W];
                            __syncwarp();
                        }
                        rhit = false;
                    }
                    if (++p == Pp) {
                        p = 0;
                        ++s;
                    }
                    if (P == 1) __syncwarp();
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
    case 12: return launch_w<Tin, 12>(plan, a, s);
    case 16: return launch_w<Tin, 16>(plan, a, s);
    case 24: return launch_w<Tin, 24>(plan, a, s);
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
    case 12: return occupancy_w<Tin, 12>(block, smem);
    case 16: return occupancy_w<Tin, 16>(block, smem);
    case 24: return occupancy_w<Tin, 24>(block, smem);
    case 32: return occupancy_w<Tin, 32>(block, smem);
    default: return 0;
    }
}

}  // namespace

bool fwd_width_supported(sdtw_dtype, int W) { return W == 8 || W == 12 || W == 16 || W == 24 || W == 32; }

int fwd_smem_bytes(sdtw_dtype, int N, int P, int W, int K)
{
    // ring [P][kRing] and column buffer [Npad/2] of 16-byte edges, query samples
    // [Npad] and the reduction (value, index)[P], 4-byte elements; with
    // checkpoints (K > 0) the row staging [P][32][W] and its bases [P][32] and
    // the column staging [P][32W/K][2*kChunk] floats
    const int npad = (N + 1) & ~1;
    int bytes = 16 * (P * kRing + npad / 2) + 4 * (npad + 2 * P);
    if (K > 0) bytes += 4 * P * (32 * W + 32 + (32 * W / K) * 2 * kChunk);
    return bytes;
}

int64_t fwd_total_steps(int64_t M, int N, int W, int P)
{
    const int64_t S = static_cast<int64_t>(32) * P * W;
    const int64_t nsw = (M + S - 1) / S;
    const int64_t lag_last = static_cast<int64_t>(P - 1) * (32 + kChunk) + 31;
    const int64_t npairs = (N + 1) / 2;
    const int64_t Pp = std::max<int64_t>(npairs, lag_last + kChunk);
    return (nsw - 1) * Pp + npairs + lag_last;
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
