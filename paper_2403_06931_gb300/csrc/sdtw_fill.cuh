// Forward sDTW fill: minimum cost and end column of every query of a batch.
//
// The recurrence is Eq. 1 of the paper (Section 2) with a free start and free
// end in the reference; one CTA owns one query (Section 5.2 gives each query
// its own block).
//
// Schedule.  The CTA's L = 32*P threads form a chain; thread l owns a strip of
// W consecutive reference columns (the paper's "segment", Section 5.2) and
// keeps the strip's reference samples and its latest DP row in registers.  At
// every step a thread advances its strip by RT query rows (an RT x W register
// tile, RT = 2, 4 or 8), and thread l runs one step behind thread l-1, so one
// step fills an anti-diagonal of tiles.  Inside the tile, cell j of row r and
// cell j-1 of row r+1 are independent, so each thread runs RT dependency
// chains; the tile's first RT-1 rows go to short-lived scratch registers and
// its last row overwrites the previous row RT-1 columns behind the first, so
// no register has to be moved between steps.  The tile's RT right-hand cells
// travel to the next thread by __shfl_up_sync inside a warp; between warps
// they go through a small shared-memory ring, and warp w runs kChunk+1 steps
// further behind warp w-1 so that one CTA barrier every kChunk steps orders
// every ring write before its read.
//
// The chain covers S = L*W columns per sweep.  Sweeps are continuous: when a
// thread finishes the last tile of rows of sweep s it starts the first tile of
// sweep s+1 (columns shifted by S) on the next step, and the chain's last
// thread leaves the sweep's right-hand column in a shared-memory column buffer
// that the first thread reads one sweep later (the paper's double-buffered
// column between wavefronts, Section 5.2, kept as one buffer indexed by tile).
// Threads never idle between sweeps; only the chain's start and end are
// ragged.  Chunks in which no thread of a warp starts a sweep or reaches the
// bottom row run a fast path without per-step bookkeeping.
//
// The bottom-row minimum (Section 5.2 aggregates it while the last row is
// produced) is kept per thread as a running (value, column) pair updated with
// a strict '<' in increasing column order -- from the strip's latest row after
// the tile when the query's last row ends a tile, else inside the tile that
// holds it, on the steps where some lane of the warp holds that tile -- then
// reduced over the CTA lexicographically, so the smallest end column wins
// exact ties.
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
// Optional checkpoints for the backward pass (a separate instantiation, so the
// plain forward carries none of it).  At the end of every chunk every thread
// stores its state as the next chunk will find it before its rebase: the
// strip's latest row relative to its base, the right-hand cells of its tile's
// other rows, its diagonal input and the base (the backward redoes the
// rebase).  Since thread l is one tile behind thread l-1, the rows stored at
// one chunk end form an anti-diagonal staircase, the wavefront; all lanes
// store on the same step, so the stores are whole-warp and coalesced.  The
// strip whose first column is a multiple of K also stores the left inputs it
// uses, already converted into its own base.  From a chunk's wavefront and
// those columns the backward recomputes any K-column window of the chunk with
// the forward's own operations, bit for bit.  Checkpoints go out with the
// streaming (evict-first) store hint.
#pragma once

#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>
#include <cstring>
#include <type_traits>

#include "sdtw_cell.cuh"
#include "sdtw_internal.h"

namespace sdtw {
namespace {

// The RT right-hand cells of one tile of a strip, with their base.
template <typename V, int RT>
struct alignas(16) Edge {
    V v[RT];
    float b;
};

template <typename V, int RT>
struct VecOf;
template <>
struct VecOf<float, 2> { using T = float2; };
template <>
struct VecOf<float, 4> { using T = float4; };
template <>
struct VecOf<int32_t, 2> { using T = int2; };
template <>
struct VecOf<int32_t, 4> { using T = int4; };
template <>
struct VecOf<__half2, 2> { using T = uint2; };
template <>
struct VecOf<__half2, 4> { using T = uint4; };

// Four consecutive input samples as one load: 16 bytes of float, 8 of binary16,
// 4 of int8 or uint8 codes.
template <typename Tin>
struct Vec4Of;
template <>
struct Vec4Of<float> { using T = float4; };
template <>
struct Vec4Of<__half> { using T = uint2; };
template <>
struct Vec4Of<int8_t> { using T = char4; };
template <>
struct Vec4Of<uint8_t> { using T = uchar4; };

// A strip's W reference samples from column base: W/4 vector loads when the
// strip lies inside the reference and the reference is aligned for them (the
// strip's first column is a multiple of 4), else one load per column with the
// columns past the reference set to zero.
template <typename Md, typename Tin, int W>
__device__ __forceinline__ void load_strip(const Tin* ref, int base, int M, bool vec_ok, typename Md::V (&y)[W])
{
    static_assert(W % 4 == 0, "strips are whole vectors");
    using V4 = typename Vec4Of<Tin>::T;
    if (vec_ok && base + W <= M) {
        const V4* p4 = reinterpret_cast<const V4*>(ref + base);
#pragma unroll
        for (int k4 = 0; k4 < W / 4; ++k4) {
            const V4 v = p4[k4];
            Tin e[4];
            memcpy(e, &v, sizeof(v));
#pragma unroll
            for (int u = 0; u < 4; ++u) y[4 * k4 + u] = Md::widen(e[u]);
        }
    } else {
#pragma unroll
        for (int k = 0; k < W; ++k) y[k] = base + k < M ? Md::widen(ref[base + k]) : Md::zero();
    }
}

// the RT query samples of tile p (xs is 16-byte aligned and zero padded)
template <int RT, typename V>
__device__ __forceinline__ void load_x(const V* xs, int p, V (&x)[RT])
{
    if constexpr (RT == 8) {
        // eight 4-byte samples (float, int32 or a binary16 pair): two 16-byte loads
        static_assert(sizeof(V) == 4, "4-byte samples");
        const uint4* p4 = reinterpret_cast<const uint4*>(xs) + 2 * p;
        const uint4 u = p4[0], w = p4[1];
        const uint32_t b[8] = {u.x, u.y, u.z, u.w, w.x, w.y, w.z, w.w};
#pragma unroll
        for (int r = 0; r < 8; ++r) memcpy(&x[r], &b[r], 4);
        return;
    } else {
    const auto v = reinterpret_cast<const typename VecOf<V, RT>::T*>(xs)[p];
    if constexpr (std::is_same<V, __half2>::value) {
        x[0] = Mode<__half>::from_bits(v.x);
        x[1] = Mode<__half>::from_bits(v.y);
        if constexpr (RT == 4) {
            x[2] = Mode<__half>::from_bits(v.z);
            x[3] = Mode<__half>::from_bits(v.w);
        }
    } else {
        x[0] = v.x;
        x[1] = v.y;
        if constexpr (RT == 4) {
            x[2] = v.z;
            x[3] = v.w;
        }
    }
    }
}

// One RT x W tile, walking its anti-diagonals so that its rows form RT
// independent chains.
//   prev   in: the strip's previous row; out: the tile's last row
//   A      out: the tile's other rows (only A[r][W-1] outlives the step)
//   diag   D of the row above the tile in the column left of the strip
//   left   D of each tile row in the column left of the strip
// With BOT, the values of tile row bot_row (relative to base B) update the
// running bottom-row minimum as they are produced.
template <typename Md, int W, int RT, bool BOT, bool PRUNE = false>
__device__ __forceinline__ void tile_step(typename Md::V (&prev)[W], typename Md::V (&A)[RT - 1][W],
                                          const typename Md::V (&y)[W], const typename Md::V (&x)[RT],
                                          typename Md::V diag, const typename Md::V (&left)[RT], int bot_row,
                                          float B, int base, int M, typename Md::V& best,
                                          typename Md::Col& best_col, int gap = 0)
{
    using V = typename Md::V;
    // the inputs of cell (rr, j) of the tile
    auto inputs = [&](int rr, int j, V& up, V& dg, V& lf) {
        if (rr == 0) {
            up = prev[j];
            dg = j == 0 ? diag : prev[j - 1];
        } else {
            up = A[rr - 1][j];
            dg = j == 0 ? left[rr - 1] : A[rr - 1][j - 1];
        }
        if (j == 0)
            lf = left[rr];
        else if (rr == RT - 1)
            lf = prev[j - 1];
        else
            lf = A[rr][j - 1];
    };
    // its result: the last row overwrites the previous row in place; with BOT
    // the bottom row updates the running minimum
    auto result = [&](int rr, int j, V nv) {
        if (rr == RT - 1)
            prev[j] = nv;
        else
            A[rr][j] = nv;
        if constexpr (BOT) {
            if (rr == bot_row) {
                if constexpr (Md::kPair) {
                    if (base + j < M) Md::bot_update(nv, base + j, best, best_col);
                } else {
                    V v = nv;
                    if constexpr (Md::kRebase) v = nv + B;
                    if (base + j < M && v < best) {
                        best = v;
                        best_col = base + j;
                    }
                }
            }
        }
    };
#pragma unroll
    for (int k = 0; k < W + RT - 1; ++k) {
        if constexpr (Md::kPack2) {
            // anti-diagonal k holds cells (rr, k - rr): rows rr and rr + 1 are
            // independent and go through one packed multiply-add when both
            // cells lie in the strip (inputs gathered before either is written)
#pragma unroll
            for (int rr = 0; rr < RT; rr += 2) {
                const int j0 = k - rr, j1 = k - rr - 1;
                const bool in0 = j0 >= 0 && j0 < W, in1 = j1 >= 0 && j1 < W;
                if (in0 && in1) {
                    V up0, dg0, lf0, up1, dg1, lf1;
                    inputs(rr, j0, up0, dg0, lf0);
                    inputs(rr + 1, j1, up1, dg1, lf1);
                    const float2 nv = Md::cell2(x[rr], y[j0], up0, dg0, lf0, x[rr + 1], y[j1], up1, dg1, lf1);
                    result(rr, j0, nv.x);
                    result(rr + 1, j1, nv.y);
                } else if (in0) {
                    V up, dg, lf;
                    inputs(rr, j0, up, dg, lf);
                    result(rr, j0, Md::cell(x[rr], y[j0], up, dg, lf));
                } else if (in1) {
                    V up, dg, lf;
                    inputs(rr + 1, j1, up, dg, lf);
                    result(rr + 1, j1, Md::cell(x[rr + 1], y[j1], up, dg, lf));
                }
            }
        } else {
#pragma unroll
            for (int rr = 0; rr < RT; ++rr) {
                const int j = k - rr;
                if (j < 0 || j >= W) continue;
                V up, dg, lf;
                inputs(rr, j, up, dg, lf);
                if constexpr (PRUNE)
                    result(rr, j, Md::cell_pruned(x[rr], y[j], up, dg, lf, gap));
                else
                    result(rr, j, Md::cell(x[rr], y[j], up, dg, lf));
            }
        }
    }
}

// The running bottom-row minimum over the strip's latest row, when that row is
// the query's last: strict '<' in increasing column order (the smallest column
// of exact ties), as the in-tile update of tile_step does.
template <typename Md, int W>
__device__ __forceinline__ void bottom_min_prev(const typename Md::V (&prev)[W], float B, int base, int M,
                                                typename Md::V& best, typename Md::Col& best_col)
{
    using V = typename Md::V;
#pragma unroll
    for (int j = 0; j < W; ++j) {
        if constexpr (Md::kPair) {
            if (base + j < M) Md::bot_update(prev[j], base + j, best, best_col);
        } else {
            V v = prev[j];
            if constexpr (Md::kRebase) v = v + B;
            if (base + j < M && v < best) {
                best = v;
                best_col = base + j;
            }
        }
    }
}

// FP32 mode: a left input far below the strip's base.  A horizontal run of
// the path entering from a cheaper strip carries values far below the bases
// the strips it crosses took from their own cells, and every cell of the run
// would then round at the scale of that gap.  When the tile's first-row left
// input lies more than kRebaseBelow under the base, the strip is rebased to
// it (an integer base again, so the shift is an integer) before the tile:
// the previous row, the diagonal input and the tile's left inputs move with
// it.  The decision uses the first row only, which the backward's replay of
// the band also has when it recomputes that row.
template <bool VOTE, int W, int RT>
__device__ __forceinline__ bool rebase_to_left(float (&prev)[W], float& diag, float (&left)[RT], float& B)
{
    // decided per lane; with VOTE (all 32 lanes present) applied under a warp
    // vote, lanes that keep their base shifting by 0, so that the common step
    // (no lane rebases) takes no divergent branch
    const bool low = left[0] < -kRebaseBelow;
    if (VOTE ? !__any_sync(0xffffffffu, low) : !low) return false;
    const float bn = low ? floorf(B + left[0]) : B;
    const float dl = bn - B;
#pragma unroll
    for (int k = 0; k < W; ++k) prev[k] -= dl;
    diag -= dl;
#pragma unroll
    for (int rr = 0; rr < RT; ++rr) left[rr] -= dl;
    B = bn;
    return true;
}

// The RT left inputs of a tile at dst + off, for the threads whose dst is not
// null, as vector stores (the destination is 4 * RT-byte aligned: windows are
// ck_rows(N) floats apart).  One thread in eight stores a window's boundary
// column, and a branch around its store split the tile's instruction schedule
// in every step, so the stores are predicated (0.15-0.26 ms faster checkpointing
// fills on the paper batch).  Checkpoints are written once and read by a later
// kernel, so they carry the streaming (evict-first) hint: plain stores
// measurably slowed the fill.
template <int RT>
__device__ __forceinline__ void store_rows_if(const float* dst, int off, const float (&v)[RT])
{
    const uint64_t ad = reinterpret_cast<uint64_t>(dst) + 4u * static_cast<uint32_t>(off);
    const int pr = dst != nullptr ? 1 : 0;
    if constexpr (RT == 2) {
        asm volatile("{ .reg .pred p; setp.ne.b32 p, %0, 0; @p st.global.cs.v2.f32 [%1], {%2, %3}; }"
                     :: "r"(pr), "l"(ad), "f"(v[0]), "f"(v[1]));
    } else {
        asm volatile("{ .reg .pred p; setp.ne.b32 p, %0, 0; @p st.global.cs.v4.f32 [%1], {%2, %3, %4, %5}; }"
                     :: "r"(pr), "l"(ad), "f"(v[0]), "f"(v[1]), "f"(v[2]), "f"(v[3]));
        if constexpr (RT == 8)
            asm volatile("{ .reg .pred p; setp.ne.b32 p, %0, 0; @p st.global.cs.v4.f32 [%1], {%2, %3, %4, %5}; }"
                         :: "r"(pr), "l"(ad + 16), "f"(v[4]), "f"(v[5]), "f"(v[6]), "f"(v[7]));
    }
}

// Register cap per segment width and tile height: the strip's samples and
// previous row (2W), the tile's short-lived values and bookkeeping, leaving
// room for several CTAs per SM.
// (one template argument, W * 16 + RT, as the attribute takes a single expression)
template <int WRT>
constexpr int fwd_reg_cap()
{
    constexpr int W = WRT / 16, RT = WRT % 16;
    if (RT == 8) return W <= 16 ? 112 : W <= 20 ? 120 : 128;
    return W <= 8 ? (RT == 2 ? 72 : 80) : W <= 16 ? (RT == 2 ? 88 : 96) : W <= 20 ? (RT == 2 ? 104 : 112) : W <= 24 ? (RT == 2 ? 112 : 120) : 128;
}

template <typename Tin, int W, int RT, bool CKPT, bool PRUNE>
__global__ void __maxnreg__(fwd_reg_cap<W * 16 + RT>())
fwd_chain_kernel(const FwdArgs a)
{
    using Md = Mode<Tin>;
    using V = typename Md::V;
    using E = Edge<V, RT>;
    static_assert(RT == 2 || RT == 4 || RT == 8, "tiles of 2, 4 or 8 rows");

    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_query;

    const int P = blockDim.x >> 5;
    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;
    const int N = a.N;
    const int Npad = (N + RT - 1) / RT * RT;
    const int M = static_cast<int>(a.M);
    const int S = blockDim.x * W;
    const int nsw = (M + S - 1) / S;

    // shared memory: ring [P][kRing] and column buffer [Npad/RT] of edges;
    // query samples [Npad] (zero padded); reduction scratch (value, index)[P].
    // Every part is 16-byte aligned.
    E* ring = reinterpret_cast<E*>(smem_raw);
    E* colbuf = ring + P * kRing;
    V* xs = reinterpret_cast<V*>(colbuf + Npad / RT);  // [Npad]
    V* red_v = xs + Npad;                              // [P]
    int* red_i = reinterpret_cast<int*>(red_v + P);    // [P]

    const Tin* ref = static_cast<const Tin*>(a.ref);
    const Tin* queries = static_cast<const Tin*>(a.queries);
    // strips are loaded as vectors of four samples when the reference allows it
    const bool ref_vec = reinterpret_cast<uintptr_t>(ref) % (4 * sizeof(Tin)) == 0;

    const int wlag = warp * (32 + kChunk);
    const int lag = wlag + lane;
    const int lag_last = (P - 1) * (32 + kChunk) + 31;
    const E* ring_in = ring + warp * kRing;
    E* ring_out = ring + (warp + 1) * kRing;
    const V INF = Md::inf();
    const int gap = a.prune_gap;  // integer modes with pruning: the largest sample difference that is not pruned
    constexpr int EREC = fwd_record_floats(RT);  // floats of a thread's checkpoint record
    const int L = blockDim.x;

    for (int it = 0;; ++it) {
        int q;
        if (a.queue) {
            if (threadIdx.x == 0) s_query = atomicAdd(a.queue, 1);
            __syncthreads();
            q = s_query;
            if constexpr (Md::kPair) {
                // binary16 pairs (uniform batches): work item q is queries 2q, 2q+1
                if (2 * q >= a.B) break;
                q = a.q0 + 2 * q;
            } else {
                if (q >= a.B) break;
                q = a.order ? a.order[q] : a.q0 + q;
            }
        } else {
            if (it > 0) break;
            q = a.q0 + (Md::kPair ? 2 : 1) * static_cast<int>(blockIdx.x);
        }

        int64_t start;
        int n;
        int qb = q;  // binary16 pairs: the query in the high halves (the last pair of an odd batch repeats q)
        if constexpr (Md::kPair) {
            // uniform batches only: the CTA's two queries, both N long
            qb = min(q + 1, a.q0 + a.B - 1);
            start = static_cast<int64_t>(q) * N;
            n = N;
        } else if (a.offsets) {
            // 0 <= offsets[q] <= offsets[q+1] <= offsets[B]: the query lies inside the batch
            start = a.offsets[q];
            const int64_t stop = a.offsets[q + 1];
            const int64_t len = stop - start;
            bool bad = start < 0 || len < 0 || len > N || stop > a.offsets[a.B_total] || (a.q_limit > 0 && stop > a.q_limit);
            if (bad) {
                // flagged, and the outputs get the empty query's values, so that
                // no caller reads a stale cost or end for it
                if (threadIdx.x == 0) {
                    atomicOr(a.status, kStatusBadLength);
                    static_cast<V*>(a.cost)[q] = Md::empty_cost();
                    a.end[q] = -1;
                }
                __syncthreads();
                continue;
            }
            n = static_cast<int>(len);
        } else {
            start = static_cast<int64_t>(q) * N;
            n = N;
        }
        if constexpr (!Md::kPair) {
            if (n == 0) {
                if (threadIdx.x == 0) {
                    static_cast<V*>(a.cost)[q] = Md::empty_cost();
                    a.end[q] = -1;
                }
                __syncthreads();
                continue;
            }
        }

        const int nt = (n + RT - 1) / RT;  // tiles of rows per sweep
        if constexpr (Md::kPair) {
            const int64_t startb = static_cast<int64_t>(qb) * N;
            for (int i = threadIdx.x; i < nt * RT; i += blockDim.x)
                xs[i] = i < n ? Md::pack(queries[start + i], queries[startb + i]) : Md::zero();
        } else {
            for (int i = threadIdx.x; i < nt * RT; i += blockDim.x)
                xs[i] = i < n ? Md::widen(queries[start + i]) : Md::zero();  // dummy rows complete the last tile
        }
        __syncthreads();

        const int lastt = nt - 1;                 // the tile holding row n-1
        const int bot = (n - 1) - RT * lastt;     // ... as its row bot
        const int Pp = max(nt, lag_last + kChunk);  // sweep period in steps
        const int total = (nsw - 1) * Pp + nt + lag_last;

        V y[W], prev[W], A[RT - 1][W];
#pragma unroll
        for (int k = 0; k < W; ++k) {
            y[k] = Md::zero();
            prev[k] = Md::zero();
#pragma unroll
            for (int rr = 0; rr < RT - 1; ++rr) A[rr][k] = Md::zero();
        }
        V diag = Md::zero();
        float B = 0.f;  // FP32 mode: this thread's base (absolute D = B + D')
        V best = INF;
        typename Md::Col best_col;
        if constexpr (Md::kPair)
            best_col = make_int2(INT_MAX, INT_MAX);
        else
            best_col = INT_MAX;
        int p = -lag;   // tile of this thread's strip in sweep s (negative: not started)
        int s = 0;      // sweep
        int base = threadIdx.x * W;  // first column of the strip in sweep s
        // checkpoints of this query: the wavefront slot and, for a strip that
        // starts at a multiple of K, its boundary column
        float* frq = CKPT ? a.fr + static_cast<int64_t>(q - a.q0) * a.fr_slot : nullptr;
        float* ck = nullptr;

        // checkpointing: the wavefront is stored every ks steps (16, 32 or 64),
        // so a chunk runs as segments of seg steps with a store between them
        const int ks = CKPT ? a.ck_stride : kChunk;
        const int seg = CKPT ? min(ks, kChunk) : kChunk;
        for (int t0 = 0; t0 < total; t0 += kChunk) {
            // rebase at the start of every rebase period (a whole number of
            // chunks: one, or two with 64-step checkpoints, so that the
            // checkpoints always fall on rebase boundaries or between them;
            // a plain fill in a context that keeps checkpoints rebases like
            // its checkpointing fill, so that both return the same costs)
            const bool do_rebase = (t0 & (a.rebase_period - 1)) == 0;
            if constexpr (Md::kRebase) if (do_rebase) {
                // new base: the integer part of the strip's first column; bases
                // are integers (exact below 2^24), so base differences, the
                // shift and every conversion between threads add no rounding
                const float bn = floorf(B + prev[0]);
                const float dl = bn - B;
#pragma unroll
                for (int k = 0; k < W; ++k) prev[k] -= dl;
#pragma unroll
                for (int rr = 0; rr < RT - 1; ++rr) A[rr][W - 1] -= dl;
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
                fast = gmax / Pp == sw && sw < nsw && gmin - sw * Pp >= 1 && gmax - sw * Pp <= lastt - 1;
            }
            for (int ub = 0; ub < kChunk; ub += seg) {
                const int ue = ub + seg;
                if (fast) {
                    // base difference to the left neighbour: fixed between rebases
                    float dconv = 0.f;
                    if constexpr (Md::kRebase) dconv = __shfl_up_sync(0xffffffffu, B, 1) - B;
#pragma unroll 1
                    for (int u = ub; u < ue; ++u) {
                        const int t = t0 + u;
                        V x[RT];
                        load_x<RT>(xs, p, x);
                        V recv[RT];
#pragma unroll
                        for (int rr = 0; rr < RT; ++rr)
                            recv[rr] = __shfl_up_sync(0xffffffffu, rr < RT - 1 ? A[rr][W - 1] : prev[W - 1], 1);
                        float dd = dconv;
                        if (lane == 0) {
                            if (warp > 0) {
                                const E e = ring_in[(t - kChunk - 1) & (kRing - 1)];
#pragma unroll
                                for (int rr = 0; rr < RT; ++rr) recv[rr] = e.v[rr];
                                dd = e.b - B;
                            } else if (s > 0) {
                                const E e = colbuf[p];
#pragma unroll
                                for (int rr = 0; rr < RT; ++rr) recv[rr] = e.v[rr];
                                dd = e.b - B;
                            } else {
#pragma unroll
                                for (int rr = 0; rr < RT; ++rr) recv[rr] = INF;
                                dd = 0.f;
                            }
                        }
                        V left[RT];
#pragma unroll
                        for (int rr = 0; rr < RT; ++rr) {
                            left[rr] = recv[rr];
                            if constexpr (Md::kRebase) left[rr] = recv[rr] + dd;
                        }
                        if constexpr (CKPT) {
                            store_rows_if<RT>(ck, RT * p, left);  // as converted, before any shift
                        }
                        if constexpr (Md::kRebase) {
                            // a lane that rebased changes its own and its right neighbour's conversion
                            if (rebase_to_left<true, W, RT>(prev, diag, left, B))
                                dconv = __shfl_up_sync(0xffffffffu, B, 1) - B;
                        }
                        tile_step<Md, W, RT, false, PRUNE>(prev, A, y, x, diag, left, 0, B, base, M, best, best_col, gap);
                        diag = left[RT - 1];
                        if (lane == 31) {
                            E e;
#pragma unroll
                            for (int rr = 0; rr < RT; ++rr) e.v[rr] = rr < RT - 1 ? A[rr][W - 1] : prev[W - 1];
                            e.b = B;
                            if (warp < P - 1)
                                ring_out[t & (kRing - 1)] = e;
                            else
                                colbuf[p] = e;
                        }
                        ++p;
                        // a one-warp chain reads and rewrites the column buffer less than
                        // a chunk apart: order those accesses within the warp
                        if (P == 1) __syncwarp();
                    }
                } else {
#pragma unroll 1
                    for (int u = ub; u < ue; ++u) {
                        const int t = t0 + u;
                        V recv[RT];
#pragma unroll
                        for (int rr = 0; rr < RT; ++rr)
                            recv[rr] = __shfl_up_sync(0xffffffffu, rr < RT - 1 ? A[rr][W - 1] : prev[W - 1], 1);
                        float rb = 0.f;
                        if constexpr (Md::kRebase) rb = __shfl_up_sync(0xffffffffu, B, 1);
                        const bool act = static_cast<unsigned>(p) < static_cast<unsigned>(nt) && s < nsw;
                        if (lane == 0) {
                            if (warp > 0) {
                                const E e = ring_in[(t - kChunk - 1) & (kRing - 1)];
#pragma unroll
                                for (int rr = 0; rr < RT; ++rr) recv[rr] = e.v[rr];
                                rb = e.b;
                            } else if (act && s > 0) {
                                const E e = colbuf[p];
#pragma unroll
                                for (int rr = 0; rr < RT; ++rr) recv[rr] = e.v[rr];
                                rb = e.b;
                            } else {
#pragma unroll
                                for (int rr = 0; rr < RT; ++rr) recv[rr] = INF;
                                rb = 0.f;
                            }
                        }
                        if (act) {
                            if (p == 0) {
                                // new sweep: load the strip's reference samples; the
                                // previous row is the virtual all-zero row -1
                                base = s * S + threadIdx.x * W;
                                load_strip<Md, Tin, W>(ref, base, M, ref_vec, y);
#pragma unroll
                                for (int k = 0; k < W; ++k) prev[k] = Md::zero();
                                diag = Md::zero();
                                B = 0.f;
                                if constexpr (CKPT) {
                                    // a strip starting a K-column window (not the first)
                                    // keeps its left inputs for the backward
                                    ck = nullptr;
                                    if (base % a.K == 0 && base > 0 && base < M)
                                        ck = a.colck + static_cast<int64_t>(q - a.q0) * a.ck_slot +
                                             static_cast<int64_t>(base / a.K - 1) * ck_rows(N);
                                }
                            }
                            V left[RT];
#pragma unroll
                            for (int rr = 0; rr < RT; ++rr) {
                                left[rr] = recv[rr];
                                if constexpr (Md::kRebase) left[rr] = recv[rr] + (rb - B);  // into this thread's base
                            }
                            if constexpr (CKPT) {
                                // as converted, before any shift; padding rows fall in the padded slot
                                store_rows_if<RT>(ck, RT * p, left);
                            }
                            if constexpr (Md::kRebase) rebase_to_left<false, W, RT>(prev, diag, left, B);
                            V x[RT];
                            load_x<RT>(xs, p, x);
                            if (bot == RT - 1) {
                                // the query's last row is a tile's last row (RT divides n):
                                // the plain tile, then the minimum over that row for the one
                                // lane that holds it; updating the minimum inside every
                                // cell of the tile measured 17-21% of the whole fill
                                tile_step<Md, W, RT, false, PRUNE>(prev, A, y, x, diag, left, 0, B, base, M, best, best_col, gap);
                                if (p == lastt) bottom_min_prev<Md, W>(prev, B, base, M, best, best_col);
                            } else if (__any_sync(__activemask(), p == lastt)) {
                                // the last row inside a tile: update the minimum in the cells,
                                // only on the steps where some lane of the warp holds that tile
                                tile_step<Md, W, RT, true, PRUNE>(prev, A, y, x, diag, left, p == lastt ? bot : -1, B,
                                                                  base, M, best, best_col, gap);
                            } else {
                                tile_step<Md, W, RT, false, PRUNE>(prev, A, y, x, diag, left, 0, B, base, M, best, best_col, gap);
                            }
                            diag = left[RT - 1];
                            if (lane == 31) {
                                E e;
#pragma unroll
                                for (int rr = 0; rr < RT; ++rr) e.v[rr] = rr < RT - 1 ? A[rr][W - 1] : prev[W - 1];
                                e.b = B;
                                if (warp < P - 1)
                                    ring_out[t & (kRing - 1)] = e;
                                else
                                    colbuf[p] = e;
                            }
                        }
                        if (++p == Pp) {
                            p = 0;
                            ++s;
                        }
                        if (P == 1) __syncwarp();
                    }
                }
                if constexpr (CKPT) {
                    // the wavefront as this segment leaves it (the state at the
                    // start of step tend, before a rebase due there), if this thread
                    // has computed a tile (p == 0 of a later sweep still holds the
                    // previous sweep's last tile when the period has no idle steps)
                    const int tend = t0 + ue;
                    const int c1 = tend / ks;
                    if (tend - c1 * ks == 0 && tend < total &&
                        ((p >= 1 && p <= nt && s < nsw) || (p == 0 && s >= 1 && Pp == nt))) {
                        float4* f4 = reinterpret_cast<float4*>(frq + static_cast<int64_t>(c1) * L * (W + EREC)) +
                                     threadIdx.x;
#pragma unroll
                        for (int k = 0; k < W / 4; ++k)
                            __stcs(f4 + k * L, make_float4(prev[4 * k], prev[4 * k + 1], prev[4 * k + 2], prev[4 * k + 3]));
                        if constexpr (RT == 2) {
                            __stcs(f4 + (W / 4) * L, make_float4(A[0][W - 1], diag, B, 0.f));
                        } else if constexpr (RT == 8) {
                            __stcs(f4 + (W / 4) * L, make_float4(A[0][W - 1], A[1][W - 1], A[2][W - 1], A[3][W - 1]));
                            __stcs(f4 + (W / 4 + 1) * L, make_float4(A[4][W - 1], A[5][W - 1], A[6][W - 1], diag));
                            __stcs(f4 + (W / 4 + 2) * L, make_float4(B, 0.f, 0.f, 0.f));
                        } else {
                            __stcs(f4 + (W / 4) * L, make_float4(A[0][W - 1], A[1][W - 1], A[2][W - 1], diag));
                            __stcs(f4 + (W / 4 + 1) * L, make_float4(B, 0.f, 0.f, 0.f));
                        }
                    }
                }
            }  // segments
            __syncthreads();
        }

        if constexpr (Md::kPair) {
            // each half's lexicographic (value, column) minimum over the CTA;
            // a last row that overflowed to +inf everywhere ends at column 0,
            // the smallest column attaining the minimum
            float b0 = __low2float(best), b1 = __high2float(best);
            int c0 = best_col.x, c1 = best_col.y;
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) {
                const float o0 = __shfl_down_sync(0xffffffffu, b0, off), o1 = __shfl_down_sync(0xffffffffu, b1, off);
                const int k0 = __shfl_down_sync(0xffffffffu, c0, off), k1 = __shfl_down_sync(0xffffffffu, c1, off);
                if (o0 < b0 || (o0 == b0 && k0 < c0)) {
                    b0 = o0;
                    c0 = k0;
                }
                if (o1 < b1 || (o1 == b1 && k1 < c1)) {
                    b1 = o1;
                    c1 = k1;
                }
            }
            float* red_f = reinterpret_cast<float*>(red_v);  // [P] floats, then the columns [2P]
            if (lane == 0) {
                red_f[warp] = b0;
                red_i[2 * warp] = c0;
                red_i[2 * warp + 1] = c1;
            }
            __syncthreads();
            float* red_f1 = reinterpret_cast<float*>(red_i + 2 * P);  // [P]
            if (lane == 0) red_f1[warp] = b1;
            __syncthreads();
            if (threadIdx.x == 0) {
                float v0 = red_f[0], v1 = red_f1[0];
                int e0 = red_i[0], e1 = red_i[1];
                for (int w = 1; w < P; ++w) {
                    if (red_f[w] < v0 || (red_f[w] == v0 && red_i[2 * w] < e0)) {
                        v0 = red_f[w];
                        e0 = red_i[2 * w];
                    }
                    if (red_f1[w] < v1 || (red_f1[w] == v1 && red_i[2 * w + 1] < e1)) {
                        v1 = red_f1[w];
                        e1 = red_i[2 * w + 1];
                    }
                }
                static_cast<float*>(a.cost)[q] = v0;
                a.end[q] = e0 == INT_MAX ? 0 : e0;
                if (qb != q) {
                    static_cast<float*>(a.cost)[qb] = v1;
                    a.end[qb] = e1 == INT_MAX ? 0 : e1;
                }
            }
            __syncthreads();
        } else {
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
            if constexpr (PRUNE) {
                // every cell of the last row pruned away: no path, no end column
                if (bv == INF) {
                    bv = Md::empty_cost();
                    bc = -1;
                }
            }
            static_cast<V*>(a.cost)[q] = bv;
            a.end[q] = bc;
            if constexpr (CKPT) {
                a.ck_cost[q - a.q0] = bv;
                a.ck_end[q - a.q0] = bc;
            }
        }
        __syncthreads();
        }  // scalar modes
    }
}

template <typename Tin, int W, int RT, bool CKPT, bool PRUNE = false>
struct Inst {
    static cudaError_t launch(const FwdPlan& plan, const FwdArgs& a, cudaStream_t s)
    {
        auto k = fwd_chain_kernel<Tin, W, RT, CKPT, PRUNE>;
        if (plan.smem < 0 || plan.smem > kMaxSmemBytes) return cudaErrorInvalidValue;
        const int smem = static_cast<int>(plan.smem);
        if (smem > 48 * 1024) {
            cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
            if (e != cudaSuccess) return e;
        }
        k<<<plan.grid, plan.block, smem, s>>>(a);
        return cudaGetLastError();
    }
    static int occupancy(int block, int64_t smem64)
    {
        if (smem64 < 0 || smem64 > kMaxSmemBytes) return 0;
        const int smem = static_cast<int>(smem64);
        int n = 0;
        auto k = fwd_chain_kernel<Tin, W, RT, CKPT, PRUNE>;
        if (smem > 48 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, block, smem) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        return n;
    }
};

}  // namespace
}  // namespace sdtw
