// Backward sDTW: the gradient of each query's cost along its warp path.
//
// The path is the paper's walk-back (Section 2): from the end cell (n-1, e)
// step to the neighbour (i-1,j-1), (i,j-1) or (i-1,j) with the smallest
// accumulated cost, exact ties to the first of that list, column 0 upwards,
// stopping at row 0.  Along the path the cost is a sum of (x_i - y_j)^2, so
//   d cost / d x_i = sum over the path's cells in row i    of  2 (x_i - y_j)
//   d cost / d y_j = sum over the path's cells in column j of -2 (x_i - y_j).
//
// The n x M matrix is never stored.  The checkpointing forward left, at the
// end of every chunk of kChunk steps, its wavefront (each thread's latest
// row, the right-hand cells of its tile's other rows, its diagonal input and
// its integer base: an anti-diagonal staircase of rows, stored before the
// next chunk's rebase, which is redone here), and the left inputs of every
// strip that starts a K-column window (K = 8 W).  The cells that the
// eight strips of one window computed during one chunk form a band, a
// parallelogram (each strip one tile higher than its left neighbour).  The
// walk proceeds band by band, one warp per query:
//   * the warp recomputes the band's rows down to the current cell from the
//     chunk's wavefront and the window's boundary column, with the forward's
//     own operations in the forward's own bases (four lanes per strip, W/4
//     columns each, lane l one row behind lane l-1), so every value is the
//     forward's bit for bit; each cell's walk-back choice (two bits) is read
//     off the minimum by equality (diagonal first, then left, then up -- the
//     tie order of the walk-back);
//   * the walk itself is cooperative: the 32 lanes read 32 cells of the
//     current row at once and a ballot finds where the path leaves the row,
//     so a horizontal run of the path costs one step per 32 cells; the row's
//     gradient is a warp sum and finished columns are written in parallel.
// At the first band the recomputed end cell must equal the forward's cost
// exactly; a mismatch sets a status bit.
//
// Per-query reference gradients go to rows of a scratch buffer, only over the
// path's column span; a second kernel sums them over queries in query order,
// so grad_ref is deterministic.
#include <cuda_runtime.h>

#include <cstdint>

#include "sdtw_cell.cuh"
#include "sdtw_internal.h"

namespace sdtw {
namespace {

template <int WB>
struct DirWord;
template <>
struct DirWord<2> { using T = uint8_t; };
template <>
struct DirWord<4> { using T = uint8_t; };
template <>
struct DirWord<5> { using T = uint16_t; };
template <>
struct DirWord<6> { using T = uint16_t; };
template <>
struct DirWord<7> { using T = uint16_t; };
template <>
struct DirWord<8> { using T = uint16_t; };

constexpr int kDiag = 0, kLeft = 1, kUp = 2, kOutside = 3;

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

template <int WB>
__global__ void __launch_bounds__(32) bwd_band_kernel(const BwdArgs a)
{
    using DW = typename DirWord<WB>::T;
    constexpr int W = 4 * WB;    // forward segment width: four lanes per strip
    constexpr int KW = 32 * WB;  // window width K = 8 W
    const int RT = a.RT;
    const int L = 32 * a.P;
    const int S = L * W;
    const int lane = threadIdx.x;
    const int N = a.N;
    const int M = static_cast<int>(a.M);
    const int ql = blockIdx.x;  // query within this launch
    const int q = a.q0 + ql;    // query within the batch
    const float INF = __int_as_float(0x7f800000);

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* xs = reinterpret_cast<float*>(smem_raw);  // [N] query samples
    float* ys = xs + N;                              // [KW] reference samples of the window
    float* lcol = ys + KW;                           // [RT*kChunk] the window's boundary column
    DW* dirs = reinterpret_cast<DW*>(lcol + RT * kChunk);  // [2*steps][32] walk-back choices (two masks)

    int64_t start;
    int n;
    if (a.offsets) {
        start = a.offsets[q];
        const int64_t stop = a.offsets[q + 1];
        const int64_t len = stop - start;
        if (start < 0 || len < 0 || len > N || stop > a.offsets[a.B_total]) {
            if (lane == 0) {
                atomicOr(a.status, kStatusBadLength);
                a.span[2 * ql] = 0;
                a.span[2 * ql + 1] = -1;
            }
            return;
        }
        n = static_cast<int>(len);
    } else {
        start = static_cast<int64_t>(q) * N;
        n = N;
    }
    if (n == 0) {
        if (lane == 0) {
            a.span[2 * ql] = 0;
            a.span[2 * ql + 1] = -1;
        }
        return;
    }
    const int64_t e64 = a.end[q];
    if (e64 < 0 || e64 >= a.M) {
        if (lane == 0) {
            atomicOr(a.status, kStatusBadEnd);
            a.span[2 * ql] = 0;
            a.span[2 * ql + 1] = -1;
        }
        return;
    }
    const bool grads = a.grad_queries != nullptr;  // false: the path only
    const float g2 = grads ? 2.f * a.grad_cost[q] : 0.f;
    const float* x = a.queries + start;
    for (int i = lane; i < n; i += 32) xs[i] = x[i];
    float* gyq = a.gyq + static_cast<int64_t>(ql) * a.M;
    float* gq = grads ? a.grad_queries + start : nullptr;
    int32_t* path = a.path ? a.path + 2 * start : nullptr;

    // the forward's schedule for this query (sdtw_forward.cu)
    const int lag_last = (a.P - 1) * (32 + kChunk) + 31;
    const int nt = (n + RT - 1) / RT;
    const int Pp = max(nt, lag_last + kChunk);
    const int erec = fwd_record_floats(RT);
    const float* frq = a.fr + static_cast<int64_t>(ql) * a.fr_slot;
    const float* ckq = a.colck + static_cast<int64_t>(ql) * a.ck_slot;

    // walk state, identical in every lane: current cell (wi, wj), the
    // gradient of row wi and of column wj accumulated so far
    int wi = n - 1, wj = static_cast<int>(e64);
    float ax = 0.f, ay = 0.f;
    bool done = false, first = true;
    if (lane == 0 && path) path[2 * wi + 1] = wj;

    const int d = lane >> 2;    // this lane's strip in the window
    const int sub = lane & 3;   // and its quarter of the strip

    // every band holds at least the walk's current cell, so a path of at most
    // n + M cells needs at most that many bands
    for (int64_t guard = 0; !done; ++guard) {
        // ---- the band holding (wi, wj): window b, chunk c
        const int b = wj / KW, c0 = b * KW, s = c0 / S;
        const int tau0 = (c0 - s * S) / W;   // forward thread of the window's first strip
        const int lag0 = (tau0 >> 5) * (32 + kChunk) + (tau0 & 31);  // strips of a window share a warp
        const int dj = (wj - c0) / W;
        const int c = (wi / RT + lag0 + dj + s * Pp) / kChunk;
        const int ps0 = c * kChunk - lag0 - s * Pp;  // strip 0's tile at the chunk start
        const int rtop = RT * (ps0 - 7);             // lane l handles row r at step r - rtop + l
        const int ps = ps0 - d;                      // this lane's strip
        const int rf = RT * max(0, ps);              // its rows in the band: [rf, re)
        const int re = min(n, RT * min(nt, ps + kChunk));
        const int rf_left = RT * max(0, ps + 1);     // the strip on the left starts here
        const int rf0 = RT * max(0, ps0);
        const int re0 = min(min(n, RT * min(nt, ps0 + kChunk)), wi + 1);
        if (guard > static_cast<int64_t>(n) + M || wi < RT * max(0, ps0 - dj) ||
            wi >= min(n, RT * min(nt, ps0 - dj + kChunk))) {
            // the current cell is not in its band: report and give up on this query
            if (lane == 0) {
                atomicOr(a.status, kStatusReplay);
                a.span[2 * ql] = 0;
                a.span[2 * ql + 1] = -1;
            }
            return;
        }

        __syncwarp();
        for (int k = lane; k < KW; k += 32) ys[k] = c0 + k < M ? a.ref[c0 + k] : 0.f;
        if (b > 0)
            for (int k = lane; k < re0 - rf0; k += 32) lcol[k] = ckq[static_cast<int64_t>(b - 1) * ck_rows(N) + rf0 + k];

        // ---- the lane's starting state: the chunk's wavefront, or the virtual
        // zero row -1 for a strip that starts its sweep inside the chunk
        const float* frc = frq + static_cast<int64_t>(c) * L * (W + erec);
        const int tau = tau0 + d;
        auto fr_at = [&](int j, int th) { return frc[((j >> 2) * L + th) * 4 + (j & 3)]; };
        auto rec_at = [&](int e, int th) { return frc[(((W >> 2) + (e >> 2)) * L + th) * 4 + (e & 3)]; };
        // the forward stored its state before the chunk's rebase: redo it
        // (new base: the integer part of the strip's first column)
        auto rebase = [&](int th, float& bn, float& dl) {
            const float b0 = rec_at(RT == 2 ? 2 : 4, th);
            bn = floorf(b0 + fr_at(0, th));
            dl = bn - b0;
        };
        float D[WB], y[WB];
        float Bl = 0.f, dg = 0.f;
        if (ps >= 1 && ps <= nt) {
            float dl;
            rebase(tau, Bl, dl);
#pragma unroll
            for (int k = 0; k < WB; ++k) D[k] = fr_at(sub * WB + k, tau) - dl;
            dg = (sub == 0 ? rec_at(RT - 1, tau) : fr_at(sub * WB - 1, tau)) - dl;
        } else {
#pragma unroll
            for (int k = 0; k < WB; ++k) D[k] = 0.f;
        }
        // the first lane of strips 1..7: the left strip's last tile before the
        // band (rows RT*ps .. RT*ps + RT-1, its right-hand cells) and its base
        float e0 = 0.f, e1 = 0.f, e2 = 0.f, e3 = 0.f, dd = 0.f;
        if (sub == 0 && d >= 1) {
            float Bsrc = 0.f;
            if (ps + 1 >= 1 && ps + 1 <= nt) {
                float dl;
                rebase(tau - 1, Bsrc, dl);
                e0 = rec_at(0, tau - 1) - dl;
                if (RT == 2) {
                    e1 = fr_at(W - 1, tau - 1) - dl;
                } else {
                    e1 = rec_at(1, tau - 1) - dl;
                    e2 = rec_at(2, tau - 1) - dl;
                    e3 = fr_at(W - 1, tau - 1) - dl;
                }
            }
            dd = Bsrc - Bl;
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < WB; ++k) y[k] = ys[lane * WB + k];

        // ---- recompute the band's rows down to row wi, recording choices.
        // Lane l handles rows r and r+1 (r - rtop even) at step (r - rtop)/2 + l:
        // the two rows are two dependency chains, row r+1 one column behind.
        const int steps = (wi - rtop) / 2 + 32;
        const int hi = min(re, wi + 1);  // this lane's rows end here
        float lastA = 0.f, lastB = 0.f;  // right-hand cells of the lane's previous row pair
        for (int sg = 0; sg < steps; ++sg) {
            const float recvA = __shfl_up_sync(0xffffffffu, lastA, 1);
            const float recvB = __shfl_up_sync(0xffffffffu, lastB, 1);
            const int r = rtop + 2 * (sg - lane);
            if (r >= rf && r < hi) {
                const bool vb = r + 1 < hi;  // row r+1 is in the band (else: last row)
                float lA, lB;
                if (sub != 0) {
                    lA = recvA;  // same strip, same base
                    lB = recvB;
                } else if (d == 0) {
                    lA = b == 0 ? INF : lcol[r - rf0];  // already in this strip's base
                    lB = (b == 0 || !vb) ? INF : lcol[r + 1 - rf0];
                } else {
                    float vA = recvA, vB = recvB;
                    if (r < rf_left) {
                        // the left strip's last tile before the band (rows RT*ps ..)
                        const int e = r - RT * ps;
                        vA = e == 0 ? e0 : e2;
                        vB = e == 0 ? e1 : e3;
                    }
                    lA = vA + dd;  // into this strip's base, as the forward converts
                    lB = vB + dd;
                }
                const float xA = xs[r];
                const float xB = vb ? xs[r + 1] : 0.f;
                const float convA = lA, convB = lB;
                float dgA = dg, dgB = lA;
                // walk-back choices as two masks per row: bit k of nd is set
                // unless the minimum is the diagonal; bit k of nu is set when it
                // is neither the diagonal nor the left cell (the cell above)
                uint32_t ndA = 0, nuA = 0, ndB = 0, nuB = 0;
#pragma unroll
                for (int k = 0; k < WB; ++k) {
                    const float up = D[k];
                    const float vA = min3_f32(up, dgA, lA);
                    if (vA != dgA) {
                        ndA |= 1u << k;
                        if (vA != lA) nuA |= 1u << k;
                    }
                    const float tA = xA - y[k];
                    const float nA = fmaf(tA, tA, vA);
                    dgA = up;
                    lA = nA;
                    const float vB = min3_f32(nA, dgB, lB);
                    if (vB != dgB) {
                        ndB |= 1u << k;
                        if (vB != lB) nuB |= 1u << k;
                    }
                    const float tB = xB - y[k];
                    const float nB = fmaf(tB, tB, vB);
                    dgB = nA;
                    lB = nB;
                    D[k] = vb ? nB : nA;
                }
                lastA = lA;
                lastB = lB;
                dg = vb ? convB : convA;
                dirs[(2 * sg) * 32 + lane] = static_cast<DW>(ndA | (nuA << WB));
                dirs[(2 * sg + 1) * 32 + lane] = static_cast<DW>(ndB | (nuB << WB));
            }
        }

        if (first) {
            // the recomputed end cell against the forward's cost (when the
            // walk starts at the forward's own end)
            const int lj = (wj - c0) / WB, kj = (wj - c0) - lj * WB;
            float v = 0.f;
#pragma unroll
            for (int k = 0; k < WB; ++k)
                if (k == kj) v = D[k];
            v = __shfl_sync(0xffffffffu, v + Bl, lj);
            if (lane == 0 && a.ck_end[ql] == e64 && v != a.ck_cost[ql]) atomicOr(a.status, kStatusReplay);
            first = false;
        }
        __syncwarp();

        // ---- follow the path through the band, 32 cells of a row at a time
        for (;;) {
            const float xi = xs[wi];
            if (wi == 0) {
                // the path starts here: only this cell of row 0 is on it
                const float cg = g2 * (xi - ys[wj - c0]);
                if (lane == 0) {
                    if (grads) {
                        gq[0] = ax + cg;
                        gyq[wj] = ay - cg;
                    }
                    if (path) path[0] = wj;
                    a.span[2 * ql] = wj;
                    a.span[2 * ql + 1] = e64;
                }
                done = true;
                break;
            }
            const int jk = wj - lane;
            int code = kOutside;
            if (jk >= c0) {
                const int cc = jk - c0, lam = cc / WB;
                if (wi >= RT * max(0, ps0 - (lam >> 2))) {  // row wi is in the band in that strip
                    if (jk == 0) {
                        code = kUp;
                    } else {
                        const uint32_t m = dirs[(wi - rtop + 2 * lam) * 32 + lam] >> (cc - lam * WB);
                        code = !(m & 1u) ? kDiag : ((m >> WB) & 1u) ? kUp : kLeft;
                    }
                }
            }
            const unsigned stop = __ballot_sync(0xffffffffu, code != kLeft);
            const int f = stop ? __ffs(stop) - 1 : 32;        // first lane whose cell leaves the row
            const int fcode = f < 32 ? __shfl_sync(0xffffffffu, code, f) : kLeft;
            const int last = fcode == kOutside ? f - 1 : (f < 32 ? f : 31);  // last lane on the path
            const bool on = lane <= last;
            const float cg = on ? g2 * (xi - ys[jk - c0]) : 0.f;
            ax += warp_sum(cg);
            // column of lane k: finished unless the path goes up from it
            float vy = -cg;
            if (lane == 0) vy += ay;
            const int lcode = (lane == last && fcode != kOutside && f < 32) ? fcode : kLeft;
            if (grads && on && lcode != kUp) gyq[jk] = vy;
            const float vlast = __shfl_sync(0xffffffffu, vy, last);
            ay = (f < 32 && fcode == kUp) ? vlast : 0.f;
            if (f < 32 && fcode != kOutside) {
                // the row ends at (wi, wj - last); move up or diagonally
                const int jl = wj - last;
                if (lane == 0) {
                    if (grads) gq[wi] = ax;
                    if (path) path[2 * wi] = jl;
                }
                ax = 0.f;
                wi -= 1;
                wj = fcode == kDiag ? jl - 1 : jl;
                if (lane == 0 && path) path[2 * wi + 1] = wj;
            } else {
                wj -= last + 1;  // the run continues to the left
            }
            if (wj < c0 || wi < RT * max(0, ps0 - (wj - c0) / W)) break;  // left the band
        }
    }
}

// grad_ref[j] (+)= sum over queries q (in order) whose path spans column j of gyq[q][j]
__global__ void grad_ref_reduce_kernel(const float* __restrict__ gyq, const int64_t* __restrict__ span,
                                       int32_t B, int64_t M, bool accumulate, float* __restrict__ grad_ref)
{
    const int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (j >= M) return;
    float acc = accumulate ? grad_ref[j] : 0.f;
    for (int q = 0; q < B; ++q) {
        const int64_t lo = span[2 * q], hi = span[2 * q + 1];
        if (j >= lo && j <= hi) acc += gyq[static_cast<int64_t>(q) * M + j];
    }
    grad_ref[j] = acc;
}

template <int WB>
cudaError_t launch_walk_wb(const BwdArgs& a, cudaStream_t s)
{
    const int smem = bwd_smem_bytes(a.N, 4 * WB, a.RT);
    auto k = bwd_band_kernel<WB>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    k<<<a.B, 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool bwd_width_supported(int W) { return W == 8 || W == 16 || W == 20 || W == 24 || W == 28 || W == 32; }

int bwd_smem_bytes(int N, int W, int RT)
{
    // query samples, the window's samples and boundary column, and the
    // choices of up to RT*kChunk + 7*RT + 64 rows of 32 lanes (W/2 bits each)
    const int word = W <= 16 ? 1 : 2;
    return 4 * (N + 8 * W + RT * kChunk) + (RT * kChunk + 7 * RT + 64) * 32 * word;
}

cudaError_t launch_backward_walk(const BwdArgs& a, cudaStream_t s)
{
    if (a.B <= 0) return cudaSuccess;
    if (a.K != 8 * a.W || (a.RT != 2 && a.RT != 4)) return cudaErrorInvalidValue;
    switch (a.W) {
    case 8: return launch_walk_wb<2>(a, s);
    case 16: return launch_walk_wb<4>(a, s);
    case 20: return launch_walk_wb<5>(a, s);
    case 24: return launch_walk_wb<6>(a, s);
    case 28: return launch_walk_wb<7>(a, s);
    case 32: return launch_walk_wb<8>(a, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_grad_ref_reduce(const float* gyq, const int64_t* span, int32_t B, int64_t M,
                                   bool accumulate, float* grad_ref, cudaStream_t s)
{
    if (M <= 0) return cudaSuccess;
    const int threads = 256;
    const int64_t blocks = (M + threads - 1) / threads;
    grad_ref_reduce_kernel<<<static_cast<unsigned>(blocks), threads, 0, s>>>(gyq, span, B, M, accumulate, grad_ref);
    return cudaGetLastError();
}

}  // namespace sdtw
