// Backward sDTW: the gradient of each query's cost along its warp path.
//
// The path is the paper's walk-back (Section 2): from the end cell (n-1, e)
// step to the neighbour (i-1,j-1), (i,j-1) or (i-1,j) with the smallest
// accumulated cost, exact ties to the first of that list, column 0 upwards,
// stopping at row 0.  Along the path the cost is a sum of (x_i - y_j)^2, so
//   d cost / d x_i = sum over the path's cells in row i    of  2 (x_i - y_j)
//   d cost / d y_j = sum over the path's cells in column j of -2 (x_i - y_j).
//
// The n x M matrix is never stored.  The forward pass left absolute D values
// along every K-th column and every R-th row (its checkpoints), so the matrix
// splits into R x K tiles whose top row and left column are known.  The walk
// proceeds tile by tile, one warp per query:
//   * the warp recomputes the tile's rows down to the current cell from the
//     checkpoint row above and the checkpoint column on the left (FP32
//     relative to per-lane integer bases, rebased every kChunk rows as in the
//     forward), with the same three-input minimum as the forward on the
//     dependency chain; each cell's walk-back choice (two bits) is derived
//     off the chain by equality with that minimum (diagonal first, then left,
//     then up -- the tie order of the walk-back);
//   * the walk itself is cooperative: the 32 lanes read 32 cells of the
//     current row at once and a ballot finds where the path leaves the row,
//     so a horizontal run of the path costs one step per 32 cells; the row's
//     gradient is a warp sum and finished columns are written in parallel.
// Paths that stretch far along the reference (a query rescaled by its own
// z-normalisation typically moves several columns per row) cross many tiles,
// so tiles are wider (K = 256) than tall (R = 64 by default).
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
struct DirWord<8> { using T = uint16_t; };

constexpr int kDiag = 0, kLeft = 1, kUp = 2, kOutside = 3;

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    return v;
}

template <int WB>
__global__ void __launch_bounds__(32) bwd_tile_kernel(const BwdArgs a)
{
    using DW = typename DirWord<WB>::T;
    constexpr int KC = 32 * WB;  // tile columns
    const int R = a.R;           // tile rows
    const int lane = threadIdx.x;
    const int N = a.N;
    const int M = static_cast<int>(a.M);
    const int ql = blockIdx.x;  // query within this launch
    const int q = a.q0 + ql;    // query within the batch
    const float INF = __int_as_float(0x7f800000);

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* xs = reinterpret_cast<float*>(smem_raw);  // [N]  query samples
    float* ys = xs + N;                              // [KC] reference samples of the tile
    float* top = ys + KC;                            // [KC] D of the row above the tile (absolute)
    float* lcol = top + KC;                          // [R]  D of the column left of the tile (absolute)
    DW* dirs = reinterpret_cast<DW*>(lcol + R);      // [R][32] walk-back choices, 2 bits per cell

    const int64_t first_start = a.offsets ? a.offsets[a.q0] : static_cast<int64_t>(a.q0) * N;
    int64_t start;
    int n;
    if (a.offsets) {
        start = a.offsets[q];
        const int64_t stop = a.offsets[q + 1];
        const int64_t len = stop - start;
        if (start < first_start || len < 0 || len > N || stop > a.offsets[a.B_total] ||
            (stop - first_start) > a.ckpt_rows) {
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
    const float g2 = 2.f * a.grad_cost[q];
    const float* x = a.queries + start;
    for (int i = lane; i < n; i += 32) xs[i] = x[i];
    const float* cck = a.ckpt + (start - first_start) * a.nblk;      // [nblk][n]
    const float* rck = a.rowck + ((start - first_start) / R) * a.M;  // [n/R][M]
    float* gyq = a.gyq + static_cast<int64_t>(ql) * a.M;
    float* gq = a.grad_queries + start;
    int32_t* path = a.path ? a.path + 2 * start : nullptr;

    // walk state, identical in every lane: current cell (wi, wj), the
    // gradient of row wi and of column wj accumulated so far
    int wi = n - 1, wj = static_cast<int>(e64);
    float ax = 0.f, ay = 0.f;
    bool done = false;
    if (lane == 0 && path) path[2 * wi + 1] = wj;

    while (!done) {
        const int rb = wi / R, cb = wj / KC;
        const int r0 = rb * R, c0 = cb * KC;
        const int rows = wi - r0 + 1;  // recompute rows r0..wi of the tile

        __syncwarp();
        for (int k = lane; k < KC; k += 32) {
            const int col = c0 + k;
            ys[k] = col < M ? a.ref[col] : 0.f;
            top[k] = (rb > 0 && col < M) ? rck[static_cast<int64_t>(rb - 1) * a.M + col] : 0.f;
        }
        for (int k = lane; k < rows; k += 32)
            lcol[k] = cb > 0 ? cck[static_cast<int64_t>(cb - 1) * n + r0 + k] : INF;
        // D(r0-1, c0-1): the virtual row -1 is zero, the virtual column -1 infinite
        const float corner = rb == 0 ? 0.f : (cb > 0 ? rck[static_cast<int64_t>(rb - 1) * a.M + c0 - 1] : INF);
        __syncwarp();

        // ---- recompute rows r0..wi of the tile, recording walk-back choices
        {
            float y[WB], D[WB];
            float B = floorf(top[lane * WB]);  // per-lane base: absolute D = B + D'
#pragma unroll
            for (int k = 0; k < WB; ++k) {
                y[k] = ys[lane * WB + k];
                D[k] = top[lane * WB + k] - B;
            }
            float diag = (lane == 0 ? corner : top[lane * WB - 1]) - B;
            const int steps = rows + 31;
            for (int t = 0; t < steps; ++t) {
                if (t > 0 && (t & (kChunk - 1)) == 0) {
                    const float bn = floorf(B + D[0]);
                    const float dl = bn - B;
#pragma unroll
                    for (int k = 0; k < WB; ++k) D[k] -= dl;
                    diag -= dl;
                    B = bn;
                }
                float recv = __shfl_up_sync(0xffffffffu, D[WB - 1], 1);
                float rbs = __shfl_up_sync(0xffffffffu, B, 1);
                const int r = t - lane;
                const bool act = static_cast<unsigned>(r) < static_cast<unsigned>(rows);
                if (lane == 0) {
                    recv = act ? lcol[r] : INF;  // absolute values
                    rbs = 0.f;
                }
                if (act) {
                    const float xv = xs[r0 + r];
                    float left = recv + (rbs - B);
                    const float conv = left;
                    uint32_t code = 0;
#pragma unroll
                    for (int k = 0; k < WB; ++k) {
                        const float up = D[k];
                        const float v = min3_f32(up, diag, left);
                        const uint32_t c = v == diag ? kDiag : (v == left ? kLeft : kUp);
                        const float d = xv - y[k];
                        const float nv = fmaf(d, d, v);
                        code |= c << (2 * k);
                        diag = up;
                        left = nv;
                        D[k] = nv;
                    }
                    diag = conv;
                    dirs[r * 32 + lane] = static_cast<DW>(code);
                }
            }
        }
        __syncwarp();

        // ---- follow the path through the tile, 32 cells of a row at a time
        for (;;) {
            const float xi = xs[wi];
            if (wi == 0) {
                // the path starts here: only this cell of row 0 is on it
                const float c = g2 * (xi - ys[wj - c0]);
                if (lane == 0) {
                    gq[0] = ax + c;
                    gyq[wj] = ay - c;
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
                if (jk == 0) {
                    code = kUp;
                } else {
                    const int cc = jk - c0;
                    code = (dirs[(wi - r0) * 32 + cc / WB] >> (2 * (cc % WB))) & 3;
                }
            }
            const unsigned stop = __ballot_sync(0xffffffffu, code != kLeft);
            const int f = stop ? __ffs(stop) - 1 : 32;        // first lane whose cell leaves the row
            const int fcode = f < 32 ? __shfl_sync(0xffffffffu, code, f) : kLeft;
            const int last = fcode == kOutside ? f - 1 : (f < 32 ? f : 31);  // last lane on the path
            const bool on = lane <= last;
            const float c = on ? g2 * (xi - ys[jk - c0]) : 0.f;
            ax += warp_sum(c);
            // column of lane k: finished unless the path goes up from it
            float vy = -c;
            if (lane == 0) vy += ay;
            const int lcode = (lane == last && fcode != kOutside && f < 32) ? fcode : kLeft;
            if (on && lcode != kUp) gyq[jk] = vy;
            const float vlast = __shfl_sync(0xffffffffu, vy, last);
            ay = (f < 32 && fcode == kUp) ? vlast : 0.f;
            if (f < 32 && fcode != kOutside) {
                // the row ends at (wi, wj - last); move up or diagonally
                const int jl = wj - last;
                if (lane == 0) {
                    gq[wi] = ax;
                    if (path) path[2 * wi] = jl;
                }
                ax = 0.f;
                wi -= 1;
                wj = fcode == kDiag ? jl - 1 : jl;
                if (lane == 0 && path) path[2 * wi + 1] = wj;
            } else {
                wj -= last + 1;  // the run continues to the left
            }
            if (wj < c0 || wi < r0) break;
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
    const int smem = bwd_smem_bytes(a.N, 32 * WB, a.R);
    auto k = bwd_tile_kernel<WB>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    k<<<a.B, 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool bwd_stride_supported(int K) { return K == 64 || K == 128 || K == 256; }

// at least 64: the forward stages a checkpoint row per warp and needs the
// 32 lanes' captures of one row to finish before lane 0 reaches the next
bool bwd_row_stride_supported(int R) { return R == 64 || R == 128 || R == 256; }

int bwd_smem_bytes(int N, int K, int R)
{
    const int word = K == 256 ? 2 : 1;
    return 4 * (N + 2 * K + R) + R * 32 * word;
}

size_t ckpt_floats_per_query(int64_t N, int64_t M, int K, int R)
{
    // a column every K columns (N values each) and a row every R rows (M values each)
    return static_cast<size_t>(N) * static_cast<size_t>(M / K) + static_cast<size_t>(N / R) * static_cast<size_t>(M);
}

cudaError_t launch_backward_walk(const BwdArgs& a, cudaStream_t s)
{
    if (a.B <= 0) return cudaSuccess;
    switch (a.K) {
    case 64: return launch_walk_wb<2>(a, s);
    case 128: return launch_walk_wb<4>(a, s);
    case 256: return launch_walk_wb<8>(a, s);
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
