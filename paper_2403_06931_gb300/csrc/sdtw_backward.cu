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
// along every K-th column and every K-th row (its checkpoints), so the matrix
// splits into K x K tiles whose top row and left column are known.  The walk
// proceeds tile by tile: one warp recomputes the rows of the current tile up
// to the current cell from the checkpoint row above and the checkpoint column
// on the left (FP32 relative to per-lane integer bases, rebased every kChunk
// rows as in the forward), records for each cell which neighbour the
// walk-back would take (two bits), and lane 0 then follows the path through
// the tile, accumulating the gradient, until it leaves the tile upwards or to
// the left.  A path visits about (its column span + n) / K tiles, each
// recomputed in K + 31 steps.
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

template <int WB>
__global__ void __launch_bounds__(32) bwd_tile_kernel(const BwdArgs a)
{
    using DW = typename DirWord<WB>::T;
    constexpr int K = 32 * WB;  // tile side (rows and columns)
    const int lane = threadIdx.x;
    const int N = a.N;
    const int M = static_cast<int>(a.M);
    const int ql = blockIdx.x;  // query within this launch
    const int q = a.q0 + ql;    // query within the batch
    const float INF = __int_as_float(0x7f800000);

    extern __shared__ __align__(16) unsigned char smem_raw[];
    float* xs = reinterpret_cast<float*>(smem_raw);  // [N]  query samples
    float* ys = xs + N;                              // [K]  reference samples of the tile
    float* top = ys + K;                             // [K]  D of the row above the tile (absolute)
    float* lcol = top + K;                           // [K]  D of the column left of the tile (absolute)
    DW* dirs = reinterpret_cast<DW*>(lcol + K);      // [K][32] walk-back choices, 2 bits per cell

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
    const float g = a.grad_cost[q];
    const float* x = a.queries + start;
    for (int i = lane; i < n; i += 32) xs[i] = x[i];
    const float* cck = a.ckpt + (start - first_start) * a.nblk;          // [nblk][n]
    const float* rck = a.rowck + ((start - first_start) / K) * a.M;      // [n/K][M]
    float* gyq = a.gyq + static_cast<int64_t>(ql) * a.M;
    float* gq = a.grad_queries + start;
    int32_t* path = a.path ? a.path + 2 * start : nullptr;

    // walk state (meaningful in lane 0; broadcast after each tile)
    int wi = n - 1, wj = static_cast<int>(e64);
    float ax = 0.f, ay = 0.f;
    bool done = false;
    if (lane == 0 && path) path[2 * wi + 1] = wj;

    while (!done) {
        const int rb = wi / K, cb = wj / K;
        const int r0 = rb * K, c0 = cb * K;
        const int rows = wi - r0 + 1;  // recompute rows r0..wi of the tile

        __syncwarp();
        for (int k = lane; k < K; k += 32) {
            const int col = c0 + k;
            ys[k] = col < M ? a.ref[col] : 0.f;
            top[k] = (rb > 0 && col < M) ? rck[static_cast<int64_t>(rb - 1) * a.M + col] : 0.f;
            lcol[k] = (cb > 0 && k < rows) ? cck[static_cast<int64_t>(cb - 1) * n + r0 + k] : INF;
        }
        // D(r0-1, c0-1): the virtual row -1 is zero, the virtual column -1 infinite
        const float corner = rb == 0 ? 0.f : (cb > 0 ? rck[static_cast<int64_t>(rb - 1) * a.M + c0 - 1] : INF);
        __syncwarp();

        float y[WB], D[WB];
        const float B0 = floorf(top[lane * WB]);
        float B = B0;  // per-lane base, as in the forward: absolute D = B + D'
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
                    // walk-back choice: smallest D, ties in the order diag, left, up
                    float v = diag;
                    uint32_t c = 0;
                    if (left < v) { v = left; c = 1; }
                    if (up < v) { v = up; c = 2; }
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
        __syncwarp();

        if (lane == 0) {
            // follow the path through this tile
            for (;;) {
                const float d2 = 2.f * g * (xs[wi] - ys[wj - c0]);
                ax += d2;
                ay -= d2;
                if (wi == 0) {
                    done = true;
                    break;
                }
                int code;
                if (wj == 0) {
                    code = 2;
                } else {
                    const int cc = wj - c0;
                    code = (dirs[(wi - r0) * 32 + cc / WB] >> (2 * (cc % WB))) & 3;
                }
                const bool row_change = code != 1;
                const bool col_change = code != 2;
                if (row_change) {
                    gq[wi] = ax;
                    ax = 0.f;
                    if (path) path[2 * wi] = wj;
                }
                if (col_change) {
                    gyq[wj] = ay;
                    ay = 0.f;
                }
                if (code == 0) { --wi; --wj; }
                else if (code == 1) { --wj; }
                else { --wi; }
                if (row_change && path) path[2 * wi + 1] = wj;
                if (wj < c0 || wi < r0) break;
            }
            if (done) {
                gq[0] = ax;
                gyq[wj] = ay;
                if (path) path[0] = wj;
                a.span[2 * ql] = wj;
                a.span[2 * ql + 1] = e64;
            }
        }
        wi = __shfl_sync(0xffffffffu, wi, 0);
        wj = __shfl_sync(0xffffffffu, wj, 0);
        done = __shfl_sync(0xffffffffu, done, 0);
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
    const int smem = bwd_smem_bytes(a.N, 32 * WB);
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

int bwd_smem_bytes(int N, int K)
{
    const int word = K == 256 ? 2 : 1;
    return 4 * (N + 3 * K) + K * 32 * word;
}

size_t ckpt_floats_per_query(int64_t N, int64_t M, int K)
{
    // a column every K columns (N values each) and a row every K rows (M values each)
    return static_cast<size_t>(N) * static_cast<size_t>(M / K) + static_cast<size_t>(N / K) * static_cast<size_t>(M);
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
