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
// start of every KS-th step (KS = 16, 32 or 64), its wavefront (each thread's latest
// row, the right-hand cells of its tile's other rows, its diagonal input and
// its integer base: an anti-diagonal staircase of rows, stored before a
// rebase due at that step, which is redone here), and the left inputs of every
// strip that starts a K-column window (K = 8 W).  The cells that the
// eight strips of one window computed during the KS steps after one
// checkpoint form a band, a parallelogram (each strip one tile higher than
// its left neighbour).  The
// walk proceeds band by band, one warp per query:
//   * the warp recomputes the band's rows down to the current cell from the
//     checkpointed wavefront and the window's boundary column, with the forward's
//     own operations in the forward's own bases (four lanes per strip, W/4
//     columns each; each step a lane advances RS rows, RS dependency chains,
//     one step behind lane l-1), so every value is the
//     forward's bit for bit; each cell's walk-back choice (two bits) is read
//     off the minimum by equality (diagonal first, then left, then up -- the
//     tie order of the walk-back);
//   * the walk itself is cooperative: the 32 lanes read 32 cells of the
//     current row at once and a ballot finds where the path leaves the row,
//     so a horizontal run of the path costs one step per 32 cells; finished
//     columns are written in parallel, and each lane keeps its share of the
//     current row's gradient, to be summed over lanes (in lane order) for all
//     the band's rows at once when the walk leaves the band -- a sum per row
//     on the walk's own chain of dependent steps would stall it.
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

// Rows a lane advances per step of the band recompute, for bands of tiles of
// RT rows: more rows give the lane more independent dependency chains, but
// lengthen the 32-step fill and drain of the lane chain.
constexpr int rows_per_step(int) { return 2; }

// One lane's step of the band recompute: RS consecutive rows over the lane's
// WB columns (D: the row above on entry, l: each row's left input, dg: the
// diagonal of the first row), recording each cell's walk-back choice as two
// bit masks per row.  Cells of row h depend on row h-1 in the same column and
// on row h in the column to the left: RS dependency chains, each one column
// behind the one above.  On exit D holds row RS-1, or with EXACT the last of
// the v valid rows (rows at or below the band's end are computed from
// placeholder inputs and never read), and l[h] holds row h's last column.
template <int WB, int RS, bool EXACT>
__device__ __forceinline__ void tile_rows(float (&D)[WB], const float (&y)[WB], const float (&x)[RS], float (&l)[RS],
                                          float dg, int v, uint32_t (&nd)[RS], uint32_t (&nu)[RS])
{
    float dgs[RS];
    dgs[0] = dg;
#pragma unroll
    for (int h = 1; h < RS; ++h) dgs[h] = l[h - 1];
#pragma unroll
    for (int h = 0; h < RS; ++h) nd[h] = nu[h] = 0u;
#pragma unroll
    for (int k = 0; k < WB; ++k) {
        float up = D[k];
        float row_v = up;
#pragma unroll
        for (int h = 0; h < RS; ++h) {
            // bit k of nd: the minimum is not the diagonal; of nu: neither the
            // diagonal nor the left cell (the cell above).  Written as selects:
            // branches here stall a warp that runs alone on its scheduler.
            const float m = min3_f32(up, dgs[h], l[h]);
            const bool not_diag = m != dgs[h];
            const bool is_up = not_diag & (m != l[h]);
            nd[h] |= not_diag ? (1u << k) : 0u;
            nu[h] |= is_up ? (1u << k) : 0u;
            const float t = x[h] - y[k];
            const float nv = fmaf(t, t, m);
            dgs[h] = up;
            l[h] = nv;
            up = nv;
            if constexpr (EXACT) {
                if (h < v) row_v = nv;
            }
        }
        D[k] = EXACT ? row_v : up;
    }
}

template <int WB, int RT, int RS>
__global__ void __launch_bounds__(32) bwd_band_kernel(const BwdArgs a)
{
    static_assert(RT % RS == 0, "a step's rows lie in one tile");
    using DW = typename DirWord<WB>::T;
    constexpr int W = 4 * WB;    // forward segment width: four lanes per strip
    constexpr int KW = 32 * WB;  // window width K = 8 W
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
    const int KS = a.KS;                             // a band's height in forward steps
    float* lcol = ys + KW;                           // [RT*KS] the window's boundary column
    float* gqs = lcol + RT * KS;                     // [N] the query's gradient, summed band by band
    float* rowpart = gqs + N;                        // [band rows][33] per-lane shares of each row's gradient
    DW* dirs = reinterpret_cast<DW*>(rowpart + (RT * KS + 7 * RT) * 33);  // [RS*steps][32] walk-back choices

    int64_t start;
    int n;
    if (a.offsets) {
        start = a.offsets[q];
        const int64_t stop = a.offsets[q + 1];
        const int64_t len = stop - start;
        if (start < 0 || len < 0 || len > N || stop > a.offsets[a.B_total] || (a.q_limit > 0 && stop > a.q_limit)) {
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
    for (int i = lane; i < n; i += 32) {
        xs[i] = x[i];
        gqs[i] = 0.f;
    }
    float* gyq = a.gyq + static_cast<int64_t>(ql) * a.M;
    float* gq = grads ? a.grad_queries + start : nullptr;
    int32_t* path = a.path ? a.path + 2 * start : nullptr;

    // the forward's schedule for this query (sdtw_fill.cuh)
    const int lag_last = (a.P - 1) * (32 + kChunk) + 31;
    const int nt = (n + RT - 1) / RT;
    const int Pp = max(nt, lag_last + kChunk);
    const int erec = fwd_record_floats(RT);
    const float* frq = a.fr + static_cast<int64_t>(ql) * a.fr_slot;
    const float* ckq = a.colck + static_cast<int64_t>(ql) * a.ck_slot;

    // walk state: the current cell (wi, wj), identical in every lane, and the
    // gradients of its row (each lane's share) and column accumulated so far
    int wi = n - 1, wj = static_cast<int>(e64);
    float axl = 0.f, ay = 0.f;  // this lane's share of row wi's gradient; column wj's so far
    bool done = false, first = true;
    if (lane == 0 && path) path[2 * wi + 1] = wj;

    const int d = lane >> 2;    // this lane's strip in the window
    const int sub = lane & 3;   // and its quarter of the strip

    // every band holds at least the walk's current cell, so a path of at most
    // n + M cells needs at most that many bands
    for (int64_t guard = 0; !done; ++guard) {
        // ---- the band holding (wi, wj): window b, checkpoint c
        const int b = wj / KW, c0 = b * KW, s = c0 / S;
        const int tau0 = (c0 - s * S) / W;   // forward thread of the window's first strip
        const int lag0 = (tau0 >> 5) * (32 + kChunk) + (tau0 & 31);  // strips of a window share a warp
        const int dj = (wj - c0) / W;
        const int c = (wi / RT + lag0 + dj + s * Pp) / KS;  // the checkpoint the band starts from
        const int ps0 = c * KS - lag0 - s * Pp;  // strip 0's tile at the band's first step
        const int rtop = RT * (ps0 - 7);             // the top of the band's rightmost strip
        const int ps = ps0 - d;                      // this lane's strip
        const int rf = RT * max(0, ps);              // its rows in the band: [rf, re)
        const int re = min(n, RT * min(nt, ps + KS));
        const int rf_left = RT * max(0, ps + 1);     // the strip on the left starts here
        const int rf0 = RT * max(0, ps0);
        const int re0 = min(min(n, RT * min(nt, ps0 + KS)), wi + 1);
        if (guard > static_cast<int64_t>(n) + M || wi < RT * max(0, ps0 - dj) ||
            wi >= min(n, RT * min(nt, ps0 - dj + KS))) {
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

        // ---- the lane's starting state: the checkpointed wavefront, or the virtual
        // zero row -1 for a strip that starts its sweep inside the band
        const float* frc = frq + static_cast<int64_t>(c) * L * (W + erec);
        const int tau = tau0 + d;
        auto fr_at = [&](int j, int th) { return frc[((j >> 2) * L + th) * 4 + (j & 3)]; };
        auto rec_at = [&](int e, int th) { return frc[(((W >> 2) + (e >> 2)) * L + th) * 4 + (e & 3)]; };
        // the forward stored its state before a rebase due at the band's
        // first step: redo it (new base: the integer part of the strip's first
        // column); a checkpoint between rebases is already in its base
        const bool redo = (c * KS) % a.rebase_period == 0;
        auto rebase = [&](int th, float& bn, float& dl) {
            const float b0 = rec_at(RT == 2 ? 2 : 4, th);
            bn = redo ? floorf(b0 + fr_at(0, th)) : b0;
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
        float e[RT], Bsrc = 0.f;
#pragma unroll
        for (int h = 0; h < RT; ++h) e[h] = 0.f;
        if (sub == 0 && d >= 1) {
            if (ps + 1 >= 1 && ps + 1 <= nt) {
                float dl;
                rebase(tau - 1, Bsrc, dl);
#pragma unroll
                for (int h = 0; h < RT - 1; ++h) e[h] = rec_at(h, tau - 1) - dl;
                e[RT - 1] = fr_at(W - 1, tau - 1) - dl;
            }
        }
        __syncwarp();
#pragma unroll
        for (int k = 0; k < WB; ++k) y[k] = ys[lane * WB + k];

        // ---- recompute the band's rows down to row wi, recording choices.
        // Lane l handles rows r .. r+RS-1 (r - rtop a multiple of RS, inside
        // one tile) at step (r - rtop)/RS + l.  A lane's last step in the band
        // may reach past row hi-1: those rows take a left input of +inf (or
        // the left lane's equally invalid rows) and a sample of 0, and are
        // never read -- the walk reads rows up to wi, and a strip's right
        // neighbour ends its band no lower.  The walk moves up and left from
        // (wi, wj), so the strips right of wj's strip dj are not needed either:
        // the schedule ends when strip dj's last lane has computed row wi.
        const int steps = (wi - rtop) / RS + 4 * dj + 4;
        const int hi = min(re, wi + 1);  // this lane's rows end here
        float last[RS];                  // right-hand cells of the lane's previous rows
#pragma unroll
        for (int h = 0; h < RS; ++h) last[h] = 0.f;
        // no lane has rows before its first step in the band: start at the
        // earliest of those (the rightmost strip's top is up to 7 tiles above
        // the others', so the first steps are often empty)
        const int sg0 = __reduce_min_sync(0xffffffffu, static_cast<unsigned>(rf < hi ? (rf - rtop) / RS + lane : steps));
        // the forward's rebases to a left input far below the base, replayed:
        // a strip's first lane decides at each tile's first row (the left input
        // of that row, as the forward converted it) and the strip's other
        // lanes follow the base their left lane's values arrive in
        float Btile = Bl, dltile = 0.f;  // first lanes: the base the tile's inputs were converted into, and the shift
        for (int sg = sg0; sg < steps; ++sg) {
            float recv[RS];
#pragma unroll
            for (int h = 0; h < RS; ++h) recv[h] = __shfl_up_sync(0xffffffffu, last[h], 1);
            const float Brecv = __shfl_up_sync(0xffffffffu, Bl, 1);  // the base of the values received
            const int r = rtop + RS * (sg - lane);
            if (r >= rf && r < hi) {
                const int v = min(RS, hi - r);  // valid rows of this step
                // left inputs: a strip's first lane converts its left strip's
                // values (from the left lane, or the stored record for the
                // strip's first tile) into its own base as the forward did,
                // the window's first strip reads the stored boundary column;
                // the other lanes take their left lane's values as they are
                const bool from_rec = sub == 0 && r < rf_left;  // a strip's first tile, first lane
                const bool tile_start = (r & (RT - 1)) == 0;
                const int eo = r - rf;                           // ... and the step's rows in it
                // a strip's other lanes follow the base their left lane's values
                // arrive in (the first lane rebased at these rows); the first
                // lane's own rebase is decided below, once its inputs are converted
                const float follow = sub != 0 ? Brecv - Bl : 0.f;
                if (tile_start) Btile = Bl;
                const float dconv = (from_rec ? Bsrc : Brecv) - Btile;
                float l[RS], x[RS];
#pragma unroll
                for (int h = 0; h < RS; ++h) {
                    float ev = e[h];
#pragma unroll
                    for (int o = RS; o < RT; o += RS)
                        if (eo == o) ev = e[h + o];
                    float lv = recv[h];
                    if (sub == 0) lv = (from_rec ? ev : recv[h]) + dconv;
                    if (d == 0 && sub == 0) lv = INF;
                    if (d == 0 && sub == 0 && b > 0 && h < v) lv = lcol[r + h - rf0];
                    l[h] = lv;
                    x[h] = h < v ? xs[r + h] : 0.f;
                }
                // the first lane's rebase at a tile's first row, as the forward
                // decides it; the tile's later rows take the same shift.  The
                // shift is applied without a branch: a lane without one shifts
                // by 0, which changes no value (x - 0 == x, signed zeros
                // included), and a divergent branch here costs more than the
                // subtractions in this latency-bound loop
                const bool trig = sub == 0 && tile_start && l[0] < -kRebaseBelow;
                const float dlt = trig ? floorf(Bl + l[0]) - Bl : 0.f;
                if (sub == 0 && tile_start) dltile = dlt;
                const float sh = sub != 0 ? follow : dlt;
#pragma unroll
                for (int k = 0; k < WB; ++k) D[k] -= sh;
                dg -= sh;
                Bl += sh;
#pragma unroll
                for (int h = 0; h < RS; ++h) l[h] -= dltile;
                const float dg_next = l[RS - 1];
                uint32_t nd[RS], nu[RS];
                if (first)
                    tile_rows<WB, RS, true>(D, y, x, l, dg, v, nd, nu);
                else
                    tile_rows<WB, RS, false>(D, y, x, l, dg, v, nd, nu);
#pragma unroll
                for (int h = 0; h < RS; ++h) {
                    last[h] = l[h];
                    dirs[(RS * sg + h) * 32 + lane] = static_cast<DW>(nd[h] | (nu[h] << WB));
                }
                dg = dg_next;
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
        const int wtop = wi;  // the band's rows the walk visits: [wlo, wtop]
        int wlo = wi;
        for (;;) {
            const float xi = xs[wi];
            if (wi == 0) {
                // the path starts here: only this cell of row 0 is on it
                const float cg = g2 * (xi - ys[wj - c0]);
                if (lane == 0) {
                    axl += cg;
                    if (grads) gyq[wj] = ay - cg;
                    if (path) path[0] = wj;
                    a.span[2 * ql] = wj;
                    a.span[2 * ql + 1] = e64;
                }
                rowpart[(wi - rtop) * 33 + lane] = axl;
                wlo = 0;
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
                        const uint32_t m = dirs[(wi - rtop + RS * lam) * 32 + lam] >> (cc - lam * WB);
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
            axl += cg;
            // column of lane k: finished unless the path goes up from it
            float vy = -cg;
            if (lane == 0) vy += ay;
            const int lcode = (lane == last && fcode != kOutside && f < 32) ? fcode : kLeft;
            if (grads && on && lcode != kUp) gyq[jk] = vy;
            const float vlast = __shfl_sync(0xffffffffu, vy, last);
            ay = (f < 32 && fcode == kUp) ? vlast : 0.f;
            const bool row_ends = f < 32 && fcode != kOutside;
            if (row_ends) {
                // the row ends at (wi, wj - last); move up or diagonally
                const int jl = wj - last;
                rowpart[(wi - rtop) * 33 + lane] = axl;
                axl = 0.f;
                wlo = wi;
                if (lane == 0 && path) path[2 * wi] = jl;
                wi -= 1;
                wj = fcode == kDiag ? jl - 1 : jl;
                if (lane == 0 && path) path[2 * wi + 1] = wj;
            } else {
                wj -= last + 1;  // the run continues to the left
            }
            if (wj < c0 || wi < RT * max(0, ps0 - (wj - c0) / W)) {
                // left the band; a row left unfinished continues in the next band
                if (!row_ends) {
                    rowpart[(wi - rtop) * 33 + lane] = axl;
                    axl = 0.f;
                    wlo = wi;
                }
                break;
            }
        }
        // the rows' gradients: each lane sums rows of the band over the 32
        // shares in lane order and adds them to the query's gradient (the rows
        // are 33 floats apart, so the lanes read distinct banks)
        __syncwarp();
        if (grads) {
            for (int i = wlo + lane; i <= wtop; i += 32) {
                const float* rp = rowpart + (i - rtop) * 33;
                float sum = 0.f;
#pragma unroll 8
                for (int k = 0; k < 32; ++k) sum += rp[k];
                gqs[i] += sum;
            }
        }
        __syncwarp();
    }
    if (grads)
        for (int i = lane; i < n; i += 32) gq[i] = gqs[i];
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
    const int64_t smem64 = bwd_smem_bytes(a.N, 4 * WB, a.RT, a.KS);
    if (smem64 < 0 || smem64 > kMaxSmemBytes) return cudaErrorInvalidValue;
    const int smem = static_cast<int>(smem64);
    auto k = a.RT == 2 ? bwd_band_kernel<WB, 2, rows_per_step(2)> : bwd_band_kernel<WB, 4, rows_per_step(4)>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    k<<<a.B, 32, smem, s>>>(a);
    return cudaGetLastError();
}

}  // namespace

bool bwd_width_supported(int W) { return W == 8 || W == 16 || W == 20 || W == 24 || W == 28 || W == 32; }

int64_t bwd_smem_bytes(int64_t N, int W, int RT, int KS)
{
    // query samples and gradient, the window's samples and boundary column,
    // the lanes' shares of the band's row gradients (33 floats per row), and
    // the choices of up to RT*KS + 7*RT + 32*RS rows of 32 lanes (W/2 bits
    // each): the band's rows below the top of its rightmost strip, and the
    // lag of RS rows per lane
    const int64_t word = W <= 16 ? 1 : 2;
    const int64_t RS = rows_per_step(RT);
    const int64_t rows = static_cast<int64_t>(RT) * KS;
    if (N < 0) N = 0;
    return 4 * (2 * N + 8 * W + rows) + 4 * (rows + 7 * RT) * 33 + (rows + 7 * RT + 32 * RS) * 32 * word;
}

cudaError_t launch_backward_walk(const BwdArgs& a, cudaStream_t s)
{
    if (a.B <= 0) return cudaSuccess;
    if (a.K != 8 * a.W || (a.RT != 2 && a.RT != 4) || !ckpt_stride_supported(a.KS) ||
        a.rebase_period != ckpt_rebase_period(a.KS))
        return cudaErrorInvalidValue;
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
