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
// start of every KS-th step (KS = 8, 16, 32 or 64), its wavefront (each thread's latest
// row, the right-hand cells of its tile's other rows, its diagonal input and
// its integer base: an anti-diagonal staircase of rows, stored before a
// rebase due at that step, which is redone here), and the left inputs of every
// strip that starts a K-column window (K = 8 W).  The cells that the
// eight strips of one window computed during the KS steps after one
// checkpoint form a band, a parallelogram (each strip one tile higher than
// its left neighbour).  The walk proceeds band by band, one CTA per query
// whose first warp walks (the walker); its other warps (helpers) recompute,
// into shared-memory band slots, the bands the walker predicts (those a path
// staying on its current row would visit next: the band changes of a long
// horizontal run, most of a long path's bands), and the walker takes a band
// from a slot when one holds it:
//   * a warp recomputes the band's rows down to the current cell from the
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
// exactly; a mismatch sets a status bit.  Every band is recomputed by the same
// code whichever warp runs it, so the results do not depend on the number of
// helpers.
//
// Per-query reference gradients go to rows of a scratch buffer, only over the
// path's column span; a second kernel sums them over queries in query order,
// so grad_ref is deterministic.
#include <cuda_runtime.h>

#include <algorithm>
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
    if constexpr (RS == 2) {
        // The cells (0, k) and (1, k-1) lie on one anti-diagonal and are
        // independent: their multiply-adds run as one f32x2 FMA (each lane
        // rounded once, exactly as fmaf), the same values as cell by cell.
        // Row 0 at column k: up D[k], diagonal g0, left l0; row 1 at column
        // k-1: up (row 0 at k-1) l0, diagonal g1, left l1.  Choice bits as
        // below.
        uint32_t nd0 = 0u, nu0 = 0u, nd1 = 0u, nu1 = 0u;
        float g0 = dg, l0 = l[0], g1 = l[0], l1 = l[1];
        {
            const float u0 = D[0];
            const float m0 = min3_f32(u0, g0, l0);
            nd0 |= m0 != g0 ? 1u : 0u;
            nu0 |= m0 != l0 ? 1u : 0u;
            const float t0 = x[0] - y[0];
            g0 = u0;
            l0 = fmaf(t0, t0, m0);
        }
#pragma unroll
        for (int k = 1; k < WB; ++k) {
            const float u0 = D[k], u1 = l0;
            const float m0 = min3_f32(u0, g0, l0);
            const float m1 = min3_f32(u1, g1, l1);
            nd0 |= m0 != g0 ? (1u << k) : 0u;
            nu0 |= m0 != l0 ? (1u << k) : 0u;
            nd1 |= m1 != g1 ? (1u << (k - 1)) : 0u;
            nu1 |= m1 != l1 ? (1u << (k - 1)) : 0u;
            const float2 t = make_float2(x[0] - y[k], x[1] - y[k - 1]);
            const float2 nv = __ffma2_rn(t, t, make_float2(m0, m1));
            D[k - 1] = EXACT && v < 2 ? u1 : nv.y;  // the last valid row
            g0 = u0;
            l0 = nv.x;
            g1 = u1;
            l1 = nv.y;
        }
        {
            const float u1 = l0;
            const float m1 = min3_f32(u1, g1, l1);
            nd1 |= m1 != g1 ? (1u << (WB - 1)) : 0u;
            nu1 |= m1 != l1 ? (1u << (WB - 1)) : 0u;
            const float t1 = x[1] - y[WB - 1];
            l1 = fmaf(t1, t1, m1);
            D[WB - 1] = EXACT && v < 2 ? u1 : l1;
        }
        l[0] = l0;
        l[1] = l1;
        nd[0] = nd0;
        nu[0] = nu0;
        nd[1] = nd1;
        nu[1] = nu1;
        return;
    }
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
            // bit k of nd: the minimum is not the diagonal; of nu: it is not the
            // left cell (the walk reads nu only where nd is set, so there nu
            // means the cell above).  Written as selects: branches here stall a
            // warp that runs alone on its scheduler.
            const float m = min3_f32(up, dgs[h], l[h]);
            const bool not_diag = m != dgs[h];
            const bool is_up = m != l[h];
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

// The band holding a cell: the cells the eight strips of K-column window b
// computed during the KS forward steps after checkpoint c.
struct Band {
    int b, c0;  // window and its first column
    int c;      // checkpoint the band starts from
    int ps0;    // strip 0's tile at the band's first step
    int tau0;   // forward thread of the window's first strip
    int rtop;   // the top row of the band's rightmost strip
};

// The forward's schedule for one query (sdtw_fill.cuh)
struct Sched {
    int n, nt, Pp, S, KS;
    int wps;     // windows per sweep, S / K = 4 P
    float rwps;  // 1 / wps
    int kslog;   // log2 KS (8, 16, 32 or 64)
};

template <int WB, int RT>
__device__ __forceinline__ Band band_at(const Sched& sc, int wi, int wj)
{
    constexpr int W = 4 * WB, KW = 32 * WB;
    Band g;
    g.b = wj / KW;
    g.c0 = g.b * KW;
    // the sweep s = b / wps without an integer division (b < 2^24: the float
    // quotient is off by at most one)
    int s = __float2int_rz(static_cast<float>(g.b) * sc.rwps);
    s += (s + 1) * sc.wps <= g.b;
    s -= s * sc.wps > g.b;
    g.tau0 = 8 * (g.b - s * sc.wps);  // (c0 - s S) / W, as K = 8 W
    const int lag0 = (g.tau0 >> 5) * (32 + kChunk) + (g.tau0 & 31);  // strips of a window share a warp
    const int dj = (wj - g.c0) / W;
    g.c = (wi / RT + lag0 + dj + s * sc.Pp) >> sc.kslog;
    g.ps0 = g.c * sc.KS - lag0 - s * sc.Pp;
    g.rtop = RT * (g.ps0 - 7);
    return g;
}

// Recompute the rows of band g down to row wi in strips 0..dj, recording each
// cell's walk-back choice: row RS*(sg - sg0) + h of `dirs` holds the choices of
// step sg's row h, lane by lane.  Fills the window's samples `ys` and boundary
// column `lcol` first.  Returns sg0 (the first step at which some lane has
// rows), or -1 if the steps would not fit in `drows` rows (never for the sizes
// that bwd_smem_bytes reserves).  With EXACT, D and Bl return this lane's last
// valid row and its base (the end-cell check of the first band).
template <int WB, int RT, int RS, bool EXACT, typename DW>
__device__ __forceinline__ int recompute_band(const BwdArgs& a, const Sched& sc, const Band& g, int wi, int dj,
                                              const float* __restrict__ xs, float* ys, float* lcol, DW* dirs,
                                              int drows, const float* frq, const float* ckq, int lane,
                                              float (&D)[WB], float& Bl)
{
    constexpr int W = 4 * WB;    // forward segment width: four lanes per strip
    constexpr int KW = 32 * WB;  // window width K = 8 W
    const int L = 32 * a.P;
    const int N = a.N;
    const int M = static_cast<int>(a.M);
    const int n = sc.n, nt = sc.nt, KS = sc.KS;
    const float INF = __int_as_float(0x7f800000);
    const int d = lane >> 2;   // this lane's strip in the window
    const int sub = lane & 3;  // and its quarter of the strip
    const int ps = g.ps0 - d;                    // this lane's strip's tile at the band's first step
    const int rf = RT * max(0, ps);              // its rows in the band: [rf, re)
    const int re = min(n, RT * min(nt, ps + KS));
    const int rf_left = RT * max(0, ps + 1);     // the strip on the left starts here
    const int rf0 = RT * max(0, g.ps0);
    const int re0 = min(min(n, RT * min(nt, g.ps0 + KS)), wi + 1);

    __syncwarp();
    for (int k = lane; k < KW; k += 32) ys[k] = g.c0 + k < M ? a.ref[g.c0 + k] : 0.f;
    if (g.b > 0)
        for (int k = lane; k < re0 - rf0; k += 32) lcol[k] = ckq[static_cast<int64_t>(g.b - 1) * ck_rows(N) + rf0 + k];

    // ---- the lane's starting state: the checkpointed wavefront, or the virtual
    // zero row -1 for a strip that starts its sweep inside the band
    const int erec = fwd_record_floats(RT);
    const float* frc = frq + static_cast<int64_t>(g.c) * L * (W + erec);
    const int tau = g.tau0 + d;
    auto fr_at = [&](int j, int th) { return frc[((j >> 2) * L + th) * 4 + (j & 3)]; };
    auto rec_at = [&](int e, int th) { return frc[(((W >> 2) + (e >> 2)) * L + th) * 4 + (e & 3)]; };
    // the forward stored its state before a rebase due at the band's
    // first step: redo it (new base: the integer part of the strip's first
    // column); a checkpoint between rebases is already in its base
    const bool redo = (g.c * KS) % a.rebase_period == 0;
    auto rebase = [&](int th, float& bn, float& dl) {
        const float b0 = rec_at(RT, th);  // the record: RT-1 right-hand cells, diag, base
        bn = redo ? floorf(b0 + fr_at(0, th)) : b0;
        dl = bn - b0;
    };
    float y[WB];
    float dg = 0.f;
    Bl = 0.f;
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
    // the cell it enters the band at, so strips right of dj are not needed:
    // the schedule ends after the last step at which a lane of strips 0..dj
    // has a row (for the entry strip's last lane, row wi)
    const int hi = min(re, wi + 1);  // this lane's rows end here
    const int steps = 1 + static_cast<int>(__reduce_max_sync(
                              0xffffffffu, d <= dj && rf < hi ? static_cast<unsigned>((hi - 1 - g.rtop) / RS + lane) : 0u));
    float last[RS];                  // right-hand cells of the lane's previous rows
#pragma unroll
    for (int h = 0; h < RS; ++h) last[h] = 0.f;
    // no lane has rows before its first step in the band: start at the
    // earliest of those (the rightmost strip's top is up to 7 tiles above
    // the others', so the first steps are often empty)
    const int sg0 = __reduce_min_sync(0xffffffffu, static_cast<unsigned>(rf < hi ? (rf - g.rtop) / RS + lane : steps));
    if (RS * (steps - sg0) > drows) return -1;
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
        const int r = g.rtop + RS * (sg - lane);
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
                if (d == 0 && sub == 0 && g.b > 0 && h < v) lv = lcol[r + h - rf0];
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
            tile_rows<WB, RS, EXACT>(D, y, x, l, dg, v, nd, nu);
#pragma unroll
            for (int h = 0; h < RS; ++h) {
                last[h] = l[h];
                dirs[(RS * (sg - sg0) + h) * 32 + lane] = static_cast<DW>(nd[h] | (nu[h] << WB));
            }
            dg = dg_next;
        }
    }
    return sg0;
}

// Shared-memory bookkeeping of the band slots: per slot its state, the band
// (window b, checkpoint c) and the cell it was computed for (rows down to wi,
// strips 0..dj), and the first step of its choice rows.
constexpr int kDiag = 0, kLeft = 1, kUp = 2, kOutside = 3;  // a cell's walk-back choice
constexpr int kSlotFree = 0, kSlotAssigned = 1, kSlotReady = 2, kSlotOwn = 3;
constexpr int kMetaInts = 8;  // state, b, c, wi, wj, dj, sg0, spare
constexpr int kMaxSlots = 4;
constexpr int kHeaderBytes = 4 * (kMaxSlots * kMetaInts + kMaxSlots + 4);  // metadata, mailboxes, done flag
constexpr long long kWaitNs = 2000000000LL;   // the walker's wait for a helper's band gives up after 2 s
constexpr long long kIdleNs = 20000000000LL;  // a helper without work gives up after 20 s
constexpr int kDefaultBwdWarps = 3;          // the walker and two helpers

__device__ __forceinline__ long long global_ns()
{
    long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One CTA per query.  Warp 0 walks the path band by band; with more warps,
// warps 1.. are helpers: when the walk enters a band, the walker hands them
// the next bands a path staying on the current row would visit (the band
// changes of a long horizontal run, most of a long path's bands), and the
// helpers recompute those into shared-memory slots while the walker works.
// A band the walk enters is taken from a slot that holds it (computed down to
// a row at or below the entry cell), else recomputed by the walker.  Slot
// states and the helpers' mailboxes live in shared memory; every wait on them
// gives up after kWaitNs (status kStatusTimeout).
template <int WB, int RT, int RS>
__global__ void __launch_bounds__(32 * kMaxSlots) bwd_band_kernel(const BwdArgs a, const int drows)
{
    static_assert(RT % RS == 0, "a step's rows lie in one tile");
    using DW = typename DirWord<WB>::T;
    constexpr int W = 4 * WB;    // forward segment width: four lanes per strip
    constexpr int KW = 32 * WB;  // window width K = 8 W
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int NS = blockDim.x >> 5;  // band slots: one per warp
    const int H = NS - 1;            // helpers
    const int N = a.N;
    const int M = static_cast<int>(a.M);
    const int KS = a.KS;
    const int ql = blockIdx.x;  // query within this launch
    const int q = a.q0 + ql;    // query within the batch

    extern __shared__ __align__(16) unsigned char smem_raw[];
    volatile int* meta = reinterpret_cast<volatile int*>(smem_raw);  // [kMaxSlots][kMetaInts]
    volatile int* mailbox = meta + kMaxSlots * kMetaInts;            // helper h: the slot to compute, or -1
    volatile int* done_flag = mailbox + kMaxSlots;                   // set when the walk ends
    float* xs = reinterpret_cast<float*>(smem_raw + kHeaderBytes);  // [N] query samples
    float* gqs = xs + N;                                             // [N] the query's gradient, summed band by band
    float* rowpart = gqs + N;                                        // [band rows][33] per-lane shares of each row's gradient
    unsigned char* slot_base = reinterpret_cast<unsigned char*>(rowpart + (RT * KS + 7 * RT) * 33);
    const int slot_bytes = 4 * (KW + RT * KS) + drows * 32 * static_cast<int>(sizeof(DW));
    // slot s: the window's samples [KW], its boundary column [RT*KS], choices [drows][32]
    auto slot_ys = [&](int s) { return reinterpret_cast<float*>(slot_base + s * slot_bytes); };
    auto slot_lcol = [&](int s) { return slot_ys(s) + KW; };
    auto slot_dirs = [&](int s) { return reinterpret_cast<DW*>(slot_ys(s) + KW + RT * KS); };

    int64_t start;
    int n;
    if (a.offsets) {
        start = a.offsets[q];
        const int64_t stop = a.offsets[q + 1];
        const int64_t len = stop - start;
        if (start < 0 || len < 0 || len > N || stop > a.offsets[a.B_total] || (a.q_limit > 0 && stop > a.q_limit)) {
            if (threadIdx.x == 0) {
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
        if (threadIdx.x == 0) {
            a.span[2 * ql] = 0;
            a.span[2 * ql + 1] = -1;
        }
        return;
    }
    const int64_t e64 = a.end[q];
    if (e64 < 0 || e64 >= a.M) {
        if (threadIdx.x == 0) {
            atomicOr(a.status, kStatusBadEnd);
            a.span[2 * ql] = 0;
            a.span[2 * ql + 1] = -1;
        }
        return;
    }
    const bool grads = a.grad_queries != nullptr;  // false: the path only
    const float g2 = grads ? 2.f * a.grad_cost[q] : 0.f;
    const float* x = a.queries + start;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        xs[i] = x[i];
        gqs[i] = 0.f;
    }
    if (threadIdx.x < kMaxSlots) {
        meta[threadIdx.x * kMetaInts] = kSlotFree;
        mailbox[threadIdx.x] = -1;
    }
    if (threadIdx.x == 0) *done_flag = 0;
    __syncthreads();

    // the forward's schedule for this query (sdtw_fill.cuh)
    const int lag_last = (a.P - 1) * (32 + kChunk) + 31;
    const int nt = (n + RT - 1) / RT;
    const Sched sc{n, nt, max(nt, lag_last + kChunk), 32 * a.P * W, KS, 4 * a.P, 1.f / (4 * a.P), __ffs(KS) - 1};
    const float* frq = a.fr + static_cast<int64_t>(ql) * a.fr_slot;
    const float* ckq = a.colck + static_cast<int64_t>(ql) * a.ck_slot;

    if (warp > 0) {
        // ---- a helper: recompute the bands handed to it until the walk ends
        if (a.idle_helpers) return;  // tests of the walker's bounded wait
        const int h = warp - 1;
        float Dd[WB], Bd;
        long long t_idle = global_ns();  // lane 0: when this helper last had work
        for (;;) {
            // lane 0 decides: a slot to compute, -2 the walk ended, -3 idle too
            // long, -1 nothing yet
            int cmd = -1;
            if (lane == 0) {
                const int s2 = mailbox[h];
                cmd = s2 >= 0 ? s2 : *done_flag ? -2 : global_ns() - t_idle > kIdleNs ? -3 : -1;
            }
            cmd = __shfl_sync(0xffffffffu, cmd, 0);
            if (cmd >= 0) {
                __threadfence_block();
                const int pwi = meta[cmd * kMetaInts + 3], pwj = meta[cmd * kMetaInts + 4];
                const Band g = band_at<WB, RT>(sc, pwi, pwj);
                const int sg0 = recompute_band<WB, RT, RS, false>(a, sc, g, pwi, 7, xs, slot_ys(cmd), slot_lcol(cmd),
                                                                  slot_dirs(cmd), drows, frq, ckq, lane, Dd, Bd);
                __threadfence_block();
                __syncwarp();
                if (lane == 0) {
                    meta[cmd * kMetaInts + 6] = sg0;
                    __threadfence_block();
                    meta[cmd * kMetaInts] = kSlotReady;
                    __threadfence_block();
                    mailbox[h] = -1;
                    t_idle = global_ns();
                }
                __syncwarp();
            } else if (cmd == -2) {
                return;
            } else if (cmd == -3) {
                if (lane == 0) atomicOr(a.status, kStatusTimeout);
                return;
            } else {
                __nanosleep(200);
            }
        }
    }

    // ---- the walker.  Walk state: the current cell (wi, wj), identical in
    // every lane, and the gradients of its row (each lane's share) and column
    // accumulated so far
    float* gyq = a.gyq + static_cast<int64_t>(ql) * a.M;
    float* gq = grads ? a.grad_queries + start : nullptr;
    int32_t* path = a.path ? a.path + 2 * start : nullptr;
    int wi = n - 1, wj = static_cast<int>(e64);
    float axl = 0.f, ay = 0.f;  // this lane's share of row wi's gradient; column wj's so far
    bool done = false, first = true;
    if (lane == 0 && path) path[2 * wi + 1] = wj;
    auto give_up = [&](int bit) {  // report, end the helpers' loops, and leave this query
        if (lane == 0) {
            atomicOr(a.status, bit);
            a.span[2 * ql] = 0;
            a.span[2 * ql + 1] = -1;
            *done_flag = 1;
        }
    };
    int cur = 0;  // the slot of the band the walk is in

    // every band holds at least the walk's current cell, so a path of at most
    // n + M cells needs at most that many bands
    for (int64_t guard = 0; !done; ++guard) {
        // ---- the band holding (wi, wj)
        const Band g = band_at<WB, RT>(sc, wi, wj);
        const int c0 = g.c0, ps0 = g.ps0, rtop = g.rtop;
        const int dj = (wj - c0) / W;
        if (guard > static_cast<int64_t>(n) + M || wi < RT * max(0, ps0 - dj) ||
            wi >= min(n, RT * min(nt, ps0 - dj + KS))) {
            give_up(kStatusReplay);  // the current cell is not in its band
            return;
        }
        // Slot bookkeeping, lane-parallel: lane s < NS reads slot s, ballots
        // combine the lanes' findings, and lane 0 writes hand-outs.
        // A slot that holds this band (a helper's), else the walker recomputes
        // it into the slot of the band it leaves (the walk never returns to a band)
        const bool slot_lane = lane < NS;
        int st_l = kSlotOwn, kb = -1, kc = -1, kw = -1, kd = -1;  // lane s: slot s's state and band
        if (slot_lane) {
            const volatile int* m = meta + lane * kMetaInts;
            st_l = m[0];
            kb = m[1];
            kc = m[2];
            kw = m[3];
            kd = m[5];
        }
        const unsigned found = __ballot_sync(0xffffffffu, slot_lane && lane != cur && st_l != kSlotFree &&
                                                              kb == g.b && kc == g.c && kw >= wi && kd >= dj);
        const bool hit = found != 0u;
        if (lane == cur) {
            st_l = hit ? kSlotFree : kSlotOwn;
            meta[cur * kMetaInts] = st_l;
        }
        if (hit) cur = __ffs(found) - 1;
        // the bands a path staying on row wi would visit next, left of this one
        int pb[kMaxSlots - 1], pc[kMaxSlots - 1], pj[kMaxSlots - 1];
        int np = 0;
        {
            int jj = c0 + max(0, ps0 - wi / RT) * W - 1;  // left of the band's leftmost cell of row wi
#pragma unroll
            for (int k = 0; k < kMaxSlots - 1; ++k) {
                pb[k] = pc[k] = pj[k] = -1;
                if (k < H && jj >= 0) {
                    const Band gp = band_at<WB, RT>(sc, wi, jj);
                    pb[k] = gp.b;
                    pc[k] = gp.c;
                    pj[k] = jj;
                    np = k + 1;
                    jj = gp.c0 + max(0, gp.ps0 - wi / RT) * W - 1;
                } else {
                    jj = -1;
                }
            }
        }
        // hand the predicted bands that no slot holds to idle helpers; finished
        // slots that no prediction names are freed.  Run at band entry (so that
        // the helpers work during the walker's own recompute or wait) and again
        // once the band is ready (a helper that finished meanwhile takes the
        // next prediction at once)
        auto predict = [&](bool reread) {
            if (H == 0) return;
            if (reread && slot_lane && lane != cur) st_l = meta[lane * kMetaInts];
            const bool mine = slot_lane && lane != cur && st_l != kSlotFree && st_l != kSlotOwn;
            bool named = false;
            unsigned have = 0u;
#pragma unroll
            for (int k = 0; k < kMaxSlots - 1; ++k) {
                const bool nk = mine && k < np && kb == pb[k] && kc == pc[k] && kw >= wi && kd >= 7;
                named |= nk;
                if (__ballot_sync(0xffffffffu, nk)) have |= 1u << k;
            }
            // a finished band no prediction names is dropped (a helper's band in
            // flight runs to its end: stopping it measured slower, as such bands
            // are often visited after all)
            if (mine && !named && st_l == kSlotReady) {
                st_l = kSlotFree;
                meta[lane * kMetaInts] = kSlotFree;
            }
            unsigned fm = __ballot_sync(0xffffffffu, slot_lane && lane != cur && st_l == kSlotFree);
            unsigned im = __ballot_sync(0xffffffffu, lane < H && mailbox[lane < H ? lane : 0] < 0);
#pragma unroll
            for (int k = 0; k < kMaxSlots - 1; ++k) {
                if (k >= np || (have >> k) & 1u || fm == 0u || im == 0u) continue;
                const int fs = __ffs(fm) - 1, fh = __ffs(im) - 1;
                fm &= fm - 1u;
                im &= im - 1u;
                if (lane == fs) {
                    // this lane's view of its slot follows the hand-out
                    st_l = kSlotAssigned;
                    kb = pb[k];
                    kc = pc[k];
                    kw = wi;
                    kd = 7;
                }
                if (lane == 0) {
                    volatile int* m = meta + fs * kMetaInts;
                    m[1] = pb[k];
                    m[2] = pc[k];
                    m[3] = wi;
                    m[4] = pj[k];
                    m[5] = 7;
                    m[6] = -1;
                    __threadfence_block();
                    m[0] = kSlotAssigned;
                    __threadfence_block();
                    mailbox[fh] = fs;
                }
            }
        };
        predict(false);
        __syncwarp();

        int sg0;
        float D[WB], Bl;
        if (!hit) {
            sg0 = first ? recompute_band<WB, RT, RS, true>(a, sc, g, wi, dj, xs, slot_ys(cur), slot_lcol(cur),
                                                           slot_dirs(cur), drows, frq, ckq, lane, D, Bl)
                        : recompute_band<WB, RT, RS, false>(a, sc, g, wi, dj, xs, slot_ys(cur), slot_lcol(cur),
                                                            slot_dirs(cur), drows, frq, ckq, lane, D, Bl);
        } else {
            // the helper's slot, once it is ready
            const long long t0 = global_ns();
            for (;;) {
                int st = 0;
                if (lane == 0) st = meta[cur * kMetaInts] == kSlotReady ? 1 : global_ns() - t0 > kWaitNs ? 2 : 0;
                st = __shfl_sync(0xffffffffu, st, 0);
                if (st == 1) break;
                if (st == 2) {
                    give_up(kStatusTimeout);
                    return;
                }
                __nanosleep(64);
            }
            __threadfence_block();
            sg0 = meta[cur * kMetaInts + 6];
        }
        if (sg0 < 0) {
            give_up(kStatusReplay);  // the band's steps exceed the slot
            return;
        }
        predict(true);
        __syncwarp();
        const float* ys = slot_ys(cur);
        const DW* dirs = slot_dirs(cur);
        const int doff = RS * sg0;  // choices of step sg, row h: row RS*sg + h - doff

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
                        const uint32_t m = dirs[(wi - rtop + RS * lam - doff) * 32 + lam] >> (cc - lam * WB);
                        code = !(m & 1u) ? kDiag : ((m >> WB) & 1u) ? kUp : kLeft;
                    }
                }
            }
            // the first lane whose cell leaves the row, and its code, from ballots
            // (a shuffle of the code would add its latency to the walk's chain)
            const unsigned stop = __ballot_sync(0xffffffffu, code != kLeft);
            const unsigned bdiag = __ballot_sync(0xffffffffu, code == kDiag);
            const unsigned bup = __ballot_sync(0xffffffffu, code == kUp);
            const int f = stop ? __ffs(stop) - 1 : 32;
            const unsigned fbit = stop & (0u - stop);
            const int fcode = !stop ? kLeft : (bdiag & fbit) ? kDiag : (bup & fbit) ? kUp : kOutside;
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
    if (lane == 0) *done_flag = 1;  // the helpers' loops end
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
    const int drows = bwd_dir_rows(a.RT, a.KS);
    const int warps = bwd_warps(a.N, 4 * WB, a.RT, a.KS, a.warps);
    if (warps < 1) return cudaErrorInvalidValue;
    const int smem = static_cast<int>(bwd_smem_bytes(a.N, 4 * WB, a.RT, a.KS, warps));
    auto k = bwd_band_kernel<WB, 4, rows_per_step(4)>;
    if (a.RT == 2) k = bwd_band_kernel<WB, 2, rows_per_step(2)>;
    if constexpr (WB >= 4 && WB <= 7) {  // 8-row tiles: segments of 16 to 28 columns
        if (a.RT == 8) k = bwd_band_kernel<WB, 8, rows_per_step(8)>;
    }
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (e != cudaSuccess) return e;
    }
    k<<<a.B, 32 * warps, smem, s>>>(a, drows);
    return cudaGetLastError();
}

}  // namespace

bool bwd_width_supported(int W) { return W == 8 || W == 16 || W == 20 || W == 24 || W == 28 || W == 32; }

// Rows of choices one band slot holds: RS rows per step, from the first step
// at which some lane has rows (no earlier than RT*7/RS: lane 4d+sub's first row
// lies RT*(7-d) rows below the rightmost strip's top, and the lane runs 4d+sub
// steps behind lane 0) to the last step of a band of KS steps (the last lane
// of the entry strip dj, for the band's bottom row in that strip, over every dj).
int bwd_dir_rows(int RT, int KS)
{
    const int RS = rows_per_step(RT);
    int most = 0;
    for (int dj = 0; dj < 8; ++dj) most = std::max(most, (RT * (KS + 7 - dj) - 1) / RS + 4 * dj + 4);
    return RS * (most - RT * 7 / RS);
}

int64_t bwd_smem_bytes(int64_t N, int W, int RT, int KS, int warps)
{
    // the slots' and helpers' bookkeeping, the query samples and gradient,
    // the lanes' shares of the band's row gradients (33 floats per row), and
    // one band slot per warp: the window's samples and boundary column and
    // the choices (W/2 bits per lane and row)
    const int64_t word = W <= 16 ? 1 : 2;
    const int64_t rows = static_cast<int64_t>(RT) * KS;
    if (N < 0) N = 0;
    const int64_t slot = 4 * (8 * W + rows) + static_cast<int64_t>(bwd_dir_rows(RT, KS)) * 32 * word;
    return kHeaderBytes + 4 * 2 * N + 4 * (rows + 7 * RT) * 33 + warps * slot;
}

int bwd_warps(int64_t N, int W, int RT, int KS, int requested)
{
    if (requested < 0 || requested > kMaxSlots) return 0;
    int w = requested > 0 ? requested : kDefaultBwdWarps;
    while (w > 1 && bwd_smem_bytes(N, W, RT, KS, w) > kMaxSmemBytes) --w;
    return bwd_smem_bytes(N, W, RT, KS, w) <= kMaxSmemBytes ? w : 0;
}

cudaError_t launch_backward_walk(const BwdArgs& a, cudaStream_t s)
{
    if (a.B <= 0) return cudaSuccess;
    if (a.K != 8 * a.W || (a.RT != 2 && a.RT != 4 && !(a.RT == 8 && a.W >= 16 && a.W <= 28)) ||
        !ckpt_stride_supported(a.KS) ||
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
