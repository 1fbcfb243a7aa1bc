"""CPU model of the backward checkpoints and of the backward's band replay.

The checkpointing forward (csrc/sdtw_fill.cuh) stores, every KS steps
(KS = 8, 16, 32 or 64), the state of its wavefront: each thread's latest row (its
strip of W columns, relative to the thread's integer base), the right-hand
cells of its tile's other rows, its diagonal input and its base, as they stand
before a rebase due at that step (the backward redoes that rebase; the fill
rebases every max(kChunk, KS) steps, so a 16-step checkpoint between rebases
is already in its base).  The rows a wavefront holds form an anti-diagonal
staircase (thread l is one tile behind thread l-1), so these are checkpoints
along anti-diagonals, one every KS steps.  Beside them, the strip that starts at every K-th column stores the left
inputs it used (its boundary column, already converted into its own base).

The backward (csrc/sdtw_backward.cu) recomputes one band at a time: the cells
that the strips of one K-column window computed during the KS steps after one
checkpoint, a parallelogram.  Starting from the chunk's stored wavefront and the window's
stored boundary column, with the forward's own operations, it reproduces the
forward's FP32 values bit for bit.

This file replays both in plain Python with FP32 rounding (struct casts; the
fused multiply-add is rounded once) and checks, on shapes with several warps,
sweeps, ragged tails and both tile heights:

* every cell of every band is reproduced exactly (value and base);
* the band lookup used by the walk-back assigns every cell to one band whose
  replay covers it;
* a walk-back driven band by band from those replays follows the same path as
  a walk over the whole FP32 matrix, and ends at the forward's cost.
"""
import math
import struct

import numpy as np
import pytest

K_CHUNK = 32   # csrc/sdtw_internal.h kChunk
REBASE_BELOW = 256.0   # csrc/sdtw_internal.h kRebaseBelow
STRIDES = (8, 16, 32, 64)   # checkpoint strides the library supports
INF = float("inf")


def r32(v):
    """Round a Python float to the nearest FP32 value (ties to even)."""
    return struct.unpack("f", struct.pack("f", v))[0]


def _next32(v, toward):
    return float(np.nextafter(np.float32(v), np.float32(toward)))


def fma32(a, b, c):
    """a*b + c rounded once to FP32 (a, b, c FP32 values)."""
    p = a * b                      # exact: two 24-bit significands
    s = p + c
    bb = s - p
    e = (p - (s - bb)) + (c - bb)  # s + e == p + c exactly (TwoSum)
    r = r32(s)
    if r != s and e != 0.0:
        o = _next32(r, INF if s > r else -INF)
        if (r + o) / 2 == s:       # s is a tie between r and o: e decides
            if (e > 0) == (o > r):
                r = o
    return r


DIAG, LEFT, UP = 0, 1, 2


def cell(xv, yv, up, dg, lf):
    """(D, walk-back choice): the choice is read off the minimum by equality,
    diagonal first, then left, then up (the walk-back's tie order)."""
    d = r32(xv - yv)
    m = min(up, dg, lf)
    return fma32(d, d, m), (DIAG if m == dg else LEFT if m == lf else UP)


def rebase(B, first):
    """A thread's new integer base at a chunk start and the shift applied to
    its values (the forward's rebase, replayed by the backward)."""
    bn = float(math.floor(r32(B + first)))
    return bn, r32(bn - B)


def rebase_to_left(B, left0):
    """The forward's rebase to a left input far below the strip's base: (new
    base, shift), or None when the tile's first-row left input is not that low."""
    if not left0 < -REBASE_BELOW:
        return None
    bn = float(math.floor(r32(B + left0)))
    return bn, r32(bn - B)


def frontier_state(fw, pl, c, tau):
    """A thread's state at checkpoint c (step c * KS), after the rebase when
    one is due at that step."""
    prev, alast, diag, B = fw["frontier"][(c, tau)]
    if (c * pl.KS) % pl.R:
        return prev[:], alast[:], diag, B
    bn, dl = rebase(B, prev[0])
    return [r32(v - dl) for v in prev], [r32(v - dl) for v in alast], r32(diag - dl), bn


class Plan:
    def __init__(self, n, M, P, W, RT, K, KS=K_CHUNK):
        self.n, self.M, self.P, self.W, self.RT, self.K = n, M, P, W, RT, K
        self.KS = KS                      # steps between wavefront checkpoints
        self.R = max(K_CHUNK, KS)         # steps between rebases
        self.L = 32 * P
        self.S = self.L * W
        self.nsw = -(-M // self.S)
        self.lag = [(t // 32) * (32 + K_CHUNK) + t % 32 for t in range(self.L)]
        self.lag_last = self.lag[-1]
        self.nt = -(-n // RT)
        self.Pp = max(self.nt, self.lag_last + K_CHUNK)
        self.total = (self.nsw - 1) * self.Pp + self.nt + self.lag_last
        self.ckpts = -(-self.total // KS)

    def band_of(self, i, j):
        """(checkpoint, window) of the band holding cell (i, j)."""
        s, tau = j // self.S, (j % self.S) // self.W
        t = i // self.RT + self.lag[tau] + s * self.Pp
        return t // self.KS, j // self.K


def model_forward(x, y, pl):
    """FP32 model of the checkpointing forward: every cell (value, base), the
    wavefront checkpoints, the boundary columns and (cost, end)."""
    n, M, W, RT, K, L = pl.n, pl.M, pl.W, pl.RT, pl.K, pl.L
    xs = [r32(v) for v in x] + [0.0] * (RT * pl.nt - n)
    ys = [r32(v) for v in y]
    prev = [[0.0] * W for _ in range(L)]
    alast = [[0.0] * (RT - 1) for _ in range(L)]
    diag = [0.0] * L
    B = [0.0] * L
    p = [-pl.lag[t] for t in range(L)]
    s = [0] * L
    base = [t * W for t in range(L)]
    yv = [[0.0] * W for _ in range(L)]
    ring, colbuf = {}, {}
    frontier, colck, D = {}, {}, {}
    best, best_col = INF, None
    triggers = 0
    for t in range(pl.total):
        if t % pl.KS == 0:
            # the wavefront as the previous steps left it (before a rebase due now)
            c = t // pl.KS
            for tau in range(L):
                pp, ss = p[tau], s[tau]
                if (1 <= pp <= pl.nt and ss < pl.nsw) or (pp == 0 and ss >= 1 and pl.Pp == pl.nt):
                    frontier[(c, tau)] = (prev[tau][:], alast[tau][:], diag[tau], B[tau])
        if t % pl.R == 0:
            for tau in range(L):
                bn, dl = rebase(B[tau], prev[tau][0])
                prev[tau] = [r32(v - dl) for v in prev[tau]]
                alast[tau] = [r32(v - dl) for v in alast[tau]]
                diag[tau] = r32(diag[tau] - dl)
                B[tau] = bn
        # the step's inputs: registers as they stand before anyone computes
        recv, rb = [None] * L, [0.0] * L
        for tau in range(L):
            lane, w = tau % 32, tau // 32
            act = 0 <= p[tau] < pl.nt and s[tau] < pl.nsw
            if lane > 0:
                recv[tau], rb[tau] = alast[tau - 1] + [prev[tau - 1][W - 1]], B[tau - 1]
            elif w > 0:
                recv[tau], rb[tau] = ring.get((w, t - K_CHUNK - 1), ([INF] * RT, 0.0))
            elif act and s[tau] > 0:
                recv[tau], rb[tau] = colbuf[p[tau]]
            else:
                recv[tau], rb[tau] = [INF] * RT, 0.0
        for tau in range(L):
            if not (0 <= p[tau] < pl.nt and s[tau] < pl.nsw):
                continue
            pt = p[tau]
            if pt == 0:
                base[tau] = s[tau] * pl.S + tau * W
                yv[tau] = [ys[base[tau] + k] if base[tau] + k < M else 0.0 for k in range(W)]
                prev[tau] = [0.0] * W
                diag[tau] = 0.0
                B[tau] = 0.0
            dd = r32(rb[tau] - B[tau])
            left = [r32(v + dd) for v in recv[tau]]
            b0 = base[tau]
            if b0 % K == 0 and 0 < b0 < M:
                for rr in range(RT):                 # stored as converted, before any shift
                    if RT * pt + rr < n:
                        colck[(b0 // K, RT * pt + rr)] = left[rr]
            shift = rebase_to_left(B[tau], left[0])
            if shift:
                triggers += 1
                B[tau], dl = shift
                prev[tau] = [r32(v - dl) for v in prev[tau]]
                diag[tau] = r32(diag[tau] - dl)
                left = [r32(v - dl) for v in left]
            rows, codes, above, dg0 = [], [], prev[tau], diag[tau]
            for rr in range(RT):
                xv = xs[RT * pt + rr]
                cur, cc = [], []
                for j in range(W):
                    up = above[j]
                    dg = dg0 if j == 0 else above[j - 1]
                    lf = left[rr] if j == 0 else cur[j - 1]
                    v, code = cell(xv, yv[tau][j], up, dg, lf)
                    cur.append(v)
                    cc.append(code)
                rows.append(cur)
                codes.append(cc)
                above, dg0 = cur, left[rr]
            alast[tau] = [rows[rr][W - 1] for rr in range(RT - 1)]
            prev[tau] = rows[RT - 1]
            diag[tau] = left[RT - 1]
            for rr in range(RT):
                i = RT * pt + rr
                if i >= n:
                    continue
                for j in range(W):
                    if b0 + j < M:
                        D[(i, b0 + j)] = (rows[rr][j], B[tau], codes[rr][j])
                if i == n - 1:
                    for j in range(W):
                        if b0 + j < M:
                            v = r32(rows[rr][j] + B[tau])
                            if v < best:
                                best, best_col = v, b0 + j
            if tau % 32 == 31:
                e = (alast[tau] + [prev[tau][W - 1]], B[tau])
                if tau // 32 < pl.P - 1:
                    ring[(tau // 32 + 1, t)] = e
                else:
                    colbuf[pt] = e
        for tau in range(L):
            p[tau] += 1
            if p[tau] == pl.Pp:
                p[tau] = 0
                s[tau] += 1
    return {"D": D, "frontier": frontier, "colck": colck, "cost": best, "end": best_col, "x": xs, "y": ys,
            "triggers": triggers}


def model_replay(fw, pl, c, b):
    """Recompute band (c, b) from its checkpoints, strip by strip, row by row
    (the backward's replay, without its lane layout):
    {(i, j): (value, base, walk-back choice)}."""
    n, M, W, RT, K = pl.n, pl.M, pl.W, pl.RT, pl.K
    c0 = b * K
    s, tau0, nstrip = c0 // pl.S, (c0 % pl.S) // W, K // W
    out = {}
    info = []
    for d in range(nstrip):
        tau = tau0 + d
        ps = c * pl.KS - pl.lag[tau] - s * pl.Pp
        r0, r1 = RT * max(0, ps), min(n, RT * min(pl.nt, ps + pl.KS))
        if ps > pl.nt:
            info.append((ps, r0, r1, 0.0, None))   # finished before this band
            continue
        if ps >= 1:
            # the strip's state after tile ps-1; with ps == nt its band is empty
            # but its last tile's right-hand cells feed the next strip
            pr, al, dg, Bd = frontier_state(fw, pl, c, tau)
            edge = al + [pr[W - 1]]          # rows RT*(ps-1) .. RT*ps-1, last column
        else:
            pr, dg, Bd, edge = [0.0] * W, 0.0, 0.0, None
        info.append((ps, r0, r1, Bd, edge))
        cols = [c0 + d * W + k for k in range(W)]
        yv = [fw["y"][j] if j < M else 0.0 for j in cols]
        above = pr
        Btile, dltile = Bd, 0.0
        for r in range(r0, r1):
            tile_start = r % RT == 0
            if tile_start:
                Btile = Bd                   # the tile's left inputs are converted into this base
            if d == 0:
                lf = INF if b == 0 else fw["colck"][(b, r)]
            else:
                ps_l, r0_l, _, B_l, edge_l = info[d - 1]
                if r >= r0_l:
                    v, B_src, _ = out[(r, c0 + d * W - 1)]
                else:
                    v, B_src = edge_l[r - RT * (ps_l - 1)], B_l
                lf = r32(v + r32(B_src - Btile))
            if tile_start:
                # the forward's rebase to a far lower left input, decided on the tile's first row
                dltile = 0.0
                shift = rebase_to_left(Bd, lf)
                if shift:
                    Bd, dltile = shift
                    above = [r32(u - dltile) for u in above]
                    dg = r32(dg - dltile)
            if dltile != 0.0:
                lf = r32(lf - dltile)
            cur = []
            for k in range(W):
                up = above[k]
                dgk = dg if k == 0 else above[k - 1]
                lfk = lf if k == 0 else cur[k - 1]
                v, code = cell(fw["x"][r], yv[k], up, dgk, lfk)
                cur.append(v)
                out[(r, cols[k])] = (v, Bd, code)
            above, dg = cur, lf
    return out


CASES = [
    # (P, W, RT, n, M)
    (2, 4, 2, 150, 700),    # two warps, three sweeps
    (2, 4, 4, 151, 700),    # 4-row tiles, ragged last tile
    (1, 8, 2, 70, 900),     # one warp, query shorter than the chain lag (padded period)
    (2, 4, 4, 9, 333),      # tiny query
    (3, 4, 2, 61, 1500),    # three warps, partial last sweep
    (1, 4, 2, 160, 600),    # sweep period equal to the query's tiles (no idle steps)
    (1, 4, 4, 299, 500),    # the same with 4-row tiles and a ragged last tile
    (2, 4, 8, 151, 700),    # 8-row tiles, ragged last tile
    (1, 8, 8, 64, 900),     # 8-row tiles, the query shorter than the chain lag
]


def _setup(P, W, RT, n, M, seed, KS=K_CHUNK):
    rng = np.random.default_rng(seed)
    y = np.cumsum(rng.standard_normal(M))
    y = (y - y.mean()) / y.std()
    o = int(rng.integers(0, max(1, M - n)))
    x = y[o:o + n] if o + n <= M else rng.standard_normal(n)
    x = x + 0.1 * rng.standard_normal(n)
    x = (x - x.mean()) / (x.std() or 1.0)
    pl = Plan(n, M, P, W, RT, 8 * W, KS)
    return pl, model_forward(x, y, pl)


@pytest.mark.parametrize("KS", STRIDES)
@pytest.mark.parametrize("P,W,RT,n,M", CASES)
def test_band_replay_is_bit_exact(P, W, RT, n, M, KS):
    pl, fw = _setup(P, W, RT, n, M, seed=n * 7 + M, KS=KS)
    D = fw["D"]
    assert len(D) == n * M
    covered = {}
    for c in range(pl.ckpts):
        for b in range(-(-M // pl.K)):
            for key, val in model_replay(fw, pl, c, b).items():
                if key[1] >= M:
                    continue
                assert key not in covered, f"cell {key} in bands {covered[key]} and {(c, b)}"
                covered[key] = (c, b)
                assert val == D[key], f"band {(c, b)} cell {key}: {val} != {D[key]}"
    assert len(covered) == n * M
    for (i, j), cb in covered.items():
        assert pl.band_of(i, j) == cb


def _walk(code_of, n, end):
    """The walk-back from (n-1, end) following each cell's recorded choice;
    column 0 goes up and the walk stops at row 0."""
    i, j, path = n - 1, end, [(n - 1, end)]
    while i > 0:
        c = UP if j == 0 else code_of(i, j)
        if c == DIAG:
            i, j = i - 1, j - 1
        elif c == LEFT:
            j -= 1
        else:
            i -= 1
        path.append((i, j))
    return path


@pytest.mark.parametrize("KS", STRIDES)
@pytest.mark.parametrize("P,W,RT,n,M", CASES[:3])
def test_walk_through_bands_matches_full_matrix(P, W, RT, n, M, KS):
    pl, fw = _setup(P, W, RT, n, M, seed=n * 11 + M, KS=KS)
    full = _walk(lambda i, j: fw["D"][(i, j)][2], n, fw["end"])
    cache = {}

    def banded_code(i, j):
        cb = pl.band_of(i, j)
        if cb not in cache:
            cache[cb] = model_replay(fw, pl, *cb)
        return cache[cb][(i, j)][2]

    banded = _walk(banded_code, n, fw["end"])
    assert banded == full
    assert len(cache) > 1
    # the replay reaches the forward's cost at the end cell
    v, Bv, _ = model_replay(fw, pl, *pl.band_of(n - 1, fw["end"]))[(n - 1, fw["end"])]
    assert r32(v + Bv) == fw["cost"]


# ---------------------------------------------------------------------------
# The backward kernel's own schedule (csrc/sdtw_backward.cu bwd_band_kernel),
# transliterated: the flat checkpoint layouts the forward writes, the warp's
# 32 lanes (four per strip, W/4 columns each, one tile of rows per step, lane l
# one step behind lane l-1),
# the per-lane band bounds, and the cooperative walk with its band exits.

def flat_checkpoints(fw, pl):
    """The forward's checkpoint arrays in their device layouts (one query)."""
    W, RT, L = pl.W, pl.RT, pl.L
    E = record_floats(RT)
    fr = np.full(pl.ckpts * L * (W + E), np.nan)
    for (c, tau), (prev, alast, diag, B) in fw["frontier"].items():
        base = c * L * (W + E)
        for k in range(W // 4):                       # float4 [W/4][L]: prev
            for e in range(4):
                fr[base + (k * L + tau) * 4 + e] = prev[4 * k + e]
        rec = (alast + [diag, B] + [0.0] * 8)[:E]     # float4 [E/4][L]: record
        for e in range(E):
            fr[base + ((W // 4 + e // 4) * L + tau) * 4 + e % 4] = rec[e]
    nwin = -(-pl.M // pl.K)
    rows = ck_rows(pl.n)
    ck = np.full(max(0, nwin - 1) * rows, np.nan)
    for (b, i), v in fw["colck"].items():
        ck[(b - 1) * rows + i] = v
    return fr, ck


def record_floats(RT):
    """Floats of a thread's checkpoint record (csrc/sdtw_internal.h
    fwd_record_floats): RT-1 right-hand cells, diag and base, in float4s."""
    return {2: 4, 4: 8, 8: 12}[RT]


def ck_rows(n):
    """Rows of a window's boundary column (csrc/sdtw_internal.h ck_rows):
    padded to a multiple of 8, so an 8-row tile's store stays in its window."""
    return -(-n // 8) * 8


def rows_per_step(RT):
    """Rows a lane advances per step (csrc/sdtw_backward.cu rows_per_step)."""
    return 2


def kernel_backward(fw, pl, end, RS=None):
    """The warp's walk from (n-1, end) with RS rows per lane step: (cells of
    the path, recomputed D at the end cell, number of bands)."""
    RS = rows_per_step(pl.RT) if RS is None else RS
    n, M, W, RT, L, S, Pp, nt = pl.n, pl.M, pl.W, pl.RT, pl.L, pl.S, pl.Pp, pl.nt
    WB, KW, KC = W // 4, 32 * (W // 4), pl.KS     # KC: a band's height in steps
    E = record_floats(RT)
    fr, ck = flat_checkpoints(fw, pl)
    xs, ys_all = fw["x"], fw["y"]
    lag = lambda tau: (tau >> 5) * (32 + K_CHUNK) + (tau & 31)  # noqa: E731
    wi, wj = n - 1, end
    cells, first, v_end, bands = [], True, None, 0
    done = False
    while not done:
        bands += 1
        b = wj // KW
        c0 = b * KW
        s = c0 // S
        tau0 = (c0 - s * S) // W
        lag0 = lag(tau0)
        dj = (wj - c0) // W
        c = (wi // RT + lag0 + dj + s * Pp) // KC
        ps0 = c * KC - lag0 - s * Pp
        rtop = RT * (ps0 - 7)
        assert RT * max(0, ps0 - dj) <= wi < min(n, RT * min(nt, ps0 - dj + KC)), "cell outside its band"
        rf0 = RT * max(0, ps0)
        re0 = min(min(n, RT * min(nt, ps0 + KC)), wi + 1)
        ys = [ys_all[c0 + k] if c0 + k < M else 0.0 for k in range(KW)]
        lcol = [ck[(b - 1) * ck_rows(n) + rf0 + k] for k in range(re0 - rf0)] if b > 0 else []
        frc = c * L * (W + E)
        redo = (c * KC) % pl.R == 0       # a rebase was due at the band's first step
        rb = (lambda B0, f: rebase(B0, f)) if redo else (lambda B0, f: (B0, 0.0))  # noqa: E731
        fr_at = lambda j, th: fr[frc + ((j >> 2) * L + th) * 4 + (j & 3)]             # noqa: E731
        rec_at = lambda e, th: fr[frc + (((W >> 2) + (e >> 2)) * L + th) * 4 + (e & 3)]  # noqa: E731
        lanes = []
        for lane in range(32):
            d, sub = lane >> 2, lane & 3
            ps = ps0 - d
            st = dict(d=d, sub=sub, ps=ps, rf=RT * max(0, ps), re=min(n, RT * min(nt, ps + KC)),
                      rf_left=RT * max(0, ps + 1), e=[0.0] * RT, dd=0.0)
            tau = tau0 + d
            if 1 <= ps <= nt:
                Bn, dl = rb(rec_at(RT, tau), fr_at(0, tau))
                st["D"] = [r32(fr_at(sub * WB + k, tau) - dl) for k in range(WB)]
                st["B"] = Bn
                st["dg"] = r32((rec_at(RT - 1, tau) if sub == 0 else fr_at(sub * WB - 1, tau)) - dl)
            else:
                st["D"], st["B"], st["dg"] = [0.0] * WB, 0.0, 0.0
            st["bsrc"] = 0.0
            if sub == 0 and d >= 1:
                if 1 <= ps + 1 <= nt:
                    st["bsrc"], dl = rb(rec_at(RT, tau - 1), fr_at(0, tau - 1))
                    e = [rec_at(h, tau - 1) for h in range(RT - 1)] + [fr_at(W - 1, tau - 1)]
                    st["e"] = [r32(v - dl) for v in e]
            st["btile"], st["dltile"] = st["B"], 0.0
            st["y"] = ys[lane * WB:(lane + 1) * WB]
            lanes.append(st)
        # lane l handles rows r .. r+RS-1 (r - rtop a multiple of RS, inside one
        # tile) at step (r - rtop) / RS + l; rows at or below its band end are
        # computed too (from a left input of +inf, or the neighbour's equally
        # invalid rows, and a query sample of 0) but never read.  After each
        # step D holds the step's last row, except in the first band, where it
        # holds the last valid row (the end cell's row) for the check below.
        steps = (wi - rtop) // RS + 4 * dj + 4   # strips right of wj's are not needed
        dirs = {}
        for st in lanes:
            st["last"] = [0.0] * RS
        # the kernel starts at the earliest step at which some lane has rows
        sg0 = min((st["rf"] - rtop) // RS + lane if st["rf"] < min(st["re"], wi + 1) else steps
                  for lane, st in enumerate(lanes))
        for sg in range(sg0, steps):
            recv = [lanes[max(0, lane - 1)]["last"][:] for lane in range(32)]
            brecv = [lanes[max(0, lane - 1)]["B"] for lane in range(32)]
            for lane, st in enumerate(lanes):
                r = rtop + RS * (sg - lane)
                hi = min(st["re"], wi + 1)
                if not (st["rf"] <= r < hi):
                    continue
                v = min(RS, hi - r)            # valid rows of this step
                tile_start = r % RT == 0
                if st["sub"] != 0 and brecv[lane] != st["B"]:
                    # the strip's first lane rebased at these rows: follow it
                    dl = r32(brecv[lane] - st["B"])
                    st["D"] = [r32(u - dl) for u in st["D"]]
                    st["dg"] = r32(st["dg"] - dl)
                    st["B"] = brecv[lane]
                if tile_start:
                    st["btile"] = st["B"]
                from_rec = r < st["rf_left"]
                dconv = r32((st["bsrc"] if from_rec else brecv[lane]) - st["btile"])
                lefts = []
                for h in range(RS):
                    rr = r + h
                    if st["sub"] != 0:
                        lefts.append(recv[lane][h])
                    elif st["d"] == 0:
                        lefts.append(INF if (b == 0 or h >= v) else lcol[rr - rf0])
                    else:
                        src = recv[lane][h] if not from_rec else st["e"][rr - RT * st["ps"]]
                        lefts.append(r32(src + dconv))
                if st["sub"] == 0:
                    if tile_start:
                        st["dltile"] = 0.0
                        shift = rebase_to_left(st["B"], lefts[0])
                        if shift:
                            st["B"], st["dltile"] = shift
                            st["D"] = [r32(u - st["dltile"]) for u in st["D"]]
                            st["dg"] = r32(st["dg"] - st["dltile"])
                    if st["dltile"] != 0.0:
                        lefts = [r32(u - st["dltile"]) for u in lefts]
                xv = [xs[r + h] if h < v else 0.0 for h in range(RS)]
                ls = lefts[:]
                dgs = [st["dg"]] + lefts[:-1]  # row h's diagonal at the strip's first column
                codes = [[] for _ in range(RS)]
                for k in range(WB):
                    up = st["D"][k]
                    rows = []
                    for h in range(RS):
                        nv, cd = cell(xv[h], st["y"][k], up, dgs[h], ls[h])
                        codes[h].append(cd)
                        dgs[h], ls[h] = up, nv
                        up = nv
                        rows.append(nv)
                    st["D"][k] = rows[v - 1] if first else rows[RS - 1]
                st["last"] = ls[:]
                st["dg"] = lefts[RS - 1]
                for h in range(RS):
                    # the kernel's shared choice buffer holds RT*kChunk + 7*RT + 32*RS rows
                    assert 0 <= RS * sg + h < RT * KC + 7 * RT + 32 * RS, (sg, h)
                    dirs[(RS * sg + h, lane)] = codes[h]
        if first:
            lj, kj = (wj - c0) // WB, (wj - c0) % WB
            v_end = r32(lanes[lj]["D"][kj] + lanes[lj]["B"])
            first = False
        # the walk, 32 cells of a row at a time
        while True:
            # the kernel's per-row gradient shares: RT*kChunk + 7*RT rows from rtop
            assert 0 <= wi - rtop < RT * KC + 7 * RT, (wi, rtop)
            if wi == 0:
                cells.append((0, wj))
                done = True
                break
            codes = []
            for lane in range(32):
                jk, code = wj - lane, 3
                if jk >= c0:
                    cc = jk - c0
                    lam = cc // WB
                    if wi >= RT * max(0, ps0 - (lam >> 2)):
                        code = UP if jk == 0 else dirs[(wi - rtop + RS * lam, lam)][cc - lam * WB]
                codes.append(code)
            f = next((k for k in range(32) if codes[k] != LEFT), 32)
            fcode = codes[f] if f < 32 else LEFT
            last = f - 1 if fcode == 3 else (f if f < 32 else 31)
            cells.extend((wi, wj - k) for k in range(last + 1))
            if f < 32 and fcode != 3:
                jl = wj - last
                wi -= 1
                wj = jl - 1 if fcode == DIAG else jl
            else:
                wj -= last + 1
            if wj < c0 or wi < RT * max(0, ps0 - (wj - c0) // W):
                break
    # a cell of a row can be listed twice (the row's end and the next start)
    out = []
    for cl in cells:
        if not out or out[-1] != cl:
            out.append(cl)
    return out, v_end, bands


KERNEL_CASES = [
    # (P, W, RT, n, M): the kernel's windows are 8 strips of W columns
    (2, 4, 2, 150, 700),
    (2, 4, 4, 151, 700),
    (1, 8, 2, 70, 900),
    (1, 4, 4, 299, 500),
    (2, 8, 4, 97, 1300),
    (1, 8, 4, 150, 800),    # the last tile holds two of the query's rows
    (2, 4, 8, 151, 700),    # 8-row tiles: the band's tilt equals the lane chain's
    (1, 8, 8, 150, 800),    # ... the last tile holds six of the query's rows
]


@pytest.mark.parametrize("KS", STRIDES)
@pytest.mark.parametrize("two_rows", [False, True])
@pytest.mark.parametrize("P,W,RT,n,M", KERNEL_CASES)
def test_kernel_band_schedule_and_walk(P, W, RT, n, M, two_rows, KS):
    """Both step heights a band of 4- or 8-row tiles can take (2 rows or the
    tile), every checkpoint stride."""
    if two_rows and RT == 2:
        pytest.skip("2-row tiles take 2-row steps")
    pl, fw = _setup(P, W, RT, n, M, seed=n * 13 + M, KS=KS)
    cells, v_end, bands = kernel_backward(fw, pl, fw["end"], RS=2 if two_rows else RT)
    assert v_end == fw["cost"]
    full = _walk(lambda i, j: fw["D"][(i, j)][2], n, fw["end"])
    assert cells == full
    assert bands > 1


def test_kernel_schedule_random_shapes():
    """Seeded random plans, shapes and step heights for the backward's lane
    schedule: the banded walk equals the walk over the whole FP32 matrix and
    the end cell is recomputed bit for bit."""
    rng = np.random.default_rng(4242)
    for _ in range(24):
        P, W, RT = int(rng.choice([1, 2])), int(rng.choice([4, 8])), int(rng.choice([2, 4, 8]))
        RS = int(rng.choice([1, 2, RT]))
        KS = int(rng.choice(STRIDES))
        n, M = int(rng.integers(1, 240)), int(rng.integers(2, 1300))
        pl, fw = _setup(P, W, RT, n, M, seed=int(rng.integers(0, 10**6)), KS=KS)
        cells, v_end, _ = kernel_backward(fw, pl, fw["end"], RS=RS)
        assert v_end == fw["cost"], (P, W, RT, RS, KS, n, M)
        assert cells == _walk(lambda i, j: fw["D"][(i, j)][2], n, fw["end"]), (P, W, RT, RS, KS, n, M)


def _stretched(seed, M=1400, step=8, n=150, scale=8.0):
    """A query that is the reference subsampled by `step` (plus a little noise):
    its optimal path runs horizontally for about `step` columns per row, so
    cheap values cross strips whose own cells are far more expensive -- the
    case the forward's rebase to a low left input exists for.  Both series are
    scaled by `scale` so that costs reach the rebase threshold on a small case."""
    rng = np.random.default_rng(seed)
    y = np.cumsum(rng.standard_normal(M))
    y = (y - y.mean()) / y.std()
    x = y[100:100 + step * n:step] + 0.05 * rng.standard_normal(n)
    return scale * (x - x.mean()) / x.std(), scale * y


@pytest.mark.parametrize("KS", STRIDES)
@pytest.mark.parametrize("P,W,RT", [(1, 4, 2), (2, 4, 4), (1, 8, 4), (1, 4, 8)])
def test_rebase_to_low_left_inputs_is_replayed(P, W, RT, KS):
    """With many rebases to low left inputs: every band replays bit for bit,
    and the lane schedule's walk equals the walk over the whole FP32 matrix."""
    for k in range(6):   # the first seeded input on which the forward rebases to a left input
        x, y = _stretched(seed=10 * W + RT + KS + 1000 * k)
        pl = Plan(len(x), len(y), P, W, RT, 8 * W, KS)
        fw = model_forward(x, y, pl)
        if fw["triggers"] > 0:
            break
    assert fw["triggers"] > 0
    for c in range(pl.ckpts):
        for b in range(-(-pl.M // pl.K)):
            for key, val in model_replay(fw, pl, c, b).items():
                if key[1] < pl.M:
                    assert val == fw["D"][key], (c, b, key)
    cells, v_end, _ = kernel_backward(fw, pl, fw["end"])
    assert v_end == fw["cost"]
    assert cells == _walk(lambda i, j: fw["D"][(i, j)][2], pl.n, fw["end"])


def _dir_rows(RT, KS, RS=2):
    """The band-slot size the library reserves (bwd_dir_rows in the backward):
    RS rows per step from the earliest first step (RT*7/RS) to the latest last
    step of a band (over every entry strip dj)."""
    most = max((RT * (KS + 7 - dj) - 1) // RS + 4 * dj + 4 for dj in range(8))
    return RS * (most - RT * 7 // RS)


@pytest.mark.parametrize("RT", [2, 4, 8])
@pytest.mark.parametrize("KS", STRIDES)
def test_band_slot_rows_bound(RT, KS):
    # the backward's lane schedule for a band: lane l (strip d = l // 4) has rows
    # [rf, hi) and handles row r at step (r - rtop) / RS + l; the band starts at
    # the first step any lane has a row (sg0) and, for an entry cell (wi, strip
    # dj), ends after the last step at which a lane of strips 0..dj has one
    # (the walker: dj = the entry strip; a helper: dj = 7).  Every band of every
    # geometry must fit the reserved rows, and the bound must be reached.
    RS = 2
    bound, worst = _dir_rows(RT, KS), 0
    for n in (1, 37, 64, 2000):
        nt = (n + RT - 1) // RT
        for ps0 in range(-KS - 3, min(nt, 3 * KS) + 3):
            rtop = RT * (ps0 - 7)
            for wi in range(max(0, rtop), min(n, RT * (ps0 + KS + 1))):
                inside = [RT * max(0, ps0 - d) <= wi < min(n, RT * min(nt, ps0 - d + KS)) for d in range(8)]
                for dj in [d for d in range(8) if inside[d]] + ([7] if any(inside) else []):
                    firsts, lasts = [], []
                    for lane in range(32):
                        d = lane >> 2
                        rf = RT * max(0, ps0 - d)
                        hi = min(min(n, RT * min(nt, ps0 - d + KS)), wi + 1)
                        if rf < hi:
                            firsts.append((rf - rtop) // RS + lane)
                            if d <= dj:
                                lasts.append((hi - 1 - rtop) // RS + lane)
                    steps = 1 + (max(lasts) if lasts else 0)
                    sg0 = min(firsts) if firsts else steps
                    need = RS * max(0, steps - sg0)
                    assert need <= bound, (RT, KS, n, ps0, wi, dj, need, bound)
                    worst = max(worst, need)
    assert worst == bound


# ---------------------------------------------------------------------------
# The band recompute's two-row lane step (csrc/sdtw_backward.cu tile_rows) runs
# the cells (0, k) and (1, k-1) of one anti-diagonal together, their two
# multiply-adds as one f32x2 FMA.  The model below follows that order and must
# give the cell-by-cell step's values, last-column left inputs and choice bits.

def _two_row_step_by_cells(D, y, x, l, dg, v, exact):
    D, l = list(D), list(l)
    dgs = [dg, l[0]]
    nd, nu = [0, 0], [0, 0]
    for k in range(len(D)):
        up, row_v = D[k], D[k]
        for h in range(2):
            m = min(up, dgs[h], l[h])
            nd[h] |= (1 << k) if m != dgs[h] else 0
            nu[h] |= (1 << k) if m != l[h] else 0
            t = r32(x[h] - y[k])
            nv = fma32(t, t, m)
            dgs[h], l[h], up = up, nv, nv
            if exact and h < v:
                row_v = nv
        D[k] = row_v if exact else up
    return D, l, nd, nu


def _two_row_step_by_antidiagonals(D, y, x, l, dg, v, exact):
    D, WB = list(D), len(D)
    nd0 = nu0 = nd1 = nu1 = 0
    g0, l0, g1, l1 = dg, l[0], l[0], l[1]
    u0 = D[0]
    m0 = min(u0, g0, l0)
    nd0 |= 1 if m0 != g0 else 0
    nu0 |= 1 if m0 != l0 else 0
    t0 = r32(x[0] - y[0])
    g0, l0 = u0, fma32(t0, t0, m0)
    for k in range(1, WB):
        u0, u1 = D[k], l0
        m0, m1 = min(u0, g0, l0), min(u1, g1, l1)
        nd0 |= (1 << k) if m0 != g0 else 0
        nu0 |= (1 << k) if m0 != l0 else 0
        nd1 |= (1 << (k - 1)) if m1 != g1 else 0
        nu1 |= (1 << (k - 1)) if m1 != l1 else 0
        ta, tb = r32(x[0] - y[k]), r32(x[1] - y[k - 1])
        na, nb = fma32(ta, ta, m0), fma32(tb, tb, m1)   # the two lanes of one f32x2 FMA
        D[k - 1] = u1 if (exact and v < 2) else nb
        g0, l0, g1, l1 = u0, na, u1, nb
    u1 = l0
    m1 = min(u1, g1, l1)
    nd1 |= (1 << (WB - 1)) if m1 != g1 else 0
    nu1 |= (1 << (WB - 1)) if m1 != l1 else 0
    t1 = r32(x[1] - y[WB - 1])
    l1 = fma32(t1, t1, m1)
    D[WB - 1] = u1 if (exact and v < 2) else l1
    return D, [l0, l1], [nd0, nd1], [nu0, nu1]


def test_two_row_step_pairs_anti_diagonals():
    rng = np.random.default_rng(2718)
    for _ in range(3000):
        WB = int(rng.choice([2, 4, 5, 6, 7, 8]))
        ties = bool(rng.integers(0, 2))   # integer-valued inputs make exact ties common

        def vals(n, nonneg=False):
            a = rng.standard_normal(n) * 3
            a = np.round(a) if ties else a
            return [r32(abs(float(t)) if nonneg else float(t)) for t in a]
        D, y, x, l = vals(WB, True), vals(WB), vals(2), vals(2, True)
        dg = vals(1, True)[0]
        if rng.random() < 0.1:
            l[0] = INF                     # the window's first strip above the query
        v, exact = int(rng.integers(1, 3)), bool(rng.integers(0, 2))
        a = _two_row_step_by_cells(D, y, x, l, dg, v, exact)
        b = _two_row_step_by_antidiagonals(D, y, x, l, dg, v, exact)
        assert a == b, (WB, v, exact)
