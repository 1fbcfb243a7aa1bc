"""CPU model of the forward kernel's schedule (paper Section 5.2 wavefront).

The CUDA forward (csrc/sdtw_fill.cuh) runs a chain of 32*P threads, each
owning W reference columns and advancing two query rows per step (a 2 x W
tile); thread l lags thread l-1 by one step inside a warp, warp w lags warp
w-1 by 32 + kChunk steps, tile edges cross warps through a ring of kRing
shared-memory slots and cross sweeps through a column buffer indexed by row
pair, with one CTA barrier after every kChunk steps.  Chunks in which no
thread of a warp starts a sweep, idles or meets the bottom row take a fast
path.  This test replays exactly that index arithmetic step by step (numpy
over threads) and checks, for many shapes including ragged tails, odd and tiny
queries and short references:

* every shared-memory read sees the edge written for the same row pair by the
  producer thread, written in an earlier barrier interval (no race);
* no slot is overwritten before its reader's barrier interval has passed;
* the fast-path test admits only chunks in which every thread of the warp is
  active, past its sweep's first pair and before its last pair;
* the bottom row it produces equals the oracle's last DP row exactly
  (float64 arithmetic), and the (cost, end) reduction matches;
* checkpoint columns land at the documented offsets with the DP's values.

It exercises the schedule, not the CUDA code; the GPU tests cover the latter.
"""
import numpy as np
import pytest

from paper_2403_06931_gb300 import inputs

K_CHUNK = 32   # csrc/sdtw_internal.h kChunk
K_RING = 128   # csrc/sdtw_internal.h kRing


def simulate_forward(x, y, P, W, K=None, RT=2, R=None):
    n, M = len(x), len(y)
    L, S = 32 * P, 32 * P * W
    nsw = -(-M // S)
    lane_ids = np.arange(L)
    warp, lane = lane_ids // 32, lane_ids % 32
    lag = warp * (32 + K_CHUNK) + lane
    lag_last = (P - 1) * (32 + K_CHUNK) + 31
    nt = -(-n // RT)
    lastt = nt - 1
    Pp = max(nt, lag_last + K_CHUNK)
    total = (nsw - 1) * Pp + nt + lag_last
    xs = np.concatenate([x, [0.0] * (RT * nt - n)])
    chunk = lambda t: t // K_CHUNK  # noqa: E731  (barrier after every K_CHUNK steps)
    R = R or K
    G = min(32, R // RT) if R else 32

    INF = np.inf
    prev = np.zeros((L, W))             # latest row of each strip
    a_last = np.zeros((L, RT - 1))      # right-hand cells of the tile's other rows
    yv = np.zeros((L, W))
    diag = np.zeros(L)
    p = -lag.copy()
    s = np.zeros(L, dtype=np.int64)
    base = lane_ids * W
    ring = np.zeros((P, K_RING, RT))
    ring_w = np.full((P, K_RING), -10**9)
    ring_r = np.full((P, K_RING), -10**9)
    col = np.zeros((nt, RT))
    col_w = np.full(nt, -10**9)
    col_r = np.full(nt, -10**9)
    last_row = np.full(M, np.nan)
    ckpt = {}
    stage = {}                          # row checkpoint staging: lane -> (sweep, tile, strip values)
    fast_chunks = 0
    for t in range(total):
        if t % K_CHUNK == 0:
            for w in range(P):
                gmin = t - w * (32 + K_CHUNK) - 31
                gmax = t - w * (32 + K_CHUNK) + K_CHUNK - 1
                fast = gmin >= 0
                if fast:
                    sw = gmin // Pp
                    fast = gmax // Pp == sw and sw < nsw and gmin - sw * Pp >= 1 and gmax - sw * Pp <= lastt - 1
                if fast:
                    fast_chunks += 1
                    for u in range(K_CHUNK):
                        for l in range(32 * w, 32 * w + 32):
                            pp = p[l] + u
                            assert 1 <= pp <= lastt - 1 and s[l] < nsw, "fast path admitted a special step"
        send = np.concatenate([a_last, prev[:, W - 1:W]], axis=1)
        recv = np.roll(send, 1, axis=0)
        act = (p >= 0) & (p < nt) & (s < nsw)
        for l in np.nonzero(lane == 0)[0]:
            w = warp[l]
            if w > 0:
                slot = (t - K_CHUNK - 1) & (K_RING - 1)
                if act[l]:
                    assert ring_w[w, slot] == t - K_CHUNK - 1, "ring read of a different tile"
                    assert chunk(ring_w[w, slot]) < chunk(t), "ring read without a barrier"
                    ring_r[w, slot] = t
                recv[l] = ring[w, slot]
            elif act[l] and s[l] > 0:
                pp = p[l]
                assert col_w[pp] == (s[l] - 1) * Pp + pp + lag_last, "column read of a different sweep"
                assert chunk(col_w[pp]) < chunk(t), "column read without a barrier"
                col_r[pp] = t
                recv[l] = col[pp]
            else:
                recv[l] = INF
        hits = []
        for l in np.nonzero(act)[0]:
            if p[l] == 0:
                base[l] = s[l] * S + l * W
                cols = base[l] + np.arange(W)
                yv[l] = np.where(cols < M, y[np.minimum(cols, M - 1)], 0.0)
                prev[l] = 0.0
                diag[l] = 0.0
            xr = xs[RT * p[l]:RT * p[l] + RT]
            left = recv[l]
            A = np.zeros((RT - 1, W))
            for k in range(W + RT - 1):     # the tile's anti-diagonals, in kernel order
                for rr in range(RT):
                    j = k - rr
                    if j < 0 or j >= W:
                        continue
                    if rr == 0:
                        up = prev[l, j]
                        dg = diag[l] if j == 0 else prev[l, j - 1]
                    else:
                        up = A[rr - 1, j]
                        dg = left[rr - 1] if j == 0 else A[rr - 1, j - 1]
                    lf = left[rr] if j == 0 else (prev[l, j - 1] if rr == RT - 1 else A[rr, j - 1])
                    d = xr[rr] - yv[l, j]
                    v = d * d + min(up, dg, lf)
                    if rr == RT - 1:
                        prev[l, j] = v
                    else:
                        A[rr, j] = v
            a_last[l] = A[:, W - 1]
            diag[l] = left[RT - 1]
            if p[l] == lastt:
                b = (n - 1) - RT * lastt
                row = prev[l] if b == RT - 1 else A[b]
                for k in range(W):
                    if base[l] + k < M:
                        last_row[base[l] + k] = row[k]
            if lane[l] == 31:
                edge = np.concatenate([A[:, W - 1], prev[l, W - 1:W]])
                if warp[l] < P - 1:
                    w2, slot = warp[l] + 1, t & (K_RING - 1)
                    if ring_r[w2, slot] > ring_w[w2, slot]:     # the value there was consumed:
                        assert chunk(ring_r[w2, slot]) < chunk(t), "ring overwrite race"
                    ring[w2, slot] = edge
                    ring_w[w2, slot] = t
                else:
                    pp = p[l]
                    if col_w[pp] >= 0 and s[l] > 0:
                        assert col_r[pp] > col_w[pp], "column value overwritten before it was read"
                        if P == 1:
                            # reader and writer are lanes of one warp: the per-step
                            # warp synchronisation orders the read before the write
                            assert col_r[pp] < t, "column overwrite race"
                        else:
                            assert chunk(col_r[pp]) < chunk(t), "column overwrite race"
                    col[pp] = edge
                    col_w[pp] = t
            if K:
                e = base[l] + W
                if e % K == 0 and e // K <= M // K:
                    vals = list(A[:, W - 1]) + [prev[l, W - 1]]
                    for rr in range(RT):
                        if RT * p[l] + rr < n:
                            ckpt[(e // K - 1, RT * p[l] + rr)] = vals[rr]
                if ((p[l] + 1) * RT) % R == 0 and RT * p[l] + RT - 1 < n:
                    # stage the strip; the slot must not hold a row still waiting to be written
                    assert l not in stage, "row staging slot overwritten before its row was written"
                    stage[l] = (s[l], p[l], prev[l].copy())
                    hits.append(l)
        # write out each group of G lanes whose last lane staged just now
        for l in hits:
            if lane[l] % G == G - 1:
                g0 = l - (G - 1)
                sg, pg = stage[l][0], stage[l][1]
                m = (pg + 1) * RT // R - 1
                for ll in range(g0, l + 1):
                    assert ll in stage and stage[ll][:2] == (sg, pg), "group staged different rows"
                    bcol = sg * S + ll * W
                    for k in range(W):
                        if bcol + k < M:
                            ckpt[("row", m, bcol + k)] = stage[ll][2][k]
                    del stage[ll]
        p += 1
        wrap = p == Pp
        p[wrap] = 0
        s[wrap] += 1
    assert not stage, "staged rows never written"
    return last_row, ckpt, fast_chunks


CASES = [
    # (P, W, n, M)
    (1, 4, 40, 300),     # one warp, several sweeps, ragged tail
    (2, 4, 41, 600),     # inter-warp ring, odd query shorter than the chain lag (padded period)
    (2, 2, 420, 700),    # query longer than the chain lag: fast-path chunks
    (1, 2, 301, 900),    # odd query, one warp, fast-path chunks
    (3, 2, 5, 1000),     # three warps, tiny query
    (2, 4, 1, 333),      # one-row query
    (2, 4, 2, 333),      # one pair
    (2, 8, 70, 20),      # reference shorter than one sweep
    (1, 2, 33, 1),       # one-column reference
]


@pytest.mark.parametrize("RT", [2, 4])
@pytest.mark.parametrize("P,W,n,M", CASES)
def test_schedule_reproduces_last_row(oracle_mod, P, W, n, M, RT):
    rng = np.random.default_rng(100 * P + 10 * W + n)
    x = rng.standard_normal(n)
    y = rng.standard_normal(M)
    last_row, _, fast = simulate_forward(x, y, P, W, RT=RT)
    c, e, row = oracle_mod.forward(x, y, last_row=True)
    if n > 300:
        assert fast > 0
    assert not np.isnan(last_row).any()
    assert np.array_equal(last_row, row)
    assert np.min(last_row) == c and int(np.argmin(last_row)) == e


@pytest.mark.parametrize("RT,R,N", [(2, 64, 200), (4, 64, 300), (4, 128, 301), (2, 128, 150)])
def test_schedule_checkpoints(oracle_mod, RT, R, N):
    # columns every K = 16 (W = 4: every fourth thread's strip edge), rows every
    # R; RT = 4 with R = 64 writes rows out in groups of 16 lanes
    w = inputs.tiny(B=1, N=N, M=700, seed=5)
    x = w.query(0).astype(np.float64)
    y = w.ref.astype(np.float64)
    K = 16
    _, ck, _ = simulate_forward(x, y, 2, 4, K=K, RT=RT, R=R)
    rows = {k: v for k, v in ck.items() if k[0] == "row"}
    assert len(ck) - len(rows) == (len(y) // K) * len(x)
    assert len(rows) == (len(x) // R) * len(y)
    for m in range(len(x) // R):
        i = (m + 1) * R - 1
        _, _, row = oracle_mod.forward(x[:i + 1], y, last_row=True)
        assert all(rows[("row", m, j)] == row[j] for j in range(len(y)))
    for b in (0, 5, len(y) // K - 1):
        c = (b + 1) * K - 1
        for i in (0, 33, len(x) - 1):
            _, _, row = oracle_mod.forward(x[:i + 1], y[:c + 1], last_row=True)
            assert ck[(b, i)] == row[c]
    for b in (0, 3, len(y) // K - 1):
        col = (b + 1) * K - 1
        for i in (0, 7, len(x) - 1):
            # D(i, col): last row of the query prefix x[:i+1] at column col
            _, _, row = oracle_mod.forward(x[:i + 1], y[:col + 1], last_row=True)
            assert ck[(b, i)] == row[col]


def test_schedule_random_shapes(oracle_mod):
    """Seeded random plans and shapes (lengths not multiples of the tile, the
    strip or the sweep; queries shorter than a warp; references shorter than a
    strip): every shared-memory access checked, the last row equal to the
    oracle's, the end column its first minimum."""
    rng = np.random.default_rng(2024)
    for _ in range(20):
        P, W, RT = int(rng.choice([1, 2, 3])), int(rng.choice([2, 4, 8])), int(rng.choice([2, 4]))
        n, M = int(rng.integers(1, 300)), int(rng.integers(1, 2000))
        x, y = rng.standard_normal(n), rng.standard_normal(M)
        last_row, _, _ = simulate_forward(x, y, P, W, RT=RT)
        c, e, row = oracle_mod.forward(x, y, last_row=True)
        assert np.array_equal(last_row, row), (P, W, RT, n, M)
        assert np.min(last_row) == c and int(np.argmin(last_row)) == e
