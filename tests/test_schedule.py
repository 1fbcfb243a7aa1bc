"""CPU model of the forward kernel's schedule (paper Section 5.2 wavefront).

The CUDA forward (csrc/sdtw_forward.cu) runs a chain of 32*P threads, each
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


def simulate_forward(x, y, P, W, K=None):
    n, M = len(x), len(y)
    L, S = 32 * P, 32 * P * W
    nsw = -(-M // S)
    lane_ids = np.arange(L)
    warp, lane = lane_ids // 32, lane_ids % 32
    lag = warp * (32 + K_CHUNK) + lane
    lag_last = (P - 1) * (32 + K_CHUNK) + 31
    npairs = (n + 1) // 2
    lastp = npairs - 1
    Pp = max(npairs, lag_last + K_CHUNK)
    total = (nsw - 1) * Pp + npairs + lag_last
    xs = np.concatenate([x, [0.0] * (2 * npairs - n)])
    chunk = lambda t: t // K_CHUNK  # noqa: E731  (barrier after every K_CHUNK steps)

    INF = np.inf
    prev = np.zeros((L, W))        # latest row of each strip
    a_last = np.zeros(L)           # right-hand cell of the pair's first row
    yv = np.zeros((L, W))
    diag = np.zeros(L)
    p = -lag.copy()
    s = np.zeros(L, dtype=np.int64)
    base = lane_ids * W
    ring = np.zeros((P, K_RING, 2))
    ring_w = np.full((P, K_RING), -10**9)
    ring_r = np.full((P, K_RING), -10**9)
    col = np.zeros((npairs, 2))
    col_w = np.full(npairs, -10**9)
    col_r = np.full(npairs, -10**9)
    last_row = np.full(M, np.nan)
    ckpt = {}
    fast_chunks = 0
    for t in range(total):
        if t % K_CHUNK == 0:
            for w in range(P):
                gmin = t - w * (32 + K_CHUNK) - 31
                gmax = t - w * (32 + K_CHUNK) + K_CHUNK - 1
                fast = gmin >= 0
                if fast:
                    sw = gmin // Pp
                    fast = gmax // Pp == sw and sw < nsw and gmin - sw * Pp >= 1 and gmax - sw * Pp <= lastp - 1
                if fast:
                    fast_chunks += 1
                    for u in range(K_CHUNK):
                        for l in range(32 * w, 32 * w + 32):
                            pp = p[l] + u
                            assert 1 <= pp <= lastp - 1 and s[l] < nsw, "fast path admitted a special step"
        send = np.stack([a_last, prev[:, W - 1]], axis=1)
        recv = np.roll(send, 1, axis=0)
        act = (p >= 0) & (p < npairs) & (s < nsw)
        for l in np.nonzero(lane == 0)[0]:
            w = warp[l]
            if w > 0:
                slot = (t - K_CHUNK - 1) & (K_RING - 1)
                if act[l]:
                    assert ring_w[w, slot] == t - K_CHUNK - 1, "ring read of a different pair"
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
        for l in np.nonzero(act)[0]:
            if p[l] == 0:
                base[l] = s[l] * S + l * W
                cols = base[l] + np.arange(W)
                yv[l] = np.where(cols < M, y[np.minimum(cols, M - 1)], 0.0)
                prev[l] = 0.0
                diag[l] = 0.0
            x0, x1 = xs[2 * p[l]], xs[2 * p[l] + 1]
            left0, left1 = recv[l]
            A = np.zeros(W)
            for k in range(W + 1):          # the tile's anti-diagonals, in kernel order
                if k < W:
                    up = prev[l, k]
                    dg = diag[l] if k == 0 else prev[l, k - 1]
                    lf = left0 if k == 0 else A[k - 1]
                    d = x0 - yv[l, k]
                    A[k] = d * d + min(up, dg, lf)
                if k >= 1:
                    j = k - 1
                    up = A[j]
                    dg = left0 if j == 0 else A[j - 1]
                    lf = left1 if j == 0 else prev[l, j - 1]
                    d = x1 - yv[l, j]
                    prev[l, j] = d * d + min(up, dg, lf)
            a_last[l] = A[W - 1]
            diag[l] = left1
            if p[l] == lastp:
                row = A if n % 2 else prev[l]
                for k in range(W):
                    if base[l] + k < M:
                        last_row[base[l] + k] = row[k]
            if lane[l] == 31:
                edge = (A[W - 1], prev[l, W - 1])
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
                    ckpt[(e // K - 1, 2 * p[l])] = A[W - 1]
                    if 2 * p[l] + 1 < n:
                        ckpt[(e // K - 1, 2 * p[l] + 1)] = prev[l, W - 1]
                if (2 * p[l] + 2) % K == 0 and 2 * p[l] + 1 < n:
                    for k in range(W):
                        if base[l] + k < M:
                            ckpt[("row", (2 * p[l] + 2) // K - 1, base[l] + k)] = prev[l, k]
        p += 1
        wrap = p == Pp
        p[wrap] = 0
        s[wrap] += 1
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


@pytest.mark.parametrize("P,W,n,M", CASES)
def test_schedule_reproduces_last_row(oracle_mod, P, W, n, M):
    rng = np.random.default_rng(100 * P + 10 * W + n)
    x = rng.standard_normal(n)
    y = rng.standard_normal(M)
    last_row, _, fast = simulate_forward(x, y, P, W)
    c, e, row = oracle_mod.forward(x, y, last_row=True)
    if n > 300:
        assert fast > 0
    assert not np.isnan(last_row).any()
    assert np.array_equal(last_row, row)
    assert np.min(last_row) == c and int(np.argmin(last_row)) == e


def test_schedule_checkpoints(oracle_mod):
    # K = 16 columns with W = 4: every fourth thread's strip edge is a checkpoint
    w = inputs.tiny(B=1, N=24, M=300, seed=5)
    x = w.query(0).astype(np.float64)
    y = w.ref.astype(np.float64)
    K = 16
    _, ck, _ = simulate_forward(x, y, 2, 4, K=K)
    rows = {k: v for k, v in ck.items() if k[0] == "row"}
    assert len(ck) - len(rows) == (len(y) // K) * len(x)
    assert len(rows) == (len(x) // K) * len(y)
    for m in range(len(x) // K):
        i = (m + 1) * K - 1
        _, _, row = oracle_mod.forward(x[:i + 1], y, last_row=True)
        assert all(rows[("row", m, j)] == row[j] for j in range(len(y)))
    for b in (0, 3, len(y) // K - 1):
        col = (b + 1) * K - 1
        for i in (0, 7, len(x) - 1):
            # D(i, col): last row of the query prefix x[:i+1] at column col
            _, _, row = oracle_mod.forward(x[:i + 1], y[:col + 1], last_row=True)
            assert ck[(b, i)] == row[col]
