"""CPU model of the forward kernel's schedule (paper Section 5.2 wavefront).

The CUDA forward (csrc/sdtw_forward.cu) runs a chain of 32*P threads, each
owning W reference columns; thread l lags thread l-1 by one step inside a
warp, warp w lags warp w-1 by 32 + kChunk steps, values cross warps through a
ring of kRing shared-memory slots and cross sweeps through a column buffer,
with one CTA barrier after every kChunk steps.  This test replays exactly
that index arithmetic step by step (numpy over threads) and checks, for many
shapes including ragged tails, tiny queries and short references:

* every shared-memory read sees the value written for the same query row by
  the producer thread, written in an earlier barrier interval (no race);
* no slot is overwritten before its reader's barrier interval has passed;
* the bottom row it produces equals the oracle's last DP row exactly
  (float64 arithmetic), and the (cost, end) reduction matches;
* checkpoint columns land at the documented offsets with the DP's values.

It exercises the schedule, not the CUDA code; the GPU tests cover the latter.
"""
import numpy as np
import pytest

from paper_2403_06931_gb300 import inputs

K_CHUNK = 16   # csrc/sdtw_internal.h kChunk
K_RING = 64    # csrc/sdtw_internal.h kRing


def simulate_forward(x, y, P, W, K=None):
    n, M = len(x), len(y)
    L, S = 32 * P, 32 * P * W
    nsw = -(-M // S)
    lane_ids = np.arange(L)
    warp, lane = lane_ids // 32, lane_ids % 32
    lag = warp * (32 + K_CHUNK) + lane
    lag_last = (P - 1) * (32 + K_CHUNK) + 31
    Np = max(n, lag_last + K_CHUNK)
    total = (nsw - 1) * Np + n + lag_last
    chunk = lambda t: t // K_CHUNK  # noqa: E731  (barrier after every K_CHUNK steps)

    INF = np.inf
    D = np.zeros((L, W))
    yv = np.zeros((L, W))
    diag = np.zeros(L)
    r = -lag.copy()
    s = np.zeros(L, dtype=np.int64)
    base = lane_ids * W
    ring_val = np.zeros((P, K_RING))
    ring_wstep = np.full((P, K_RING), -10**9)
    ring_rstep = np.full((P, K_RING), -10**9)
    col_val = np.zeros(n)
    col_wstep = np.full(n, -10**9)
    col_rstep = np.full(n, -10**9)
    last_row = np.full(M, np.nan)
    ckpt = {}
    for t in range(total):
        last = D[:, W - 1].copy()
        recv = np.roll(last, 1)
        act = (r >= 0) & (r < n) & (s < nsw)
        for l in np.nonzero(lane == 0)[0]:
            w = warp[l]
            if w > 0:
                slot = (t - K_CHUNK - 1) & (K_RING - 1)
                if act[l]:
                    assert ring_wstep[w, slot] == t - K_CHUNK - 1, "ring read of a different row"
                    assert chunk(ring_wstep[w, slot]) < chunk(t), "ring read without a barrier"
                    ring_rstep[w, slot] = t
                recv[l] = ring_val[w, slot]
            else:
                if act[l] and s[l] > 0:
                    rr = r[l]
                    assert col_wstep[rr] == (s[l] - 1) * Np + rr + lag_last, "column read of a different sweep"
                    assert chunk(col_wstep[rr]) < chunk(t), "column read without a barrier"
                    col_rstep[rr] = t
                    recv[l] = col_val[rr]
                else:
                    recv[l] = INF
        for l in np.nonzero(act)[0]:
            if r[l] == 0:
                base[l] = s[l] * S + l * W
                cols = base[l] + np.arange(W)
                yv[l] = np.where(cols < M, y[np.minimum(cols, M - 1)], 0.0)
                D[l] = 0.0
                diag[l] = 0.0
            xv = x[r[l]]
            left = recv[l]
            for k in range(W):
                up = D[l, k]
                d = xv - yv[l, k]
                nv = d * d + min(up, diag[l], left)
                diag[l] = up
                left = nv
                D[l, k] = nv
            diag[l] = recv[l]
            if r[l] == n - 1:
                for k in range(W):
                    if base[l] + k < M:
                        last_row[base[l] + k] = D[l, k]
            if lane[l] == 31:
                if warp[l] < P - 1:
                    w2, slot = warp[l] + 1, t & (K_RING - 1)
                    assert chunk(ring_rstep[w2, slot]) < chunk(t) or ring_rstep[w2, slot] < 0, "ring overwrite race"
                    assert ring_wstep[w2, slot] < 0 or ring_rstep[w2, slot] > ring_wstep[w2, slot] or \
                        ring_wstep[w2, slot] < 0, "ring value overwritten before it was read"
                    ring_val[w2, slot] = D[l, W - 1]
                    ring_wstep[w2, slot] = t
                else:
                    rr = r[l]
                    if col_wstep[rr] >= 0 and s[l] > 0:
                        assert col_rstep[rr] > col_wstep[rr], "column value overwritten before it was read"
                        assert chunk(col_rstep[rr]) < chunk(t), "column overwrite race"
                    col_val[rr] = D[l, W - 1]
                    col_wstep[rr] = t
            if K:
                edge = base[l] + W
                if edge % K == 0 and edge // K <= M // K:
                    ckpt[(edge // K - 1, r[l])] = D[l, W - 1]
        r += 1
        wrap = r == Np
        r[wrap] = 0
        s[wrap] += 1
    return last_row, ckpt


CASES = [
    # (P, W, n, M)
    (1, 4, 40, 300),     # one warp, several sweeps, ragged tail
    (2, 4, 40, 600),     # inter-warp ring, query shorter than the chain lag (padded period)
    (2, 2, 130, 700),    # query longer than the chain lag
    (3, 2, 5, 1000),     # three warps, tiny query
    (2, 4, 1, 333),      # one-row query
    (2, 8, 70, 20),      # reference shorter than one sweep
    (1, 2, 33, 1),       # one-column reference
]


@pytest.mark.parametrize("P,W,n,M", CASES)
def test_schedule_reproduces_last_row(oracle_mod, P, W, n, M):
    rng = np.random.default_rng(100 * P + 10 * W + n)
    x = rng.standard_normal(n)
    y = rng.standard_normal(M)
    last_row, _ = simulate_forward(x, y, P, W)
    c, e, row = oracle_mod.forward(x, y, last_row=True)
    assert not np.isnan(last_row).any()
    assert np.array_equal(last_row, row)
    assert np.min(last_row) == c and int(np.argmin(last_row)) == e


def test_schedule_checkpoints(oracle_mod):
    # K = 16 columns with W = 4: every fourth thread's strip edge is a checkpoint
    w = inputs.tiny(B=1, N=24, M=300, seed=5)
    x = w.query(0).astype(np.float64)
    y = w.ref.astype(np.float64)
    K = 16
    _, ck = simulate_forward(x, y, 2, 4, K=K)
    assert len(ck) == (len(y) // K) * len(x)
    for b in (0, 3, len(y) // K - 1):
        col = (b + 1) * K - 1
        for i in (0, 7, len(x) - 1):
            # D(i, col): last row of the query prefix x[:i+1] at column col
            _, _, row = oracle_mod.forward(x[:i + 1], y[:col + 1], last_row=True)
            assert ck[(b, i)] == row[col]
