"""CPU oracle for batched subsequence DTW (sDTW) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` import this package.  The CUDA library and its Python binding
never import it, and it shares no code with them.

The arithmetic lives in ``sdtw_oracle.c`` (double / int64, a plain row-by-row
loop over Eq. 1 of the paper, Section 2); this module compiles it with gcc,
loads it with ctypes and adds:

* batch drivers that run one query per worker thread (ctypes releases the GIL,
  so the threads run the C loop in parallel);
* the walk-back (Section 2) returned as a list of cells;
* warp-path helpers written from the definitions: a path's cost is the sum of
  d(x_i, y_j) = (x_i - y_j)^2 over its cells, and the gradient of that sum is
  d/dx_i = sum over the path's cells in row i of 2 (x_i - y_j), and
  d/dy_j = sum over the path's cells in column j of -2 (x_i - y_j).

Pinning: every function here is checked in ``tests/test_oracle.py`` against
brute-force enumeration of all warp paths, closed forms, invariants, worked
examples derived by hand from Eq. 1, and FP64 central differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdtw_oracle.c")
_LIB = os.path.join(_HERE, "_sdtw_oracle.so")
_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i = ctypes.POINTER(ctypes.c_int64)


def build(force: bool = False) -> str:
    """Compile sdtw_oracle.c into a shared object next to it (portable flags)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.sdtw_oracle_forward_f64.argtypes = [_d, ctypes.c_int64, _d, ctypes.c_int64, _d, _i, _d]
            lib.sdtw_oracle_forward_i64.argtypes = [_i, ctypes.c_int64, _i, ctypes.c_int64, _i, _i, _i]
            lib.sdtw_oracle_walkback_f64.argtypes = [_d, ctypes.c_int64, _d, ctypes.c_int64, ctypes.c_int64,
                                                     _i, _i, _i, _d]
            lib.sdtw_oracle_znorm_f64.argtypes = [_d, ctypes.c_int64, _d]
            lib.sdtw_oracle_forward_f16.argtypes = [_d, ctypes.c_int64, _d, ctypes.c_int64, _d, _i, _d]
            lib.sdtw_oracle_round_f16.argtypes = [_d, ctypes.c_int64, _d]
            lib.sdtw_oracle_fma_f16.argtypes = [_d, _d, _d, ctypes.c_int64, _d]
            lib.sdtw_oracle_forward_pruned_i64.argtypes = [_i, ctypes.c_int64, _i, ctypes.c_int64, ctypes.c_int64,
                                                           _i, _i]
            for f in (lib.sdtw_oracle_forward_f64, lib.sdtw_oracle_forward_i64, lib.sdtw_oracle_walkback_f64,
                      lib.sdtw_oracle_znorm_f64, lib.sdtw_oracle_forward_f16, lib.sdtw_oracle_round_f16,
                      lib.sdtw_oracle_fma_f16, lib.sdtw_oracle_forward_pruned_i64):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _p(a, t):
    return a.ctypes.data_as(t)


def _is_int(a) -> bool:
    return np.issubdtype(np.asarray(a).dtype, np.integer)


def forward(x, y, last_row: bool = False):
    """sDTW of one query against one reference.

    Integer inputs run the exact int64 loop, anything else runs in double.
    Returns (cost, end) or (cost, end, D(n-1, :)).
    """
    lib = _load()
    if _is_int(x) and _is_int(y):
        xa = np.ascontiguousarray(x, dtype=np.int64)
        ya = np.ascontiguousarray(y, dtype=np.int64)
        c, e = ctypes.c_int64(), ctypes.c_int64()
        row = np.empty(ya.shape[0], dtype=np.int64) if last_row else None
        rc = lib.sdtw_oracle_forward_i64(_p(xa, _i), xa.shape[0], _p(ya, _i), ya.shape[0],
                                         ctypes.byref(c), ctypes.byref(e),
                                         _p(row, _i) if last_row else None)
    else:
        xa = np.ascontiguousarray(x, dtype=np.float64)
        ya = np.ascontiguousarray(y, dtype=np.float64)
        c, e = ctypes.c_double(), ctypes.c_int64()
        row = np.empty(ya.shape[0], dtype=np.float64) if last_row else None
        rc = lib.sdtw_oracle_forward_f64(_p(xa, _d), xa.shape[0], _p(ya, _d), ya.shape[0],
                                         ctypes.byref(c), ctypes.byref(e),
                                         _p(row, _d) if last_row else None)
    if rc != 0:
        raise ValueError(f"oracle forward failed (code {rc}) for n={np.size(x)}, m={np.size(y)}")
    return (c.value, e.value, row) if last_row else (c.value, e.value)


PRUNED_INF = 1 << 62   # the pruned oracle's +inf


def forward_pruned(x, y, gap: int):
    """Integer sDTW with the early-INF pruning of Section 8: a cell whose
    samples differ by more than gap costs +inf, and +inf absorbs every sum.
    Returns (cost, end); cost PRUNED_INF and end -1 when every last-row cell
    is pruned away."""
    xv = np.ascontiguousarray(x, dtype=np.int64)
    yv = np.ascontiguousarray(y, dtype=np.int64)
    c = ctypes.c_int64()
    e = ctypes.c_int64()
    rc = _load().sdtw_oracle_forward_pruned_i64(_p(xv, _i), len(xv), _p(yv, _i), len(yv), int(gap),
                                                ctypes.byref(c), ctypes.byref(e))
    if rc != 0:
        raise ValueError(f"oracle pruned forward failed (code {rc})")
    return c.value, e.value


def round_f16(values):
    """Each value rounded to the nearest IEEE binary16 value (ties to even),
    as float64 (beyond 65504 by half a unit or more: +-inf)."""
    v = np.ascontiguousarray(values, dtype=np.float64).reshape(-1)
    out = np.empty_like(v)
    _load().sdtw_oracle_round_f16(_p(v, _d), len(v), _p(out, _d))
    return out.reshape(np.shape(values))


def fma_f16(a, b, c):
    """fl16(a * b + c) for binary16 values, rounded once, element by element."""
    a, b, c = (np.ascontiguousarray(np.broadcast_to(t, np.broadcast(a, b, c).shape), dtype=np.float64).reshape(-1)
               for t in (a, b, c))
    out = np.empty_like(a)
    _load().sdtw_oracle_fma_f16(_p(a, _d), _p(b, _d), _p(c, _d), len(a), _p(out, _d))
    return out


def forward_f16(x, y, last_row: bool = False):
    """sDTW in the paper's binary16 precision (Section 5.2): Eq. 1 with every
    operation rounded to binary16 (the local cost's subtraction, then one
    fused multiply-add).  x and y must hold binary16 values (e.g. float16
    arrays).  Returns (cost, end[, last row]) with the cost as a float."""
    xv = np.ascontiguousarray(x, dtype=np.float64)
    yv = np.ascontiguousarray(y, dtype=np.float64)
    c = ctypes.c_double()
    e = ctypes.c_int64()
    row = np.empty(len(yv), dtype=np.float64) if last_row else None
    rc = _load().sdtw_oracle_forward_f16(_p(xv, _d), len(xv), _p(yv, _d), len(yv), ctypes.byref(c), ctypes.byref(e),
                                         _p(row, _d) if last_row else None)
    if rc != 0:
        raise ValueError(f"oracle binary16 forward failed (code {rc}): inputs must be binary16 values")
    return (c.value, e.value, row) if last_row else (c.value, e.value)


def znormalize(x):
    """Eq. 2 z-normalisation of one series in float64 (population statistics,
    two passes; a series with zero spread is only centred)."""
    xv = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(xv)
    st = _load().sdtw_oracle_znorm_f64(_p(xv, _d), len(xv), _p(out, _d))
    if st != 0:
        raise ValueError(f"oracle znorm failed ({st})")
    return out


def znormalize_vjp(x, gz):
    """The derivative of Eq. 2 applied to a gradient, in float64.

    For z = (x - mean) / S with the population spread S (S == 0: z = x - mean),
    and g = d cost / d z, returns d cost / d x.  Differentiating mean = sum(x)/n
    and S = sqrt(sum((x - mean)^2) / n) gives d z_i / d x_k =
    (delta_ik - 1/n - z_i z_k / n) / S, hence
    d cost / d x_k = (g_k - mean(g) - z_k mean(g z)) / S; with S == 0 the
    series is only centred and the result is g - mean(g)."""
    xv = np.asarray(x, dtype=np.float64)
    g = np.asarray(gz, dtype=np.float64)
    n = xv.shape[0]
    mu = xv.sum() / n
    c = xv - mu
    var = (c * c).sum() / n
    inv = 1.0 / np.sqrt(var) if var > 0 else 1.0
    z = c * inv
    return inv * (g - g.mean() - z * (g * z).mean())


def znormalize_batch(values, offsets=None, N=None):
    """znormalize every series of a batch stored back to back ([B][N] or by offsets)."""
    v = np.asarray(values, dtype=np.float64).reshape(-1)
    out = np.empty_like(v)
    if offsets is None:
        bounds = [(i, i + N) for i in range(0, len(v), N)]
    else:
        bounds = [(int(offsets[q]), int(offsets[q + 1])) for q in range(len(offsets) - 1)]
    for a, b in bounds:
        out[a:b] = znormalize(v[a:b])
    return out


def codebook_fit(ref, sigmas: float = 4.0):
    """The reference codebook of the paper's Section 8 (future work): the bulk
    of the reference's value distribution divided evenly into the 256 uint8
    codes, outliers clamped to the extreme codes.  The bulk is read here as
    mean +- sigmas * S with the population spread S (FP64, two passes).
    Returns (lo, step): code k covers [lo + k step, lo + (k + 1) step).  A
    reference with zero spread gets step 1 and lo = mean - 128."""
    y = np.asarray(ref, dtype=np.float64)
    mu = y.sum() / y.shape[0]
    c = y - mu
    s = np.sqrt((c * c).sum() / y.shape[0])
    if not s > 0.0:
        return mu - 128.0, 1.0
    return mu - sigmas * s, 2.0 * sigmas * s / 256.0


def codebook_encode(values, lo, inv_step):
    """uint8 codes of values under a codebook: clamp(floor((x - lo) * inv_step),
    0, 255), the subtraction and the product each rounded to float32 -- the
    precision in which the library decides a code, so that both sides take
    every decision alike (lo and inv_step are float32 parameters)."""
    x = np.asarray(values, dtype=np.float32)
    t = (x - np.float32(lo)) * np.float32(inv_step)
    return np.clip(np.floor(t), 0, 255).astype(np.uint8)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def forward_batch(ref, queries, offsets=None, indices=None, threads: int | None = None,
                  last_row: bool = False):
    """Run ``forward`` for each query of a uniform [B, N] or ragged (flat, offsets) batch.

    ``indices`` restricts the run to those queries.  Returns (costs, ends) as
    arrays over the selected queries (float64 or int64 costs), plus the list of
    last rows when ``last_row`` is set.
    """
    B = (len(offsets) - 1) if offsets is not None else len(queries)
    idx = list(range(B)) if indices is None else [int(q) for q in indices]

    def one(q):
        xq = queries[offsets[q]:offsets[q + 1]] if offsets is not None else queries[q]
        return forward(xq, ref, last_row=last_row)

    with ThreadPoolExecutor(max_workers=threads or default_threads()) as ex:
        res = list(ex.map(one, idx))
    integer = _is_int(ref) and _is_int(queries)
    costs = np.array([r[0] for r in res], dtype=np.int64 if integer else np.float64)
    ends = np.array([r[1] for r in res], dtype=np.int64)
    if last_row:
        return costs, ends, [r[2] for r in res]
    return costs, ends


def walkback(x, y, end: int, max_cells: int = 200_000_000):
    """Walk-back of Section 2 from (n-1, end) over the fully filled matrix.

    Returns (cells, margins): cells is an int64 array [L, 2] of (i, j) from the
    end cell back to row 0; margins[k] is the gap between the best and the
    second-best neighbour at step k (-1 where there was no choice).
    """
    xa = np.ascontiguousarray(x, dtype=np.float64)
    ya = np.ascontiguousarray(y, dtype=np.float64)
    n, m = xa.shape[0], ya.shape[0]
    if n * m > max_cells:
        raise ValueError(f"walkback matrix {n}x{m} exceeds max_cells={max_cells}")
    cap = n + m
    pi = np.empty(cap, dtype=np.int64)
    pj = np.empty(cap, dtype=np.int64)
    mg = np.empty(cap, dtype=np.float64)
    L = ctypes.c_int64()
    rc = _load().sdtw_oracle_walkback_f64(_p(xa, _d), n, _p(ya, _d), m, int(end),
                                          _p(pi, _i), _p(pj, _i), ctypes.byref(L), _p(mg, _d))
    if rc != 0:
        raise ValueError(f"oracle walkback failed (code {rc})")
    k = L.value
    return np.stack([pi[:k], pj[:k]], axis=1), mg[:k]


# ----------------------------------------------------------- path helpers --

def path_is_valid(cells, n: int, m: int, end: int) -> bool:
    """A warp path listed from (n-1, end) back to row 0.

    Each step back moves to (i-1, j-1), (i, j-1) or (i-1, j) (Eq. 1's three
    neighbours), every cell is inside the n x m matrix, and the path stops at
    its first row-0 cell.
    """
    c = np.asarray(cells, dtype=np.int64)
    if c.ndim != 2 or c.shape[1] != 2 or c.shape[0] < 1:
        return False
    if c[0, 0] != n - 1 or c[0, 1] != end:
        return False
    if (c[:, 0] < 0).any() or (c[:, 0] >= n).any() or (c[:, 1] < 0).any() or (c[:, 1] >= m).any():
        return False
    if c[-1, 0] != 0 or (c[:-1, 0] == 0).any():
        return False
    step = c[:-1] - c[1:]
    ok = ((step == [1, 1]).all(axis=1) | (step == [0, 1]).all(axis=1) | (step == [1, 0]).all(axis=1))
    return bool(ok.all())


def path_cost(x, y, cells) -> float:
    """Sum of (x_i - y_j)^2 over the path's cells, in double."""
    c = np.asarray(cells, dtype=np.int64)
    d = np.asarray(x, dtype=np.float64)[c[:, 0]] - np.asarray(y, dtype=np.float64)[c[:, 1]]
    return float(np.sum(d * d))


def path_gradient(x, y, cells, g: float = 1.0):
    """Gradient of g * path_cost with respect to x and y (double).

    d/dx_i = g * sum over cells (i, j) of 2 (x_i - y_j);
    d/dy_j = g * sum over cells (i, j) of -2 (x_i - y_j).
    """
    xa = np.asarray(x, dtype=np.float64)
    ya = np.asarray(y, dtype=np.float64)
    c = np.asarray(cells, dtype=np.int64)
    d = 2.0 * g * (xa[c[:, 0]] - ya[c[:, 1]])
    gx = np.zeros_like(xa)
    gy = np.zeros_like(ya)
    np.add.at(gx, c[:, 0], d)
    np.add.at(gy, c[:, 1], -d)
    return gx, gy


def cells_from_intervals(lo, hi):
    """Expand a per-row column interval form [lo_i, hi_i] into cells (end first)."""
    out = []
    for i in range(len(lo) - 1, -1, -1):
        for j in range(int(hi[i]), int(lo[i]) - 1, -1):
            out.append((i, j))
    return np.asarray(out, dtype=np.int64).reshape(-1, 2)


def intervals_from_cells(cells, n: int):
    """Per-row [first column, last column] of a monotone warp path."""
    c = np.asarray(cells, dtype=np.int64)
    lo = np.full(n, -1, dtype=np.int64)
    hi = np.full(n, -1, dtype=np.int64)
    for i, j in c:
        lo[i] = j if lo[i] < 0 else min(lo[i], j)
        hi[i] = max(hi[i], j)
    return lo, hi


# ------------------------------------------------- per-row interval form --
# A monotone warp path visits, in each row i, one contiguous run of columns
# [lo_i, hi_i].  The helpers below evaluate the same definitions as
# path_is_valid / path_cost / path_gradient on that form without expanding
# the cells (the sums over a run use prefix sums of y and y^2, in double).

def intervals_are_valid(lo, hi, m: int, end: int) -> bool:
    """Runs of a valid warp path ending at (n-1, end): 0 <= lo_i <= hi_i < m,
    hi_{n-1} = end, and between rows the path steps up (lo_i = hi_{i-1}) or
    diagonally (lo_i = hi_{i-1} + 1)."""
    lo = np.asarray(lo, dtype=np.int64)
    hi = np.asarray(hi, dtype=np.int64)
    if lo.shape != hi.shape or lo.ndim != 1 or lo.size < 1:
        return False
    if (lo < 0).any() or (hi >= m).any() or (lo > hi).any() or hi[-1] != end:
        return False
    step = lo[1:] - hi[:-1]
    return bool(((step == 0) | (step == 1)).all())


def intervals_cost(x, y, lo, hi) -> float:
    """sum_i sum_{j=lo_i..hi_i} (x_i - y_j)^2 in double."""
    xa = np.asarray(x, dtype=np.float64)
    ya = np.asarray(y, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.int64)
    hi = np.asarray(hi, dtype=np.int64)
    s1 = np.concatenate([[0.0], np.cumsum(ya)])
    s2 = np.concatenate([[0.0], np.cumsum(ya * ya)])
    cnt = (hi - lo + 1).astype(np.float64)
    sy = s1[hi + 1] - s1[lo]
    syy = s2[hi + 1] - s2[lo]
    return float(np.sum(cnt * xa * xa - 2.0 * xa * sy + syy))


def intervals_gradient(x, y, lo, hi, g: float = 1.0):
    """Gradient of g * intervals_cost: d/dx_i = 2 g sum_j (x_i - y_j) over the
    row's run; d/dy_j = -2 g sum over rows whose run covers j of (x_i - y_j)."""
    xa = np.asarray(x, dtype=np.float64)
    ya = np.asarray(y, dtype=np.float64)
    lo = np.asarray(lo, dtype=np.int64)
    hi = np.asarray(hi, dtype=np.int64)
    m = ya.shape[0]
    s1 = np.concatenate([[0.0], np.cumsum(ya)])
    cnt = (hi - lo + 1).astype(np.float64)
    gx = 2.0 * g * (cnt * xa - (s1[hi + 1] - s1[lo]))
    # rows covering column j: difference arrays of the count and of sum x_i
    dc = np.zeros(m + 1)
    dx = np.zeros(m + 1)
    np.add.at(dc, lo, 1.0)
    np.add.at(dc, hi + 1, -1.0)
    np.add.at(dx, lo, xa)
    np.add.at(dx, hi + 1, -xa)
    c = np.cumsum(dc)[:m]
    sx = np.cumsum(dx)[:m]
    gy = -2.0 * g * (sx - c * ya)
    return gx, gy
