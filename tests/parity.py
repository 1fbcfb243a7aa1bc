"""Parity rules shared by the GPU tests (FP32 against the FP64/int64 oracle).

Cost: |c_gpu - c_oracle| <= 1e-5 * |c_oracle| + 1e-6 * N (the absolute term
only matters for costs near zero, e.g. exact cuts).  End column: equal to the
oracle's, or a column whose oracle value D(N-1, g) is within the same
tolerance of the optimum (the oracle's best two costs are then tied within
FP32 resolution).  Integer mode: bit-exact cost and end.
"""
import numpy as np

import oracle

RTOL = 1e-5


def cost_tol(c_oracle, n):
    return RTOL * np.abs(c_oracle) + 1e-6 * n


def check_forward_f32(ref, queries_of, idx, cost, end, threads=None):
    """Compare the GPU (cost, end) of the queries in idx with the oracle."""
    ref64 = np.asarray(ref, dtype=np.float64)
    qs = [np.asarray(queries_of(q), dtype=np.float64) for q in idx]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=threads or oracle.default_threads()) as ex:
        res = list(ex.map(lambda x: oracle.forward(x, ref64, last_row=True), qs))
    bad = []
    for k, q in enumerate(idx):
        oc, oe, row = res[k]
        n = len(qs[k])
        c, e = float(cost[q]), int(end[q])
        if not abs(c - oc) <= cost_tol(oc, n):
            bad.append((q, "cost", c, oc))
        if e != oe and not (0 <= e < len(row) and abs(row[e] - oc) <= cost_tol(oc, n)):
            bad.append((q, "end", e, oe))
    return bad


def check_forward_i8(ref, queries_of, idx, cost, end, threads=None):
    """Bit-exact comparison of int32 costs and end columns with the int64 oracle."""
    ref64 = np.asarray(ref, dtype=np.int64)
    qs = [np.asarray(queries_of(q), dtype=np.int64) for q in idx]
    from concurrent.futures import ThreadPoolExecutor
    with ThreadPoolExecutor(max_workers=threads or oracle.default_threads()) as ex:
        res = list(ex.map(lambda x: oracle.forward(x, ref64), qs))
    return [(q, int(cost[q]), res[k][0], int(end[q]), res[k][1]) for k, q in enumerate(idx)
            if int(cost[q]) != res[k][0] or int(end[q]) != res[k][1]]
