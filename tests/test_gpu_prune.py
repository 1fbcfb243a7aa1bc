"""GPU early-INF pruning (paper Section 8, opt-in) against the CPU oracle.

With prune_gap > 0 an integer-mode cell whose samples differ by more than the
gap costs +inf and +inf absorbs every sum.  The GPU's int32 costs and end
columns must equal the pruned int64 oracle's bit for bit (a query whose every
last-row cell is pruned away reports INT32_MAX and end -1), and a gap that
prunes nothing must reproduce the exact fill.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest
import torch

import oracle
from paper_2403_06931_gb300 import capi, inputs
from paper_2403_06931_gb300.sdtw import SdtwContext, codebook_encode, codebook_fit

pytestmark = pytest.mark.gpu

I32_MAX = np.iinfo(np.int32).max


def run(dev, ref, queries, dtype, gap, offsets=None, N=None, **kw):
    r = torch.from_numpy(np.ascontiguousarray(ref)).to(dev)
    q = torch.from_numpy(np.ascontiguousarray(queries)).to(dev)
    o = torch.from_numpy(offsets).to(dev) if offsets is not None else None
    B = len(offsets) - 1 if offsets is not None else queries.shape[0]
    Nmax = N if N is not None else queries.shape[1]
    ctx = SdtwContext(dtype=dtype, max_ref_len=len(ref), max_batch=B, max_query_len=Nmax,
                      max_total_query_len=max(q.numel(), 1), prune_gap=gap, **kw)
    cost, end = ctx.forward(r, q, offsets=o, N=Nmax if offsets is not None else None)
    assert ctx.device_status() == capi.SDTW_OK
    ctx.close()
    return cost.cpu().numpy(), end.cpu().numpy()


def check(ref, queries_of, idx, gap, cost, end):
    y = np.asarray(ref, dtype=np.int64)
    with ThreadPoolExecutor(max_workers=oracle.default_threads()) as ex:
        res = list(ex.map(lambda q: oracle.forward_pruned(np.asarray(queries_of(q), np.int64), y, gap), idx))
    bad = []
    for q, (c, e) in zip(idx, res):
        want = (I32_MAX, -1) if c == oracle.PRUNED_INF else (c, e)
        if (int(cost[q]), int(end[q])) != want:
            bad.append((q, int(cost[q]), int(end[q]), want))
    return bad


@pytest.mark.parametrize("gap", [1, 4, 12, 40])
@pytest.mark.parametrize("RT", [2, 4, 8])
@pytest.mark.parametrize("W", [8, 24, 32])
def test_pruned_u8_every_plan(gpu, W, RT, gap):
    if RT == 8 and not 16 <= W <= 28:
        pytest.skip("8-row tiles are built for 16 to 28 columns")
    rng = np.random.default_rng(100 + W + RT + gap)
    cref = np.clip(np.cumsum(rng.integers(-6, 7, 4000)) + 128, 0, 255).astype(np.uint8)
    cq = np.stack([cref[o:o + 90] for o in rng.integers(0, 3900, 4)]).astype(np.int64)
    cq = np.clip(cq + rng.integers(-3, 4, cq.shape), 0, 255).astype(np.uint8)
    cq[3] = 255 - cq[3]            # a query far from most of the reference: heavy pruning
    cost, end = run(gpu, cref, cq, "u8", gap, seg_width=W, tile_rows=RT, warps_per_query=2)
    assert check(cref, lambda q: cq[q], range(4), gap, cost, end) == []


def test_pruned_i8_ragged_and_fully_pruned(gpu):
    rng = np.random.default_rng(7)
    lengths = np.array([5, 0, 1, 200, 64, 33], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    ref = rng.integers(-20, 21, 3000).astype(np.int8)
    flat = rng.integers(-20, 21, int(offs[-1])).astype(np.int8)
    flat[offs[5]:offs[6]] = 127               # every cell of this query differs by more than the gap
    gap = 30
    cost, end = run(gpu, ref, flat, "i8", gap, offsets=offs, N=200)
    nz = [q for q in range(len(lengths)) if lengths[q] > 0]
    assert check(ref, lambda q: flat[offs[q]:offs[q + 1]], nz, gap, cost, end) == []
    assert cost[5] == I32_MAX and end[5] == -1
    assert cost[1] == I32_MAX and end[1] == -1     # the empty query


def test_gap_that_prunes_nothing_is_the_exact_fill(gpu):
    w = inputs.paper_i8(B=6, N=300, M=20000, seed=71)
    gap = int(np.abs(w.queries.astype(np.int64)).max() + np.abs(w.ref.astype(np.int64)).max())
    c0, e0 = run(gpu, w.ref, w.queries, "i8", 0)
    c1, e1 = run(gpu, w.ref, w.queries, "i8", gap)
    assert np.array_equal(c0, c1) and np.array_equal(e0, e1)


def test_pruned_codebook_paper_shape(gpu):
    """The codebook pipeline on 64 paper-shaped queries (2,000 x 100,000) with a
    gap of 32 codes (one standard deviation of the reference): bit-exact
    against the pruned oracle on every query."""
    w = inputs.paper_fp32(B=64)
    r = torch.from_numpy(w.ref).to(gpu)
    params = codebook_fit(r)
    cr = codebook_encode(r, params).cpu().numpy()
    cq = codebook_encode(torch.from_numpy(w.queries).to(gpu), params).cpu().numpy()
    cost, end = run(gpu, cr, cq, "u8", 32)
    assert check(cr, lambda q: cq[q], range(w.B), 32, cost, end) == []
