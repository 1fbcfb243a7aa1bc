"""Query z-normalisation inside the library (SDTW_FLAG_ZNORM_QUERIES, the
paper's Eq. 2 applied before the fill of Eq. 1).

On raw queries, a context with the flag must give exactly what a plain context
gives on the same queries normalised by sdtw_znormalize: the same normaliser
writes the copy the fill reads, so costs, ends, paths and the reference
gradient are equal bit for bit.  The query gradient is then the gradient with
respect to the raw samples: the FP64 derivative of Eq. 2 (oracle
``znormalize_vjp``, pinned by central differences) applied to the plain
context's gradient with respect to the normalised queries, within float
rounding of that sum.
"""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2403_06931_gb300 import capi, inputs
from paper_2403_06931_gb300.sdtw import SdtwContext, sdtw_cost, znormalize

pytestmark = pytest.mark.gpu

VTOL = 1e-5   # |g - o| <= VTOL * max|o| + 1e-6 for the carried gradient


def _raw(w, seed):
    """Un-normalised queries: each a random affine image of the workload's."""
    rng = np.random.default_rng(seed)
    q = w.queries.astype(np.float64).copy()
    bounds = [(w.offsets[i], w.offsets[i + 1]) for i in range(w.B)] if w.offsets is not None else \
        [(i * w.N, (i + 1) * w.N) for i in range(w.B)]
    flat = q.reshape(-1)
    for a, b in bounds:
        flat[a:b] = flat[a:b] * rng.uniform(0.3, 40.0) + rng.uniform(-500.0, 500.0)
    return flat.reshape(q.shape).astype(np.float32), bounds


def _run(dev, w, raw, **kw):
    ref = torch.from_numpy(w.ref).to(dev)
    qr = torch.from_numpy(raw).to(dev)
    offs = torch.from_numpy(w.offsets).to(dev) if w.offsets is not None else None
    N = int(w.lengths.max())
    Nk = N if offs is not None else None
    common = dict(max_ref_len=w.M, max_batch=w.B, max_query_len=N, max_total_query_len=qr.numel(),
                  grad=True, keep_checkpoints=True, **kw)
    cz = SdtwContext(znorm_queries=True, **common)
    cp = SdtwContext(**common)
    qz = znormalize(qr, offsets=offs)
    g = torch.from_numpy(np.random.default_rng(5).uniform(-2, 2, w.B).astype(np.float32)).to(dev)
    out = {}
    for name, ctx, q in (("z", cz, qr), ("p", cp, qz)):
        cost, end = ctx.forward(ref, q, offsets=offs, N=Nk)
        gq, gr, path = ctx.backward(ref, q, end, g, offsets=offs, N=Nk, want_path=True)
        assert ctx.device_status() == capi.SDTW_OK
        out[name] = [t.cpu().numpy() for t in (cost, end, gq, gr, path)]
        ctx.close()
    return out, qz.cpu().numpy(), g.cpu().numpy()


def _check(w, raw, bounds, out, qz, g):
    cz, ez, gqz, grz, pz = out["z"]
    cp, ep, gqp, grp, pp = out["p"]
    assert np.array_equal(cz, cp) and np.array_equal(ez, ep)
    assert np.array_equal(pz, pp) and np.array_equal(grz, grp)
    flat_raw = raw.reshape(-1).astype(np.float64)
    fz, fp = gqz.reshape(-1), gqp.reshape(-1).astype(np.float64)
    for a, b in bounds:
        if b <= a:
            continue
        o = oracle.znormalize_vjp(flat_raw[a:b], fp[a:b])
        assert np.all(np.abs(fz[a:b] - o) <= VTOL * np.abs(o).max() + 1e-6), (a, b)
    # and the costs and ends are those of the FP64-normalised queries
    bad = parity.check_forward_f32(w.ref, lambda q: oracle.znormalize(flat_raw[bounds[q][0]:bounds[q][1]]),
                                   [q for q in range(w.B) if bounds[q][1] > bounds[q][0]], cz, ez)
    assert not bad, bad[:4]


def test_uniform_batch(gpu):
    w = inputs.tiny(B=6, N=96, M=3000, seed=301)
    raw, bounds = _raw(w, 1)
    out, qz, g = _run(gpu, w, raw)
    _check(w, raw, bounds, out, qz, g)


def test_uniform_batch_length_not_a_multiple_of_four(gpu):
    w = inputs.tiny(B=5, N=157, M=2600, seed=302)
    raw, bounds = _raw(w, 2)
    out, qz, g = _run(gpu, w, raw, seg_width=16, tile_rows=2, warps_per_query=2)
    _check(w, raw, bounds, out, qz, g)


def test_ragged_batch(gpu):
    w = inputs.ragged_fp32(B=7, n_lo=2, n_hi=300, M=2500, seed=303)
    raw, bounds = _raw(w, 3)
    out, qz, g = _run(gpu, w, raw)
    _check(w, raw, bounds, out, qz, g)


def test_autograd_gives_the_raw_query_gradient(gpu):
    w = inputs.tiny(B=4, N=60, M=900, seed=304)
    raw, _ = _raw(w, 4)
    ctx = SdtwContext(max_ref_len=w.M, max_batch=w.B, max_query_len=w.N, grad=True, keep_checkpoints=True,
                      znorm_queries=True)
    ref = torch.from_numpy(w.ref).to(gpu).requires_grad_(True)
    qs = torch.from_numpy(raw).to(gpu).requires_grad_(True)
    cost, end = sdtw_cost(ref, qs, ctx)
    wts = torch.tensor([1.0, -0.5, 2.0, 0.25], device=gpu)
    (cost * wts).sum().backward()
    gq, gr, _ = ctx.backward(ref.detach(), qs.detach(), end, wts)
    assert torch.equal(qs.grad, gq) and torch.equal(ref.grad, gr)
    # a shift and a scale of a query change neither its cost nor its end
    c2, e2 = ctx.forward(ref.detach(), qs.detach() * 3.0 + 11.0)
    assert torch.allclose(c2, cost.detach(), rtol=1e-5, atol=1e-5)
    ctx.close()


def test_ragged_query_past_the_copy_is_flagged(gpu):
    """Offsets that reach past max_total_query_len: the query is reported and
    skipped (it gets the empty query's outputs), nothing is read or written
    outside the context's copy."""
    w = inputs.ragged_fp32(B=3, n_lo=40, n_hi=60, M=800, seed=305)
    total = int(w.offsets[-1])
    ctx = SdtwContext(max_ref_len=w.M, max_batch=w.B, max_query_len=int(w.lengths.max()),
                      max_total_query_len=total - 5, znorm_queries=True)
    ref = torch.from_numpy(w.ref).to(gpu)
    qs = torch.from_numpy(w.queries).to(gpu)
    offs = torch.from_numpy(w.offsets).to(gpu)
    cost = torch.full((w.B,), -7.0, device=gpu)
    end = torch.full((w.B,), -9, dtype=torch.int64, device=gpu)
    ctx.forward(ref, qs, offsets=offs, N=int(w.lengths.max()), out=(cost, end))
    assert ctx.device_status() & 1            # a ragged query longer than allowed
    c = cost.cpu().numpy()
    assert np.isinf(c[-1]) and c[-1] > 0 and end.cpu().numpy()[-1] == -1   # the last query was skipped
    ctx.close()


def _ckpt_floats_per_query(M, N, W, P, RT, KS):
    """Backward workspace per query (floats) of a checkpointing plan, as the
    library documents it: the wavefront slot (a record per thread every KS
    steps), the boundary columns, a gradient row and 7 scalars."""
    S, lag_last = 32 * P * W, (P - 1) * 64 + 31
    nsw, nt = -(-M // S), -(-N // RT)
    total = (nsw - 1) * max(nt, lag_last + 32) + nt + lag_last
    fr = -(-total // KS) * 32 * P * (W + (4 if RT == 2 else 8))
    ck = (-(-M // (8 * W)) - 1) * (-(-N // 4) * 4)
    return fr + ck + M + 7


def test_chunked_backward_with_normalised_queries(gpu):
    """Kept checkpoints, a backward that re-runs the forward, and a memory cap
    that holds the checkpoints of 4 of the 9 queries (chunks of 4, 4 and 1,
    each re-running its forward on the normalised copy) agree bit for bit."""
    w = inputs.tiny(B=9, N=200, M=4000, seed=306)
    raw, _ = _raw(w, 6)
    st = dict(seg_width=16, tile_rows=4, warps_per_query=2, ckpt_stride=16)
    ref = torch.from_numpy(w.ref).to(gpu)
    qr = torch.from_numpy(raw).to(gpu)
    g = torch.from_numpy(np.linspace(-1.5, 2.0, w.B).astype(np.float32)).to(gpu)

    def run(keep, cap=0):
        ctx = SdtwContext(max_ref_len=w.M, max_batch=w.B, max_query_len=w.N, grad=True, keep_checkpoints=keep,
                          znorm_queries=True, mem_cap_bytes=cap, **st)
        cost, end = ctx.forward(ref, qr)
        gq, gr, path = ctx.backward(ref, qr, end, g, want_path=True)
        assert ctx.device_status() == capi.SDTW_OK
        ctx.close()
        return [t.cpu().numpy() for t in (cost, end, gq, gr, path)]

    a = run(True)
    b = run(False)
    # status, work counter and order (8 + 4 B bytes), the normalised copy (4 B N),
    # per-query cost and end scratch (12 B), then the arena
    fixed = 8 + 4 * w.B + 4 * w.B * w.N + 12 * w.B
    per_q = _ckpt_floats_per_query(w.M, w.N, 16, 2, 4, 16)
    c = run(False, fixed + 4 * (4 * per_q + 32) + 8)
    for u, v in ((a, b), (a, c)):
        for k in range(5):
            assert np.array_equal(u[k], v[k])
