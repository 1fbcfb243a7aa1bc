"""GPU backward (walk-back gradient) against the CPU oracle, through the C ABI.

What is unique is compared exactly: where the oracle's walk-back meets no
near-tie (every step's best neighbour beats the runner-up by more than FP32
can blur), the GPU path must be the oracle's path and its gradients must match
the oracle's path gradient.  Where several paths are optimal within FP32
resolution, the GPU path must be valid, its FP64 cost must equal the optimum
within the cost tolerance, and the GPU gradients must equal the FP64 path
gradient of the GPU's own path.  grad_ref must be the sum of the per-query
path gradients.
"""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2403_06931_gb300 import capi, inputs
from paper_2403_06931_gb300.sdtw import SdtwContext, sdtw_cost

pytestmark = pytest.mark.gpu

GTOL = 1e-4   # gradients: |g - o| <= GTOL * max|o| + 1e-6


def run_bwd(dev, w, grad_cost=None, keep=True, **kw):
    ref = torch.from_numpy(w.ref).to(dev)
    qs = torch.from_numpy(w.queries).to(dev)
    offs = torch.from_numpy(w.offsets).to(dev) if w.offsets is not None else None
    N = int(w.lengths.max())
    ctx = SdtwContext(max_ref_len=w.M, max_batch=w.B, max_query_len=N, max_total_query_len=qs.numel(),
                      grad=True, keep_checkpoints=keep, **kw)
    cost, end = ctx.forward(ref, qs, offsets=offs, N=N if offs is not None else None)
    g = torch.from_numpy(np.asarray(grad_cost, dtype=np.float32)).to(dev) if grad_cost is not None \
        else torch.ones(w.B, device=dev)
    gq, gr, path = ctx.backward(ref, qs, end, g, offsets=offs, N=N if offs is not None else None, want_path=True)
    assert ctx.device_status() == capi.SDTW_OK
    ctx.close()
    return (cost.cpu().numpy(), end.cpu().numpy(), gq.cpu().numpy(), gr.cpu().numpy(),
            path.cpu().numpy().reshape(-1, 2), g.cpu().numpy())


def _rows(w, path, q):
    a = w.offsets[q] if w.offsets is not None else q * w.N
    n = int(w.lengths[q])
    return path[a:a + n, 0], path[a:a + n, 1]


def _gq(w, gq, q):
    if w.offsets is not None:
        return gq[w.offsets[q]:w.offsets[q + 1]]
    return gq[q]


def check_validity(w, cost, end, gq, gr, path, g, idx, oracle_costs):
    """Path valid and optimal; gradients equal the FP64 gradient of the GPU's path."""
    y = w.ref.astype(np.float64)
    gy_sum = np.zeros(w.M)
    for k, q in enumerate(idx):
        x = w.query(q).astype(np.float64)
        lo, hi = _rows(w, path, q)
        assert oracle.intervals_are_valid(lo, hi, w.M, int(end[q])), q
        pc = oracle.intervals_cost(x, y, lo, hi)
        oc = oracle_costs[k]
        # the forward that stored the checkpoints returned the right cost
        assert abs(float(cost[q]) - oc) <= parity.cost_tol(oc, len(x)), (q, float(cost[q]), oc)
        assert abs(pc - oc) <= parity.cost_tol(oc, len(x)), (q, pc, oc)
        gx, gyq = oracle.intervals_gradient(x, y, lo, hi, g=float(g[q]))
        scale = max(np.abs(gx).max(), 1e-12)
        assert np.all(np.abs(_gq(w, gq, q) - gx) <= GTOL * scale + 1e-6), q
        gy_sum += gyq
    return gy_sum


TIE = 1e-5    # a walk-back step is a near-tie when its two best neighbours differ by < TIE * cost


def compare_with_oracle_paths(w, end, gq, path, g, idx, oracle_costs, oracle_ends):
    """Follow the GPU path and the oracle's walk-back from the end cell: they must
    agree until their first divergence, and a divergence may only start at a step
    where the oracle's best two neighbours are within FP32 resolution (a near-tie).
    Where the whole path agrees, the gradients must match the oracle's.
    Returns (queries with identical paths, matched cells, total cells)."""
    y = w.ref.astype(np.float64)
    same = matched = total = 0
    for k, q in enumerate(idx):
        if int(end[q]) != int(oracle_ends[k]):
            continue                      # a tied end: covered by the end-index rule
        x = w.query(q).astype(np.float64)
        cells, margins = oracle.walkback(x, y, int(oracle_ends[k]))
        lo, hi = _rows(w, path, q)
        gcells = oracle.cells_from_intervals(lo, hi)
        L = min(len(cells), len(gcells))
        diff = np.nonzero((cells[:L] != gcells[:L]).any(axis=1))[0]
        total += len(cells)
        if len(diff) == 0 and len(cells) == len(gcells):
            same += 1
            matched += len(cells)
            gx, _ = oracle.path_gradient(x, y, cells, g=float(g[q]))
            assert np.all(np.abs(_gq(w, gq, q) - gx) <= GTOL * np.abs(gx).max() + 1e-6), q
            continue
        first = int(diff[0]) if len(diff) else L
        matched += first
        assert first >= 1, q              # the end cell itself is shared
        tol = TIE * oracle_costs[k] + 1e-6 * len(x)
        assert 0 <= margins[first - 1] <= tol, (q, first, margins[first - 1], tol)
    return same, matched, total


def test_grad_subset_matches_oracle_paths(gpu):
    """8 x 64 vs 512: the walk-back follows the oracle's up to FP32 near-ties."""
    w = inputs.grad_subset()
    g = np.linspace(0.5, 2.0, w.B)
    cost, end, gq, gr, path, gd = run_bwd(gpu, w, grad_cost=g)
    oc, oe = oracle.forward_batch(w.ref, w.queries)
    gy_sum = check_validity(w, cost, end, gq, gr, path, gd, range(w.B), oc)
    assert np.all(np.abs(gr - gy_sum) <= GTOL * np.abs(gy_sum).max() + 1e-6)
    same, matched, total = compare_with_oracle_paths(w, end, gq, path, gd, range(w.B), oc, oe)
    assert same >= 2 and matched >= 0.5 * total


def test_walkback_tie_rule_on_many_queries(gpu):
    """48 queries x 64..200 samples: every divergence from the oracle's path starts at a near-tie."""
    w = inputs.tiny(B=48, N=150, M=3000, seed=97)
    cost, end, gq, gr, path, g = run_bwd(gpu, w)
    oc, oe = oracle.forward_batch(w.ref, w.queries)
    check_validity(w, cost, end, gq, gr, path, g, range(w.B), oc)
    same, matched, total = compare_with_oracle_paths(w, end, gq, path, g, range(w.B), oc, oe)
    assert same >= 5 and matched >= 0.5 * total


@pytest.mark.parametrize("B,N,M,W,RT,P", [(4, 50, 700, 8, 2, 1), (3, 300, 2000, 16, 4, 2), (2, 129, 5000, 32, 2, 4),
                                          (3, 1, 300, 8, 4, 2), (2, 40, 1, 8, 2, 1), (2, 700, 600, 16, 2, 1),
                                          (2, 600, 3000, 24, 4, 4), (3, 257, 1100, 24, 2, 3),
                                          (2, 1000, 40000, 24, 4, 4), (2, 333, 20000, 32, 4, 8),
                                          (3, 1, 300, 16, 8, 2), (2, 600, 3000, 24, 8, 4), (3, 257, 1100, 16, 8, 3),
                                          (2, 1000, 40000, 20, 8, 4), (2, 333, 20000, 28, 8, 8)])
def test_backward_shapes(gpu, B, N, M, W, RT, P):
    # band replays across warps, sweeps, ragged last tiles, a one-row query,
    # a one-column reference and queries longer than the reference
    w = inputs.tiny(B=B, N=N, M=M, seed=500 + B + N + M)
    cost, end, gq, gr, path, g = run_bwd(gpu, w, seg_width=W, tile_rows=RT, warps_per_query=P)
    oc, _ = oracle.forward_batch(w.ref, w.queries)
    gy_sum = check_validity(w, cost, end, gq, gr, path, g, range(B), oc)
    assert np.all(np.abs(gr - gy_sum) <= GTOL * max(np.abs(gy_sum).max(), 1.0) + 1e-6)


@pytest.mark.parametrize("P", [2, 5])
@pytest.mark.parametrize("RT", [2, 4, 8])
@pytest.mark.parametrize("W", [8, 16, 20, 24, 28, 32])
def test_backward_every_tile_height_and_width(gpu, RT, W, P):
    # checkpoints taken by every checkpointing forward variant
    if RT == 8 and not 16 <= W <= 28:
        pytest.skip("8-row tiles take 16 to 28 columns")
    w = inputs.tiny(B=3, N=700, M=9000, seed=400 + RT + W)
    cost, end, gq, gr, path, g = run_bwd(gpu, w, seg_width=W, tile_rows=RT, warps_per_query=P)
    oc, _ = oracle.forward_batch(w.ref, w.queries)
    check_validity(w, cost, end, gq, gr, path, g, range(w.B), oc)


@pytest.mark.parametrize("KS", [8, 16, 32, 64])
@pytest.mark.parametrize("RT", [2, 4, 8])
def test_backward_every_checkpoint_stride(gpu, RT, KS):
    # bands of 8, 16, 32 or 64 forward steps, with several warps and sweeps
    w = inputs.tiny(B=4, N=600, M=12000, seed=430 + RT + KS)
    cost, end, gq, gr, path, g = run_bwd(gpu, w, seg_width=24, tile_rows=RT, warps_per_query=3, ckpt_stride=KS)
    oc, _ = oracle.forward_batch(w.ref, w.queries)
    gy_sum = check_validity(w, cost, end, gq, gr, path, g, range(w.B), oc)
    assert np.all(np.abs(gr - gy_sum) <= GTOL * max(np.abs(gy_sum).max(), 1.0) + 1e-6)


@pytest.mark.parametrize("KS", [8, 16, 32, 64])
@pytest.mark.parametrize("RT", [4, 8])
def test_backward_stretched_paths(gpu, KS, RT):
    # long horizontal runs, scaled so that costs reach the forward's rebase to
    # low left inputs: the backward must replay every such rebase to reproduce
    # the forward's values (the device checks the end cell bit for bit)
    w = inputs.stretched(B=8, N=300, M=30000, scale=8.0)
    cost, end, gq, gr, path, g = run_bwd(gpu, w, ckpt_stride=KS, tile_rows=RT, seg_width=32 if RT == 4 else 28)
    oc, _ = oracle.forward_batch(w.ref, w.queries)
    check_validity(w, cost, end, gq, gr, path, g, range(w.B), oc)


def test_backward_long_vertical_runs_cross_bands(gpu):
    # a query far longer than the reference forces long vertical runs, so the
    # walk climbs through many bands of one window
    w = inputs.tiny(B=2, N=2500, M=300, seed=61)
    cost, end, gq, gr, path, g = run_bwd(gpu, w, seg_width=8, tile_rows=2, warps_per_query=1)
    oc, _ = oracle.forward_batch(w.ref, w.queries)
    check_validity(w, cost, end, gq, gr, path, g, range(w.B), oc)


def test_backward_ragged(gpu):
    w = inputs.ragged_fp32(B=7, n_lo=1, n_hi=300, M=2500, seed=71)
    cost, end, gq, gr, path, g = run_bwd(gpu, w)
    oc, _ = oracle.forward_batch(w.ref, w.queries, offsets=w.offsets)
    gy_sum = check_validity(w, cost, end, gq, gr, path, g, range(w.B), oc)
    assert np.all(np.abs(gr - gy_sum) <= GTOL * np.abs(gy_sum).max() + 1e-6)


@pytest.mark.parametrize("case", ["stretched16", "stretched64", "stretched_rt8", "tiny_rt2", "w8", "ragged", "vertical"])
def test_backward_helpers_give_identical_results(gpu, case):
    # the walker alone (bwd_warps=1) and with 1 to 3 helpers recomputing the
    # predicted bands: the same path, gradients and reference gradient, bit for bit
    w, st = {
        "stretched16": (inputs.stretched(B=6, N=300, M=30000, scale=8.0), dict(ckpt_stride=16)),
        "stretched64": (inputs.stretched(B=4, N=300, M=30000), dict(ckpt_stride=64, tile_rows=2)),
        "stretched_rt8": (inputs.stretched(B=6, N=300, M=30000, scale=8.0), dict(ckpt_stride=8, tile_rows=8)),
        "tiny_rt2": (inputs.tiny(B=5, N=500, M=8000, seed=91), dict(seg_width=24, tile_rows=2, warps_per_query=3)),
        "w8": (inputs.tiny(B=4, N=400, M=6000, seed=92), dict(seg_width=8, tile_rows=4, warps_per_query=2)),
        "ragged": (inputs.ragged_fp32(B=9, n_lo=1, n_hi=500, M=7000, seed=93), {}),
        "vertical": (inputs.tiny(B=2, N=2500, M=300, seed=61), dict(seg_width=8, tile_rows=2, warps_per_query=1)),
    }[case]
    runs = [run_bwd(gpu, w, bwd_warps=k, **st) for k in (1, 2, 3, 4)]
    for r in runs[1:]:
        for k in range(5):
            assert np.array_equal(runs[0][k], r[k]), k
    oc, _ = oracle.forward_batch(w.ref, w.queries, offsets=w.offsets)
    check_validity(w, *runs[3], range(w.B), oc)


def test_walker_wait_runs_out_when_helpers_never_answer(gpu):
    # a test flag keeps the helper warps from taking work: the walker's wait for
    # a band it handed out ends at its time limit (about 2 s) with SDTW_E_TIMEOUT
    # in the device status, and the device stays usable
    w = inputs.stretched(B=4, N=300, M=30000)
    ref = torch.from_numpy(w.ref).to(gpu)
    qs = torch.from_numpy(w.queries).to(gpu)
    ctx = SdtwContext(max_ref_len=w.M, max_batch=w.B, max_query_len=w.N, grad=True, keep_checkpoints=True,
                      bwd_warps=3, extra_flags=capi.SDTW_FLAG_TEST_IDLE_HELPERS)
    cost, end = ctx.forward(ref, qs)
    ctx.backward(ref, qs, end, torch.ones(w.B, device=gpu))
    assert ctx.device_status() == capi.SDTW_E_TIMEOUT
    ctx.close()
    cost, end, gq, gr, path, g = run_bwd(gpu, w)     # a fresh context works (its status is checked)
    oc, _ = oracle.forward_batch(w.ref, w.queries)
    check_validity(w, cost, end, gq, gr, path, g, range(w.B), oc)


def _ckpt_floats_per_query(M, N, W, P, RT, KS):
    """Backward workspace per query (floats) of a checkpointing plan: the
    wavefront slot (one record of W + 4, W + 8 or W + 12 floats per thread and
    checkpoint for 2-, 4- or 8-row tiles, one checkpoint every KS steps), the
    boundary columns every 8 W columns (rows padded to 8), a gradient row and
    7 scalars (the layout the library documents)."""
    S, lag_last = 32 * P * W, (P - 1) * 64 + 31
    nsw, nt = -(-M // S), -(-N // RT)
    total = (nsw - 1) * max(nt, lag_last + 32) + nt + lag_last
    fr = -(-total // KS) * 32 * P * (W + {2: 4, 4: 8, 8: 12}[RT])
    ck = (-(-M // (8 * W)) - 1) * (-(-N // 8) * 8)
    return fr + ck + M + 7


@pytest.mark.parametrize("KS", [8, 16, 32, 64])
def test_chunked_and_recomputed_backward_are_identical(gpu, KS):
    w = inputs.tiny(B=9, N=200, M=4000, seed=81)
    st = dict(seg_width=16, tile_rows=4, warps_per_query=2, ckpt_stride=KS)
    a = run_bwd(gpu, w, keep=True, **st)                          # checkpoints from the forward
    b = run_bwd(gpu, w, keep=False, **st)                         # backward re-runs the forward
    # a cap that holds the checkpoints of 4 queries: chunks of 4, 4 and 1
    fixed = 8 + 4 * w.B + 12 * w.B
    per_q = _ckpt_floats_per_query(w.M, w.N, 16, 2, 4, KS)
    c = run_bwd(gpu, w, keep=False, mem_cap_bytes=fixed + 4 * (4 * per_q + 32) + 8, **st)
    for u, v in ((a, b), (a, c)):
        for k in range(5):
            assert np.array_equal(u[k], v[k])
    # too small a cap for one query fails at creation
    with pytest.raises(capi.SdtwError):
        run_bwd(gpu, w, keep=False, mem_cap_bytes=fixed + 4 * per_q // 2, **st)


def test_path_entry_point_matches_backward(gpu):
    # sdtw_path: the walk-back without gradients, from kept checkpoints and from
    # a re-run forward, equals the backward's path
    for w in (inputs.tiny(B=6, N=300, M=5000, seed=87), inputs.ragged_fp32(B=5, n_lo=1, n_hi=400, M=3000, seed=88)):
        cost, end, gq, gr, path, g = run_bwd(gpu, w)
        ref = torch.from_numpy(w.ref).to(gpu)
        qs = torch.from_numpy(w.queries).to(gpu)
        offs = torch.from_numpy(w.offsets).to(gpu) if w.offsets is not None else None
        Nq = int(w.lengths.max())
        for keep in (True, False):
            ctx = SdtwContext(max_ref_len=w.M, max_batch=w.B, max_query_len=Nq, max_total_query_len=qs.numel(),
                              grad=True, keep_checkpoints=keep)
            c2, e2 = ctx.forward(ref, qs, offsets=offs, N=Nq if offs is not None else None)
            p2 = ctx.path(ref, qs, e2, offsets=offs, N=Nq if offs is not None else None)
            assert ctx.device_status() == capi.SDTW_OK
            assert np.array_equal(e2.cpu().numpy(), end) and np.array_equal(p2.cpu().numpy(), path)
            ctx.close()


def test_differentiable_step_replays_from_a_cuda_graph(gpu):
    # forward with checkpoints + backward allocate nothing after the context is
    # created, so the whole step can be captured once and replayed
    w = inputs.tiny(B=6, N=300, M=6000, seed=89)
    ref = torch.from_numpy(w.ref).to(gpu)
    qs = torch.from_numpy(w.queries).to(gpu)
    ctx = SdtwContext(max_ref_len=w.M, max_batch=w.B, max_query_len=w.N, grad=True, keep_checkpoints=True)
    cost = torch.empty(w.B, device=gpu)
    end = torch.empty(w.B, dtype=torch.int64, device=gpu)
    g = torch.linspace(0.5, 1.5, w.B, device=gpu)
    gq = torch.empty_like(qs)
    gr = torch.empty_like(ref)
    path = torch.empty(qs.numel() * 2, dtype=torch.int32, device=gpu)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())

    def step():
        ctx.forward(ref, qs, out=(cost, end), stream=s)
        ctx.backward(ref, qs, end, g, out=(gq, gr, path), stream=s)

    with torch.cuda.stream(s):
        step()                                   # warm-up outside the capture
    torch.cuda.synchronize()
    want = [t.clone() for t in (cost, end, gq, gr, path)]
    for t in (cost, gq, gr):
        t.fill_(float("nan"))
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        step()
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    assert ctx.device_status() == capi.SDTW_OK
    for a, b in zip(want, (cost, end, gq, gr, path)):
        assert torch.equal(a, b)
    ctx.close()


def test_host_forward_backward_matches_device(gpu):
    w = inputs.tiny(B=5, N=120, M=2000, seed=91)
    cost, end, gq, gr, path, g = run_bwd(gpu, w)
    ctx = SdtwContext(max_ref_len=w.M, max_batch=w.B, max_query_len=w.N, grad=True, keep_checkpoints=True)
    hc = np.empty(w.B, np.float32)
    he = np.empty(w.B, np.int64)
    hgq = np.empty_like(w.queries)
    hgr = np.empty_like(w.ref)
    hp = np.empty(w.queries.size * 2, np.int32)
    gc = np.ones(w.B, np.float32)
    st = capi.sdtw_forward_backward_host(ctx.handle, w.ref.ctypes.data, w.M, w.queries.ctypes.data, None, w.B,
                                         w.N, gc.ctypes.data, hc.ctypes.data, he.ctypes.data, hgq.ctypes.data,
                                         hgr.ctypes.data, hp.ctypes.data, None)
    assert st == capi.SDTW_OK
    assert np.array_equal(hc, cost) and np.array_equal(he, end) and np.array_equal(hgq, gq)
    assert np.array_equal(hgr, gr) and np.array_equal(hp.reshape(-1, 2), path)
    ctx.close()


def test_autograd_function(gpu):
    w = inputs.tiny(B=4, N=60, M=900, seed=93)
    ctx = SdtwContext(max_ref_len=w.M, max_batch=w.B, max_query_len=w.N, grad=True, keep_checkpoints=True)
    ref = torch.from_numpy(w.ref).to(gpu).requires_grad_(True)
    qs = torch.from_numpy(w.queries).to(gpu).requires_grad_(True)
    cost, end = sdtw_cost(ref, qs, ctx)
    wts = torch.tensor([1.0, -0.5, 2.0, 0.25], device=gpu)
    (cost * wts).sum().backward()
    gq, gr, _ = ctx.backward(ref.detach(), qs.detach(), end, wts)
    assert torch.equal(qs.grad, gq) and torch.equal(ref.grad, gr)
    ctx.close()


def test_autograd_raises_on_a_device_side_error(gpu):
    # a ragged query longer than N is flagged on the device by the forward; the
    # autograd backward reads the status word and raises instead of returning
    # a gradient computed past the error
    lengths = np.array([30, 80, 30], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    rng = np.random.default_rng(96)
    ref = torch.from_numpy(rng.standard_normal(600).astype(np.float32)).to(gpu).requires_grad_(True)
    flat = torch.from_numpy(rng.standard_normal(int(offs[-1])).astype(np.float32)).to(gpu).requires_grad_(True)
    o = torch.from_numpy(offs).to(gpu)
    ctx = SdtwContext(max_ref_len=600, max_batch=3, max_query_len=80, max_total_query_len=int(offs[-1]),
                      grad=True, keep_checkpoints=True)
    cost, end = sdtw_cost(ref, flat, ctx, offsets=o, N=40)
    assert end[1].item() == -1 and cost[1].item() == float("inf")
    with pytest.raises(capi.SdtwError):
        cost[[0, 2]].sum().backward()
    assert ctx.device_status() == capi.SDTW_OK     # read and cleared by the backward
    ctx.close()


def test_backward_rejections(gpu):
    ctx = SdtwContext(dtype="i8", max_ref_len=100, max_batch=2, max_query_len=10)
    z = torch.zeros(100, dtype=torch.int8, device=gpu)
    st = capi.sdtw_backward(ctx.handle, z.data_ptr(), 100, z.data_ptr(), None, 2, 10, z.data_ptr(),
                            z.data_ptr(), z.data_ptr(), z.data_ptr(), None, None)
    assert st == capi.SDTW_E_UNSUPPORTED
    ctx.close()
    ctx = SdtwContext(max_ref_len=100, max_batch=2, max_query_len=10)       # no grad flag
    f = torch.zeros(100, device=gpu)
    st = capi.sdtw_backward(ctx.handle, f.data_ptr(), 100, f.data_ptr(), None, 2, 10, f.data_ptr(),
                            f.data_ptr(), f.data_ptr(), f.data_ptr(), None, None)
    assert st == capi.SDTW_E_INVALID
    ctx.close()


def test_backward_bad_end_is_flagged(gpu):
    w = inputs.tiny(B=2, N=20, M=300, seed=95)
    ctx = SdtwContext(max_ref_len=w.M, max_batch=w.B, max_query_len=w.N, grad=True)
    ref = torch.from_numpy(w.ref).to(gpu)
    qs = torch.from_numpy(w.queries).to(gpu)
    end = torch.tensor([5, 300], dtype=torch.int64, device=gpu)     # 300 is outside [0, M)
    ctx.backward(ref, qs, end, torch.ones(2, device=gpu))
    assert ctx.device_status() == capi.SDTW_E_INVALID
    ctx.close()


def test_paper_batch_backward_full_size(gpu):
    """512 x 2,000 vs 100,000 with checkpoints kept by the forward (the bench's
    configuration): every path valid; 12 sampled queries checked against the
    oracle's cost and their gradients; grad_ref equals the sum of path gradients."""
    w = inputs.paper_fp32()
    cost, end, gq, gr, path, g = run_bwd(gpu, w)
    y = w.ref.astype(np.float64)
    gy_all = np.zeros(w.M)
    for q in range(w.B):
        lo, hi = _rows(w, path, q)
        assert oracle.intervals_are_valid(lo, hi, w.M, int(end[q])), q
        _, gyq = oracle.intervals_gradient(w.query(q).astype(np.float64), y, lo, hi, g=1.0)
        gy_all += gyq
    assert np.all(np.abs(gr - gy_all) <= GTOL * np.abs(gy_all).max() + 1e-5)
    idx = sorted(np.random.default_rng(5).choice(w.B, size=12, replace=False).tolist())
    oc, _ = oracle.forward_batch(w.ref, w.queries, indices=idx)
    check_validity(w, cost, end, gq, gr, path, g, idx, oc)
    # the library's choice of helpers against the walker alone: identical
    alone = run_bwd(gpu, w, bwd_warps=1)
    for k, v in enumerate((cost, end, gq, gr, path)):
        assert np.array_equal(v, alone[k]), k
