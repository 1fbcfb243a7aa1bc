"""GPU forward parity against the CPU oracle, through the C ABI.

FP32 costs within 1e-5 relative of the FP64 oracle, end columns exact except
where the oracle's best columns tie within that tolerance; int8 mode bit-exact.
Shapes span several strips, warps and sweeps with ragged tails, the paper's
batch at full size (sampled queries), and the edge cases of the method
(one-sample queries or reference, queries longer than the reference, exact
cuts with zero cost, empty queries in a ragged batch).
"""
import numpy as np
import pytest
import torch

import parity
from paper_2403_06931_gb300 import capi, inputs
from paper_2403_06931_gb300.sdtw import SdtwContext

pytestmark = pytest.mark.gpu


def run_fwd(dev, ref, queries, offsets=None, N=None, dtype="f32", **kw):
    r = torch.from_numpy(np.ascontiguousarray(ref)).to(dev)
    q = torch.from_numpy(np.ascontiguousarray(queries)).to(dev)
    o = torch.from_numpy(offsets).to(dev) if offsets is not None else None
    B = len(offsets) - 1 if offsets is not None else queries.shape[0]
    Nmax = N if N is not None else (queries.shape[1] if offsets is None else int(np.diff(offsets).max(initial=1)))
    ctx = SdtwContext(dtype=dtype, max_ref_len=len(ref), max_batch=max(B, 1), max_query_len=max(Nmax, 1),
                      max_total_query_len=max(q.numel(), 1), **kw)
    cost, end = ctx.forward(r, q, offsets=o, N=Nmax if offsets is not None else None)
    assert ctx.device_status() == capi.SDTW_OK
    ctx.close()
    return cost.cpu().numpy(), end.cpu().numpy()


def test_small_batch_fp32(gpu):
    w = inputs.small_fp32()
    cost, end = run_fwd(gpu, w.ref, w.queries)
    assert parity.check_forward_f32(w.ref, w.query, range(w.B), cost, end) == []


SHAPES = [
    # (B, N, M) -- several strips/warps/sweeps with ragged tails, and edge cases
    (3, 37, 1000), (2, 200, 5000), (5, 1, 777), (4, 64, 1), (3, 300, 129), (2, 1000, 999),
    (1, 5, 4096), (1, 5, 4097), (7, 130, 8193),
]


@pytest.mark.parametrize("B,N,M", SHAPES)
def test_shapes_fp32(gpu, B, N, M):
    w = inputs.tiny(B=B, N=N, M=M, seed=1000 + B * N + M)
    cost, end = run_fwd(gpu, w.ref, w.queries)
    assert parity.check_forward_f32(w.ref, w.query, range(B), cost, end) == []


@pytest.mark.parametrize("RT", [2, 4, 8])
@pytest.mark.parametrize("W", [8, 16, 20, 24, 28, 32])
@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 8, 16])
def test_every_plan_fp32(gpu, W, P, RT):
    if RT == 8 and not 16 <= W <= 28:
        pytest.skip("8-row tiles are built for 16 to 28 columns")
    w = inputs.tiny(B=3, N=91, M=6000, seed=77)
    cost, end = run_fwd(gpu, w.ref, w.queries, seg_width=W, warps_per_query=P, tile_rows=RT)
    assert parity.check_forward_f32(w.ref, w.query, range(w.B), cost, end) == []


@pytest.mark.parametrize("RT", [2, 4, 8])
@pytest.mark.parametrize("W", [8, 16, 20, 24, 28, 32])
@pytest.mark.parametrize("P", [1, 4, 5, 16])
def test_every_plan_i8_bit_exact(gpu, W, P, RT):
    if RT == 8 and not 16 <= W <= 28:
        pytest.skip("8-row tiles are built for 16 to 28 columns")
    w = inputs.paper_i8(B=4, N=70, M=5000, seed=78)
    cost, end = run_fwd(gpu, w.ref, w.queries, dtype="i8", seg_width=W, warps_per_query=P, tile_rows=RT)
    assert cost.dtype == np.int32
    assert parity.check_forward_i8(w.ref, w.query, range(w.B), cost, end) == []


@pytest.mark.parametrize("RT", [2, 4, 8])
@pytest.mark.parametrize("W", [8, 16, 28, 32])
@pytest.mark.parametrize("P", [1, 2, 4])
def test_fast_path_plans(gpu, W, P, RT):
    # queries long enough that most chunks take the fast path; lengths of every residue mod 8
    if RT == 8 and not 16 <= W <= 28:
        pytest.skip("8-row tiles are built for 16 to 28 columns")
    for N in (1501, 1202, 1403, 1200, 1605, 1206, 1207):
        w = inputs.tiny(B=2, N=N, M=20000, seed=79 + N)
        cost, end = run_fwd(gpu, w.ref, w.queries, seg_width=W, warps_per_query=P, tile_rows=RT)
        assert parity.check_forward_f32(w.ref, w.query, range(w.B), cost, end) == []
        wi = inputs.paper_i8(B=2, N=N, M=20000, seed=80 + N)
        cost, end = run_fwd(gpu, wi.ref, wi.queries, dtype="i8", seg_width=W, warps_per_query=P, tile_rows=RT)
        assert parity.check_forward_i8(wi.ref, wi.query, range(wi.B), cost, end) == []


@pytest.mark.parametrize("scale", [1.0, 8.0])
@pytest.mark.parametrize("W", [16, 24, 32])
def test_stretched_paths_fp32(gpu, W, scale):
    # queries subsampled from the reference: their paths run long horizontal
    # stretches into strips whose own cells cost far more (the FP32 fill
    # rebases a strip to such a low left input; without it these costs drift
    # past the tolerance); scaled by 8, costs reach that rebase on this shape
    w = inputs.stretched(scale=scale)
    cost, end = run_fwd(gpu, w.ref, w.queries, seg_width=W)
    assert parity.check_forward_f32(w.ref, w.query, range(w.B), cost, end) == []


@pytest.mark.parametrize("dtype", ["f32", "i8", "f16"])
def test_unaligned_reference_matches_aligned(gpu, dtype):
    # strips are loaded as vectors of four samples only when the reference is
    # aligned for them; a reference that starts one sample into a buffer takes
    # the per-sample loads and must give the same results
    w = inputs.tiny(B=4, N=120, M=5003, seed=83)
    tdt = {"f32": torch.float32, "i8": torch.int8, "f16": torch.float16}[dtype]
    if dtype == "i8":
        ref_h, q_h = inputs.quantize_i8(w.ref), inputs.quantize_i8(w.queries)
    else:
        ref_h, q_h = w.ref, w.queries
    buf = torch.zeros(w.M + 1, dtype=tdt, device=gpu)
    buf[1:] = torch.from_numpy(np.ascontiguousarray(ref_h)).to(gpu).to(tdt)
    unaligned = buf[1:]
    aligned = unaligned.clone()
    q = torch.from_numpy(np.ascontiguousarray(q_h)).to(gpu).to(tdt)
    ctx = SdtwContext(dtype=dtype, max_ref_len=w.M, max_batch=w.B, max_query_len=w.N)
    c0, e0 = ctx.forward(aligned, q)
    c1, e1 = ctx.forward(unaligned, q)
    assert ctx.device_status() == capi.SDTW_OK
    assert torch.equal(c0, c1) and torch.equal(e0, e1)
    ctx.close()


def test_exact_cut_has_zero_cost(gpu):
    w = inputs.tiny(B=1, N=10, M=3000, seed=5)
    y = w.ref
    offs = [0, 1234, 2990 - 128]
    qs = np.stack([y[o:o + 128] for o in offs]).astype(np.float32)
    cost, end = run_fwd(gpu, y, qs)
    assert (cost == 0).all()
    assert end.tolist() == [o + 127 for o in offs]


def test_int8_extremes_bit_exact(gpu):
    # largest local costs (254^2) and long queries: int32 accumulation stays exact
    rng = np.random.default_rng(3)
    ref = rng.choice(np.array([-127, 127], dtype=np.int8), size=3000)
    qs = rng.choice(np.array([-127, 127], dtype=np.int8), size=(3, 2500))
    cost, end = run_fwd(gpu, ref, qs, dtype="i8")
    assert parity.check_forward_i8(ref, lambda q: qs[q], range(3), cost, end) == []


def test_int8_min_is_exact_on_small_integers(gpu):
    # costs below 2^23 are subnormal float patterns: the three-input float
    # minimum must order them like the integers they are
    ref = np.array([0, 1, 0, 2, 0, 1, 1, 0], dtype=np.int8)
    qs = np.array([[0, 1, 1], [1, 0, 0], [2, 2, 2]], dtype=np.int8)
    cost, end = run_fwd(gpu, ref, qs, dtype="i8")
    assert parity.check_forward_i8(ref, lambda q: qs[q], range(3), cost, end) == []


def test_ragged_with_empty_and_single_queries(gpu):
    rng = np.random.default_rng(11)
    lengths = np.array([5, 0, 1, 300, 17, 0, 64, 1024, 2], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    ref = rng.standard_normal(4000).astype(np.float32)
    flat = rng.standard_normal(int(offs[-1])).astype(np.float32)
    cost, end = run_fwd(gpu, ref, flat, offsets=offs, N=1024)
    nz = [q for q in range(len(lengths)) if lengths[q] > 0]
    assert parity.check_forward_f32(ref, lambda q: flat[offs[q]:offs[q + 1]], nz, cost, end) == []
    for q in range(len(lengths)):
        if lengths[q] == 0:
            assert np.isinf(cost[q]) and cost[q] > 0 and end[q] == -1


@pytest.mark.parametrize("RT", [4, 8])
def test_ragged_every_residue(gpu, RT):
    # ragged lengths of every residue modulo the tile height, in one persistent launch
    rng = np.random.default_rng(14)
    lengths = np.array([1, 2, 3, 4, 5, 6, 7, 8, 9, 15, 16, 17, 255, 256, 257, 700, 703], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    ref = inputs.znorm(np.cumsum(rng.standard_normal(9000))).astype(np.float32)
    flat = rng.standard_normal(int(offs[-1])).astype(np.float32)
    cost, end = run_fwd(gpu, ref, flat, offsets=offs, N=703, seg_width=24, tile_rows=RT)
    assert parity.check_forward_f32(ref, lambda q: flat[offs[q]:offs[q + 1]], range(len(lengths)), cost, end) == []


def test_ragged_i8(gpu):
    rng = np.random.default_rng(12)
    lengths = rng.integers(0, 400, size=20).astype(np.int64)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    ref = rng.integers(-127, 128, size=3000).astype(np.int8)
    flat = rng.integers(-127, 128, size=int(offs[-1])).astype(np.int8)
    cost, end = run_fwd(gpu, ref, flat, offsets=offs, N=400, dtype="i8")
    nz = [q for q in range(20) if lengths[q] > 0]
    assert parity.check_forward_i8(ref, lambda q: flat[offs[q]:offs[q + 1]], nz, cost, end) == []


def test_ragged_query_longer_than_N_is_flagged(gpu):
    lengths = np.array([10, 50, 10], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    ref = torch.randn(500, device=gpu)
    flat = torch.randn(int(offs[-1]), device=gpu)
    o = torch.from_numpy(offs).to(gpu)
    ctx = SdtwContext(max_ref_len=500, max_batch=3, max_query_len=64, max_total_query_len=200)
    cost = torch.full((3,), -7.0, device=gpu)
    end = torch.full((3,), -7, dtype=torch.int64, device=gpu)
    ctx.forward(ref, flat, offsets=o, N=20, out=(cost, end))
    assert ctx.device_status() == capi.SDTW_E_INVALID
    assert ctx.device_status() == capi.SDTW_OK      # cleared
    # the flagged query gets the empty query's outputs, never a stale value
    assert cost[1].item() == float("inf") and end[1].item() == -1
    assert end[0].item() >= 0 and end[2].item() >= 0
    ctx.close()


def test_invalid_arguments_queue_nothing(gpu):
    ctx = SdtwContext(max_ref_len=100, max_batch=4, max_query_len=10)
    ref = torch.randn(100, device=gpu)
    qs = torch.randn(4, 10, device=gpu)
    cost = torch.empty(4, device=gpu)
    end = torch.empty(4, dtype=torch.int64, device=gpu)
    h = ctx.handle
    s = torch.cuda.current_stream().cuda_stream
    P = lambda t: t.data_ptr()  # noqa: E731
    assert capi.sdtw_forward(h, P(ref), 101, P(qs), None, 4, 10, P(cost), P(end), s) == capi.SDTW_E_INVALID
    assert capi.sdtw_forward(h, P(ref), 100, P(qs), None, 5, 10, P(cost), P(end), s) == capi.SDTW_E_INVALID
    assert capi.sdtw_forward(h, P(ref), 100, P(qs), None, 4, 11, P(cost), P(end), s) == capi.SDTW_E_INVALID
    assert capi.sdtw_forward(h, P(ref), 0, P(qs), None, 4, 10, P(cost), P(end), s) == capi.SDTW_E_INVALID
    assert capi.sdtw_forward(h, None, 100, P(qs), None, 4, 10, P(cost), P(end), s) == capi.SDTW_E_INVALID
    assert capi.sdtw_forward(h, P(ref), 100, P(qs), None, 0, 10, None, None, s) == capi.SDTW_OK
    ctx.close()


def test_host_entry_point_matches_device(gpu):
    w = inputs.tiny(B=6, N=100, M=3000, seed=9)
    cost_d, end_d = run_fwd(gpu, w.ref, w.queries)
    ctx = SdtwContext(max_ref_len=w.M, max_batch=w.B, max_query_len=w.N)
    cost = np.empty(w.B, dtype=np.float32)
    end = np.empty(w.B, dtype=np.int64)
    st = capi.sdtw_forward_host(ctx.handle, w.ref.ctypes.data, w.M, w.queries.ctypes.data, None, w.B, w.N,
                                cost.ctypes.data, end.ctypes.data, None)
    assert st == capi.SDTW_OK
    assert np.array_equal(cost, cost_d) and np.array_equal(end, end_d)
    ctx.close()


def test_autotune_keeps_results(gpu):
    w = inputs.tiny(B=8, N=256, M=20000, seed=10)
    r = torch.from_numpy(w.ref).to(gpu)
    q = torch.from_numpy(w.queries).to(gpu)
    ctx = SdtwContext(max_ref_len=w.M, max_batch=w.B, max_query_len=w.N)
    c0, e0 = ctx.forward(r, q)
    plan = ctx.autotune(r, q)
    assert plan["tuned"] == 1 and plan["seg_width"] in (8, 16, 20, 24, 28, 32)
    c1, e1 = ctx.forward(r, q)
    assert torch.equal(e0, e1)
    assert parity.check_forward_f32(w.ref, w.query, range(w.B), c1.cpu().numpy(), e1.cpu().numpy()) == []
    ctx.close()


# ---------------------------------------------------------------- full size --

def _sample(B, k, seed):
    rng = np.random.default_rng(seed)
    return sorted(rng.choice(B, size=min(k, B), replace=False).tolist())


def test_paper_batch_fp32_full_size(gpu):
    """512 x 2,000 vs 100,000 in the bench's launch configuration: every query."""
    w = inputs.paper_fp32()
    cost, end = run_fwd(gpu, w.ref, w.queries)
    assert np.isfinite(cost).all() and (cost >= 0).all() and ((end >= 0) & (end < w.M)).all()
    assert parity.check_forward_f32(w.ref, w.query, range(w.B), cost, end) == []


def test_paper_batch_i8_full_size(gpu):
    """The integer workload at full size: all 512 queries bit-exact against the int64 oracle."""
    w = inputs.paper_i8()
    cost, end = run_fwd(gpu, w.ref, w.queries, dtype="i8")
    assert parity.check_forward_i8(w.ref, w.query, range(w.B), cost, end) == []


def _ragged_check_set(w, extra, seed):
    """Every query of at most 400 samples (the oracle finishes those in
    seconds against 10^6 columns) plus a few sampled longer ones."""
    short = np.nonzero(w.lengths <= 400)[0].tolist()
    return sorted(set(short + _sample(w.B, extra, seed)))


def test_ragged_full_size(gpu):
    """2,048 queries, lengths U[200, 4000], vs 1,000,000: all queries of <= 400 samples, and 3 others."""
    w = inputs.ragged_fp32()
    cost, end = run_fwd(gpu, w.ref, w.queries, offsets=w.offsets, N=int(w.lengths.max()))
    assert np.isfinite(cost).all() and ((end >= 0) & (end < w.M)).all()
    idx = _ragged_check_set(w, 3, 3)
    assert len(idx) >= 90
    assert parity.check_forward_f32(w.ref, w.query, idx, cost, end) == []


@pytest.mark.parametrize("full", [False, True])
def test_ragged_persistent_form_replays_from_a_cuda_graph(gpu, full):
    """The ragged call captured once in a CUDA graph (the length ordering, the
    work-counter reset and the persistent launch), replayed twice with the
    outputs overwritten in between: bit-for-bit the eager call's results, and
    the oracle's on checked queries.  full: the 2,048-query, 10^6-column
    workload the bench replays (bench.py repeats the replay-equals-eager check
    on the plan its autotuner picks)."""
    if full:
        w = inputs.ragged_fp32()
    else:
        w = inputs.ragged_fp32(B=300, n_lo=1, n_hi=900, M=40000, seed=641)
    Nr = int(w.lengths.max())
    ref = torch.from_numpy(w.ref).to(gpu)
    qs = torch.from_numpy(w.queries).to(gpu)
    offs = torch.from_numpy(w.offsets).to(gpu)
    ctx = SdtwContext(max_ref_len=w.M, max_batch=w.B, max_query_len=Nr, max_total_query_len=qs.numel())
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    cost = torch.empty(w.B, device=gpu)
    end = torch.empty(w.B, dtype=torch.int64, device=gpu)
    with torch.cuda.stream(s):
        ctx.forward(ref, qs, offsets=offs, N=Nr, out=(cost, end), stream=s)   # eager, outside the capture
    torch.cuda.synchronize()
    assert ctx.device_status() == capi.SDTW_OK
    want_c, want_e = cost.clone(), end.clone()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s):
        ctx.forward(ref, qs, offsets=offs, N=Nr, out=(cost, end), stream=s)
    for _ in range(2):
        cost.fill_(float("nan"))
        end.fill_(-7)
        graph.replay()
        torch.cuda.synchronize()
        assert torch.equal(cost, want_c) and torch.equal(end, want_e)
    assert ctx.device_status() == capi.SDTW_OK
    ctx.close()
    c, e = cost.cpu().numpy(), end.cpu().numpy()
    if full:
        idx = sorted(set(np.argsort(w.lengths, kind="stable")[:6].tolist() + _sample(w.B, 2, 7)))
    else:
        idx = list(range(w.B))
    assert parity.check_forward_f32(w.ref, w.query, idx, c, e) == []
