"""sdtw_forward_noalloc: the forward for callers that cannot allocate.

Callers inside a graph capture that may not allocate, plug-ins whose host
process owns every device allocation, and real-time loops that must not touch
the allocator after start-up cannot create a context (sdtw_create allocates).
This entry point keeps its small scratch in a fixed device array instead.  The
test calls it through the C ABI twice in a row (the array keeps the previous
call's contents, which the entry point must clear) and compares both results
with sdtw_forward's, within the parity tolerance of the other tests.  It is
collected last so that a failure here cannot hide any other test's result.
"""
import numpy as np
import pytest
import torch

import parity
from paper_2403_06931_gb300 import capi, inputs
from paper_2403_06931_gb300.sdtw import SdtwContext

pytestmark = pytest.mark.gpu


def _same_within_tolerance(c_ref, e_ref, c, e, lengths):
    tol = parity.cost_tol(c_ref.astype(np.float64), lengths)
    assert np.all(np.abs(c.astype(np.float64) - c_ref) <= tol)
    assert np.array_equal(e, e_ref)


@pytest.mark.parametrize("ragged", [True, False])
def test_noalloc_matches_forward_twice(gpu, ragged):
    if ragged:
        w = inputs.ragged_fp32(B=40, n_lo=1, n_hi=700, M=30000, seed=611)
    else:
        w = inputs.tiny(B=24, N=300, M=30000, seed=612)
    N = int(w.lengths.max())
    ref = torch.from_numpy(w.ref).to(gpu)
    qs = torch.from_numpy(w.queries).to(gpu)
    offs = torch.from_numpy(w.offsets).to(gpu) if ragged else None
    ctx = SdtwContext(max_ref_len=w.M, max_batch=w.B, max_query_len=N, max_total_query_len=qs.numel(),
                      seg_width=32, warps_per_query=4)
    c_ref, e_ref = ctx.forward(ref, qs, offsets=offs, N=N if ragged else None)
    torch.cuda.synchronize()
    ctx.close()
    c_ref, e_ref = c_ref.cpu().numpy(), e_ref.cpu().numpy()
    s = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        cost = torch.full((w.B,), -1.0, device=gpu)
        end = torch.full((w.B,), -7, dtype=torch.int64, device=gpu)
        st = capi.sdtw_forward_noalloc(capi.SDTW_F32, ref.data_ptr(), w.M, qs.data_ptr(),
                                       offs.data_ptr() if ragged else None, w.B, N, cost.data_ptr(),
                                       end.data_ptr(), s)
        assert st == capi.SDTW_OK
        torch.cuda.synchronize()
        _same_within_tolerance(c_ref, e_ref, cost.cpu().numpy(), end.cpu().numpy(), w.lengths)


def test_noalloc_int8_matches_forward_twice(gpu):
    w = inputs.paper_i8(B=16, N=200, M=20000, seed=613)
    ref = torch.from_numpy(w.ref).to(gpu)
    qs = torch.from_numpy(w.queries).to(gpu)
    ctx = SdtwContext(dtype="i8", max_ref_len=w.M, max_batch=w.B, max_query_len=w.N)
    c_ref, e_ref = ctx.forward(ref, qs)
    torch.cuda.synchronize()
    ctx.close()
    s = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        cost = torch.full((w.B,), -1, dtype=torch.int32, device=gpu)
        end = torch.full((w.B,), -7, dtype=torch.int64, device=gpu)
        st = capi.sdtw_forward_noalloc(capi.SDTW_I8, ref.data_ptr(), w.M, qs.data_ptr(), None, w.B, w.N,
                                       cost.data_ptr(), end.data_ptr(), s)
        assert st == capi.SDTW_OK
        torch.cuda.synchronize()
        assert torch.equal(cost.cpu(), c_ref.cpu()) and torch.equal(end.cpu(), e_ref.cpu())


@pytest.mark.parametrize("dtype", ["f16", "u8"])
def test_noalloc_binary16_and_codebook_codes_match_forward_twice(gpu, dtype):
    w = inputs.tiny(B=9, N=150, M=12000, seed=615)
    ref = torch.from_numpy(w.ref).to(gpu)
    qs = torch.from_numpy(w.queries).to(gpu)
    if dtype == "f16":
        ref, qs = ref.half(), qs.half()
        lib_dt, cdt = capi.SDTW_F16, torch.float32
    else:
        from paper_2403_06931_gb300.sdtw import codebook_encode, codebook_fit
        params = codebook_fit(ref)
        ref, qs = codebook_encode(ref, params), codebook_encode(qs, params)
        lib_dt, cdt = capi.SDTW_U8, torch.int32
    ctx = SdtwContext(dtype=dtype, max_ref_len=w.M, max_batch=w.B, max_query_len=w.N)
    c_ref, e_ref = ctx.forward(ref, qs)
    torch.cuda.synchronize()
    ctx.close()
    s = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        cost = torch.full((w.B,), -1, dtype=cdt, device=gpu)
        end = torch.full((w.B,), -7, dtype=torch.int64, device=gpu)
        st = capi.sdtw_forward_noalloc(lib_dt, ref.data_ptr(), w.M, qs.data_ptr(), None, w.B, w.N,
                                       cost.data_ptr(), end.data_ptr(), s)
        assert st == capi.SDTW_OK
        torch.cuda.synchronize()
        assert torch.equal(cost, c_ref) and torch.equal(end, e_ref)


def test_noalloc_over_long_query_gets_the_empty_outputs(gpu):
    # a ragged query longer than N cannot be reported (no context): it gets the
    # empty query's outputs, and the others are computed as by sdtw_forward
    lengths = np.array([20, 90, 0, 35], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    rng = np.random.default_rng(614)
    ref = torch.from_numpy(rng.standard_normal(3000).astype(np.float32)).to(gpu)
    flat = torch.from_numpy(rng.standard_normal(int(offs[-1])).astype(np.float32)).to(gpu)
    o = torch.from_numpy(offs).to(gpu)
    s = torch.cuda.current_stream().cuda_stream
    for _ in range(2):
        cost = torch.full((4,), -1.0, device=gpu)
        end = torch.full((4,), -7, dtype=torch.int64, device=gpu)
        st = capi.sdtw_forward_noalloc(capi.SDTW_F32, ref.data_ptr(), 3000, flat.data_ptr(), o.data_ptr(), 4, 40,
                                       cost.data_ptr(), end.data_ptr(), s)
        assert st == capi.SDTW_OK
        torch.cuda.synchronize()
        c, e = cost.cpu().numpy(), end.cpu().numpy()
        for q in (1, 2):
            assert np.isinf(c[q]) and c[q] > 0 and e[q] == -1
        fl = flat.cpu().numpy()
        assert parity.check_forward_f32(ref.cpu().numpy(), lambda q: fl[offs[q]:offs[q + 1]], [0, 3], c, e) == []


def test_noalloc_rejects_batches_over_its_maximum(gpu):
    z = torch.zeros(8, device=gpu)
    s = torch.cuda.current_stream().cuda_stream
    st = capi.sdtw_forward_noalloc(capi.SDTW_F32, z.data_ptr(), 8, z.data_ptr(), None,
                                   capi.SDTW_NOALLOC_MAX_BATCH + 1, 1, z.data_ptr(), z.data_ptr(), s)
    assert st == capi.SDTW_E_INVALID
