"""GPU reference codebook (paper Section 8) against the CPU oracle, through the C ABI.

The fit (mean +- 4 S of the reference, 256 equal bins) is compared with the
oracle's FP64 fit to float precision; the encoding is bit-exact against the
oracle's float32 decisions given the same (float32) parameters; the uint8 DP
on the codes is bit-exact against the int64 oracle on the same codes.
"""
import numpy as np
import pytest
import torch

import oracle
import parity
from paper_2403_06931_gb300 import capi, inputs
from paper_2403_06931_gb300.sdtw import SdtwContext, codebook_encode, codebook_fit

pytestmark = pytest.mark.gpu


def _fit_and_codes(dev, ref, values):
    r = torch.from_numpy(np.ascontiguousarray(ref, dtype=np.float32)).to(dev)
    params = codebook_fit(r)
    v = torch.from_numpy(np.ascontiguousarray(values, dtype=np.float32)).to(dev)
    codes = codebook_encode(v, params)
    torch.cuda.synchronize()
    return params.cpu().numpy(), codes.cpu().numpy()


@pytest.mark.parametrize("M", [1, 2, 1000, 100_000, 1_000_003])
def test_fit_matches_oracle(gpu, M):
    y = inputs.znorm(np.cumsum(np.random.default_rng(M).standard_normal(M))) * 3.0 + 1.5 if M > 1 \
        else np.array([0.7])
    p, _ = _fit_and_codes(gpu, y, y[:4])
    lo, step = oracle.codebook_fit(y.astype(np.float32).astype(np.float64))
    assert abs(p[0] - lo) <= 1e-6 * max(1.0, abs(lo))
    assert abs(p[2] - step) <= 1e-6 * step
    assert p[1] == np.float32(1.0 / np.float64(np.float32(p[2]))) or abs(p[1] * p[2] - 1.0) <= 2e-7


@pytest.mark.parametrize("n,offset", [(4096, 0), (4099, 0), (4096, 1), (1, 0), (3_000_000, 0)])
def test_encode_bit_exact(gpu, n, offset):
    rng = np.random.default_rng(n + offset)
    ref = inputs.znorm(np.cumsum(rng.standard_normal(50_000)))
    vals = np.concatenate([rng.standard_normal(n) * 1.7, [9.0, -9.0, 1e20, -1e20]]).astype(np.float32)
    r = torch.from_numpy(ref.astype(np.float32)).to(gpu)
    params = codebook_fit(r)
    buf = torch.from_numpy(vals).to(gpu)
    x = buf[offset:]                        # offset 1: not 16-byte aligned (scalar path)
    codes = codebook_encode(x.contiguous() if offset == 0 else x, params)
    torch.cuda.synchronize()
    p = params.cpu().numpy()
    want = oracle.codebook_encode(vals[offset:], p[0], p[1])
    assert np.array_equal(codes.cpu().numpy(), want)


def test_encode_rejects_bad_arguments(gpu):
    s = torch.cuda.current_stream().cuda_stream
    z = torch.zeros(4, device=gpu)
    assert capi.sdtw_codebook_encode(None, 4, z.data_ptr(), z.data_ptr(), s) == capi.SDTW_E_INVALID
    assert capi.sdtw_codebook_encode(z.data_ptr(), -1, z.data_ptr(), z.data_ptr(), s) == capi.SDTW_E_INVALID
    assert capi.sdtw_codebook_encode(None, 0, None, None, s) == capi.SDTW_OK
    assert capi.sdtw_codebook_fit(z.data_ptr(), 4, 0.0, z.data_ptr(), s) == capi.SDTW_E_INVALID
    assert capi.sdtw_codebook_fit(z.data_ptr(), 0, 4.0, z.data_ptr(), s) == capi.SDTW_E_INVALID


def _u8_forward(dev, cref, cq, offsets=None, N=None, **kw):
    r = torch.from_numpy(cref).to(dev)
    q = torch.from_numpy(cq).to(dev)
    o = torch.from_numpy(offsets).to(dev) if offsets is not None else None
    B = len(offsets) - 1 if offsets is not None else cq.shape[0]
    Nmax = N if N is not None else cq.shape[1]
    ctx = SdtwContext(dtype="u8", max_ref_len=len(cref), max_batch=B, max_query_len=Nmax,
                      max_total_query_len=max(q.numel(), 1), **kw)
    cost, end = ctx.forward(r, q, offsets=o, N=Nmax if offsets is not None else None)
    assert ctx.device_status() == capi.SDTW_OK
    ctx.close()
    assert cost.dtype == torch.int32
    return cost.cpu().numpy(), end.cpu().numpy()


@pytest.mark.parametrize("RT", [2, 4, 8])
@pytest.mark.parametrize("W", [8, 16, 24, 32])
@pytest.mark.parametrize("P", [1, 4])
def test_u8_every_plan_bit_exact(gpu, W, P, RT):
    if RT == 8 and not 16 <= W <= 28:
        pytest.skip("8-row tiles are built for 16 to 28 columns")
    rng = np.random.default_rng(70 + W + P + RT)
    cref = rng.integers(0, 256, size=5000).astype(np.uint8)
    cq = rng.integers(0, 256, size=(4, 70)).astype(np.uint8)
    cost, end = _u8_forward(gpu, cref, cq, seg_width=W, warps_per_query=P, tile_rows=RT)
    assert parity.check_forward_i8(cref, lambda q: cq[q], range(4), cost, end) == []


def test_u8_extreme_codes_bit_exact(gpu):
    # codes 0 and 255 only: the largest local cost, 255^2, on every cell
    rng = np.random.default_rng(9)
    cref = rng.choice(np.array([0, 255], np.uint8), size=3000)
    cq = rng.choice(np.array([0, 255], np.uint8), size=(3, 2500))
    cost, end = _u8_forward(gpu, cref, cq)
    assert parity.check_forward_i8(cref, lambda q: cq[q], range(3), cost, end) == []


def test_u8_ragged_bit_exact(gpu):
    rng = np.random.default_rng(13)
    lengths = np.array([3, 0, 1, 250, 77, 400], dtype=np.int64)
    offs = np.concatenate([[0], np.cumsum(lengths)]).astype(np.int64)
    cref = rng.integers(0, 256, size=4000).astype(np.uint8)
    flat = rng.integers(0, 256, size=int(offs[-1])).astype(np.uint8)
    cost, end = _u8_forward(gpu, cref, flat, offsets=offs, N=400)
    nz = [q for q in range(len(lengths)) if lengths[q] > 0]
    assert parity.check_forward_i8(cref, lambda q: flat[offs[q]:offs[q + 1]], nz, cost, end) == []
    assert cost[1] == np.iinfo(np.int32).max and end[1] == -1


def test_codebook_pipeline_paper_batch_full_size(gpu):
    """The paper-shaped batch (512 x 2,000 vs 100,000): codebook fitted on the
    reference, reference and queries encoded on the GPU, the uint8 DP; every
    query bit-exact against the oracle's encoding (float32, the GPU's
    parameters) followed by the int64 DP."""
    w = inputs.paper_fp32()
    r = torch.from_numpy(w.ref).to(gpu)
    q = torch.from_numpy(w.queries).to(gpu)
    params = codebook_fit(r)
    cr, cq = codebook_encode(r, params), codebook_encode(q, params)
    ctx = SdtwContext(dtype="u8", max_ref_len=w.M, max_batch=w.B, max_query_len=w.N)
    cost, end = ctx.forward(cr, cq)
    assert ctx.device_status() == capi.SDTW_OK
    ctx.close()
    p = params.cpu().numpy()
    ocr = oracle.codebook_encode(w.ref, p[0], p[1])
    ocq = oracle.codebook_encode(w.queries, p[0], p[1])
    assert np.array_equal(cr.cpu().numpy(), ocr) and np.array_equal(cq.cpu().numpy(), ocq)
    c, e = cost.cpu().numpy(), end.cpu().numpy()
    assert parity.check_forward_i8(ocr, lambda k: ocq[k], range(w.B), c, e) == []
