"""GPU batch z-normalisation (sdtw_znormalize, paper Section 5.1, Eq. 2)
against the FP64 oracle, element by element.

The kernel works in float only: compensated sums of the samples shifted by the
first one, reductions and the mean as float pairs (hi + lo), the centred values
as (x - hi) - lo.  Each output then
carries a few float roundings at the scale of max(|z|, 1): the bound checked
is |z - o| <= 2^-21 (|o| + 1).  (A float32 emulation of the kernel on random
walks, offsets of 1e4 and 1e6 and long series stays below 2.7e-7.)
"""
import numpy as np
import pytest
import torch

import oracle
from paper_2403_06931_gb300 import capi
from paper_2403_06931_gb300.sdtw import znormalize

pytestmark = pytest.mark.gpu


def _check(z, o):
    z = np.asarray(z, dtype=np.float64)
    bad = np.abs(z - o) > 2.0 ** -21 * (np.abs(o) + 1.0)
    assert not bad.any(), (int(np.argmax(bad)), z[bad][:3], o[bad][:3])


def _walks(B, N, seed, offset=0.0, scale=1.0):
    rng = np.random.default_rng(seed)
    return (offset + scale * np.cumsum(rng.standard_normal((B, N)), axis=1)).astype(np.float32)


def test_uniform_batch_paper_shape(gpu):
    x = _walks(512, 2000, 1, offset=3.0, scale=2.5)
    z = znormalize(torch.from_numpy(x).to(gpu)).cpu().numpy()
    _check(z.reshape(-1), oracle.znormalize_batch(x, N=2000))


def test_ragged_batch_with_edge_series(gpu):
    rng = np.random.default_rng(2)
    lens = [0, 1, 2, 3, 255, 256, 257, 4000, 0, 17]
    series = [rng.standard_normal(n).astype(np.float32) * 4 + 1 for n in lens]
    series[5][:] = 7.25                       # zero spread: centred only
    series[6] = (1e4 + rng.standard_normal(257)).astype(np.float32)   # large mean, small spread
    flat = np.concatenate(series).astype(np.float32)
    offs = np.concatenate([[0], np.cumsum(lens)]).astype(np.int64)
    sentinel = np.float32(-123.5)
    out = torch.full((flat.size + 1,), float(sentinel), device=gpu)[:flat.size]
    znormalize(torch.from_numpy(flat).to(gpu), offsets=torch.from_numpy(offs).to(gpu), out=out)
    z = out.cpu().numpy()
    _check(z, oracle.znormalize_batch(flat, offsets=offs))
    assert np.array_equal(z[offs[5]:offs[6]], np.zeros(256, np.float32))


def test_in_place_and_long_series(gpu):
    x = _walks(1, 1_000_000, 3, offset=-50.0).reshape(-1)
    t = torch.from_numpy(x).to(gpu)
    znormalize(t, out=t)                      # in place, one CTA over 10^6 samples
    _check(t.cpu().numpy(), oracle.znormalize(x))


@pytest.mark.parametrize("N", [1, 2, 4, 33, 2048, 2052, 16384, 16385])
def test_uniform_lengths_across_kernels(gpu, N):
    # series of a multiple of 4 samples up to 2,048 stay in a warp's registers,
    # others up to 16,384 take a warp each (16-byte accesses when N % 4 == 0),
    # longer ones a CTA each
    x = _walks(9, N, 10 + N, offset=1.0)
    x[4] = 2.5                                # a constant series
    z = znormalize(torch.from_numpy(x).to(gpu)).cpu().numpy()
    _check(z.reshape(-1), oracle.znormalize_batch(x, N=N))
    assert np.array_equal(z[4], np.zeros(N, np.float32))


def test_invalid_arguments(gpu):
    f = torch.zeros(8, device=gpu)
    assert capi.sdtw_znormalize(f.data_ptr(), f.data_ptr(), None, -1, 8, None) == capi.SDTW_E_INVALID
    assert capi.sdtw_znormalize(f.data_ptr(), f.data_ptr(), None, 1, 0, None) == capi.SDTW_E_INVALID
    assert capi.sdtw_znormalize(None, f.data_ptr(), None, 1, 8, None) == capi.SDTW_E_INVALID
    assert capi.sdtw_znormalize(None, None, None, 0, 8, None) == capi.SDTW_OK
