"""The C ABI library without a GPU: it builds, loads, exports every function
include/sdtw.h declares, its struct layouts match the header, and argument
checks fail cleanly before any device work."""
import ctypes
import os
import re
import subprocess

import pytest
import torch

from paper_2403_06931_gb300 import build as libbuild
from paper_2403_06931_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sdtw.h")


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return capi.load()


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*[A-Za-z_][\w \*]*?\b(sdtw_\w+)\s*\(", text, flags=re.M)))


def test_every_declared_function_is_exported_and_bound(lib):
    names = declared_functions()
    assert len(names) >= 14
    bound = {n for n, _, _ in capi.SIGNATURES}
    for n in names:
        assert hasattr(lib, n), f"{n} not exported by libsdtw.so"
        assert n in bound, f"{n} has no binding in capi.py"
    assert bound == set(names)


def test_struct_layouts_match_header(tmp_path):
    src = tmp_path / "layout.c"
    fields_cfg = [f for f, _ in capi.sdtw_config._fields_]
    fields_plan = [f for f, _ in capi.sdtw_plan._fields_]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sdtw.h"', "int main(void) {",
             'printf("config %zu\\n", sizeof(sdtw_config));', 'printf("plan %zu\\n", sizeof(sdtw_plan));']
    lines += [f'printf("config.{f} %zu\\n", offsetof(sdtw_config, {f}));' for f in fields_cfg]
    lines += [f'printf("plan.{f} %zu\\n", offsetof(sdtw_plan, {f}));' for f in fields_plan]
    lines += ["return 0; }"]
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.check_call(["gcc", "-std=c11", "-I", os.path.dirname(HEADER), str(src), "-o", str(exe)])
    out = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    assert int(out["config"]) == ctypes.sizeof(capi.sdtw_config)
    assert int(out["plan"]) == ctypes.sizeof(capi.sdtw_plan)
    for f in fields_cfg:
        assert int(out[f"config.{f}"]) == getattr(capi.sdtw_config, f).offset, f
    for f in fields_plan:
        assert int(out[f"plan.{f}"]) == getattr(capi.sdtw_plan, f).offset, f


def test_abi_version_and_status_strings(lib):
    assert capi.sdtw_abi_version() == capi.ABI_VERSION
    for s in range(6):
        assert capi.sdtw_status_string(s).startswith("SDTW_")
    assert "unknown" in capi.sdtw_status_string(99)


def test_config_defaults(lib):
    cfg = capi.sdtw_config_init()
    assert cfg.dtype == capi.SDTW_F32 and cfg.max_ref_len == 100_000
    assert cfg.max_batch == 512 and cfg.max_query_len == 2000 and cfg.flags == 0


def test_argument_checks_before_device_work(lib):
    assert lib.sdtw_config_init(None) == capi.SDTW_E_INVALID
    assert lib.sdtw_create(None, None) == capi.SDTW_E_INVALID
    cfg = capi.sdtw_config_init()
    cfg.dtype = 7
    assert capi.sdtw_create(cfg)[0] == capi.SDTW_E_INVALID
    cfg = capi.sdtw_config_init()
    cfg.max_batch = 0
    assert capi.sdtw_create(cfg)[0] == capi.SDTW_E_INVALID
    cfg = capi.sdtw_config_init()
    cfg.dtype = capi.SDTW_I8
    cfg.flags = capi.SDTW_FLAG_GRAD
    assert capi.sdtw_create(cfg)[0] == capi.SDTW_E_INVALID       # no backward in int8 mode
    cfg = capi.sdtw_config_init()
    cfg.flags = capi.SDTW_FLAG_KEEP_CHECKPOINTS
    assert capi.sdtw_create(cfg)[0] == capi.SDTW_E_INVALID       # checkpoints need SDTW_FLAG_GRAD
    cfg = capi.sdtw_config_init()
    cfg.seg_width = 5
    assert capi.sdtw_create(cfg)[0] == capi.SDTW_E_INVALID
    cfg = capi.sdtw_config_init()
    cfg.dtype = capi.SDTW_I8
    cfg.flags = capi.SDTW_FLAG_ZNORM_QUERIES
    assert capi.sdtw_create(cfg)[0] == capi.SDTW_E_INVALID       # query normalisation is FP32 only
    assert capi.sdtw_forward(None, 1, 10, 1, None, 1, 5, 1, 1, None) == capi.SDTW_E_INVALID
    assert capi.sdtw_backward(None, 1, 10, 1, None, 1, 5, 1, 1, 1, 1, None, None) == capi.SDTW_E_INVALID
    assert capi.sdtw_last_device_status(None, None) == capi.SDTW_E_INVALID
    assert capi.sdtw_get_plan(None, 1, 1, 1, 0, 0)[0] == capi.SDTW_E_INVALID
    assert capi.sdtw_destroy(None) == capi.SDTW_OK
    assert capi.sdtw_workspace_bytes(None) == 0


@pytest.mark.skipif(torch.cuda.is_available(), reason="checks the no-GPU failure path")
def test_create_without_gpu_reports_cuda_error(lib):
    st, h = capi.sdtw_create(capi.sdtw_config_init())
    assert st == capi.SDTW_E_CUDA and h is None


def test_binding_fails_loudly_without_library(tmp_path):
    import importlib
    saved = capi._lib
    try:
        capi._lib = None
        with pytest.raises(ImportError):
            capi.load(str(tmp_path / "missing.so"))
    finally:
        capi._lib = saved
        importlib.reload  # keep the module state as it was


# A query length whose shared-memory size, computed in 32-bit arithmetic, would
# wrap to a small positive number (12 * 357,913,944 + 16,416 = 2^32 + 16,448 for
# four warps of 4-row tiles).  Every entry point must reject it on the host,
# before any device work, so these calls are safe without a GPU.
WRAPPING_N = 357_913_944


def test_query_lengths_beyond_shared_memory_are_rejected_on_the_host(lib):
    cfg = capi.sdtw_config_init()
    cfg.max_query_len = WRAPPING_N
    cfg.max_total_query_len = WRAPPING_N
    assert capi.sdtw_create(cfg)[0] == capi.SDTW_E_UNSUPPORTED
    cfg.max_query_len = 1 << 20
    assert capi.sdtw_create(cfg)[0] == capi.SDTW_E_UNSUPPORTED
    fake = 256  # never dereferenced: the calls return before touching the device
    for dtype in (capi.SDTW_F32, capi.SDTW_I8):
        for offsets in (None, fake):
            for n in (WRAPPING_N, 2_000_000_000, 40_000):
                if dtype == capi.SDTW_I8 and n > 32_896:
                    want = capi.SDTW_E_INVALID          # the int32 cost bound comes first
                else:
                    want = capi.SDTW_E_UNSUPPORTED
                st = capi.sdtw_forward_noalloc(dtype, fake, 1000, fake, offsets, 3, n, fake, fake, None)
                assert st == want, (dtype, offsets, n, st)


def test_reserved_spin_limit_must_be_zero(lib):
    cfg = capi.sdtw_config_init()
    cfg.spin_limit = 1000
    assert capi.sdtw_create(cfg)[0] == capi.SDTW_E_INVALID


def test_checkpoint_strides_accepted_by_create(lib):
    # 8, 16, 32 and 64 steps are the strides the library has; any other
    # positive stride is rejected before any device work (a negative one is invalid)
    for ks, want in ((48, capi.SDTW_E_UNSUPPORTED), (4, capi.SDTW_E_UNSUPPORTED), (12, capi.SDTW_E_UNSUPPORTED),
                     (128, capi.SDTW_E_UNSUPPORTED), (-16, capi.SDTW_E_INVALID)):
        cfg = capi.sdtw_config_init()
        cfg.ckpt_stride = ks
        cfg.flags = capi.SDTW_FLAG_GRAD
        assert capi.sdtw_create(cfg)[0] == want, ks


def test_prune_gap_accepted_only_for_integer_modes(lib):
    for dtype, gap, want in ((capi.SDTW_F32, 5, capi.SDTW_E_INVALID), (capi.SDTW_F16, 5, capi.SDTW_E_INVALID),
                             (capi.SDTW_I8, -1, capi.SDTW_E_INVALID), (capi.SDTW_U8, -3, capi.SDTW_E_INVALID)):
        cfg = capi.sdtw_config_init()
        cfg.dtype = dtype
        cfg.prune_gap = gap
        assert capi.sdtw_create(cfg)[0] == want, (dtype, gap)


def test_backward_warps_range(lib):
    for v in (-1, 5, 32):
        cfg = capi.sdtw_config_init()
        cfg.bwd_warps = v
        assert capi.sdtw_create(cfg)[0] == capi.SDTW_E_INVALID, v


def test_eight_row_tiles_only_for_16_to_28_columns(lib):
    for dtype, flags, width in ((capi.SDTW_F32, capi.SDTW_FLAG_GRAD, 32), (capi.SDTW_F32, capi.SDTW_FLAG_GRAD, 8),
                                (capi.SDTW_F32, 0, 32), (capi.SDTW_F32, 0, 8),
                                (capi.SDTW_I8, 0, 32), (capi.SDTW_U8, 0, 8), (capi.SDTW_F16, 0, 32)):
        cfg = capi.sdtw_config_init()
        cfg.dtype = dtype
        cfg.flags = flags
        cfg.seg_width = width
        cfg.tile_rows = 8
        assert capi.sdtw_create(cfg)[0] == capi.SDTW_E_INVALID, (dtype, flags, width)
