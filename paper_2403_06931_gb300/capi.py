"""ctypes binding of the C ABI in include/sdtw.h -- argument marshalling only.

Every function here has the name and argument order of its C counterpart;
pointers are passed as integers (device addresses from torch tensors'
``data_ptr()``, or host addresses), streams as ``cudaStream_t`` integers.
All computation happens inside libsdtw.so: there is no Python or CPU path.
Loading fails with an ImportError when the library has not been built.
"""
from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsdtw.so")

# sdtw_status
SDTW_OK = 0
SDTW_E_INVALID = 1
SDTW_E_NOMEM = 2
SDTW_E_CUDA = 3
SDTW_E_TIMEOUT = 4
SDTW_E_UNSUPPORTED = 5

# sdtw_dtype
SDTW_F32 = 0
SDTW_I8 = 1
SDTW_U8 = 2
SDTW_F16 = 3

SDTW_FLAG_GRAD = 0x1
SDTW_FLAG_KEEP_CHECKPOINTS = 0x2
SDTW_FLAG_NO_AUTOTUNE = 0x4
SDTW_FLAG_ZNORM_QUERIES = 0x8
SDTW_FLAG_TEST_IDLE_HELPERS = 0x10

ABI_VERSION = 5


class sdtw_config(ctypes.Structure):
    _fields_ = [
        ("dtype", ctypes.c_int),
        ("device", ctypes.c_int32),
        ("max_ref_len", ctypes.c_int64),
        ("max_total_query_len", ctypes.c_int64),
        ("max_batch", ctypes.c_int32),
        ("max_query_len", ctypes.c_int32),
        ("seg_width", ctypes.c_int32),
        ("warps_per_query", ctypes.c_int32),
        ("ckpt_stride", ctypes.c_int32),
        ("prune_gap", ctypes.c_int32),
        ("mem_cap_bytes", ctypes.c_size_t),
        ("spin_limit", ctypes.c_uint64),
        ("flags", ctypes.c_uint32),
        ("tile_rows", ctypes.c_int32),
        ("bwd_warps", ctypes.c_int32),
    ]


class sdtw_plan(ctypes.Structure):
    _fields_ = [
        ("seg_width", ctypes.c_int32),
        ("warps_per_query", ctypes.c_int32),
        ("ctas_per_query", ctypes.c_int32),
        ("persistent", ctypes.c_int32),
        ("grid", ctypes.c_int64),
        ("block", ctypes.c_int32),
        ("smem_bytes", ctypes.c_int32),
        ("ckpt_stride", ctypes.c_int32),
        ("tuned", ctypes.c_int32),
        ("sweep_cols", ctypes.c_int64),
        ("tile_rows", ctypes.c_int32),
        ("ckpt_cols", ctypes.c_int32),
        ("bwd_warps", ctypes.c_int32),
    ]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_ST = ctypes.c_int

# (name, restype, argtypes) of every exported function of include/sdtw.h
SIGNATURES = [
    ("sdtw_abi_version", _I32, []),
    ("sdtw_status_string", ctypes.c_char_p, [_ST]),
    ("sdtw_config_init", _ST, [ctypes.POINTER(sdtw_config)]),
    ("sdtw_create", _ST, [ctypes.POINTER(_P), ctypes.POINTER(sdtw_config)]),
    ("sdtw_destroy", _ST, [_P]),
    ("sdtw_forward", _ST, [_P, _P, _I64, _P, _P, _I32, _I32, _P, _P, _P]),
    ("sdtw_backward", _ST, [_P, _P, _I64, _P, _P, _I32, _I32, _P, _P, _P, _P, _P, _P]),
    ("sdtw_path", _ST, [_P, _P, _I64, _P, _P, _I32, _I32, _P, _P, _P]),
    ("sdtw_forward_host", _ST, [_P, _P, _I64, _P, _P, _I32, _I32, _P, _P, _P]),
    ("sdtw_forward_backward_host", _ST, [_P, _P, _I64, _P, _P, _I32, _I32, _P, _P, _P, _P, _P, _P, _P]),
    ("sdtw_autotune", _ST, [_P, _P, _I64, _P, _P, _I32, _I32, _P, _P, _P, ctypes.POINTER(sdtw_plan)]),
    ("sdtw_get_plan", _ST, [_P, _I32, _I32, _I64, _I32, _I32, ctypes.POINTER(sdtw_plan)]),
    ("sdtw_forward_noalloc", _ST, [ctypes.c_int, _P, _I64, _P, _P, _I32, _I32, _P, _P, _P]),
    ("sdtw_znormalize", _ST, [_P, _P, _P, _I32, _I32, _P]),
    ("sdtw_codebook_fit", _ST, [_P, _I64, ctypes.c_float, _P, _P]),
    ("sdtw_codebook_encode", _ST, [_P, _I64, _P, _P, _P]),
    ("sdtw_last_device_status", _ST, [_P, _P]),
    ("sdtw_last_error", ctypes.c_char_p, [_P]),
    ("sdtw_workspace_bytes", ctypes.c_size_t, [_P]),
]

_lib = None


def load(path: str = LIB_PATH):
    """Load libsdtw.so and declare its signatures (ImportError if missing)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(
            f"libsdtw.so not found at {path}: build it first "
            "(python -c 'import __graft_entry__ as g; g.build()')")
    lib = ctypes.CDLL(path)
    for name, res, args in SIGNATURES:
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if lib.sdtw_abi_version() != ABI_VERSION:
        raise ImportError(f"libsdtw.so ABI {lib.sdtw_abi_version()} != binding ABI {ABI_VERSION}")
    _lib = lib
    return lib


class SdtwError(RuntimeError):
    def __init__(self, status: int, where: str, detail: str = ""):
        self.status = status
        msg = load().sdtw_status_string(status).decode()
        super().__init__(f"{where}: {msg}" + (f" ({detail})" if detail else ""))


def check(status: int, where: str, ctx=None) -> None:
    if status != SDTW_OK:
        detail = load().sdtw_last_error(ctx).decode() if ctx else ""
        raise SdtwError(status, where, detail)


# ------------------------------------------------- same-name thin wrappers --

def sdtw_abi_version() -> int:
    return load().sdtw_abi_version()


def sdtw_status_string(status: int) -> str:
    return load().sdtw_status_string(status).decode()


def sdtw_config_init() -> sdtw_config:
    cfg = sdtw_config()
    check(load().sdtw_config_init(ctypes.byref(cfg)), "sdtw_config_init")
    return cfg


def sdtw_create(cfg: sdtw_config):
    """Returns (status, ctx handle or None)."""
    h = _P()
    st = load().sdtw_create(ctypes.byref(h), ctypes.byref(cfg))
    return st, (h.value if st == SDTW_OK else None)


def sdtw_destroy(ctx) -> int:
    return load().sdtw_destroy(ctx)


def sdtw_forward(ctx, ref, M, queries, offsets, B, N, cost, end, stream) -> int:
    return load().sdtw_forward(ctx, ref, M, queries, offsets, B, N, cost, end, stream)


def sdtw_backward(ctx, ref, M, queries, offsets, B, N, end, grad_cost, grad_queries, grad_ref, path,
                  stream) -> int:
    return load().sdtw_backward(ctx, ref, M, queries, offsets, B, N, end, grad_cost, grad_queries, grad_ref,
                                path, stream)


def sdtw_path(ctx, ref, M, queries, offsets, B, N, end, path, stream) -> int:
    return load().sdtw_path(ctx, ref, M, queries, offsets, B, N, end, path, stream)


def sdtw_forward_host(ctx, ref, M, queries, offsets, B, N, cost, end, stream) -> int:
    return load().sdtw_forward_host(ctx, ref, M, queries, offsets, B, N, cost, end, stream)


def sdtw_forward_backward_host(ctx, ref, M, queries, offsets, B, N, grad_cost, cost, end, grad_queries,
                               grad_ref, path, stream) -> int:
    return load().sdtw_forward_backward_host(ctx, ref, M, queries, offsets, B, N, grad_cost, cost, end,
                                             grad_queries, grad_ref, path, stream)


def sdtw_autotune(ctx, ref, M, queries, offsets, B, N, cost, end, stream):
    """Returns (status, sdtw_plan)."""
    plan = sdtw_plan()
    st = load().sdtw_autotune(ctx, ref, M, queries, offsets, B, N, cost, end, stream, ctypes.byref(plan))
    return st, plan


def sdtw_get_plan(ctx, B, N, M, ragged, backward):
    plan = sdtw_plan()
    st = load().sdtw_get_plan(ctx, B, N, M, ragged, backward, ctypes.byref(plan))
    return st, plan


def sdtw_forward_noalloc(dtype, ref, M, queries, offsets, B, N, cost, end, stream) -> int:
    return load().sdtw_forward_noalloc(dtype, ref, M, queries, offsets, B, N, cost, end, stream)


SDTW_NOALLOC_MAX_BATCH = 65536


def sdtw_znormalize(inp, out, offsets, B, N, stream) -> int:
    return load().sdtw_znormalize(inp, out, offsets, B, N, stream)


def sdtw_codebook_fit(ref, M, sigmas, params, stream) -> int:
    return load().sdtw_codebook_fit(ref, M, sigmas, params, stream)


def sdtw_codebook_encode(inp, n, params, out, stream) -> int:
    return load().sdtw_codebook_encode(inp, n, params, out, stream)


def sdtw_last_device_status(ctx, stream) -> int:
    return load().sdtw_last_device_status(ctx, stream)


def sdtw_last_error(ctx) -> str:
    return load().sdtw_last_error(ctx).decode()


def sdtw_workspace_bytes(ctx) -> int:
    return load().sdtw_workspace_bytes(ctx)
