"""PyTorch front end of the sDTW library.

PyTorch supplies device memory and streams; every step of the computation runs
in libsdtw.so (see capi.py).  Tensors must already be on the context's CUDA
device, contiguous, with the element type of the context (float32; int8 for
the integer mode; uint8 codebook codes; float16 for the binary16 mode);
nothing is converted or copied here.

    ctx = SdtwContext(max_ref_len=M, max_batch=B, max_query_len=N)
    cost, end = ctx.forward(ref, queries)              # uniform [B, N]
    cost, end = ctx.forward(ref, flat, offsets=offs)   # ragged

    cost = sdtw_cost(ref, queries, ctx=grad_ctx)       # differentiable
"""
from __future__ import annotations

import torch

from . import capi


def _stream_ptr(stream) -> int:
    s = stream if stream is not None else torch.cuda.current_stream()
    return int(s.cuda_stream)


def _ptr(t) -> int:
    return 0 if t is None else int(t.data_ptr())


class SdtwContext:
    """Owns one sdtw_ctx (include/sdtw.h): device workspace and tuned plans."""

    def __init__(self, dtype: str = "f32", device: int | None = None, max_ref_len: int = 100_000,
                 max_batch: int = 512, max_query_len: int = 2000, max_total_query_len: int | None = None,
                 grad: bool = False, keep_checkpoints: bool = False, seg_width: int = 0,
                 warps_per_query: int = 0, ckpt_stride: int = 0, mem_cap_bytes: int = 0, tile_rows: int = 0,
                 znorm_queries: bool = False, check_status: bool = True, prune_gap: int = 0,
                 bwd_warps: int = 0, extra_flags: int = 0):
        lib_dtype = {"f32": capi.SDTW_F32, "i8": capi.SDTW_I8, "u8": capi.SDTW_U8, "f16": capi.SDTW_F16}[dtype]
        cfg = capi.sdtw_config_init()
        cfg.dtype = lib_dtype
        cfg.device = torch.cuda.current_device() if device is None else int(device)
        cfg.max_ref_len = int(max_ref_len)
        cfg.max_batch = int(max_batch)
        cfg.max_query_len = int(max_query_len)
        cfg.max_total_query_len = int(max_total_query_len or max_batch * max_query_len)
        cfg.seg_width = int(seg_width)
        cfg.warps_per_query = int(warps_per_query)
        cfg.ckpt_stride = int(ckpt_stride)
        cfg.mem_cap_bytes = int(mem_cap_bytes)
        cfg.tile_rows = int(tile_rows)
        cfg.bwd_warps = int(bwd_warps)
        cfg.prune_gap = int(prune_gap)
        cfg.flags = (capi.SDTW_FLAG_GRAD if grad or keep_checkpoints else 0) | \
            (capi.SDTW_FLAG_KEEP_CHECKPOINTS if keep_checkpoints else 0) | \
            (capi.SDTW_FLAG_ZNORM_QUERIES if znorm_queries else 0) | int(extra_flags)
        st, h = capi.sdtw_create(cfg)
        capi.check(st, "sdtw_create")
        self.handle = h
        self.dtype = dtype
        self.device = cfg.device
        self.cfg = cfg
        self.grad = bool(cfg.flags & capi.SDTW_FLAG_GRAD)
        # SdtwFunction.backward reads the device status word after each backward
        # (one stream synchronisation) and raises on a device-side error
        self.check_status = bool(check_status)

    # -- helpers --------------------------------------------------------------
    def _dims(self, ref, queries, offsets, N):
        M = ref.numel()
        if offsets is None:
            if queries.dim() != 2:
                raise ValueError("uniform queries must be [B, N]")
            B, N = queries.shape
        else:
            B = offsets.numel() - 1
            if N is None:
                raise ValueError("ragged batches need N (an upper bound on query length)")
        return int(B), int(N), int(M)

    def _check(self, *ts):
        for t in ts:
            if t is not None and (not t.is_cuda or not t.is_contiguous()):
                raise ValueError("tensors must be contiguous CUDA tensors")

    # -- calls ----------------------------------------------------------------
    def forward(self, ref, queries, offsets=None, N=None, stream=None, out=None):
        """(cost [B], end [B] int64) of every query (sdtw_forward)."""
        self._check(ref, queries, offsets)
        B, N, M = self._dims(ref, queries, offsets, N)
        cdt = torch.float32 if self.dtype in ("f32", "f16") else torch.int32
        if out is None:
            cost = torch.empty(B, dtype=cdt, device=ref.device)
            end = torch.empty(B, dtype=torch.int64, device=ref.device)
        else:
            cost, end = out
        st = capi.sdtw_forward(self.handle, _ptr(ref), M, _ptr(queries), _ptr(offsets), B, N, _ptr(cost),
                               _ptr(end), _stream_ptr(stream))
        capi.check(st, "sdtw_forward", self.handle)
        return cost, end

    def backward(self, ref, queries, end, grad_cost, offsets=None, N=None, want_path=False, stream=None,
                 out=None):
        """(grad_queries, grad_ref, path or None) (sdtw_backward)."""
        self._check(ref, queries, offsets, end, grad_cost)
        B, N, M = self._dims(ref, queries, offsets, N)
        if out is None:
            gq = torch.empty_like(queries)
            gr = torch.empty_like(ref)
            path = torch.empty(queries.numel() * 2, dtype=torch.int32, device=ref.device) if want_path else None
        else:
            gq, gr, path = out
        st = capi.sdtw_backward(self.handle, _ptr(ref), M, _ptr(queries), _ptr(offsets), B, N, _ptr(end),
                                _ptr(grad_cost), _ptr(gq), _ptr(gr), _ptr(path), _stream_ptr(stream))
        capi.check(st, "sdtw_backward", self.handle)
        return gq, gr, path

    def path(self, ref, queries, end, offsets=None, N=None, stream=None, out=None):
        """Per query row, the first and last column of the warp path (sdtw_path):
        int32 [total samples, 2]."""
        self._check(ref, queries, offsets, end)
        B, N, M = self._dims(ref, queries, offsets, N)
        path = out if out is not None else torch.empty(queries.numel() * 2, dtype=torch.int32, device=ref.device)
        st = capi.sdtw_path(self.handle, _ptr(ref), M, _ptr(queries), _ptr(offsets), B, N, _ptr(end), _ptr(path),
                            _stream_ptr(stream))
        capi.check(st, "sdtw_path", self.handle)
        return path.view(-1, 2)

    def autotune(self, ref, queries, offsets=None, N=None, stream=None):
        """Time the candidate plans on this batch and keep the fastest (sdtw_autotune)."""
        self._check(ref, queries, offsets)
        B, N, M = self._dims(ref, queries, offsets, N)
        cdt = torch.float32 if self.dtype in ("f32", "f16") else torch.int32
        cost = torch.empty(B, dtype=cdt, device=ref.device)
        end = torch.empty(B, dtype=torch.int64, device=ref.device)
        st, plan = capi.sdtw_autotune(self.handle, _ptr(ref), M, _ptr(queries), _ptr(offsets), B, N,
                                      _ptr(cost), _ptr(end), _stream_ptr(stream))
        capi.check(st, "sdtw_autotune", self.handle)
        return plan.as_dict()

    def plan(self, B, N, M, ragged=False, backward=False):
        st, plan = capi.sdtw_get_plan(self.handle, int(B), int(N), int(M), int(ragged), int(backward))
        capi.check(st, "sdtw_get_plan", self.handle)
        return plan.as_dict()

    def device_status(self, stream=None) -> int:
        """sdtw_last_device_status: syncs the stream, returns and clears the status."""
        return capi.sdtw_last_device_status(self.handle, _stream_ptr(stream))

    def workspace_bytes(self) -> int:
        return capi.sdtw_workspace_bytes(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            capi.sdtw_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SdtwFunction(torch.autograd.Function):
    """cost = sDTW(ref, queries); backward via sdtw_backward's walk-back gradient."""

    @staticmethod
    def forward(fctx, ref, queries, offsets, N, sctx):
        cost, end = sctx.forward(ref, queries, offsets=offsets, N=N)
        fctx.save_for_backward(ref, queries, end)
        fctx.offsets = offsets
        fctx.N = N
        fctx.sctx = sctx
        fctx.mark_non_differentiable(end)
        return cost, end

    @staticmethod
    def backward(fctx, grad_cost, grad_end):
        ref, queries, end = fctx.saved_tensors
        sctx = fctx.sctx
        gq, gr, _ = sctx.backward(ref, queries, end, grad_cost.contiguous(), offsets=fctx.offsets, N=fctx.N)
        if sctx.check_status:
            # the status word collects what the forward and the backward found
            # on the device (a ragged query longer than N, an end outside the
            # reference, a recompute that missed the forward's cost): a gradient
            # computed past any of these is not returned
            st = sctx.device_status()
            if st != capi.SDTW_OK:
                raise capi.SdtwError(st, "sdtw_backward (device status)")
        return gr, gq, None, None, None


def znormalize(x, offsets=None, out=None, stream=None):
    """Eq. 2 z-normalisation of a batch (sdtw_znormalize): x is [B, N] (or 1-D
    with offsets [B+1]), float32 on a CUDA device; returns out (in place if
    out is x)."""
    if not x.is_cuda or not x.is_contiguous() or x.dtype != torch.float32:
        raise ValueError("x must be a contiguous float32 CUDA tensor")
    if offsets is None:
        if x.dim() == 1:
            B, N = 1, x.numel()
        else:
            B, N = x.shape
    else:
        B, N = offsets.numel() - 1, 1
    if out is None:
        out = torch.empty_like(x)
    st = capi.sdtw_znormalize(_ptr(x), _ptr(out), _ptr(offsets), int(B), int(N), _stream_ptr(stream))
    capi.check(st, "sdtw_znormalize")
    return out


def codebook_fit(ref, sigmas: float = 4.0, stream=None):
    """The reference codebook (sdtw_codebook_fit): a float32 CUDA tensor
    [lo, 1/step, step, 0] for 256 equal bins over mean +- sigmas * S."""
    if not ref.is_cuda or not ref.is_contiguous() or ref.dtype != torch.float32:
        raise ValueError("ref must be a contiguous float32 CUDA tensor")
    params = torch.empty(4, dtype=torch.float32, device=ref.device)
    st = capi.sdtw_codebook_fit(_ptr(ref), ref.numel(), float(sigmas), _ptr(params), _stream_ptr(stream))
    capi.check(st, "sdtw_codebook_fit")
    return params


def codebook_encode(x, params, out=None, stream=None):
    """uint8 codes of x under a codebook (sdtw_codebook_encode); same shape as x."""
    if not x.is_cuda or not x.is_contiguous() or x.dtype != torch.float32:
        raise ValueError("x must be a contiguous float32 CUDA tensor")
    if out is None:
        out = torch.empty(x.shape, dtype=torch.uint8, device=x.device)
    st = capi.sdtw_codebook_encode(_ptr(x), x.numel(), _ptr(params), _ptr(out), _stream_ptr(stream))
    capi.check(st, "sdtw_codebook_encode")
    return out


def sdtw_cost(ref, queries, ctx: SdtwContext, offsets=None, N=None):
    """Differentiable (cost, end); ctx must be an f32 context created with grad=True."""
    if not ctx.grad:
        raise ValueError("the context was created without grad=True")
    return SdtwFunction.apply(ref, queries, offsets, N, ctx)
