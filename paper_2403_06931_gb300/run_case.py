"""Run the library on one seeded workload from the command line.

    python -m paper_2403_06931_gb300.run_case --workload paper --B 152 --reps 3 [--backward] [--dtype i8]

Used to profile a single kernel on a chosen shape (e.g. under ncu) and as a
quick end-to-end check: prints the plan, the mean kernel time and GCUPS.
"""
from __future__ import annotations

import argparse
import json

import torch

from . import inputs
from .sdtw import SdtwContext


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", default="paper", choices=["paper", "ragged", "small", "grad", "stretched"])
    ap.add_argument("--B", type=int, default=None, help="queries (default: the workload's)")
    ap.add_argument("--N", type=int, default=None)
    ap.add_argument("--M", type=int, default=None)
    ap.add_argument("--dtype", default="f32", choices=["f32", "i8", "u8", "f16"],
                    help="u8: the batch encoded with the reference codebook; f16: the batch rounded to binary16")
    ap.add_argument("--reps", type=int, default=3, help="timed runs after one warm-up")
    ap.add_argument("--backward", action="store_true")
    ap.add_argument("--autotune", action="store_true")
    ap.add_argument("--seg-width", type=int, default=0)
    ap.add_argument("--warps", type=int, default=0)
    ap.add_argument("--tile-rows", type=int, default=0)
    ap.add_argument("--ckpt-stride", type=int, default=0, help="steps between wavefront checkpoints (8, 16, 32, 64)")
    ap.add_argument("--bwd-warps", type=int, default=0,
                    help="warps per query in the backward (1 = the walker alone; 0 = the library's choice)")
    ap.add_argument("--prune-gap", type=int, default=0,
                    help="integer modes: early-INF pruning of cells whose samples differ by more than this")
    ap.add_argument("--keep-checkpoints", action="store_true",
                    help="the forward stores backward checkpoints (implied by --backward)")
    ap.add_argument("--znorm", action="store_true",
                    help="time the batch z-normalisation (Eq. 2) of B x N raw random walks instead of the fill")
    a = ap.parse_args()
    if a.znorm:
        return run_znorm(a)

    kw = {k: v for k, v in (("B", a.B), ("N", a.N), ("M", a.M)) if v is not None}
    if a.workload == "ragged":
        kw = {k: v for k, v in (("B", a.B), ("M", a.M)) if v is not None}
        w = inputs.ragged_fp32(**kw)
    elif a.workload == "paper":
        w = inputs.paper_i8(**kw) if a.dtype == "i8" else inputs.paper_fp32(**kw)
    else:
        w = inputs.by_name(a.workload)
    dev = torch.device("cuda", torch.cuda.current_device())
    ref = torch.from_numpy(w.ref).to(dev)
    qs = torch.from_numpy(w.queries).to(dev)
    offs = torch.from_numpy(w.offsets).to(dev) if w.offsets is not None else None
    if a.dtype == "f16":
        ref, qs = ref.to(torch.float16), qs.to(torch.float16)
    elif a.dtype == "u8":
        from .sdtw import codebook_encode, codebook_fit
        params = codebook_fit(ref)
        ref, qs = codebook_encode(ref, params), codebook_encode(qs, params)
    N = int(w.lengths.max())
    ctx = SdtwContext(dtype=a.dtype, max_ref_len=w.M, max_batch=w.B, max_query_len=N,
                      max_total_query_len=qs.numel(), grad=a.backward or a.keep_checkpoints,
                      keep_checkpoints=a.backward or a.keep_checkpoints,
                      seg_width=a.seg_width, warps_per_query=a.warps, tile_rows=a.tile_rows,
                      ckpt_stride=a.ckpt_stride, prune_gap=a.prune_gap,
                      bwd_warps=a.bwd_warps)
    if a.autotune:
        ctx.autotune(ref, qs, offsets=offs, N=N if offs is not None else None)
    Nr = N if offs is not None else None
    times, fwd_times = [], []
    for rep in range(a.reps + 1):  # the first run is an untimed warm-up
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record()
        cost, end = ctx.forward(ref, qs, offsets=offs, N=Nr)
        e1.record()
        if a.backward:
            ctx.backward(ref, qs, end, torch.ones(w.B, device=dev), offsets=offs, N=Nr)
        e2.record()
        e2.synchronize()
        if rep > 0:
            times.append(e0.elapsed_time(e2))
            fwd_times.append(e0.elapsed_time(e1))
    status = ctx.device_status()
    ms = sum(times) / len(times)
    fms = sum(fwd_times) / len(fwd_times)
    print(json.dumps({"workload": w.name, "B": w.B, "N": N, "M": w.M, "dtype": a.dtype, "backward": a.backward,
                      "plan": ctx.plan(w.B, N, w.M, ragged=offs is not None), "ms": round(ms, 3),
                      "fwd_ms": round(fms, 3), "bwd_ms": round(ms - fms, 3),
                      "gcups": round(w.cells / (ms * 1e-3) / 1e9, 2), "device_status": status}))
    ctx.close()
    if status != 0:
        raise SystemExit(f"device status {status}")


def run_znorm(a):
    from .sdtw import znormalize
    B, N = a.B or 512, a.N or 2000
    dev = torch.device("cuda", torch.cuda.current_device())
    x = torch.from_numpy(inputs.random_walks(B, N, seed=11)).to(dev)
    z = torch.empty_like(x)
    times = []
    for rep in range(a.reps + 1):  # the first run is an untimed warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        znormalize(x, out=z)
        e1.record()
        e1.synchronize()
        if rep > 0:
            times.append(e0.elapsed_time(e1))
    ms = sum(times) / len(times)
    print(json.dumps({"workload": f"znorm_{B}x{N}", "B": B, "N": N, "ms": round(ms, 4),
                      "gbs": round(8 * B * N / (ms * 1e-3) / 1e9, 1)}))


if __name__ == "__main__":
    main()
