"""Throughput of batched subsequence DTW on one GB300 (or N, one rank each).

Step = one differentiable pass over the paper's batch (Section 6: 512 queries
of 2,000 samples against a 100,000-sample reference, z-normalised random
walks): sdtw_forward (cost and end of every query, checkpoints kept) followed
by sdtw_backward (walk-back gradients w.r.t. queries and reference), through
the C ABI with device-resident inputs.  value = GCUPS of that step
(B*N*M cells / step seconds); the forward alone, the backward alone, the int8
mode and the ragged persistent form (2,048 queries of U[200,4000] samples vs
1,000,000, one persistent launch replayed from a CUDA graph) are reported
beside it under "forms".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the CPU oracle (FP64, all host cores) on a bounded
sample of the same workload.  Under torchrun (N > 1) every rank runs its own
batch (weak scaling); value and e2e are whole-job throughputs over the slowest
rank's time, and the host baseline is reported on the 1-GPU line only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GCUPS fwd/bwd, 512×2000 queries vs 100k ref, 1 GB300; % ALU roofline; vs host oracle"
OPS_PER_CELL = 6          # instruction-issue roofline: ops per DP cell (subtract, 2 min, FMA + overheads)
LANES_PER_SM = 128        # 4 schedulers x 32 lanes
L2_FLUSH_BYTES = 512 << 20

# ncu DRAM traffic of one checkpointing forward launch on the paper batch, per
# plan (seg_width, tile_rows, warps_per_query, ckpt_stride), valid only while
# the forward kernel's code hashes to FWD_SRC_SHA (else, or for another plan,
# reported as null).  Captured on 128 of the 512 queries (the writes are the
# per-query checkpoints) and scaled by 4 to the 512-query launch;
# profiles/fwd_chain_kernel_f32_ckpt_W32_RT4_KS16_paper_512x2000_vs_100000.md
FWD_SRC_SHA = "54359229b4890b5f"
FWD_TRAFFIC_BYTES = {
    (32, 4, 4, 16): 4 * (2_547_968 + 2_388_259_840),
    (32, 4, 4, 32): 4 * (2_154_240 + 1_364_210_432),
    (28, 8, 4, 16): 4 * (8_784_640 + 1_548_449_792),
    (28, 8, 4, 8): 4 * (17_545_984 + 2_702_749_952),
    (28, 4, 4, 32): 4 * (2_135_296 + 1_429_650_432),
    (28, 4, 4, 16): 4 * (2_383_360 + 2_460_893_696),
    (32, 4, 4, 8): 4 * (3_400_704 + 4_436_850_944),
    (28, 8, 4, 32): 4 * (4_549_888 + 971_104_768),
    (24, 8, 4, 16): 4 * (9_507_584 + 1_694_594_048),
    (24, 8, 4, 8): 4 * (21_463_808 + 2_920_252_928),
}


def src_sha(*paths):
    """Hash of CUDA sources' code: comments and blank lines do not count, so
    a comment edit keeps counters taken on the kernel valid."""
    import re
    text = ""
    for path in paths:
        with open(path) as f:
            text += f.read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = [ln.split("//", 1)[0].rstrip() for ln in text.splitlines()]
    code = "\n".join(ln for ln in lines if ln.strip())
    return hashlib.sha256(code.encode()).hexdigest()[:16]


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f), "measured"
    except OSError:
        return {"sm_max_mhz": 2070.0, "hbm_gbs": 6800.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms.  Entering the
    context waits for the first sample, so that the samples counted (those
    written between entering and leaving) fall inside the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples (the JSON line carries their summary): SDTW_CLOCKS_DIR, else the temp directory
        self.path = os.path.join(os.environ.get("SDTW_CLOCKS_DIR") or tempfile.gettempdir(),
                                 f"sdtw_clocks_gpu{gpu_index}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "20"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None
            return self
        t0 = time.perf_counter()
        while self._lines() < 1 and time.perf_counter() - t0 < 5.0 and self.proc.poll() is None:
            time.sleep(0.02)
        self.n0 = self._lines()
        return self

    def _lines(self):
        try:
            with open(self.path) as f:
                return sum(1 for _ in f)
        except OSError:
            return 0

    def __exit__(self, *exc):
        if self.proc is not None:
            self.n1 = self._lines()
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        with open(self.path) as f:
            lines = f.readlines()
        # the samples written while the timed region ran; a region shorter than
        # the interval keeps the first sample after it began
        lines = lines[self.n0:max(self.n1, self.n0 + 1)]
        for line in lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[2]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        seen = sorted({names[k] for _, _, r in rows for k in range(4) if r[k].lower() == "active"})
        sm = [r[0] for r in rows]
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(r[1] for r in rows),
                "samples": len(rows), "reasons": seen}


# ------------------------------------------------------------------ ours --

def max_over_ranks(value, world, dev):
    """The largest of a per-rank value over all ranks (the job's step time is
    its slowest rank's); a plain float when running alone."""
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64)
    if world > 1:
        import torch.distributed as dist
        t = t.to(dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gcups(world, cells_per_rank, step_ms_max):
    """Whole-job throughput: every rank processes its own batch of cells_per_rank
    cells (weak scaling, no collective on the data path) in at most step_ms_max."""
    return world * cells_per_rank / (step_ms_max * 1e-3) / 1e9


def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_2403_06931_gb300 import build as libbuild
    from paper_2403_06931_gb300 import capi, inputs
    from paper_2403_06931_gb300.sdtw import SdtwContext

    libbuild.build()
    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)

    w = inputs.paper_fp32(seed=inputs.SEED_BASE + 2 + rank)
    B, N, M = w.B, w.N, w.M
    cells = B * N * M
    ref = torch.from_numpy(w.ref).to(dev)
    qs = torch.from_numpy(w.queries).to(dev)
    cost = torch.empty(B, device=dev)
    end = torch.empty(B, dtype=torch.int64, device=dev)
    gc = torch.ones(B, device=dev)
    gq = torch.empty_like(qs)
    gr = torch.empty_like(ref)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    ctx = SdtwContext(max_ref_len=M, max_batch=B, max_query_len=N, grad=True, keep_checkpoints=True)
    if not args.no_autotune:
        ctx.autotune(ref, qs)
    tuned = ctx.plan(B, N, M, backward=True)
    h = ctx.handle
    P = lambda t: t.data_ptr()  # noqa: E731

    def fwd():
        capi.check(capi.sdtw_forward(h, P(ref), M, P(qs), None, B, N, P(cost), P(end), sp), "sdtw_forward", h)

    def bwd():
        capi.check(capi.sdtw_backward(h, P(ref), M, P(qs), None, B, N, P(end), P(gc), P(gq), P(gr), None, sp),
                   "sdtw_backward", h)

    def step():
        fwd()
        bwd()

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if ctx.device_status() != capi.SDTW_OK:
        raise RuntimeError("device status error during warm-up")

    # timed region: K steps, L2 flushed before each (outside the events)
    e_f0, e_f1, e_b1 = [ev() for _ in range(args.steps)], [ev() for _ in range(args.steps)], \
        [ev() for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local_rank) as clk:
        t_wall = time.perf_counter()
        for k in range(args.steps):
            flush.zero_()
            e_f0[k].record(stream)
            fwd()
            e_f1[k].record(stream)
            bwd()
            e_b1[k].record(stream)
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall
    if world > 1:
        dist.barrier()
    fwd_ms = [e_f0[k].elapsed_time(e_f1[k]) for k in range(args.steps)]
    bwd_ms = [e_f1[k].elapsed_time(e_b1[k]) for k in range(args.steps)]
    step_ms = sum(fwd_ms) / args.steps + sum(bwd_ms) / args.steps
    if ctx.device_status() != capi.SDTW_OK:
        raise RuntimeError("device status error in the timed region")
    step_ms_max = max_over_ranks(step_ms, world, dev)
    clocks = clk.summary()

    # e2e: host buffers through the C ABI, copies inside the timed region
    href = w.ref.copy()
    hq = w.queries.copy()
    pin = lambda a: torch.from_numpy(a).pin_memory()  # noqa: E731
    t_ref, t_q, t_gc = pin(href), pin(hq), pin(np.ones(B, np.float32))
    t_cost, t_end = pin(np.empty(B, np.float32)), pin(np.empty(B, np.int64))
    t_gq, t_gr = pin(np.empty_like(hq)), pin(np.empty_like(href))
    e2e_ctx = SdtwContext(max_ref_len=M, max_batch=B, max_query_len=N, grad=True, keep_checkpoints=True)

    def e2e_step():
        capi.check(capi.sdtw_forward_backward_host(
            e2e_ctx.handle, P(t_ref), M, P(t_q), None, B, N, P(t_gc), P(t_cost), P(t_end), P(t_gq), P(t_gr), None,
            sp), "sdtw_forward_backward_host", e2e_ctx.handle)

    if not args.no_autotune:
        e2e_ctx.autotune(ref, qs)
    for _ in range(2):
        e2e_step()
    e2e_ms = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e2e_step()
        e2e_ms.append((time.perf_counter() - t0) * 1e3)
    e2e_ctx.close()
    # whole-job end-to-end throughput: every rank's own median, the slowest rank's
    e2e_ms_max = max_over_ranks(statistics.median(e2e_ms), world, dev)
    h2d = href.nbytes + hq.nbytes + 4 * B
    d2h = 4 * B + 8 * B + hq.nbytes + href.nbytes

    forms = {}
    if rank == 0 and not args.no_forms:
        forms["autograd"] = run_autograd_form(args, ctx, ref, qs, B, N, M, flush, stream)
        forms.update(run_forms(args, ctx, w, ref, qs, cost, end, flush, stream, dev))

    ctx.close()
    if rank != 0:
        return None

    pk, pk_kind = peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    f_max = float(pk.get("sm_max_mhz", 2070.0))
    peak_gcups = sms * LANES_PER_SM * f_max * 1e6 / OPS_PER_CELL / 1e9
    fwd_avg = sum(fwd_ms) / len(fwd_ms)
    achieved = cells / (fwd_avg * 1e-3) / 1e9
    csrc = os.path.join(ROOT, "paper_2403_06931_gb300", "csrc")
    fwd_sha = src_sha(os.path.join(csrc, "sdtw_fill.cuh"), os.path.join(csrc, "sdtw_cell.cuh"))
    pkey = (tuned["seg_width"], tuned["tile_rows"], tuned["warps_per_query"], tuned["ckpt_stride"])
    traffic = FWD_TRAFFIC_BYTES.get(pkey) if FWD_SRC_SHA == fwd_sha else None
    roof = {"bound": "alu", "kernel": "fwd_chain_kernel", "achieved": round(achieved, 1),
            "peak": round(peak_gcups, 1), "unit": "GCUPS", "frac": round(achieved / peak_gcups, 4),
            "traffic": traffic,
            "peak_basis": f"{sms} SMs x {LANES_PER_SM} lanes x {f_max:.0f} MHz ({pk_kind} max SM clock) "
                          f"/ {OPS_PER_CELL} ops per cell"}
    if clocks.get("sm_mhz"):
        roof["frac_at_sampled_clock"] = round(achieved / (sms * LANES_PER_SM * clocks["sm_mhz"] * 1e6
                                                          / OPS_PER_CELL / 1e9), 4)
    value = job_gcups(world, cells, step_ms_max)
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": "GCUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms_max, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"sdtw_fp32_{B}x{N}_vs_{M}: forward (cost, end, checkpoints) + backward "
                               "(walk-back gradients)", "B": B, "N": N, "M": M, "cells_per_step": cells,
                   "seed": inputs.SEED_BASE + 2 + rank, "plan": tuned,
                   "l2": "flushed (512 MiB write) before every timed step",
                   "parallelism": f"replicas x{world}, no collective on the data path"},
        "fwd_gcups": round(cells / (fwd_avg * 1e-3) / 1e9, 2),
        "bwd_gcups": round(cells / (sum(bwd_ms) / len(bwd_ms) * 1e-3) / 1e9, 2),
        "fwd_ms": round(fwd_avg, 3), "bwd_ms": round(sum(bwd_ms) / len(bwd_ms), 3),
        "wall_ms_per_step_incl_flush": round(t_wall * 1e3 / args.steps, 3),
        "roofline": roof,
        "e2e": {"value": round(job_gcups(world, cells, e2e_ms_max), 2), "unit": "GCUPS",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": round(e2e_ms_max, 3),
                "api": "sdtw_forward_backward_host (pinned host buffers)"},
        "gpu_launches": 3 * args.steps,
        "clocks": clocks,
        "device": {"name": torch.cuda.get_device_name(dev), "sms": sms},
        "forms": forms,
    }
    if not args.no_cpu_baseline and world == 1:   # the host baseline belongs to the 1-GPU line
        out["cpu_baseline"] = cpu_baseline(args, w)
    return out


def run_autograd_form(args, ctx, ref, qs, B, N, M, flush, stream):
    """The differentiable step as a PyTorch user runs it: sdtw_cost (the
    torch.autograd.Function over sdtw_forward) and .backward() (sdtw_backward,
    then the device-status check, which synchronises the stream), on the
    headline's context and batch, L2 flushed before each step."""
    import torch

    from paper_2403_06931_gb300.sdtw import sdtw_cost

    r = ref.detach().clone().requires_grad_(True)
    x = qs.detach().clone().requires_grad_(True)
    gc = torch.ones(B, device=ref.device)

    def step():
        r.grad = None
        x.grad = None
        c, _ = sdtw_cost(r, x, ctx)
        c.backward(gc)

    for _ in range(2):
        step()
    torch.cuda.synchronize()
    ts = []
    for _ in range(max(3, args.steps // 4)):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ms = sum(ts) / len(ts)
    return {"gcups": round(B * N * M / (ms * 1e-3) / 1e9, 2), "ms": round(ms, 3),
            "api": "sdtw_cost(ref, queries, ctx) then cost.backward(): forward with checkpoints, backward, "
                   "device-status check"}


def run_forms(args, ctx, w, ref, qs, cost, end, flush, stream, dev):
    """Forward alone, int8, binary16 and codebook forwards, the normaliser, and
    the ragged persistent form under a CUDA graph."""
    import torch

    from paper_2403_06931_gb300 import capi, inputs
    from paper_2403_06931_gb300.sdtw import SdtwContext

    forms = {}
    B, N, M = w.B, w.N, w.M
    cells = B * N * M

    def timed(fn, reps):
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return sum(ts) / len(ts)

    # forward only, no checkpoints
    fctx = SdtwContext(max_ref_len=M, max_batch=B, max_query_len=N)
    fplan = fctx.plan(B, N, M) if args.no_autotune else fctx.autotune(ref, qs)
    fctx.forward(ref, qs, out=(cost, end))
    ms = timed(lambda: fctx.forward(ref, qs, out=(cost, end)), 5)
    forms["forward_f32"] = {"gcups": round(cells / (ms * 1e-3) / 1e9, 2), "ms": round(ms, 3), "plan": fplan}
    fctx.close()

    # int8 inputs, int32 costs
    wi = inputs.paper_i8()
    ri = torch.from_numpy(wi.ref).to(dev)
    qi = torch.from_numpy(wi.queries).to(dev)
    ci = torch.empty(B, dtype=torch.int32, device=dev)
    ictx = SdtwContext(dtype="i8", max_ref_len=M, max_batch=B, max_query_len=N)
    iplan = ictx.plan(B, N, M) if args.no_autotune else ictx.autotune(ri, qi)
    ictx.forward(ri, qi, out=(ci, end))
    ms = timed(lambda: ictx.forward(ri, qi, out=(ci, end)), 5)
    forms["forward_i8"] = {"gcups": round(cells / (ms * 1e-3) / 1e9, 2), "ms": round(ms, 3), "plan": iplan}
    ictx.close()

    # binary16 (the paper's precision, Section 5.2): two queries per thread as
    # __half2; the same batch rounded to binary16.  Its difference from the FP64
    # DP of the same samples is reported on a few queries (the oracle on the
    # host), beside the throughput.
    h_ref, h_q = ref.to(torch.float16), qs.to(torch.float16)
    hctx = SdtwContext(dtype="f16", max_ref_len=M, max_batch=B, max_query_len=N)
    hplan = hctx.plan(B, N, M) if args.no_autotune else hctx.autotune(h_ref, h_q)
    hc, he = hctx.forward(h_ref, h_q)
    ms = timed(lambda: hctx.forward(h_ref, h_q, out=(hc, he)), 5)
    forms["forward_f16"] = {"gcups": round(cells / (ms * 1e-3) / 1e9, 2), "ms": round(ms, 3), "plan": hplan,
                            "arithmetic": "binary16, two queries per thread (__half2), no rebasing"}
    if not args.no_cpu_baseline:
        import oracle
        k = 4
        y64 = h_ref.cpu().numpy().astype(np.float64)
        x64 = h_q[:k].cpu().numpy().astype(np.float64)
        c64, _ = oracle.forward_batch(y64, x64, threads=min(k, host_threads()))
        c16 = hc[:k].cpu().numpy().astype(np.float64)
        forms["forward_f16"]["rel_err_vs_fp64"] = {"queries": k, "max": float(np.max(np.abs(c16 - c64) / c64)),
                                                   "mean": float(np.mean(np.abs(c16 - c64) / c64))}
    hctx.close()

    # the reference codebook of Section 8: fit on the reference, encode the
    # batch to uint8 codes, the exact int32 DP on the codes
    from paper_2403_06931_gb300.sdtw import codebook_encode, codebook_fit
    params = codebook_fit(ref)
    cr, cq = codebook_encode(ref, params), codebook_encode(qs, params)
    ms_enc = timed(lambda: codebook_encode(qs, params, out=cq), 5)
    uctx = SdtwContext(dtype="u8", max_ref_len=M, max_batch=B, max_query_len=N)
    uplan = uctx.plan(B, N, M) if args.no_autotune else uctx.autotune(cr, cq)
    ui = torch.empty(B, dtype=torch.int32, device=dev)
    uctx.forward(cr, cq, out=(ui, end))
    ms = timed(lambda: uctx.forward(cr, cq, out=(ui, end)), 5)
    forms["forward_u8_codebook"] = {"gcups": round(cells / (ms * 1e-3) / 1e9, 2), "ms": round(ms, 3), "plan": uplan,
                                    "encode_ms": round(ms_enc, 4),
                                    "encode_gbs": round(5 * B * N / (ms_enc * 1e-3) / 1e9, 1),
                                    "codebook": "mean +- 4 S of the reference, 256 equal bins"}
    uctx.close()
    # early-INF pruning (Section 8, opt-in, changes results): cells whose codes
    # differ by more than 32 (one standard deviation of the reference) cost +inf
    pctx = SdtwContext(dtype="u8", max_ref_len=M, max_batch=B, max_query_len=N, prune_gap=32)
    pplan = pctx.plan(B, N, M) if args.no_autotune else pctx.autotune(cr, cq)
    pctx.forward(cr, cq, out=(ui, end))
    ms = timed(lambda: pctx.forward(cr, cq, out=(ui, end)), 5)
    forms["forward_u8_codebook_pruned"] = {"gcups": round(cells / (ms * 1e-3) / 1e9, 2), "ms": round(ms, 3),
                                           "plan": pplan, "prune_gap": 32,
                                           "queries_with_no_path": int((end < 0).sum().item())}
    pctx.close()

    # batch z-normalisation (Section 5.1, Eq. 2) of query batches shaped like
    # the paper's (512 x 2,000 samples, as its Table 1 times it).  HBM-bound:
    # one read and one write per sample.  A microsecond kernel after an L2
    # flush would mostly measure the flush's write-back, so one launch covers
    # 32 such batches (131 MB, more than L2) and the time is reported per batch.
    from paper_2403_06931_gb300.sdtw import znormalize
    nb = 32
    zin = torch.from_numpy(inputs.random_walks(nb * B, N, seed=11)).to(dev)
    zout = torch.empty_like(zin)
    znormalize(zin, out=zout)
    ts = []
    for _ in range(10):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        znormalize(zin, out=zout)
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    ms = sum(ts) / len(ts)
    zbytes = 8 * nb * B * N
    pk, pk_kind = peaks()
    hbm = pk.get("hbm_gbs")
    forms["znormalize"] = {"series": f"{nb} batches of {B} x {N}", "ms_per_batch": round(ms / nb, 5),
                           "gsps": round(nb * B * N / (ms * 1e-3) / 1e9, 2),
                           "gbs": round(zbytes / (ms * 1e-3) / 1e9, 1),
                           "hbm_frac": round(zbytes / (ms * 1e-3) / 1e9 / hbm, 4) if hbm else None,
                           "bytes_per_launch": zbytes, "peak_basis": f"hbm_gbs, {pk_kind}",
                           "note": "one read and one write per sample; inputs larger than L2, one launch"}
    del zin, zout
    rin = torch.from_numpy(inputs.random_walks(1, M, seed=12).reshape(-1)).to(dev)
    ms = timed(lambda: znormalize(rin, out=rin), 5)
    forms["znormalize"]["reference_ms"] = round(ms, 4)

    if not args.no_ragged:
        wr = inputs.ragged_fp32()
        Nr = int(wr.lengths.max())
        rr = torch.from_numpy(wr.ref).to(dev)
        qr = torch.from_numpy(wr.queries).to(dev)
        orr = torch.from_numpy(wr.offsets).to(dev)
        cr = torch.empty(wr.B, device=dev)
        er = torch.empty(wr.B, dtype=torch.int64, device=dev)
        rctx = SdtwContext(max_ref_len=wr.M, max_batch=wr.B, max_query_len=Nr, max_total_query_len=qr.numel())
        if args.no_autotune:
            rplan = rctx.plan(wr.B, Nr, wr.M, ragged=True)
        else:
            # tuned on a seeded sample of 2 x 608 queries (twice the resident
            # CTAs, so that the persistent queue balances as on the whole batch;
            # the same shape class) at about 60% of the whole batch's time
            k = min(wr.B, 1216)
            pick = np.sort(np.random.default_rng(5).choice(wr.B, size=k, replace=False))
            sub = np.concatenate([wr.query(int(q)) for q in pick]).astype(np.float32)
            soff = np.zeros(k + 1, dtype=np.int64)
            soff[1:] = np.cumsum(wr.lengths[pick])
            rctx.autotune(rr, torch.from_numpy(sub).to(dev), offsets=torch.from_numpy(soff).to(dev), N=Nr)
            rplan = rctx.plan(wr.B, Nr, wr.M, ragged=True)
        rctx.forward(rr, qr, offsets=orr, N=Nr, out=(cr, er))
        torch.cuda.synchronize()
        eager_c, eager_e = cr.clone(), er.clone()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            rctx.forward(rr, qr, offsets=orr, N=Nr, out=(cr, er))
        # the replayed graph must reproduce the eager call bit for bit before it is timed
        cr.fill_(float("nan"))
        er.fill_(-7)
        g.replay()
        torch.cuda.synchronize()
        if not (torch.equal(cr, eager_c) and torch.equal(er, eager_e)):
            raise RuntimeError("ragged forward replayed from a CUDA graph differs from the eager call")
        ms = timed(g.replay, 3)
        assert rctx.device_status() == capi.SDTW_OK
        forms["ragged_persistent_graph"] = {
            "workload": wr.name, "cells": wr.cells, "gcups": round(wr.cells / (ms * 1e-3) / 1e9, 2),
            "ms": round(ms, 3), "plan": rplan, "launch": "one persistent kernel, replayed from a CUDA graph",
            "replay_equals_eager": True}
        rctx.close()
    return forms


# ------------------------------------------------------------ CPU oracle --

def mem_available_bytes():
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 8 << 30


def walkback_threads(w, threads):
    """Concurrent walk-backs allowed: each holds an N x M double matrix; use at
    most a quarter of the host's available memory."""
    per = 8 * w.N * w.M
    return max(1, min(threads, int(0.25 * mem_available_bytes() // per)))


def oracle_step(w, idx, threads):
    """The oracle's differentiable step on queries idx: forward (cost, end) on
    all threads, then walk-back over the filled matrix and the path gradient
    (memory-bounded concurrency)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    y = w.ref.astype(np.float64)
    xs = [w.query(q).astype(np.float64) for q in idx]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        fw = list(ex.map(lambda x: oracle.forward(x, y), xs))

    def back(k):
        cells, _ = oracle.walkback(xs[k], y, fw[k][1])
        return oracle.path_gradient(xs[k], y, cells)

    with ThreadPoolExecutor(max_workers=walkback_threads(w, threads)) as ex:
        list(ex.map(back, range(len(idx))))


def cpu_model():
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    import platform
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith("model name"):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return platform.processor() or platform.machine()


def host_threads():
    return max(1, len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1))


def sample_size(threads):
    return max(1, min(threads, 16))


def cpu_baseline(args, w=None):
    from paper_2403_06931_gb300 import inputs
    import oracle
    oracle.build()
    w = w or inputs.paper_fp32()
    threads = min(host_threads(), 16)
    k = sample_size(threads)
    idx = list(range(k))
    t0 = time.perf_counter()
    oracle_step(w, idx, threads)
    dt = time.perf_counter() - t0
    cells = k * w.N * w.M
    # one core: the forward and walk-back of one query on a single thread
    t1 = time.perf_counter()
    oracle_step(w, [k % w.B], 1)
    dt1 = time.perf_counter() - t1
    return {"value": round(cells / dt / 1e9, 4), "unit": "GCUPS", "cores": threads, "kind": "oracle",
            "cpu": cpu_model(),
            "sample": f"{k} of {w.B} queries ({w.N} x {w.M}): FP64 forward on {threads} threads, then walk-back "
                      f"+ path gradient on {walkback_threads(w, threads)} threads, {dt:.1f} s",
            "one_core": {"value": round(w.N * w.M / dt1 / 1e9, 4), "unit": "GCUPS",
                         "sample": f"1 query, forward + walk-back + path gradient on 1 thread, {dt1:.1f} s"}}


def run_reference(args):
    from paper_2403_06931_gb300 import inputs
    import oracle
    oracle.build()
    w = inputs.paper_fp32()
    threads = min(host_threads(), 16)
    k = sample_size(threads)
    idx = list(range(k))
    for _ in range(args.warmup):
        oracle_step(w, idx[:1], 1)
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle_step(w, idx, threads)
        ts.append(time.perf_counter() - t0)
    ms = 1e3 * sum(ts) / len(ts)
    cells = k * w.N * w.M
    v = round(cells / (ms * 1e-3) / 1e9, 4)
    return {"metric": METRIC, "value": v, "unit": "GCUPS", "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 3), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": f"sdtw_fp32_{w.B}x{w.N}_vs_{w.M}: oracle forward + walk-back gradient, "
                                   f"{k}-query sample per step", "B": w.B, "N": w.N, "M": w.M},
            "cpu_baseline": {"value": v, "unit": "GCUPS", "cores": threads, "kind": "oracle", "cpu": cpu_model(),
                             "sample": f"{k} of {w.B} queries per step, warm-up on 1 query"},
            "e2e": {"value": v, "unit": "GCUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-forms", action="store_true", help="skip the forward/int8/ragged side measurements")
    ap.add_argument("--no-ragged", action="store_true", help="skip the ragged persistent form")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the library's default plans instead of timing candidates (for profiling runs)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps(run_reference(args)), flush=True)
        return

    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    out = run_ours(args, rank, world, local_rank)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
