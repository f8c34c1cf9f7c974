#!/usr/bin/env python
"""Throughput of SymPix preconditioner blocks on one GB300 (or N, weak scaling).

A step is one pass of the whole hot path over one operator at l_max = 3000,
FWHM 5': kernel table (FP64) -> block sampling D^ + B^T N^-1 B^ -> FP64
Cholesky of every block.  The headline `value` is the mixed path (FP32
contraction); the FP64 and split-FP32 contractions are timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own independent problem (the inverse-noise
map of rank r uses seed 4 + r), so the per-GPU work is fixed as N grows.
"""
from __future__ import annotations

import argparse
import csv
import io
import json
import math
import os
import subprocess
import sys
import tempfile
import time
from concurrent.futures import ThreadPoolExecutor

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "preconditioner block elements/s at l_max=3000: mixed vs FP64, % of roofline"
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP64_NOMINAL = 1.25e12   # dense FP64 FLOP/s, GB300 nominal (recipe table)
FP32_NOMINAL = 152 * 128 * 2 * 2.07e9  # FP32 FMA lanes x 2 x max SM clock


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="lmax3000")
    ap.add_argument("--precision", default="fp32:fp32",
                    help="headline arithmetic as contraction:factor (fp64, fp32x2 or fp32 each)")
    ap.add_argument("--launch", default="graph", choices=["graph", "eager"],
                    help="replay the step as captured CUDA graphs, or call the entry points directly")
    ap.add_argument("--no-autotune", action="store_true", help="keep the default launch shapes")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--arms", default="fp64:fp64,fp32x2:fp32x2",
                    help="other contraction:factor arithmetics timed beside the headline")
    return ap.parse_args()


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except OSError:
        return {}


# -- oracle sample (CPU baseline and reference arm) ---------------------------------------

def oracle_rings(og, nmax=2048, count=16, shift=0):
    """A bounded sample: `count` rings spread over the polar caps whose rings
    hold <= nmax pixels (the oracle's dense Cholesky is O(n^3) per ring)."""
    cand = [j for j in range(og["nrings"]) if og["nring"][j] <= nmax]
    idx = np.linspace(0, len(cand) - 1, count).round().astype(int)
    return [cand[(i + shift) % len(cand)] for i in idx]


def run_oracle_sample(wl, og, ninv, rings, threads):
    from oracle import oracle as O

    def one(j):
        M, _ = O.block(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], ninv, j)
        L, info = O.cholesky(M)
        n = M.shape[0]
        q = np.arange(n)
        nz = np.nonzero(M)
        if len(nz[0]):
            dist = np.minimum((nz[0] - nz[1]) % n, (nz[1] - nz[0]) % n)
            w = int(dist.max())
        else:
            w = 0
        return n * (w + 1) if 2 * w + 1 < n else n * (n + 1) // 2

    t0 = time.perf_counter()
    with ThreadPoolExecutor(max_workers=threads) as ex:
        elems = list(ex.map(one, rings))
    dt = time.perf_counter() - t0
    return int(sum(elems)), dt


# -- clocks ----------------------------------------------------------------------------

class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.3)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r for r in csv.reader(io.StringIO(self.f.read())) if len(r) >= 9]
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.strip().lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(rows[0][2]),
                "power_w_max": max(float(r[3]) for r in rows if r[3].strip() not in ("", "[N/A]")),
                "samples": len(rows), "reasons": sorted(reasons)}


# -- the GPU arm ---------------------------------------------------------------------------

S_BLOCK_PBAND = 0  # the C header's SYMPIX_BLOCK_PBAND


def factor_flops(plan):
    tot = 0.0
    for o in range(plan.nops):
        for j in range(plan.ring0, plan.ring1):
            _, n, w, fmt = plan.block_layout("pband", o, j)
            if fmt == 0:
                m = n - w
                tot += 2.0 * (m * w * (w + 1) / 2 + w * m * w + n * w * (w + 1) / 2) + 2.0 * n
            else:
                tot += n ** 3 / 3.0
    return tot


ALU_PEAK = {"fp64": (FP64_NOMINAL, "nominal FP64 1.25 TFLOP/s (a DFMA probe measured 1.197)"),
            "fp32": (FP32_NOMINAL, "nominal FP32 80.5 TFLOP/s (an FFMA probe measured 73.1)"),
            "fp32x2": (FP32_NOMINAL, "nominal FP32 80.5 TFLOP/s; a split product costs ~16 FP32 flops")}

# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel from one ncu capture of (workload, precision), as summarised under
# profiles/; an entry is removed when its kernel changes.
TRAFFIC = {
    # profiles/dram_lmax3000_mixed_step.md
    ("lmax3000_fwhm5", "fp32:fp32", "k_f32_fused"): 1669556992,
    ("lmax3000_fwhm5", "fp32:fp32", "k_table"): 854528,
}


def kernel_work(plan, grid, wl, elements, sprec, fprec):
    """Algorithmic work of one launch of each kernel: (bound, amount, type),
    amount in bytes for "hbm" and flops for "alu" (type = the arithmetic)."""
    geo = [plan.block_layout("pband", o, j) for o in range(plan.nops) for j in range(plan.ring0, plan.ring1)]
    f32 = [(n, w) for _, n, w, fmt in geo if fmt == S_BLOCK_PBAND and w <= 16]
    band = sum(n * (w + 1) for n, w in f32)
    l11 = sum((n - w) * (w + 1) for n, w in f32)
    l21 = sum(w * (n - w) for n, w in f32)
    npix = grid.npix * plan.nops
    sample_flops = 2.0 * plan.ntriples + plan.nmults
    sample_bytes = elements * 8 + npix * (8 if sprec == "fp64" else 16)
    t_hbm = sample_bytes / (peaks().get("hbm_gbs", 6800.0) * 1e9)
    t_alu = sample_flops / ALU_PEAK[sprec][0]
    return {
        "k_table": ("alu", plan.nslots * plan.nops * (wl.lmax - 1) * 7.0, "fp64"),
        "k_table_coeffs": ("hbm", (wl.lmax + 1) * plan.nops * 32.0, "fp64"),
        "k_split_ninv": ("hbm", npix * 16.0, sprec),
        "k_sample_pband": ("hbm", sample_bytes, sprec) if t_hbm >= t_alu else ("alu", sample_flops, sprec),
        "k_f32_shadow_in": ("hbm", band * 12.0, "fp32"),
        "k_f32_band_pass": ("alu", float(sum((n - w) * (w * (w + 1) + w + 2) for n, w in f32)), "fp32"),
        "k_f32_border_pass": ("alu", float(sum((n - w) * (2 * w * w + w + w * (w + 1)) for n, w in f32)), "fp32"),
        "k_f32_out": ("hbm", (l11 + l21) * 12.0, "fp32"),
        "k_f32_fused": ("alu", float(sum((n - w) * (w * (w + 1) + w + 2 + 2 * w * w + w + w * (w + 1))
                                         for n, w in f32 if w <= 12)), "fp32"),
        "k_factor_band": ("alu", factor_flops(plan), fprec),
    }


def rank_workload(wl, rank):
    """Rank r's independent problem: the workload with every seed shifted by r."""
    from paper_1504_04653_gb300 import workloads as W
    return W.Workload(wl.name, wl.lmax, wl.fwhm_arcmin, wl.band_deg, [s + rank for s in wl.seeds], wl.desc)


def max_over_ranks(x, world, device):
    """The largest x over the ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def job_value(elements_per_rank, ms_max, world):
    """Whole-job throughput: every rank's elements over the slowest rank's time."""
    return world * elements_per_rank / (ms_max * 1e-3)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return reference_arm(args, rank, world)

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__
    if rank == 0:
        __graft_entry__.build()
    if world > 1:
        torch.distributed.barrier()
    from paper_1504_04653_gb300 import sympix as S
    from paper_1504_04653_gb300 import workloads as W

    wl = W.WORKLOADS[args.workload]
    wl = rank_workload(wl, rank)
    grid = S.Grid(wl.lmax)
    plan = S.Plan(grid, wl.radii())
    nbytes, elements = plan.blocks_size("pband")
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    ninv_h = wl.ninv(colat)
    bl_h, dl_h = wl.beams(), wl.priors()
    bl = torch.tensor(bl_h, dtype=torch.float64, device=dev)
    dl = torch.tensor(dl_h, dtype=torch.float64, device=dev)
    ninv = torch.tensor(ninv_h, dtype=torch.float64, device=dev)
    blocks = torch.empty(nbytes // 8, dtype=torch.float64, device=dev)
    info = torch.empty(plan.nblocks, dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.Stream(device=dev)

    # launch shapes: timed on this workload before anything is captured
    tune = None
    if not args.no_autotune:
        sp0, fp0 = args.precision.split(":")
        tune = plan.autotune(bl, dl, ninv, blocks, info, "pband", sp0, fp0, stream=stream)
        torch.cuda.synchronize()
    graphs = {}

    def graph_step(prec):
        if prec not in graphs:
            sprec, fprec = prec.split(":")
            graphs[prec] = S.Step(plan, bl, dl, ninv, blocks, info, "pband", sprec, fprec)
        return graphs[prec]

    def step(prec, ev=None):
        if args.launch == "graph":
            # one graph replay per stage, events between the stages
            g = graph_step(prec)
            for i, bit in enumerate((S.STAGE_TABLE, S.STAGE_SAMPLE, S.STAGE_FACTOR)):
                if ev:
                    ev[i].record(stream)
                g.launch(bit, stream=stream)
            if ev:
                ev[3].record(stream)
            return
        sprec, fprec = prec.split(":")
        if ev:
            ev[0].record(stream)
        S.sympix_kernel_table(plan, bl, dl, stream=stream)
        if ev:
            ev[1].record(stream)
        S.sympix_sample_blocks(plan, ninv, precision=sprec, storage="pband", out=blocks, stream=stream)
        if ev:
            ev[2].record(stream)
        S.sympix_factor_blocks(plan, blocks, storage="pband", precision=fprec, info=info, stream=stream)
        if ev:
            ev[3].record(stream)

    def timed(prec, K, W_):
        with torch.cuda.stream(stream):
            for _ in range(W_):
                step(prec)
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for k in range(K):
            with torch.cuda.stream(stream):
                flush.fill_(float(k))          # evict L2 between steps (outside the events)
                step(prec, evs[k])
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if world > 1:
            torch.distributed.barrier()
        st = np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(3)] for k in range(K)])
        return st, wall

    clocks = Clocks(local)
    main_st, main_wall = timed(args.precision, args.steps, args.warmup)
    clk = clocks.stop()
    info_h = info.cpu().numpy()
    sampled_main = None
    ms_step = float(main_st.sum(axis=1).mean())
    ms_max = max_over_ranks(ms_step, world, dev)
    value = job_value(elements, ms_max, world)

    # other contraction arms (same steps) and their accuracy against FP64
    arms = {}
    ref64 = None
    for prec in [a for a in args.arms.split(",") if a and a != args.precision]:
        st, _ = timed(prec, args.steps, 1)
        arms[prec] = {"value": elements / (float(st.sum(axis=1).mean()) * 1e-3),
                      "ms_per_step": float(st.sum(axis=1).mean()),
                      "stages_ms": dict(zip(["table", "sample", "factor"], st.mean(axis=0).round(4).tolist()))}
    # accuracy against the FP64 GPU path, normwise per block over every
    # (operator, ring) block: sampled blocks of each contraction, and the
    # factors of each full arm on the blocks both arms factored
    acc = {}
    not_pd = {}
    if rank == 0:
        lay = [plan.block_layout("pband", op, j) for op in range(plan.nops) for j in range(plan.ring0, plan.ring1)]
        nb = len(lay)
        starts = torch.tensor([o for o, _, _, _ in lay], dtype=torch.int64, device=dev)
        lens = torch.tensor([n * (2 * w + 1) if fmt == S.BLOCK_PBAND else n * n for _, n, w, fmt in lay],
                            dtype=torch.int64, device=dev)
        bid = torch.repeat_interleave(torch.arange(nb, device=dev), lens)
        first = torch.cumsum(lens, 0) - lens
        pos = starts[bid] + torch.arange(bid.numel(), device=dev) - first[bid]

        def run_once(prec, factored):
            sprec, fprec = prec.split(":")
            with torch.cuda.stream(stream):
                S.sympix_kernel_table(plan, bl, dl, stream=stream)
                S.sympix_sample_blocks(plan, ninv, precision=sprec, storage="pband", out=blocks, stream=stream)
                if factored:
                    S.sympix_factor_blocks(plan, blocks, storage="pband", precision=fprec, info=info, stream=stream)
            torch.cuda.synchronize()
            return blocks[pos], info.clone()

        def blockwise(a, b):
            num = torch.zeros(nb, dtype=torch.float64, device=dev).scatter_reduce_(0, bid, (a - b).abs(), "amax")
            den = torch.zeros(nb, dtype=torch.float64, device=dev).scatter_reduce_(0, bid, b.abs(), "amax")
            return num / den.clamp_min(1e-300)

        for factored in (False, True):
            ref, ref_info = run_once("fp64:fp64", factored)
            if factored:
                not_pd["fp64:fp64"] = int((ref_info != 0).sum())
            for prec in sorted({args.precision, *[a for a in args.arms.split(",") if a]} - {"fp64:fp64"}):
                got, got_info = run_once(prec, factored)
                err = blockwise(got, ref)
                if factored:
                    not_pd[prec] = int((got_info != 0).sum())
                    acc[f"{prec}_info_mismatches_vs_fp64"] = int((got_info != ref_info).sum())
                    err = err[(got_info == 0) & (ref_info == 0)]
                key = f"{prec}_{'factor' if factored else 'blocks'}_vs_fp64_normwise_max"
                acc[key] = float(err.max()) if err.numel() else 0.0
                del got
            del ref
        del pos, bid

    # e2e: the same step through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        bl_p = torch.tensor(bl_h, dtype=torch.float64).pin_memory()
        dl_p = torch.tensor(dl_h, dtype=torch.float64).pin_memory()
        ninv_p = torch.tensor(ninv_h, dtype=torch.float64).pin_memory()
        out_p = torch.empty(nbytes // 8, dtype=torch.float64).pin_memory()
        info_p = torch.empty(plan.nblocks, dtype=torch.int32).pin_memory()

        def e2e_step():
            bl.copy_(bl_p, non_blocking=True)
            dl.copy_(dl_p, non_blocking=True)
            ninv.copy_(ninv_p, non_blocking=True)
            step(args.precision)
            out_p.copy_(blocks, non_blocking=True)
            info_p.copy_(info, non_blocking=True)

        with torch.cuda.stream(stream):
            for _ in range(max(1, args.warmup)):
                e2e_step()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
            for _ in range(args.steps):
                e2e_step()
            e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        h2d = (bl_p.numel() + dl_p.numel() + ninv_p.numel()) * 8
        d2h = out_p.numel() * 8 + info_p.numel() * 4
        e2e = {"value": world * elements / (ms * 1e-3), "unit": "elements/s", "ms_per_step": ms,
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}

    # per-kernel device times: a traced pass of the same steps (direct calls,
    # an event after every launch), then the roofline of the dominant kernel
    # against the peak of the arithmetic (or memory) that bounds it
    pk = peaks()
    hbm = pk.get("hbm_gbs", 6800.0) * 1e9
    stages = dict(zip(["table", "sample", "factor"], main_st.mean(axis=0).tolist()))
    sprec, fprec = args.precision.split(":")
    per_kernel = {}
    plan.set_trace(True)
    sp, fp = args.precision.split(":")
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(float(k))
            plan.trace_read()  # drop anything recorded before this step
            S.sympix_kernel_table(plan, bl, dl, stream=stream)
            S.sympix_sample_blocks(plan, ninv, precision=sp, storage="pband", out=blocks, stream=stream)
            S.sympix_factor_blocks(plan, blocks, storage="pband", precision=fp, info=info, stream=stream)
        for name, ms in plan.trace_read():
            per_kernel.setdefault(name, []).append(ms)
    plan.set_trace(False)
    kern_ms = {k: float(np.mean(v)) for k, v in per_kernel.items()}
    dominant = max(kern_ms, key=kern_ms.get)
    work = kernel_work(plan, grid, wl, elements, sprec, fprec)
    bound, amount, ktype = work.get(dominant, ("alu", 0.0, fprec))
    if bound == "hbm":
        roof = {"kernel": dominant, "bound": "hbm", "achieved": amount / (kern_ms[dominant] * 1e-3) / 1e9,
                "peak": hbm / 1e9, "unit": "GB/s", "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)",
                "algorithmic_bytes_per_launch": amount}
    else:
        peak, src = ALU_PEAK[ktype]
        roof = {"kernel": dominant, "bound": "alu", "achieved": amount / (kern_ms[dominant] * 1e-3) / 1e12,
                "peak": peak / 1e12, "unit": "TFLOP/s", "peak_source": src, "algorithmic_flops_per_launch": amount}
    roof["frac"] = roof["achieved"] / roof["peak"]
    roof["traffic"] = TRAFFIC.get((wl.name, args.precision, dominant))
    roof["kernel_ms"] = kern_ms[dominant]
    roof["timing"] = "CUDA events around each launch on the launching stream, traced pass of the same steps"
    # every kernel against its own bound, for context
    kernels = {}
    for name, ms in kern_ms.items():
        b, a, t = work.get(name, ("alu", 0.0, fprec))
        if b == "hbm":
            kernels[name] = {"ms": round(ms, 4), "bound": "hbm", "gbs": a / (ms * 1e-3) / 1e9,
                             "frac": a / (ms * 1e-3) / hbm}
        else:
            kernels[name] = {"ms": round(ms, 4), "bound": "alu", "tflops": a / (ms * 1e-3) / 1e12,
                             "frac": a / (ms * 1e-3) / ALU_PEAK[t][0]}

    # the pixel-domain convolution g = B^ f on the same plan and table (the
    # N^-1 map stands in for f): FP32 against HBM, FP64 against the FP64 pipe
    conv = {}
    gbuf = torch.empty_like(ninv)
    S.sympix_kernel_table(plan, bl, dl, stream=stream)
    for cp in ("fp32", "fp64"):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for _ in range(max(1, args.warmup)):
                S.sympix_convolve(plan, ninv, precision=cp, out=gbuf, stream=stream)
            for k in range(args.steps):
                flush.fill_(float(k))
                evs[k][0].record(stream)
                S.sympix_convolve(plan, ninv, precision=cp, out=gbuf, stream=stream)
                evs[k][1].record(stream)
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
        px = grid.npix * plan.nops
        ent = {"ms": ms, "pixels_per_s": px / (ms * 1e-3)}
        if cp == "fp32":
            ent.update({"bound": "hbm", "gbs": px * 16.0 / (ms * 1e-3) / 1e9,
                        "frac": px * 16.0 / (ms * 1e-3) / hbm})
        else:
            ent.update({"bound": "alu", "tflops": 2.0 * plan.nmults / (ms * 1e-3) / 1e12,
                        "frac": 2.0 * plan.nmults / (ms * 1e-3) / FP64_NOMINAL})
        conv[cp] = ent

    if args.launch == "graph":
        launches = graph_step(args.precision).kernels(S.STAGE_ALL)
    else:
        launches = sum(plan.launches("pband", sprec, fprec))
    line = {
        "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {"fp32:fp32x2": "f64 kernel table, f32 contraction, split-f32 Cholesky",
                  "fp32:fp32": "f64 kernel table, f32 contraction, f32 Cholesky",
                  "fp64:fp64": "f64"}.get(args.precision, args.precision),
        "data": "synthetic",
        "config": {"workload": wl.name, "lmax": wl.lmax, "fwhm_arcmin": wl.fwhm_arcmin[0], "nops": plan.nops,
                   "npix": int(grid.npix), "elements": int(elements), "storage": "pband",
                   "precision": args.precision, "triples": int(plan.ntriples), "kernel_slots": int(plan.nslots),
                   "l2": "256 MB buffer written between steps, outside the step events",
                   "launch": "one CUDA graph replay per stage" if args.launch == "graph" else "direct calls",
                   "launch_shapes": {"table_cta": plan.tuning()[0], "border_threads": plan.tuning()[1],
                                     "autotuned": tune is not None},
                   "parallelism": f"independent problem per GPU x{world}"},
        "stages_ms": {k: round(v, 4) for k, v in stages.items()},
        "kernel_rooflines": kernels,
        "arms": arms, "accuracy": acc, "roofline": roof, "e2e": e2e,
        "convolution": {"op": "g = B^ f, pixel domain (Eq. convolution-pixel); 16 B algorithmic per pixel",
                        **conv},
        "gpu_launches": launches * args.steps, "clocks": clk,
        "blocks": int(plan.nblocks),
        "blocks_not_positive_definite": not_pd or int((info_h != 0).sum()),
    }

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        og = O.grid(wl.lmax)
        rings = oracle_rings(og)
        threads = min(16, os.cpu_count() or 1)
        el, dt = run_oracle_sample(wl, og, ninv_h[0], rings, threads)
        line["cpu_baseline"] = {"value": el / dt, "unit": "elements/s", "cores": threads, "kind": "oracle",
                                "sample": f"{len(rings)} polar-cap rings (n <= 2048) of the same workload, "
                                          f"one thread each: {el} elements in {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def reference_arm(args, rank, world):
    """The oracle timed as it stands, on the host cores (rank 0 only)."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1504_04653_gb300 import workloads as W
    O.build()
    wl = W.WORKLOADS[args.workload]
    og = O.grid(wl.lmax)
    colat = W.pixel_colatitude(og["theta"], og["nring"], og["ring_offset"], og["ring_stride"], og["npix"])
    ninv = wl.ninv(colat)[0]
    threads = min(16, os.cpu_count() or 1)
    for s in range(args.warmup):
        run_oracle_sample(wl, og, ninv, oracle_rings(og, count=threads, shift=s), threads)
    tot_el, tot_t = 0, 0.0
    for s in range(args.steps):
        el, dt = run_oracle_sample(wl, og, ninv, oracle_rings(og, count=threads, shift=1000 + s), threads)
        tot_el += el
        tot_t += dt
    v = tot_el / tot_t
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "elements/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "lmax": wl.lmax, "fwhm_arcmin": wl.fwhm_arcmin[0]},
        "cpu_baseline": {"value": v, "unit": "elements/s", "cores": threads, "kind": "oracle",
                         "sample": f"per step {threads} polar-cap rings (n <= 2048), one thread each"},
        "e2e": {"value": v, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


if __name__ == "__main__":
    main()
