#!/usr/bin/env python
"""Throughput of SymPix preconditioner blocks on one GB300 (or N, weak scaling).

A step is one pass of the whole hot path over one operator at l_max = 3000,
FWHM 5': kernel table (FP64) -> block sampling D^ + B^T N^-1 B^ -> Cholesky
of every block.  The headline `value` is the mixed path (FP32 contraction,
FP32 factor with FP64 rescue); the FP64 and split-FP32 arms are timed beside
it, and further workloads (l_max = 1500 with an FP64 factor, 32 operators at
l_max = 1000, and the band blocks of the paper's DP grid at l_max = 500,
k = 8) are timed as sub-lines under "configs".

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own independent problem (the inverse-noise
map of rank r uses seed 4 + r), so the per-GPU work is fixed as N grows.
"""
from __future__ import annotations

import argparse
import csv
import hashlib
import io
import json
import math
import os
import platform
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
CSRC = os.path.join(ROOT, "paper_1504_04653_gb300", "csrc")
FP64_NOMINAL = 1.25e12   # dense FP64 FLOP/s, GB300 nominal
FP32_NOMINAL = 152 * 128 * 2 * 2.07e9  # FP32 FMA lanes x 2 x max SM clock
SPLIT_COST = 8.0  # FP32 operations per split-FP32 (hi + lo) multiply-add, roughly


def parse(argv=None):
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
    ap.add_argument("--narrow-factor", type=int, default=None, choices=[-1, 0, 1, 2, 3],
                    help="kernel for bands w <= 12: 0 G-lane, 1 earlier kernels, 2 band pass and chunked "
                         "border on a shadow of the arithmetic, 3 FP32 split CTAs, -1 per arithmetic (default: "
                         "the autotuner's choice)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-configs", action="store_true", help="skip the l_max 1500 and 32-operator sub-lines")
    ap.add_argument("--arms", default="fp64:fp64,fp32x2:fp32x2",
                    help="other contraction:factor arithmetics timed beside the headline")
    return ap.parse_args(argv)


def peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f)
    except OSError:
        return {}


def host_cores():
    """Cores this process may run on (affinity mask), and the CPU model."""
    try:
        cores = len(os.sched_getaffinity(0))
    except (AttributeError, OSError):
        cores = os.cpu_count() or 1
    model = platform.processor() or platform.machine()
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                k = line.split(":")[0].strip().lower()
                if k in ("model name", "cpu model", "hardware"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return cores, model


# -- oracle sample (CPU baseline and reference arm) ---------------------------------------

def oracle_ring(wl, og, ninv, j):
    """One ring of the whole path in the oracle: the block, then its Cholesky.
    Returns (stored elements, seconds)."""
    from oracle import oracle as O
    t0 = time.perf_counter()
    M, _ = O.block(og, wl.beams()[0], wl.priors()[0], wl.radii()[0], ninv, j)
    O.cholesky(M)
    dt = time.perf_counter() - t0
    n = M.shape[0]
    nz = np.nonzero(M)
    w = int(np.max(np.minimum((nz[0] - nz[1]) % n, (nz[1] - nz[0]) % n))) if len(nz[0]) else 0
    return (n * (w + 1) if 2 * w + 1 < n else n * (n + 1) // 2), dt


def stratified_rings(og, nmax, count, shift=0):
    """`count` rings whose sizes span the distinct ring sizes up to nmax
    (quantiles of the distinct sizes), both hemispheres alternately."""
    sizes = sorted({int(v) for v in og["nring"] if v <= nmax})
    picks = np.unique(np.linspace(0, len(sizes) - 1, count).round().astype(int))
    N = og["nrings"]
    rings = []
    for k, i in enumerate(picks):
        cand = [j for j in range(N) if og["nring"][j] == sizes[i]]
        rings.append(cand[(k + shift) % len(cand)])
    return rings


def oracle_extrapolate(wl, og, ninv, rings, threads):
    """Time the oracle on `rings` (one thread per ring, all at once), fit the
    per-ring cost t(n) = a n^2 + b n^3 + c n l_max (the pair sums, the dense
    Cholesky, the kernel evaluations) by non-negative least squares, and
    extrapolate to every ring of the workload on `threads` cores."""
    from scipy.optimize import nnls
    with ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(lambda j: oracle_ring(wl, og, ninv, j), rings))
    n = np.array([og["nring"][j] for j in rings], dtype=np.float64)
    t = np.array([r[1] for r in res])
    X = np.stack([n ** 2, n ** 3, n * og["lmax"]], axis=1)
    coef, _ = nnls(X / t[:, None], np.ones_like(t))  # relative residuals
    nall = og["nring"].astype(np.float64)
    t_all = float(np.sum(np.stack([nall ** 2, nall ** 3, nall * og["lmax"]], axis=1) @ coef))
    sample_el = int(sum(r[0] for r in res))
    return {"sample_elements": sample_el, "sample_cpu_s": float(t.sum()), "sample_wall_s": float(t.max()),
            "sample_max_n": int(n.max()), "predicted_cpu_s_all_rings": t_all, "fit": coef.tolist()}


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


# -- roofline model --------------------------------------------------------------------------

S_BLOCK_PBAND = 0  # the C header's SYMPIX_BLOCK_PBAND


def pipe_peaks(dev):
    """Measured FP64 and FP32 (non-tensor) rates: cuBLAS DGEMM and SGEMM with
    TF32 off, n = 4096, best of 5 (library GEMMs stand in for the pipes'
    peaks); the nominal figures where a GEMM measures implausibly high."""
    import torch
    out = {}
    tf32 = torch.backends.cuda.matmul.allow_tf32
    torch.backends.cuda.matmul.allow_tf32 = False
    try:
        for dt, nom, key in ((torch.float64, FP64_NOMINAL, "fp64"), (torch.float32, FP32_NOMINAL, "fp32")):
            n = 4096
            a = torch.randn(n, n, dtype=dt, device=dev)
            b = torch.randn(n, n, dtype=dt, device=dev)
            c = a @ b
            best = 1e30
            for _ in range(5):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                torch.matmul(a, b, out=c)
                e1.record()
                torch.cuda.synchronize()
                best = min(best, e0.elapsed_time(e1) * 1e-3)
            meas = 2.0 * n ** 3 / best
            if meas > 1.05 * nom:
                out[key] = (nom, f"nominal {nom / 1e12:.2f} TFLOP/s (the GEMM measured {meas / 1e12:.1f}, "
                                 f"not a plain-pipe rate)")
            else:
                out[key] = (meas, f"measured: cuBLAS {'DGEMM' if key == 'fp64' else 'SGEMM (TF32 off)'} "
                                  f"n=4096, {meas / 1e12:.3f} TFLOP/s")
            del a, b, c
    finally:
        torch.backends.cuda.matmul.allow_tf32 = tf32
    out["fp32x2"] = (out["fp32"][0] / SPLIT_COST,
                     f"FP32 rate / {SPLIT_COST:g} (a split-FP32 multiply-add costs about "
                     f"{SPLIT_COST:g} FP32 operations)")
    return out


def factor_work(n, w, pband):
    """(flops, bytes) of factoring one block: periodic band (L11 band, L21 =
    A21 L11^-T, corner) or dense n^3/3; bytes: 16 per stored element (the
    sampled FP64 element read and its factor written)."""
    if pband:
        m = n - w
        flops = 2.0 * (m * w * (w + 1) / 2 + w * m * w + n * w * (w + 1) / 2) + 2.0 * n
        byt = 16.0 * n * (w + 1)
    else:
        flops = n ** 3 / 3.0
        byt = 16.0 * n * (n + 1) / 2
    return flops, byt


def kernel_models(plan, grid, sprec, fprec):
    """Algorithmic work of every traced span of one step, as
    {name: (bytes, flops, arithmetic of the flops)}: bytes the algorithm
    itself must move to or from HBM, flops it must perform (sparse triples,
    band updates; no padding).  flops None = not modelled."""
    geo = [plan.block_layout("pband", o, j) for o in range(plan.nops) for j in range(plan.ring0, plan.ring1)]
    pb = [(n, w) for _, n, w, fmt in geo if fmt == S_BLOCK_PBAND]
    dn = [n for _, n, w, fmt in geo if fmt != S_BLOCK_PBAND]
    lmax = grid.lmax
    npix = grid.npix * plan.nops
    chunks = 0
    left = plan.nops
    while left > 0:
        left -= 8 if left >= 8 else 4 if left >= 4 else 2 if left >= 2 else 1
        chunks += 1

    def fsum(items, pband):
        f = b = 0.0
        for it in items:
            ff, bb = factor_work(it[0], it[1], True) if pband else factor_work(it, 0, False)
            f += ff
            b += bb
        return b, f

    narrow = [x for x in pb if x[1] <= 16]
    wide = [x for x in pb if 16 < x[1] <= 64]
    el_pb = sum(n * (w + 1) for n, w in pb)
    map_bytes = {"fp64": 8, "fp32": 4, "fp32x2": 8}[sprec]
    narrow_prec = fprec
    wide_prec = "fp64" if fprec == "fp32x2" else fprec
    m = {
        "k_table_coeffs": ((lmax + 1) * plan.nops * 32.0 + 16.0 * (lmax + 1), 0.0, "fp64"),
        # one product and three FMAs of the recurrence per chunk, an FMA per operator, per (slot, l)
        "k_table": (plan.nslots * (12.0 + 48.0 * plan.nops),
                    plan.nslots * lmax * (7.0 * chunks + 2.0 * plan.nops), "fp64"),
        "k_split_ninv": (npix * 16.0, 0.0, "fp32"),
        "k_sample_pband": (el_pb * 8.0 + npix * map_bytes, 2.0 * plan.ntriples + plan.nmults, sprec),
        "k_sample_dense": (sum(n * n for n in dn) * 8.0, None, sprec),
        "k_pband_chol": (*fsum(narrow, True), narrow_prec),
        "k_factor_band": (*fsum(narrow, True), narrow_prec),
        "k_factor_wide": (*fsum(wide, True), wide_prec),
        "k_factor_dense": (*fsum([n for n in dn if n <= 1024], False), "fp64"),
        "k_factor_dense_cta": (*fsum([n for n in dn if n > 1024], False), "fp64"),
    }
    # spans whose work depends on the data (blocks refactored in FP64 after an
    # FP32 pivot fell below the floor; none in a well-conditioned step)
    for name in ("k_pband_chol_rescue", "k_factor_rescue", "k_factor_wide_rescue"):
        m[name] = (0.0, None, "fp64")
    # the FP32 factor on a band copy: the transposes move the copy, the
    # factor kernels are charged the factorisation's own 16 B per element
    band = sum(n * (w + 1) for n, w in narrow)
    l21 = sum(w * (n - w) for n, w in narrow)
    fl = sum(factor_work(n, w, True)[0] for n, w in narrow)
    fl12 = sum(factor_work(n, w, True)[0] for n, w in narrow if w <= 12)
    b12 = 16.0 * sum(n * (w + 1) for n, w in narrow if w <= 12)
    fl8 = sum(factor_work(n, w, True)[0] for n, w in narrow if w <= 8)
    b8 = 16.0 * sum(n * (w + 1) for n, w in narrow if w <= 8)
    # the split launch (option 3) factors the w <= 8 blocks; its span ends on
    # the main stream, and the w 9..12 path beside it shows only as the
    # remainder after it ("k_f32_split"), which is not a kernel's own time
    m.update({"k_f32_split_w8": (b8, fl8, "fp32"), "k_f32_fused_w8": (b8, fl8, "fp32"),
              "k_f32_split": (0.0, None, "fp32", "the w 9..12 path's time beyond the w <= 8 launch, not a kernel")})
    # option 2 (band pass of every slice, border rows by column chunks): its
    # chunk kernels are not modelled separately
    for name in ("k_l21_transfer", "k_l21_carry", "k_l21_solve", "k_l21_cornerpart", "k_l21_corner"):
        m[name] = (0.0, None, "fp32", "a phase of the chunked border solve, not modelled alone")
    if fprec in ("fp64", "fp32x2"):
        # FP64 / split FP32 on a shadow of 8-byte elements (option 2, w <= 12):
        # the transposes move 16 B per element (FP64 read or written, the
        # shadow element written or read), the band pass reads and writes its
        # rows (16 B) and does the band third of the factor's flops
        band_lo = sum(n * (w + 1) for n, w in narrow if w <= 12)
        l21_lo = sum(w * (n - w) for n, w in narrow if w <= 12)
        fl_band = sum((n - w) * w * (w + 1) + 2.0 * n for n, w in narrow if w <= 12)
        m.update({"k_f32_shadow_in": (band_lo * 16.0, 0.0, fprec), "k_f32_out": ((band_lo + l21_lo) * 16.0, 0.0, fprec),
                  "k_f64_band_pass": (band_lo * 16.0, fl_band, "fp64"),
                  "k_df_band_pass": (band_lo * 16.0, fl_band, "fp32x2")})
        for name in ("k_l21_transfer", "k_l21_carry", "k_l21_solve", "k_l21_cornerpart", "k_l21_corner"):
            m[name] = (0.0, None, fprec, "a phase of the chunked border solve, not modelled alone")
        return m
    m.update({"k_f32_shadow_in": (band * 12.0, 0.0, "fp32"), "k_f32_out": (band * 4.0 + l21 * 12.0, 0.0, "fp32"),
              "k_f32_fused": (b12, fl12, "fp32"), "k_f32_band_pass": (16.0 * band - b12, (fl - fl12) / 3, "fp32"),
              "k_f32_border_pass": (0.0, 2 * (fl - fl12) / 3, "fp32"),
              "k_chol_commit": (12.0 * sum((n - w) * (w + 1) for n, w in narrow if w <= 12), 0.0, "fp32")})
    return m


def roofline(name, ms, model, hbm, pk):
    """The kernel against whichever bound is larger: bytes / HBM bandwidth,
    or flops / the peak of their arithmetic."""
    if name not in model:
        return {"kernel": name, "ms": ms, "bound": "unmodelled", "frac": None}
    byt, fl, typ = model[name][:3]
    note = model[name][3] if len(model[name]) > 3 else "work depends on the data"
    t_hbm = byt / hbm
    t_alu = (fl / pk[typ][0]) if fl else 0.0
    r = {"kernel": name, "ms": ms, "bytes": byt, "flops": fl, "flop_type": typ,
         "t_hbm_ms": t_hbm * 1e3, "t_alu_ms": t_alu * 1e3}
    if fl is None and byt == 0.0:
        r.update({"bound": "unmodelled", "frac": None, "note": note})
    elif t_hbm >= t_alu:
        r.update({"bound": "hbm", "achieved": byt / (ms * 1e-3) / 1e9, "peak": hbm / 1e9, "unit": "GB/s",
                  "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)"})
    else:
        r.update({"bound": "alu", "achieved": fl / (ms * 1e-3) / 1e12, "peak": pk[typ][0] / 1e12,
                  "unit": "TFLOP/s", "peak_source": pk[typ][1]})
    if "achieved" in r:
        r["frac"] = r["achieved"] / r["peak"]
    if fl is None and byt > 0:
        r["note"] = "flops not modelled; bytes bound only"
    return r


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) of a
# kernel from one ncu capture of (workload, precision), valid only while the
# kernel's sources hash to the digest recorded with the capture.
KERNEL_SOURCES = {
    "k_table": ["sympix_table.cu"],
    "k_f32_fused": ["sympix_factor_fused.cu", "sympix_factor_kernels.cuh", "sympix_arith.cuh"],
    "k_f32_split_w8": ["sympix_factor_split.cu", "sympix_factor_kernels.cuh", "sympix_arith.cuh"],
    "k_pband_chol": ["sympix_chol.cuh", "sympix_chol_f32.cu", "sympix_chol_f64.cu", "sympix_chol_f2.cu",
                     "sympix_arith.cuh"],
    "k_sample_pband": ["sympix_sample_kernels.cuh", "sympix_sample_f32.cu", "sympix_sample.cu"],
}
TRAFFIC = {
    # (workload, precision, kernel): (bytes per launch, source digest, capture)
    ("lmax3000_fwhm5", "fp32:fp32", "k_table"): (
        799488, "e053756e1e7a",
        "ncu dram__bytes_read.sum + dram__bytes_write.sum, one pass over the bench's own mixed step"),
    ("lmax3000_fwhm5", "fp32:fp32", "k_f32_split_w8"): (
        1555681024, "ecc07086edd3",
        "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_f32_split<8,256,2> (759.2 + 796.5 MB), one pass "
        "over the bench's own mixed step (--steps 1 --warmup 1 --no-autotune), the timed step's launch"),
}


def source_digest(kernel):
    h = hashlib.sha256()
    for f in KERNEL_SOURCES.get(kernel, []):
        p = os.path.join(CSRC, f)
        if os.path.exists(p):
            with open(p, "rb") as fh:
                h.update(fh.read())
    return h.hexdigest()[:12]


def traffic_of(workload, precision, kernel, per_step_launches=1):
    ent = TRAFFIC.get((workload, precision, kernel))
    if ent is None:
        return None, "no ncu capture of this kernel's current source"
    byt, digest, how = ent
    if digest != source_digest(kernel):
        return None, "the kernel changed since its ncu capture"
    return byt, how


# -- helpers used by the rank tests ----------------------------------------------------------

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


# -- the GPU arm ---------------------------------------------------------------------------

class Problem:
    """One workload on the device: grid, plan, inputs and buffers, and the
    timed step in any contraction:factor arithmetic."""

    def __init__(self, S, W, wl, dev, stream, flush, launch="graph"):
        import torch
        self.S, self.wl, self.dev, self.stream, self.flush, self.launch = S, wl, dev, stream, flush, launch
        self.grid = S.Grid(wl.lmax)
        self.plan = S.Plan(self.grid, wl.radii())
        self.nbytes, self.elements = self.plan.blocks_size("pband")
        g = self.grid
        colat = W.pixel_colatitude(g.theta, g.nring, g.ring_offset, g.ring_stride, g.npix)
        self.ninv_h = wl.ninv(colat)
        self.bl_h, self.dl_h = wl.beams(), wl.priors()
        self.bl = torch.tensor(self.bl_h, dtype=torch.float64, device=dev)
        self.dl = torch.tensor(self.dl_h, dtype=torch.float64, device=dev)
        self.ninv = torch.tensor(self.ninv_h, dtype=torch.float64, device=dev)
        self.blocks = torch.empty(self.nbytes // 8, dtype=torch.float64, device=dev)
        self.info = torch.empty(self.plan.nblocks, dtype=torch.int32, device=dev)
        self.graphs = {}
        self.tune = None

    def autotune(self, prec):
        sp, fp = prec.split(":")
        self.tune = self.plan.autotune(self.bl, self.dl, self.ninv, self.blocks, self.info, "pband", sp, fp,
                                       stream=self.stream)

    def graph(self, prec):
        if prec not in self.graphs:
            sp, fp = prec.split(":")
            self.graphs[prec] = self.S.Step(self.plan, self.bl, self.dl, self.ninv, self.blocks, self.info,
                                            "pband", sp, fp)
        return self.graphs[prec]

    def step(self, prec, ev=None):
        S, st = self.S, self.stream
        if self.launch == "graph":
            g = self.graph(prec)
            for i, bit in enumerate((S.STAGE_TABLE, S.STAGE_SAMPLE, S.STAGE_FACTOR)):
                if ev:
                    ev[i].record(st)
                g.launch(bit, stream=st)
            if ev:
                ev[3].record(st)
            return
        sp, fp = prec.split(":")
        if ev:
            ev[0].record(st)
        S.sympix_kernel_table(self.plan, self.bl, self.dl, stream=st)
        if ev:
            ev[1].record(st)
        S.sympix_sample_blocks(self.plan, self.ninv, precision=sp, storage="pband", out=self.blocks, stream=st)
        if ev:
            ev[2].record(st)
        S.sympix_factor_blocks(self.plan, self.blocks, storage="pband", precision=fp, info=self.info, stream=st)
        if ev:
            ev[3].record(st)

    def timed(self, prec, K, W_, world=1):
        """Stage times [K, 3] (ms) of K steps after W_ warm-up steps, L2
        flushed between steps outside the events."""
        import torch
        with torch.cuda.stream(self.stream):
            for _ in range(W_):
                self.step(prec)
        torch.cuda.synchronize()
        evs = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(K)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        for k in range(K):
            with torch.cuda.stream(self.stream):
                self.flush.fill_(float(k))
                self.step(prec, evs[k])
        torch.cuda.synchronize()
        if world > 1:
            torch.distributed.barrier()
        return np.array([[evs[k][i].elapsed_time(evs[k][i + 1]) for i in range(3)] for k in range(K)])

    def traced(self, prec, K):
        """Per-kernel device times (ms per step, spans of one name summed within
        a step) from K direct-call steps with an event after every launch."""
        import torch
        S, st = self.S, self.stream
        sp, fp = prec.split(":")
        per = {}
        self.plan.set_trace(True)
        for k in range(K):
            with torch.cuda.stream(st):
                self.flush.fill_(float(k))
                self.plan.trace_read()
                S.sympix_kernel_table(self.plan, self.bl, self.dl, stream=st)
                S.sympix_sample_blocks(self.plan, self.ninv, precision=sp, storage="pband", out=self.blocks,
                                       stream=st)
                S.sympix_factor_blocks(self.plan, self.blocks, storage="pband", precision=fp, info=self.info,
                                       stream=st)
            step = {}
            for name, ms in self.plan.trace_read():
                step[name] = step.get(name, 0.0) + ms
            for name, ms in step.items():
                per.setdefault(name, []).append(ms)
        self.plan.set_trace(False)
        return {k: float(np.mean(v)) for k, v in per.items()}

    def rooflines(self, prec, K, hbm, pk):
        sp, fp = prec.split(":")
        kern = self.traced(prec, K)
        model = kernel_models(self.plan, self.grid, sp, fp)
        rows = {name: roofline(name, ms, model, hbm, pk) for name, ms in kern.items()}
        dom = max(kern, key=kern.get)
        return rows, dict(rows[dom])


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

    wl = rank_workload(W.WORKLOADS[args.workload], rank)
    stream = torch.cuda.Stream(device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    P = Problem(S, W, wl, dev, stream, flush, args.launch)
    plan, grid, elements = P.plan, P.grid, P.elements
    if not args.no_autotune and args.narrow_factor is None:
        P.autotune(args.precision)
        torch.cuda.synchronize()
    if args.narrow_factor is not None:
        plan.set_narrow_factor(args.narrow_factor)

    clocks = Clocks(local)
    main_st = P.timed(args.precision, args.steps, args.warmup, world)
    clk = clocks.stop()
    info_h = P.info.cpu().numpy()
    ms_step = float(main_st.sum(axis=1).mean())
    ms_max = max_over_ranks(ms_step, world, dev)
    value = job_value(elements, ms_max, world)

    pk = pipe_peaks(dev)
    hbm = peaks().get("hbm_gbs", 6800.0) * 1e9

    # other arithmetic arms (same steps), each with its dominant kernel's roofline
    arms = {}
    for prec in [a for a in args.arms.split(",") if a and a != args.precision]:
        st = P.timed(prec, args.steps, 1)
        _, roof = P.rooflines(prec, max(2, args.steps // 2), hbm, pk)
        arms[prec] = {"value": elements / (float(st.sum(axis=1).mean()) * 1e-3),
                      "ms_per_step": float(st.sum(axis=1).mean()),
                      "stages_ms": dict(zip(["table", "sample", "factor"], st.mean(axis=0).round(4).tolist())),
                      "roofline": roof}

    # accuracy against the FP64 GPU path, normwise per block over every
    # (operator, ring) block: sampled blocks of each contraction, and the
    # factors of each full arm on the blocks both arms factored
    acc, not_pd = {}, {}
    if rank == 0:
        acc, not_pd = accuracy(P, args)

    e2e = None if args.no_e2e else end_to_end(P, args, world)

    # per-kernel device times of the headline arithmetic and the roofline of
    # the dominant kernel against whichever bound is larger
    kernels, roof = P.rooflines(args.precision, args.steps, hbm, pk)
    tr, tsrc = traffic_of(wl.name, args.precision, roof["kernel"])
    roof["traffic"] = tr
    roof["traffic_source"] = tsrc
    roof["timing"] = "CUDA events around each launch on the launching stream, traced pass of the same steps"

    conv = convolution(P, args, hbm, pk)
    apply_ = apply_timing(P, args, hbm, pk)

    launches = P.graph(args.precision).kernels(S.STAGE_ALL) if args.launch == "graph" else \
        sum(plan.launches("pband", *args.precision.split(":")))
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
                   "launch_shapes": {**dict(zip(("table_cta", "border_threads"), plan.tuning())),
                                     "narrow_factor_kernel": plan.narrow_kernels()},
                   "autotuned": P.tune is not None,
                   "parallelism": f"independent problem per GPU x{world}"},
        "stages_ms": dict(zip(["table", "sample", "factor"], main_st.mean(axis=0).round(4).tolist())),
        "kernel_rooflines": kernels, "pipe_peaks": {k: {"tflops": v[0] / 1e12, "source": v[1]} for k, v in pk.items()},
        "arms": arms, "accuracy": acc, "roofline": roof, "e2e": e2e,
        "convolution": {"op": "g = B^ f, pixel domain (Eq. convolution-pixel); 16 B algorithmic per pixel", **conv},
        "apply": apply_,
        "gpu_launches": launches * args.steps, "clocks": clk,
        "blocks": int(plan.nblocks),
        "blocks_not_positive_definite": not_pd or int((info_h != 0).sum()),
    }
    del P
    torch.cuda.empty_cache()

    if rank == 0 and world == 1 and not args.no_configs:
        line["configs"] = sub_configs(S, W, args, dev, stream, flush, hbm, pk)

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        from oracle import oracle as O
        line["cpu_baseline"] = cpu_baseline(wl, O.grid(grid.lmax), P_ninv0(wl, grid), elements)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def P_ninv0(wl, grid):
    from paper_1504_04653_gb300 import workloads as W
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    return wl.ninv(colat)[0]


def accuracy(P, args):
    import torch
    S, plan, dev, stream = P.S, P.plan, P.dev, P.stream
    lay = [plan.block_layout("pband", op, j) for op in range(plan.nops) for j in range(plan.ring0, plan.ring1)]
    nb = len(lay)
    starts = torch.tensor([o for o, _, _, _ in lay], dtype=torch.int64, device=dev)
    lens = torch.tensor([n * (2 * w + 1) if fmt == S.BLOCK_PBAND else n * n for _, n, w, fmt in lay],
                        dtype=torch.int64, device=dev)
    bid = torch.repeat_interleave(torch.arange(nb, device=dev), lens)
    first = torch.cumsum(lens, 0) - lens
    pos = starts[bid] + torch.arange(bid.numel(), device=dev) - first[bid]

    def run_once(prec, factored):
        sp, fp = prec.split(":")
        with torch.cuda.stream(stream):
            S.sympix_kernel_table(plan, P.bl, P.dl, stream=stream)
            S.sympix_sample_blocks(plan, P.ninv, precision=sp, storage="pband", out=P.blocks, stream=stream)
            if factored:
                S.sympix_factor_blocks(plan, P.blocks, storage="pband", precision=fp, info=P.info, stream=stream)
        torch.cuda.synchronize()
        return P.blocks[pos], P.info.clone()

    def blockwise(a, b):
        num = torch.zeros(nb, dtype=torch.float64, device=dev).scatter_reduce_(0, bid, (a - b).abs(), "amax")
        den = torch.zeros(nb, dtype=torch.float64, device=dev).scatter_reduce_(0, bid, b.abs(), "amax")
        return num / den.clamp_min(1e-300)

    acc, not_pd = {}, {}
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
    return acc, not_pd


def end_to_end(P, args, world):
    """The same step through the public API with pinned host buffers: inputs
    copied in and the factored blocks and info copied out every step."""
    import torch
    bl_p = torch.tensor(P.bl_h, dtype=torch.float64).pin_memory()
    dl_p = torch.tensor(P.dl_h, dtype=torch.float64).pin_memory()
    ninv_p = torch.tensor(P.ninv_h, dtype=torch.float64).pin_memory()
    out_p = torch.empty(P.nbytes // 8, dtype=torch.float64).pin_memory()
    info_p = torch.empty(P.plan.nblocks, dtype=torch.int32).pin_memory()

    def e2e_step():
        P.bl.copy_(bl_p, non_blocking=True)
        P.dl.copy_(dl_p, non_blocking=True)
        P.ninv.copy_(ninv_p, non_blocking=True)
        P.step(args.precision)
        out_p.copy_(P.blocks, non_blocking=True)
        info_p.copy_(P.info, non_blocking=True)

    with torch.cuda.stream(P.stream):
        for _ in range(max(1, args.warmup)):
            e2e_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(P.stream):
        e0.record(P.stream)
        for _ in range(args.steps):
            e2e_step()
        e1.record(P.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    h2d = (bl_p.numel() + dl_p.numel() + ninv_p.numel()) * 8
    d2h = out_p.numel() * 8 + info_p.numel() * 4
    return {"value": world * P.elements / (ms * 1e-3), "unit": "elements/s", "ms_per_step": ms,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h)}


def convolution(P, args, hbm, pk):
    """g = B^ f on the same plan and table (the N^-1 map stands in for f):
    FP32 against HBM, FP64 against the FP64 rate."""
    import torch
    S, plan, stream = P.S, P.plan, P.stream
    out = {}
    gbuf = torch.empty_like(P.ninv)
    S.sympix_kernel_table(plan, P.bl, P.dl, stream=stream)
    for cp in ("fp32", "fp64"):
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        with torch.cuda.stream(stream):
            for _ in range(max(1, args.warmup)):
                S.sympix_convolve(plan, P.ninv, precision=cp, out=gbuf, stream=stream)
            for k in range(args.steps):
                P.flush.fill_(float(k))
                evs[k][0].record(stream)
                S.sympix_convolve(plan, P.ninv, precision=cp, out=gbuf, stream=stream)
                evs[k][1].record(stream)
        torch.cuda.synchronize()
        ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
        px = P.grid.npix * plan.nops
        model = {"k_convolve": (px * 16.0, 2.0 * plan.nmults, cp)}
        ent = roofline("k_convolve", ms, model, hbm, pk)
        ent["pixels_per_s"] = px / (ms * 1e-3)
        out[cp] = ent
    return out


def apply_timing(P, args, hbm, pk):
    """y = M^-1 x with the factored diagonal ring blocks (block Jacobi,
    sympix_apply, FP64) on the factors of the headline step: algorithmic
    bytes = the stored factor elements read (band and border rows) plus x
    read and y written, 8 B each; flops 4 per stored factor element."""
    import torch
    S, plan, stream = P.S, P.plan, P.stream
    P.step(args.precision)
    torch.cuda.synchronize()
    x = torch.randn_like(P.ninv)
    y = torch.empty_like(x)
    geo = [plan.block_layout("pband", o, j) for o in range(plan.nops) for j in range(plan.ring0, plan.ring1)]
    fel = sum(n * (2 * w + 1) if fmt == 0 else n * (n + 1) // 2 for _, n, w, fmt in geo)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with torch.cuda.stream(stream):
        for _ in range(max(1, args.warmup)):
            S.sympix_apply(plan, P.blocks, P.info, x, out=y, stream=stream)
        for k in range(args.steps):
            P.flush.fill_(float(k))
            evs[k][0].record(stream)
            S.sympix_apply(plan, P.blocks, P.info, x, out=y, stream=stream)
            evs[k][1].record(stream)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    px = P.grid.npix * plan.nops
    ent = roofline("k_apply", ms, {"k_apply": (8.0 * fel + 16.0 * px, 4.0 * fel, "fp64")}, hbm, pk)
    ent.update({"op": "y = M^-1 x, block Jacobi with the factored ring blocks (forward and back substitution)",
                "pixels_per_s": px / (ms * 1e-3)})
    return ent


def coupling_timing(S, P, args, hbm, pk):
    """The blocks between neighbouring rings (ring offset 1, FP64) of a
    workload: planned, the table re-evaluated with d at every class, then
    timed; algorithmic bytes = the stored entries written, 8 B each."""
    import torch
    nbytes, el = P.plan.coupling_size(1)
    S.sympix_kernel_table(P.plan, P.bl, P.dl, stream=P.stream)
    out = torch.empty(max(1, nbytes // 8), dtype=torch.float64, device=P.dev)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(3)]
    with torch.cuda.stream(P.stream):
        S.sympix_sample_coupling(P.plan, P.ninv, 1, out=out, stream=P.stream)
        for k in range(3):
            P.flush.fill_(float(k))
            evs[k][0].record(P.stream)
            S.sympix_sample_coupling(P.plan, P.ninv, 1, out=out, stream=P.stream)
            evs[k][1].record(P.stream)
    torch.cuda.synchronize()
    ms = float(np.mean([a.elapsed_time(b) for a, b in evs]))
    ent = roofline("k_sample_coupling", ms, {"k_sample_coupling": (8.0 * el, None, "fp64")}, hbm, pk)
    ent.update({"op": "blocks between rings j and j+1 (FP64)", "elements": int(el),
                "elements_per_s": el / (ms * 1e-3)})
    del out
    return ent


def dp_timing(S, W, args, hbm, pk, lmax=500, k=8):
    """The paper's DP grid with k x k tiles (f2): one block per band of k rings
    under tile adjacency, l_max = 500, k = 8 (64 bands of up to 8640
    pixels), one operator with a beam narrower than a tile.  Times the kernel
    table and the band-block sampling (FP64 and FP32) with CUDA events on
    the stream, L2 flushed before each; the dense factor of these bands (one
    CTA per band) is not timed."""
    import torch
    grid = S.Grid(lmax, k=k, layout="dp", polar_thr=0.0)
    fwhm = 60.0 * 180.0 / lmax * k / 4.0
    wl = W.Workload(f"dp_lmax{lmax}_k{k}", lmax, [fwhm], [20.0], [41])
    plan = S.Plan(grid, wl.radii())
    colat = W.pixel_colatitude(grid.theta, grid.nring, grid.ring_offset, grid.ring_stride, grid.npix)
    bl = torch.tensor(wl.beams(), device="cuda")
    dl = torch.tensor(wl.priors(), device="cuda")
    ninv = torch.tensor(wl.ninv(colat), device="cuda")
    nb = plan.nblocks
    stored = sum(plan.block_layout("pband", 0, g)[1] ** 2 for g in range(nb))
    nbytes, _ = plan.blocks_size("pband")
    out = torch.empty(nbytes // 8, dtype=torch.float64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    st = torch.cuda.current_stream()
    reps = max(2, min(args.steps, 5))

    def timed(fn):
        fn()
        ts = []
        for _ in range(reps):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(st)
            fn()
            b.record(st)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.mean(ts))

    ent = {"workload": wl.name, "lmax": lmax, "k": k, "npix": int(grid.npix), "bands": nb,
           "largest_band": int(max(plan.block_layout("pband", 0, g)[1] for g in range(nb))),
           "stored_elements": int(stored), "table_slots": int(plan.nslots),
           "multiply_adds": int(plan.ntriples)}
    ent["table_ms"] = timed(lambda: S.sympix_kernel_table(plan, bl, dl))
    for prec in ("fp64", "fp32"):
        ms = timed(lambda: S.sympix_sample_blocks(plan, ninv, precision=prec, out=out))
        model = {"k_sample_tiles": (8.0 * stored, 2.0 * plan.ntriples, prec)}
        r = roofline("k_sample_tiles", ms, model, hbm, pk)
        r.update({"elements_per_s": stored / (ms * 1e-3), "note": "includes zeroing the blocks buffer"})
        ent[prec] = r
    del out, flush
    torch.cuda.empty_cache()
    return ent


def sub_configs(S, W, args, dev, stream, flush, hbm, pk):
    """Two more workloads, each timed the same way (graph replay, L2 flushed,
    CUDA events): l_max = 1500 with an FP64 factor after the mixed and the
    FP64 contraction, and 32 operators at l_max = 1000 (FWHM 10'-60', mask
    bands 0-30 deg) mixed and FP64."""
    import torch
    out = {}
    for key, precs in (("lmax1500", ("fp32:fp64", "fp64:fp64")), ("batched32", ("fp32:fp32", "fp64:fp64"))):
        wl = W.WORKLOADS[key]
        P = Problem(S, W, wl, dev, stream, flush, "graph")
        P.autotune(precs[0])
        ent = {"workload": wl.name, "lmax": wl.lmax, "nops": P.plan.nops, "elements": int(P.elements),
               "blocks": int(P.plan.nblocks), "storage": "pband"}
        for prec in precs:
            st = P.timed(prec, max(3, args.steps // 2), args.warmup)
            ms = float(st.sum(axis=1).mean())
            _, roof = P.rooflines(prec, 2, hbm, pk)
            ent[prec] = {"value": P.elements / (ms * 1e-3), "unit": "elements/s", "ms_per_step": ms,
                         "stages_ms": dict(zip(["table", "sample", "factor"], st.mean(axis=0).round(4).tolist())),
                         "roofline": roof, "blocks_not_positive_definite": int((P.info != 0).sum()),
                         "gpu_launches_per_step": P.graph(prec).kernels(S.STAGE_ALL)}
        if key == "lmax1500":
            ent["coupling"] = coupling_timing(S, P, args, hbm, pk)
        out[key] = ent
        del P
        torch.cuda.empty_cache()
    out["dp_lmax500_k8"] = dp_timing(S, W, args, hbm, pk)
    return out


def cpu_baseline(wl, og, ninv0, elements):
    """The oracle as it stands on this host's cores: a stratified sample of
    ring sizes (up to n = 3000, all timed at once, one thread per ring),
    extrapolated to every ring of the workload by the fitted per-ring cost."""
    cores, model = host_cores()
    rings = stratified_rings(og, 3000, min(cores, 16))
    ex = oracle_extrapolate(wl, og, ninv0, rings, min(cores, len(rings)))
    wall_all = ex["predicted_cpu_s_all_rings"] / cores
    return {"value": elements / wall_all, "unit": "elements/s", "cores": cores, "kind": "oracle",
            "cpu_model": model, "extrapolated": True,
            "sample": (f"{len(rings)} rings of distinct sizes n <= {ex['sample_max_n']} timed at once "
                       f"({ex['sample_elements']} elements, {ex['sample_cpu_s']:.1f} CPU s, "
                       f"{ex['sample_wall_s']:.1f} s wall); per-ring cost t(n) = a n^2 + b n^3 + c n l_max "
                       f"fitted and summed over all {og['nrings']} rings ({ex['predicted_cpu_s_all_rings']:.0f} "
                       f"CPU s), spread over {cores} cores"),
            "fit_a_b_c": ex["fit"]}


def reference_arm(args, rank, world):
    """The oracle timed as it stands, on the host cores (rank 0 only): each
    step a stratified sample of ring sizes up to n = 1500, extrapolated to
    the whole workload by the fitted per-ring cost."""
    if rank != 0:
        return
    from oracle import oracle as O
    from paper_1504_04653_gb300 import workloads as W
    O.build()
    wl = W.WORKLOADS[args.workload]
    og = O.grid(wl.lmax)
    colat = W.pixel_colatitude(og["theta"], og["nring"], og["ring_offset"], og["ring_stride"], og["npix"])
    ninv = wl.ninv(colat)[0]
    cores, model = host_cores()
    count = min(cores, 12)
    for s in range(args.warmup):
        oracle_extrapolate(wl, og, ninv, stratified_rings(og, 1500, count, shift=s), count)
    preds, wall = [], 0.0
    for s in range(args.steps):
        t0 = time.perf_counter()
        ex = oracle_extrapolate(wl, og, ninv, stratified_rings(og, 1500, count, shift=1000 + s), count)
        wall += time.perf_counter() - t0
        preds.append(ex["predicted_cpu_s_all_rings"])
    elements = workload_elements(og, wl)
    v = elements / (float(np.mean(preds)) / cores)
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "elements/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / max(1, args.steps),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": wl.name, "lmax": wl.lmax, "fwhm_arcmin": wl.fwhm_arcmin[0]},
        "cpu_baseline": {"value": v, "unit": "elements/s", "cores": cores, "kind": "oracle", "cpu_model": model,
                         "extrapolated": True,
                         "sample": (f"per step {count} rings of distinct sizes n <= 1500 timed at once, the "
                                    f"per-ring cost a n^2 + b n^3 + c n l_max fitted and summed over all "
                                    f"{og['nrings']} rings, spread over {cores} cores")},
        "e2e": {"value": v, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def workload_elements(og, wl):
    """Stored elements of every block of the workload, from the oracle's
    support: n (w+1) for a periodic band, n (n+1)/2 for a ring whose coupling
    wraps, with w the largest ring offset of any pixel pair within 2 r_s."""
    r_s = float(wl.radii()[0])
    total = 0
    th, nr = og["theta"], og["nring"]
    for j in range(og["nrings"]):
        n = int(nr[j])
        # offsets d with some pair of ring-j pixels q, q-d at angle <= 2 r_s
        # (the same-ring separation grows with d, so count until it exceeds)
        w = 0
        while w + 1 < n:
            d = w + 1
            dphi = 2 * math.pi * min(d, n - d) / n
            cosg = math.cos(th[j]) ** 2 + math.sin(th[j]) ** 2 * math.cos(dphi)
            if math.acos(max(-1.0, min(1.0, cosg))) > 2 * r_s:
                break
            w = d
        total += n * (w + 1) if 2 * w + 1 < n else n * (n + 1) // 2
    return total


if __name__ == "__main__":
    main()
