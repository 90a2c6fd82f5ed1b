#!/usr/bin/env python
"""Benchmark of the simplex-domain hot path on GB300.

Headline workload (one "step"): the Axilrod-Teller-Muto triple-dipole energy
and its adjoint forces F = -dE/dx over all i < j < k of n = 16384 points
uniform in a cube of side 20 (seed 6), nu = 1, eps = 1e-4: 732,873,539,584
triples on the lambda-mapped 3-simplex grid (two-branch recursive map plus
the J = K plane), one call of simplex_atm_forces (force tables over the
2-simplex of blocks, the forces kernel, the FP64 reduction of the energy),
FP32 per triple, FP64 force and energy sums.  Metric: triples per second
(whole job), with the same step timed for the bounding-box and linear
(cube-root) maps, the forces kernel timed live against the FP32 ALU
roofline, an end-to-end number through the C ABI with host buffers, and the
FP64 CPU oracle timed on all host cores (a bounded sample, extrapolated).

``--rows`` (default on at one GPU) also times every other kernel on the path
at its own configuration (coverage m = 2, 3, 4; EDM n = 1024 d = 3,
n = 32768 d = 256, n = 65536 d = 64 in both layouts; ATM energy n = 1024,
energy and forces n = 4096; stress loss forward/backward n = 65536 d = 64;
and non-powers of two: EDM n = 49152, ATM n = 3000 and n = 12000, coverage
n = 12000), each row with its own CPU oracle baseline.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs one replica per GPU under torchrun (the workload is independent
per rank, no data collective; "scaling": "weak").
"""
from __future__ import annotations

import argparse
import concurrent.futures as cf
import hashlib
import json
import math
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

METRIC = "pairs/s and triplets/s, λ-map vs bounding-box on 1 GB300; % of HBM/FP32 roofline"
WORKLOAD = "atm_n16384"
NU, EPS = 1.0, 1e-4
# Algorithmic FP32 flops per triple of the energy kernel with the pair terms
# hoisted into tables (edge vectors scaled by r^(3/2), and r^3): three
# 3-vector dot products (3 x 5), the product of the three (2, the second as
# an FMA into one accumulator) and r_ik^3 r_jk^3 into the other (1 FMA, 2):
# 20 flops (r_ij^3 and the combination r_ij^3 s0 - 3 s1 once per pair).
FLOPS_PER_TRIPLE = 20
# The same count (an FMA is 2 flops) for a triple of the forces kernel, which
# forms e and its three derivatives by the squared sides: the three unit-vector
# dot products (15), the cosine products p1, p2, c_ik, C_p (4), X, Y, Z with
# their r products (6), R^3 (2), e accumulated (4), H = 1 + 5 C_p (2), 1.5 R^3
# (1), S = Y - X - Z (2), the three derivatives (15) and their sums into the
# (i,j), (i,k) and (j,k) accumulators (2.5): 53.5.
FORCE_FLOPS_PER_TRIPLE = 53.5
FP32_LANES_PER_SM = 128
L2_FLUSH_BYTES = 512 << 20
PROFILES = os.path.join(ROOT, "profiles")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--rows", choices=["auto", "on", "off"], default="auto")
    ap.add_argument("--row", default=None, help="time only this row (no headline line)")
    return ap.parse_args()


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
            "sm_max_mhz": 2070.0}, "fallback"


def stated_traffic(summary: str):
    """DRAM bytes (read + write) per launch of a kernel from an ncu summary
    under profiles/: its line
      <!-- bench: source=<file> sha256=<hash> traffic_bytes_per_launch=<B> -->
    names the kernel's source file as captured; the figure is used only while
    that file is unchanged (else None: the counters predate the kernel)."""
    path = os.path.join(PROFILES, summary)
    if not os.path.exists(path):
        return None, f"{summary}: missing"
    m = re.search(r"<!-- bench: source=(\S+) sha256=([0-9a-f]+) traffic_bytes_per_launch=([0-9.e+]+)"
                  r"(?: scale=(\S+))? -->", open(path).read())
    if not m:
        return None, f"{summary}: no bench line"
    src = os.path.join(ROOT, m.group(1))
    cur = hashlib.sha256(open(src, "rb").read()).hexdigest() if os.path.exists(src) else ""
    if cur != m.group(2):
        return None, f"{summary}: {m.group(1)} changed since the capture"
    note = f"ncu capture summarised in profiles/{summary}"
    if m.group(4):
        note += f" ({m.group(4).replace('_', ' ')})"
    return float(m.group(3)), note


class Clocks:
    """nvidia-smi sampling of SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(prefix="clocks_", suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.1)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def time_steps(torch, fn, steps, warmup, flush=None, label="step"):
    """CUDA-event time of each step (ms) on the current stream, L2 flushed
    (untimed) before every step when `flush` is given.  Each timed step is an
    NVTX range named `label`, the warm-up one range, for profiler filters."""
    torch.cuda.nvtx.range_push(f"{label}:warmup")
    for _ in range(warmup):
        fn()
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for a, b in ev:
        if flush is not None:
            flush()
        torch.cuda.nvtx.range_push(label)
        a.record()
        fn()
        b.record()
        torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def triples(n):
    return n * (n - 1) * (n - 2) // 6


def row_triples(n, i):
    """Triples i < j < k < n with the given i."""
    return (n - 1 - i) * (n - 2 - i) // 2


def job_rate(ms_local: float, units_per_rank: int, world: int, dist=None, device=None):
    """Whole-job throughput of independent replicas: every rank processes
    `units_per_rank`; the job's step time is the slowest rank's (MAX
    all-reduce, the only collective; it carries a timing, not data).
    Returns (units per second for the job, job step ms)."""
    ms = ms_local
    if world > 1:
        import torch
        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return world * units_per_rank / (ms / 1e3), ms


# ------------------------------------------------------------------ oracle on the host

def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def host_parallel(fn, tasks, workers):
    """Runs fn over tasks on `workers` host threads (the oracle's ctypes calls
    release the GIL); returns (results, wall seconds)."""
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        res = list(ex.map(fn, tasks))
    return res, time.perf_counter() - t0


def oracle_rate(work, tasks, units, workers, kind="oracle"):
    """Units per second of the FP64 oracle over `tasks` on `workers` threads
    (one task per thread at a time), and on one thread for the first task."""
    _, wall = host_parallel(work, tasks, workers)
    _, one = host_parallel(work, tasks[:1], 1)
    return {"value": sum(units) / wall, "cores": workers, "kind": kind,
            "single_core": units[0] / one, "seconds": wall + one}


def cpu_atm(x, rows, forces: bool, workers):
    """The oracle's energy (or energy and gradient) over whole i-rows of the
    3-simplex: one row per task.  Extrapolates to the full sum by triples."""
    import oracle
    oracle.build()
    n = len(x)
    xd = x.astype(np.float64)

    def work(i):
        if forces:
            oracle.atm_energy_grad_slice(xd, i, i + 1, NU, EPS)
        else:
            oracle.atm_energy_slice(xd, i, i + 1, NU, EPS)

    units = [row_triples(n, i) for i in rows]
    r = oracle_rate(work, list(rows), units, workers)
    what = "energy and gradient" if forces else "energy"
    r.update({"unit": "triplets/s", "extrapolated": True,
              "sample": f"FP64 C oracle, {what} of the triples with i in {len(rows)} rows "
                        f"{rows[0]}..{rows[-1]} ({sum(units)} of {triples(n)} triples), one row per "
                        f"host thread; rate extrapolated to the whole sum by triple count"})
    return r


def rows_with(n, target, count):
    """`count` consecutive i-rows whose triple counts are near `target` each."""
    i = max(0, min(n - 3, n - 1 - int(math.isqrt(2 * target))))
    i = min(i, max(0, n - 3 - count))
    return list(range(i, i + count))


def cpu_edm(x, count, workers, seed=90):
    """The oracle's squared distances of `count` seeded pairs, split over the
    host threads; extrapolated to the whole triangle by pair count."""
    import oracle
    oracle.build()
    n = len(x)
    pr = synth.sample_pairs(count, n, seed)
    chunks = np.array_split(pr, workers)
    r = oracle_rate(lambda c: oracle.edm_pairs(x, c), chunks, [len(c) for c in chunks], workers)
    r.update({"unit": "pairs/s", "extrapolated": True,
              "sample": f"FP64 C oracle, squared distances of {count} seeded pairs, split over the "
                        f"host threads; extrapolated to n(n+1)/2 pairs by count"})
    return r


def cpu_stress(x, y, rows, workers):
    """The oracle's loss terms over whole rows (forward) and gradient rows
    (backward), one row block per thread."""
    import oracle
    oracle.build()
    n = len(x)
    blocks = np.array_split(np.asarray(rows), workers)
    fwd = oracle_rate(lambda b: oracle.stress_loss_rows(x, y, int(b[0]), int(b[-1]) + 1), blocks,
                      [int(sum(int(i) for i in b)) for b in blocks], workers)
    bwd = oracle_rate(lambda b: oracle.stress_grad_rows(x, y, b), blocks,
                      [len(b) * (n - 1) for b in blocks], workers)
    # a backward row touches n - 1 pairs from one side; each pair has two
    # sides, so pairs/s of the whole backward is half the rows' pair rate
    bwd["value"] /= 2
    bwd["single_core"] /= 2
    for r, what in ((fwd, "loss terms (D - delta)^2 of the pairs j < i"), (bwd, "gradient rows")):
        r.update({"unit": "pairs/s", "extrapolated": True,
                  "sample": f"FP64 C oracle, {what} of {len(rows)} rows {rows[0]}..{rows[-1]}, "
                            f"split over the host threads; extrapolated by pair count"})
    return {"fwd": fwd, "bwd": bwd}


def cpu_cover(m, n, rho):
    """The oracle's coverage count (map table walk, one thread) of the same
    problem, whole."""
    import oracle
    oracle.build()
    fn = {2: oracle.cover2, 3: oracle.cover3, 4: oracle.cover4}[m]
    t0 = time.perf_counter()
    fn(n, rho, "lambda")
    el = time.perf_counter() - t0
    vol = math.comb(n + m - 1, m)
    return {"value": vol / el, "unit": "elements/s", "cores": 1, "kind": "oracle", "extrapolated": False,
            "sample": f"FP64 C oracle, the whole lambda coverage of n={n}, rho={rho} on one thread",
            "seconds": el}
# ------------------------------------------------------------------ rows

def _median_ms(torch, fn, steps, warmup=1):
    return statistics.median(time_steps(torch, fn, steps, warmup))


def _kernel_ms(torch, sx, fn, steps=3, warmup=1):
    """Average duration of the entry point's main kernel (library event pairs)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    sx.simplex_profile(True)
    for _ in range(steps):
        fn()
    ms, k, _ = sx.simplex_profile_read()
    sx.simplex_profile(False)
    return ms / max(k, 1)


def _fp32_peak(torch):
    sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
    return sms * FP32_LANES_PER_SM * 2 * 2070e6 / 1e12


def row_edm_n1024_d3(torch, sx, peaks):
    """EDM n=1024, d=3: 524,800 FP32 outputs (2.1 MB); one launch is a few
    microseconds, so a step replays a CUDA graph of 1000 launches (no host
    launch overhead) and the output stays L2-resident."""
    x = torch.from_numpy(synth.make_points("edm_n1024_d3")).cuda()
    o = torch.empty(1024 * 1025 // 2, device="cuda")
    pairs = o.numel()
    reps = 1000
    r = {"unit": "pairs/s", "pairs": pairs, "prec": "fp32",
         "note": f"CUDA graph of {reps} launches per timed step; output L2-resident"}
    for mp in ("lambda", "bbox", "linear", "rb"):
        side = torch.cuda.Stream()
        side.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(side):
            for _ in range(3):
                sx.simplex_edm_packed(x, o, mp, "fp32")
        torch.cuda.current_stream().wait_stream(side)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            for _ in range(reps):
                sx.simplex_edm_packed(x, o, mp, "fp32")
        ms = _median_ms(torch, g.replay, 5) / reps
        r[mp] = pairs / (ms / 1e3)
        r[mp + "_us"] = ms * 1e3
        r[mp + "_hbm_gbs"] = 4 * pairs / (ms / 1e3) / 1e9
        del g
    r["lambda_vs_bbox"] = r["lambda"] / r["bbox"]
    r["lambda_vs_rb"] = r["lambda"] / r["rb"]
    r["cpu_baseline"] = cpu_edm(synth.make_points("edm_n1024_d3"), 4_000_000, host_cores())
    return r


def _edm_big(torch, sx, peaks, x, prec, maps=("lambda", "bbox", "rb"), out=None):
    n, d = x.shape
    o = out if out is not None else torch.empty(n * (n + 1) // 2, device="cuda")
    pairs = o.numel()
    ws = {mp: sx.workspace("edm", n, d, mp, prec) for mp in maps}
    r = {"unit": "pairs/s", "pairs": pairs, "prec": prec}
    for mp in maps:
        ms = _kernel_ms(torch, sx, lambda: sx.simplex_edm_packed(x, o, mp, prec, ws[mp]))
        r[mp] = pairs / (ms / 1e3)
        r[mp + "_ms"] = ms
    r["lambda_vs_bbox"] = r["lambda"] / r["bbox"]
    if "rb" in r:
        r["lambda_vs_rb"] = r["lambda"] / r["rb"]
    t = r["lambda_ms"] / 1e3
    r["hbm_gbs_lambda"] = 4.0 * pairs / t / 1e9          # packed output written
    r["hbm_frac_lambda"] = r["hbm_gbs_lambda"] / peaks["hbm_gbs"]
    if prec != "fp32":
        r["tensor_tflops_lambda"] = 6.0 * d * pairs / t / 1e12   # hi.hi + hi.lo + lo.hi
        r["tensor_frac_lambda"] = r["tensor_tflops_lambda"] / peaks["bf16_tflops"]
    sx.simplex_device_errors()
    return r


def _edm_error(torch, o, xh, seed, count=1_000_000, tile=128):
    """Relative error of packed EDM entries against the squared distance in
    FP64 (computed here from the FP32 inputs, by the definition): `count`
    seeded pairs over the whole triangle and as many pairs inside diagonal
    tiles of `tile` points (where the Gram form cancels most), plus the
    exact-zero diagonal.  Reported, not asserted (the tests assert)."""
    n = len(xh)
    x64 = xh.astype(np.float64)
    pr = synth.sample_pairs(count, n, seed)
    near = synth.sample_pairs(count, tile, seed + 1)
    base = (synth.splitmix64(seed + 2, count) % np.uint64(max(n // tile, 1))).astype(np.int64) * tile
    near = np.minimum(near + base[:, None], n - 1)
    near = np.stack([np.maximum(near[:, 0], near[:, 1]), np.minimum(near[:, 0], near[:, 1])], axis=1)
    out = {}
    for name, p in (("sampled", pr), ("diagonal_tiles", near)):
        i, j = p[:, 0], p[:, 1]
        got = o[torch.from_numpy(i * (i + 1) // 2 + j).cuda()].double().cpu().numpy()
        rel = np.empty(len(i))
        for c in range(0, len(i), 100_000):
            sl = slice(c, c + 100_000)
            ref = ((x64[i[sl]] - x64[j[sl]]) ** 2).sum(axis=1)
            off = i[sl] != j[sl]
            rel[sl] = np.where(off, np.abs(got[sl] - ref) / np.maximum(ref, 1e-30), 0.0)
        out[name] = {"pairs": int(len(i)), "max_rel": float(rel.max()),
                     "p99_rel": float(np.percentile(rel, 99))}
    d = np.arange(0, n, max(n // 4096, 1), dtype=np.int64)
    out["diagonal_exact_zero"] = bool((o[torch.from_numpy(d * (d + 1) // 2 + d).cuda()] == 0).all())
    out["reference"] = "FP64 squared distance of the FP32 inputs"
    out["tolerance"] = 1e-5
    return out


def row_edm_n32768_d256(torch, sx, peaks):
    """EDM n=32768, d=256 on tensor cores (BF16 hi+lo split): 536,887,296
    outputs, 2.15 GB written; FP32 SIMT path alongside."""
    xh = synth.make_points("edm_n32768_d256")
    x = torch.from_numpy(xh).cuda()
    o = torch.empty(len(xh) * (len(xh) + 1) // 2, device="cuda")
    r = _edm_big(torch, sx, peaks, x, "bf16x3", out=o)
    sx.simplex_edm_packed(x, o, "lambda", "bf16x3", sx.workspace("edm", x.shape[0], x.shape[1], "lambda", "bf16x3"))
    r["error_lambda"] = _edm_error(torch, o, xh, seed=21)
    r["fp32_simt_lambda"] = _edm_big(torch, sx, peaks, x, "fp32", ("lambda", "bbox"), out=o)["lambda"]
    del o
    torch.cuda.empty_cache()
    t = _edm_tiles(torch, sx, peaks, x)
    t["tensor_tflops_lambda"] = 6.0 * x.shape[1] * t["pairs"] / (t["lambda_ms"] / 1e3) / 1e12
    t["tensor_frac_lambda"] = t["tensor_tflops_lambda"] / peaks["bf16_tflops"]
    r["tiles"] = t
    r["cpu_baseline"] = cpu_edm(xh, 2_000_000, host_cores())
    return r


def row_edm_n65536_d64(torch, sx, peaks):
    """EDM n=65536, d=64 on tensor cores: 2,147,516,416 outputs, 8.6 GB."""
    w = synth.WORKLOADS["stress_n65536_d64"]
    xh = synth.normal(w["n"], w["d"], w["seed"])
    x = torch.from_numpy(xh).cuda()
    o = torch.empty(len(xh) * (len(xh) + 1) // 2, device="cuda")
    r = _edm_big(torch, sx, peaks, x, "bf16x3", out=o)
    sx.simplex_edm_packed(x, o, "lambda", "bf16x3", sx.workspace("edm", x.shape[0], x.shape[1], "lambda", "bf16x3"))
    r["error_lambda"] = _edm_error(torch, o, xh, seed=22)
    del o
    torch.cuda.empty_cache()
    r["tiles"] = _edm_tiles(torch, sx, peaks, x)
    r["cpu_baseline"] = cpu_edm(xh, 4_000_000, host_cores())
    return r


def _edm_tiles(torch, sx, peaks, x, prec="bf16x3", maps=("lambda", "bbox", "rb")):
    """The tile-packed layout (simplex_edm_tiles: each 128 x 128 tile one
    contiguous 64 KB block, written by TMA tensor stores of 4 KB boxes).
    Rates count the n(n+1)/2 pairs; the HBM figure counts the bytes the call
    writes (the whole diagonal tiles and the padding: 0.2% more than the
    packed rows at n = 65536)."""
    n, d = x.shape
    o = torch.empty(sx.simplex_edm_tiles_len(n), device="cuda")
    pairs = n * (n + 1) // 2
    ws = {mp: sx.workspace("edm", n, d, mp, prec) for mp in maps}
    r = {"unit": "pairs/s", "pairs": pairs, "bytes_written": 4 * o.numel(), "prec": prec}
    for mp in maps:
        ms = _kernel_ms(torch, sx, lambda: sx.simplex_edm_tiles(x, o, mp, prec, ws[mp]))
        r[mp] = pairs / (ms / 1e3)
        r[mp + "_ms"] = ms
    r["lambda_vs_bbox"] = r["lambda"] / r["bbox"]
    if "rb" in r:
        r["lambda_vs_rb"] = r["lambda"] / r["rb"]
    t = r["lambda_ms"] / 1e3
    r["hbm_gbs_lambda"] = 4.0 * o.numel() / t / 1e9
    r["hbm_frac_lambda"] = r["hbm_gbs_lambda"] / peaks["hbm_gbs"]
    sx.simplex_device_errors()
    del o
    return r


def row_edm_n16384_d64(torch, sx, peaks):
    """EDM n=16384, d=64 on tensor cores (134M outputs, 537 MB): a smaller
    case of the same kernel, sized for profiler captures."""
    x = torch.from_numpy(synth.normal(16384, 64, seed=4)).cuda()
    r = _edm_big(torch, sx, peaks, x, "bf16x3")
    r["tiles"] = _edm_tiles(torch, sx, peaks, x)
    return r


def row_edm_n16384_d256(torch, sx, peaks):
    """EDM n=16384, d=256 on tensor cores (the d >= 128 kernel, 134M outputs):
    a smaller case of the n=32768 configuration, sized for profiler captures."""
    x = torch.from_numpy(synth.normal(16384, 256, seed=2)).cuda()
    return _edm_big(torch, sx, peaks, x, "bf16x3")


def _atm_row(torch, sx, x, maps=("lambda", "bbox", "linear"), steps=3, warmup=1):
    """ATM energy (pair tables + energy kernel + FP64 reduction) and energy
    with forces (force tables + forces kernel) per map: whole-call rates,
    L2 not flushed (the tables of a call are larger than L2 from n = 4096)."""
    n = len(x)
    r = {"unit": "triplets/s", "triples": triples(n), "n": n}
    e = torch.empty((), dtype=torch.float64, device="cuda")
    for mp in maps:
        ws = sx.workspace("atm_energy", n, 3, mp)
        ms = _median_ms(torch, lambda: sx.simplex_atm_energy(x, NU, EPS, e, mp, ws), steps, warmup)
        r["energy_" + mp] = triples(n) / (ms / 1e3)
        del ws
    f = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    for mp in maps:
        ws = sx.workspace("atm_forces", n, 3, mp)
        ms = _median_ms(torch, lambda: sx.simplex_atm_forces(x, NU, EPS, e, f, mp, ws), steps, warmup)
        r["energy_forces_" + mp] = triples(n) / (ms / 1e3)
        del ws
        torch.cuda.empty_cache()
    for k in ("energy", "energy_forces"):
        r[k + "_lambda_vs_bbox"] = r[k + "_lambda"] / r[k + "_bbox"]
        if "linear" in maps:
            r[k + "_lambda_vs_linear"] = r[k + "_lambda"] / r[k + "_linear"]
    r["energy_fp32_frac"] = FLOPS_PER_TRIPLE * r["energy_lambda"] / 1e12 / _fp32_peak(torch)
    r["energy_forces_fp32_frac"] = FORCE_FLOPS_PER_TRIPLE * r["energy_forces_lambda"] / 1e12 / _fp32_peak(torch)
    return r


def _atm_cpu(xh, target):
    w = host_cores()
    rows = rows_with(len(xh), target, w)
    return {"energy": cpu_atm(xh, rows, False, w), "energy_forces": cpu_atm(xh, rows, True, w)}


def row_atm_n4096(torch, sx, peaks):
    """ATM n=4096 (differentiation config): energy, energy+forces."""
    xh = synth.make_points("atm_n4096")
    r = _atm_row(torch, sx, torch.from_numpy(xh).cuda())
    r["cpu_baseline"] = _atm_cpu(xh, 8_000_000)
    return r


def row_atm_n3000(torch, sx, peaks):
    """ATM n=3000 (a non-power of two: lambda pads the 94 blocks to 128 and
    filters, Sec. III-A "approach n from above"), uniform in a cube of side
    20, seed 7."""
    xh = synth.uniform_cube(3000, 3, 20.0, seed=7)
    r = _atm_row(torch, sx, torch.from_numpy(xh).cuda())
    r["grid_blocks"] = {mp: sx.simplex_grid_blocks(3, -(-3000 // 32), mp) for mp in ("lambda", "bbox", "linear")}
    r["cpu_baseline"] = _atm_cpu(xh, 4_000_000)
    return r


def row_atm_n12000(torch, sx, peaks):
    """ATM n=12000 (375 blocks, padded to 512 by lambda), uniform in a cube
    of side 20, seed 8: 2.88e11 triples."""
    xh = synth.uniform_cube(12000, 3, 20.0, seed=8)
    r = _atm_row(torch, sx, torch.from_numpy(xh).cuda(), steps=2)
    r["grid_blocks"] = {mp: sx.simplex_grid_blocks(3, -(-12000 // 32), mp) for mp in ("lambda", "bbox", "linear")}
    r["cpu_baseline"] = _atm_cpu(xh, 20_000_000)
    return r


def row_atm_n1024(torch, sx, peaks, steps=100):
    """ATM energy alone, n=1024 (the 3-simplex plain config, 178,433,024
    triples): the step is the pair tables, the energy kernel and the FP64
    reduction, L2 flushed between steps; the energy kernel against the FP32
    ALU roofline; the energy against the oracle's FP64 sum."""
    xh = synth.make_points("atm_n1024")
    x = torch.from_numpy(xh).cuda()
    n = len(xh)
    units = triples(n)
    e = torch.empty((), dtype=torch.float64, device="cuda")
    flush_buf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    flush = lambda: flush_buf.fill_(1)  # noqa: E731
    r = {"unit": "triplets/s", "triples": units}
    e_gpu = None
    for mp in ("lambda", "bbox", "linear"):
        ws = sx.workspace("atm_energy", n, 3, mp)
        step = lambda: sx.simplex_atm_energy(x, NU, EPS, e, mp, ws)  # noqa: E731
        ts = time_steps(torch, step, steps, 3, flush, label="energy_n1024_" + mp)
        r[mp] = units / (sum(ts) / len(ts) / 1e3)
        r[mp + "_ms"] = sum(ts) / len(ts)
        if mp == "lambda":
            sx.simplex_profile(True)
            time_steps(torch, step, 20, 0, flush, label="energy_n1024_kernel")
            k_ms, k, _ = sx.simplex_profile_read()
            sx.simplex_profile(False)
            k_ms /= max(k, 1)
            r["kernel"] = "k_atm_energy_tab<lambda>"
            r["kernel_ms"] = k_ms
            r["kernel_tflops"] = FLOPS_PER_TRIPLE * units / (k_ms / 1e3) / 1e12
            r["kernel_fp32_frac"] = r["kernel_tflops"] / _fp32_peak(torch)
            e_gpu = float(e.item())
    del flush_buf
    r["lambda_vs_bbox"] = r["lambda"] / r["bbox"]
    r["lambda_vs_linear"] = r["lambda"] / r["linear"]
    import oracle
    oracle.build()
    r["cpu_baseline"] = cpu_atm(xh, list(range(0, n - 2)), False, host_cores())
    r["cpu_baseline"]["extrapolated"] = False
    r["cpu_baseline"]["sample"] = "FP64 C oracle, the whole n=1024 sum, one i-row per task on the host threads"
    e_ref = oracle.atm_energy(xh, NU, EPS)
    r["accuracy"] = {"energy": e_gpu, "energy_oracle": e_ref, "rel_err": abs(e_gpu - e_ref) / abs(e_ref),
                     "tolerance": 1e-6}
    return r


def row_stress_n65536_d64(torch, sx, peaks):
    """Stress loss n=65536, d=64: forward (loss only) and backward."""
    w = synth.WORKLOADS["stress_n65536_d64"]
    xn = synth.normal(w["n"], w["d"], w["seed"])
    yn = synth.perturbed(xn, w["sigma"], w["y_seed"])
    x = torch.from_numpy(xn).cuda()
    y = torch.from_numpy(yn).cuda()
    n = w["n"]
    pairs = n * (n - 1) // 2
    r = {"unit": "pairs/s", "pairs": pairs}
    loss = torch.empty((), dtype=torch.float64, device="cuda")
    ws = sx.workspace("stress_fwd", n, w["d"], "lambda")
    ms = _median_ms(torch, lambda: sx.simplex_stress_fwd(x, y, None, loss, "lambda", "fp32", ws), 2)
    r["fwd_lambda"] = pairs / (ms / 1e3)
    g = torch.empty_like(x)
    ms = _median_ms(torch, lambda: sx.simplex_stress_bwd(x, y, 1.0, g, "lambda", "fp32"), 2)
    r["bwd_lambda"] = pairs / (ms / 1e3)
    # algorithmic FP32 flops per pair: forward 4d (two FMAs per coordinate),
    # backward 8d (the residual plus the two tile products)
    d = w["d"]
    fp32 = _fp32_peak(torch)
    r["fwd_tflops"] = 4 * d * r["fwd_lambda"] / 1e12
    r["bwd_tflops"] = 8 * d * r["bwd_lambda"] / 1e12
    r["fwd_fp32_frac"] = r["fwd_tflops"] / fp32
    r["bwd_fp32_frac"] = r["bwd_tflops"] / fp32
    r.update(_stress_tensor(torch, sx, peaks, x, y, ("lambda", "bbox", "linear", "rb")))
    w_ = host_cores()
    r["cpu_baseline"] = cpu_stress(xn, yn, list(range(n - 4 * w_, n)), w_)
    return r


def _stress_tensor(torch, sx, peaks, x, y, maps):
    """Tensor-core stress forward and backward (BF16 hi+lo products): pairs/s
    per map and the issued MMA rate of the lambda map against the measured
    BF16 peak.  Per 128 x 128 tile the forward issues three K = 2d products,
    the backward adds three K = 128 products of N = d + 16 for each side;
    the rate of the pass that returns loss and gradient together as well."""
    n, d = x.shape
    pairs = n * (n - 1) // 2
    nb = -(-n // 128)
    tiles = nb * (nb + 1) // 2
    f_mma = tiles * 128 * 128 * 2 * (2 * d) * 3
    b_mma = f_mma + tiles * 2 * 128 * (d + 16) * 2 * 128 * 3
    r = {}
    loss = torch.empty((), dtype=torch.float64, device="cuda")
    g = torch.empty_like(x)
    for mp in maps:
        wf = sx.workspace("stress_fwd", n, d, mp, "bf16x3")
        ms = _median_ms(torch, lambda: sx.simplex_stress_fwd(x, y, None, loss, mp, "bf16x3", wf), 3)
        r["tc_fwd_" + mp] = pairs / (ms / 1e3)
        if mp == "lambda":
            r["tc_fwd_ms"] = ms
            r["tc_fwd_mma_tflops"] = f_mma / (ms / 1e3) / 1e12
        del wf
        wb = sx.workspace("stress_bwd", n, d, mp, "bf16x3")
        ms = _median_ms(torch, lambda: sx.simplex_stress_bwd(x, y, 1.0, g, mp, "bf16x3", wb), 3)
        r["tc_bwd_" + mp] = pairs / (ms / 1e3)
        if mp == "lambda":
            r["tc_bwd_ms"] = ms
            r["tc_bwd_mma_tflops"] = b_mma / (ms / 1e3) / 1e12
        del wb
    # loss and gradient in one pass (the backward kernel summing the loss too)
    wfb = sx.workspace("stress_fwd_bwd", n, d, "lambda", "bf16x3")
    ms = _median_ms(torch, lambda: sx.simplex_stress_fwd_bwd(x, y, 1.0, g, loss, "lambda", "bf16x3", wfb), 3)
    r["tc_fwd_bwd_lambda"] = pairs / (ms / 1e3)
    r["tc_fwd_bwd_ms"] = ms
    del wfb
    bf16 = peaks.get("bf16_tflops") if peaks else None
    if bf16:
        r["tc_fwd_bf16_frac"] = r["tc_fwd_mma_tflops"] / bf16
        r["tc_bwd_bf16_frac"] = r["tc_bwd_mma_tflops"] / bf16
    return r


def row_stress_n16384_d64(torch, sx, peaks):
    """Stress loss n=16384, d=64 on tensor cores: a smaller case of the same
    kernels, sized for profiler captures."""
    xn = synth.normal(16384, 64, seed=4)
    x = torch.from_numpy(xn).cuda()
    y = torch.from_numpy(synth.perturbed(xn, 0.1, seed=5)).cuda()
    return _stress_tensor(torch, sx, peaks, x, y, ("lambda",))


def _cover_row(torch, sx, m, n, rho, cpu=True):
    """Coverage of the m-simplex with one thread per element: each map's grid
    launched as is, every thread decoding its block and counting its element
    (an atomic increment) or itself as idle.  The per-element work is one
    atomic, so here the threads a map launches outside the simplex weigh as
    much as the work itself (the parallel space of Sec. III)."""
    vol = math.comb(n + m - 1, m)
    count = torch.empty(vol, dtype=torch.int32, device="cuda")
    idle = torch.empty(1, dtype=torch.int64, device="cuda")
    fn = {2: sx.simplex_map2, 3: sx.simplex_map3, 4: sx.simplex_map4}[m]
    r = {"unit": "elements/s", "elements": vol, "rho": rho}
    maps = {2: ("lambda", "bbox", "linear", "rb"), 3: ("lambda", "bbox", "linear"), 4: ("lambda", "bbox")}[m]
    for mp in maps:
        ms = _median_ms(torch, lambda: fn(n, rho, mp, count, idle), 5)
        r[mp] = vol / (ms / 1e3)
        r[mp + "_ms"] = ms
        r[mp + "_idle_threads"] = int(idle.item())
        r[mp + "_threads_per_element"] = (int(idle.item()) + vol) / vol
    r["lambda_vs_bbox"] = r["lambda"] / r["bbox"]
    if m == 2:
        r["lambda_vs_rb"] = r["lambda"] / r["rb"]
        r["lambda_vs_linear"] = r["lambda"] / r["linear"]
    if cpu:
        r["cpu_baseline"] = cpu_cover(m, n, rho)
    return r


def row_cover2_n16384(torch, sx, peaks):
    """Coverage of the 2-simplex, n=16384, 16x16 threads per block."""
    return _cover_row(torch, sx, 2, 16384, 16)


def row_cover3_n1024(torch, sx, peaks):
    """Coverage of the 3-simplex, n=1024, 8x8x8 threads per block."""
    return _cover_row(torch, sx, 3, 1024, 8)


def row_cover4_n256(torch, sx, peaks):
    """Coverage of the 4-simplex, n=256, 4^4 threads per block: the lambda
    map of the r = 1/2, beta = 2 set (plus the m = 3 map for the plane
    K = L) against the bounding box's 64^4 blocks."""
    return _cover_row(torch, sx, 4, 256, 4)


def row_cover2_n12000(torch, sx, peaks):
    """Coverage of the 2-simplex at a non-power of two, n=12000, 16x16
    threads per block (750 blocks: lambda pads to 1024)."""
    r = _cover_row(torch, sx, 2, 12000, 16)
    r["grid_blocks"] = {mp: sx.simplex_grid_blocks(2, 750, mp) for mp in ("lambda", "bbox", "linear", "rb")}
    return r


def row_edm_n49152_d64(torch, sx, peaks):
    """EDM at a non-power of two, n=49152 (384 tiles of 128, 192 super-blocks
    of 256: lambda pads them to 256), d=64, N(0,1) seed 9: both layouts,
    every map."""
    xh = synth.normal(49152, 64, seed=9)
    x = torch.from_numpy(xh).cuda()
    maps = ("lambda", "bbox", "linear", "rb")
    r = _edm_big(torch, sx, peaks, x, "bf16x3", maps)
    torch.cuda.empty_cache()
    r["tiles"] = _edm_tiles(torch, sx, peaks, x, maps=maps)
    r["grid_blocks_256"] = {mp: sx.simplex_grid_blocks(2, 192, mp) for mp in maps}
    r["cpu_baseline"] = cpu_edm(xh, 4_000_000, host_cores())
    return r


ROWS = {
    "cover2_n16384": row_cover2_n16384,
    "cover3_n1024": row_cover3_n1024,
    "cover4_n256": row_cover4_n256,
    "edm_n1024_d3": row_edm_n1024_d3,
    "edm_n32768_d256": row_edm_n32768_d256,
    "edm_n65536_d64": row_edm_n65536_d64,
    "atm_n1024": row_atm_n1024,
    "atm_n4096": row_atm_n4096,
    "stress_n65536_d64": row_stress_n65536_d64,
    # non-powers of two (lambda pads to the next power and filters)
    "cover2_n12000": row_cover2_n12000,
    "edm_n49152_d64": row_edm_n49152_d64,
    "atm_n3000": row_atm_n3000,
    "atm_n12000": row_atm_n12000,
}
# profiling-only cases (not part of the default rows)
PROFILE_ROWS = {"edm_n16384_d64": row_edm_n16384_d64, "edm_n16384_d256": row_edm_n16384_d256,
                "stress_n16384_d64": row_stress_n16384_d64}


def rows_measure(torch, sx, peaks, names=None):
    """Every other kernel of the path at its own configuration."""
    out = {}
    for name, fn in ROWS.items():
        if names is None or name in names:
            out[name] = fn(torch, sx, peaks)
            torch.cuda.empty_cache()
    return out


def row_only(args):
    """--row NAME: just that row (for profiling one kernel)."""
    import torch
    import paper_1610_07394_gb300 as sx
    sx.lib()
    peaks, _ = measured_peaks()
    fn = ROWS.get(args.row) or PROFILE_ROWS[args.row]
    print(json.dumps({"row": args.row, **fn(torch, sx, peaks)}), flush=True)


# ------------------------------------------------------------------ the headline workload

def config_block():
    w = synth.WORKLOADS[WORKLOAD]
    return {"workload": f"ATM triple-dipole energy and adjoint forces (E, F = -dE/dx) over i<j<k, "
                        f"n={w['n']} uniform in a cube of side {w['side']:g}, seed {w['seed']}, nu=1, "
                        f"eps=1e-4 ({triples(w['n'])} triples)",
            "map": "lambda (two-branch recursive 3-simplex map + J=K plane)",
            "n": w["n"], "triples": triples(w["n"]),
            "l2": f"flushed before every timed step ({L2_FLUSH_BYTES >> 20} MB write); the call's "
                  f"force tables (9.7 GB) exceed L2 as well"}


def headline_cpu_rows(n, workers):
    """The i-rows the oracle times for the headline (about 1e7 triples each,
    one per host thread)."""
    return rows_with(n, 10_000_000, workers)


def reference_arm(args):
    """The FP64 oracle on the host cores (all of them, one i-row of the
    3-simplex per thread) on the headline's metric: each step the energy and
    gradient of a bounded sample of the n=16384 triples."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    x = synth.make_points(WORKLOAD)
    import oracle
    oracle.build()
    n = len(x)
    xd = x.astype(np.float64)
    workers = host_cores()
    rows = headline_cpu_rows(n, workers)
    units = sum(row_triples(n, i) for i in rows)

    def work(i):
        oracle.atm_energy_grad_slice(xd, i, i + 1, NU, EPS)

    for _ in range(args.warmup):
        host_parallel(work, rows, workers)
    ts = [host_parallel(work, rows, workers)[1] for _ in range(args.steps)]
    ms = 1e3 * sum(ts) / len(ts)
    value = units / (ms / 1e3)
    sample = (f"energy and gradient of the triples with i in rows {rows[0]}..{rows[-1]} of the n={n} "
              f"workload ({units} of {triples(n)} triples) per step, FP64 C oracle, one row per host "
              f"thread ({workers} threads); rate extrapolated to the whole sum by triple count")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "triplets/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": config_block(),
        "cpu_baseline": {"value": value, "unit": "triplets/s", "cores": workers, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "triplets/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def our_arm(args):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    import paper_1610_07394_gb300 as sx
    sx.lib()  # fails loudly when the CUDA library is missing

    peaks, peak_src = measured_peaks()
    props = torch.cuda.get_device_properties(local)
    sms = props.multi_processor_count
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    fp32_peak = sms * FP32_LANES_PER_SM * 2 * sm_max * 1e6 / 1e12   # TFLOP/s

    w = synth.WORKLOADS[WORKLOAD]
    n = w["n"]
    xh = synth.make_points(WORKLOAD)
    x = torch.from_numpy(xh).cuda()
    e = torch.empty((), dtype=torch.float64, device="cuda")
    f = torch.empty((n, 3), dtype=torch.float64, device="cuda")
    units = triples(n)
    flush_buf = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    flush = lambda: flush_buf.fill_(1)  # noqa: E731
    ws = sx.workspace("atm_forces", n, 3, "lambda")

    def step(mp="lambda", wsp=None):
        sx.simplex_atm_forces(x, NU, EPS, e, f, mp, ws if wsp is None else wsp)

    clocks = Clocks(local)
    clocks.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    # the timed steps run without the library's event pairs (profile(1) then
    # (0) clears the counters; the launch counter keeps counting), and a
    # second pass of a few steps with the event pairs on times the forces
    # kernel for the roofline
    sx.simplex_profile(True)
    sx.simplex_profile(False)
    times = time_steps(torch, step, args.steps, 0, flush, label="energy_forces_lambda")
    _, _, launches = sx.simplex_profile_read()
    sx.simplex_profile(True)
    time_steps(torch, step, min(args.steps, 3), 0, flush, label="energy_forces_kernel")
    main_ms, main_k, _ = sx.simplex_profile_read()
    sx.simplex_profile(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    value, ms_step = job_rate(sum(times) / len(times), units, world, dist, "cuda")
    k_ms = main_ms / max(main_k, 1)
    achieved = FORCE_FLOPS_PER_TRIPLE * units / (k_ms / 1e3) / 1e12
    e_step = float(e.item())
    f_step = f.cpu().numpy()

    # the same step on the other maps (same kernel body, same tile)
    maps = {"lambda": units / (ms_step / 1e3)}
    other = min(args.steps, 2)
    for mp in ("bbox", "linear"):
        wsm = sx.workspace("atm_forces", n, 3, mp)
        tt = time_steps(torch, lambda: step(mp, wsm), other, 1, flush, label="energy_forces_" + mp)
        maps[mp] = units / (sum(tt) / len(tt) / 1e3)
        maps[mp + "_energy_rel_diff"] = abs(float(e.item()) - e_step) / abs(e_step)
        del wsm
        torch.cuda.empty_cache()
    maps["lambda_vs_bbox"] = maps["lambda"] / maps["bbox"]
    maps["lambda_vs_linear"] = maps["lambda"] / maps["linear"]
    maps["grid_blocks"] = {mp: sx.simplex_grid_blocks(3, -(-n // sx.simplex_block_rho("atm_forces")), mp)
                           for mp in ("lambda", "bbox", "linear")}
    maps["steps_each"] = other

    # end to end through the public API with host buffers: the C ABI called
    # through the package's ctypes binding, with the H2D copy of x and the
    # D2H copies of E and F (pinned host memory) inside every timed step
    xp = torch.from_numpy(xh).pin_memory()
    ep = torch.empty((), dtype=torch.float64).pin_memory()
    fp = torch.empty((n, 3), dtype=torch.float64).pin_memory()

    def e2e_step():
        x.copy_(xp, non_blocking=True)
        step()
        ep.copy_(e, non_blocking=True)
        fp.copy_(f, non_blocking=True)

    te = time_steps(torch, e2e_step, min(args.steps, 5), 1, flush, label="energy_forces_e2e")
    e2e_value, _ = job_rate(sum(te) / len(te), units, world, dist, "cuda")
    e2e = {"value": e2e_value, "unit": "triplets/s",
           "h2d_bytes_per_step": int(xp.numel() * xp.element_size()),
           "d2h_bytes_per_step": int(ep.numel() * ep.element_size() + fp.numel() * fp.element_size()),
           "path": "simplex_atm_forces through the package's ctypes binding; torch copies from and to "
                   "pinned host buffers on the same stream", "steps": min(args.steps, 5)}
    del ws
    torch.cuda.empty_cache()

    do_rows = args.rows == "on" or (args.rows == "auto" and world == 1)
    rows = rows_measure(torch, sx, peaks) if (do_rows and rank == 0) else None
    clk = clocks.stop()

    traffic, traffic_note = stated_traffic("k_atm_forces_n16384.md")
    line = {
        "metric": METRIC, "value": value, "unit": "triplets/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": config_block(),
        "maps": maps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": fp32_peak, "unit": "TFLOP/s",
                     "frac": achieved / fp32_peak, "traffic": traffic, "traffic_source": traffic_note,
                     "algorithmic_bytes": 12 * n + 24 * n + 8,
                     "kernel": "k_atm_forces<lambda>", "kernel_ms": k_ms,
                     "flops_per_triple": FORCE_FLOPS_PER_TRIPLE,
                     "peak_basis": f"{sms} SMs x {FP32_LANES_PER_SM} FP32 lanes x 2 x {sm_max:g} MHz "
                                   f"(unit counts and max clock; the {peak_src} peaks file has no FP32 "
                                   f"figure)"},
        "e2e": e2e,
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0 and world == 1:
        workers = host_cores()
        line["cpu_baseline"] = cpu_atm(xh, headline_cpu_rows(n, workers), True, workers)
        # the step's forces on seeded atoms against the oracle's analytic
        # gradient (parity of the measured run; the energy is compared
        # across maps above, the oracle's O(n^3) sum being out of reach)
        import oracle
        oracle.build()
        atoms = synth.sample_indices(8, n, seed=6 + 10 ** 6)
        g_ref, _ = host_parallel(lambda a: oracle.atm_grad_atoms(xh, [int(a)], NU, EPS)[0], list(atoms), workers)
        g_ref = np.array(g_ref)
        err = np.linalg.norm(f_step[atoms] + g_ref, axis=1) / np.linalg.norm(g_ref, axis=1)
        line["accuracy"] = {"forces_max_rel_err": float(err.max()), "atoms": len(atoms),
                            "reference": "FP64 oracle gradient rows", "tolerance": 1e-4,
                            "energy": e_step}
    if rows is not None:
        line["rows"] = rows
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def main():
    args = parse()
    if args.row:
        row_only(args)
    elif args.impl == "reference":
        reference_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
