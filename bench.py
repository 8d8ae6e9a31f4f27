#!/usr/bin/env python3
"""Benchmark of the spinor polarizability chi0_GG'(q, i w) on GB300.

One step = the whole hot path for one q-point of the Si-like workload
(FCC a = 10.26 bohr, 24^3 FFT box, ~2000 plane waves per spinor component,
N_G = 350, 4x4x4 k-grid (N_k = 64), N_v = 8, N_c = 200, omega = 0 plus 4
imaginary frequencies up to 40 eV, q = (1/4, 0, 0)): every k-point's spinor
coefficients go to the real-space grid, every (v, c, k) pair's matrix
elements are formed and contracted into chi0, and chi0 is finalised.
Inputs are seeded synthetic states of that shape (no DFT data).

Prints one JSON line (metric q-points/s); see --help.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    "si24": (dict(), "Si-like FCC a=10.26 bohr, 24^3 box, N_w~2000 per spinor component, N_G=350, "
             "N_k=64 (4x4x4), N_v=8, N_c=200, 5 imaginary freqs (0..40 eV), q=(1/4,0,0)"),
    # profiling case: the same per-launch shapes on a 2x2x2 k-grid (< 1 GB on the device)
    "si24_small": (dict(kgrid=(2, 2, 2), q=(0.5, 0, 0)),
                   "si24 shapes (24^3, N_G=350, N_v=8, N_c=200, 5 freqs) on a 2x2x2 k-grid, q=(1/2,0,0)"),
    "gasb32": ("gasb32", "GaSb-like FCC a=11.53 bohr, 32^3 box, N_w~5000 per spinor component, "
                         "N_G=800, N_k=216 (6x6x6), N_v=18, N_c=400, 16 imaginary freqs, q=(1/6,0,0)"),
    # profiling case: the GaSb-like per-launch shapes on a 2x2x2 k-grid (~2 GB on the device)
    "gasb32_small": (dict(config="gasb32", kgrid=(2, 2, 2), q=(0.5, 0, 0)),
                     "gasb32 shapes (32^3, N_G=800, N_v=18, N_c=400, 16 freqs) on a 2x2x2 k-grid, q=(1/2,0,0)"),
    "gasb32_batch": ("batch", "40 q-points of the GaSb-like 6x6x6 grid in one accumulate call: "
                              "32^3 box, N_G(q)~U{700..900}, N_c(q)~U{300..500}, N_v=18, 16 freqs"),
    "bi2se3": ("bi2se3", "Bi2Se3-like rhombohedral cell (hex a=4.143 A, c=28.636 A), 64^3 box, "
                         "N_w~9000 per spinor component, N_G=2000, N_k=216 (6x6x6), N_v=48, N_c=1000, "
                         "8 imaginary freqs, q=(1/6,0,0); real-space grids streamed through 8 slots"),
    # profiling case: the 64^3 box and N_G = 2000 on a 2x2x2 k-grid with 8 + 40 bands (~1.5 GB)
    "bi2se3_small": ("bi2se3_small", "Bi2Se3-like cell, 64^3 box, N_G=2000, 2x2x2 k-grid, N_v=8, N_c=40, "
                                     "2 freqs, q=(1/2,0,0)"),
}
METRIC = "spinor chi0 q-points/s and TFLOP/s, FP64 vs mixed at ≤2e-5 rel. Frobenius error"

# FP64 issue rate of GB300 derived from its nominal 1.25 TFLOP/s over 152 SMs
# at the 2070 MHz maximum clock: 1.25e12 / (152 * 2.07e9) ~ 4 flop/clk/SM,
# i.e. 2 DFMA per clock per SM.  Peak = 152 * 2 * 2 * 2.07e9.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# cuBLAS DGEMM 8192^3 through torch.matmul on this GPU type
# (profiles/alu_peaks_gb300.md; `bench.py --alu-peaks` measures it again).
MEASURED_DGEMM_TFLOPS = 1.101

# FP32 FFMA peak from unit counts and clocks: 152 SMs x 128 lanes x 2 flop x
# 2.07 GHz (cuBLAS SGEMM measures 69.7 TFLOP/s on this GPU type).
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12

# DRAM bytes (read + write) of one launch, from one ncu capture of the
# full-size workload with that k-chunk (profiles/traffic_si24.md); valid for
# the kernel sources they were taken on.  Keyed by (workload, kernel, k-chunk).
TRAFFIC = {("si24", "k4_herk_f64", 4): 36.19e6 + 44.94e6,
           ("si24", "k4_herk_f64", 16): 145.66e6 + 67.13e6,
           ("si24", "k5_gemm", 16): 477.86e6 + 3.10e6}


def traffic(workload, kernel, kchunk):
    return TRAFFIC.get((workload, kernel, kchunk))


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp64", "mixed"], default="fp64")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision comparison")
    ap.add_argument("--no-autotune", action="store_true", help="default tiles and k-chunk")
    ap.add_argument("--check-fp64", type=int, default=0, metavar="NQ",
                    help="with --precision mixed: compare the first NQ q-points with one FP64 run")
    ap.add_argument("--check-kspan", type=int, default=0, metavar="NK",
                    help="restrict the FP64 comparison to k-points 0..NK-1 (both precisions)")
    ap.add_argument("--grid-slots", type=int, default=-1,
                    help="real-space grid slots (0 = all k resident; default 8 for bi2se3, else 0)")
    ap.add_argument("--kchunk", type=int, default=0, help="k-chunk when not autotuning")
    ap.add_argument("--k1-path", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="sphere -> grid kernels: 0 automatic, 1 per axis, 2 one kernel per band component, "
                         "3 eight lanes per line (cubic 32/40/48/64), 4 one kernel without the shared cube")
    ap.add_argument("--mtxel-lanes", type=int, default=0, choices=[0, 1, 8],
                    help="FFT lanes per line of the matrix-element kernels (0 automatic)")
    ap.add_argument("--defer-k1", type=int, default=1, choices=[0, 1],
                    help="1 (default): build the grids of a step's uploads together at the accumulate "
                         "(one launch per 64 k-points where the box allows); 0: at each upload")
    ap.add_argument("--copy-ahead", type=int, default=1, choices=[0, 1],
                    help="1 (default): host uploads copy on a second stream, overlapping the transforms; "
                         "0: on the context stream")
    ap.add_argument("--overlap", type=int, default=1, choices=[0, 1],
                    help="mixed path: 1 (default) contracts each k-chunk on a second stream while the next "
                         "chunk's matrix elements run; 0: one stream")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="si24")
    ap.add_argument("--alu-peaks", action="store_true",
                    help="only time cuBLAS FP64 and FP32 (no TF32) GEMMs of 8192^3 through torch.matmul "
                         "and print them (the measured ALU ceilings for the roofline)")
    return ap.parse_args()


def alu_peaks():
    """Library GEMM rates that bound hand-written FP64 / FP32 arithmetic on
    this GPU: torch.matmul (cuBLAS) on 8192^3, FP64 and FP32 with TF32 off,
    CUDA events, 2 warm-ups, median of 5."""
    import torch
    torch.backends.cuda.matmul.allow_tf32 = False
    out = {}
    n = 8192
    for name, dt in (("fp64_gemm_tflops", torch.float64), ("fp32_gemm_tflops", torch.float32)):
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        c = torch.empty(n, n, dtype=dt, device="cuda")
        ts = []
        for i in range(7):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            torch.matmul(a, b, out=c)
            e1.record()
            torch.cuda.synchronize()
            if i >= 2:
                ts.append(e0.elapsed_time(e1))
        out[name] = 2 * n ** 3 / (statistics.median(ts) * 1e-3) / 1e12
        del a, b, c
    out["gpu"] = torch.cuda.get_device_name()
    return out


# ----------------------------------------------------------- distributed --

def dist_setup():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Dist:
    def __init__(self, world, rank, backend):
        self.world, self.rank = world, rank
        self.pg = None
        if world > 1:
            import torch.distributed as dist
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# ---------------------------------------------------------------- clocks --

class ClockSampler:
    """nvidia-smi samples (every 200 ms) while the timed region runs."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.rows, self.proc = [], None
        self.dev = device_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


# ------------------------------------------------------------ flop model --

def flop_model(p):
    """Algorithmic FLOPs of one step over every q-point of the workload."""
    parts = [flop_model_q(p, iq) for iq in range(len(p.qs))]
    out = {k: sum(x[k] for x in parts) for k in parts[0]}
    out["wfn_to_grid"] = parts[0]["wfn_to_grid"]   # grids are built once per step
    out["total"] = out["wfn_to_grid"] + out["mtxel"] + out["contraction"]
    return out


def flop_model_q(p, iq=0):
    """Algorithmic FLOPs of one q-point: pruned radix FFTs (5 L log2 L per
    line of length L), the pair density (8 flops per point and spin
    component) and the Hermitian contraction (8 flops per complex MAC over
    N_G(N_G+1)/2 entries per pair and frequency)."""
    q, geps, nc = p.qs[iq]
    n = np.array(p.box, float)
    L = float(np.log2(n[0]))
    w = geps.max(0) - geps.min(0) + 1
    per_pair_fft = 5 * n[0] * L * (n[0] * n[1] + n[0] * w[1] + w[1] * w[2])
    per_pair_rho = 8 * 2 * np.prod(n)
    pairs = p.nk * p.nv * nc
    band_fft = 0.0
    for ik in range(p.nk):
        ws = p.gvec[ik].max(0) - p.gvec[ik].min(0) + 1
        band_fft += 2 * p.nbands * 5 * n[0] * L * (ws[1] * ws[2] + n[0] * ws[2] + n[0] * n[1])
    ng = len(geps)
    herk = 8.0 * pairs * len(p.freq) * ng * (ng + 1) / 2
    return {"wfn_to_grid": band_fft, "mtxel": pairs * (per_pair_fft + per_pair_rho),
            "contraction": herk, "total": band_fft + pairs * (per_pair_fft + per_pair_rho) + herk}


def byte_model(p, csize):
    """Least DRAM bytes of the two FFT stages in one step (every q-point):
    the sphere -> grid transform reads each band's coefficients (complex128)
    and writes its grid once; the matrix elements read the grids of the
    valence bands at k and the conduction bands at k+q once and write M once
    (csize bytes per complex value of the path's precision)."""
    vol = float(np.prod(p.box))
    coeff = sum(p.nbands * 2 * len(g) * 16.0 for g in p.gvec)
    grids = p.nk * p.nbands * 2 * vol * csize
    mtxel = 0.0
    for q, geps, nc in p.qs:
        mtxel += p.nk * (p.nv + nc) * 2 * vol * csize + p.nk * p.nv * nc * len(geps) * csize
    return {"wfn_to_grid": coeff + grids, "mtxel": mtxel}


# ---------------------------------------------------------------- oracle --

def oracle_sample(p, k_indices):
    """Time the CPU oracle on the given k-points of one q (all bands, all G,
    all frequencies); returns (seconds, threads)."""
    import oracle
    oracle.build()
    t0 = time.perf_counter()
    oracle.chi0(p, k_indices=k_indices)
    dt = time.perf_counter() - t0
    threads = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return dt, threads


def cpu_baseline(p):
    ks = [0]
    dt, cores = oracle_sample(p, ks)
    qps = 1.0 / (dt * p.nk / len(ks))
    return {"value": qps, "unit": "q-points/s", "cores": cores, "kind": "oracle",
            "sample": f"{len(ks)} of {p.nk} k-points of one q (all {p.nv}x{p.qs[0][2]} pairs, "
                      f"N_G={len(p.qs[0][1])}, {len(p.freq)} freqs) in {dt:.1f} s, scaled x{p.nk}"}


# ------------------------------------------------------------------ arms --

def make_workload(name):
    from paper_2206_00808_gb300 import synthetic as syn
    over, desc = WORKLOADS[name]
    if over == "batch":
        return syn.make_batched_problem(), desc
    if over == "bi2se3":
        return syn.make_bi2se3_problem(), desc
    if over == "bi2se3_small":
        # generated on the host (torch CPU QR): profilers run this case, and the
        # device QR's lazily loaded library is not found under them
        p = syn.make_bi2se3_problem(kgrid=(2, 2, 2), nv=8, nc=40, q=(0.5, 0, 0), nfreq=2, device="cpu")
        p.coeff = [c.numpy() for c in p.coeff]
        return p, desc
    if isinstance(over, str):
        return syn.make_problem(over), desc
    over = dict(over)
    return syn.make_problem(over.pop("config", "si24"), **over), desc


def run_reference(args, world, rank):
    if rank != 0:
        return 0
    p, desc = make_workload(args.workload)
    for _ in range(args.warmup and 1):
        oracle_sample(p, [0])
    times = []
    cores = 1
    for _ in range(args.steps):
        dt, cores = oracle_sample(p, [0])
        times.append(dt * p.nk)
    ms = 1e3 * statistics.mean(times)
    value = 1e3 / ms
    line = {"metric": METRIC, "value": value, "unit": "q-points/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": desc, "precision": "fp64"},
            "cpu_baseline": {"value": value, "unit": "q-points/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: 1 of {p.nk} k-points, scaled x{p.nk}"},
            "e2e": {"value": value, "unit": "q-points/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")


def bf16_peaks():
    """(burst, sustained) dense BF16 TFLOP/s measured on this machine, else the
    fallback figures."""
    try:
        with open(MEASURED_PEAKS) as f:
            d = json.load(f)
        return float(d["bf16_tflops"]), float(d["bf16_tflops_sustained"]), "measured"
    except (OSError, KeyError, ValueError):
        return 1900.0, 1700.0, "fallback"


def measured_hbm_gbs():
    """The measured copy rate (read + write bytes) of this machine, else the
    fallback figure."""
    try:
        with open(MEASURED_PEAKS) as f:
            return float(json.load(f)["hbm_gbs"])
    except (OSError, KeyError, ValueError):
        return 6800.0


def measure(B, torch, p, precision, args, dist, stream, dev_in, local, with_clocks):
    """Time `args.steps` full steps of one precision; returns a dict.

    The steps run as one captured CUDA graph replayed K times (value); a
    profiled eager pass of K steps gives the per-stage breakdown."""
    nf = len(p.freq)
    outs = [torch.empty((nf, len(g), len(g)), dtype=torch.complex128, device="cuda") for _, g, _ in p.qs]
    torch.cuda.synchronize()
    ctx = B.Chi0Context(p, precision, stream)
    if args.grid_slots > 0:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_GRID_SLOTS, args.grid_slots)
    # FP64 has no tile to tune; its k-chunk is fixed at 4 k-points per launch
    # (the fastest in the autotuner's timings on si24, and the configuration
    # whose DRAM traffic was captured for the roofline line)
    fixed_fp64 = precision == "fp64" and not args.no_autotune and args.kchunk == 0
    if args.kchunk > 0 or fixed_fp64:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_KCHUNK, args.kchunk if args.kchunk > 0 else min(4, p.nk))
    if args.k1_path > 0:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_K1_PATH, args.k1_path)
    if args.mtxel_lanes > 0:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_MTXEL_LANES, args.mtxel_lanes)
    if args.defer_k1:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_DEFER_K1, 1)
    if args.copy_ahead:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_COPY_AHEAD, 1)
    if args.overlap and precision == "mixed":
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_OVERLAP, 1)
    ctx.upload(device_inputs=dev_in)
    tune_span = min(p.nk, 16)
    if fixed_fp64:
        tuning = {"kchunk": min(4, p.nk), "pair_tile": [0, 0], "autotuned": False}
    else:
        tuning = ctx.autotune(0, tune_span) if not args.no_autotune else None

    def step():
        ctx.reset()
        ctx.upload(device_inputs=dev_in)
        ctx.accumulate()
        for iq, o in enumerate(outs):
            B.bgw_chi0_finalize(ctx.ctx, iq, o)

    def timed(fn, n):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(n):
            fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        dist.barrier()
        torch.cuda.synchronize()
        return dist.max(ev0.elapsed_time(ev1))

    for _ in range(max(3, args.warmup)):
        step()
    # eager, profiled: stage breakdown and per-kernel times, on one stream so
    # that each kernel's events bracket it alone
    ovl = args.overlap and precision == "mixed"
    if ovl:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_OVERLAP, 0)
    B.bgw_profile(ctx.ctx, True)
    ms_eager = timed(step, args.steps)
    prof = B.bgw_profile_read(ctx.ctx)
    B.bgw_profile(ctx.ctx, False)
    if ovl:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_OVERLAP, 1)
    # graph of one step, replayed
    B.bgw_graph_begin(ctx.ctx)
    step()
    B.bgw_graph_end(ctx.ctx)
    for _ in range(3):
        B.bgw_graph_launch(ctx.ctx)
    clk = ClockSampler(local) if with_clocks else None
    if clk:
        clk.__enter__()
    ms_total = timed(lambda: B.bgw_graph_launch(ctx.ctx), args.steps)
    if clk:
        clk.__exit__(None, None, None)
    res = {"ctx": ctx, "out": outs[0], "outs": outs, "ms": ms_total / args.steps,
           "ms_eager": ms_eager / args.steps,
           "prof": prof, "clocks": clk.summary() if clk else None, "tuning": tuning}
    res["stages"] = {s: {"ms_per_step": sms / args.steps, "share": sms / max(1e-9, ms_eager),
                         "launch_groups": calls, "kernels": kern}
                     for s, (sms, calls, kern) in prof.items() if calls}
    res["gpu_launches"] = sum(v["kernels"] for v in res["stages"].values())
    # achieved algorithmic rate and roofline fraction of each stage with a FLOP model
    fl = flop_model(p)
    burst, sustained, _ = bf16_peaks()
    peaks = ({"wfn_to_grid": (FP64_PEAK_TFLOPS, "FP64 ALU (derived)"),
              "mtxel": (FP64_PEAK_TFLOPS, "FP64 ALU (derived)"),
              "contraction": (FP64_PEAK_TFLOPS, "FP64 ALU (derived)")}
             if precision == "fp64" else
             {"wfn_to_grid": (FP32_PEAK_TFLOPS, "FP32 ALU (derived)"),
              "mtxel": (FP32_PEAK_TFLOPS, "FP32 ALU (derived)"),
              "contraction": (sustained / 3, "BF16 sustained / 3 products")})
    bm = byte_model(p, 16 if precision == "fp64" else 8)
    hbm = measured_hbm_gbs()
    for name, st in res["stages"].items():
        if name in peaks and st["ms_per_step"] > 0:
            tf = fl[name] / (st["ms_per_step"] * 1e-3) / 1e12
            st.update({"tflops": tf, "peak_tflops": peaks[name][0], "roofline_frac": tf / peaks[name][0],
                       "peak": peaks[name][1]})
        if name in bm and st["ms_per_step"] > 0:
            gbs = bm[name] / (st["ms_per_step"] * 1e-3) / 1e9
            st.update({"hbm_bytes_min": bm[name], "hbm_gbs_min": gbs, "hbm_frac_min": gbs / hbm})
    return res


def epsinv_measure(B, torch, p, res, stream, reps=3):
    """The step after chi0: W = eps^-1 v of every frequency of the first
    q-point from the device chi0 of the last timed step (bgw_epsinv, FP64),
    timed with CUDA events on the bench stream; FLOPs = 8 N_G^3 per matrix
    (complex Gauss-Jordan inversion)."""
    q, geps, _ = p.qs[0]
    s = B.bgw_coulomb_sqrt(p.avec, q, geps)
    chi = res["outs"][0]
    nf, ng = chi.shape[0], chi.shape[1]
    ws = torch.empty(B.bgw_epsinv_workspace_bytes(ng, nf), dtype=torch.uint8, device="cuda")
    times = []
    for _ in range(reps + 1):
        t = chi.clone()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.bgw_epsinv(t, s, "W", work=ws, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times[1:])
    tf = 8.0 * ng ** 3 * nf / (ms * 1e-3) / 1e12
    return {"what": "W = eps^-1 v(q+G') for every frequency of one q (FP64, blocked Gauss-Jordan on "
                    "the symmetrised eps)", "n_g": ng, "n_freq": nf, "ms_per_q": ms, "tflops": tf,
            "peak_tflops": FP64_PEAK_TFLOPS, "roofline_frac": tf / FP64_PEAK_TFLOPS}


def unfold_measure(B, torch, p, dev_in, stream, reps=3):
    """Spinor symmetry unfolding by one operation of the FCC lattice with a
    fractional translation, on as many bands as the step uploads in all (the
    band sets of every k-point, here on the sphere of k-point 0 in one call so
    that one launch is timed, not 64 host round trips), timed with CUDA
    events.  DRAM-bound: 64 bytes read and written per band, spin pair and
    plane wave, against the measured copy rate."""
    A = np.asarray(p.avec).T
    Rc = np.array([[0.0, 0.0, 1.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])   # 120 degrees about (1,1,1)
    R_lat = np.rint(np.linalg.inv(A) @ Rc @ A).astype(np.int32)
    tau = (0.25, 0.25, 0.25)
    nb = sum(int(c.shape[0]) for c, _ in dev_in)
    ngw = len(p.gvec[0])
    g = torch.Generator(device="cuda")
    g.manual_seed(7)
    cin = torch.randn((nb, 2, ngw), dtype=torch.complex128, device="cuda", generator=g)
    cout = torch.empty_like(cin)
    times = []
    for _ in range(reps + 1):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        B.bgw_unfold_spinor(p.avec, R_lat, tau, p.gvec[0], cin, cout, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times[1:])
    nbytes = 2 * cin.numel() * cin.element_size()
    gbs = nbytes / (ms * 1e-3) / 1e9
    hbm = measured_hbm_gbs()
    # per band, spin pair and plane wave: the 2 x 2 complex product, 16 FP64
    # fused multiply-adds (the phase is folded into U once per plane wave)
    dfma = 16.0 * nb * ngw
    dfma_peak = FP64_PEAK_TFLOPS * 1e12 / 2              # DFMA instructions per second
    del cin, cout
    return {"what": "c(G) -> U c(R^-1 G) e^{-iG.tau} (FP64), one launch over the bands of every k of the step",
            "bands": nb, "plane_waves": ngw, "bytes": nbytes, "ms": ms, "gbs": gbs, "peak_gbs": hbm,
            "hbm_frac": gbs / hbm if hbm else None,
            "fp64_fma_per_s": dfma / (ms * 1e-3), "fp64_frac": dfma / (ms * 1e-3) / dfma_peak,
            "bound": "alu (FP64): 16 DFMA per 64 bytes outruns the DRAM time on this part"}


def e2e_measure(B, torch, p, res, args, dist, stream):
    """Same step from pinned host buffers, chi0 read back to host."""
    ctx = res["ctx"]
    q, geps, nc = p.qs[0]
    ng, nf = len(geps), len(p.freq)
    pin = [(torch.from_numpy(np.ascontiguousarray(p.coeff[ik])).pin_memory(),
            torch.from_numpy(np.ascontiguousarray(p.energy[ik])).pin_memory()) for ik in range(p.nk)]
    host_out = torch.empty((nf, ng, ng), dtype=torch.complex128).pin_memory()
    h2d = sum(c.numel() * c.element_size() + e.numel() * e.element_size() for c, e in pin)
    d2h = host_out.numel() * host_out.element_size()

    def e2e_step():
        ctx.reset()
        ctx.upload(device_inputs=pin)
        ctx.accumulate()
        B.bgw_chi0_finalize(ctx.ctx, 0, host_out.numpy())

    for _ in range(max(3, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    dist.barrier()

    def pipelined(n):
        # each step's inputs are uploaded while the previous step accumulates
        # (copy-ahead host uploads); every step still copies its inputs in and
        # reads its chi0 back to host
        ctx.reset()
        ctx.upload(device_inputs=pin)
        for i in range(n):
            ctx.accumulate()
            if i + 1 < n:
                ctx.upload(device_inputs=pin)
            B.bgw_chi0_finalize(ctx.ctx, 0, host_out.numpy())
            ctx.reset()

    def timed(fn):
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        dist.barrier()
        ev0.record(stream)
        fn()
        ev1.record(stream)
        torch.cuda.synchronize()
        return dist.max(ev0.elapsed_time(ev1)) / args.e2e_steps

    seq_ms = timed(lambda: [e2e_step() for _ in range(args.e2e_steps)])
    ems = seq_ms
    out = {"unit": "q-points/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
           "sequential": {"ms_per_step": seq_ms, "value": dist.world * 1e3 / seq_ms}}
    if args.copy_ahead:
        pipelined(2)
        ems = timed(lambda: pipelined(args.e2e_steps))
        out["pipelined"] = {"ms_per_step": ems, "value": dist.world * 1e3 / ems,
                            "how": "step s+1's uploads (copy-ahead) issued before step s's finalize"}
    out["matches_device_step"] = bool(np.array_equal(host_out.numpy(), res["outs"][0].cpu().numpy()))
    out.update({"value": dist.world * 1e3 / ems, "ms_per_step": ems})
    return out


def rel_fro(a, b):
    return float(np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()))


def run_ours(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    dist = Dist(world, rank, "nccl")
    from paper_2206_00808_gb300 import build
    build.build()
    from paper_2206_00808_gb300 import binding as B

    p, desc = make_workload(args.workload)
    if args.grid_slots < 0:
        args.grid_slots = 8 if args.workload == "bi2se3" else 0
    q, geps, nc = p.qs[0]
    ng, nf = len(geps), len(p.freq)
    stream = torch.cuda.Stream()      # graph capture needs a non-default stream

    def dev(x):
        return x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x)).cuda()

    dev_in = [(dev(p.coeff[ik]), dev(p.energy[ik])) for ik in range(p.nk)]
    fl = flop_model(p)
    steps = args.steps

    nq = len(p.qs)
    head = measure(B, torch, p, args.precision, args, dist, stream, dev_in, local, True)
    ms = head["ms"]
    value = world * nq * 1e3 / ms
    con_ms, con_calls, _ = head["prof"]["contraction"]
    # algorithmic contraction FLOPs of the profiled steps over the kernel's summed device time
    achieved = fl["contraction"] * steps / (con_ms * 1e-3) / 1e12
    burst, sustained, src = bf16_peaks()
    head_kchunk = head["tuning"]["kchunk"] if head["tuning"] else max(1, args.kchunk)
    if args.precision == "fp64":
        # The kernel forms conj(M_g) M_g' once per pair (4 FP64 operations) and
        # weights it per frequency (2 FMAs each): (4 + 2 N_w) operations per
        # entry and pair where the algorithmic count is 4 N_w multiply-adds.
        nwc = -(-nf // 5)
        ops_ratio = (4.0 * nwc + 2.0 * nf) / (4.0 * nf)
        executed = achieved * ops_ratio
        roofline = {"bound": "alu", "kernel": "k4_herk_f64", "achieved": achieved,
                    "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP64_PEAK_TFLOPS,
                    "executed_fp64_tflops": executed, "executed_frac": executed / FP64_PEAK_TFLOPS,
                    "executed_over_algorithmic_ops": ops_ratio,
                    "traffic": traffic(args.workload, "k4_herk_f64", head_kchunk),
                    "peak_source": "derived: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz "
                                   "(nominal FP64 1.25 TFLOP/s)",
                    "measured_dgemm_tflops": MEASURED_DGEMM_TFLOPS,
                    "executed_frac_of_dgemm": executed / MEASURED_DGEMM_TFLOPS}
    else:
        roofline = {"bound": "tensor", "kernel": "k5_gemm", "achieved": achieved,
                    "peak": sustained / 3, "unit": "TFLOP/s", "frac": achieved / (sustained / 3),
                    "traffic": traffic(args.workload, "k5_gemm", head_kchunk),
                    "peak_source": f"{src} BF16 sustained {sustained} / 3 products"}
    epsinv = epsinv_measure(B, torch, p, head, stream) if args.precision == "fp64" else None
    unfold = unfold_measure(B, torch, p, dev_in, stream) if args.precision == "fp64" else None
    e2e = None if args.no_e2e else e2e_measure(B, torch, p, head, args, dist, stream)
    check = None
    if args.precision == "mixed" and args.check_fp64 > 0:
        import copy
        sub = copy.copy(p)
        sub.qs = p.qs[:args.check_fp64]
        kspan = args.check_kspan if args.check_kspan > 0 else p.nk
        res = {}
        for prec in ("fp64", "mixed"):
            cx = B.Chi0Context(sub, prec, stream)
            if args.grid_slots > 0:
                B.bgw_set_option(cx.ctx, B.BGW_OPT_GRID_SLOTS, args.grid_slots)
            cx.upload(device_inputs=dev_in)
            t0 = time.perf_counter()
            cx.accumulate(0, kspan)
            res[prec] = [cx.finalize(iq) for iq in range(len(sub.qs))]
            res[prec + "_s"] = time.perf_counter() - t0
            cx.close()
        errs = [rel_fro(g, r) for g, r in zip(res["mixed"], res["fp64"])]
        check = {"q_points_checked": len(sub.qs), "k_points": kspan,
                 "rel_fro_err_vs_fp64_max": max(errs), "fp64_seconds": res["fp64_s"],
                 "error_reference": "the FP64 GPU path (itself within 1e-10 of the CPU oracle)"}

    other = None
    if args.precision == "fp64" and not args.no_mixed:
        refs = [o.cpu().numpy() for o in head["outs"]]
        mix = measure(B, torch, p, "mixed", args, dist, stream, dev_in, local, False)
        gots = [o.cpu().numpy() for o in mix["outs"]]
        ref, got = refs[0], gots[0]
        gm_ms, gm_calls, _ = mix["prof"]["contraction"]
        gm_ach = fl["contraction"] * steps / (gm_ms * 1e-3) / 1e12
        pad_r = -(-2 * ng // 128) * 128
        nt = pad_r // 128
        kc = mix["tuning"]["kchunk"] if mix["tuning"] else 1
        pad_k = -(-(kc * p.nv * nc) // 64) * 64
        executed = 3 * 2.0 * nt * (nt + 1) / 2 * 128 * 128 * pad_k * nf * gm_calls
        offd = ~np.eye(ng, dtype=bool)
        other = {"precision": "mixed (FP32 grids/FFT, complex64 M, split-BF16 x3 tcgen05, "
                              "FP64 weights and k-reduction)",
                 "value": world * nq * 1e3 / mix["ms"], "unit": "q-points/s", "ms_per_step": mix["ms"],
                 "ms_per_step_eager": mix["ms_eager"],
                 "speedup_vs_fp64": ms / mix["ms"],
                 "rel_fro_err_vs_fp64": max(rel_fro(g, r) for g, r in zip(gots, refs)),
                 "rel_fro_err_per_freq_max": max(rel_fro(got[j], ref[j]) for j in range(nf)),
                 "offdiag_rel_fro_err": max(rel_fro(got[j][offd], ref[j][offd]) for j in range(nf)),
                 "max_entry_err_rel_to_max": float(np.abs(got - ref).max() / np.abs(ref).max()),
                 "error_reference": "the FP64 GPU path (itself within 1e-10 of the CPU oracle)",
                 "tflops": fl["total"] / (mix["ms"] * 1e-3) / 1e12,
                 "stages": mix["stages"], "gpu_launches": mix["gpu_launches"],
                 "tuning": mix["tuning"],
                 "roofline": {"bound": "tensor", "kernel": "k5_gemm", "achieved": gm_ach,
                              "peak": sustained / 3, "unit": "TFLOP/s",
                              "frac": gm_ach / (sustained / 3),
                              "executed_bf16_tflops": executed / (gm_ms * 1e-3) / 1e12,
                              "executed_frac_of_bf16": executed / (gm_ms * 1e-3) / 1e12 / sustained,
                              "traffic": traffic(args.workload, "k5_gemm", kc),
                              "peak_source": f"{src} BF16 sustained {sustained} TFLOP/s / 3 products"}}
        mix["ctx"].close()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(p)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "q-points/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "ms_per_step_eager": head["ms_eager"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64" if args.precision == "fp64" else "f32+bf16x3",
                "data": "synthetic",
                "config": {"workload": desc, "precision": args.precision,
                           "timing": "one captured CUDA graph per step, replayed; stages from an "
                                     "eager profiled pass of the same steps on one stream",
                           "q_points": nq, "pairs_per_q": p.pairs(), "defer_k1": args.defer_k1,
                           "copy_ahead": args.copy_ahead, "overlap": args.overlap,
                           "l2": "inputs larger than L2 (coefficients "
                           f"{sum(c.nbytes for c in p.coeff) / 1e9:.2f} GB, grids resident per step)"},
                "tflops": fl["total"] / (ms * 1e-3) / 1e12,
                "pairs_per_s": value / nq * sum(p.pairs(i) for i in range(nq)),
                "stages": head["stages"],
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "epsinv": epsinv, "unfold": unfold,
                "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
                "tuning": head["tuning"], "fp64_check": check,
                "mixed": other}
        print(json.dumps(line), flush=True)
    head["ctx"].close()
    dist.close()
    return 0


def main():
    if "--alu-peaks" in sys.argv:
        print(json.dumps({"alu_peaks": alu_peaks()}))
        return 0
    args = parse_args()
    world, rank, local = dist_setup()
    if args.impl == "reference":
        return run_reference(args, world, rank)
    return run_ours(args, world, rank, local)


if __name__ == "__main__":
    sys.exit(main())
