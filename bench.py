#!/usr/bin/env python3
"""Benchmark of the spinor polarizability chi0_GG'(q, i w) on GB300.

Default workload (the mixed-precision configuration of the metric): the
GaSb-like cell (FCC a = 11.53 bohr), 32^3 FFT box, ~5000 plane waves per
spinor component, N_G = 800, 6x6x6 k-grid (N_k = 216), N_v = 18, N_c = 400,
16 imaginary frequencies in [0, 40] eV, q = (1/6, 0, 0).  One step = the whole
hot path for one q-point: every k-point's spinor coefficients go to the
real-space grid, every (v, c, k) pair's matrix elements are formed and
contracted into chi0 (FP32 FFTs, complex64 M, split-BF16 x3 tensor-core
contraction, FP64 weights and k reduction), and chi0 is finalised.  The FP64
path runs in the same line on a labelled k-subset (per-k time x N_k), with
the mixed path's error against it and both paths' error against the CPU
oracle on the oracle's timed sample.  Inputs are seeded synthetic states of
that shape (no DFT data).  The Si-like 24^3 case (FP64 and mixed) is reported
beside it.

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
    "gasb32": (dict(config="gasb32"), "GaSb-like FCC a=11.53 bohr, 32^3 box, N_w~5000 per spinor component, "
                                      "N_G=800, N_k=216 (6x6x6), N_v=18, N_c=400, 16 imaginary freqs (0..40 eV), "
                                      "q=(1/6,0,0)"),
    "si24": (dict(config="si24"), "Si-like FCC a=10.26 bohr, 24^3 box, N_w~2000 per spinor component, N_G=350, "
                                  "N_k=64 (4x4x4), N_v=8, N_c=200, 5 imaginary freqs (0..40 eV), q=(1/4,0,0)"),
    # profiling case: the same per-launch shapes on a 2x2x2 k-grid (< 1 GB on the device)
    "si24_small": (dict(config="si24", kgrid=(2, 2, 2), q=(0.5, 0, 0)),
                   "si24 shapes (24^3, N_G=350, N_v=8, N_c=200, 5 freqs) on a 2x2x2 k-grid, q=(1/2,0,0)"),
    # profiling case: the GaSb-like per-launch shapes on a 2x2x2 k-grid (~2 GB on the device)
    "gasb32_small": (dict(config="gasb32", kgrid=(2, 2, 2), q=(0.5, 0, 0)),
                     "gasb32 shapes (32^3, N_G=800, N_v=18, N_c=400, 16 freqs) on a 2x2x2 k-grid, q=(1/2,0,0)"),
    "gasb32_batch": ("batch", "40 q-points of the GaSb-like 6x6x6 grid in one accumulate call: "
                              "32^3 box, N_G(q)~U{700..900}, N_c(q)~U{300..500}, N_v=18, 16 freqs"),
    "bi2se3": ("bi2se3", "Bi2Se3-like rhombohedral cell (hex a=4.143 A, c=28.636 A), 64^3 box, "
                         "N_w~9000 per spinor component, N_G=2000, N_k=216 (6x6x6), N_v=48, N_c=1000, "
                         "8 imaginary freqs, q=(1/6,0,0); real-space grids streamed through 8 slots"),
    "bi2se3_48": ("bi2se3_48", "Bi2Se3-like rhombohedral cell, literal 48^3 box with the largest alias-free "
                               "wavefunction sphere (32.5 Ry, N_w~3000 per spinor component), N_G=2000, "
                               "N_k=216 (6x6x6), N_v=48, N_c=1000, 8 imaginary freqs, q=(1/6,0,0); grids "
                               "streamed through 8 slots"),
    # profiling case: the 64^3 box and N_G = 2000 on a 2x2x2 k-grid with 8 + 40 bands (~1.5 GB)
    "bi2se3_small": ("bi2se3_small", "Bi2Se3-like cell, 64^3 box, N_G=2000, 2x2x2 k-grid, N_v=8, N_c=40, "
                                     "2 freqs, q=(1/2,0,0)"),
}
METRIC = "spinor chi0 q-points/s and TFLOP/s, FP64 vs mixed at ≤2e-5 rel. Frobenius error"

# FP64 issue rate of GB300 derived from its nominal 1.25 TFLOP/s over 152 SMs
# at the 2070 MHz maximum clock: 1.25e12 / (152 * 2.07e9) ~ 4 flop/clk/SM,
# i.e. 2 DFMA per clock per SM.  Peak = 152 * 2 * 2 * 2.07e9.  The roofline
# denominator of FP64 ALU stages is the DGEMM rate measured in the same run.
FP64_PEAK_DERIVED_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12

# FP32 FFMA peak from unit counts and clocks: 152 SMs x 128 lanes x 2 flop x
# 2.07 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12


def parse_args():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=sorted(WORKLOADS), default="gasb32")
    ap.add_argument("--precision", choices=["fp64", "mixed", "tf32x3", "tf32"], default="mixed",
                    help="precision of the headline value (default mixed = split-BF16 x3)")
    ap.add_argument("--no-formats", action="store_true",
                    help="skip the TF32 contraction forms on the FP64 leg's k-subset (mixed headline)")
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-other", action="store_true",
                    help="skip the other precision (FP64 k-subset leg of a mixed headline, or the mixed "
                         "comparison of an FP64 one)")
    ap.add_argument("--no-secondary", action="store_true", help="skip the Si-like 24^3 secondary lines")
    ap.add_argument("--fp64-ks", type=int, default=4, metavar="N",
                    help="FP64 leg of a mixed headline: k-points 0..N-1 and the first N k-points with an "
                         "umklapp (k+q = k'+G0, G0 != 0)")
    ap.add_argument("--fp64-dfma", action="store_true",
                    help="FP64 path: contract on the FP64 pipe (FMA kernel) instead of the tensor cores")
    ap.add_argument("--no-autotune", action="store_true", help="default tiles and k-chunk")
    ap.add_argument("--grid-slots", type=int, default=-1,
                    help="real-space grid slots (0 = all k resident; default 8 for bi2se3, else 0)")
    ap.add_argument("--kchunk", type=int, default=0, help="k-chunk when not autotuning")
    ap.add_argument("--pair-tile", type=int, nargs=2, default=None, metavar=("TV", "TC"),
                    help="pair tile of the FP32 matrix-element kernel when not autotuning")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the hot path only: no eps^-1/W, unfolding, e2e, other precision, CPU baseline or "
                         "secondary workload (for profiler launch lists)")
    ap.add_argument("--k1-path", type=int, default=0, choices=[0, 1, 2, 3, 4],
                    help="sphere -> grid kernels: 0 automatic, 1 per axis, 2 one kernel per band component, "
                         "3 eight lanes per line (cubic 32/40/48/64), 4 one kernel without the shared cube")
    ap.add_argument("--mtxel-zy", type=int, default=0, choices=[0, 1, 2],
                    help="FP32 pair density + z + y kernel: 0 automatic, 1 plane kernel, 2 streamed")
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
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="DRAM bytes (read + write) per launch of the dominant kernel from an ncu capture of "
                         "this configuration and the current sources; without it roofline.traffic is null")
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


def dgemm_tflops(n=8192, reps=3):
    """cuBLAS FP64 GEMM rate (torch.matmul, n^3, CUDA events, median of
    `reps` after one warm-up): the measured ceiling of FP64 ALU stages."""
    import torch
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = torch.empty(n, n, dtype=torch.float64, device="cuda")
    ts = []
    for i in range(reps + 1):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        torch.cuda.synchronize()
        if i:
            ts.append(e0.elapsed_time(e1))
    del a, b, c
    return 2 * n ** 3 / (statistics.median(ts) * 1e-3) / 1e12


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
    out["total"] = out["wfn_to_grid"] + out["mtxel"] + out["mtxel_x"] + out["contraction"]
    return out


def flop_model_q(p, iq=0):
    """Algorithmic FLOPs of one q-point: pruned radix FFTs (5 L log2 L per
    line of length L), the pair density (8 flops per point and spin
    component) and the Hermitian contraction (8 flops per complex MAC over
    N_G(N_G+1)/2 entries per pair and frequency).  The matrix elements are
    split as profiled: "mtxel" the pair density with the z and y passes,
    "mtxel_x" the x pass (its sphere gather moves data only)."""
    q, geps, nc = p.qs[iq]
    n = np.array(p.box, float)
    L = float(np.log2(n[0]))
    w = geps.max(0) - geps.min(0) + 1
    per_pair_zy = 5 * n[0] * L * (n[0] * n[1] + n[0] * w[1])
    per_pair_x = 5 * n[0] * L * w[1] * w[2]
    per_pair_rho = 8 * 2 * np.prod(n)
    pairs = p.nk * p.nv * nc
    band_fft = 0.0
    for ik in range(p.nk):
        ws = p.gvec[ik].max(0) - p.gvec[ik].min(0) + 1
        band_fft += 2 * p.nbands * 5 * n[0] * L * (ws[1] * ws[2] + n[0] * ws[2] + n[0] * n[1])
    ng = len(geps)
    herk = 8.0 * pairs * len(p.freq) * ng * (ng + 1) / 2
    zy = pairs * (per_pair_zy + per_pair_rho)
    x = pairs * per_pair_x
    return {"wfn_to_grid": band_fft, "mtxel": zy, "mtxel_x": x, "contraction": herk,
            "total": band_fft + zy + x + herk}


def byte_model(p, csize):
    """Least DRAM bytes of the FFT stages in one step (every q-point): the
    sphere -> grid transform reads each band's coefficients (complex128) and
    writes its grid once; the matrix elements read the grids of the valence
    bands at k and the conduction bands at k+q once (z and y passes) and
    write M once (x pass); csize bytes per complex value of the path's
    precision."""
    vol = float(np.prod(p.box))
    coeff = sum(p.nbands * 2 * len(g) * 16.0 for g in p.gvec)
    grids = p.nk * p.nbands * 2 * vol * csize
    mtxel, mx = 0.0, 0.0
    for q, geps, nc in p.qs:
        mtxel += p.nk * (p.nv + nc) * 2 * vol * csize
        mx += p.nk * p.nv * nc * len(geps) * csize
    return {"wfn_to_grid": coeff + grids, "mtxel": mtxel, "mtxel_x": mx}


# ---------------------------------------------------------------- oracle --

def umklapp_ks(p, iq=0):
    """k-points whose k + q leaves the grid's unit cell (k + q = k' + G0 with
    G0 != 0), in index order."""
    q = np.asarray(p.qs[iq][0], float)
    t = np.asarray(p.kcrys, float) + q[None, :]
    return [int(i) for i in np.nonzero((np.floor(t + 1e-9) != 0).any(1))[0]]


def sample_nc(p, flop_target=5e10):
    """Conduction bands of the oracle's per-k sample: all valence bands and as
    many conduction bands as keep one k-point near `flop_target` flops of
    convolution (8 per complex MAC over both spinor components of the sphere
    per G) and contraction (8 per complex MAC per frequency)."""
    q, geps, nc = p.qs[0]
    ngw = float(np.mean([len(g) for g in p.gvec]))
    per_pair = len(geps) * 2 * ngw * 8 + len(p.freq) * len(geps) ** 2 * 8
    return int(max(1, min(nc, round(flop_target / per_pair / p.nv))))


def with_partners(p, ks):
    """ks and the grid index of each k + q."""
    q = np.asarray(p.qs[0][0], float)
    need = set(ks)
    for ik in ks:
        t = np.asarray(p.kcrys[ik]) + q
        d = np.asarray(p.kcrys) - (t - np.floor(t + 1e-9))[None, :]
        need.add(int(np.argmin(np.abs(d - np.round(d)).sum(1))))
    return sorted(need)


def host_problem(p, ks):
    """A copy of problem p holding only the coefficients of ks and their
    k + q partners, as numpy arrays (device tensors are copied to the host,
    missing ones generated on the host); every other k's are None."""
    import copy
    h = copy.copy(p)
    need = with_partners(p, ks)
    h.coeff = [None] * p.nk
    for ik in need:
        c = p.coeff[ik]
        if c is None:
            from paper_2206_00808_gb300 import synthetic as syn
            syn.fill_coefficients(h, [ik], on="host")
        else:
            h.coeff[ik] = c if isinstance(c, np.ndarray) else c.cpu().numpy()
    return h


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
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
    import platform
    return platform.machine()


def host_threads():
    """Threads the oracle's OpenMP loops use: OMP_NUM_THREADS, else the CPUs
    this process may run on."""
    if os.environ.get("OMP_NUM_THREADS"):
        return int(os.environ["OMP_NUM_THREADS"])
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


_SINGLE_THREAD = r"""
import sys, time, numpy as np
sys.path.insert(0, sys.argv[1])
import oracle
from paper_2206_00808_gb300 import synthetic as syn
d = np.load(sys.argv[2], allow_pickle=True)
p = d["problem"].item()
oracle.build()
t0 = time.perf_counter()
oracle.chi0(p, k_indices=[int(d["k"])], nc=int(d["nc"]))
print(time.perf_counter() - t0)
"""


def cpu_baseline(p, with_single_thread=True):
    """The oracle as it stands on the host cores: all N_v valence bands and a
    sample of conduction bands at k = 0 and at the first umklapp k-point, all
    G and frequencies; q-points/s scaled by (N_k / 2) x (N_c / sample).  Also
    a single-thread run of one k-point with an eighth of that sample.
    Returns (baseline dict, sampled chi0, sample)."""
    import oracle
    oracle.build()
    ks = [0, umklapp_ks(p)[0]]
    ncs = sample_nc(p)
    hp = host_problem(p, ks)
    t0 = time.perf_counter()
    chi = oracle.chi0(hp, k_indices=ks, nc=ncs)
    dt = time.perf_counter() - t0
    nc = p.qs[0][2]
    scale = (p.nk / len(ks)) * (nc / ncs)
    out = {"value": 1.0 / (dt * scale), "unit": "q-points/s", "cores": host_threads(), "kind": "oracle",
           "cpu_model": cpu_model(),
           "sample": f"k-points {ks} of {p.nk} (the second with an umklapp G0) x all {p.nv} valence x "
                     f"{ncs} of {nc} conduction bands, N_G={len(p.qs[0][1])}, {len(p.freq)} freqs: "
                     f"{dt:.1f} s, scaled x{scale:.0f}"}
    if with_single_thread:
        import tempfile
        nc1 = max(1, ncs // 8)
        sub = host_problem(hp, ks[:1])
        with tempfile.TemporaryDirectory() as td:
            path = os.path.join(td, "sample.npz")
            np.savez(path, problem=np.array(sub, dtype=object), k=ks[0], nc=nc1)
            env = dict(os.environ, OMP_NUM_THREADS="1")
            r = subprocess.run([sys.executable, "-c", _SINGLE_THREAD, ROOT, path], capture_output=True,
                               text=True, env=env, timeout=600)
        if r.returncode == 0:
            t1 = float(r.stdout.strip().splitlines()[-1])
            sc1 = p.nk * (nc / nc1)
            out["single_thread"] = {"value": 1.0 / (t1 * sc1), "unit": "q-points/s", "cores": 1,
                                    "sample": f"k-point {ks[0]} x all {p.nv} valence x {nc1} conduction bands: "
                                              f"{t1:.1f} s, scaled x{sc1:.0f}"}
        else:
            out["single_thread"] = {"error": r.stderr[-300:]}
    return out, chi, {"ks": ks, "nc": ncs}


# ------------------------------------------------------------------ arms --

def make_workload(name, coeff_on="cuda"):
    """(problem, description); coefficients made on the device ("cuda"), on
    the host ("host"), or left for fill_coefficients (None)."""
    from paper_2206_00808_gb300 import synthetic as syn
    over, desc = WORKLOADS[name]
    if over == "batch":
        return syn.make_batched_problem(), desc
    if over == "bi2se3":
        return syn.make_bi2se3_problem(device=coeff_on), desc
    if over == "bi2se3_48":
        return syn.make_bi2se3_problem(box=(48, 48, 48), ecut_wfn=32.5, device=coeff_on), desc
    if over == "bi2se3_small":
        # generated on the host (torch CPU QR): profilers run this case, and the
        # device QR's lazily loaded library is not found under them
        p = syn.make_bi2se3_problem(kgrid=(2, 2, 2), nv=8, nc=40, q=(0.5, 0, 0), nfreq=2, device="cpu")
        p.coeff = [c.numpy() for c in p.coeff]
        return p, desc
    over = dict(over)
    if name.endswith("_small") and coeff_on is not None:
        coeff_on = "host"      # profilers run these; the device QR's lazily loaded library is not found under them
    return syn.make_problem(over.pop("config"), coeff_on=coeff_on, **over), desc


def run_reference(args, world, rank):
    """The oracle as it stands, timed on the host cores on this arm's
    workload and metric: each step one k-point (k = 0 and the first umklapp
    k-point in turn) with all valence bands and a quarter of the cpu_baseline
    sample of conduction bands, scaled to one q-point."""
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    p, desc = make_workload(args.workload, coeff_on=None)
    ks = [0, umklapp_ks(p)[0]]
    hp = host_problem(p, ks)
    nc = p.qs[0][2]
    ncs = max(1, sample_nc(p) // 4)
    scale = p.nk * (nc / ncs)

    def one(i):
        t0 = time.perf_counter()
        oracle.chi0(hp, k_indices=[ks[i % 2]], nc=ncs)
        return time.perf_counter() - t0

    for i in range(args.warmup):
        one(i)
    times = [one(i) * scale for i in range(args.steps)]
    ms = 1e3 * statistics.mean(times)
    value = 1e3 / ms
    cores = host_threads()
    line = {"metric": METRIC, "value": value, "unit": "q-points/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": desc, "precision": "fp64 (CPU oracle)"},
            "cpu_baseline": {"value": value, "unit": "q-points/s", "cores": cores, "kind": "oracle",
                             "cpu_model": cpu_model(),
                             "sample": f"each step: k-point {ks[0]} or {ks[1]} of {p.nk} x all {p.nv} valence x "
                                       f"{ncs} of {nc} conduction bands, all G and freqs, scaled x{scale:.0f}"},
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
    if args.pair_tile:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_PAIR_TILE_V, args.pair_tile[0])
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_PAIR_TILE_C, args.pair_tile[1])
    if args.k1_path > 0:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_K1_PATH, args.k1_path)
    if args.mtxel_lanes > 0:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_MTXEL_LANES, args.mtxel_lanes)
    if args.mtxel_zy > 0:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_MTXEL_ZY, args.mtxel_zy)
    if args.defer_k1:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_DEFER_K1, 1)
    if args.copy_ahead:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_COPY_AHEAD, 1)
    if args.overlap and precision != "fp64":
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_OVERLAP, 1)
    if precision == "fp64" and args.fp64_dfma:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_FP64_CONTRACTION, 1)
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
    ovl = args.overlap and precision != "fp64"
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
    f64 = (args.fp64_peak, args.fp64_peak_label)
    f64c = f64 if args.fp64_dfma else (sustained / 15, "BF16 sustained / 15 digit products")
    peaks = ({"wfn_to_grid": f64, "mtxel": f64, "mtxel_x": f64, "contraction": f64c}
             if precision == "fp64" else
             {"wfn_to_grid": (FP32_PEAK_TFLOPS, "FP32 ALU (derived)"),
              "mtxel": (FP32_PEAK_TFLOPS, "FP32 ALU (derived)"),
              "mtxel_x": (FP32_PEAK_TFLOPS, "FP32 ALU (derived)"),
              "contraction": contraction_peak(precision, sustained, "")})
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


def epsinv_measure(B, torch, p, res, stream, fp64_peak, reps=3):
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
            "peak_tflops": fp64_peak, "peak": "FP64 DGEMM (measured in this run)",
            "roofline_frac": tf / fp64_peak, "derived_fp64_peak_tflops": FP64_PEAK_DERIVED_TFLOPS}


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
    nb = min(16384, sum(int(c.shape[0]) for c, _ in dev_in))
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
    dfma_peak = FP64_PEAK_DERIVED_TFLOPS * 1e12 / 2      # DFMA instructions per second
    del cin, cout
    return {"what": "c(G) -> U c(R^-1 G) e^{-iG.tau} (FP64), one launch over the bands of the step's "
                    "k-points (at most 16384) on the sphere of k-point 0",
            "bands": nb, "plane_waves": ngw, "bytes": nbytes, "ms": ms, "gbs": gbs, "peak_gbs": hbm,
            "hbm_frac": gbs / hbm if hbm else None,
            "fp64_fma_per_s": dfma / (ms * 1e-3), "fp64_frac": dfma / (ms * 1e-3) / dfma_peak,
            "bound": "alu (FP64): 16 DFMA per 64 bytes outruns the DRAM time on this part"}


def e2e_measure(B, torch, p, res, args, dist, stream):
    """Same step from pinned host buffers, chi0 read back to host."""
    ctx = res["ctx"]
    q, geps, nc = p.qs[0]
    ng, nf = len(geps), len(p.freq)
    def pinned(x):
        # a user's inputs arrive from host memory (files): fill the pinned
        # buffers by a host copy.  (Pinned buffers last written by a
        # device-to-host copy were read back by host-to-device copies at about a
        # third of the rate on GB300's coherent host memory: 300 vs 70 ms for
        # the same 14.7 GB.)
        t = x.cpu() if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x))
        return torch.empty(t.shape, dtype=t.dtype, pin_memory=True).copy_(t)

    pin = [(pinned(p.coeff[ik]), pinned(p.energy[ik])) for ik in range(p.nk)]
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


def error_stats(got, ref):
    """Relative Frobenius error overall and per frequency, the off-diagonal
    part's, and the largest entry error relative to the largest entry."""
    nf, ng = ref.shape[0], ref.shape[1]
    offd = ~np.eye(ng, dtype=bool)
    per = [rel_fro(got[j], ref[j]) for j in range(nf)]
    return {"rel_fro": rel_fro(got, ref), "rel_fro_per_freq": per, "rel_fro_per_freq_max": max(per),
            "offdiag_rel_fro_max": max(rel_fro(got[j][offd], ref[j][offd]) for j in range(nf)),
            "max_entry_err_rel_to_max": float(np.abs(got - ref).max() / np.abs(ref).max())}


def k_runs(ks):
    """Contiguous [a, b) runs of a sorted k list."""
    out = []
    for k in ks:
        if out and out[-1][1] == k:
            out[-1][1] = k + 1
        else:
            out.append([k, k + 1])
    return [tuple(r) for r in out]


def chi0_on(B, ctx, qlist, freq, ks):
    """A new running sum over k-points ks on a context; chi0 of the first q (host)."""
    B.bgw_chi0_reset(ctx.ctx)
    for a, b in k_runs(sorted(ks)):
        B.bgw_chi0_accumulate(ctx.ctx, qlist, freq, a, b)
    ng = len(qlist[0][1])
    out = np.zeros((len(freq), ng, ng), dtype=np.complex128)
    B.bgw_chi0_finalize(ctx.ctx, 0, out)
    return out


def subset_leg(B, torch, p, args, stream, dev_in, ks, prec="fp64", kchunk=None, reps=2):
    """One precision (FP64 by default) on k-points ks of the workload: every
    run re-uploads the k-points it reads (so each includes the sphere-to-grid
    transforms of ks and of their k + q partners), accumulates ks and
    finalises to the device.  Grids live in a few streaming slots, not all
    N_k.  CUDA events on the stream, one warm-up run, median of `reps`."""
    need = with_partners(p, ks)
    ctx = B.Chi0Context(p, prec, stream)
    if len(need) + 2 < p.nk:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_GRID_SLOTS, len(need) + 2)
    B.bgw_set_option(ctx.ctx, B.BGW_OPT_KCHUNK, kchunk or (args.kchunk if args.kchunk > 0 else 4))
    if prec == "fp64" and args.fp64_dfma:
        B.bgw_set_option(ctx.ctx, B.BGW_OPT_FP64_CONTRACTION, 1)
    ctx.upload(device_inputs=dev_in)
    q, geps, nc = p.qs[0]
    ng, nf = len(geps), len(p.freq)
    out = torch.empty((nf, ng, ng), dtype=torch.complex128, device="cuda")

    def run():
        ctx.upload(device_inputs=dev_in, ks=need)
        B.bgw_chi0_reset(ctx.ctx)
        for a, b in k_runs(sorted(ks)):
            ctx.accumulate(a, b)
        B.bgw_chi0_finalize(ctx.ctx, 0, out)

    run()
    times = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        run()
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    B.bgw_profile(ctx.ctx, True)
    run()
    prof = B.bgw_profile_read(ctx.ctx)
    B.bgw_profile(ctx.ctx, False)
    stages = {k: v[0] / len(ks) for k, v in prof.items() if v[1]}
    return ctx, out.cpu().numpy(), ms / len(ks), stages


TF32_PER_BF16 = 1.1 / 2.25      # nominal dense TF32 / BF16 tensor rates of GB300


def contraction_peak(precision, sustained, src):
    """Ceiling of the mixed contraction in algorithmic FLOP/s: the measured
    sustained BF16 rate over the products per term, scaled by the nominal
    TF32/BF16 ratio for the TF32 forms (no TF32 rate is measured)."""
    if precision == "tf32x3":
        return (sustained * TF32_PER_BF16 / 3,
                f"{src} BF16 sustained {sustained} TFLOP/s x nominal TF32/BF16 1.1/2.25 / 3 products".strip())
    if precision == "tf32":
        return (sustained * TF32_PER_BF16,
                f"{src} BF16 sustained {sustained} TFLOP/s x nominal TF32/BF16 1.1/2.25, 1 product".strip())
    return sustained / 3, f"{src} BF16 sustained {sustained} TFLOP/s / 3 products".strip()


DTYPES = {"fp64": "f64", "mixed": "f32+bf16x3", "tf32x3": "f32+tf32x3", "tf32": "f32+tf32"}


def format_legs(B, torch, p, args, stream, dev_in, ks, head, chi64):
    """The contraction forms of the FP32 path (split-BF16 x3, split-TF32 x3,
    one TF32 product) on the FP64 leg's k-subset at the headline's k-chunk:
    per-k contraction time (the profiled stage, k5_split + k5_gemm) and the
    error against the FP64 GPU path on the same k-points."""
    kc = max(1, B.bgw_get_option(head["ctx"].ctx, B.BGW_OPT_KCHUNK))
    _, sustained, src = bf16_peaks()
    fl = flop_model(p)["contraction"] / p.nk
    out = {"k_subset": ks, "kchunk": kc}
    for prec in ("mixed", "tf32x3", "tf32"):
        ctx, chi, per_k, st = subset_leg(B, torch, p, args, stream, dev_in, ks, prec, kchunk=kc)
        ctx.close()
        ct = st.get("contraction", 0.0) + st.get("operand_split", 0.0)
        pk, lab = contraction_peak(prec, sustained, src)
        out[DTYPES[prec]] = {"ms_per_k": per_k, "contraction_ms_per_k": ct,
                             "gemm_ms_per_k": st.get("contraction", 0.0),
                             "gemm_tflops": fl / max(1e-9, st.get("contraction", 0.0) * 1e-3) / 1e12,
                             "gemm_peak": pk, "peak_source": lab,
                             "vs_fp64_on_subset": error_stats(chi, chi64)}
    return out


def nq_of(p):
    return len(p.qs)


def zy_kernel_name(p, precision, zy):
    """The kernel of the pair density + z + y stage for this box and choice
    (the library's rule: FP64 separate passes; eight lanes per line on cubic
    48^3/64^3; else the streamed kernel on even boxes up to 32 unless the
    plane kernel was chosen)."""
    n = p.box[1]
    if precision == "fp64":
        return "k2_zpass + k2_ypass (FP64)"
    if p.box[0] == p.box[1] == p.box[2] and n in (48, 64):
        return "k2_zy_oct"
    if zy != 1 and n % 2 == 0 and n <= 32 and n not in (22, 26, 28):
        return "k2_zy_stream"
    return "k2_zy_plane"


# Per-launch DRAM bytes (read + write) of a kernel, from one ncu capture of
# the same launch shape: kernel, workload shapes, precision, k-chunk and the
# SHA-256 prefix of the kernel's source file when it was captured (any later
# edit of that file voids the figure).  k5_gemm: the GaSb-like shapes, one
# k-chunk of 2 (14,400 pairs, 1456 work items): 2.972 GB read, 0.086 GB written.
CAPTURED_TRAFFIC = {
    ("k5_gemm", "gasb32", "mixed", 2): ("paper_2206_00808_gb300/csrc/bgw_chi0_mixed.cu", "5e421338b6571e70",
                                        2.971712e9 + 0.086362624e9),
}


def captured_traffic(kernel, workload, precision, kchunk):
    """(bytes per launch, None) for a captured configuration whose kernel
    source is unchanged, else (None, reason)."""
    import hashlib
    hit = CAPTURED_TRAFFIC.get((kernel, workload, precision, kchunk))
    if hit is None:
        return None, (f"null: no ncu capture of {kernel} at this launch shape ({workload}, {precision}, "
                      f"k-chunk {kchunk}); pass --traffic-bytes")
    path, digest, nbytes = hit
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), path), "rb") as f:
            now = hashlib.sha256(f.read()).hexdigest()[:16]
    except OSError:
        now = None
    if now != digest:
        return None, f"null: {path} changed since the capture of {kernel}"
    return nbytes, None


def gemm_operand_bytes(p, kchunk):
    """Algorithmic operand bytes of one split-BF16 contraction launch: the
    X and w_j X planes, hi and lo, 2 B each, rows padded to 128 and pairs to
    64, every plane read once."""
    q, geps, nc = p.qs[0]
    rows = -(-2 * len(geps) // 128) * 128
    pairs = -(-kchunk * p.nv * nc // 64) * 64
    return 2 * (1 + len(p.freq)) * rows * pairs * 2


def head_roofline(p, res, precision, args, steps):
    """Roofline of the dominant kernel of the headline: the contraction
    GEMM or the pair density + z + y kernel of the matrix elements (their x
    pass is profiled apart), whichever takes longer; achieved = algorithmic
    FLOPs of the profiled steps over that kernel's summed device time."""
    fl = flop_model(p)
    burst, sustained, src = bf16_peaks()
    st = res["stages"]
    mt = st.get("mtxel", {}).get("ms_per_step", 0.0)
    ct = st.get("contraction", {}).get("ms_per_step", 0.0)
    traffic = args.traffic_bytes
    note = None if traffic else ("null: per-launch DRAM bytes come from an ncu capture of this configuration "
                                 "and these sources (pass --traffic-bytes); none is taken by the timed run")
    kchunk = (res.get("tuning") or {}).get("kchunk") or args.kchunk
    if ct >= mt and not traffic and precision == "mixed" and nq_of(p) == 1:
        traffic, why = captured_traffic("k5_gemm", args.workload, precision, kchunk)
        note = why or (f"from an ncu capture of the same launch shape (k-chunk {kchunk}); algorithmic operand "
                       f"bytes per launch {gemm_operand_bytes(p, kchunk):.4g}")
    if ct >= mt:
        ach = fl["contraction"] / (ct * 1e-3) / 1e12
        if precision == "fp64" and args.fp64_dfma:
            r = {"bound": "alu", "kernel": "k4_herk_f64", "achieved": ach, "peak": args.fp64_peak,
                 "unit": "TFLOP/s", "frac": ach / args.fp64_peak,
                 "peak_source": args.fp64_peak_label,
                 "derived_fp64_peak_tflops": FP64_PEAK_DERIVED_TFLOPS}
        elif precision == "fp64":
            r = {"bound": "tensor", "kernel": "k5z_gemm (with its exponent and digit-split passes)",
                 "achieved": ach, "peak": sustained / 15, "unit": "TFLOP/s", "frac": ach / (sustained / 15),
                 "peak_source": f"{src} BF16 sustained {sustained} TFLOP/s / 15 digit products"}
        else:
            pk, lab = contraction_peak(precision, sustained, src)
            r = {"bound": "tensor", "kernel": "k5_gemm", "achieved": ach, "peak": pk,
                 "unit": "TFLOP/s", "frac": ach / pk, "peak_source": lab}
    else:
        ach = fl["mtxel"] / (mt * 1e-3) / 1e12
        pk = args.fp64_peak if precision == "fp64" else FP32_PEAK_TFLOPS
        kern = zy_kernel_name(p, precision, (res.get("tuning") or {}).get("mtxel_zy", args.mtxel_zy))
        r = {"bound": "alu", "kernel": kern + " (pair density + pruned z and y FFT passes)",
             "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
             "peak_source": (args.fp64_peak_label if precision == "fp64" else
                             "FP32 FFMA from unit counts: 152 SMs x 128 lanes x 2 flop x 2.07 GHz")}
    r["traffic"] = traffic
    if note:
        r["traffic_note"] = note
    return r


def secondary(B, torch, args, dist, stream, local, name="si24"):
    """A smaller workload in both precisions (5 steps after 3 warm-ups each):
    q-points/s, the mixed/FP64 speedup and the mixed error against FP64."""
    import copy
    p, desc = make_workload(name, coeff_on="cuda")
    dev_in = [(p.coeff[ik], torch.from_numpy(np.ascontiguousarray(p.energy[ik])).cuda())
              for ik in range(p.nk)]
    a2 = copy.copy(args)
    a2.steps, a2.warmup, a2.grid_slots = 5, 3, 0
    f = measure(B, torch, p, "fp64", a2, dist, stream, dev_in, local, False)
    ref = [o.cpu().numpy() for o in f["outs"]]
    f["ctx"].close()
    m = measure(B, torch, p, "mixed", a2, dist, stream, dev_in, local, False)
    got = [o.cpu().numpy() for o in m["outs"]]
    m["ctx"].close()
    nq = len(p.qs)
    return {"workload": desc,
            "fp64": {"value": nq * 1e3 / f["ms"], "unit": "q-points/s", "ms_per_step": f["ms"],
                     "stages": {k: v["ms_per_step"] for k, v in f["stages"].items()}},
            "mixed": {"value": nq * 1e3 / m["ms"], "unit": "q-points/s", "ms_per_step": m["ms"],
                      "stages": {k: v["ms_per_step"] for k, v in m["stages"].items()}, "tuning": m["tuning"]},
            "speedup_mixed_vs_fp64": f["ms"] / m["ms"],
            "mixed_vs_fp64": error_stats(got[0], ref[0])}


def run_ours(args, world, rank, local):
    import torch
    torch.cuda.set_device(local)
    dist = Dist(world, rank, "nccl")
    from paper_2206_00808_gb300 import build
    build.build()
    from paper_2206_00808_gb300 import binding as B

    if args.no_extras:
        args.no_e2e = args.no_other = args.no_cpu_baseline = args.no_secondary = True
    args.fp64_peak = dgemm_tflops() if not args.no_extras else FP64_PEAK_DERIVED_TFLOPS
    args.fp64_peak_label = ("FP64 DGEMM (measured in this run)" if not args.no_extras else
                            "FP64 from unit counts: 152 SMs x 2 DFMA/clk x 2 flop x 2.07 GHz")
    p, desc = make_workload(args.workload, coeff_on="cuda")
    if args.grid_slots < 0:
        args.grid_slots = 8 if args.workload in ("bi2se3", "bi2se3_48") else 0
    q, geps, nc = p.qs[0]
    ng, nf = len(geps), len(p.freq)
    stream = torch.cuda.Stream()      # graph capture needs a non-default stream

    def dev(x):
        return x if isinstance(x, torch.Tensor) else torch.from_numpy(np.ascontiguousarray(x)).cuda()

    dev_in = [(dev(p.coeff[ik]), dev(p.energy[ik])) for ik in range(p.nk)]
    fl = flop_model(p)
    steps = args.steps
    nq = len(p.qs)
    other_prec = "mixed" if args.precision == "fp64" else "fp64"

    head = measure(B, torch, p, args.precision, args, dist, stream, dev_in, local, True)
    ms = head["ms"]
    value = world * nq * 1e3 / ms
    roofline = head_roofline(p, head, args.precision, args, steps)
    epsinv = None if args.no_extras else epsinv_measure(B, torch, p, head, stream, args.fp64_peak)
    unfold = None if args.no_extras else unfold_measure(B, torch, p, dev_in, stream)
    e2e = None if args.no_e2e else e2e_measure(B, torch, p, head, args, dist, stream)

    # the other precision: FP64 on a labelled k-subset (mixed headline), or
    # the whole mixed step (FP64 headline)
    other, octx = None, None
    if not args.no_other and nq == 1:
        if args.precision != "fp64":
            n = min(args.fp64_ks, p.nk)
            umk = umklapp_ks(p)
            ks = sorted(set(range(n)) | set(umk[:n]))
            octx, chi64, per_k, st64 = subset_leg(B, torch, p, args, stream, dev_in, ks)
            chimx = chi0_on(B, head["ctx"], [(q, geps, nc)], p.freq, ks)
            ms64 = per_k * p.nk
            other = {"precision": "fp64 (FP64 grids, FFTs, M and contraction)",
                     "k_subset": ks, "k_subset_note": f"k = 0..{n - 1} and the first {n} k-points with an "
                                                      "umklapp; per-k time x N_k",
                     "contraction": "FP64 FMA kernel" if args.fp64_dfma else
                                    "tensor cores, exact BF16 digit slices (FP64 accuracy)",
                     "ms_per_k": per_k, "ms_per_q_extrapolated": ms64,
                     "stage_ms_per_k": st64,
                     "value": world * 1e3 / ms64, "unit": "q-points/s (extrapolated from the k-subset)",
                     "speedup_mixed_vs_fp64": ms64 / ms,
                     "mixed_vs_fp64_on_subset": error_stats(chimx, chi64),
                     "error_reference": "the FP64 GPU path on the same k-subset"}
            if not args.no_formats:
                other["contraction_formats"] = format_legs(B, torch, p, args, stream, dev_in, ks, head, chi64)
        else:
            mix = measure(B, torch, p, "mixed", args, dist, stream, dev_in, local, False)
            ref = head["outs"][0].cpu().numpy()
            got = mix["outs"][0].cpu().numpy()
            other = {"precision": "mixed (FP32 grids/FFT, complex64 M, split-BF16 x3 tcgen05, "
                                  "FP64 weights and k-reduction)",
                     "value": world * nq * 1e3 / mix["ms"], "unit": "q-points/s", "ms_per_step": mix["ms"],
                     "speedup_mixed_vs_fp64": ms / mix["ms"],
                     "mixed_vs_fp64": error_stats(got, ref),
                     "stages": mix["stages"], "tuning": mix["tuning"],
                     "roofline": head_roofline(p, mix, "mixed", args, steps)}
            octx = mix["ctx"]

    cpu, oracle_check = None, None
    if rank == 0 and world == 1 and not args.no_cpu_baseline and nq == 1:
        cpu, chis, smp = cpu_baseline(p)
        ql = [(q, geps, smp["nc"])]
        oracle_check = {"sample": f"k-points {smp['ks']}, all {p.nv} valence x {smp['nc']} conduction bands, "
                                  f"all {ng} G and {nf} freqs (the cpu_baseline run)"}
        for prec, cx in ((args.precision, head["ctx"]), (other_prec, octx)):
            if cx is not None:
                oracle_check[prec] = error_stats(chi0_on(B, cx, ql, p.freq, smp["ks"]), chis)
    if octx is not None:
        octx.close()

    sec = None
    if rank == 0 and not args.no_secondary and args.workload != "si24":
        head["ctx"].close()
        head["ctx"] = None
        sec = secondary(B, torch, args, dist, stream, local)

    if rank == 0:
        coeff_gb = sum(c.numel() * c.element_size() for c, _ in dev_in) / 1e9
        line = {"metric": METRIC, "value": value, "unit": "q-points/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "ms_per_step_eager": head["ms_eager"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPES[args.precision],
                "data": "synthetic",
                "config": {"workload": desc, "precision": args.precision,
                           "timing": "one captured CUDA graph per step, replayed; stages from an "
                                     "eager profiled pass of the same steps on one stream",
                           "q_points": nq, "pairs_per_q": p.pairs(), "defer_k1": args.defer_k1,
                           "copy_ahead": args.copy_ahead, "overlap": args.overlap,
                           "l2": f"inputs larger than L2 (coefficients {coeff_gb:.2f} GB, grids resident "
                                 "per step)"},
                "tflops": fl["total"] / (ms * 1e-3) / 1e12,
                "pairs_per_s": value / nq * sum(p.pairs(i) for i in range(nq)),
                "stages": head["stages"],
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": head["gpu_launches"], "clocks": head["clocks"],
                "tuning": head["tuning"], "fp64_dgemm_tflops": args.fp64_peak,
                "other_precision": other, "oracle_check": oracle_check,
                "epsinv": epsinv, "unfold": unfold, "secondary": sec}
        print(json.dumps(line), flush=True)
    if head["ctx"] is not None:
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
