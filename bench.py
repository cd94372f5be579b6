"""Throughput of the 2-D PIC space-charge step on one GB300.

Metric: particle-SC-kicks/s = particles x space-charge kicks / time, one kick
being deposit + open-boundary solve + gather/kick + push to the next
space-charge location.  Workload (default): 1e6 macroparticles, 128x128 grid
(256x256 padded), the synthetic 72-cell FODO ring with 216 kicks per turn.
One bench step = one turn (216 kicks) through sc_track_turns.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|tf32x3]
  python bench.py --impl reference      # the FP64 CPU oracle, bounded sample

Prints ONE JSON line on rank 0.
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
sys.path.insert(0, ROOT)

METRIC = "particle-SC-kicks/s at 1e6 particles,128² grid; batched split-TF32 vs plain FP64"
UNIT = "particle-kicks/s"
WORKLOAD = ("c2: 1e6 macroparticles (4D Gaussian, sigma_x=4 mm, sigma_y=3 mm, 0.2 mrad, 4-sigma cut), "
            "128x128 grid over +-5 sigma (256x256 padded open-boundary solve), 72-cell FODO ring with "
            "2 thin-sextupole families, bare tunes (22.40, 20.75), 216 SC kicks/turn")
WORKLOADS = {
    "c1": "c1: 2e4 macroparticles (sigma 2 mm), 64x64 grid, 24-cell FODO ring, 48 SC kicks/turn",
    "c2": WORKLOAD,
    "c3": "c3: 4e6 macroparticles, 256x256 grid (512x512 padded), the c2 ring, 216 SC kicks/turn",
    "c4": ("c4: 64 independent bunches, counts log-uniform 1e4-2e6 (2.37e7 total), grids 64^2/128^2/256^2 by "
           "count, 8x8 working points of the c2 ring, 216 SC kicks/turn"),
    "c5": ("c5: 1e7 macroparticles, Gaussian bunch sigma_z = 15 m cut at 4 sigma_z, sorted by sigma, 32 slices "
           "over +-4 sigma_z each with its own 128x128 grid, 1e13 protons, the c2 ring, 216 SC kicks/turn"),
}

# FP64-pipe thread instructions per particle in kick_push_kernel (the turn
# graph's variant), by segment content, from ncu's
# sm__thread_inst_executed_pipe_fp64_pred_on per launch on the three segment
# types of the bench ring (1e6 particles), fitted to the segments' element mix
# (profiles/kick_push_c2.md gives the per-segment counts and the commands);
# base = gather + kick + fused deposit.  The quadrupole reads its matrix
# entries from the per-particle family cache (51.0 when it computes them).
# The counts belong to the kernel sources whose SHA-256 (first 16 hex digits)
# is FP64_INST_SOURCES_SHA (the three segment types measured on them: 55.8,
# 68.0 and 18.0, mean 47.2 per particle-kick, the model's own figure); the
# bench reports whether the sources still match.
FP64_INST = {"base": 17.5, "drift": 12.2, "quad": 20.6, "sext": 5.0, "bend": 16.0, "rf": 30.0}
FP64_INST_QUAD_UNCACHED = 51.0  # with the longitudinal kick (psigma changes at every kick: no cache); earlier build
# split-TF32 form: float32 gather from the cached fixed-point weights
FP64_INST_BASE_F32 = 5.8
# sliced grids: the slice index (one subtract, one multiply; the floor is integer work) per locate
FP64_INST_SLICE = 2.0
# Bezier gather instead of bilinear fields (extra per particle-kick), and the
# longitudinal kick (bilinear / Bezier potentials of two slices plus the
# psigma-dependent quantities recomputed): measured with ncu like FP64_INST
FP64_INST_BEZIER = 103.7
FP64_INST_LON = 25.6
FP64_INST_LON_BEZIER = 83.7
# the same in the split form (float32 potential and Bezier surface)
FP64_INST_BEZIER_F32 = 3.85
FP64_INST_LON_F32 = 13.95
FP64_INST_LON_BEZIER_F32 = 13.95
# DRAM bytes (read + write) per kick_push launch, split form, from ncu (cold
# cache; c2: mean of the three segment types), with the kernel sources'
# SHA-256 (first 16 hex digits) they were captured on: the roofline's
# "traffic" while the sources still match; other workloads report null.
KP_TRAFFIC_TF32 = {"c2": (122.4e6, "741f33f43b3df3e1"),  # 1e6 particles (the working set partly stays in L2)
                   "c4": (3860.0e6, "052c41cbfc714941"),  # 2.37e7 particles, batched (kick_push_traffic_c4_c5.md)
                   "c5": (1594.1e6, "052c41cbfc714941")}  # 1e7 particles in 32 slices
# GB300: 152 SMs x 2 FP64 instructions per SM clock x 2.07 GHz maximum clock
FP64_PIPE_PEAK_TINST = 152 * 2 * 2.07e9 / 1e12
# FP64-pipe instructions per particle of the stand-alone deposit (xi and eta: a
# subtract and a multiply each, 4.23 measured with ncu
# sm__thread_inst_executed_pipe_fp64_pred_on, profiles/deposit_c2.md; the
# slice index two more)
DEP_FP64_INST = 4.23
DEP_FP64_INST_SLICE = 2.0
KP_SOURCES = ("kick_push.cu", "maps.cuh", "cic.cuh", "fixpt.h", "sc_internal.cuh")
FP64_INST_SOURCES_SHA = "741f33f43b3df3e1"
# HBM bytes per particle-kick that the fused kick/push must move (algorithmic):
# the six float64 coordinates read (48 B) and the five a kick and a push
# change written back (40 B: psigma changes only in RF cavities); 96 B when
# psigma is written too.
KP_ALGORITHMIC_BYTES = 88
KP_ALGORITHMIC_BYTES_RF = 96


def kp_sources_sha():
    import hashlib
    h = hashlib.sha256()
    for f in KP_SOURCES:
        with open(os.path.join(ROOT, "paper_2010_11540_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]

# arithmetic of each form: particle state and push, solve
DTYPE_LABEL = {"fp64": "f64", "tf32x3": "f64 state and push / tf32x3 solve (fp32 accumulate, fp32 fields)",
               "bf16x3": "f64 state and push / bf16x3 solve (fp32 accumulate, fp32 fields)",
               "pipe_fp64": "f64", "pipe_tf32x3": "f64 state and push / tf32x3 solve (fp32 accumulate, fp32 fields)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="tf32x3", choices=["fp64", "tf32x3", "bf16x3"],
                    help="solve form of the headline number; the other forms are timed beside it")
    ap.add_argument("--compare", default=None,
                    help="comma-separated solve forms timed beside the headline one (default: the plain FP64 form, "
                         "or split-TF32 when the headline is FP64; c3: both other forms)")
    ap.add_argument("--no-compare", action="store_true", help="skip timing the other solve forms")
    ap.add_argument("--config", default="c2")
    ap.add_argument("--cpu-kicks", type=int, default=0,
                    help="oracle sample size in kicks (0: as many as take about 10 s, from a 2-kick probe)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--boundary", default="open", choices=["open", "pipe"],
                    help="pipe: conducting rectangular pipe on the grid's outer nodes (Sec. IV-B), one more node "
                         "per axis over the same extent, float64 sine-transform solve")
    ap.add_argument("--gather", default="bilinear", choices=["bilinear", "bezier"],
                    help="bezier: Bezier surface of the potential (Sec. IV-C), pipe grids only")
    ap.add_argument("--longitudinal", action="store_true",
                    help="longitudinal space-charge kick (Sec. IV), sliced pipe grids (c5 --boundary pipe)")
    ap.add_argument("--tiling", default=None,
                    help="force the split-TF32 solve's kernel variant per phase, e.g. 0,1,2,1 (default: tuned)")
    ap.add_argument("--kp-shape", default=None,
                    help="force the kick/push launch shape (default: tuned): block size and traversal "
                         "(0 grid stride, 1 chunks) for single-bunch configs, e.g. 768,1; block size and "
                         "waves per launch for c4, e.g. 768,4")
    return ap.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------- helpers
def element_mix(lat):
    """Elements per turn by kind (space-charge locations as "kicks")."""
    from paper_2010_11540_gb300 import synth
    t = lat["type"]
    per = {synth.DRIFT: "drift", synth.QUAD: "quad", synth.SEXT: "sext", synth.BEND: "bend", synth.RF: "rf"}
    mix = {name: int((t == code).sum()) for code, name in per.items()}
    mix["kicks"] = int((t == synth.MARK).sum())
    return mix


def fp64_inst_per_turn(lat, precision):
    """FP64-pipe instructions per particle per turn from the element mix, and kicks/turn."""
    mix = element_mix(lat)
    f = mix["kicks"] * (FP64_INST["base"] if precision == "fp64" else FP64_INST_BASE_F32)
    for name in ("drift", "quad", "sext", "bend", "rf"):
        f += mix[name] * FP64_INST[name]
    return f, mix["kicks"]


def probe_peaks(stream):
    """Live machine probes from libsc_probe.so (bench_probe.cu, built beside
    this file; not part of libsc): conflict-free and random-word shared u64
    atomics per second, FP64 FMA instructions per second."""
    import ctypes
    from paper_2010_11540_gb300 import build
    L = ctypes.CDLL(build.build_probe())
    L.scb_probe_peaks.argtypes = [ctypes.POINTER(ctypes.c_double)] * 3 + [ctypes.c_void_p]
    L.scb_probe_peaks.restype = ctypes.c_int
    a, r, f = ctypes.c_double(0), ctypes.c_double(0), ctypes.c_double(0)
    code = L.scb_probe_peaks(ctypes.byref(a), ctypes.byref(r), ctypes.byref(f), int(stream.cuda_stream))
    if code != 0:
        raise RuntimeError(f"machine probes failed ({code})")
    return a.value, r.value, f.value


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


def cpu_baseline(config, n_kicks, boundary="open", gather="bilinear", longitudinal=False, threads=1):
    """The FP64 oracle as it stands on `threads` host threads (None: every
    core; its OpenMP particle loops give the same bits for any count), on a
    bounded sample: the full particle set (c4: its largest bunch) through the
    first n_kicks kicks of turn 1."""
    import oracle
    from paper_2010_11540_gb300 import synth
    oracle.set_threads(threads)
    slices = None
    if config == "c4":
        bunches = synth.c4_bunches()
        parts, b, grid, lat = max(bunches, key=lambda u: len(u[0]["x"]))
        what = "c4 largest bunch"
    else:
        parts, b, grid, lat = synth.workload(config)
        what = f"{config} full particle set"
        if "n_slices" in synth.CONFIGS[config]:
            slices = oracle.Slices(*synth.slices(config))
    if boundary == "pipe":
        grid = (grid[0] + 1, grid[1] + 1) + tuple(grid[2:])
        what += f", conducting pipe, {gather} gather" + (", longitudinal kick" if longitudinal else "")
    g = oracle.Geometry(*grid)
    oracle.lib()
    if n_kicks <= 0:
        # about 10 s of oracle work: the per-kick time from a 2-kick probe
        st = oracle.copy_state(parts)
        t0 = time.perf_counter()
        oracle.track(g, st, b, lat, 1, max_kicks=2, slices=slices, boundary=boundary, gather=gather,
                     longitudinal=longitudinal)
        per_kick = (time.perf_counter() - t0) / 2
        n_kicks = max(2, min(10000, int(10.0 / max(per_kick, 1e-6))))
    per_turn = max(1, int((lat["type"] == synth.MARK).sum()))
    turns = -(-n_kicks // per_turn)
    st = oracle.copy_state(parts)
    t0 = time.perf_counter()
    done = oracle.track(g, st, b, lat, turns, max_kicks=n_kicks, slices=slices, boundary=boundary, gather=gather,
                        longitudinal=longitudinal)
    dt = time.perf_counter() - t0
    n = len(parts["x"])
    span = "of turn 1" if turns == 1 else f"over {turns} turns"
    cores = oracle.threads()
    oracle.set_threads(1)
    return {"value": n * done / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{what} ({n}), first {done} SC kicks {span}, {dt:.1f} s on {cores} thread(s)"}


def cpu_baselines(config, n_kicks, boundary="open", gather="bilinear", longitudinal=False):
    """The oracle on every host core (the reported baseline) and on one."""
    allc = cpu_baseline(config, n_kicks, boundary, gather, longitudinal, threads=None)
    one = cpu_baseline(config, n_kicks, boundary, gather, longitudinal, threads=1)
    allc["single_thread"] = {"value": one["value"], "cores": 1, "sample": one["sample"]}
    allc["threads_note"] = ("OpenMP particle loops and per-thread integer charge grids: bit-identical to one thread "
                            "(tests/test_oracle_track.py::test_threads_bit_identical)")
    return allc


# --------------------------------------------------------------------------- reference arm
def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    kicks = max(1, args.cpu_kicks // 4) if args.cpu_kicks > 0 else 6  # a bounded sample per step
    for _ in range(args.warmup):
        cpu_baseline(args.config, 1, threads=None)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(args.config, kicks, threads=None))
    wall = time.perf_counter() - t0
    value = statistics.mean(v["value"] for v in vals)
    cb = dict(vals[0])
    cb["value"] = value
    cb["sample"] = f"each step: {cb['sample']}"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * wall / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOADS.get(args.config, args.config),
                                            "step": f"{kicks} SC kicks on the CPU oracle"},
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- our arm
KEYS = ("x", "px", "y", "py", "sigma", "psigma")


class SingleRun:
    """One bunch on one grid (c1-c3), or one bunch on a sliced grid (c5): sc_track_turns."""

    kernel = "kick_push_kernel (gather+kick, push, fused CIC deposit)"

    def __init__(self, config, rank, stream, args=None):
        from paper_2010_11540_gb300 import synth
        self.parts, self.b, self.grid, self.lat = synth.workload(config, seed=12345 + rank)
        self.slices = synth.slices(config) if "n_slices" in synth.CONFIGS[config] else None
        self.pipe = args is not None and args.boundary == "pipe"
        self.gather = args.gather if args is not None else "bilinear"
        self.longitudinal = args is not None and args.longitudinal
        if self.pipe:  # walls on the outer nodes: n - 1 a power of two
            self.grid = (self.grid[0] + 1, self.grid[1] + 1) + tuple(self.grid[2:])
        self.n = len(self.parts["x"])
        self.stream = stream
        self.n_classes = 1
        # several ranks: each holds its own seeded share of one bunch of world x n particles, and the
        # ranks' charges are summed by an NCCL all-reduce captured in the turn (sc_set_charge_reduce)
        self.world = int(os.environ.get("WORLD_SIZE", 1))

    @staticmethod
    def allreduce(q, stream):
        import torch
        import torch.distributed as dist
        with torch.cuda.stream(stream):
            dist.all_reduce(q)

    def make(self, precision):
        import torch
        from paper_2010_11540_gb300 import sc
        dev = {k: torch.from_numpy(self.parts[k]).cuda() for k in KEYS}
        g = sc.create_grid(*self.grid, precision=precision, stream=self.stream, slices=self.slices)
        if self.world > 1:
            # one eager all-reduce of the (still zero) charge first: the communicator is set up
            # outside the turn's graph capture, which then records the collective only
            self.allreduce(sc.charge_tensor(g), self.stream)
            self.stream.synchronize()
            sc.set_charge_reduce(g, self.allreduce, self.world * self.n)
        if precision in ("tf32x3", "pipe_tf32x3", "bf16x3") and self.tiling:
            sc.set_solver_tiling(g, self.tiling)
        if self.kp_shape:
            sc.set_kick_push_shape(g, *self.kp_shape)
        if precision in ("pipe_fp64", "pipe_tf32x3"):
            if self.gather == "bezier":
                sc.set_gather(g, "bezier")
            if self.longitudinal:
                sc.set_longitudinal_kick(g)
        return g, dev

    def tiling_desc(self, h):
        from paper_2010_11540_gb300 import sc
        if h[0].precision not in ("tf32x3", "pipe_tf32x3", "bf16x3"):
            return None
        v, d = sc.get_solver_tiling(h[0])
        return {"variants": v, "grid": d}

    def solver_work(self, h):
        from paper_2010_11540_gb300 import sc
        return sc.solver_work(h[0])

    def shape_desc(self, h):
        from paper_2010_11540_gb300 import sc
        t, v, us = sc.get_kick_push_shape(h[0])
        return {"threads": t, "traversal": ("grid stride", "chunks")[v],
                "trial_us_first_16_sc_steps": round(us, 1) or None,
                "chosen": "fixed" if self.kp_shape else ("tuned" if us > 0 else "default")}

    def turns(self, h, n):
        from paper_2010_11540_gb300 import sc
        sc.track_turns(h[0], h[1], self.b, self.lat, n)

    def trace(self, h, on):
        from paper_2010_11540_gb300 import sc
        sc.trace_enable(h[0], on)

    def trace_read(self, h):
        from paper_2010_11540_gb300 import sc
        return sc.trace_read(h[0])

    def pinned(self):
        import torch
        return {k: torch.from_numpy(self.parts[k].copy()).pin_memory() for k in KEYS}

    def host_turn(self, h, pinned):
        from paper_2010_11540_gb300 import sc
        sc.track_turns_host(h[0], pinned, self.b, self.lat, 1)

    def close(self, h):
        h[0].close()

    def cufft_reference(self, flush, reps=20):
        """Context line: the open-boundary solve as the paper does it, with cuFFT
        (through torch.fft, float64): forward real 2-D transform of the
        zero-padded charge, times two field spectra, two inverse transforms;
        median of `reps`, L2 flushed.  Not on the product path."""
        import torch
        if self.pipe or self.slices:
            return None
        nx, ny = self.grid[0], self.grid[1]
        gen = torch.Generator(device="cuda").manual_seed(7)
        q = torch.zeros(2 * ny, 2 * nx, dtype=torch.float64, device="cuda")
        q[:ny, :nx] = torch.rand(ny, nx, generator=gen, dtype=torch.float64, device="cuda")
        gx = torch.randn(2 * ny, nx + 1, generator=gen, dtype=torch.complex128, device="cuda")
        gy = torch.randn(2 * ny, nx + 1, generator=gen, dtype=torch.complex128, device="cuda")
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps + 3)]
        with torch.cuda.stream(self.stream):
            for i, (a, c) in enumerate(ev):
                flush.zero_()
                a.record(self.stream)
                f = torch.fft.rfft2(q)
                ex = torch.fft.irfft2(f * gx, s=q.shape)
                ey = torch.fft.irfft2(f * gy, s=q.shape)
                c.record(self.stream)
            torch.cuda.synchronize()
        del ex, ey
        ms = sorted(a.elapsed_time(c) for a, c in ev[3:])[reps // 2]
        return {"solve_us": ms * 1e3, "what": f"cuFFT (torch.fft, float64) rfft2 of the {2 * nx}x{2 * ny} "
                                             "zero-padded charge, x2 spectra, 2 irfft2; context only"}

    def deposit_roofline(self, h, flush, atom_random, atom_conflict_free, reps=20):
        """sc_deposit alone (the deposit kernel) on the workload's particles:
        4 shared-memory u64 atomic adds per particle inside the grid, against
        the probed conflict-free rate of such atomics (the random-word rate of
        a 128 KB table as context)."""
        import torch
        from paper_2010_11540_gb300 import sc
        g, dev = h
        with torch.cuda.stream(self.stream):
            out0 = sc.grid_read(g)[3]
            sc.deposit(g, dev)
            n_in = self.n - (sc.grid_read(g)[3] - out0)  # particles inside the grid (one deposit)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for a, c in ev:
                flush.zero_()
                a.record(self.stream)
                sc.deposit(g, dev)
                c.record(self.stream)
            torch.cuda.synchronize()
        ms = sorted(a.elapsed_time(c) for a, c in ev)[reps // 2]
        atomics = 4 * n_in
        rate = atomics / (ms * 1e-3)
        # the same bunch ordered by cell (sc_sort_particles, on a copy): warps combine equal cells
        with torch.cuda.stream(self.stream):
            od = {k: v.clone() for k, v in dev.items()}
            sc.sort_particles(g, od)
            sc.deposit(g, od)
            ev2 = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            for a, c in ev2:
                flush.zero_()
                a.record(self.stream)
                sc.deposit(g, od)
                c.record(self.stream)
            torch.cuda.synchronize()
        ms_o = sorted(a.elapsed_time(c) for a, c in ev2)[reps // 2]
        del od
        ordered = {"avg_launch_ms": ms_o, "achieved": atomics / (ms_o * 1e-3) / 1e9,
                   "frac": atomics / (ms_o * 1e-3) / atom_conflict_free,
                   "what": "the same particles ordered by cell (sc_sort_particles): each warp combines the weights "
                           "of neighbouring particles in one cell before its atomic adds; achieved counts the "
                           "4 algorithmic atomics per particle"}
        return {"bound": "shared-atomics", "kernel": "deposit_kernel (stand-alone sc_deposit)",
                "achieved": rate / 1e9, "peak": atom_conflict_free / 1e9, "unit": "G shared-u64-atomics/s",
                "frac": rate / atom_conflict_free, "avg_launch_ms": ms, "atomics_per_launch": atomics,
                "peak_source": "live probe (libsc_probe.so): conflict-free shared u64 atomicAdd, each warp on 32 "
                               "consecutive words, measured in this run",
                "context_peak_random_words": atom_random / 1e9,
                "frac_of_random_words": rate / atom_random, "ordered_bunch": ordered,
                # what binds it: the locate's FP64 subtract and multiply per axis (the cell, fraction and
                # weights are decoded from the bits with integer instructions), on the 2-per-clock FP64 pipe
                "fp64_pipe": {"fp64_inst_per_particle": DEP_FP64_INST + (DEP_FP64_INST_SLICE if self.slices else 0),
                              "achieved": (DEP_FP64_INST + (DEP_FP64_INST_SLICE if self.slices else 0)) * self.n
                              / (ms * 1e-3) / 1e12,
                              "peak": FP64_PIPE_PEAK_TINST, "unit": "T FP64-inst/s",
                              "frac": (DEP_FP64_INST + (DEP_FP64_INST_SLICE if self.slices else 0)) * self.n
                              / (ms * 1e-3) / 1e12 / FP64_PIPE_PEAK_TINST,
                              "ceiling_atomics_frac": 4 / (DEP_FP64_INST + (DEP_FP64_INST_SLICE if self.slices else 0))
                              * FP64_PIPE_PEAK_TINST * 1e12 / atom_conflict_free,
                              "note": "at the FP64 peak the deposit adds 4 atomics per 4 FP64 instructions: the "
                                      "ceiling_atomics_frac of the conflict-free atomic rate"}}

    def grid_desc(self):
        d = {"grid": [self.grid[0], self.grid[1]]}
        if self.slices:
            d["slices"] = list(self.slices)
        if self.pipe:
            d["boundary"] = "conducting rectangular pipe on the outer nodes"
            d["gather"] = self.gather
            d["longitudinal_kick"] = self.longitudinal
        return d


class BatchRun:
    """Many bunches in one batch (c4): sc_batch_track_turns."""

    kernel = "kick_push_batched (all bunches: gather+kick, push, fused CIC deposit)"

    def __init__(self, config, rank, stream):
        from paper_2010_11540_gb300 import synth
        self.bunches = synth.c4_bunches(seed=12345 + 1000 * rank)
        self.n = sum(len(p["x"]) for p, _, _, _ in self.bunches)
        self.lat = self.bunches[0][3]
        self.stream = stream
        self.grids = [g for _, _, g, _ in self.bunches]
        self.beams = [b for _, b, _, _ in self.bunches]
        self.lats = [l for _, _, _, l in self.bunches]
        self.n_classes = len(set(self.grids))

    def make(self, precision):
        import torch
        from paper_2010_11540_gb300 import sc
        devs = [{k: torch.from_numpy(p[k]).cuda() for k in KEYS} for p, _, _, _ in self.bunches]
        B = sc.create_batch(self.grids, precision=precision, stream=self.stream)
        if precision in ("tf32x3", "bf16x3") and self.tiling:
            sc.batch_set_solver_tiling(B, self.tiling)
        if self.kp_shape:
            sc.batch_set_kick_push_shape(B, *self.kp_shape)
        return B, devs

    def tiling_desc(self, h):
        from paper_2010_11540_gb300 import sc
        if h[0].precision not in ("tf32x3", "bf16x3"):
            return None
        out = {}
        for i, g in enumerate(self.grids):
            key = f"{g[0]}x{g[1]}"
            if key not in out:
                out[key] = sc.batch_get_solver_tiling(h[0], i)[1]
        return out

    def solver_work(self, h):
        return None  # the grid classes' solves run side by side on their own streams

    def shape_desc(self, h):
        from paper_2010_11540_gb300 import sc
        t, w, us = sc.batch_get_kick_push_shape(h[0])
        return {"threads": t, "waves": w, "trial_us_first_16_sc_steps": round(us, 1) or None,
                "chosen": "fixed" if self.kp_shape else ("tuned" if us > 0 else "default")}

    def turns(self, h, n):
        from paper_2010_11540_gb300 import sc
        sc.batch_track_turns(h[0], h[1], self.beams, self.lats, n)

    def trace(self, h, on):
        from paper_2010_11540_gb300 import sc
        sc.batch_trace_enable(h[0], on)

    def trace_read(self, h):
        from paper_2010_11540_gb300 import sc
        return sc.batch_trace_read(h[0])

    def pinned(self):
        import torch
        return [{k: torch.from_numpy(p[k].copy()).pin_memory() for k in KEYS} for p, _, _, _ in self.bunches]

    def host_turn(self, h, pinned):
        from paper_2010_11540_gb300 import sc
        sc.batch_track_turns_host(h[0], pinned, self.beams, self.lats, 1)

    def close(self, h):
        pass

    def grid_desc(self):
        sizes = sorted({g[0] for g in self.grids})
        return {"bunches": len(self.bunches), "grids": {f"{s}x{s}": sum(1 for g in self.grids if g[0] == s)
                                                        for s in sizes},
                "working_points": "8x8 tune scan +-0.1 around (22.40, 20.75)"}


def run_ours(args):
    import torch

    from paper_2010_11540_gb300 import build, sc, synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    build.build()
    sc.load()
    stream = torch.cuda.Stream()
    W = BatchRun(args.config, rank, stream) if args.config == "c4" else SingleRun(args.config, rank, stream, args)
    if args.boundary == "pipe":
        if args.config == "c4":
            raise SystemExit("--boundary pipe: single-bunch configs only")
        args.precision = "pipe_fp64" if args.precision == "fp64" else "pipe_tf32x3"
    W.tiling = [int(v) for v in args.tiling.split(",")] if args.tiling else None
    W.kp_shape = [int(v) for v in args.kp_shape.split(",")] if args.kp_shape else None
    n = W.n
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()

    def timed_turns(precision):
        """Warm-up turns, then exactly args.steps timed turns, L2 flushed between
        turns; returns (handle, total ms (max over ranks), wall s, clocks)."""
        h = W.make(precision)
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                W.turns(h, 1)
            stream.synchronize()
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(args.steps)]
            clocks = ClockSampler(local)
            clocks.start()
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()
            t_wall = time.perf_counter()
            for s in range(args.steps):
                flush.zero_()
                ev[s][0].record(stream)
                W.turns(h, 1)
                ev[s][1].record(stream)
            torch.cuda.synchronize()
            wall = time.perf_counter() - t_wall
            if world > 1:
                torch.distributed.barrier()
            clk = clocks.stop()
        ms = sum(a.elapsed_time(c) for a, c in ev)
        if world > 1:
            t = torch.tensor([ms], device="cuda")
            torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
            ms = float(t.item())
        return h, ms, wall, clk

    inst_turn, n_kicks = fp64_inst_per_turn(W.lat, {"pipe_fp64": "fp64", "pipe_tf32x3": "tf32x3",
                                                    "bf16x3": "tf32x3"}.get(args.precision,
                                                                                                 args.precision))
    if getattr(W, "slices", None):
        inst_turn += n_kicks * FP64_INST_SLICE
    f32 = args.precision in ("tf32x3", "pipe_tf32x3", "bf16x3")
    if args.gather == "bezier":
        inst_turn += n_kicks * (FP64_INST_BEZIER_F32 if f32 else FP64_INST_BEZIER)
    if args.longitudinal:
        inst_turn += n_kicks * ((FP64_INST_LON_BEZIER_F32 if f32 else FP64_INST_LON_BEZIER) if args.gather == "bezier"
                                else (FP64_INST_LON_F32 if f32 else FP64_INST_LON))
        from paper_2010_11540_gb300 import synth
        inst_turn += int((W.lat["type"] == synth.QUAD).sum()) * (FP64_INST_QUAD_UNCACHED - FP64_INST["quad"])
    h, ms, wall, clk = timed_turns(args.precision)
    value = world * n * n_kicks * args.steps / (ms * 1e-3)
    compare = None
    if not args.no_compare:
        if args.compare:
            others = args.compare.split(",")
        elif args.config == "c3":
            others = [f for f in ("fp64", "tf32x3", "bf16x3") if f != args.precision]
        else:
            others = [{"tf32x3": "fp64", "fp64": "tf32x3", "bf16x3": "fp64", "pipe_tf32x3": "pipe_fp64"}[args.precision]]
        forms = []
        for other in others:
            h2, ms2, _, clk2 = timed_turns(other)
            forms.append({"precision": other, "value": world * n * n_kicks * args.steps / (ms2 * 1e-3),
                          "ms_per_step": ms2 / args.steps, "clocks": clk2})
            W.close(h2)
            del h2
        compare = forms[0] if len(forms) == 1 else forms

    # ---------------- dominant kernel, timed inside the turn graph (library tracing:
    # CUDA events on the grid's stream around every solve and kick/push launch)
    W.trace(h, True)
    with torch.cuda.stream(stream):
        W.turns(h, 1)  # capture + warm
        W.trace_read(h)
        W.turns(h, 2)
    kp_ms, solve_ms, traced = W.trace_read(h)
    W.trace(h, False)
    kp_avg_ms = kp_ms / traced
    inst_per_kick = inst_turn / n_kicks
    achieved = inst_per_kick * n / (kp_avg_ms * 1e-3) / 1e12
    sha = kp_sources_sha()
    mix = element_mix(W.lat)
    rf = mix["rf"] > 0 or args.longitudinal
    kp_bytes = KP_ALGORITHMIC_BYTES_RF if rf else KP_ALGORITHMIC_BYTES
    hbm_peak = measured_peaks().get("hbm_gbs", 6800.0)
    hbm_achieved = kp_bytes * n / (kp_avg_ms * 1e-3) / 1e9
    roofline = {"bound": "alu", "kernel": W.kernel,
                "achieved": achieved, "peak": FP64_PIPE_PEAK_TINST, "unit": "T FP64-inst/s",
                "frac": achieved / FP64_PIPE_PEAK_TINST,
                "traffic": (KP_TRAFFIC_TF32[args.config][0]
                            if (args.config in KP_TRAFFIC_TF32 and args.precision == "tf32x3"
                                and args.gather == "bilinear" and args.boundary == "open"
                                and sha == KP_TRAFFIC_TF32[args.config][1]) else None),
                "traffic_unit": "DRAM bytes per launch (ncu, cold cache, mean of the ring's three segment types)",
                "peak_source": None,  # after the live probe below
                "avg_launch_ms": kp_avg_ms,
                "fp64_inst_per_particle_kick": inst_per_kick,
                "fp64_inst_model": {"per_element": dict(FP64_INST, base_split_form=FP64_INST_BASE_F32),
                                    "element_mix_per_turn": mix,
                                    "source": "ncu sm__thread_inst_executed_pipe_fp64_pred_on per launch, "
                                              "profiles/kick_push_c2.md",
                                    "fitted_on_sources_sha": FP64_INST_SOURCES_SHA, "current_sources_sha": sha,
                                    "current": sha == FP64_INST_SOURCES_SHA},
                "hbm": {"achieved": hbm_achieved, "peak": hbm_peak, "unit": "GB/s", "frac": hbm_achieved / hbm_peak,
                        "algorithmic_bytes_per_particle_kick": kp_bytes,
                        "peak_source": "of measured: MEASURED_PEAKS.json hbm_gbs"},
                "solve_avg_ms": solve_ms / traced, "share_kick_push": kp_ms / (kp_ms + solve_ms)}

    # ---------------- the solve on the tensor cores (split-TF32 forms): tensor flops per traced solve
    roofline_solve = None
    work = W.solver_work(h)
    if work is not None and work[0] > 0:
        solve_s = solve_ms / traced * 1e-3
        bf16 = args.precision == "bf16x3"
        tensor_peak = measured_peaks().get("bf16_tflops", 1900.0) / (1 if bf16 else 2)
        roofline_solve = {
            "bound": "tensor",
            "kernel": "dft_gemm (split-%s DFT GEMMs on tcgen05, all phases of one solve)" % ("BF16" if bf16 else "TF32"),
            "achieved": work[0] / solve_s / 1e12, "peak": tensor_peak, "unit": "TFLOP/s",
            "frac": work[0] / solve_s / 1e12 / tensor_peak,
            "peak_source": ("of measured: MEASURED_PEAKS.json bf16_tflops (burst)" if bf16 else
                            "of measured: MEASURED_PEAKS.json bf16_tflops (burst) x 1/2, the nominal dense "
                            "TF32/BF16 ratio"),
            "tensor_flops_per_solve": work[0], "fft_equivalent_flops_per_solve": work[1],
            "fft_equivalent_tflops": work[1] / solve_s / 1e12, "solve_us_traced": solve_s * 1e6,
            "note": "latency-bound: a few microseconds of tensor work per phase; traced solves are serialised "
                    "with events (in the turn graph programmatic dependent launch overlaps the phases)"}

    # ---------------- live machine probes and the stand-alone deposit (shared-atomic roofline)
    atom_cf, atom_rand, fp64_probe = probe_peaks(stream)
    roofline["peak_probe_fp64_tinst"] = fp64_probe / 1e12
    roofline["peak_source"] = ("derived: 152 SMs x 2 FP64 instructions/clk x 2.07 GHz; the FMA probe of this run "
                               "reaches %.2f/clk/SM at 2.07 GHz" % (fp64_probe / 152 / 2.07e9))
    deposit = W.deposit_roofline(h, flush, atom_rand, atom_cf) if hasattr(W, "deposit_roofline") else None
    cufft = W.cufft_reference(flush) if hasattr(W, "cufft_reference") else None

    # ---------------- end to end: host buffers through the public API
    pinned = W.pinned()
    e2e_steps = max(3, args.steps // 2)
    with torch.cuda.stream(stream):
        W.host_turn(h, pinned)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(e2e_steps):
            W.host_turn(h, pinned)
        torch.cuda.synchronize()
        e2e_s = (time.perf_counter() - t0) / e2e_steps
    e2e = {"value": world * n * n_kicks / e2e_s, "unit": UNIT, "h2d_bytes_per_step": 6 * 8 * n,
           "d2h_bytes_per_step": 6 * 8 * n}

    solve_kernels = {"fp64": 3, "tf32x3": 4, "bf16x3": 4, "pipe_fp64": 4, "pipe_tf32x3": 5}[args.precision]
    config = {"workload": WORKLOADS.get(args.config, args.config),
              "step": f"one turn = {n_kicks} SC kicks via "
                      f"{'sc_batch_track_turns' if args.config == 'c4' else 'sc_track_turns'} (CUDA graph)",
              "solve": {"fp64": "fp64 FFT convolution", "tf32x3": "tf32x3 DFT GEMMs on tcgen05",
                        "bf16x3": "bf16x3 DFT GEMMs on tcgen05 (kind::f16)",
                        "pipe_fp64": "fp64 sine transforms (conducting pipe)",
                        "pipe_tf32x3": "tf32x3 sine-transform GEMMs on tcgen05 (conducting pipe)"}[args.precision],
              "particles": n, **W.grid_desc(),
              "solve_tiling": W.tiling_desc(h), "kick_push_shape": W.shape_desc(h),
              "l2": "256 MB buffer written between timed turns",
              "parallelism": (f"replicas x{world}" if world == 1 or args.config == "c4" else
                              f"one bunch sharded over {world} ranks ({n} particles each), uint64 charge all-reduce "
                              "per space-charge kick captured in the turn graph")}
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": DTYPE_LABEL[args.precision], "data": "synthetic", "config": config,
            "roofline": roofline, "roofline_deposit": deposit, "roofline_solve": roofline_solve,
            "reference_cufft_solve": cufft, "e2e": e2e,
            "clocks": clk, "compare_form": compare,
            "gpu_launches": args.steps * n_kicks * (W.n_classes * solve_kernels + 1),
            "wall_s_timed": wall}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baselines(args.config, args.cpu_kicks, args.boundary, args.gather,
                                             args.longitudinal)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
