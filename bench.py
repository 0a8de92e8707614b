"""Throughput of the fused Maxwell-Stefan MRT stream-collide on GB300.

Headline workload (--workload tube, the default): ternary two-bulb
(Loschmidt-like) diffusion on D3Q7, 256^3 nodes, FP32, no-flux bounce-back
walls on all six faces, left half x = (0, 0.5, 0.5), right half
x = (0.5, 0.5, 0) joined by a tanh interface of width 4 cells,
D12 : D13 : D23 = 5 : 4 : 1 scaled to max lattice D = 0.1.

One bench step is one lattice Boltzmann time step of the whole grid: pull
streaming with the boundary faces, mole fractions, the per-node
Maxwell-Stefan relaxation matrices, collision and store (the last step of
each timed region also writes the per-species mass partials).  The timed
region is --steps steps, bracketed by barrier + synchronize and timed with
CUDA events on the launching stream; it is repeated until about a second
has been timed and the median is reported.

Metric: GLUPS = evolved-species node updates per second, S * cells * steps / s
with S = n - 1 distributions per node (the n-th species follows from the
closure); the n-counted figure is reported beside it.  The rest of the
metric is timed in the same run, at the same --steps, under "workloads":
five species on D2Q9 2048^2 (blobs), the FP64 D2Q5 128^2 run (sine), the
4096 batched solves (solves/s) and the adjoint/forward cost of the 512^2
gradient (at its own 4000 steps).  --workload selects another headline
(also D3Q15, D3Q6, D2Q4 and D1Q3 workloads) and --no-extras skips the rest.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
sample of the same workload.
"""

from __future__ import annotations

import argparse
import glob
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time
from dataclasses import dataclass

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUPS (species-node updates/s) and % of HBM roofline; batched solves/s; adjoint/fwd cost"
KERNEL_SOURCES = sorted(
    os.path.relpath(p_, os.path.dirname(os.path.abspath(__file__)))
    for p_ in glob.glob(os.path.join(os.path.dirname(os.path.abspath(__file__)),
                                     "paper_1808_06787_gb300", "csrc", "*.cuh")))


@dataclass
class Workload:
    key: str
    lattice: str
    Q: int
    grid: tuple
    n: int
    f64: bool
    bc: tuple
    description: str
    traffic_file: str

    @property
    def S(self):
        return self.n - 1

    @property
    def cells(self):
        return self.grid[0] * self.grid[1] * self.grid[2]

    @property
    def es(self):
        return 8 if self.f64 else 4

    def D(self):
        import synthetic as sy

        if self.key == "blobs":
            return sy.random_D(self.n, seed=1003)
        return sy.D_from_pairs(3, {(1, 2): 0.10, (1, 3): 0.08, (2, 3): 0.02})

    def x0(self, grid=None):
        import synthetic as sy

        nx, ny, nz = grid or self.grid
        if self.key in ("tube", "tube15", "tube6", "plane4", "plane5", "line"):
            return sy.two_bulb(nx, ny, nz, width=4.0)
        if self.key == "blobs":
            return sy.gaussian_blobs(self.n, nx, ny, seed=1003)
        return sy.sin_modes(3, nx, ny, amp=0.05, seed=1001)

    def sample_grid(self, cells_target: int):
        """A block of the workload with about cells_target nodes (oracle timing)."""
        nx, ny, nz = self.grid
        if self.key in ("tube", "tube15", "tube6"):  # x-slab of the closed tube: same physics per node
            sy_ = max(1, min(ny, cells_target // nx))
            sz = max(1, min(nz, cells_target // (nx * sy_)))
            return (nx, sy_, sz)
        if self.key == "line":
            return (int(max(64, min(nx, cells_target))), 1, 1)
        side = int(max(8, min(nx, cells_target ** 0.5)))
        return (side, side, 1)


def make_workload(key: str, grid_edge: int) -> Workload:
    P, W = "periodic", "noflux"
    if key == "tube":
        g = (grid_edge, grid_edge, grid_edge)
        return Workload("tube", "D3Q7", 7, g, 3, False, (W,) * 6,
                        "D3Q7 %d^3 ternary two-bulb closed tube, FP32, D12:D13:D23=5:4:1 "
                        "(max lattice D 0.1), no-flux walls" % grid_edge,
                        "traffic_d3q7_256cube_f32.json")
    if key == "blobs":
        e = grid_edge if grid_edge != 256 else 2048
        return Workload("blobs", "D2Q9", 9, (e, e, 1), 5, False, (P,) * 6,
                        "D2Q9 %d^2 five species, FP32, periodic, seeded Gaussian blobs "
                        "(sigma 32, amplitude 0.2), D_ij uniform in [0.01, 0.12]" % e,
                        "traffic_d2q9_2048sq_n5_f32.json")
    if key == "tube15":
        g = (grid_edge, grid_edge, grid_edge)
        return Workload("tube15", "D3Q15", 15, g, 3, False, (W,) * 6,
                        "D3Q15 %d^3 ternary two-bulb closed tube, FP32, D = (0.10, 0.08, 0.02), "
                        "no-flux walls" % grid_edge,
                        "traffic_d3q15_256cube_f32.json")
    if key == "tube6":
        g = (grid_edge, grid_edge, grid_edge)
        return Workload("tube6", "D3Q6", 6, g, 3, False, (W,) * 6,
                        "D3Q6 %d^3 ternary two-bulb closed tube, FP32, D = (0.10, 0.08, 0.02), "
                        "no-flux walls" % grid_edge,
                        "traffic_d3q6_256cube_f32.json")
    if key == "plane4":
        e = 8192 if grid_edge == 256 else grid_edge
        return Workload("plane4", "D2Q4", 4, (e, e, 1), 3, False, (W, W, P, P, P, P),
                        "D2Q4 %d^2 ternary two-bulb, FP32, D = (0.10, 0.08, 0.02), no-flux x "
                        "faces, periodic y" % e,
                        "traffic_d2q4_8192sq_f32.json")
    if key == "plane5":
        e = 8192 if grid_edge == 256 else grid_edge
        return Workload("plane5", "D2Q5", 5, (e, e, 1), 3, False, (W, W, P, P, P, P),
                        "D2Q5 %d^2 ternary two-bulb, FP32, D = (0.10, 0.08, 0.02), no-flux x "
                        "faces, periodic y" % e,
                        "traffic_d2q5_8192sq_f32.json")
    if key == "line":
        nx = 1 << 26 if grid_edge == 256 else grid_edge
        return Workload("line", "D1Q3", 3, (nx, 1, 1), 3, False, (W, W, P, P, P, P),
                        "D1Q3 line of %d nodes, ternary two-bulb, FP32, D = (0.10, 0.08, 0.02), "
                        "no-flux ends" % nx,
                        "traffic_d1q3_64M_f32.json")
    e = grid_edge if grid_edge != 256 else 128
    return Workload("sine", "D2Q5", 5, (e, e, 1), 3, True, (P,) * 6,
                    "D2Q5 %d^2 ternary, FP64, periodic, seeded sine modes, "
                    "D = (0.10, 0.08, 0.02)" % e,
                    "traffic_d2q5_128sq_f64.json")


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(fname: str, grid):
    """DRAM bytes per launch of a kernel from its committed ncu record, or None
    when the kernel sources changed since it was taken or the size differs."""
    try:
        with open(os.path.join(ROOT, "profiles", fname)) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_hash") != kernel_hash() or list(rec.get("grid", ())) != list(grid):
        return None
    return rec.get("dram_bytes_per_launch")


def measured_traffic(wl: Workload):
    """DRAM bytes per launch of the workload's step kernel (see recorded_traffic)."""
    return recorded_traffic(wl.traffic_file, wl.grid)


def hbm_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "measured"
    except (OSError, ValueError, KeyError):
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self._t.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [v.strip() for v in ln.split(",")]
            if len(p) < 7:
                continue
            try:
                sm.append(float(p[0]))
                mx.append(float(p[1]))
            except ValueError:
                continue
            for nm, v in zip(names, p[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# FP64 work of the D2Q5 ternary step per node, counted by ncu on the kernel
# (DADD + DMUL + 2 DFMA: 59 + 21 + 2 x 36 per node).  GB300 issues 2 DFMA per SM
# and cycle (ncu's peak_sustained of 304 per cycle over its 152 SMs).
D2Q5_TERNARY_FP64_FLOPS_PER_NODE = 152.0
DFMA_PER_SM_CLK = 2


def fp64_peak_tflops(sms: int, sm_mhz: float) -> float:
    """FP64-pipe peak: SMs x DFMA per SM and clock x 2 flops x SM clock."""
    return sms * DFMA_PER_SM_CLK * 2 * sm_mhz * 1e6 / 1e12


def fp64_roofline(wl: "Workload", step_ms: float, sms: int, sm_mhz: float) -> dict:
    """ALU roofline of the L2-resident FP64 workload: its step kernel is bound by the
    FP64 pipes (57 % of their issue slots busy under ncu), not by HBM.  The peak
    uses the device's SM count and the SM clock sampled while it ran."""
    flops = D2Q5_TERNARY_FP64_FLOPS_PER_NODE * wl.cells
    achieved = flops / (step_ms * 1e-3) / 1e12
    peak = fp64_peak_tflops(sms, sm_mhz)
    return {
        "bound": "alu",
        "achieved": round(achieved, 4),
        "peak": round(peak, 4),
        "unit": "TFLOP/s",
        "frac": round(achieved / peak, 4),
        "traffic": measured_traffic(wl),
        "peak_source": "derived: %d SMs x %d DFMA/clk x 2 flops x %.0f MHz (sampled SM clock; FP64 pipe)"
                       % (sms, DFMA_PER_SM_CLK, sm_mhz),
        "algorithmic_flops_per_launch": flops,
        "note": "FP64 flops per node counted by ncu on this kernel; state L2-resident",
    }


def dist_context(backend: str = "nccl"):
    """(world, rank, local_rank, dist-or-None) from the torchrun environment.

    The rank's GPU is selected before the process group exists, so that NCCL's
    communicators bind to it.  Single-solve workloads shard one grid over the
    ranks (halo exchange every step, masses by one all-reduce); batches and the
    adjoint run one independent problem per rank."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist

        if backend == "nccl" and torch.cuda.is_available():
            torch.cuda.set_device(local)
        if not dist.is_initialized():
            dist.init_process_group(backend)
    return world, rank, local, dist


def max_over_ranks(dist, values, device="cuda"):
    """Element-wise maximum over ranks: the slowest replica sets the job time."""
    if dist is None:
        return [float(v) for v in values]
    import torch

    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_rate(units_per_rank: float, world: int, t_ms: float) -> float:
    """Whole-job throughput: the units all ranks processed over the job time."""
    return units_per_rank * world / (t_ms * 1e-3)


MIN_TIMED_S = 1.0  # repeats of the K-step region fill at least this long (clock samples)
MAX_REPEATS = 1000


def timed_repeats(run_steps, stream, steps: int, barrier, min_repeats: int = 5):
    """Device time of `steps` steps (CUDA events on the launching stream, barrier +
    synchronize on both sides), repeated until at least MIN_TIMED_S has been spent
    (and at least min_repeats times); returns (median ms, list of ms)."""
    import torch

    times = []
    spent = 0.0
    while len(times) < min_repeats or (spent < MIN_TIMED_S * 1e3 and len(times) < MAX_REPEATS):
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        run_steps(steps)
        ev1.record(stream)
        barrier()
        times.append(ev0.elapsed_time(ev1))
        spent += times[-1]
    return statistics.median(times), times


E2E_REPEATS = 5


def e2e_median(run, barrier, repeats: int = E2E_REPEATS):
    """Wall time of `run()` (host buffers in and out, so the host clock with a
    barrier + synchronize on both sides): one untimed run, then the median of
    `repeats` timed runs; returns (median s, list of s)."""
    run()
    barrier()
    times = []
    for _ in range(repeats):
        barrier()
        t0 = time.perf_counter()
        run()
        barrier()
        times.append(time.perf_counter() - t0)
    return statistics.median(times), times


def local_barrier():
    import torch

    torch.cuda.synchronize()


def measure_single(wl: Workload, steps: int, warmup: int, barrier=local_barrier, keep=False):
    """Time `steps` steps of a single-solve workload (inputs resident in HBM)."""
    import numpy as np
    import torch

    from paper_1808_06787_gb300 import Solver

    tdtype = torch.float64 if wl.f64 else torch.float32
    x0_host = torch.from_numpy(wl.x0()).to(tdtype).pin_memory()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = Solver(wl.lattice, wl.D(), wl.grid, bc=wl.bc, dtype=tdtype, stream=stream)
        s.set_state(x0_host.cuda(non_blocking=True))
        mass0 = s.mass()
        s.step(warmup)
        torch.cuda.synchronize()
        ms, reps = timed_repeats(s.step, stream, steps, barrier)
        flags = s.status()
        mass = s.mass()
    out = {"ms": ms, "repeats_ms": reps, "status_flags": flags,
           "mass_drift_rel": float(np.max(np.abs(mass - mass0) / np.abs(mass0))),
           "x0_host": x0_host, "stream": stream}
    if keep:
        out["solver"] = s
    else:
        s.close()
    return out


def hbm_roofline(bytes_per_launch: float, launch_ms: float, traffic) -> dict:
    peak, peak_kind = hbm_peak()
    achieved = bytes_per_launch / (launch_ms * 1e-3) / 1e9
    return {
        "bound": "hbm",
        "achieved": round(achieved, 1),
        "peak": peak,
        "unit": "GB/s",
        "frac": round(achieved / peak, 4),
        "traffic": traffic,
        "peak_source": peak_kind,
        "algorithmic_bytes_per_launch": bytes_per_launch,
    }


def single_line(wl: Workload, m: dict, steps: int, world: int, t_ms: float, sms: int, sm_mhz: float):
    """GLUPS, roofline and identification of a single-solve measurement."""
    glups = job_rate(float(wl.S) * wl.cells * steps, world, t_ms) / 1e9
    bytes_per_launch = 2.0 * wl.S * wl.Q * wl.es * wl.cells
    state_gb = bytes_per_launch / 1e9
    roof = (fp64_roofline(wl, t_ms / steps, sms, sm_mhz) if wl.key == "sine"
            else hbm_roofline(bytes_per_launch, t_ms / steps, measured_traffic(wl)))
    return {
        "value": round(glups, 4),
        "unit": "GLUPS",
        "steps": steps,
        "ms_per_step": round(t_ms / steps, 6),
        "repeats": len(m["repeats_ms"]),
        "repeat_ms_min_max": [round(min(m["repeats_ms"]), 4), round(max(m["repeats_ms"]), 4)],
        "dtype": "f64" if wl.f64 else "f32",
        "config": {
            "workload": wl.description,
            "lattice": wl.lattice, "grid": list(wl.grid), "n_species": wl.n,
            "evolved_species": wl.S,
            "bc": {"tube": "no-flux all faces", "tube15": "no-flux all faces",
                   "tube6": "no-flux all faces", "plane4": "no-flux x, periodic y",
                   "plane5": "no-flux x, periodic y",
                   "line": "no-flux ends"}.get(wl.key, "periodic"),
            "relax": "MRT, Lambda_2 by Eq. 3-16",
            "glups_n_counted": round(glups * wl.n / wl.S, 4),
            "l2": ("state %.2f GB per step vs 129 MB L2; no flush" % state_gb) if state_gb > 0.5
            else ("state %.1f MB per step is L2-resident: L2/latency bound, not an HBM test"
                  % (state_gb * 1e3)),
        },
        "roofline": roof,
        "gpu_launches": steps,
        "status_flags": m["status_flags"],
        "mass_drift_rel": m["mass_drift_rel"],
    }


def _split(wl: Workload) -> int:
    from paper_1808_06787_gb300.slab import split_axis

    return split_axis(wl.lattice)


def device_sms(local: int) -> int:
    import torch

    return int(torch.cuda.get_device_properties(local).multi_processor_count)


def sharded_grid(wl: Workload, world: int):
    """Global grid of the sharded solve: every rank owns one workload-sized slab,
    stacked along the lattice's split axis (weak scaling)."""
    from paper_1808_06787_gb300.slab import split_axis

    g = list(wl.grid)
    g[split_axis(wl.lattice)] *= world
    return tuple(g)


def measure_sharded(wl: Workload, steps: int, warmup: int, dist, barrier, keep=False):
    """Time `steps` steps of one grid sharded over the ranks (slab decomposition,
    one slab per GPU, halo exchange by point-to-point messages every step).  Each
    rank's slab is the workload's grid and holds the workload's initial field, so
    the global field is the workload's field repeated along the split axis
    (continuous for the x-only two-bulb profile and the periodic fields)."""
    import numpy as np
    import torch

    from paper_1808_06787_gb300 import DistSlabSolver

    tdtype = torch.float64 if wl.f64 else torch.float32
    x0_host = torch.from_numpy(wl.x0()).to(tdtype).pin_memory()
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = DistSlabSolver(wl.lattice, wl.D(), sharded_grid(wl, dist.get_world_size()), dist, bc=wl.bc,
                           dtype=tdtype, stream=stream)
        s.set_state(x0_host.cuda(non_blocking=True))
        mass0 = s.mass()
        s.step(warmup)
        torch.cuda.synchronize()
        ms, reps = timed_repeats(s.step, stream, steps, barrier)
        flags = s.status()
        mass = s.mass()
    out = {"ms": ms, "repeats_ms": reps, "status_flags": flags,
           "mass_drift_rel": float(np.max(np.abs(mass - mass0) / np.abs(mass0))),
           "x0_host": x0_host, "stream": stream}
    if keep:
        out["solver"] = s
    else:
        s.close()
    return out


def run_ours(args, wl: Workload):
    import torch

    world, rank, local, dist = dist_context()
    torch.cuda.set_device(local)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        m = measure_sharded(wl, args.steps, args.warmup, dist, barrier, keep=True)
    else:
        m = measure_single(wl, args.steps, args.warmup, barrier, keep=True)
    clocks = sampler.stop()
    s, stream, x0_host = m["solver"], m["stream"], m["x0_host"]
    tdtype = x0_host.dtype

    # end to end through the public API with host buffers: pinned x0 in,
    # K steps, mole fractions and masses back to pinned host memory
    field_shape = s.solver.field_shape if world > 1 else s.field_shape
    x_host = torch.empty(field_shape, dtype=tdtype).pin_memory()
    e2e_s = None
    if not args.no_e2e:
        def e2e_run():
            s.set_state(x0_host)
            s.step(args.steps)
            if world > 1:
                x_host.copy_(s.moments())
            else:
                s.moments(x_host)
            s.mass()

        with torch.cuda.stream(stream):
            e2e_s, _ = e2e_median(e2e_run, barrier)
    s.close()
    e2e_ms = e2e_s * 1e3 if e2e_s is not None else float("nan")
    t_ms, e2e_ms = max_over_ranks(dist, [m["ms"], e2e_ms])
    extras = None
    if world == 1 and not args.no_extras:
        extras = measure_extras(args, wl, local)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    sms = device_sms(local)
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    line = single_line(wl, m, args.steps, world, t_ms, sms, mhz)
    updates = float(wl.S) * wl.cells * args.steps * world
    out = {
        "metric": METRIC,
        "value": line["value"],
        "unit": "GLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": line["ms_per_step"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": line["dtype"],
        "data": "synthetic (seeded %s; no dataset)" % {"tube": "two-bulb tanh profile",
                                                      "tube15": "two-bulb tanh profile",
                                                      "tube6": "two-bulb tanh profile",
                                                      "plane4": "two-bulb tanh profile",
                                                      "plane5": "two-bulb tanh profile",
                                                      "line": "two-bulb tanh profile",
                                                      "blobs": "Gaussian blobs",
                                                      "sine": "sine modes"}[wl.key],
        "config": dict(line["config"],
                       parallelism=("slab decomposition: grid %s split along %s into %d slabs of %s, one "
                                    "per GPU; one halo exchange per step (point-to-point), masses by one "
                                    "all-reduce" % (list(sharded_grid(wl, world)), "xyz"[_split(wl)], world,
                                                    list(wl.grid))) if world > 1 else "single GPU",
                       timing="median of %d repeats of the %d-step region (CUDA events, max over ranks)"
                              % (line["repeats"], args.steps)),
        "roofline": line["roofline"],
        "e2e": None if args.no_e2e else {
            "value": round(updates / (e2e_ms * 1e-3) / 1e9, 4),
            "unit": "GLUPS",
            "h2d_bytes_per_step": round(x0_host.numel() * wl.es / args.steps, 1),
            "d2h_bytes_per_step": round((x_host.numel() * wl.es + 8 * wl.n) / args.steps, 1),
            "timing": "host clock, median of %d runs after one untimed run" % E2E_REPEATS,
        },
        "gpu_launches": line["gpu_launches"],
        "clocks": clocks,
        "repeat_ms_min_max": line["repeat_ms_min_max"],
        "status_flags": line["status_flags"],
        "mass_drift_rel": line["mass_drift_rel"],
    }
    if extras is not None:
        out["workloads"] = extras
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(wl, budget_s=args.cpu_budget)
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def measure_extras(args, headline: Workload, local: int) -> dict:
    """The other parts of the metric, timed in the same run at the same --steps:
    the other single-solve configurations (five-species D2Q9 blobs, FP64 D2Q5
    sine), the batched solves and the adjoint/forward cost."""
    import torch

    sms = device_sms(local)
    out = {}
    for key in ("blobs", "sine"):
        if key == headline.key:
            continue
        wl = make_workload(key, 256)
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.3)
        m = measure_single(wl, args.steps, args.warmup)
        clocks = sampler.stop()
        mhz = (clocks or {}).get("sm_mhz") or 2070.0
        line = single_line(wl, m, args.steps, 1, m["ms"], sms, mhz)
        line["clocks"] = clocks
        out[key] = line
        torch.cuda.empty_cache()
    out["batch"] = measure_batch(args.steps, args.warmup, local, schedule=args.batch_schedule)
    torch.cuda.empty_cache()
    out["adjoint"] = measure_adjoint(args.warmup, local)
    torch.cuda.empty_cache()
    return out


BATCH_COUNT = 4096
BATCH_SOLVE_STEPS = 5000


def measure_batch(steps: int, warmup: int, local: int, count: int = BATCH_COUNT, seed: int = 1004,
                  schedule: int = -1, barrier=local_barrier, tune_steps: int = 8, keep=False):
    """Batched workload: `count` independent ternary D2Q5 FP32 solves, square sides
    uniform in [32, 256], per-instance D_ij uniform in [0.01, 0.12], sine
    (periodic) or two-bulb tanh (no-flux x) initial fields; step schedule chosen by
    the tuner unless `schedule` >= 0."""
    import numpy as np
    import torch

    import synthetic as sy
    from paper_1808_06787_gb300 import BatchSolver

    grids, Ds, bcs = sy.batch_instances(count, seed=seed)
    stream = torch.cuda.Stream()
    sampler = ClockSampler(local)
    with torch.cuda.stream(stream):
        b = BatchSolver("D2Q5", Ds, grids, bcs=bcs, dtype=torch.float32, stream=stream)
        if schedule < 0:
            chosen, tune_ms = b.tune(trial_steps=tune_steps)
        else:
            b.set_schedule(schedule)
            chosen, tune_ms = schedule, []
        launches_per_step = b.launches_per_step()
        x0_host = torch.empty(int(b.offsets[-1]), dtype=torch.float32).pin_memory()
        for i in range(count):
            x0_host[int(b.offsets[i]):int(b.offsets[i + 1])] = torch.from_numpy(
                sy.batch_field(i, int(grids[i][0]), seed=seed).reshape(-1)).float()
        b.set_state(x0_host.cuda(non_blocking=True))
        mass0 = b.mass()
        b.step(warmup)
        torch.cuda.synchronize()
        sampler.start()
        time.sleep(0.3)
        ms, reps = timed_repeats(b.step, stream, steps, barrier)
        clocks = sampler.stop()
        flags = b.status()
        mass = b.mass()
    nodes = float(sum(int(g[0]) * int(g[1]) for g in grids))
    bytes_per_step = 2.0 * 2 * 5 * 4 * nodes
    roof = hbm_roofline(bytes_per_step, ms / steps,
                        recorded_traffic("traffic_batch_d2q5_4096_f32.json", [count, int(chosen)])
                        if chosen % 7 == 0 else None)
    roof["note"] = "algorithmic bytes of a streamed step; L2-blocked schedules move less"
    out = {
        "value": round(count * steps / BATCH_SOLVE_STEPS / (ms * 1e-3), 3),
        "unit": "solves/s",
        "steps": steps,
        "ms_per_step": round(ms / steps, 6),
        "repeats": len(reps),
        "repeat_ms_min_max": [round(min(reps), 4), round(max(reps), 4)],
        "glups": round(2.0 * nodes * steps / (ms * 1e-3) / 1e9, 3),
        "dtype": "f32",
        "config": {
            "workload": "batched: %d ternary D2Q5 FP32 solves of %d steps, sides uniform in "
                        "[32, 256] (%.1f M nodes), D_ij uniform in [0.01, 0.12], sine/periodic "
                        "and tanh/no-flux-x fields" % (count, BATCH_SOLVE_STEPS, nodes / 1e6),
            "candidate": int(chosen),
            "schedule": int(chosen) % 7,
            "nodes_per_thread": 1 + int(chosen) // 7,
            "tuner_ms_per_step": [round(float(v), 4) for v in tune_ms],
            "l2": "state %.1f GB per step vs 129 MB L2" % (bytes_per_step / 1e9),
        },
        "roofline": roof,
        "gpu_launches": steps * launches_per_step,
        "clocks": clocks,
        "status_flags": flags,
        "mass_drift_rel": float(np.max(np.abs(mass - mass0) / np.abs(mass0))),
    }
    if keep:
        out.update(solver=b, x0_host=x0_host, stream=stream, grids=grids, Ds=Ds, bcs=bcs)
    else:
        b.close()
    return out


ADJOINT_STEPS = 4000


def measure_adjoint(warmup: int, local: int, n: int = 512, steps: int = ADJOINT_STEPS,
                    e2e: bool = False):
    """Adjoint workload: gradient of the L2 misfit of the final mole fractions
    (ternary D2Q5, n^2, FP32, `steps` steps, target from D* = (0.09, 0.07, 0.02))
    with respect to the three D_ij and the initial field, by the adjoint kernels
    with sqrt(T) checkpointing; the cost is reported against the plain forward run
    of the same steps (median of 3 of each).  The ratio is measured at the
    workload's own length: checkpointing makes it depend on T."""
    import torch

    import synthetic as sy
    from paper_1808_06787_gb300 import RunSpec, Solver, simulate

    x0 = torch.from_numpy(sy.sin_modes(3, n, n, amp=0.05, seed=1005)).float().cuda()
    Dm = lambda d: sy.D_from_pairs(3, {(1, 2): d[0], (1, 3): d[1], (2, 3): d[2]})

    def forward(d):
        s = Solver("D2Q5", Dm(d), (n, n), dtype=torch.float32)
        s.set_state(x0)
        s.step(steps)
        x = s.moments()
        s.close()
        return x

    target = forward((0.09, 0.07, 0.02)).double()
    for _ in range(max(1, warmup // 10)):
        forward((0.10, 0.08, 0.02))
    # one untimed gradient pass: loads torch's own kernels used by the loss
    dpw = torch.tensor((0.10, 0.08, 0.02), dtype=torch.float64, requires_grad=True)
    lw = ((simulate(x0.clone().requires_grad_(True), dpw, RunSpec("D2Q5", (n, n, 1), steps))
           .double() - target) ** 2).sum()
    lw.backward()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    fwd, ckpt, bwd, adj_us = [], [], [], []
    for _ in range(3):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        torch.cuda.synchronize()
        ev[0].record()
        forward((0.10, 0.08, 0.02))
        ev[1].record()
        dp = torch.tensor((0.10, 0.08, 0.02), dtype=torch.float64, requires_grad=True)
        xg = x0.clone().requires_grad_(True)
        spec = RunSpec("D2Q5", (n, n, 1), steps)
        spec.stats["adjoint_events"] = []
        xT = simulate(xg, dp, spec)
        loss = ((xT.double() - target) ** 2).sum()
        ev[2].record()
        loss.backward()
        ev[3].record()
        torch.cuda.synchronize()
        fwd.append(ev[0].elapsed_time(ev[1]))
        ckpt.append(ev[1].elapsed_time(ev[2]))
        bwd.append(ev[2].elapsed_time(ev[3]))
        # the dominant kernel: the adjoint step, timed over the backward's own loops
        adj = spec.stats["adjoint_events"]
        adj_us.append(1e3 * sum(a.elapsed_time(b) for a, b, _ in adj) / sum(c for _, _, c in adj))
    # the adjoint step alone (no recomputation sharing the GPU): one segment of 64
    # steps from a mid-run state, repeated
    s = Solver("D2Q5", Dm((0.10, 0.08, 0.02)), (n, n), dtype=torch.float32)
    s.set_state(x0)
    s.step(steps // 2)
    seg = 64
    ck = s.get_state()
    rest = torch.empty((seg - 1,) + tuple(s.state_shape), dtype=torch.float32, device="cuda")
    s.recompute(ck, steps // 2, seg - 1, rest)
    lam_a, lam_b, gacc = s.adjoint_state(), s.adjoint_state(), s.adjoint_scratch()
    s.adjoint_seed(2.0 * (s.moments().double() - target).float(), lam_a)
    alone = []
    for _ in range(5):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(s.stream)
        s.adjoint_steps(ck, rest, seg, lam_a, lam_b, gacc)
        e1.record(s.stream)
        torch.cuda.synchronize()
        alone.append(e0.elapsed_time(e1) * 1e3 / seg)
    s.close()
    clocks = sampler.stop()
    t_fwd, t_ckpt, t_bwd = (statistics.median(v) for v in (fwd, ckpt, bwd))
    adj_ms = statistics.median(adj_us) * 1e-3
    alone_ms = statistics.median(alone) * 1e-3
    adj_bytes = float(n * n) * 2 * 5 * (4 + 8 + 8)  # f+ (FP32) read, lambda (8 B) read and written
    roof = hbm_roofline(adj_bytes, alone_ms,
                        recorded_traffic("traffic_adjoint_d2q5_512sq_f32.json", [n, n]))
    roof.update(kernel="k_adjoint_step<D2Q5, 2, float>", avg_launch_us=round(alone_ms * 1e3, 3),
                in_backward_launch_us=round(adj_ms * 1e3, 3),
                note="launch time of the adjoint step alone (64-step segments, CUDA events); in the "
                     "backward it shares the GPU with the recomputation of the next segment "
                     "(in_backward_launch_us); the 2 x 21 MB adjoint state is largely L2-resident")
    out = {
        "value": round((t_ckpt + t_bwd) / t_fwd, 3),
        "unit": "x forward",
        "higher_is_better": False,
        "steps": steps,
        "ms_per_step": round((t_ckpt + t_bwd) / steps, 6),
        "dtype": "f32 forward, float-pair (about 48-bit) adjoint state",
        "config": {
            "workload": "adjoint: ternary D2Q5 %d^2 FP32, %d steps, L2 misfit, gradients wrt 3 "
                        "D_ij and the initial field, sqrt(T) checkpointing" % (n, steps),
            "forward_ms": round(t_fwd, 3),
            "checkpointed_forward_ms": round(t_ckpt, 3),
            "backward_ms": round(t_bwd, 3),
            "checkpoints": spec.stats.get("checkpoints"),
            "segment_steps": spec.stats.get("segment"),
            "dL_dD": [float(v) for v in dp.grad.numpy()],
            "glups_forward": round(2.0 * n * n * steps / (t_fwd * 1e-3) / 1e9, 3),
            "timing": "median of 3 forward and 3 gradient runs (CUDA events)",
        },
        "roofline": roof,
        "gpu_launches": spec.stats.get("launches"),
        "clocks": clocks,
    }
    if e2e:
        # end to end through the public API: pinned host x0 in, gradients back to the host
        x0_host = x0.cpu().pin_memory()
        g_host = torch.empty(x0.shape, dtype=torch.float32).pin_memory()

        def e2e_run():
            xd = x0_host.cuda(non_blocking=True).requires_grad_(True)
            dpe = torch.tensor((0.10, 0.08, 0.02), dtype=torch.float64, requires_grad=True)
            le = ((simulate(xd, dpe, RunSpec("D2Q5", (n, n, 1), steps)).double() - target) ** 2).sum()
            le.backward()
            g_host.copy_(xd.grad, non_blocking=True)

        e2e_s, _ = e2e_median(e2e_run, torch.cuda.synchronize, repeats=3)
        e2e_ms = e2e_s * 1e3
        out["e2e"] = {
            "value": round(e2e_ms / t_fwd, 3),
            "unit": "x forward",
            "h2d_bytes_per_step": round(x0_host.numel() * 4 / steps, 1),
            "d2h_bytes_per_step": round((g_host.numel() * 4 + 3 * 8) / steps, 1),
            "timing": "host clock, median of 3 gradient runs after one untimed run",
        }
    return out


def run_batch(args):
    """Batched workload as the headline line (see measure_batch)."""
    import torch

    world, rank, local, dist = dist_context()
    torch.cuda.set_device(local)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    count = BATCH_COUNT if args.grid == 256 else max(1, args.grid)
    m = measure_batch(args.steps, args.warmup, local, count=count, seed=1004 + rank,
                      schedule=args.batch_schedule, barrier=barrier, tune_steps=16, keep=True)
    b, x0_host, stream = m.pop("solver"), m.pop("x0_host"), m.pop("stream")
    grids, Ds, bcs = m.pop("grids"), m.pop("Ds"), m.pop("bcs")
    e2e_s = None
    if not args.no_e2e:
        def e2e_run():
            b.set_state(x0_host)
            b.step(args.steps)
            b.moments(out_device="cpu")
            b.mass()

        with torch.cuda.stream(stream):
            e2e_s, _ = e2e_median(e2e_run, barrier)
    b.close()
    e2e_ms = e2e_s * 1e3 if e2e_s is not None else float("nan")
    t_ms, e2e_ms = max_over_ranks(dist, [m["ms_per_step"] * args.steps, e2e_ms])
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    out = {
        "metric": "batched solves/s (5000-step ternary D2Q5 solves) and GLUPS",
        "value": round(job_rate(count * args.steps / BATCH_SOLVE_STEPS, world, t_ms), 3),
        "unit": "solves/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_ms / args.steps, 6),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded sides, diffusivities, sine / tanh fields; no dataset)",
        "config": dict(m["config"], glups=m["glups"], parallelism="replicas" if world > 1 else "single GPU",
                       timing="median of %d repeats of the %d-step region (CUDA events)"
                              % (m["repeats"], args.steps)),
        "roofline": m["roofline"],
        "e2e": None if args.no_e2e else {
            "value": round(count * world * args.steps / BATCH_SOLVE_STEPS / (e2e_ms * 1e-3), 3),
            "unit": "solves/s",
            "h2d_bytes_per_step": round(x0_host.numel() * 4 / args.steps, 1),
            "d2h_bytes_per_step": round((x0_host.numel() * 4 + 8 * 3 * count) / args.steps, 1),
            "timing": "host clock, median of %d runs after one untimed run" % E2E_REPEATS,
        },
        "cpu_baseline": None if (args.no_cpu_baseline or world > 1)
        else cpu_baseline_batch(grids, Ds, bcs, 1004 + rank, budget_s=args.cpu_budget),
        "gpu_launches": m["gpu_launches"],
        "clocks": m["clocks"],
        "status_flags": m["status_flags"],
        "mass_drift_rel": m["mass_drift_rel"],
    }
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def run_adjoint(args):
    """Adjoint workload as the headline line (see measure_adjoint).  The gradient
    of one problem runs on one GPU: under torchrun rank 0 measures it and the
    other ranks exit without work."""
    import torch

    world, rank, local, dist = dist_context()
    if world > 1:
        torch.cuda.set_device(local)
        if rank != 0:
            dist.destroy_process_group()
            return
    steps = args.steps or ADJOINT_STEPS
    n = 512 if args.grid == 256 else args.grid
    m = measure_adjoint(args.warmup, 0, n=n, steps=steps, e2e=not args.no_e2e)
    out = {
        "metric": "adjoint/fwd cost (gradient wrt D_ij and x0 over plain forward)",
        "value": m["value"],
        "unit": m["unit"],
        "n_gpus": 1,
        "steps": steps,
        "warmup": args.warmup,
        "ms_per_step": m["ms_per_step"],
        "higher_is_better": False,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": m["dtype"],
        "data": "synthetic (seeded sine modes; target from D* = (0.09, 0.07, 0.02))",
        "config": m["config"],
        "roofline": m["roofline"],
        "e2e": m.get("e2e"),
        "gpu_launches": m["gpu_launches"],
        "clocks": m["clocks"],
    }
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def _oracle_sample_run(wl: Workload, cells_target: int, steps: int):
    """Time the oracle on a block of the workload with about cells_target nodes."""
    import oracle

    g = wl.sample_grid(cells_target)
    x0 = wl.x0(g)
    t0 = time.perf_counter()
    oracle.run(wl.lattice, wl.D(), x0, steps, bc=wl.bc)
    return time.perf_counter() - t0, g


def cpu_baseline(wl: Workload, budget_s: float = 20.0):
    """The oracle as it stands, timed on the host cores over a bounded sample."""
    import oracle

    oracle.build()
    probe = min(wl.cells, 65536)
    dt1, g1 = _oracle_sample_run(wl, probe, 1)
    rate = g1[0] * g1[1] * g1[2] / dt1  # node updates per second
    if rate * budget_s >= wl.cells:
        cells = wl.cells
        steps = int(max(1, min(20000, rate * budget_s / wl.cells)))
    else:
        cells, steps = int(max(64, rate * budget_s)), 1
    dt, g = _oracle_sample_run(wl, cells, steps)
    n = g[0] * g[1] * g[2]
    return {
        "value": round(wl.S * n * steps / dt / 1e9, 6),
        "unit": "GLUPS",
        "cores": oracle.get_threads(),
        "kind": "oracle",
        "sample": "%d step(s) on a %dx%dx%d block of the workload (FP64 oracle, OpenMP), %.1f s"
                  % (steps, g[0], g[1], g[2], dt),
    }


def cpu_baseline_batch(grids, Ds, bcs, seed: int, budget_s: float = 20.0):
    """The oracle on the first instances of the batch, converted to solves/s
    (5000-step solves of the batch's mean instance size)."""
    import oracle

    import synthetic as sy

    oracle.build()
    k = min(8, len(grids))
    fields = [sy.batch_field(i, int(grids[i][0]), seed=seed) for i in range(k)]

    def run(steps):
        t0 = time.perf_counter()
        for i in range(k):
            oracle.run("D2Q5", Ds[i], fields[i], steps, bc=bcs[i])
        return time.perf_counter() - t0

    probe = run(1)
    steps = int(max(1, min(5000, budget_s / max(probe, 1e-6))))
    dt = run(steps)
    nodes = sum(int(grids[i][0]) * int(grids[i][1]) for i in range(k))
    rate = nodes * steps / dt  # node updates per second
    mean_nodes = float(sum(int(g[0]) * int(g[1]) for g in grids)) / len(grids)
    return {
        "value": round(rate / (mean_nodes * BATCH_SOLVE_STEPS), 4),
        "unit": "solves/s",
        "cores": oracle.get_threads(),
        "kind": "oracle",
        "sample": "instances 0..%d (%d nodes), %d steps each, FP64 oracle, %.1f s" % (k - 1, nodes, steps, dt),
    }


def run_reference(args, wl: Workload):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    budget = args.cpu_budget * 4
    probe = min(wl.cells, 4096)
    dt1, g1 = _oracle_sample_run(wl, probe, 1)
    rate = g1[0] * g1[1] * g1[2] / dt1
    cells = int(max(64, min(wl.cells, rate * budget / max(1, args.steps + args.warmup))))
    if args.warmup:
        _oracle_sample_run(wl, cells, args.warmup)
    dt, g = _oracle_sample_run(wl, cells, args.steps)
    n = g[0] * g[1] * g[2]
    glups = wl.S * n * args.steps / dt / 1e9
    sample = ("%d timed steps (after %d warm-up) on a %dx%dx%d block of the workload, FP64 "
              "oracle, %.1f s" % (args.steps, args.warmup, g[0], g[1], g[2], dt))
    out = {
        "impl": "reference",
        "metric": METRIC,
        "value": round(glups, 6),
        "unit": "GLUPS",
        "n_gpus": int(os.environ.get("WORLD_SIZE", "1")),
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(dt * 1e3 / args.steps, 3),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic (same generator as the GPU arm; no dataset)",
        "config": {"workload": wl.description, "lattice": wl.lattice, "grid": list(wl.grid),
                   "n_species": wl.n},
        "cpu_baseline": {"value": round(glups, 6), "unit": "GLUPS", "cores": oracle.get_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(glups, 6), "unit": "GLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    global MIN_TIMED_S
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="steps per timed region (default 200; the adjoint workload: 4000)")
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=["tube", "blobs", "sine", "tube15", "tube6", "plane4",
                                           "plane5", "line", "batch", "adjoint"],
                    default="tube")
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of oracle work for the CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end run")
    ap.add_argument("--no-extras", action="store_true",
                    help="time only the headline workload (not the other parts of the metric)")
    ap.add_argument("--min-timed-s", type=float, default=MIN_TIMED_S,
                    help="repeat the timed region until this many seconds are timed (at least 5 "
                         "repeats; profiling runs use 0)")
    ap.add_argument("--batch-schedule", type=int, default=-1,
                    help="batched workload: fixed step candidate (0..13: schedule + 7 x kernel "
                         "shape) instead of the tuner's")
    ap.add_argument("--grid", type=int, default=256,
                    help="grid edge (256 selects each workload's own size)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    MIN_TIMED_S = max(0.0, args.min_timed_s)
    if args.workload != "adjoint" and args.steps is None:
        args.steps = 200
    if args.workload == "adjoint":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the adjoint workload has no "
                              "reference arm; use the single-solve workloads"}))
        else:
            run_adjoint(args)
        return
    if args.workload == "batch":
        if args.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the batched workload has no "
                              "reference arm; use the single-solve workloads"}))
        else:
            run_batch(args)
        return
    wl = make_workload(args.workload, args.grid)
    if args.impl == "reference":
        run_reference(args, wl)
    else:
        run_ours(args, wl)


if __name__ == "__main__":
    main()
