"""Throughput of the fused Maxwell-Stefan MRT stream-collide on GB300.

Workload (default): ternary two-bulb (Loschmidt-like) diffusion on D3Q7, 256^3
nodes, FP32, no-flux bounce-back walls on all six faces, left half
x = (0, 0.5, 0.5), right half x = (0.5, 0.5, 0) joined by a tanh interface of
width 4 cells, D12 : D13 : D23 = 5 : 4 : 1 scaled to max lattice D = 0.1.

One bench step is one lattice Boltzmann time step of the whole grid: pull
streaming with bounce-back, mole fractions, the per-node Maxwell-Stefan
relaxation matrices, collision and store (the last step of the timed run also
writes the FP64 per-species mass partials and reduces them).  The state is
2 x 940 MB, far larger than the 129 MB L2, so no flush is needed between steps.

Metric: GLUPS = evolved-species node updates per second, S * cells * steps / s
with S = n - 1 = 2 distributions per node (the n-th species follows from the
closure); the n-counted figure is reported beside it.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
slab of the same workload.
"""

from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NX = NY = NZ = 256  # --grid changes these (profiling of smaller copies)
N_SPECIES = 3
S_EVOLVED = N_SPECIES - 1
Q = 7
D_PAIRS = {(1, 2): 0.10, (1, 3): 0.08, (2, 3): 0.02}
METRIC = "GLUPS (species-node updates/s) and % of HBM roofline"
WORKLOAD = ("D3Q7 256^3 ternary two-bulb closed tube, FP32, D12:D13:D23=5:4:1 "
            "(max lattice D 0.1), no-flux walls")
KERNEL_SOURCES = ["paper_1808_06787_gb300/csrc/kernels.cuh",
                  "paper_1808_06787_gb300/csrc/node.cuh",
                  "paper_1808_06787_gb300/csrc/lattice.cuh"]
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "traffic_d3q7_256cube_f32.json")


def kernel_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(os.path.join(ROOT, p), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic():
    """DRAM bytes per launch of the step kernel from the committed ncu summary,
    or None when the kernel sources changed since it was taken."""
    try:
        with open(TRAFFIC_FILE) as fh:
            rec = json.load(fh)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_hash") != kernel_hash():
        return None
    return rec.get("dram_bytes_per_launch")


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


def initial_field(np):
    import synthetic as sy

    return sy.two_bulb(NX, NY, NZ, width=4.0)


def diffusivities():
    import synthetic as sy

    return sy.D_from_pairs(N_SPECIES, D_PAIRS)


def run_ours(args):
    import numpy as np
    import torch

    from paper_1808_06787_gb300 import Solver

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    D = diffusivities()
    x0_host = torch.from_numpy(initial_field(np)).float().pin_memory()
    cells = NX * NY * NZ
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        s = Solver("D3Q7", D, (NX, NY, NZ), bc="noflux", dtype=torch.float32, stream=stream)
        x0_dev = x0_host.cuda(non_blocking=True)
        s.set_state(x0_dev)
        mass0 = s.mass()
        s.step(args.warmup)
        torch.cuda.synchronize()

        sampler = ClockSampler(local)
        barrier()
        sampler.start()
        time.sleep(0.3)
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        barrier()
        ev0.record(stream)
        s.step(args.steps)
        ev1.record(stream)
        barrier()
        ms = ev0.elapsed_time(ev1)
        clocks = sampler.stop()
        flags = s.status()
        mass = s.mass()

        # end to end through the public API with host buffers: pinned x0 in,
        # K steps, mole fractions and masses back to pinned host memory
        x_host = torch.empty(s.field_shape, dtype=torch.float32).pin_memory()
        e2e_s, mass_e2e = None, None
        if not args.no_e2e:
            barrier()
            t0 = time.perf_counter()
            s.set_state(x0_host)
            s.step(args.steps)
            s.moments(x_host)
            mass_e2e = s.mass()
            barrier()
            e2e_s = time.perf_counter() - t0

    t_ms = ms
    e2e_ms = e2e_s * 1e3 if e2e_s is not None else float("nan")
    if dist is not None:
        tt = torch.tensor([ms, e2e_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_ms, e2e_ms = tt.tolist()
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    updates = float(S_EVOLVED) * cells * args.steps * world
    glups = updates / (t_ms * 1e-3) / 1e9
    bytes_per_launch = 2.0 * S_EVOLVED * Q * 4 * cells
    launch_s = t_ms * 1e-3 / args.steps
    achieved = bytes_per_launch / launch_s / 1e9
    peak, peak_kind = hbm_peak()
    traffic = measured_traffic()
    out = {
        "metric": METRIC,
        "value": round(glups, 4),
        "unit": "GLUPS",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": round(t_ms / args.steps, 6),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic (seeded two-bulb tanh profile; no dataset)",
        "config": {
            "workload": WORKLOAD if NX == 256 else WORKLOAD.replace("256^3", "%d^3" % NX),
            "lattice": "D3Q7", "grid": [NX, NY, NZ], "n_species": N_SPECIES,
            "evolved_species": S_EVOLVED, "bc": "no-flux all faces",
            "relax": "MRT, Lambda_2 by Eq. 3-16",
            "glups_n_counted": round(glups * N_SPECIES / S_EVOLVED, 4),
            "l2": "state %.2f GB per step vs 129 MB L2; no flush" % (2 * S_EVOLVED * Q * 4 * NX * NY * NZ / 1e9),
            "parallelism": "replicas" if world > 1 else "single GPU",
        },
        "roofline": {
            "bound": "hbm",
            "achieved": round(achieved, 1),
            "peak": peak,
            "unit": "GB/s",
            "frac": round(achieved / peak, 4),
            "traffic": traffic,
            "peak_source": peak_kind,
            "algorithmic_bytes_per_launch": bytes_per_launch,
        },
        "e2e": None if args.no_e2e else {
            "value": round(updates / (e2e_ms * 1e-3) / 1e9, 4),
            "unit": "GLUPS",
            "h2d_bytes_per_step": round(x0_host.numel() * 4 / args.steps, 1),
            "d2h_bytes_per_step": round((x_host.numel() * 4 + 8 * N_SPECIES) / args.steps, 1),
        },
        "gpu_launches": args.steps + 1,
        "clocks": clocks,
        "status_flags": flags,
        "mass_drift_rel": float(np.max(np.abs(mass - mass0) / np.abs(mass0))),
    }
    if world == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(budget_s=args.cpu_budget)
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


def _oracle_sample_run(cells_target: int, steps: int):
    """Time the oracle on a slab of the workload with about cells_target nodes."""
    import numpy as np

    import oracle
    import synthetic as sy

    ny = max(1, min(NY, cells_target // NX))
    nz = max(1, min(NZ, cells_target // (NX * ny)))
    x0 = sy.two_bulb(NX, ny, nz, width=4.0)
    t0 = time.perf_counter()
    oracle.run("D3Q7", diffusivities(), x0, steps, bc=("noflux",) * 6)
    dt = time.perf_counter() - t0
    return dt, (NX, ny, nz)


def cpu_baseline(budget_s: float = 20.0):
    """The oracle as it stands, timed on the host cores over a bounded sample."""
    import oracle

    oracle.build()
    dt1, _ = _oracle_sample_run(NX * NY, 1)
    rate = NX * NY / dt1  # node updates per second
    cells_full = NX * NY * NZ
    if rate * budget_s >= cells_full:
        cells = cells_full
        steps = int(max(1, min(50, rate * budget_s / cells_full)))
    else:
        cells, steps = int(max(NX, rate * budget_s)), 1
    dt, shape = _oracle_sample_run(cells, steps)
    n = shape[0] * shape[1] * shape[2]
    return {
        "value": round(S_EVOLVED * n * steps / dt / 1e9, 6),
        "unit": "GLUPS",
        "cores": oracle.get_threads(),
        "kind": "oracle",
        "sample": "%d step(s) on a %dx%dx%d block of the closed tube (FP64 oracle, OpenMP), %.1f s"
                  % (steps, shape[0], shape[1], shape[2], dt),
    }


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import oracle

    oracle.build()
    budget = args.cpu_budget * 4
    dt, _ = _oracle_sample_run(NX * 16, 1)
    rate = NX * 16 / dt
    cells = int(max(NX, min(NX * NY * NZ, rate * budget / max(1, args.steps + args.warmup))))
    _oracle_sample_run(cells, args.warmup) if args.warmup else None
    dt, shape = _oracle_sample_run(cells, args.steps)
    n = shape[0] * shape[1] * shape[2]
    glups = S_EVOLVED * n * args.steps / dt / 1e9
    sample = ("%d timed steps (after %d warm-up) on a %dx%dx%d slab of the closed tube, FP64 "
              "oracle, %.1f s" % (args.steps, args.warmup, shape[0], shape[1], shape[2], dt))
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
        "data": "synthetic (seeded two-bulb tanh profile; no dataset)",
        "config": {"workload": WORKLOAD, "lattice": "D3Q7", "grid": [NX, NY, NZ],
                   "n_species": N_SPECIES},
        "cpu_baseline": {"value": round(glups, 6), "unit": "GLUPS", "cores": oracle.get_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(glups, 6), "unit": "GLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--cpu-budget", type=float, default=20.0,
                    help="seconds of oracle work for the CPU baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end run")
    ap.add_argument("--grid", type=int, default=256,
                    help="edge of the cubic grid (256 is the benchmarked workload)")
    args = ap.parse_args()
    global NX, NY, NZ
    NX = NY = NZ = args.grid
    if args.warmup < 3:
        ap.error("--warmup must be at least 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
