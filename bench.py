"""Throughput of the fused reactive lattice Boltzmann step on GB300.

Workload (default ``--workload sweep``): the batched sweep, 512 capillaries
(widths 16-128, lengths 1024-4096, k_r log-uniform on [1e-5, 1e-2],
contact angles 20-60 degrees, tau_A / tau_B in [0.6, 1.5]; about 1e8 nodes)
advanced together, one launch per step.  A step is one pass of the whole
hot path over every node of every capillary.  The population state is far
larger than L2 (about 17 GB in FP32), so no L2 flush is needed between
steps.

Prints one JSON line: GLUPS (fluid-node updates per second / 1e9) of the
headline storage precision, the roofline of the step kernel, the FP64
oracle's throughput on the host as a baseline, and the same metric end to
end through the C ABI with host buffers.

    python bench.py [--gpus N] [--steps K] [--warmup W]
                    [--precision fp16|fp32] [--workload sweep|paper|preform]
    python bench.py --impl reference ...   # the FP64 oracle on host cores
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

METRIC = "reactive 2-comp LB GLUPS & % HBM roofline, mixed vs FP32 at stated error"

#: algorithmic bytes per fluid-node update: each of the 22 populations (18
#: D2Q9, 4 D2Q4) read once and written once at the storage precision, the
#: mask byte read once -- FP32: 22 x 4 B x 2 + 1 = 177; 16-bit storage:
#: 22 x 2 B x 2 + 1 = 89.  The roofline's `achieved` uses these.
BYTES_PER_NODE = {"fp32": 177.0, "fp16": 89.0, "bf16": 89.0}
#: bytes the layout actually stores and reloads per fluid-node update
#: (reported beside the algorithmic count): FP16 storage keeps 15 32-bit
#: words per node (8 half2 A/B deviation pairs, 2 half2 solute pairs, 2
#: half2 linear-reference pairs, 3 FP32 references), read and written:
#: 120 B, + 1 mask byte.
STORED_BYTES_PER_NODE = {"fp32": 177.0, "fp16": 121.0, "bf16": 121.0}
#: deposit read + write (FP64) at reacting (surface) nodes, per such node
DEPOSIT_BYTES = 16.0
#: DRAM bytes read + written per fluid-node update by the step kernel
#: (default tiles: 64 x 8 FP32, 64 x 4 FP16), from one ncu capture (dram__bytes_read.sum +
#: dram__bytes_write.sum) of the first 40 capillaries of the sweep -- the
#: 512-capillary state is too large to capture; traffic scales with the
#: fluid nodes a launch updates.  Reported for the sweep at the default
#: tile only.
TRAFFIC_PER_FLUID_NODE = {"fp32": 187.61, "fp16": 126.32, "bf16": None}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed
    region (every 200 ms)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,"
              "clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu),
                 "--query-gpu=" + self.FIELDS, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE,
                stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [],
                    "samples": 0}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown",
                 "sw_power_cap")
        for line in self.lines:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def build_workload(name: str, rank: int = 0, lattices: int = 512):
    from paper_1309_6726_gb300 import inputs as I
    if name == "sweep":
        members = I.sweep_members(512, seed=1236 + 1000 * rank)[:lattices]
        pairs = [I.sweep_lattice(m) for m in members]
        geoms = [g for g, _ in pairs]
        params = [p for _, p in pairs]
        desc = ("batched sweep: %d capillaries, W 16-128, L 1024-4096, "
                "k_r logU[1e-5,1e-2], theta 20-60 deg, tau_A/tau_B 0.6-1.5"
                % len(geoms))
    elif name == "paper":
        g, p, _ = I.config_paper_scale(k_r=1e-3)
        geoms, params = [g], [p]
        desc = "single capillary 4096x128, k_r 1e-3"
    elif name == "preform":
        g, p, _ = I.config_preform()
        geoms, params = [g], [p]
        desc = "disc preform 2048x2048, porosity 0.5, k_r 1e-3"
    else:
        raise SystemExit("unknown workload " + name)
    return geoms, params, desc


def fluid_nodes(geoms) -> int:
    return int(sum(int((g.solid == 0).sum()) for g in geoms))


def all_nodes(geoms) -> int:
    return int(sum(g.solid.size for g in geoms))


def surface_fraction(geoms) -> float:
    """Fluid nodes with a solid D2Q4 neighbour / fluid nodes (the nodes whose
    deposit the reaction may read and write)."""
    surf = 0
    for g in geoms:
        s = g.solid.astype(bool)
        nb = np.zeros_like(s)
        for dy, dx in ((0, 1), (1, 0), (0, -1), (-1, 0)):
            nb |= np.roll(s, (dy, dx), axis=(0, 1))
        surf += int((nb & ~s).sum())
    return surf / max(1, fluid_nodes(geoms))


def combine_ranks(ms: float, n_fluid: int, device) -> tuple[float, float]:
    """Across the ranks of the process group: the slowest rank's timed
    region (max) and the fluid nodes all ranks updated per step (sum)."""
    import torch
    import torch.distributed as td
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    td.all_reduce(t, op=td.ReduceOp.MAX)
    n = torch.tensor([float(n_fluid)], dtype=torch.float64, device=device)
    td.all_reduce(n)
    return float(t.item()), float(n.item())


def time_gpu(geoms, params, precision, steps, warmup, dist):
    import torch
    from paper_1309_6726_gb300 import lbm
    s = lbm.Solver(geoms, params, precision)
    # a stream of torch's (never the legacy default stream): the events below
    # are recorded on the stream the step kernels are launched on
    stream = torch.cuda.Stream()
    s.set_stream(stream.cuda_stream)
    s.step(warmup)
    torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    s.step(steps)
    e1.record(stream)
    torch.cuda.synchronize()
    if dist:
        torch.distributed.barrier()
    ms = e0.elapsed_time(e1)
    obs = s.observables(allow_nan=True)
    s.set_stream(None)
    s.close()
    return ms, obs


def pinned(geoms):
    """The geometries with their arrays copied into pinned (page-locked)
    host memory, where a job keeps the inputs it streams to the GPU."""
    import dataclasses
    import torch
    out = []
    for g in geoms:
        pin = {k: torch.from_numpy(np.ascontiguousarray(getattr(g, k), t))
               .pin_memory().numpy()
               for k, t in (("solid", np.uint8), ("rho_a", np.float32),
                            ("rho_b", np.float32), ("conc", np.float32))}
        out.append(dataclasses.replace(g, **pin))
    return out


def time_e2e(geoms, params, precision, steps, observe_every):
    """Whole job through the C ABI with host buffers: create (host->device
    copy of geometry and initial fields from pinned host memory), steps,
    observables read back every `observe_every` steps and at the end, final
    solid masks of every lattice read back (one call, into pinned host
    memory)."""
    import torch
    from paper_1309_6726_gb300 import lbm
    geoms = pinned(geoms)
    # the masks come back into pinned memory, as the inputs go from it
    masks = torch.empty(sum(g.solid.size for g in geoms), dtype=torch.uint8,
                        pin_memory=True).numpy()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s = lbm.Solver(geoms, params, precision)
    n_obs = 0
    done = 0
    while done < steps:
        k = min(observe_every, steps - done)
        s.step(k)
        done += k
        s.observables_array(allow_nan=True)
        n_obs += 1
    s.solid_masks(out=masks)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    s.close()
    h2d = sum(g.solid.size * (1 + 4 * 3) for g in geoms)
    d2h = n_obs * 144 * len(geoms) + sum(g.solid.size for g in geoms)
    return dt, h2d, d2h


def cpu_baseline(geoms, params, budget_s: float = 12.0):
    """The FP64 oracle, as it stands, on this host: one capillary of the
    workload stepped until about `budget_s` seconds have passed."""
    from oracle.lattice import Lattice, Params
    # the capillary nearest the workload's mean size
    sizes = np.array([g.solid.size for g in geoms])
    k = int(np.argmin(np.abs(sizes - sizes.mean())))
    g, p = geoms[k], params[k]
    lat = Lattice(Params(**p.as_dict(), cap_x0=g.cap_x0, cap_x1=g.cap_x1),
                  g.solid, g.rho_a, g.rho_b, g.conc)
    lat.step(1)
    steps = 0
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < budget_s:
        lat.step(5)
        steps += 5
    dt = time.perf_counter() - t0
    fl = int((g.solid == 0).sum())
    return {"value": fl * steps / dt / 1e9, "unit": "GLUPS", "cores": 1,
            "kind": "oracle",
            "sample": "capillary %d (%dx%d) of the workload, %d steps, "
                      "%.1f s, single thread FP64" % (k, g.nx, g.ny, steps, dt)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    geoms, params, desc = build_workload(args.workload, 0, args.lattices)
    times = []
    from oracle.lattice import Lattice, Params
    sizes = np.array([g.solid.size for g in geoms])
    k = int(np.argmin(np.abs(sizes - sizes.mean())))
    g, p = geoms[k], params[k]
    lat = Lattice(Params(**p.as_dict(), cap_x0=g.cap_x0, cap_x1=g.cap_x1),
                  g.solid, g.rho_a, g.rho_b, g.conc)
    fl = int((g.solid == 0).sum())
    per_step = 3
    for _ in range(args.warmup):
        lat.step(per_step)
    for _ in range(args.steps):
        t0 = time.perf_counter()
        lat.step(per_step)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = fl * per_step * args.steps / total / 1e9
    sample = ("capillary %d (%dx%d) of the workload, %d oracle steps per "
              "bench step, single thread FP64" % (k, g.nx, g.ny, per_step))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value,
        "unit": "GLUPS", "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": desc, "lattices": len(geoms),
                   "fluid_nodes": fluid_nodes(geoms),
                   "all_nodes": all_nodes(geoms),
                   "parallelism": "host oracle, one capillary per step"},
        "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": 1,
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--precision", default="fp16", choices=["fp16", "bf16", "fp32"])
    ap.add_argument("--compare", default="fp32",
                    help="second precision timed for the mixed-vs-FP32 ratio"
                         " ('none' to skip)")
    ap.add_argument("--workload", default="sweep",
                    choices=["sweep", "paper", "preform"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=50)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--lattices", type=int, default=512,
                    help="sweep only: the first N capillaries (a smaller "
                         "case for profiling; the benchmark is N = 512)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = world > 1
    if dist:
        torch.distributed.init_process_group("nccl")
    torch.cuda.set_device(local)
    import __graft_entry__
    if rank == 0 or not dist:
        __graft_entry__.build()
    if dist:
        torch.distributed.barrier()
    __graft_entry__.build()

    geoms, params, desc = build_workload(args.workload, rank, args.lattices)
    n_fluid = fluid_nodes(geoms)
    n_all = all_nodes(geoms)
    f_s = surface_fraction(geoms)

    clocks = ClockSampler(local)
    clocks.start()
    ms, obs = time_gpu(geoms, params, args.precision, args.steps,
                       args.warmup, dist)
    clk = clocks.stop()
    if dist:
        ms, n_fluid_all = combine_ranks(ms, n_fluid, "cuda")
    else:
        n_fluid_all = float(n_fluid)
    ms_step = ms / args.steps
    glups = n_fluid_all * args.steps / (ms / 1e3) / 1e9
    compare = None
    if args.compare not in ("none", args.precision):
        ms2, _ = time_gpu(geoms, params, args.compare, args.steps,
                          args.warmup, dist)
        g2 = n_fluid * args.steps / (ms2 / 1e3) / 1e9
        compare = {"precision": args.compare, "glups_per_gpu": g2,
                   "ms_per_step": ms2 / args.steps,
                   "speedup_of_headline": (n_fluid * args.steps / (ms / 1e3)
                                           / 1e9) / g2}
    peak, peak_kind = load_peaks()
    traffic = None
    per_node = TRAFFIC_PER_FLUID_NODE[args.precision]
    if (args.workload == "sweep" and not os.environ.get("LBM_TILE")
            and per_node is not None):
        traffic = per_node * n_fluid
    bpn = BYTES_PER_NODE[args.precision] + DEPOSIT_BYTES * f_s
    stored = STORED_BYTES_PER_NODE[args.precision] + DEPOSIT_BYTES * f_s
    achieved = n_fluid * bpn / (ms_step / 1e3) / 1e9
    e2e = None
    if rank == 0 and args.e2e_steps > 0:
        dt, h2d, d2h = time_e2e(geoms, params, args.precision, args.e2e_steps,
                                observe_every=10)
        e2e = {"value": n_fluid * args.e2e_steps / dt / 1e9 * world,
               "unit": "GLUPS",
               "h2d_bytes_per_step": h2d / args.e2e_steps,
               "d2h_bytes_per_step": d2h / args.e2e_steps,
               "steps": args.e2e_steps}
    cpu = None
    if rank == 0 and not dist and not args.no_cpu_baseline:
        cpu = cpu_baseline(geoms, params)
    nonfinite = sum(1 for o in obs if o["nonfinite"])
    if rank == 0:
        line = {
            "metric": METRIC, "value": glups, "unit": "GLUPS",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "storage": args.precision, "data": "synthetic",
            "config": {"workload": desc, "lattices": len(geoms),
                       "fluid_nodes": n_fluid, "all_nodes": n_all,
                       "glups_all_nodes": glups * n_all / n_fluid,
                       "l2": "state > L2 (no flush needed)",
                       "parallelism": "dp%d (independent capillaries)" % world},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak,
                         "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind, "traffic": traffic,
                         "bytes_per_fluid_node": bpn,
                         "stored_bytes_per_fluid_node": stored,
                         "traffic_over_algorithmic":
                             None if traffic is None
                             else traffic / (n_fluid * bpn),
                         "kernel": "k_step_tma (one launch per step)"},
            "compare": compare,
            "cpu_baseline": cpu, "e2e": e2e, "clocks": clk,
            "gpu_launches": args.steps,
            "lattices_nonfinite": nonfinite,
        }
        print(json.dumps(line))
    if dist:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
