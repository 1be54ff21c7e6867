#!/usr/bin/env python3
"""Benchmark of the Maxwell–Bloch FDTD step: Mcell-updates/s and HBM GB/s.

Workload: one active realization of the paper-scale sample, a 320^3 Yee grid
(6.4 um box, dx = 20 nm, Courant 0.99, 8-cell CPML) holding ~8100 TiO2
spheres (d ~ normal(300 nm, 10 %), 45 % fill) with the gain medium in the
voids, N_a = 5e24 m^-3 pumped at W_p = 1e13 /s, Langevin noise on, a centre
point probe and six face probes (128 bins, 475-705 nm).  A "step" is one
full time step: H pass, fused E / gain / noise / population pass (with the
face flux), point-probe DFT, face-probe DFT.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun, one rank per GPU) every rank advances its own
realization (different disorder and noise seeds): weak scaling, no
collective on the data path; the barrier and the max over ranks of the
timed region are the only communication.  Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "MB-FDTD Mcell-updates/s & HBM GB/s at 320^3; batched and adjoint vs plain step"
UNIT = "Mcell-updates/s"
FALLBACK_HBM_GBS = 6800.0
PROFILE_DIR = os.path.join(ROOT, "profiles")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_0809_1547_gb300", "csrc", f)
                  for f in ("mb_device.cuh", "mb_tiles.cuh", "mb_passes.cu", "mb_tma.cuh",
                            "mb_fused.cu")]


# ------------------------------------------------------------------ helpers

def kernel_source_hash() -> str:
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(p, "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def algorithmic_bytes(w):
    """Algorithmic bytes per cell of one step (perfect neighbour reuse), per launch.

    H launch (H half-step + Lorentz/Langevin update of the gain cells): read E
    and H, write H (36 B); per CPML slab axis the cell lies in, read+write two
    psi_H (16 B); gain cells read+write P and J and read n1, n2 (56 B).
    E launch (E update + populations): read H and E, write E, read the
    material byte (37 B); per slab axis two psi_E (16 B); gain cells read J
    and read+write n1..n3 (36 B).
    Two-pass minimum of the whole step (the two launches above with E^n read
    once by the gain work): 73 B + 32 B per slab axis + 72 B per gain cell.
    Single-pass step (one launch per step): read E and H, write E and H to
    the other copy, read the material byte (49 B); per slab axis four psi
    read+write (32 B); gain cells read+write P, J and n1..n3 (72 B).
    """
    import numpy as np
    L = w.npml
    n = w.grid
    slab = sum(min(2 * L, nw) / nw for nw in n)   # sum over axes of the slab fraction
    g = float(np.mean(w.gain != 0)) if w.N_a > 0 else 0.0
    h_launch = 36.0 + 16.0 * slab + 56.0 * g
    e_launch = 37.0 + 16.0 * slab + 36.0 * g
    two_pass = 73.0 + 32.0 * slab + 72.0 * g
    single = 49.0 + 32.0 * slab + 72.0 * g
    # the step's reference byte count: two passes with perfect neighbour
    # reuse, all four populations stored, 64 B per slab axis
    reference = 73.0 + 80.0 * g + 64.0 * slab
    return {"h_launch": h_launch, "e_launch": e_launch, "step_two_pass_minimum": two_pass,
            "single_pass_launch": single, "step_reference": reference, "gain_fraction": g,
            "slab_fraction_sum": slab}


def traffic_from_profile(kernel: str, workload: str = "mb320_active"):
    """DRAM bytes per launch of `kernel` on `workload` from the committed ncu
    summary profiles/<kernel>_traffic_<workload>.md, if it was taken on the
    current kernel sources (else None)."""
    import re
    try:
        with open(os.path.join(PROFILE_DIR, f"{kernel}_traffic_{workload}.md")) as f:
            text = f.read()
        h = re.search(r"kernel_source_hash:\s*(\w+)", text).group(1)
        if h != kernel_source_hash():
            return None
        return float(re.search(r"bytes_per_launch_full_size:\s*([0-9.eE+]+)", text).group(1))
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms."""
    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is not None:
            time.sleep(0.15)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 10:
                        rows.append(parts)
        except Exception:
            pass
        finally:
            if self.path and os.path.exists(self.path):
                os.unlink(self.path)
        return rows

    @staticmethod
    def summarize(rows, t0, t1):
        from datetime import datetime
        sel = []
        for r in rows:
            try:
                ts = datetime.strptime(r[0], "%Y/%m/%d %H:%M:%S.%f").timestamp()
            except Exception:
                continue
            if t0 - 0.05 <= ts <= t1 + 0.05:
                sel.append(r)
        window = "timed region"
        if not sel:
            sel, window = rows, "whole run (no sample fell inside the timed region)"
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"],
                    "samples": 0}

        def num(x):
            try:
                return float(x)
            except Exception:
                return None
        sm = [num(r[2]) for r in sel if num(r[2]) is not None]
        smax = [num(r[3]) for r in sel if num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[q] for r in sel for q in range(4) if r[6 + q].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": reasons,
                "samples": len(sel), "window": window,
                "power_w_max": max((num(r[4]) or 0.0) for r in sel)}


# ---------------------------------------------------------- distributed glue

def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def init_dist(world, backend):
    if world > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            dist.init_process_group(backend=backend)


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int, device=None) -> float:
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_workload(rank: int, n: int = 320):
    """Rank r runs its own realization: disorder seed 7 + r, noise seed + r."""
    from paper_0809_1547_gb300 import inputs
    w = inputs.workload_paper(n, seed=7 + rank)
    w.seed = w.seed + rank
    return w


# ------------------------------------------------------------- CPU baseline
# The oracle is plain FP64 numpy on one thread.  It is timed on the host's
# cores by one child process per core, each stepping its own part of the
# workload (a slab of z-planes at its own depth, or one member of the
# ensemble) with the workload's materials, gain, pump and noise seed and an
# 8-cell CPML on the part's own faces.  The children set up, report ready,
# and start their timed steps together; the rate is the cells x steps of all
# children over the longest child's time.

def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def save_part(w, directory: str, tag: str, z0: int = 0, thickness: int | None = None,
              rows: int | None = None) -> str:
    """Planes z0 .. z0+thickness-1 of workload w (all of it by default) with
    its parameters, as an .npz an oracle child reads; with `rows`, only the
    middle `rows` rows (y) of those planes."""
    import numpy as np
    t = w.grid[2] - z0 if thickness is None else thickness
    r = w.grid[1] if rows is None else rows
    y0 = (w.grid[1] - r) // 2
    path = os.path.join(directory, f"{tag}.npz")
    np.savez(path, eps=np.ascontiguousarray(w.eps[z0:z0 + t, y0:y0 + r]),
             gain=np.ascontiguousarray(w.gain[z0:z0 + t, y0:y0 + r]),
             real=np.array([w.dx, w.dt, w.N_a, w.pump], dtype=np.float64),
             npml=np.array([w.npml], dtype=np.int64), seed=np.array([w.seed], dtype=np.uint64))
    return path


def oracle_child(path: str, steps: int, warm: int, kind: str):
    """One oracle child (one BLAS thread): set up the part at `path`, print
    'ready', wait for a line on stdin, time `steps` forward steps (kind
    'forward') or one adjoint gradient over `steps` steps (kind 'adjoint'),
    print [cells, seconds]."""
    import numpy as np
    from oracle.mb_oracle import MBOracle, Params
    d = np.load(path)
    eps, gain = d["eps"], d["gain"]
    dx, dt, N_a, pump = (float(v) for v in d["real"])
    nz, ny, nx = eps.shape
    o = MBOracle((nx, ny, nz), dx, dt, Params(npml=int(d["npml"][0])))
    o.set_material(eps, gain, N_a, pump)
    o.set_seed(int(d["seed"][0]))
    o.add_point_probe((nx // 2, ny // 2, nz // 2), 128, 475e-9, 705e-9)
    if kind == "forward" and warm > 0:
        o.step(warm)
    print("ready", flush=True)
    sys.stdin.readline()
    t = time.perf_counter()
    if kind == "adjoint":
        from oracle import mb_adjoint
        mb_adjoint.adjoint_energy_zface(o, steps)
    else:
        o.step(steps)
    el = time.perf_counter() - t
    print(json.dumps([nx * ny * nz, el]), flush=True)


def run_oracle_children(jobs, timeout: float = 1200.0):
    """jobs: [(path, steps, warm, kind)], one child each, all at once.
    Returns (Mcell-updates/s of all children together, the longest child's
    seconds, [(cells, seconds)] per child)."""
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    procs, res = [], []
    try:
        for path, steps, warm, kind in jobs:
            code = (f"import sys; sys.path.insert(0, {ROOT!r}); import bench; "
                    f"bench.oracle_child({path!r}, {int(steps)}, {int(warm)}, {kind!r})")
            procs.append(subprocess.Popen([sys.executable, "-c", code], stdin=subprocess.PIPE,
                                          stdout=subprocess.PIPE, stderr=subprocess.PIPE,
                                          text=True, env=env))
        for p in procs:
            if p.stdout.readline().strip() != "ready":
                p.wait(timeout=60)
                raise RuntimeError("oracle child failed: " + p.stderr.read()[-1500:])
        for p in procs:
            p.stdin.write("go\n")
            p.stdin.flush()
        for p in procs:
            out, err = p.communicate(timeout=timeout)
            if p.returncode != 0:
                raise RuntimeError("oracle child failed: " + err[-1500:])
            res.append(json.loads(out.strip().splitlines()[-1]))
    finally:
        for p in procs:
            if p.poll() is None:
                p.kill()
    work = sum(c * j[1] for (c, _), j in zip(res, jobs))
    secs = max(el for _, el in res)
    return work / secs / 1e6, secs, res


def slab_offsets(n: int, thickness: int, parts: int):
    """z0 of `parts` slabs of `thickness` planes spread over 0 .. n - thickness."""
    top = max(0, n - thickness)
    return [round(q * top / max(1, parts - 1)) for q in range(parts)]


def cpu_slab_rate(w, thickness: int, steps: int, warm: int = 1, cores: int | None = None,
                  kind: str = "forward", rows: int | None = None):
    """The oracle on `cores` slabs (thickness planes each, all rows or the
    middle `rows`) of workload w, one child per core."""
    cores = cores or host_cores()
    with tempfile.TemporaryDirectory() as d:
        jobs = [(save_part(w, d, f"slab{q}", z0, thickness, rows), steps, warm, kind)
                for q, z0 in enumerate(slab_offsets(w.grid[2], thickness, cores))]
        rate, secs, res = run_oracle_children(jobs)
    return rate, secs, res[0][0], cores


def cpu_baseline(w, cores: int | None = None, thickness: int = 32, steps: int = 12):
    """The headline oracle rate: slabs of the benchmark's own workload on every host core."""
    rate, secs, cells, cores = cpu_slab_rate(w, thickness, steps, 1, cores)
    return {"value": round(rate, 3), "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{cores} slabs of {w.grid[0]}x{w.grid[1]}x{thickness} planes ({cells} cells "
                      f"each, spread over the depth) of the {w.name} workload, each with its own "
                      f"8-cell CPML, stepped {steps} times (after 1 warm-up) by the FP64 numpy oracle "
                      f"in {cores} single-thread processes at once; {secs:.1f} s"}


def cpu_baseline_configs(cores: int | None = None):
    """The oracle on the other configurations, each on every host core
    (except the 48^3 run, one realization on one core)."""
    from paper_0809_1547_gb300 import inputs
    cores = cores or host_cores()
    out = {}
    w = inputs.workload_small_48()
    with tempfile.TemporaryDirectory() as d:
        rate, secs, res = run_oracle_children([(save_part(w, d, "w48"), w.steps, 0, "forward")])
    out["small_48_full"] = {"value": round(rate, 3), "unit": UNIT, "cores": 1,
                            "sample": f"the whole 48^3 workload, all {w.steps} steps, one process; "
                                      f"{secs:.1f} s"}
    w = inputs.workload_large_448()
    rate, secs, cells, _ = cpu_slab_rate(w, 24, 8, 1, cores)
    out["large_448"] = {"value": round(rate, 3), "unit": UNIT, "cores": cores,
                        "sample": f"{cores} slabs of 448x448x24 ({cells} cells each), 8 steps; {secs:.1f} s"}
    ws = inputs.workload_batch()
    with tempfile.TemporaryDirectory() as d:
        jobs = [(save_part(ws[q], d, f"m{q}"), 6, 1, "forward") for q in range(min(cores, len(ws)))]
        rate, secs, res = run_oracle_children(jobs)
    out["batched_members"] = {"value": round(rate, 3), "unit": UNIT, "cores": len(jobs),
                              "sample": f"the first {len(jobs)} ensemble members (whole grids of "
                                        f"{sorted({ws[q].grid[0] for q in range(len(jobs))})} cells "
                                        f"per side), one per process, 6 steps each; {secs:.1f} s"}
    w = inputs.workload_adjoint_96()
    rate, secs, cells, _ = cpu_slab_rate(w, 24, 10, 0, cores, kind="adjoint")
    out["adjoint_96"] = {"value": round(rate, 3), "unit": UNIT, "cores": cores,
                         "sample": f"{cores} slabs of 96x96x24 ({cells} cells each) of the adjoint "
                                   f"workload, one gradient over 10 steps each by the FP64 oracle "
                                   f"adjoint (forward with every state kept + reverse sweep); "
                                   f"{secs:.1f} s"}
    return out


# --------------------------------------------------------------- our arm

def bench_ours(args):
    import numpy as np
    import torch
    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    init_dist(world, "nccl")
    from paper_0809_1547_gb300 import build
    if rank == 0:
        build.build()
    barrier(world)
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params
    from paper_0809_1547_gb300.workloads import setup_simulation
    w = rank_workload(rank, args.grid)
    stream = torch.cuda.Stream()
    sim = setup_simulation(w, autotune=not args.tune, stream=stream.cuda_stream)
    if args.tune:
        th, te = (tuple(int(v) for v in part.split(",")) for part in args.tune.split(":"))
        sim.set_tuning(th, te)
    if args.single_pass == "off":
        sim.set_single_pass((0, 32, 8, 16))
    elif args.single_pass:
        sim.set_single_pass((1,) + tuple(int(v) for v in args.single_pass.split(",")))
    single = sim.single_pass()
    per_step_launches, _ = sim.launch_stats()
    blk_h, blk_e = sim.tuning()
    sim.step(args.warmup)
    sim.synchronize()
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    barrier(world)
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    t_host0 = time.time()
    ev0.record(stream)
    sim.step(args.steps)                          # the production path: CUDA-graph replay
    sim.join_probes()                             # the last steps' probe DFTs inside the region
    ev1.record(stream)
    torch.cuda.synchronize()
    t_host1 = time.time()
    barrier(world)
    clock_rows = sampler.stop()
    elapsed_ms = ev0.elapsed_time(ev1)
    elapsed_ms = max_over_ranks(elapsed_ms, world, device=torch.device("cuda", local))

    # per-launch device times (direct launches with CUDA events around each
    # launch) on the same state, for the roofline of each kernel
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    pass_ms = sim.step_timed(args.steps)
    g1.record(stream)
    torch.cuda.synchronize()
    direct_ms_per_step = g0.elapsed_time(g1) / args.steps
    U, fl = sim.energy()
    sim.close()

    cells = w.ncell
    value = cells * args.steps * world / (elapsed_ms / 1e3) / 1e6
    ab = algorithmic_bytes(w)
    peak, peak_kind = measured_peaks()
    h_avg_ms = pass_ms[0] / args.steps
    e_avg_ms = pass_ms[1] / args.steps
    if single[0]:
        # steps run in pairs of single-pass launches (an odd K ends with one two-pass step)
        n_single = args.steps - args.steps % 2
        launches = {"k_step_fused (H half-step + Lorentz/Langevin + E + populations + face flux, "
                    "one launch per step)": (h_avg_ms * args.steps / max(n_single, 1),
                                             ab["single_pass_launch"], "k_step_fused")}
    else:
        launches = {"k_hg (H half-step + gain-cell Lorentz/Langevin)": (h_avg_ms, ab["h_launch"], "k_hg"),
                    "k_e (E update + populations + face flux)": (e_avg_ms, ab["e_launch"], "k_e")}
    dom_name = max(launches, key=lambda k: launches[k][0])
    dom_ms, dom_bpc, dom_key = launches[dom_name]
    dom_bytes = dom_bpc * cells
    achieved = dom_bytes / (dom_ms / 1e3) / 1e9
    traffic = traffic_from_profile(dom_key, w.name) if args.grid == 320 else None
    step_ms = elapsed_ms / args.steps
    other = {k: {"avg_launch_ms": round(v[0], 5), "bytes_per_cell": round(v[1], 2),
                 "achieved_gbs": round(v[1] * cells / (v[0] / 1e3) / 1e9, 1)}
             for k, v in launches.items()}

    # end to end through the public API with host buffers: material upload
    # (host -> device), K steps each followed by a read of the six face
    # energies (device -> host, 48 bytes into pinned memory, consumed on the
    # host one step later while the next step runs), the final spectrum read.
    # the host buffers are page-locked (pinned), as a user streaming inputs
    # to the GPU would hold them
    eps_pin = torch.from_numpy(np.ascontiguousarray(w.eps, dtype=np.float32)).pin_memory()
    gain_pin = torch.from_numpy(np.ascontiguousarray(w.gain, dtype=np.uint8)).pin_memory()
    eps_h, gain_h = eps_pin.numpy(), gain_pin.numpy()
    sim2 = MBSimulation(w.grid, w.dx, w.dt, mb_default_params(npml=w.npml), stream=stream.cuda_stream)
    pid = sim2.add_point_probe(w.extra.get("probe", (160, 160, 160)), 128, 475e-9, 705e-9)
    sim2.add_face_probes(8, 4, 128, 475e-9, 705e-9)
    sim2.set_material(eps_h, gain_h, w.N_a, w.pump)
    sim2.set_seed(w.seed)
    # the launch shapes the timed run was tuned to (set-up, like the graphs)
    sim2.set_tuning(blk_h, blk_e)
    if single[0]:
        sim2.set_single_pass(single)
    sim2.step(2)          # graph capture outside the timed region
    sim2.set_material(eps_h, gain_h, w.N_a, w.pump)
    sim2.synchronize()
    barrier(world)
    bufs = [torch.zeros(6, dtype=torch.float64).pin_memory() for _ in range(2)]
    evs = [torch.cuda.Event() for _ in range(2)]
    # the loop's host-side calls once before the timed region (first-use
    # initialisation of the read-back path and of the host sum)
    sim2.flux_async(bufs[0])
    evs[0].record(stream)
    evs[0].synchronize()
    float(bufs[0].sum())
    sim2.probe_spectrum(pid)
    emitted = []
    t0 = time.perf_counter()
    sim2.set_material(eps_h, gain_h, w.N_a, w.pump)
    for q in range(args.steps):
        sim2.step(1)
        sim2.flux_async(bufs[q % 2])
        evs[q % 2].record(stream)
        if q > 0:
            evs[(q - 1) % 2].synchronize()
            emitted.append(float(bufs[(q - 1) % 2].sum()))
    evs[(args.steps - 1) % 2].synchronize()
    emitted.append(float(bufs[(args.steps - 1) % 2].sum()))
    S, _ = sim2.probe_spectrum(pid)
    t1 = time.perf_counter()
    assert len(emitted) == args.steps and all(np.isfinite(emitted))
    e2e_s = max_over_ranks(t1 - t0, world, device=torch.device("cuda", local))
    sim2.close()
    e2e_value = cells * args.steps * world / e2e_s / 1e6
    h2d = (eps_h.nbytes + gain_h.nbytes) / args.steps
    d2h = 48 + 16 * 3 * 128 / args.steps   # six face energies per step; the probe's bins once

    clocks = ClockSampler.summarize(clock_rows, t_host0, t_host1)
    out = {
        "metric": METRIC, "value": round(value, 2), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(elapsed_ms / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"{w.name}: {w.grid[0]}^3 Yee grid (dx 20 nm, Courant 0.99, 8-cell CPML), "
                               f"{w.n_spheres} TiO2 spheres d~N(300 nm,10%) at {w.fill:.3f} fill, gain in "
                               "the voids, N_a 5e24 m^-3, W_p 1e13/s, Langevin noise, centre point probe "
                               "+ 6 face probes (stride 8, every 4, 128 bins)",
                   "grid": list(w.grid), "cells": cells, "gain_fraction": round(ab["gain_fraction"], 4),
                   "l2": f"inputs larger than L2 (state {61 * cells / 1e9:.2f} GB per realization)",
                   "parallelism": f"replicas x{world} (one realization per GPU)",
                   "timed_path": "mb_step (CUDA-graph replay) bracketed by CUDA events; per-launch "
                                 "times from a second pass of direct launches with events around each",
                   "blocks": {"h_pass": list(blk_h), "e_pass": list(blk_e),
                              "single_pass": list(single)},
                   "direct_launch_ms_per_step": round(direct_ms_per_step, 5)},
        "roofline": {"bound": "hbm", "kernel": dom_name,
                     "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                     "frac": round(achieved / peak, 4), "peak_source": f"{peak_kind} hbm_gbs (of measured)"
                     if peak_kind == "measured" else "fallback 6.8 TB/s (of fallback)",
                     "traffic": traffic, "algorithmic_bytes_per_launch": round(dom_bytes),
                     "fractions": {
                         "own_bytes": round(achieved / peak, 4),
                         "reference_bytes": round(ab["step_reference"] * cells / (dom_ms / 1e3) / 1e9 / peak, 4),
                         "measured_traffic": (round(traffic / (dom_ms / 1e3) / 1e9 / peak, 4)
                                              if traffic else None),
                         "definition": "bytes per launch / the launch's average CUDA-event time / "
                                       "peak: own_bytes with the kernel's own algorithmic bytes "
                                       "(the frac above), reference_bytes with the step's reference "
                                       "count 73 + 80 g + 64 f B/cell, measured_traffic with ncu's "
                                       "DRAM read + write bytes of one launch (traffic)"},
                     "bytes_per_cell": round(dom_bpc, 2), "avg_launch_ms": round(dom_ms, 5),
                     "launches": other,
                     "step": {"single_pass_bytes_per_cell": round(ab["single_pass_launch"], 2),
                              "achieved_gbs": round(ab["single_pass_launch"] * cells / (step_ms / 1e3) / 1e9, 1),
                              "frac": round(ab["single_pass_launch"] * cells / (step_ms / 1e3) / 1e9 / peak, 4),
                              "reference_bytes_per_cell": round(ab["step_reference"], 2),
                              "reference_gbs": round(ab["step_reference"] * cells / (step_ms / 1e3) / 1e9, 1),
                              "reference_frac": round(ab["step_reference"] * cells / (step_ms / 1e3) / 1e9 / peak, 4),
                              "reference_definition": "Mcell-updates/s x (73 + 80 g + 64 f) B/cell / peak: the "
                                                      "two-pass step's bytes with perfect neighbour reuse "
                                                      "(g gain fraction, f summed CPML slab fractions)"},
                     "pass_ms_per_step": [round(v / args.steps, 5) for v in pass_ms]},
        "e2e": {"value": round(e2e_value, 2), "unit": UNIT, "h2d_bytes_per_step": round(h2d, 1),
                "d2h_bytes_per_step": round(d2h, 1)},
        "gpu_launches": int(per_step_launches * args.steps),
        "clocks": clocks,
        "energy_J": U,
    }
    if args.grid == 320:
        out["gp_theory"] = bench_gp()
    if not args.no_large and args.grid == 320:
        out["large_448"] = bench_large(stream, max(50, args.steps // 6), args.warmup)
    if not args.no_passive and args.grid == 320:
        out["passive"] = bench_passive(w, stream, max(50, args.steps // 3), args.warmup)
    if not args.no_batched:
        out["batched"] = bench_batched(stream, args.batched_steps, args.warmup)
    if not args.no_adjoint:
        out["adjoint"] = bench_adjoint(stream, args.warmup)
    if not args.no_split and args.grid == 320:
        out["split_z"] = bench_split(stream, max(50, args.steps // 4), args.warmup)
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.grid == 320:
        try:
            out["cpu_baseline"] = cpu_baseline(w)
        except Exception as e:   # keep the GPU line even if the CPU leg fails
            out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": host_cores(), "kind": "oracle",
                                   "sample": f"failed: {str(e)[-200:]}"}
        if not args.no_cpu_configs:
            try:
                out["cpu_baseline_configs"] = cpu_baseline_configs()
            except Exception as e:
                out["cpu_baseline_configs"] = {"failed": str(e)[-300:]}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


# ------------------------------------------------------ batched ensemble

def bench_batched(stream, steps: int, warmup: int, n_pump: int = 16, n_seed: int = 5,
                  autotune: bool = True, plain: bool = True):
    """The ensemble (16 N_a levels log-spaced 5e23-2e25 m^-3 x 5 disorder
    seeds, cubes of side 96-160, 45 % fill, gain in the voids, a centre probe
    each) advanced by the batched persistent launch, against the plain
    single-context step of the same 80 realizations one after another."""
    import numpy as np
    import torch
    from paper_0809_1547_gb300 import inputs
    from paper_0809_1547_gb300.binding import MBBatch, MBSimulation, mb_default_params, \
        MB_BATCH_PERSISTENT, MB_BATCH_CONCURRENT
    ws = inputs.workload_batch(n_pump=n_pump, n_seed=n_seed)
    p = mb_default_params(npml=ws[0].npml)
    cells = sum(int(np.prod(w.grid)) for w in ws)

    def centre(w):
        return tuple(v // 2 for v in w.grid)

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    b = MBBatch([w.grid for w in ws], ws[0].dx, ws[0].dt, p, stream=stream.cuda_stream)
    for q, w in enumerate(ws):
        b.set_instance(q, w.eps, w.gain, w.N_a, w.pump, w.seed)
        b.instances[q].add_point_probe(centre(w), 128, 475e-9, 705e-9)
    if autotune:
        b.autotune()                   # tile shape, the members' launches and the mode
    picked = b.mode
    # both modes from the same state: the persistent launch (one cooperative
    # launch per graph-replayed chunk, the design the ensemble is specified
    # with) is the headline; the members' own launches on 8 streams beside it
    times = {}
    for mode in (MB_BATCH_PERSISTENT, MB_BATCH_CONCURRENT):
        b.set_mode(mode)
        # warm-up long enough to capture every graph chunk (32 steps
        # persistent, 16 per member concurrent) outside the timed region
        b.step(max(warmup, 32))
        b.synchronize()
        times[mode] = timed(lambda: b.step(steps))
        b.synchronize()
    b.set_mode(MB_BATCH_CONCURRENT)
    launches_concurrent = sum(s_.launch_stats()[0] for s_ in b.instances) * steps
    tune = b.tuning()
    b.close()
    batch_ms = times[MB_BATCH_PERSISTENT]
    mode_name = {MB_BATCH_PERSISTENT: "persistent", MB_BATCH_CONCURRENT: "concurrent"}
    conc_ms = times[MB_BATCH_CONCURRENT]
    other = {"mode": "concurrent", "value": round(cells * steps / (conc_ms / 1e3) / 1e6, 2),
             "unit": UNIT, "ms_per_step": round(conc_ms / steps, 4),
             "launches_per_call": launches_concurrent,
             "how": "each member's own autotuned launches and graph chunks on one of 8 streams"}
    if not plain:
        return {"instances": len(ws), "cells_per_step": cells, "steps": steps,
                "value": round(cells * steps / (batch_ms / 1e3) / 1e6, 2), "unit": UNIT,
                "tile_bx_by_kz": list(tune)}

    sims = []
    for w in ws:
        s_ = MBSimulation(w.grid, w.dx, w.dt, p, stream=stream.cuda_stream)
        s_.set_material(w.eps, w.gain, w.N_a, w.pump)
        s_.set_seed(w.seed)
        s_.add_point_probe(centre(w), 128, 475e-9, 705e-9)
        s_.autotune()
        s_.step(warmup)
        sims.append(s_)

    def plain():
        for s_ in sims:
            s_.step(steps)
            s_.join_probes()
    plain_ms = timed(plain)
    for s_ in sims:
        s_.close()
    v_batch = cells * steps / (batch_ms / 1e3) / 1e6
    v_conc = cells * steps / (conc_ms / 1e3) / 1e6
    v_plain = cells * steps / (plain_ms / 1e3) / 1e6
    sides = sorted({w.grid[0] for w in ws})
    other["ratio_vs_plain"] = round(v_conc / v_plain, 4)
    return {"workload": f"{len(ws)} realizations: 16 N_a levels (5e23-2e25 m^-3, log-spaced) x 5 "
                        f"disorder seeds, cubes of side {sides} (dx 20 nm, 45% fill, d 300 nm, "
                        "8-cell CPML), gain in the voids, W_p 1e13/s, Langevin noise, a centre "
                        "probe (128 bins) each",
            "instances": len(ws), "cells_per_step": cells, "steps": steps, "warmup": warmup,
            "value": round(v_batch, 2), "unit": UNIT, "ms_per_step": round(batch_ms / steps, 4),
            "mode": "persistent", "launches_per_call": 1,
            "what": "one persistent cooperative launch advancing all members (bounded grid "
                    "barriers), replayed from a CUDA graph per chunk of steps",
            "autotuner_pick": mode_name[picked],
            "tile_bx_by_kz": list(tune), "concurrent_mode": other,
            "plain_single_instance": {"value": round(v_plain, 2), "unit": UNIT,
                                      "ms_per_step": round(plain_ms / steps, 4),
                                      "how": "each realization's own context stepped by mb_step "
                                             "(autotuned, graph replay), one after another"},
            "ratio_vs_plain": round(v_batch / v_plain, 4),
            "l2": "inputs larger than L2"}


# ------------------------------------------------------- grid split along z

def bench_split(stream, steps: int, warmup: int, parts_list=(2, 4)):
    """The 320^3 workload split along z into slab contexts on this one GPU
    (ghost planes exchanged before every step through the C ABI, then one
    step of every slab), against the same grid as one context: the cost of
    the split path's exchange and per-slab launches.  Scaling over several
    GPUs is not measured here."""
    import torch
    from paper_0809_1547_gb300 import inputs
    from paper_0809_1547_gb300.binding import mb_default_params
    from paper_0809_1547_gb300.sharded import SlabGrid
    from paper_0809_1547_gb300.workloads import (FACE_EVERY, FACE_STRIDE, LAM_MAX, LAM_MIN, N_FREQ,
                                                 setup_simulation)
    w = inputs.workload_paper_320()
    cells = w.ncell

    def timed(fn, st):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(st)
        fn()
        e1.record(st)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    whole = setup_simulation(w, autotune=True, stream=stream.cuda_stream)
    whole.step(warmup)
    t_whole = timed(lambda: (whole.step(steps), whole.join_probes()), stream)
    whole.close()
    out = {"workload": f"{w.name}: {w.grid[0]}^3, centre probe + 6 face probes (each slab keeps "
                       f"the face points on its own planes)",
           "steps": steps, "whole_grid": {"value": round(cells * steps / (t_whole / 1e3) / 1e6, 2),
                                          "unit": UNIT, "ms_per_step": round(t_whole / steps, 5)}}
    for parts in parts_list:
        sg = SlabGrid(w.grid, w.dx, w.dt, parts, mb_default_params(npml=w.npml))
        sg.set_material(w.eps, w.gain, w.N_a, w.pump)
        sg.set_seed(w.seed)
        sg.add_point_probe(tuple(v // 2 for v in w.grid), N_FREQ, LAM_MIN, LAM_MAX)
        sg.add_face_probes(FACE_STRIDE, FACE_EVERY, N_FREQ, LAM_MIN, LAM_MAX)
        for s_ in sg.slabs:
            s_.autotune()
        sg.step(warmup)
        t = timed(lambda: (sg.step(steps), [s_.join_probes() for s_ in sg.slabs]), sg._stream)
        out[f"slabs_{parts}"] = {"value": round(cells * steps / (t / 1e3) / 1e6, 2), "unit": UNIT,
                                 "ms_per_step": round(t / steps, 5), "bounds": sg.bounds,
                                 "ratio_vs_whole": round(t_whole / t, 4),
                                 "halo_bytes_per_interface_per_step": 2 * sg.slabs[0].halo_bytes}
        sg.close()
    return out


# ------------------------------------------------------------- theory side

def bench_gp(n_E: int = 512, n_grid: int = 2047):
    """Bound states of -phi'' + tau^2 phi + phi^3 = E phi for n_E eigenvalues
    (log-spaced 1.005-400) on n_grid points each, FP64 on the GPU, and the
    theory curves (linewidth, peak) of kappa = 0.14 from them."""
    import numpy as np
    from paper_0809_1547_gb300 import gp
    E = np.geomspace(1.005, 400.0, n_E)
    gp.spectral_features(E[:8], n_grid)                      # warm-up
    t0 = time.perf_counter()
    w, pk = gp.spectral_features(E, n_grid)
    secs = time.perf_counter() - t0
    kappa = 0.14
    p = gp.p_threshold(kappa) * np.array([1.01, 2.0, 5.0, 20.0])
    c = gp.theory_curves(p, kappa, n_grid)
    return {"what": f"{n_E} eigenvalues E in [1.005, 400], {n_grid}-point grids, Newton in FP64",
            "ms": round(secs * 1e3, 2), "eigenvalues_per_s": round(n_E / secs, 1),
            "kappa": kappa, "p_th": c["p_th"], "p_over_p_th": [1.01, 2.0, 5.0, 20.0],
            "W_tg": [float(v) for v in c["W_tg"]], "S_p": [float(v) for v in c["S_p"]]}


# ------------------------------------------------------------ large sweep

def bench_large(stream, steps: int, warmup: int):
    """The 448^3 sample (8.96 um box, ~22.9k spheres d = 300 nm at 45 % fill,
    gain in the voids, N_a 5e24 m^-3, noise on; 90 M cells, 5.8 GB of FP32
    state): Mcell-updates/s and the passes' algorithmic HBM rates."""
    import torch
    from paper_0809_1547_gb300 import inputs
    from paper_0809_1547_gb300.workloads import setup_simulation
    w = inputs.workload_large_448()
    sim = setup_simulation(w, autotune=True, stream=stream.cuda_stream)
    sim.step(warmup)
    sim.synchronize()
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(steps)                    # graph replay, as mb_step runs
    sim.join_probes()
    e1.record(stream)
    torch.cuda.synchronize()
    el = e0.elapsed_time(e1)
    ms = sim.step_timed(steps)         # per-launch device times
    blocks = sim.tuning()
    single = sim.single_pass()
    sim.close()
    cells = w.ncell
    ab = algorithmic_bytes(w)
    peak, _ = measured_peaks()
    gbs = lambda b, t: b * cells / (t / 1e3) / 1e9
    if single[0]:
        n_single = steps - steps % 2
        f_ms = ms[0] / steps * steps / max(n_single, 1)
        launches = {"single_pass": {"ms": round(f_ms, 5), "gbs": round(gbs(ab["single_pass_launch"], f_ms), 1),
                                    "frac": round(gbs(ab["single_pass_launch"], f_ms) / peak, 4)}}
    else:
        h_ms, e_ms = ms[0] / steps, ms[1] / steps
        launches = {"h_pass": {"ms": round(h_ms, 5), "gbs": round(gbs(ab["h_launch"], h_ms), 1),
                               "frac": round(gbs(ab["h_launch"], h_ms) / peak, 4)},
                    "e_pass": {"ms": round(e_ms, 5), "gbs": round(gbs(ab["e_launch"], e_ms), 1),
                               "frac": round(gbs(ab["e_launch"], e_ms) / peak, 4)}}
    return {"workload": f"{w.name}: {w.grid[0]}^3 Yee grid, {w.n_spheres} TiO2 spheres d 300 nm at "
                        f"{w.fill:.3f} fill, gain in the voids, N_a 5e24 m^-3, W_p 1e13/s, Langevin "
                        "noise, centre probe + 6 face probes",
            "cells": cells, "steps": steps, "value": round(cells * steps / (el / 1e3) / 1e6, 2),
            "unit": UNIT, "ms_per_step": round(el / steps, 5),
            "launches": launches,
            "step_single_pass_frac": round(gbs(ab["single_pass_launch"], el / steps) / peak, 4),
            "blocks": {"h_pass": list(blocks[0]), "e_pass": list(blocks[1]), "single_pass": list(single)},
            "l2": "inputs larger than L2 (5.8 GB state)"}


# ---------------------------------------------------------------- passive

def bench_passive(w, stream, steps: int, warmup: int):
    """The 320^3 sample with the gain off (N_a = 0): (a) the response to the
    single-cycle 532 nm pulse (tau = 1 fs, t0 = 4 tau) at the centre with the
    centre probe and the six face probes; (b) CW excitation at 586.5 nm
    (rise time 4 fs) with a whole-plane probe on the middle section z = n/2
    (one bin at 586.5 nm, every step): the mode map of a long-living mode."""
    import torch
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params
    from paper_0809_1547_gb300.workloads import setup_simulation
    cells = w.ncell
    mid = tuple(v // 2 for v in w.grid)
    out = {}

    def run(sim):
        sim.step(warmup)
        sim.synchronize()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sim.step(steps)                # graph replay, as mb_step runs
        sim.join_probes()
        e1.record(stream)
        torch.cuda.synchronize()
        el = e0.elapsed_time(e1)
        return el, sim.step_timed(steps)

    import copy
    wp = copy.copy(w)
    wp.N_a = 0.0
    sim = setup_simulation(wp, autotune=True, stream=stream.cuda_stream)
    sim.set_source(mid, 2, 532e-9, 4e-15, 1e-15, 1e9)
    el, ms = run(sim)
    sim.close()
    out["pulse"] = {"value": round(cells * steps / (el / 1e3) / 1e6, 2), "unit": UNIT,
                    "ms_per_step": round(el / steps, 5),
                    "pass_ms_per_step": [round(v / steps, 5) for v in ms]}
    sim = MBSimulation(w.grid, w.dx, w.dt, mb_default_params(npml=w.npml), stream=stream.cuda_stream)
    sim.set_material(w.eps, w.gain, 0.0, 0.0)
    sim.set_seed(w.seed)
    sim.autotune()
    sim.set_source_cw(mid, 2, 586.5e-9, 0.0, 4e-15, 1e9, 2 * steps + warmup + 10)
    sim.add_plane_probe(mid[2], 1, 1, 586.5e-9, 586.5e-9)
    el, ms = run(sim)
    m = sim.plane_mode_map(0, 0)
    sim.close()
    out["cw_mode_map"] = {"value": round(cells * steps / (el / 1e3) / 1e6, 2), "unit": UNIT,
                          "ms_per_step": round(el / steps, 5),
                          "plane_probe_ms_per_step": round(ms[3] / steps, 5),
                          "plane_cells": w.grid[0] * w.grid[1], "map_max": float(m.max())}
    out["workload"] = (f"{w.name} geometry with the gain off (N_a = 0): (a) single-cycle 532 nm "
                       "pulse at the centre, centre probe + 6 face probes; (b) CW at 586.5 nm at the "
                       "centre with a whole-plane DFT probe on the middle section (1 bin, every step)")
    out["steps"] = steps
    return out


# ---------------------------------------------------------------- adjoint

def bench_adjoint(stream, warmup: int, autotune: bool = True, steps: int = 0, ckpt: int = 0):
    """Gradient of the energy through the +z face w.r.t. eps (per cell) and the
    pump on the 96^3 workload (225 spheres, 45 % fill, gain in the voids,
    fixed pump and noise seed), 4000 steps with checkpoints every 200 steps,
    against the plain step of the same realization over the same steps
    (steps, ckpt > 0: a shorter case of the same workload, for profiling)."""
    import copy
    import torch
    from paper_0809_1547_gb300 import inputs
    from paper_0809_1547_gb300.binding import MBSimulation, mb_default_params
    w = inputs.workload_adjoint_96()
    K = ckpt if ckpt > 0 else w.extra["ckpt_every"]
    if steps > 0:
        w = copy.copy(w)
        w.steps = steps
    cells = w.ncell

    def make():
        s_ = MBSimulation(w.grid, w.dx, w.dt, mb_default_params(npml=w.npml), stream=stream.cuda_stream)
        s_.set_material(w.eps, w.gain, w.N_a, w.pump)
        s_.set_seed(w.seed)
        if autotune:
            s_.autotune()
        return s_

    def timed(fn):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    s_ = make()
    for _ in range(max(1, warmup // 3)):
        s_.adjoint_energy_zface(2 * K, K)          # warm-up (allocations, graphs)
    s_.close()
    s_ = make()
    adj_ms, (J, G, gp) = timed(lambda: s_.adjoint_energy_zface(w.steps, K))
    s_.close()
    p_ = make()
    p_.step(warmup)
    plain_ms, _ = timed(lambda: (p_.step(w.steps), p_.join_probes()))
    p_.close()
    # one store slot per step of a segment: E, J, n1..n3 of every cell and two H planes
    store_gb = (9 * cells + 2 * w.grid[0] * w.grid[1]) * 4 * (K + 1) / 1e9
    state_mb = 16 * cells * 4 / 1e6
    v_adj = cells * w.steps / (adj_ms / 1e3) / 1e6
    v_plain = cells * w.steps / (plain_ms / 1e3) / 1e6
    return {"workload": f"{w.name}: {w.grid[0]}^3 (dx 20 nm, 8-cell CPML), {w.n_spheres} TiO2 spheres "
                        f"d 300 nm at {w.fill:.3f} fill, gain in the voids, N_a 5e24 m^-3, W_p 1e13/s, "
                        f"Langevin noise; gradient of the energy through the +z face w.r.t. eps (every "
                        f"cell) and W_p over {w.steps} steps, checkpoints every {K}",
            "value": round(v_adj, 2), "unit": UNIT, "ms_total": round(adj_ms, 2),
            "ms_per_step": round(adj_ms / w.steps, 5),
            "what": "forward sweep with checkpoints + per-segment recomputation + reverse sweep",
            "plain_single_instance": {"value": round(v_plain, 2), "unit": UNIT,
                                      "ms_per_step": round(plain_ms / w.steps, 5)},
            "ratio_vs_plain": round(v_adj / v_plain, 4),
            "objective_J": J, "grad_pump": gp,
            "l2": f"state ({state_mb:.0f} MB) below L2 size; segment store ({store_gb:.1f} GB) above"}


# --------------------------------------------------------- reference arm

def bench_reference(args):
    """The reference arm: the FP64 oracle (the paper has no implementation to
    run) on the benchmark's workload, on every host core; each step is one
    step of a slab of the workload per core, sized so the whole run takes
    about --ref-budget seconds (100 by default): 17 to 48 whole planes, and
    for runs too long for 17 whole planes, 17 planes of fewer rows (at least
    64, so the 8-cell CPML takes at most a quarter of the sample's rows)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return
    try:
        w = rank_workload(0)
        cores = min(host_cores(), args.ref_cores) if args.ref_cores > 0 else host_cores()
        # calibration on every core at once (the children share the memory
        # bandwidth, so one child alone would overstate each child's rate)
        with tempfile.TemporaryDirectory() as d:
            part = save_part(w, d, "cal", 150, 17)
            rall, _, _ = run_oracle_children([(part, 1, 1, "forward")] * cores)
        r1 = rall / cores
        budget_s = float(args.ref_budget)
        cells_per_child = r1 * 1e6 * budget_s / max(1, args.steps + args.warmup)
        thickness = int(max(17, min(48, round(cells_per_child / (w.grid[0] * w.grid[1])))))
        rows = w.grid[1]
        if cells_per_child < thickness * w.grid[0] * w.grid[1]:
            rows = int(max(min(64, w.grid[1]), min(w.grid[1], round(cells_per_child / (thickness * w.grid[0])))))
        rate, secs, ncell, cores = cpu_slab_rate(w, thickness, args.steps, args.warmup, cores,
                                                 rows=rows)
    except Exception as e:
        print(json.dumps({"impl": "reference", "unavailable": "oracle run failed: " + str(e)[-300:]}))
        return
    sample = (f"each step: {cores} slabs of {w.grid[0]}x{rows}x{thickness} planes ({ncell} cells "
              f"each, spread over the depth, each with its own 8-cell CPML) of the {w.name} workload, "
              f"FP64 numpy oracle, {cores} single-thread processes at once")
    out = {"impl": "reference", "metric": METRIC, "value": round(rate, 4), "unit": UNIT,
           "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": round(secs / args.steps * 1e3, 3), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": f"{w.name} (sampled slabs)", "grid": [w.grid[0], rows, thickness],
                      "slabs_per_step": cores},
           "cpu_baseline": {"value": round(rate, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(rate, 4), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_only(args):
    """One leg on its own (for profiling): its dict on one JSON line."""
    import torch
    from paper_0809_1547_gb300 import build
    build.build()
    stream = torch.cuda.Stream()
    if args.only == "batched":
        out = bench_batched(stream, args.batched_steps, args.warmup, args.batched_pump,
                            args.batched_seeds, autotune=not args.no_autotune, plain=False)
    elif args.only == "adjoint":
        out = bench_adjoint(stream, args.warmup, autotune=not args.no_autotune, steps=args.adj_steps,
                            ckpt=args.adj_ckpt)
    elif args.only == "passive":
        out = bench_passive(rank_workload(0, 320), stream, max(50, args.steps // 3), args.warmup)
    elif args.only == "large":
        out = bench_large(stream, max(50, args.steps // 6), args.warmup)
    elif args.only == "split":
        out = bench_split(stream, max(50, args.steps // 4), args.warmup)
    else:
        out = bench_gp()
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=600)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--ref-budget", type=float, default=100.0,
                    help="--impl reference: seconds of oracle stepping the run is sized for")
    ap.add_argument("--ref-cores", type=int, default=0,
                    help="--impl reference: oracle processes (default: one per host core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-cpu-configs", action="store_true",
                    help="skip the oracle rates of the 48^3, 448^3, ensemble and adjoint configs")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-ensemble leg")
    ap.add_argument("--batched-steps", type=int, default=40)
    ap.add_argument("--no-adjoint", action="store_true", help="skip the adjoint leg")
    ap.add_argument("--no-passive", action="store_true", help="skip the passive (pulse, CW) leg")
    ap.add_argument("--no-large", action="store_true", help="skip the 448^3 leg")
    ap.add_argument("--no-split", action="store_true", help="skip the z-slab split leg")
    ap.add_argument("--only", choices=("batched", "adjoint", "passive", "large", "gp", "split"), default="",
                    help="run one leg alone and print its result (profiling)")
    ap.add_argument("--batched-pump", type=int, default=16, help="N_a levels of the ensemble")
    ap.add_argument("--batched-seeds", type=int, default=5, help="disorder seeds of the ensemble")
    ap.add_argument("--adj-steps", type=int, default=0,
                    help="--only adjoint: steps of the gradient call (default: the workload's 4000)")
    ap.add_argument("--adj-ckpt", type=int, default=0,
                    help="--only adjoint: checkpoint interval (default: the workload's 200)")
    ap.add_argument("--no-autotune", action="store_true",
                    help="--only batched/adjoint: default launch shapes (no tuning launches)")
    ap.add_argument("--tune", default="",
                    help="fixed launch shapes 'v,bx,by,bz:v,bx,by,bz' (H launch : E launch) "
                         "instead of the autotuner; for profiling a chosen variant")
    ap.add_argument("--single-pass", default="",
                    help="'bx,by,kz': force the single-pass step with that tile; 'off': force the "
                         "two passes; default: the autotuner decides")
    ap.add_argument("--grid", type=int, default=320,
                    help="cube side of the workload (320: the paper-scale sample; smaller sides "
                         "only for profiling)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.only:
        run_only(args)
        return
    if args.impl == "reference":
        bench_reference(args)
    else:
        bench_ours(args)


if __name__ == "__main__":
    main()
