"""Benchmark: Sutton-Chen Ni cluster MD on one GB300 per rank (replicas), one JSON line.

Default workload (the largest single-GPU configuration, the paper's ensemble pattern of
Sec. III C): 512 independent clusters with N_b uniform in 55..2000 (seed 5; fcc spheres,
a = 3.52 A), Maxwell-Boltzmann velocities at 2000 K (per-cluster seed 1000 + b), melted with
Langevin at 2000 K for 20 ps (1e4 steps of 2 fs, gamma = 1/ps; untimed set-up), then quenched
with Langevin at a fixed 900 K (dt = 2 fs, gamma = 1/ps), MIXED precision (FP32 pair terms,
FP64 rho, energy and integration), all pairs. One timed iteration ("step" of this benchmark) is
one md_step call of --md-steps MD steps (default 500), issued as CUDA-graph replays. L2 is
flushed (a 256 MB write) before every timed iteration and that flush is outside the timed
events.

Other configs (--config): ni2000 (one cluster, Langevin cooling 2000 -> 300 K over 2e5 steps),
ni6000, ni20000 (all pairs, MIXED), ni50000 (rcut = 8.8 A on the neighbour lists, MIXED: lists of
atoms per atom quad), ni147 (FP64 NVE), ni147x64 (64 replicas of it in one context).

value  : atom-timesteps/s over all ranks (sum of atoms x MD steps / max rank time).
e2e    : the same metric through the C ABI with host buffers every iteration
         (md_set_state from pinned host arrays, md_step, md_get_state back to the host).
roofline: the force pass (dominant kernel), FP32-pipe lane operations per launch
         (16 per ordered pair) over its mean launch time. The launch time is CUDA-event time
         over back-to-back launches on the library's stream (the same programmatic-dependent
         launch overlap as inside the step graph) right after the timed region; it must fit the
         measured MD step. Peak: the device's SM count x 128 FP32 lanes x the maximum SM clock;
         the FFMA rate measured on this device (md_fp32_peak) is reported beside it.
cpu_baseline: the FP64 oracle (plain C + OpenMP) on the host cores, on a bounded sample
         of the same workload (rank 0 only).
--impl reference: times that oracle alone as the reference arm.
Multi-GPU (torchrun): independent replicas, one per rank ("replicas only": clusters are
independent), no data-path collective; value sums the ranks' work.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "atom-timesteps/s & pair-evals/s vs FP32 peak; mixed vs FP64 at stated drift"
UNIT = "atom-timesteps/s"
FP32_LANES_PER_SM = 128
FORCE_OPS_PER_PAIR = 16    # FP32 pipe lane-ops per ordered pair, force pass, (n,m) = (9,6)
# DRAM bytes (read + write) of one force-pass launch from an ncu capture (cold caches), with the hash
# of the sources of that kernel when it was captured; reported only while those sources are unchanged.
FORCE_SOURCES = {
    "all pairs": ("paper_1210_3559_gb300/csrc/scmd_kernels.cu", "paper_1210_3559_gb300/csrc/scmd_device.cuh",
                  "paper_1210_3559_gb300/csrc/scmd_internal.cuh"),
    "neighbour lists": ("paper_1210_3559_gb300/csrc/scmd_quads.cu", "paper_1210_3559_gb300/csrc/scmd_device.cuh",
                        "paper_1210_3559_gb300/csrc/scmd_internal.cuh", "paper_1210_3559_gb300/csrc/scmd_cells.cuh"),
}
FORCE_DRAM_BYTES_PER_LAUNCH = {"batched512": (51968000 + 838144, "2a201b4d53587c99")}
DENSITY_OPS_PER_PAIR = 8   # FP32 pipe lane-ops per ordered pair, density pass


def kernel_source_hash(path_name: str) -> str:
    import hashlib
    h = hashlib.sha256()
    for rel in FORCE_SOURCES.get(path_name, ()):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def force_traffic(config: str, path_name: str):
    rec = FORCE_DRAM_BYTES_PER_LAUNCH.get(config)
    if rec is None or rec[1] != kernel_source_hash(path_name):
        return None
    return rec[0]


# ------------------------------------------------------------------ workloads
def workload(name: str, rank: int):
    from paper_1210_3559_gb300 import inputs
    seed_off = 1000 * rank  # independent replica per rank
    if name == "ni2000":
        pos = inputs.fcc_sphere(2000)
        m = inputs.masses(2000)
        vel = inputs.maxwell_boltzmann(pos, m, 2000.0, seed=2 + seed_off, dof="3N")
        return dict(sizes=[2000], pos=pos, vel=vel, mass=m, prec="mixed", dt=2.0, melt_steps=10000,
                    melt_T=2000.0, schedule=(2000.0, 300.0, 200000), gamma=1.0, seed=2 + seed_off,
                    desc="Ni~2000 FCC sphere, melt 2000 K, Langevin cooling 2000->300 K over 2e5 steps dt=2 fs")
    if name in ("ni6000", "ni20000"):
        n = int(name[2:])
        pos = inputs.fcc_sphere(n)
        m = inputs.masses(n)
        vel = inputs.maxwell_boltzmann(pos, m, 2000.0, seed=(3 if n == 6000 else 4) + seed_off, dof="3N")
        return dict(sizes=[n], pos=pos, vel=vel, mass=m, prec="mixed", dt=2.0, melt_steps=2000, melt_T=2000.0,
                    schedule=(2000.0, 300.0, 200000), gamma=1.0, seed=3 + seed_off,
                    desc=f"Ni~{n} FCC sphere, Langevin cooling 2000->300 K over 2e5 steps dt=2 fs")
    if name == "ni50000":
        pos = inputs.fcc_sphere(50000)
        m = inputs.masses(50000)
        vel = inputs.maxwell_boltzmann(pos, m, 2000.0, seed=6 + seed_off, dof="3N")
        return dict(sizes=[50000], pos=pos, vel=vel, mass=m, prec="mixed", dt=2.0, melt_steps=2000, melt_T=2000.0,
                    schedule=(2000.0, 300.0, 200000), gamma=1.0, seed=6 + seed_off, rcut=8.8,
                    desc="Ni~50000 FCC sphere, rcut 8.8 A (2.5 a) on neighbour lists, Langevin cooling "
                         "2000->300 K over 2e5 steps dt=2 fs")
    if name == "ni147":
        pos = inputs.mackay_icosahedron(3, 2.49)
        m = inputs.masses(147)
        vel = inputs.maxwell_boltzmann(pos, m, 1500.0, seed=1 + seed_off)
        return dict(sizes=[147], pos=pos, vel=vel, mass=m, prec="fp64", dt=1.0, melt_steps=0, melt_T=0.0,
                    schedule=None, gamma=0.0, seed=1 + seed_off,
                    desc="Ni147 Mackay icosahedron, 1500 K, NVE dt=1 fs, FP64")
    if name == "ni147x64":  # 64 independent replicas of the Ni147 case in one context
        p1 = inputs.mackay_icosahedron(3, 2.49)
        m1 = inputs.masses(147)
        pos = np.concatenate([p1] * 64)
        vel = np.concatenate([inputs.maxwell_boltzmann(p1, m1, 1500.0, seed=1 + 100 * b + seed_off) for b in range(64)])
        return dict(sizes=[147] * 64, pos=pos, vel=vel, mass=inputs.masses(len(pos)), prec="fp64", dt=1.0,
                    melt_steps=0, melt_T=0.0, schedule=None, gamma=0.0, seed=1 + seed_off,
                    desc="64 replicas of Ni147 Mackay icosahedron, 1500 K, NVE dt=1 fs, FP64")
    if name == "batched512":
        sizes = inputs.batched_sizes(512, 55, 2000, seed=5 + seed_off)
        parts, vels = [], []
        for b, n in enumerate(sizes):
            p = inputs.fcc_sphere(int(n))
            parts.append(p)
            vels.append(inputs.maxwell_boltzmann(p, inputs.masses(int(n)), 2000.0, seed=1000 + b + seed_off, dof="3N"))
        pos = np.concatenate(parts)
        return dict(sizes=sizes, pos=pos, vel=np.concatenate(vels), mass=inputs.masses(len(pos)), prec="mixed",
                    dt=2.0, melt_steps=10000, melt_T=2000.0, schedule=(900.0, 900.0, 250000), gamma=1.0,
                    seed=5 + seed_off,
                    desc="512 clusters N~U{55..2000}, melt 2000 K, Langevin quench at 900 K dt=2 fs")
    raise SystemExit(f"unknown config {name}")


# --------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.out = tempfile.NamedTemporaryFile(prefix="clocks", suffix=".csv", delete=False)

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.out, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.out.close()
        rows = []
        for line in open(self.out.name):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append(dict(sm=float(f[1]), smax=float(f[2]), power=float(f[3]) if f[3] not in ("[N/A]", "") else 0.0,
                                 hw=f[5], hwt=f[6], swt=f[7], swp=f[8]))
            except ValueError:
                continue
        os.unlink(self.out.name)
        if not rows:
            return None
        load = [r for r in rows if r["power"] > 0.25 * max(x["power"] for x in rows)] or rows
        reasons = set()
        for r in load:
            for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                              ("swt", "sw_thermal_slowdown"), ("swp", "sw_power_cap")):
                if r[key].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(r["sm"] for r in load), "sm_max_mhz": max(r["smax"] for r in rows),
                "samples": len(load), "reasons": sorted(reasons)}


# ------------------------------------------------------------ oracle baseline
def cpu_baseline(w, budget_s: float):
    """Time the FP64 oracle on a bounded sample of the workload (same thermostat and dt)."""
    import oracle
    cores = oracle.num_threads(os.cpu_count() or 1)
    sizes = list(map(int, w["sizes"]))
    if len(sizes) > 8:  # batched: a fixed subset of clusters, scaled by atoms
        sizes = sizes[:8]
    n = sum(sizes)
    pos, vel, mass = w["pos"][:n], w["vel"][:n], w["mass"][:n]
    b = oracle.Batch(sizes, pos, vel, mass, oracle.params(rcut=w.get("rcut", 0.0)))
    th = oracle.thermostat(oracle.LANGEVIN if w["gamma"] > 0 else oracle.NVE,
                           w["melt_T"] or 0.0, None, gamma_ps=w["gamma"] or 1.0, seed=w["seed"])
    t0 = time.perf_counter()
    b.run(1, w["dt"], th)
    t1 = time.perf_counter() - t0
    steps = max(1, min(2000, int(budget_s / max(t1, 1e-6))))
    t0 = time.perf_counter()
    b.run(steps, w["dt"], th)
    el = time.perf_counter() - t0
    out = {"value": n * steps / el, "unit": UNIT, "cores": cores, "kind": "oracle",
           "sample": f"{steps} MD steps (FP64, all pairs{cut_note(w)}) of {len(sizes)} cluster(s), {n} atoms, "
                     f"dt={w['dt']} fs, same thermostat", "s_per_step": el / steps}
    # the same oracle on one core (the paper compares against one CPU core), when it fits the budget
    if t1 * cores <= budget_s:
        oracle.num_threads(1)
        steps1 = max(1, min(200, int(0.5 * budget_s / (t1 * cores))))
        t0 = time.perf_counter()
        b.run(steps1, w["dt"], th)
        el1 = time.perf_counter() - t0
        oracle.num_threads(cores)
        out["value_1core"] = n * steps1 / el1
        out["sample_1core"] = f"{steps1} MD steps, same sample, 1 thread"
    return out


def arm_config(w, world: int) -> dict:
    """The workload both arms report (the same dict for the GPU arm and the oracle arm)."""
    return {"workload": w["desc"], "atoms_per_gpu": int(np.sum(w["sizes"])), "clusters_per_gpu": int(len(w["sizes"])),
            "dt_fs": w["dt"], "rcut_A": w.get("rcut") or None,
            "l2": "GPU arm: flushed (256 MB write) before every timed iteration, outside the timed events",
            "parallelism": f"replicas x{world}" if world > 1 else "1 GPU"}


def cut_note(w):
    return f", cutoff {w['rcut']} A tested on every pair" if w.get("rcut") else ""


def run_reference(args, rank, world):
    if rank != 0:
        return
    w = workload(args.config, 0)
    import oracle
    cores = oracle.num_threads(os.cpu_count() or 1)
    sizes = list(map(int, w["sizes"]))[:8]
    n = sum(sizes)
    b = oracle.Batch(sizes, w["pos"][:n], w["vel"][:n], w["mass"][:n], oracle.params(rcut=w.get("rcut", 0.0)))
    th = oracle.thermostat(oracle.LANGEVIN if w["gamma"] > 0 else oracle.NVE, w["melt_T"] or 0.0, None,
                           gamma_ps=w["gamma"] or 1.0, seed=w["seed"])
    for _ in range(args.warmup):
        b.run(1, w["dt"], th)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b.run(1, w["dt"], th)
    el = time.perf_counter() - t0
    val = n * args.steps / el
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": arm_config(w, world),
            "run": {"sample_atoms": n, "sample_clusters": len(sizes), "md_steps_per_step": 1, "precision": "fp64"},
            "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step = 1 MD step of {n} atoms (FP64 oracle, all pairs{cut_note(w)})"},
            "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None, help="timed iterations (default 40; ni2000: 400)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="batched512", choices=["batched512", "ni2000", "ni6000", "ni20000", "ni50000",
                                                           "ni147", "ni147x64"])
    ap.add_argument("--md-steps", type=int, default=500, help="MD steps per timed iteration")
    ap.add_argument("--precision", default=None, choices=[None, "mixed", "fp64"])
    ap.add_argument("--path", default="auto", choices=["auto", "allpairs", "half"],
                    help="pair path of the all-pairs workloads: automatic, ordered pairs, or FP64 each pair once")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--skip-cpu", action="store_true")
    ap.add_argument("--skip-fp64", action="store_true")
    ap.add_argument("--melt-steps", type=int, default=None, help="override the untimed melt length")
    ap.add_argument("--shapes", default=None, help="ipt,warps,cluster for the density and force passes (6 ints); skips tuning")
    ap.add_argument("--snapshots", type=int, default=None, help="states kept during the timed run for e_F (default 10)")
    ap.add_argument("--drift-steps", type=int, default=None, help="NVE steps of the drift runs (default: automatic)")
    ap.add_argument("--skip-analysis", action="store_true", help="no snapshots, drift runs or structure analysis")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 400 if args.config == "ni2000" else 40
    if args.warmup < 3:
        args.warmup = 3

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if args.impl == "reference":
        run_reference(args, rank, world)
        if dist:
            dist.destroy_process_group()
        return

    torch.cuda.set_device(local)
    from paper_1210_3559_gb300 import build as _build, scmd
    _build.build()
    w = workload(args.config, rank)
    if args.melt_steps is not None:
        w["melt_steps"] = args.melt_steps
    prec = args.precision or w["prec"]
    P = scmd.MD_PREC_MIXED if prec == "mixed" else scmd.MD_PREC_FP64
    stream = torch.cuda.Stream()
    path_arg = {"auto": scmd.MD_PATH_AUTO, "allpairs": scmd.MD_PATH_ALLPAIRS,
                "half": scmd.MD_PATH_ALLPAIRS_HALF}[args.path]
    cfg = scmd.config(precision=P, path=path_arg, graph_chunk=min(args.md_steps, 512), tune=0 if args.no_tune else 1,
                      stream=stream.cuda_stream)
    sizes = np.asarray(w["sizes"], dtype=np.int32)
    natoms = int(sizes.sum())
    pairs_per_eval = float(np.sum(sizes.astype(np.float64) * (sizes - 1)))
    if args.shapes:
        cfg.tune = 0
    rcut = w.get("rcut", 0.0)
    ctx = scmd.md_create(cfg, sizes, w["pos"], w["vel"], w["mass"], scmd.sc_params(rcut=rcut))
    path = scmd.md_get_path(ctx)
    cells = path in (scmd.MD_PATH_CELLS, scmd.MD_PATH_VERLET)  # a cutoff path
    path_name = {scmd.MD_PATH_CELLS: "cells", scmd.MD_PATH_VERLET: "neighbour lists",
                 scmd.MD_PATH_ALLPAIRS_HALF: "all pairs, each pair once"}.get(path, "all pairs")
    if args.shapes:
        v = [int(x) for x in args.shapes.split(",")]
        scmd.md_set_launch(ctx, 0, *v[0:3])
        scmd.md_set_launch(ctx, 1, *v[3:6])
    dt = w["dt"]
    # set-up: melt (untimed)
    if w["melt_steps"]:
        scmd.md_step(ctx, w["melt_steps"], dt, scmd.thermostat(scmd.MD_LANGEVIN, w["melt_T"], w["melt_T"],
                                                               gamma_per_ps=w["gamma"], seed=w["seed"]))
    melt_pos, melt_vel, _ = scmd.md_get_state(ctx)  # start of the NVE drift runs
    cna_melt = None if args.skip_analysis else scmd.md_cna(ctx, 3.0)  # on the device (Sec. III)
    M = args.md_steps

    def therm(k):
        if w["schedule"] is None:
            return None
        T0, T1, n = w["schedule"]
        a, b = k * M, (k + 1) * M
        return scmd.thermostat(scmd.MD_LANGEVIN, T0 + (T1 - T0) * min(a, n) / n, T0 + (T1 - T0) * min(b, n) / n,
                               gamma_per_ps=w["gamma"], seed=w["seed"] + 17)

    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")  # 256 MB > 129 MB L2
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    # warm-up iterations (not timed) advance the schedule like the timed ones
    k_iter = 0
    for _ in range(args.warmup):
        scmd.md_step(ctx, M, dt, therm(k_iter))
        k_iter += 1
    n0 = int(sizes[0])
    analysis_on = not args.skip_analysis
    n_snap = 0 if not analysis_on else (args.snapshots if args.snapshots is not None else (10 if natoms <= 20000 else 3))
    snap_every = max(1, args.steps // max(n_snap, 1))
    snaps = []
    obs_start = scmd.md_observables(ctx) if analysis_on else None
    sampler = ClockSampler(local)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    sampler.start()
    t_wall0 = time.perf_counter()
    for k in range(args.steps):
        with torch.cuda.stream(stream):
            flush.zero_()
            ev[k][0].record(stream)
        scmd.md_step(ctx, M, dt, therm(k_iter))
        with torch.cuda.stream(stream):
            ev[k][1].record(stream)
        k_iter += 1
        if len(snaps) < n_snap and (k + 1) % snap_every == 0:  # outside the events: a D2H copy of x
            snaps.append(scmd.md_get_state(ctx)[0][:n0].copy())
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop()
    t_dev = sum(a.elapsed_time(b) for a, b in ev) / 1e3  # seconds of timed device work
    t_max = t_dev
    if dist:
        t = torch.tensor([t_dev], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_max = float(t.item())
    md_steps_total = args.steps * M
    value = natoms * md_steps_total * world / t_max

    # pass timings with CUDA events on the library's stream (same state, same launch shapes)
    ms_d, ms_f, pairs = scmd.md_time_passes(ctx, 50)
    if cells:  # pairs tested at the final state (octants of the cell list, or the listed pairs)
        pairs_per_eval = pairs
    pair_rate = pairs_per_eval * md_steps_total * world / t_max
    peak_clock = (clocks or {}).get("sm_max_mhz", 2070.0)
    n_sm = torch.cuda.get_device_properties(local).multi_processor_count
    # the pair passes run on the FP32 pipe in MIXED and on the FP64 pipe (1/64 of the FP32 lanes) in FP64
    lanes = FP32_LANES_PER_SM if prec == "mixed" else FP32_LANES_PER_SM / 64
    peak_ops = n_sm * lanes * peak_clock * 1e6
    ffma_measured, _ = scmd.md_fp32_peak(10)
    # algorithmic work of a launch: every ordered pair for all pairs; the pairs closer than rcut with a
    # cutoff (the candidates the cell or neighbour lists test are reported beside)
    useful_pairs = None
    if cells:
        from scipy.spatial import cKDTree
        pf, _, _ = scmd.md_get_state(ctx)
        useful_pairs = 2.0 * len(cKDTree(pf).query_pairs(rcut, output_type="ndarray"))
    alg_pairs = useful_pairs if cells else pairs
    ops_per_pair = FORCE_OPS_PER_PAIR
    if path == scmd.MD_PATH_ALLPAIRS_HALF:  # each unordered pair once: its 16 ops plus 3 for the partner's force
        alg_pairs, ops_per_pair = pairs / 2, FORCE_OPS_PER_PAIR + 3
    achieved = ops_per_pair * alg_pairs / (ms_f * 1e-3)
    shapes = {"density": scmd.md_get_launch(ctx, 0), "force": scmd.md_get_launch(ctx, 1)}
    per_step, per_chunk = scmd.md_launch_counts(ctx)
    chunk = min(M, 512)
    launches = args.steps * (M * per_step + math.ceil(M / chunk) * per_chunk)

    # force error of the final state against the FP64 oracle (rank 0, first cluster)
    force_err = None
    pos_f, vel_f, step_f = scmd.md_get_state(ctx)
    snap_err = []
    if rank == 0:
        import oracle
        E, F = scmd.md_energy_forces(ctx)
        _, Fr, _, _ = oracle.energy_forces(pos_f[:n0], oracle.params(rcut=rcut))
        force_err = float(np.linalg.norm(F[:n0] - Fr) / np.linalg.norm(Fr))
        # the snapshots of the timed run: first cluster, fresh context of the same precision and path
        for sp in snaps:
            cs = scmd.md_create(scmd.config(precision=P, path=scmd.MD_PATH_AUTO), [n0], sp, None, w["mass"][:n0],
                                scmd.sc_params(rcut=rcut))
            _, Fs = scmd.md_energy_forces(cs)
            scmd.md_destroy(cs)
            _, Fr, _, _ = oracle.energy_forces(sp, oracle.params(rcut=rcut))
            snap_err.append(float(np.linalg.norm(Fs - Fr) / np.linalg.norm(Fr)))
    structure = None
    if rank == 0 and analysis_on:
        obs_end = scmd.md_observables(ctx)
        cna_end = scmd.md_cna(ctx, 3.0)

        def fractions(counts):  # cluster 0: other, fcc, hcp, icosahedral
            f = counts[0] / max(n0, 1)
            return {"fcc": float(f[1]), "hcp": float(f[2]), "icosahedral": float(f[3]),
                    "crystalline": float(f[1] + f[2])}
        structure = {"cluster": 0, "atoms": n0,
                     "epot_per_atom_start_eV": obs_start[0]["epot"] / n0, "epot_per_atom_end_eV": obs_end[0]["epot"] / n0,
                     "T_start_K": obs_start[0]["T"], "T_end_K": obs_end[0]["T"],
                     "crystalline_fraction_end": fractions(cna_end),
                     "crystalline_fraction_start_of_schedule": fractions(cna_melt),
                     "cna": "on the device (md_cna, neighbours closer than 3.0 A)"}

    # e2e through the C ABI with host buffers: set_state (H2D) + md_step + get_state (D2H)
    pos_h = torch.from_numpy(pos_f.copy()).pin_memory().numpy()
    vel_h = torch.from_numpy(vel_f.copy()).pin_memory().numpy()
    e2e_iters = max(3, min(args.steps, 20))
    scmd.md_set_state(ctx, pos_h, vel_h, step_f)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    s_now = step_f
    for k in range(e2e_iters):
        scmd.md_set_state(ctx, pos_h, vel_h, s_now)
        scmd.md_step(ctx, M, dt, therm(k_iter + k))
        p2, v2, s_now = scmd.md_get_state(ctx)
        pos_h[:] = p2
        vel_h[:] = v2
    e2e_t = time.perf_counter() - t0
    if dist:
        t = torch.tensor([e2e_t], dtype=torch.float64, device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_t = float(t.item())
    e2e_value = natoms * M * e2e_iters * world / e2e_t

    # FP64-on-GPU form of the same workload, short sample (mixed vs FP64)
    fp64 = None
    if not args.skip_fp64 and prec == "mixed":
        # built-in launch table: tuning FP64 at the large workloads would time hundreds of launches of
        # tens of milliseconds each
        cfg64 = scmd.config(precision=scmd.MD_PREC_FP64, graph_chunk=min(M, 512), tune=0, stream=stream.cuda_stream)
        c64 = scmd.md_create(cfg64, sizes, pos_f, vel_f, w["mass"], scmd.sc_params(rcut=rcut))
        m64 = max(10, M // 10)
        scmd.md_step(c64, m64, dt, therm(0))
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(stream):
            e0.record(stream)
        reps64 = 3
        for _ in range(reps64):
            scmd.md_step(c64, m64, dt, therm(0))
        with torch.cuda.stream(stream):
            e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3
        p64 = scmd.md_get_path(c64)
        fp64 = {"value": natoms * m64 * reps64 / t64, "unit": UNIT,
                "pair_evals_per_s": (useful_pairs if cells else pairs_per_eval) * m64 * reps64 / t64,
                "path": {scmd.MD_PATH_CELLS: "cells", scmd.MD_PATH_VERLET: "neighbour lists",
                         scmd.MD_PATH_ALLPAIRS_HALF: "all pairs, each pair once"}.get(p64, "all pairs"),
                "sample": f"{reps64} x {m64} MD steps, same state and thermostat, per GPU, built-in launch shapes"}
        scmd.md_destroy(c64)

    # NVE energy drift from the melted state, MIXED and FP64 on the GPU (first cluster, or the first 8)
    drift = None
    if rank == 0 and analysis_on:
        from paper_1210_3559_gb300 import analysis
        nb = 1 if len(sizes) == 1 else min(8, len(sizes))
        sz = sizes[:nb]
        na = int(sz.sum())
        rate64 = (fp64 or {}).get("value") or 2.0e6
        steps_d = args.drift_steps or int(min(20000, max(1000, 10.0 * rate64 / na)))
        oe = max(1, steps_d // 200)
        drift = {"start": "state after the untimed melt" if w["melt_steps"] else "initial state",
                 "clusters": int(nb), "atoms": na, "steps": steps_d, "dt_fs": dt}
        for name, pr in (("mixed", scmd.MD_PREC_MIXED), ("fp64", scmd.MD_PREC_FP64)):
            if pr == scmd.MD_PREC_FP64 and args.skip_fp64:
                continue
            cd = scmd.md_create(scmd.config(precision=pr, obs_every=oe, obs_capacity=steps_d // oe + 2,
                                            graph_chunk=min(512, steps_d), stream=stream.cuda_stream),
                                sz, melt_pos[:na], melt_vel[:na], w["mass"][:na], scmd.sc_params(rcut=rcut))
            e0 = scmd.md_observables(cd)
            scmd.md_step(cd, steps_d, dt)
            hist = scmd.md_obs_history(cd)
            scmd.md_destroy(cd)
            t = np.array([0.0] + [h[0]["time_fs"] for h in hist])
            et = np.array([sum(o["etot"] for o in e0)] + [sum(o["etot"] for o in h) for h in hist])
            drift[name] = analysis.energy_drift(t, et, na)

    cpu = None
    if rank == 0 and not args.skip_cpu:
        cpu = cpu_baseline(w, args.cpu_budget)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * t_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32" if prec == "mixed" else "f64",
            "data": "synthetic",
            "config": arm_config(w, world),
            "run": {"md_steps_per_step": M, "precision": prec, "path": path_name,
                    "launch_shapes": {k: list(v) for k, v in shapes.items()} if not cells else path_name,
                    "wall_s_timed_region": t_wall},
            "pair_evals_per_s": pair_rate if not cells else useful_pairs * md_steps_total * world / t_max,
            "candidate_pairs_per_s": pair_rate if cells else None,
            "fp32_pipe_frac_force_pass": achieved / peak_ops if prec == "mixed" else None,
            "force_err_vs_oracle": force_err,
            "force_err_snapshots": snap_err or None,
            "nve_drift": drift,
            "structure": structure,
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12,
                         "unit": "T FP32-lane-ops/s" if prec == "mixed" else "T FP64-lane-ops/s",
                         "frac": achieved / peak_ops,
                         "traffic": force_traffic(args.config, path_name) if prec == "mixed" else None,
                         "kernel": {"cells": "k_cell_force (force pass, cell list)",
                                    "neighbour lists": "k_q_force (force pass, atom lists per quad)" if prec == "mixed"
                                    else "k_v_force (force pass, neighbour lists)"}.get(
                                        path_name, "k_force (force pass)"),
                         "ms_per_launch": ms_f,
                         "density_pass_ms_per_launch": ms_d, "pairs_per_launch": alg_pairs,
                         "tested_pairs_per_launch": pairs if cells else None,
                         "peak_basis": (f"{n_sm} SMs x 128 FP32 lanes x {peak_clock:.0f} MHz (max SM clock)"
                                        if prec == "mixed" else
                                        f"{n_sm} SMs x 2 FP64 lanes (1/64 of FP32) x {peak_clock:.0f} MHz (max SM clock)"),
                         "peak_measured_ffma": ffma_measured / 1e12,
                         "frac_of_measured_ffma": achieved / ffma_measured if prec == "mixed" else None,
                         "launch_timing": "CUDA events over back-to-back launches (PDL overlap as in the step graph)",
                         "passes_ms_per_md_step": ms_d + ms_f if not cells else None,
                         "ms_per_md_step": 1e3 * t_max / md_steps_total},
            "e2e": {"value": e2e_value, "unit": UNIT,
                    "h2d_bytes_per_step": int(2 * natoms * 3 * 8), "d2h_bytes_per_step": int(2 * natoms * 3 * 8),
                    "iterations": e2e_iters},
            "gpu_launches": int(launches),
            "fp64_gpu": fp64,
            "cpu_baseline": cpu,
            "clocks": clocks,
        }
        print(json.dumps(line), flush=True)
    scmd.md_destroy(ctx)
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
