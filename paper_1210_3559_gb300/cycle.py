"""Heating-cooling cycle of icosahedral nickel clusters and the hysteresis of melting and freezing.

Usage: python -m paper_1210_3559_gb300.cycle [--replicas 8] [--shells 8] [--T-low 400] [--T-high 1400]
                                            [--rate 1.0] [--out result.json]

Independent replicas of a Mackay icosahedron (8 shells: 2057 atoms, the paper's Ni2047-2057 cluster) are
heated linearly from T-low to T-high and cooled back at the same rate (K/ps) under the Langevin
thermostat (gamma = 10/ps, dt = 1 fs, the paper's settings), all in one context on the GPU, with the total
energy per atom recorded every picosecond (the paper's cycle, Sec. III). For each replica: the melting
temperature (steepest rise of the energy with temperature on heating), the freezing temperature (the
same on cooling), their difference (the hysteresis width), and the energy per atom and crystalline fraction
(common-neighbour analysis) at T-low before and after the cycle.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs
from . import scmd


def _steepest(T: np.ndarray, e: np.ndarray, window_K: float = 40.0, smooth_K: float = 20.0) -> float:
    """Bath temperature at which the energy rises fastest with temperature: melting on a heating leg,
    freezing on a cooling leg (where the energy falls as the temperature falls). The energy is first
    averaged over smooth_K of bath temperature (a liquid cluster's energy fluctuates by ~5e-3 eV/atom
    per picosecond sample), then dE/dT is a centred difference over window_K."""
    dT = abs(T[1] - T[0])
    ns = max(1, int(round(smooth_K / dT)))
    es = np.convolve(e, np.ones(ns) / ns, mode="valid")
    Ts = T[(ns - 1) // 2:(ns - 1) // 2 + len(es)]
    w = max(1, int(round(window_K / dT / 2)))
    slope = (es[2 * w:] - es[:-2 * w]) / (Ts[2 * w:] - Ts[:-2 * w])
    k = int(np.argmax(slope))
    return float(Ts[k + w])


def run(replicas=8, shells=8, T_low=400.0, T_high=1400.0, rate_K_per_ps=1.0, dt=1.0, gamma=10.0, seed=21,
        precision=scmd.MD_PREC_MIXED, segment_ps=50.0):
    p1 = inputs.mackay_icosahedron(shells, 2.49)
    n = len(p1)
    m1 = inputs.masses(n)
    pos = np.concatenate([p1] * replicas)
    vel = np.concatenate([inputs.maxwell_boltzmann(p1, m1, T_low, seed=100 * seed + b, dof="3N") for b in range(replicas)])
    mass = inputs.masses(len(pos))
    every = max(1, int(round(1000.0 / dt)))  # one sample per ps
    ramp_ps = (T_high - T_low) / rate_K_per_ps
    seg_steps = int(round(segment_ps * 1000.0 / dt))
    n_seg = int(round(ramp_ps / segment_ps))
    cfg = scmd.config(precision=precision, obs_every=every, obs_capacity=2 * n_seg * (seg_steps // every) + 8,
                      graph_chunk=500)
    ctx = scmd.md_create(cfg, [n] * replicas, pos, vel, mass, scmd.sc_params())
    # equilibrate at T_low, then record the start
    scmd.md_step(ctx, int(round(20000.0 / dt)), dt, scmd.thermostat(scmd.MD_LANGEVIN, T_low, T_low, gamma_per_ps=gamma,
                                                                    seed=seed))
    start = scmd.md_observables(ctx)
    cna_start = scmd.md_cna(ctx, 3.0)  # per replica: other, fcc, hcp, icosahedral (on the device)
    scmd.md_clear_history(ctx)
    t0 = time.perf_counter()
    temps = []
    for leg, (Ta, Tb) in enumerate(((T_low, T_high), (T_high, T_low))):
        for s in range(n_seg):
            T0 = Ta + (Tb - Ta) * s / n_seg
            T1 = Ta + (Tb - Ta) * (s + 1) / n_seg
            th = scmd.thermostat(scmd.MD_LANGEVIN, T0, T1, gamma_per_ps=gamma, seed=seed + 1 + leg * n_seg + s)
            scmd.md_step(ctx, seg_steps, dt, th)
            # bath temperature at the samples of this segment (one at the end of every every-th step)
            k = np.arange(1, seg_steps // every + 1) * every
            temps.extend((T0 + (T1 - T0) * k / seg_steps).tolist())
    wall = time.perf_counter() - t0
    hist = scmd.md_obs_history(ctx)
    end = scmd.md_observables(ctx)
    cna_end = scmd.md_cna(ctx, 3.0)
    scmd.md_destroy(ctx)
    T = np.array(temps[:len(hist)])
    e = np.array([[h[b]["etot"] for b in range(replicas)] for h in hist]) / n
    half = len(T) // 2
    out = []
    for b in range(replicas):
        t_melt = _steepest(T[:half], e[:half, b])
        t_freeze = _steepest(T[half:], e[half:, b])
        out.append({"T_melt_K": t_melt, "T_freeze_K": t_freeze, "hysteresis_K": t_melt - t_freeze,
                    "e_start_eV_per_atom": start[b]["etot"] / n, "e_end_eV_per_atom": end[b]["etot"] / n,
                    "epot_start_eV_per_atom": start[b]["epot"] / n, "epot_end_eV_per_atom": end[b]["epot"] / n,
                    "crystalline_start": float(cna_start[b, 1] + cna_start[b, 2]) / n,
                    "crystalline_end": float(cna_end[b, 1] + cna_end[b, 2]) / n,
                    "icosahedral_start": int(cna_start[b, 3]), "icosahedral_end": int(cna_end[b, 3])})
    hyst = np.array([c["hysteresis_K"] for c in out])
    return {"replicas": replicas, "atoms_per_cluster": n, "T_low_K": T_low, "T_high_K": T_high,
            "rate_K_per_ps": rate_K_per_ps, "dt_fs": dt, "gamma_per_ps": gamma,
            "precision": "mixed" if precision == scmd.MD_PREC_MIXED else "fp64",
            "atom_steps_per_s": replicas * n * 2 * n_seg * seg_steps / wall,
            "T_melt_mean_K": float(np.mean([c["T_melt_K"] for c in out])),
            "T_freeze_mean_K": float(np.mean([c["T_freeze_K"] for c in out])),
            "hysteresis_mean_K": float(hyst.mean()), "hysteresis_sem_K": float(hyst.std(ddof=1) / np.sqrt(len(hyst)))
            if len(hyst) > 1 else None,
            "per_replica": out, "curve_T_K": T.tolist(), "curve_e_eV_per_atom": np.round(e, 6).tolist()}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--replicas", type=int, default=8)
    ap.add_argument("--shells", type=int, default=8)
    ap.add_argument("--T-low", type=float, default=400.0)
    ap.add_argument("--T-high", type=float, default=1400.0)
    ap.add_argument("--rate", type=float, default=1.0, help="K/ps")
    ap.add_argument("--seed", type=int, default=21)
    ap.add_argument("--out", default=None)
    a = ap.parse_args()
    res = run(a.replicas, a.shells, a.T_low, a.T_high, a.rate, seed=a.seed)
    if a.out:
        with open(a.out, "w") as f:
            f.write(json.dumps(res))
    print(json.dumps({k: v for k, v in res.items() if k not in ("per_replica", "curve_T_K", "curve_e_eV_per_atom")}))


if __name__ == "__main__":
    main()
