"""Quench an ensemble of clusters and report when each one solidifies.

Usage: python -m paper_1210_3559_gb300.quench [--clusters 512] [--nmin 55] [--nmax 2000] [--T 900]
                                             [--steps 250000] [--dt 2] [--gamma 1] [--out result.json]

Many independent clusters of uneven size (fcc spheres, per-cluster Maxwell-Boltzmann velocities)
are melted at 2000 K with the Langevin thermostat, then quenched to a fixed temperature and followed
with the total energy recorded every picosecond, all in one context on the GPU (the paper's
solidification runs, Sec. III; nucleation is stochastic, hence the ensemble). The solidification
time of each cluster is read from its energy trace (analysis.solidification_time; clusters that never
solidify are right-censored at the horizon), and the crystalline fraction of its final structure is
measured by common-neighbour analysis. The escape rate from the supercooled liquid is reported as
the mean lifetime's inverse over the clusters that solidified (the paper's definition, Sec. III D)
and as the exponential-decay maximum-likelihood rate with right censoring (events / total time
spent liquid), which stays unbiased when some clusters outlast the horizon.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import analysis, inputs
from . import scmd


def run(n_clusters=512, nmin=55, nmax=2000, T=900.0, steps=250000, melt_steps=10000, dt=2.0, gamma=1.0,
        seed=5, precision=scmd.MD_PREC_MIXED, bin_ps=50.0, traces=False, melt_T=2000.0):
    sizes = inputs.batched_sizes(n_clusters, nmin, nmax, seed=seed)
    parts, vels = [], []
    for b, n in enumerate(sizes):
        p = inputs.fcc_sphere(int(n))
        parts.append(p)
        vels.append(inputs.maxwell_boltzmann(p, inputs.masses(int(n)), melt_T, seed=1000 * seed + b, dof="3N"))
    pos, vel = np.concatenate(parts), np.concatenate(vels)
    mass = inputs.masses(len(pos))
    every = max(1, int(round(1000.0 / dt)))  # one sample per ps
    cfg = scmd.config(precision=precision, obs_every=every, obs_capacity=steps // every + 2, graph_chunk=500)
    ctx = scmd.md_create(cfg, sizes, pos, vel, mass, scmd.sc_params())
    scmd.md_step(ctx, melt_steps, dt, scmd.thermostat(scmd.MD_LANGEVIN, melt_T, melt_T, gamma_per_ps=gamma,
                                                      seed=seed))
    scmd.md_clear_history(ctx)
    t0 = time.perf_counter()
    scmd.md_step(ctx, steps, dt, scmd.thermostat(scmd.MD_LANGEVIN, T, T, gamma_per_ps=gamma, seed=seed + 1))
    wall = time.perf_counter() - t0
    hist = scmd.md_obs_history(ctx)
    cna = scmd.md_cna(ctx, 3.0)  # per cluster: other, fcc, hcp, icosahedral (on the device)
    scmd.md_destroy(ctx)
    e = np.array([[h[b]["etot"] for b in range(len(sizes))] for h in hist]) / np.asarray(sizes)[None, :]
    off = np.concatenate([[0], np.cumsum(sizes)])
    out = []
    for b, n in enumerate(sizes):
        tn = analysis.solidification_time(e[:, b], dt_ps=every * dt / 1000.0)
        cf = float(cna[b, 1] + cna[b, 2]) / n
        out.append({"n": int(n), "t_nuc_ps": tn, "crystalline_end": cf})
    horizon = steps * dt / 1000.0
    times = np.array([c["t_nuc_ps"] for c in out if c["t_nuc_ps"] is not None])
    edges = np.arange(0.0, horizon + bin_ps, bin_ps)
    counts, _ = np.histogram(times, bins=edges)
    at_risk = float(times.sum() + horizon * (len(out) - len(times)))
    res = {"clusters": len(sizes), "atoms": int(off[-1]), "T_K": T, "horizon_ps": horizon, "dt_fs": dt,
            "gamma_per_ps": gamma, "precision": "mixed" if precision == scmd.MD_PREC_MIXED else "fp64",
            "atom_steps_per_s": off[-1] * steps / wall,
            "solidified": int(len(times)),
            "mean_lifetime_ps": float(times.mean()) if len(times) else None,
            "lifetime_sem_ps": float(times.std(ddof=1) / np.sqrt(len(times))) if len(times) > 1 else None,
            "kappa_mean_per_ps": float(1.0 / times.mean()) if len(times) else None,
            "kappa_mle_per_ps": len(times) / at_risk if at_risk > 0 else None,
            "lifetimes_ps": sorted(times.tolist()),
            "histogram": {"bin_ps": bin_ps, "edges_ps": edges.tolist(), "counts": counts.tolist(),
                          "censored": int(sum(c["t_nuc_ps"] is None for c in out))},
            "per_cluster": out}
    if traces:  # E_tot / N of every cluster, one sample per ps (rows: clusters)
        res["traces_eV_per_atom"] = np.round(e.T, 6).tolist()
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--clusters", type=int, default=512)
    ap.add_argument("--nmin", type=int, default=55)
    ap.add_argument("--nmax", type=int, default=2000)
    ap.add_argument("--T", type=float, default=900.0)
    ap.add_argument("--steps", type=int, default=250000)
    ap.add_argument("--melt-steps", type=int, default=10000)
    ap.add_argument("--melt-T", type=float, default=2000.0)
    ap.add_argument("--dt", type=float, default=2.0, help="fs")
    ap.add_argument("--gamma", type=float, default=1.0, help="Langevin friction, 1/ps")
    ap.add_argument("--seed", type=int, default=5)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--out", default=None)
    ap.add_argument("--traces", action="store_true", help="store every cluster's energy trace in --out")
    a = ap.parse_args()
    res = run(a.clusters, a.nmin, a.nmax, a.T, a.steps, a.melt_steps, dt=a.dt, gamma=a.gamma, seed=a.seed,
              precision=scmd.MD_PREC_MIXED if a.precision == "mixed" else scmd.MD_PREC_FP64, traces=a.traces,
              melt_T=a.melt_T)
    text = json.dumps(res)
    if a.out:
        with open(a.out, "w") as f:
            f.write(text)
    h = res["histogram"]
    print(json.dumps({k: v for k, v in res.items() if k not in ("per_cluster", "traces_eV_per_atom")}))
    print(f"solidified {res['clusters'] - h['censored']} / {res['clusters']} within {res['horizon_ps']:.0f} ps")


if __name__ == "__main__":
    main()
