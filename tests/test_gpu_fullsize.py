"""GPU parity at the workloads' own sizes: all pairs at Ni~6000 and Ni~20000 (one cluster each) and
the full 512-cluster ensemble (N_b uniform in 55..2000), every atom of every cluster compared with the
FP64 oracle (Eq. 1 energy, Eq. 2 density, the derivative of Eq. 1 for the forces), at the launch
shapes the autotuner picks for the benchmark.

Tolerances are those of test_gpu_parity.py: FP64 e_F <= 1e-12, |dE|/|E| <= 1e-13, rho <= 1e-13;
MIXED e_F <= 1e-5, |dE|/|E| <= 1e-6, rho <= 2e-5 (e_F = ||F_gpu - F_ref|| / ||F_ref|| over a
cluster). In MIXED the pair coordinates are FP32 offsets from the cluster's centre of mass, so the
rounding of the coordinates alone sets a floor under e_F that grows with the cluster's radius
(ulp(x)/2 is 9.5e-7 A below 16 A, 1.9e-6 A up to 32 A, 3.8e-6 A beyond). The test
``test_mixed_coordinate_rounding_floor`` (CPU) evaluates the oracle on those rounded coordinates to
show the floor and the margin left for the FP32 sums.
"""
import numpy as np
import pytest

import oracle
from paper_1210_3559_gb300 import inputs

FP64, MIXED = 0, 1
TOL = {FP64: dict(eF=1e-12, E=1e-13, rho=1e-13), MIXED: dict(eF=1e-5, E=1e-6, rho=2e-5)}
# At these sizes the MIXED energy also meets the tighter 1e-7 of the original specification: its error comes
# from the FP32 pair terms, whose sums are folded in FP64 every 128 pairs and which average out over ~1e7 pairs.
E_FULLSIZE_MIXED = 1e-7


@pytest.fixture(scope="module")
def scmd():
    from paper_1210_3559_gb300 import build, scmd as s
    build.build()
    return s


def errors(F, E, rho, pos):
    Er, Fr, _, rhor = oracle.energy_forces(pos)
    eF = np.linalg.norm(F - Fr) / np.linalg.norm(Fr)
    eE = abs(E - Er) / abs(Er)
    erho = np.max(np.abs(rho - rhor) / rhor)
    return eF, eE, erho


def tune_for(prec):
    """MIXED: the autotuned shapes the benchmark runs; FP64: the built-in table (tuning FP64 at these
    sizes would time hundreds of launches of tens of milliseconds each)."""
    return 1 if prec == MIXED else 0


def sphere(n, amp, seed):
    return inputs.jitter(inputs.fcc_sphere(n), amp, seed)


# ------------------------------------------------------------------ CPU (no GPU)
@pytest.mark.parametrize("n,amp", [(6000, 0.1), (20000, 0.1)])
def test_mixed_coordinate_rounding_floor(n, amp):
    """The part of the MIXED force error that FP32 pair coordinates alone cause, from the oracle on
    coordinates rounded as the GPU rounds them (offsets from the centre of mass): it must leave room
    under the 1e-5 bound for the FP32 sums."""
    pos = sphere(n, amp, 7)
    o = pos.mean(axis=0)
    rounded = o + (pos - o).astype(np.float32).astype(np.float64)
    _, F, _, _ = oracle.energy_forces(pos)
    _, Fr, _, _ = oracle.energy_forces(rounded)
    floor = np.linalg.norm(Fr - F) / np.linalg.norm(F)
    assert 1e-7 < floor < 0.8e-5, floor


# ------------------------------------------------------------------ GPU
@pytest.mark.gpu
@pytest.mark.parametrize("prec", [FP64, MIXED], ids=["fp64", "mixed"])
@pytest.mark.parametrize("n,amp,seed", [(6000, 0.15, 3), (20000, 0.1, 4)], ids=["ni6000", "ni20000"])
def test_single_cluster_full_size(scmd, prec, n, amp, seed):
    pos = sphere(n, amp, seed)
    ctx = scmd.md_create(scmd.config(precision=prec, tune=tune_for(prec)), [n], pos, None, inputs.masses(n),
                         scmd.sc_params())
    E, F = scmd.md_energy_forces(ctx)
    rho = scmd.md_get_density(ctx)
    eF, eE, erho = errors(F, E[0], rho, pos)
    tol = TOL[prec]
    print(f"N={n} prec={prec} shapes={scmd.md_get_launch(ctx, 0)},{scmd.md_get_launch(ctx, 1)} "
          f"e_F={eF:.3e} dE/E={eE:.3e} rho={erho:.3e}")
    assert eF <= tol["eF"], eF
    assert eE <= (E_FULLSIZE_MIXED if prec == MIXED else tol["E"]), eE
    assert erho <= tol["rho"], erho
    scmd.md_destroy(ctx)


@pytest.mark.gpu
def test_single_cluster_full_size_liquid_state(scmd):
    """Ni~20000 after 400 Langevin steps at 2000 K (the start of the cooling schedule's melt), MIXED:
    the thermal state the benchmark times, forces compared with the oracle at that state."""
    n = 20000
    pos = inputs.fcc_sphere(n)
    m = inputs.masses(n)
    vel = inputs.maxwell_boltzmann(pos, m, 2000.0, seed=4, dof="3N")
    ctx = scmd.md_create(scmd.config(precision=MIXED, tune=1), [n], pos, vel, m, scmd.sc_params())
    scmd.md_step(ctx, 400, 2.0, scmd.thermostat(scmd.MD_LANGEVIN, 2000.0, 2000.0, gamma_per_ps=1.0, seed=4))
    p, _, _ = scmd.md_get_state(ctx)
    E, F = scmd.md_energy_forces(ctx)
    rho = scmd.md_get_density(ctx)
    eF, eE, erho = errors(F, E[0], rho, p)
    print(f"N={n} liquid e_F={eF:.3e} dE/E={eE:.3e} rho={erho:.3e}")
    assert eF <= TOL[MIXED]["eF"] and eE <= E_FULLSIZE_MIXED and erho <= TOL[MIXED]["rho"], (eF, eE, erho)
    scmd.md_destroy(ctx)


@pytest.mark.gpu
@pytest.mark.parametrize("prec", [FP64, MIXED], ids=["fp64", "mixed"])
def test_full_512_cluster_ensemble(scmd, prec):
    """The whole 512-cluster context of the ensemble workload (sizes from seed 5), every cluster."""
    sizes = inputs.batched_sizes(512, 55, 2000, seed=5)
    parts = [sphere(int(n), 0.15, 100 + b) for b, n in enumerate(sizes)]
    pos = np.concatenate(parts)
    ctx = scmd.md_create(scmd.config(precision=prec, tune=tune_for(prec)), sizes, pos, None, inputs.masses(len(pos)),
                         scmd.sc_params())
    E, F = scmd.md_energy_forces(ctx)
    rho = scmd.md_get_density(ctx)
    off = np.concatenate([[0], np.cumsum(sizes)])
    worst = [0.0, 0.0, 0.0]
    for b in range(len(sizes)):
        s, e = off[b], off[b + 1]
        err = errors(F[s:e], E[b], rho[s:e], pos[s:e])
        worst = [max(w, x) for w, x in zip(worst, err)]
    print(f"512 clusters prec={prec} worst e_F={worst[0]:.3e} dE/E={worst[1]:.3e} rho={worst[2]:.3e}")
    tol = TOL[prec]
    e_tol = E_FULLSIZE_MIXED if prec == MIXED else tol["E"]
    assert worst[0] <= tol["eF"] and worst[1] <= e_tol and worst[2] <= tol["rho"], worst
    scmd.md_destroy(ctx)
