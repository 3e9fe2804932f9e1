"""Thermostat properties of the GPU integrator that hold exactly, checked on the GPU itself (through the C ABI):

- the Langevin splitting B A O A B samples the configurations of a harmonic system exactly at any stable step
  (Leimkuhler and Matthews, 2013): 200 relaxed Ni13 icosahedra at 1 K in one batched context, whose 33
  vibrations are harmonic, give <U - U_min> = (3N - 6)/2 k_B T at dt = 20 fs (omega_max dt = 1.45), where a
  velocity-Verlet-plus-friction splitting overshoots by about 20 %;
- with tau = dt the Berendsen factor is sqrt(T_target / T_inst), so every step ends exactly on its target
  temperature, with forces acting and along a ramp. The library requires tau > dt, so the test takes
  tau = dt (1 + 1e-9), which lands within 1e-9 |T_inst - T_target| of the target.
"""
import numpy as np
import pytest

from paper_1210_3559_gb300 import inputs

pytestmark = pytest.mark.gpu
FP64, MIXED = 0, 1
KB = 8.617333262e-5


@pytest.fixture(scope="module")
def scmd():
    from paper_1210_3559_gb300 import build, scmd as s
    build.build()
    return s


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_gpu_baoab_samples_harmonic_configurations_exactly(scmd, prec):
    pos = inputs.mackay_icosahedron(1, 2.49)
    m = inputs.masses(13)
    # relax on the GPU: overdamped Langevin dynamics at 0 K
    ctx = scmd.md_create(scmd.config(precision=prec), [13], pos, None, m, scmd.sc_params())
    scmd.md_step(ctx, 3000, 2.0, scmd.thermostat(scmd.MD_LANGEVIN, 0.0, 0.0, gamma_per_ps=50.0, seed=1))
    p0 = scmd.md_get_state(ctx)[0]
    scmd.md_destroy(ctx)
    nc, T, dt, every, samples = 200, 1.0, 20.0, 20, 60
    pos_b = np.concatenate([p0 + 40.0 * b for b in range(nc)])
    ctx = scmd.md_create(scmd.config(precision=prec, obs_every=every, obs_capacity=samples + 8), [13] * nc, pos_b,
                         None, np.tile(m, nc), scmd.sc_params())
    E0, F0 = scmd.md_energy_forces(ctx)
    assert np.abs(F0).max() < (1e-9 if prec == FP64 else 2e-5)
    th = scmd.thermostat(scmd.MD_LANGEVIN, T, T, gamma_per_ps=5.0, seed=3)
    scmd.md_step(ctx, 50, dt, th)  # 1 ps: five friction times
    scmd.md_clear_history(ctx)
    scmd.md_step(ctx, every * samples, dt, th)
    hist = scmd.md_obs_history(ctx)
    scmd.md_destroy(ctx)
    assert len(hist) >= samples
    u = np.array([[h[b]["epot"] for b in range(nc)] for h in hist[-samples:]])
    ratio = ((u - E0[None, :]) / (0.5 * (3 * 13 - 6) * KB * T)).mean(axis=0)  # per cluster
    sem = ratio.std(ddof=1) / np.sqrt(nc)
    assert sem < 0.004
    assert ratio.mean() == pytest.approx(1.0, abs=0.012)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_gpu_berendsen_with_tau_equal_to_dt_lands_on_the_ramp_target_every_step(scmd, prec):
    pos = inputs.fcc_sphere(55)
    m = inputs.masses(55)
    vel = inputs.maxwell_boltzmann(pos, m, 900.0, seed=6)
    ctx = scmd.md_create(scmd.config(precision=prec), [55], pos, vel, m, scmd.sc_params())
    dt, T0, T1, n = 2.0, 700.0, 400.0, 6
    tau_ps = dt * 1e-3 * (1.0 + 1e-9)
    for k in range(n):  # one call per step: the target of a one-step call is its T0
        Tk = T0 + (T1 - T0) * k / n
        scmd.md_step(ctx, 1, dt, scmd.thermostat(scmd.MD_BERENDSEN, Tk, Tk, tau_ps=tau_ps))
        assert scmd.md_observables(ctx)[0]["T"] == pytest.approx(Tk, rel=1e-8)
    scmd.md_step(ctx, n, dt, scmd.thermostat(scmd.MD_BERENDSEN, T0, T1, tau_ps=tau_ps))
    assert scmd.md_observables(ctx)[0]["T"] == pytest.approx(T0 + (T1 - T0) * (n - 1) / n, rel=1e-8)
    scmd.md_destroy(ctx)
