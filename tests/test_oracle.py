"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed forms
(dimer, bulk FCC lattice sums, harmonic dimer period, Ornstein-Uhlenbeck and
Berendsen recursions), finite differences, exact invariants and symmetry zeros,
and the published Philox known-answer vectors. No test re-types the oracle's
own loops.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1210_3559_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def golden_params():
    vals = {}
    for line in open(os.path.join(GOLDEN, "ni_sc_params.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v, _ = line.split()
        vals[k] = float(v)
    return vals


P = golden_params()
EPS, A, C, NN, MM = P["eps"], P["a"], P["c"], int(P["n"]), int(P["m"])


def test_golden_params_match_generator_defaults():
    # the generator module carries the same printed parameter set (Sec. II A)
    assert inputs.NI_SC == dict(eps=EPS, c=C, a=A, n=NN, m=MM)


# ------------------------------------------------------------------ dimer
def dimer_closed_form(r):
    """Two atoms: rho = s^m each, so U = eps [s^n - 2 c s^(m/2)] with s = a/r."""
    s = A / r
    U = EPS * (s ** NN - 2.0 * C * s ** (MM / 2))
    dUdr = EPS * (-NN * s ** NN + C * MM * s ** (MM / 2)) / r
    return U, dUdr


@pytest.mark.parametrize("r", [1.9, 2.041345, 2.3, 2.49, 3.1, 4.5, 7.0])
def test_dimer_energy_and_force_closed_form(r):
    U_ref, dUdr = dimer_closed_form(r)
    U, F, _, rho = oracle.energy_forces([[0, 0, 0], [r, 0, 0]])
    assert U == pytest.approx(U_ref, rel=1e-13, abs=1e-15)
    # F on atom 0 points along -x when the pair attracts (dU/dr > 0)
    assert F[0, 0] == pytest.approx(dUdr, rel=1e-12, abs=1e-14)
    assert F[1, 0] == pytest.approx(-dUdr, rel=1e-12, abs=1e-14)
    assert np.allclose(F[:, 1:], 0)
    assert rho[0] == pytest.approx((A / r) ** MM, rel=1e-14)


def test_dimer_minimum():
    # dU/dr = 0 at r0 = a (n / (c m))^(1 / (n - m/2)) = 2.041345 A, U(r0) = -4.234085 eV
    r0 = A * (NN / (C * MM)) ** (1.0 / (NN - MM / 2))
    assert r0 == pytest.approx(2.041345, abs=1e-6)
    U, F, _, _ = oracle.energy_forces([[0, 0, 0], [r0, 0, 0]])
    assert U == pytest.approx(-4.234085, abs=1e-6)
    assert np.abs(F).max() < 1e-12
    assert oracle.energy([[0, 0, 0], [r0 * 1.001, 0, 0]]) > U
    assert oracle.energy([[0, 0, 0], [r0 * 0.999, 0, 0]]) > U



def symmetric_closed_form(k, r):
    """k + 1 atoms at mutual distance r (k = 2: equilateral triangle, k = 3: regular tetrahedron).
    Each atom has k neighbours at r, so rho = k s^m and U = (k + 1) eps [(k/2) s^n - c sqrt(k) s^(m/2)]
    with s = a/r; the embedding's sqrt(k) is what a pairwise form cannot give."""
    s = A / r
    U = (k + 1) * EPS * (0.5 * k * s ** NN - C * np.sqrt(k) * s ** (MM / 2))
    dUdr = (k + 1) * EPS * (-0.5 * k * NN * s ** NN + C * np.sqrt(k) * (MM / 2) * s ** (MM / 2)) / r
    return U, dUdr, k * s ** MM


@pytest.mark.parametrize("r", [2.3, 2.49, 3.0, 4.5])
def test_trimer_and_tetramer_closed_forms(r):
    tri = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0], [0.5 * r, 0.5 * np.sqrt(3.0) * r, 0.0]])
    tet = np.array([[1, 1, 1], [1, -1, -1], [-1, 1, -1], [-1, -1, 1]], dtype=np.float64) * r / (2 * np.sqrt(2.0))
    for k, pos in ((2, tri), (3, tet)):
        U_ref, dUdr, rho_ref = symmetric_closed_form(k, r)
        U, F, (e_pair, e_emb), rho = oracle.energy_forces(pos)
        assert U == pytest.approx(U_ref, rel=1e-13)
        assert e_emb == pytest.approx(-(k + 1) * EPS * C * np.sqrt(rho_ref), rel=1e-13)
        assert np.allclose(rho, rho_ref, rtol=1e-14, atol=0)
        # forces are radial from the centroid, all of one magnitude f; the virial of a uniform dilation,
        # sum_i F_i . (r_i - R) = -r dU/dr, fixes f
        d = pos - pos.mean(axis=0)
        R = np.linalg.norm(d[0])
        f = -r * dUdr / ((k + 1) * R)
        assert np.allclose(F, f * d / R, rtol=1e-12, atol=1e-14 * abs(f) + 1e-16)


# ------------------------------------------------------------ bulk lattice
def fcc_lattice_sums(kmax=36):
    """S_k = sum over FCC sites R != 0 of (a/|R|)^k, with an r^-3 continuum tail for S_6."""
    r = np.arange(-kmax, kmax + 1)
    i, j, k = np.meshgrid(r, r, r, indexing="ij")
    keep = ((i + j + k) % 2 == 0) & ((i != 0) | (j != 0) | (k != 0))
    d2 = (i[keep] ** 2 + j[keep] ** 2 + k[keep] ** 2) * 0.25  # |R|^2 / a^2
    Rc = kmax * 0.5 * 0.999
    inside = d2 < Rc * Rc
    S9 = np.sum(d2[inside] ** -4.5)
    S6 = np.sum(d2[inside] ** -3.0)
    density = 4.0  # sites per a^3
    S6 += 4 * np.pi * density / (3 * Rc ** 3)
    S9 += 4 * np.pi * density / (6 * Rc ** 6)
    return S9, S6


def test_bulk_lattice_sums_and_paper_parameters():
    S9, S6 = fcc_lattice_sums()
    assert S9 == pytest.approx(282.6741, abs=2e-3)
    assert S6 == pytest.approx(115.631, abs=2e-3)
    # zero pressure at a = 3.52 A requires c = n S9 / (m sqrt(S6)); the paper's c agrees
    assert NN * S9 / (MM * np.sqrt(S6)) == pytest.approx(C, abs=2e-3)
    assert EPS * (0.5 * S9 - C * np.sqrt(S6)) == pytest.approx(-4.4401, abs=2e-4)


def test_centre_atom_of_fcc_sphere_tends_to_bulk_cohesive_energy():
    S9, S6 = fcc_lattice_sums()
    pos = inputs.fcc_sphere(4000)
    e = oracle.atom_energies(pos)
    # finite sphere: add the missing continuum tail of rho beyond the sphere radius
    R = np.sqrt((pos ** 2).sum(1)).max() + 0.5 * A / np.sqrt(2)
    n0 = 4.0 / A ** 3
    rho_tail = 4 * np.pi * n0 * A ** 6 / (3 * R ** 3)
    rho0 = oracle.density(pos)[0]
    assert rho0 + rho_tail == pytest.approx(S6, rel=2e-3)
    e0 = e[0] - EPS * C * (np.sqrt(rho0 + rho_tail) - np.sqrt(rho0))
    assert e0 == pytest.approx(EPS * (0.5 * S9 - C * np.sqrt(S6)), abs=2e-3)


# ----------------------------------------------------------------- forces
def numeric_forces(pos, p, h=1e-5):
    F = np.zeros_like(pos)
    for i in range(len(pos)):
        for c in range(3):
            xp = pos.copy(); xp[i, c] += h
            xm = pos.copy(); xm[i, c] -= h
            F[i, c] = -(oracle.energy(xp, p) - oracle.energy(xm, p)) / (2 * h)
    return F


@pytest.mark.parametrize("n,seed", [(3, 1), (13, 2), (38, 3)])
def test_forces_match_central_differences(n, seed):
    pos = inputs.jitter(inputs.fcc_sphere(n), 0.15, seed)
    p = oracle.params()
    _, F, _, _ = oracle.energy_forces(pos, p)
    Fn = numeric_forces(pos, p)
    err = np.linalg.norm(F - Fn) / np.linalg.norm(F)
    assert err < 1e-8


def test_forces_with_cutoff_match_central_differences():
    # strict truncation r < rcut for both rho and the pair term; the jittered
    # configuration keeps every pair more than 1e-3 A away from the cutoff
    pos = inputs.jitter(inputs.fcc_sphere(43), 0.1, 7)
    rc = 5.3
    d = np.linalg.norm(pos[:, None] - pos[None], axis=-1)
    assert np.min(np.abs(d[np.triu_indices(len(pos), 1)] - rc)) > 1e-3
    p = oracle.params(rcut=rc)
    _, F, _, _ = oracle.energy_forces(pos, p)
    Fn = numeric_forces(pos, p)
    assert np.linalg.norm(F - Fn) / np.linalg.norm(F) < 1e-8
    # the truncated energy differs from the all-pairs one
    assert oracle.energy(pos, p) != pytest.approx(oracle.energy(pos), rel=1e-6)


def test_cutoff_pairs_beyond_range_vanish_and_isolated_atom_is_zero():
    p = oracle.params(rcut=8.8)
    U, F, et, rho = oracle.energy_forces([[0, 0, 0], [8.8, 0, 0]], p)  # r == rcut: excluded
    assert U == 0 and np.all(F == 0) and np.all(rho == 0)
    U, F, et, rho = oracle.energy_forces([[0, 0, 0], [8.79, 0, 0]], p)
    assert U < 0 and rho[0] > 0
    U, F, et, rho = oracle.energy_forces([[1.0, 2.0, 3.0]])  # N = 1
    assert U == 0 and np.all(F == 0) and rho[0] == 0


def test_net_force_and_torque_vanish():
    pos = inputs.jitter(inputs.fcc_sphere(300), 0.3, 11)
    _, F, _, _ = oracle.energy_forces(pos)
    scale = np.abs(F).sum()
    assert np.abs(F.sum(0)).max() < 1e-13 * scale
    torque = np.cross(pos, F).sum(0)
    assert np.abs(torque).max() < 1e-12 * scale * np.abs(pos).max()


def test_invariance_under_permutation_rotation_translation():
    pos = inputs.jitter(inputs.fcc_sphere(200), 0.2, 5)
    U, F, _, rho = oracle.energy_forces(pos)
    rng = np.random.Generator(np.random.PCG64(3))
    perm = rng.permutation(len(pos))
    U2, F2, _, rho2 = oracle.energy_forces(pos[perm])
    assert U2 == pytest.approx(U, rel=1e-13)
    assert np.allclose(F2, F[perm], rtol=0, atol=1e-12 * np.abs(F).max())
    Rm = inputs.random_rotation(9)
    shift = np.array([12.5, -7.25, 3.0])
    U3, F3, _, rho3 = oracle.energy_forces(pos @ Rm.T + shift)
    assert U3 == pytest.approx(U, rel=1e-12)
    assert np.allclose(F3, F @ Rm.T, rtol=0, atol=1e-11 * np.abs(F).max())
    assert np.allclose(rho3, rho, rtol=1e-12)


@pytest.mark.parametrize("n", [13, 19, 43, 55, 79, 87])
def test_centre_of_closed_fcc_shell_feels_no_force(n):
    pos = inputs.fcc_sphere(n)
    _, F, _, _ = oracle.energy_forces(pos)
    assert np.abs(F[0]).max() < 1e-12 * np.abs(F).max() + 1e-13


def test_mackay_icosahedron_centre_and_symmetry():
    pos = inputs.mackay_icosahedron(3, 2.49)
    assert len(pos) == 147
    U, F, _, rho = oracle.energy_forces(pos)
    assert np.abs(F[0]).max() < 1e-12
    # all 12 vertices of the first shell are equivalent
    r = np.linalg.norm(pos, axis=1)
    first = np.abs(r - 2.49 * 0.9510565162951535) < 1e-6
    assert first.sum() == 12
    assert np.ptp(rho[first]) < 1e-11 * rho[first].max()


# -------------------------------------------------------------- integrator
def conv():
    return oracle.ev_per_amu_a2_fs2()


def test_unit_constants():
    assert conv() == pytest.approx(9.648533212e-3, rel=1e-9)
    assert oracle.kb() == 8.617333262e-5


def test_dimer_small_oscillation_period_matches_harmonic_closed_form():
    # U''(r0) from the closed form of the dimer; omega^2 = U'' / mu with mu = m/2
    r0 = A * (NN / (C * MM)) ** (1.0 / (NN - MM / 2))
    s = A / r0
    Upp = EPS * (NN * (NN + 1) * s ** NN - C * (MM / 2) * (MM / 2 + 1) * 2 * s ** (MM / 2)) / r0 ** 2
    m = inputs.NI_MASS_AMU
    omega = np.sqrt(Upp * conv() / (m / 2))  # rad/fs
    period = 2 * np.pi / omega
    amp = 1e-3
    b = oracle.Batch([2], [[0, 0, 0], [r0 + amp, 0, 0]], np.zeros((2, 3)), [m, m])
    dt = 0.05
    rs = []
    for _ in range(int(3 * period / dt)):
        b.run(1, dt)
        rs.append(b.pos[1, 0] - b.pos[0, 0] - r0)
    rs = np.array(rs)
    # upward zero crossings, linear interpolation
    idx = np.where((rs[:-1] < 0) & (rs[1:] >= 0))[0]
    t = (idx + 1 - rs[idx + 1] / (rs[idx + 1] - rs[idx])) * dt
    measured = np.diff(t).mean()
    assert measured == pytest.approx(period, rel=2e-3)



def test_observables_of_a_spinning_dimer_closed_forms():
    # two atoms of unequal mass, centre of mass X moving at V, spinning at omega about z through X:
    # P = M V, L (about X) = mu r^2 omega, E_kin = 1/2 M V^2 + 1/2 mu r^2 omega^2 (Koenig), U = dimer(r)
    m1, m2, r = inputs.NI_MASS_AMU, 2.0 * inputs.NI_MASS_AMU, 2.49
    M, mu = m1 + m2, m1 * m2 / (m1 + m2)
    X, V, w = np.array([1.0, -2.0, 0.5]), np.array([0.01, 0.002, -0.003]), 0.004
    pos = np.array([X - (m2 / M) * r * np.array([1.0, 0, 0]), X + (m1 / M) * r * np.array([1.0, 0, 0])])
    vel = V + np.cross(np.array([0, 0, w]), pos - X)
    o = oracle.observables(pos, vel, [m1, m2])
    assert np.allclose(o["com"], X, rtol=0, atol=1e-14)
    assert np.allclose(o["mom"], M * V, rtol=1e-13, atol=1e-16)
    assert np.allclose(o["angmom"], [0.0, 0.0, mu * r * r * w], rtol=1e-12, atol=1e-15)
    ekin = (0.5 * M * V @ V + 0.5 * mu * r * r * w * w) / conv()
    assert o["ekin"] == pytest.approx(ekin, rel=1e-13)
    assert o["T"] == pytest.approx(2 * ekin / (3 * 2 * oracle.kb()), rel=1e-13)
    assert o["epot"] == pytest.approx(dimer_closed_form(r)[0], rel=1e-13)
    assert o["etot"] == pytest.approx(o["epot"] + o["ekin"], rel=1e-15)


def nve_fluct(dt, nsteps):
    pos = inputs.mackay_icosahedron(2, 2.49)
    m = inputs.masses(len(pos))
    vel = inputs.maxwell_boltzmann(pos, m, 600.0, seed=1)
    b = oracle.Batch([len(pos)], pos, vel, m)
    E = []
    for _ in range(nsteps):
        b.run(1, dt)
        E.append(b.observables()[0]["etot"])
    E = np.array(E)
    return E, b


def test_nve_energy_fluctuation_scales_as_dt_squared_and_conserves_momenta():
    E1, b1 = nve_fluct(1.0, 200)
    E2, _ = nve_fluct(0.5, 400)
    f1, f2 = np.std(E1), np.std(E2[1::2])
    assert 3.0 < f1 / f2 < 5.0
    assert abs(E1[-1] - E1[0]) / len(b1.pos) < 1e-4
    o = b1.observables()[0]
    assert np.abs(o["mom"]).max() < 1e-12
    assert np.abs(o["angmom"]).max() < 1e-9


def test_langevin_free_atoms_follow_exact_ornstein_uhlenbeck():
    # N = 1 clusters have U = 0, so the O step alone drives the velocities:
    # var(v_x) relaxes to k_B T / m and the lag-K autocorrelation is exp(-gamma K dt)
    n = 4000
    m = inputs.NI_MASS_AMU
    b = oracle.Batch(np.ones(n, np.int32), np.zeros((n, 3)), np.zeros((n, 3)), np.full(n, m))
    T, gamma, dt = 900.0, 20.0, 2.0
    th = oracle.thermostat(oracle.LANGEVIN, T, T, gamma_ps=gamma, seed=77)
    b.run(400, dt, th)
    v0 = b.vel.copy()
    var_target = oracle.kb() * T * conv() / m
    sv = v0.var()
    assert sv == pytest.approx(var_target, rel=4 * np.sqrt(2.0 / (3 * n)))
    K = 10
    b.run(K, dt, th)
    rho = (v0 * b.vel).mean() / np.sqrt((v0 * v0).mean() * (b.vel * b.vel).mean())
    assert rho == pytest.approx(np.exp(-gamma * 1e-3 * K * dt), abs=4 / np.sqrt(3 * n))


def test_langevin_ramp_follows_variance_recursion():
    # with a ramp T_k = T0 + (T1 - T0) k / n the variance obeys
    # s_{k+1} = c1^2 s_k + (1 - c1^2) k_B T_k / m exactly in expectation
    n, m = 6000, inputs.NI_MASS_AMU
    b = oracle.Batch(np.ones(n, np.int32), np.zeros((n, 3)), np.zeros((n, 3)), np.full(n, m))
    T0, T1, gamma, dt, steps = 2000.0, 300.0, 100.0, 2.0, 50
    b.run(steps, dt, oracle.thermostat(oracle.LANGEVIN, T0, T1, gamma_ps=gamma, seed=5))
    c1 = np.exp(-gamma * 1e-3 * dt)
    s = 0.0
    for k in range(steps):
        Tk = T0 + (T1 - T0) * k / steps
        s = c1 * c1 * s + (1 - c1 * c1) * oracle.kb() * Tk * conv() / m
    assert b.vel.var() == pytest.approx(s, rel=4 * np.sqrt(2.0 / (3 * n)))



def relaxed_icosahedron13():
    """The 13-atom Mackay icosahedron relaxed to its minimum by overdamped Langevin dynamics at 0 K."""
    pos = inputs.mackay_icosahedron(1, 2.49)
    m = inputs.masses(13)
    b = oracle.Batch([13], pos, np.zeros_like(pos), m)
    b.run(3000, 2.0, oracle.thermostat(oracle.LANGEVIN, 0.0, 0.0, gamma_ps=50.0, seed=1))
    return b.pos.copy(), m


def test_langevin_baoab_samples_harmonic_configurations_exactly():
    """The Langevin splitting B A O A B samples the configurational distribution of a harmonic system exactly
    at any stable step (Leimkuhler and Matthews, 2013), which velocity Verlet with a friction step after it,
    or a full drift before the friction step, do not. At 1 K the 33 vibrations of a relaxed Ni13 icosahedron
    are harmonic (omega 0.016 to 0.073 rad/fs), so equipartition gives <U - U_min> = (3N - 6)/2 k_B T even at
    dt = 20 fs (omega_max dt = 1.45), where those other splittings overshoot by 17-21 %. Rotation and
    translation leave U unchanged; the cluster turns by under 0.02 rad per step, so straight-line drifts add
    no measurable strain."""
    p0, m = relaxed_icosahedron13()
    U0, F0, _, _ = oracle.energy_forces(p0)
    assert np.abs(F0).max() < 1e-10
    nc, T, dt = 200, 1.0, 20.0
    B = oracle.Batch(np.full(nc, 13, np.int32), np.tile(p0, (nc, 1)), np.zeros((13 * nc, 3)), np.tile(m, nc))
    th = oracle.thermostat(oracle.LANGEVIN, T, T, gamma_ps=5.0, seed=3)
    B.run(50, dt, th)  # 1 ps: five friction times
    u = []
    for _ in range(60):
        B.run(20, dt, th)
        u.append([o["epot"] for o in B.observables()])
    ratio = ((np.array(u) - U0) / (0.5 * (3 * 13 - 6) * oracle.kb() * T)).mean(axis=0)  # per cluster
    sem = ratio.std(ddof=1) / np.sqrt(nc)
    assert sem < 0.004
    assert ratio.mean() == pytest.approx(1.0, abs=0.012)


def test_berendsen_free_atoms_follow_closed_form_relaxation():
    # U = 0: T' = lambda^2 T = T + (dt/tau)(T0 - T), so T_k = T0 + (Ti - T0)(1 - dt/tau)^k
    n, m = 50, inputs.NI_MASS_AMU
    rng = np.random.Generator(np.random.PCG64(2))
    v = rng.standard_normal((n, 3)) * 0.01
    b = oracle.Batch(np.full(1, n, np.int32), inputs.fcc_sphere(n) * 100.0, v, np.full(n, m),
                     oracle.params(rcut=5.0))
    Ti = b.observables()[0]["T"]
    T0, dt, tau = 500.0, 1.0, 0.05
    b.run(30, dt, oracle.thermostat(oracle.BERENDSEN, T0, T0, tau_ps=tau))
    expect = T0 + (Ti - T0) * (1 - dt / (tau * 1e3)) ** 30
    assert b.observables()[0]["T"] == pytest.approx(expect, rel=1e-12)



def test_berendsen_with_tau_equal_to_dt_lands_on_the_ramp_target_every_step():
    # with tau = dt the factor is sqrt(T_target / T_inst): rescaling the velocities that end the step sets
    # T to the step's target exactly, forces or not; with a ramp the target of local step k is
    # T0 + (T1 - T0) k / n
    pos = inputs.fcc_sphere(55)
    m = inputs.masses(55)
    vel = inputs.maxwell_boltzmann(pos, m, 900.0, seed=6)
    b = oracle.Batch([55], pos, vel, m)
    dt, T0, T1, n = 2.0, 700.0, 400.0, 6
    for k in range(n):  # one call per step: the target of a one-step call is its T0
        Tk = T0 + (T1 - T0) * k / n
        b.run(1, dt, oracle.thermostat(oracle.BERENDSEN, Tk, Tk, tau_ps=dt * 1e-3))
        assert b.observables()[0]["T"] == pytest.approx(Tk, rel=1e-13)
    b.run(n, dt, oracle.thermostat(oracle.BERENDSEN, T0, T1, tau_ps=dt * 1e-3))
    assert b.observables()[0]["T"] == pytest.approx(T0 + (T1 - T0) * (n - 1) / n, rel=1e-13)


def test_langevin_run_is_reproducible_and_resumable():
    pos = inputs.fcc_sphere(55)
    m = inputs.masses(55)
    vel = inputs.maxwell_boltzmann(pos, m, 1000.0, seed=4)
    th = oracle.thermostat(oracle.LANGEVIN, 1000.0, 800.0, gamma_ps=1.0, seed=9)
    a = oracle.Batch([55], pos, vel, m)
    a.run(20, 2.0, oracle.thermostat(oracle.LANGEVIN, 1000.0, 1000.0, gamma_ps=1.0, seed=9))
    b = oracle.Batch([55], pos, vel, m)
    b.run(10, 2.0, oracle.thermostat(oracle.LANGEVIN, 1000.0, 1000.0, gamma_ps=1.0, seed=9))
    b.run(10, 2.0, oracle.thermostat(oracle.LANGEVIN, 1000.0, 1000.0, gamma_ps=1.0, seed=9))
    assert np.array_equal(a.pos, b.pos) and np.array_equal(a.vel, b.vel)
    del th


# ---------------------------------------------------------- Philox, normals
def kat_vectors():
    out = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        out.append((w[0:4], w[4:6], w[6:10]))
    return out


@pytest.mark.parametrize("ctr,key,expect", kat_vectors())
def test_philox_known_answer_vectors(ctr, key, expect):
    assert list(oracle.philox4x32_10(ctr, key)) == expect


def test_philox_matches_aten_engine():
    """Cross-check against PyTorch's independent C++ Philox4x32-10 engine header."""
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    hdr = os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")
    cuda_inc = "/usr/local/cuda/include"
    if not os.path.exists(hdr) or shutil.which("g++") is None or not os.path.isdir(cuda_inc):
        pytest.skip("ATen Philox header or g++ not available")
    import tempfile
    src = r"""
#include <ATen/core/PhiloxRNGEngine.h>
#include <cstdio>
int main(){
  unsigned long long cases[3][3] = {{0ull,0ull,0ull},{0x123456789abcdefull, 77ull, 5ull},{42ull, 0xdeadbeefcafeull, 1ull<<33}};
  for (auto& c: cases){ at::Philox4_32 e(c[0], c[1], c[2]);
    for(int k=0;k<4;k++) printf("%u ", e()); printf("\n"); }
}
"""
    with tempfile.TemporaryDirectory() as d:
        cpp = os.path.join(d, "t.cpp")
        open(cpp, "w").write(src)
        exe = os.path.join(d, "t")
        r = subprocess.run(["g++", "-std=c++17", "-I", inc, "-I", cuda_inc, cpp, "-o", exe],
                           capture_output=True, text=True)
        if r.returncode != 0:
            pytest.skip("could not compile against the ATen header: " + r.stderr[-300:])
        lines = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split("\n")
    cases = [(0, 0, 0), (0x123456789ABCDEF, 77, 5), (42, 0xDEADBEEFCAFE, 1 << 33)]
    for (seed, sub, off), line in zip(cases, lines):
        got = [int(x) for x in line.split()]
        # ATen: key = seed, counter = (offset lo, offset hi, subsequence lo, subsequence hi)
        ctr = [off & 0xFFFFFFFF, off >> 32, sub & 0xFFFFFFFF, sub >> 32]
        key = [seed & 0xFFFFFFFF, seed >> 32]
        assert list(oracle.philox4x32_10(ctr, key)) == got


def test_box_muller_normals_moments_and_counter_layout():
    z = np.array([oracle.langevin_normals(123, c, s, a) for c in range(4) for s in range(50) for a in range(40)])
    assert z.shape == (8000, 3)
    n = z.size
    assert abs(z.mean()) < 4 / np.sqrt(n)
    assert z.var() == pytest.approx(1.0, abs=4 * np.sqrt(2.0 / n))
    assert abs(np.mean(z ** 4) - 3.0) < 0.25
    assert abs(np.corrcoef(z[:, 0], z[:, 1])[0, 1]) < 4 / np.sqrt(len(z))
    # the first two normals come from (w0, w1) of Philox((atom, cluster, step lo, step hi), seed)
    w = oracle.philox4x32_10([7, 3, 11, 0], [123, 0])
    u1 = (w[0] + 1.0) / 2 ** 32
    u2 = (w[1] + 1.0) / 2 ** 32
    r = np.sqrt(-2 * np.log(u1))
    zz = oracle.langevin_normals(123, 3, 11, 7)
    assert zz[0] == pytest.approx(r * np.cos(2 * np.pi * u2), rel=1e-14, abs=1e-15)
    assert zz[1] == pytest.approx(r * np.sin(2 * np.pi * u2), rel=1e-14, abs=1e-15)


# ------------------------------------------------------------- generators
def test_fcc_sphere_counts_and_shells():
    for n in [1, 13, 55, 79, 147, 2000, 2047]:
        x = inputs.fcc_sphere(n)
        assert x.shape == (n, 3)
        assert len(np.unique(np.round(x, 6), axis=0)) == n
    x = inputs.fcc_sphere(13)
    d = np.linalg.norm(x[1:], axis=1)
    assert np.allclose(d, A / np.sqrt(2))


def test_maxwell_boltzmann_temperature_and_momenta():
    pos = inputs.fcc_sphere(2000)
    m = inputs.masses(2000)
    v = inputs.maxwell_boltzmann(pos, m, 2000.0, seed=2, dof="3N")
    o = oracle.observables(pos, v, m)
    assert o["T"] == pytest.approx(2000.0, rel=1e-12)
    assert np.abs(o["mom"]).max() < 1e-12
    assert np.abs(o["angmom"]).max() < 1e-9


# ------------------------------------------------------------ shifted cutoff
@pytest.mark.parametrize("r", [2.3, 2.6, 4.0, 8.0])
def test_shifted_dimer_closed_form(r):
    """Two atoms: each has rho = (a/r)^m - (a/rc)^m, so U = eps [(a/r)^n - (a/rc)^n
    - 2 c sqrt((a/r)^m - (a/rc)^m)]; F = -dU/dr along the axis."""
    eps, c, a, n, m, rc = 1.5707e-2, 39.432, 3.52, 9, 6, 8.8
    p = oracle.params(rcut=rc, shift=True)
    U, F, _, rho = oracle.energy_forces([[0, 0, 0], [r, 0, 0]], p)
    sn, sm, cn, cm = (a / r) ** n, (a / r) ** m, (a / rc) ** n, (a / rc) ** m
    assert U == pytest.approx(eps * ((sn - cn) - 2 * c * np.sqrt(sm - cm)), rel=1e-13)
    assert rho[0] == pytest.approx(sm - cm, rel=1e-13)
    dU = eps * (-n * sn / r + c * m * sm / r / np.sqrt(sm - cm))
    assert F[1][0] == pytest.approx(-dU, rel=1e-12) and F[0][0] == pytest.approx(dU, rel=1e-12)


def test_shifted_energy_is_continuous_at_the_cutoff():
    """A dimer approaching rc from inside: the shifted energy goes to zero like sqrt(rc - r) (the
    embedding term), the truncated one keeps a finite jump. In a cluster, a pair crossing rc leaves
    the shifted energy continuous: along a path that carries one pair through rc, consecutive
    energies differ by no more than the force times the step, while the truncated energy jumps."""
    rc = 8.8
    ps, pt = oracle.params(rcut=rc, shift=True), oracle.params(rcut=rc)
    u1 = oracle.energy([[0, 0, 0], [rc - 1e-6, 0, 0]], ps)
    u2 = oracle.energy([[0, 0, 0], [rc - 1e-8, 0, 0]], ps)
    assert abs(u1) < 1e-4 and u1 / u2 == pytest.approx(10.0, rel=1e-3)
    assert oracle.energy([[0, 0, 0], [rc - 1e-8, 0, 0]], pt) < -0.07
    pos = inputs.jitter(inputs.fcc_sphere(43), 0.1, 7)
    k = int(np.argmax(np.linalg.norm(pos, axis=1)))
    u = pos[k] / np.linalg.norm(pos[k])
    # carry atom k outwards by 1 A in steps of 1e-4 A: several pairs leave rc on the way
    steps = np.arange(0, 10001) * 1e-4
    d0 = np.linalg.norm(pos - pos[k], axis=1)
    crossing = np.sum((d0 < rc) & (np.linalg.norm(pos - (pos[k] + u), axis=1) >= rc))
    assert crossing > 0
    def path(p):  # energies and the work of the force along the path (trapezoid rule)
        E, W = [], []
        for t in steps[::50]:
            q = pos.copy()
            q[k] = pos[k] + t * u
            U, F, _, _ = oracle.energy_forces(q, p)
            E.append(U)
            W.append(F[k] @ u)
        E, W = np.array(E), np.array(W)
        return np.abs(np.diff(E) + 0.5 * (W[1:] + W[:-1]) * 50e-4)  # dE = -F.dx, up to O(dx^3)

    rs, rt = path(ps), path(pt)
    assert np.max(rs) < 1e-5                  # smooth where pairs cross rc
    assert np.max(rt) > 100 * np.max(rs)      # the truncated energy jumps there


def test_shifted_forces_match_central_differences():
    pos = inputs.jitter(inputs.fcc_sphere(43), 0.1, 7)
    rc = 5.3
    d = np.linalg.norm(pos[:, None] - pos[None], axis=-1)
    assert np.min(np.abs(d[np.triu_indices(len(pos), 1)] - rc)) > 1e-3
    p = oracle.params(rcut=rc, shift=True)
    _, F, _, _ = oracle.energy_forces(pos, p)
    Fn = numeric_forces(pos, p)
    assert np.linalg.norm(F - Fn) / np.linalg.norm(F) < 1e-8
    # the shift lowers every rho by (a/rc)^m per neighbour inside rc
    _, _, _, rho_t = oracle.energy_forces(pos, oracle.params(rcut=rc))
    _, _, _, rho_s = oracle.energy_forces(pos, p)
    nin = np.sum((d < rc) & (d > 0), axis=1)
    assert np.allclose(rho_t - rho_s, nin * (3.52 / rc) ** 6, rtol=1e-10, atol=0)
