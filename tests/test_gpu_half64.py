"""FP64 all pairs with each unordered pair evaluated once (MD_PATH_ALLPAIRS_HALF) against the FP64 oracle.

The tolerances are the FP64 ones of test_gpu_parity.py (e_F <= 1e-12, |dE|/|E| <= 1e-13, rho <= 1e-13,
trajectories <= 1e-9 A); the sizes cover one and several work units (32 x 16 atoms), ragged tiles and
half-tiles, single atoms, batches of uneven clusters and the padding between them."""
import numpy as np
import pytest

import oracle
from paper_1210_3559_gb300 import inputs

pytestmark = pytest.mark.gpu
FP64, MIXED = 0, 1


@pytest.fixture(scope="module")
def scmd():
    from paper_1210_3559_gb300 import build, scmd as s
    build.build()
    return s


def half(scmd, sizes, pos, vel=None, rcut=0.0, params=None, mass=None, **cfg):
    mass = inputs.masses(int(np.sum(sizes))) if mass is None else mass
    ctx = scmd.md_create(scmd.config(precision=FP64, path=scmd.MD_PATH_ALLPAIRS_HALF, **cfg), sizes, pos, vel, mass,
                         params or scmd.sc_params(rcut=rcut))
    assert scmd.md_get_path(ctx) == scmd.MD_PATH_ALLPAIRS_HALF
    return ctx


def check(F, E, rho, pos, p=None):
    Er, Fr, _, rhor = oracle.energy_forces(pos, p)
    nF = np.linalg.norm(Fr)
    if nF > 0:
        assert np.linalg.norm(F - Fr) / nF <= 1e-12
    else:
        assert np.abs(F).max() <= 1e-12
    if Er != 0:
        assert abs(E - Er) / abs(Er) <= 1e-13, (E, Er)
    nz = rhor > 0
    assert np.all(np.abs(rho[nz] - rhor[nz]) <= 1e-13 * rhor[nz])
    assert np.all(rho[~nz] == 0)


@pytest.mark.parametrize("n", [2, 3, 13, 16, 17, 31, 32, 33, 48, 55, 147, 301, 1000, 1100])
def test_single_cluster_matches_oracle(scmd, n):
    pos = inputs.jitter(inputs.fcc_sphere(n), 0.15, n) if n > 3 else \
        np.array([[0, 0, 0], [2.3, 0.4, -0.1], [1.1, 2.1, 0.3]], float)[:n]
    ctx = half(scmd, [n], pos)
    E, F = scmd.md_energy_forces(ctx)
    check(F, E[0], scmd.md_get_density(ctx), pos)


def test_batched_uneven_clusters(scmd):
    sizes = [1, 2, 55, 64, 65, 200, 513, 31, 33]
    pos = np.concatenate([inputs.jitter(inputs.fcc_sphere(n), 0.1, 10 + k) + 25.0 * k for k, n in enumerate(sizes)])
    ctx = half(scmd, sizes, pos)
    E, F = scmd.md_energy_forces(ctx)
    rho = scmd.md_get_density(ctx)
    off = np.concatenate([[0], np.cumsum(sizes)])
    for b in range(len(sizes)):
        s, e = off[b], off[b + 1]
        check(F[s:e], E[b], rho[s:e], pos[s:e])


def test_cutoff_and_general_exponents(scmd):
    pos = inputs.jitter(inputs.fcc_sphere(400), 0.1, 8)
    ctx = half(scmd, [400], pos, rcut=8.8)
    E, F = scmd.md_energy_forces(ctx)
    check(F, E[0], scmd.md_get_density(ctx), pos, oracle.params(rcut=8.8))
    p = dict(eps=2.5415e-3, c=144.41, a=4.09, n=12, m=6)
    pos = inputs.jitter(inputs.fcc_sphere(120, a=4.09), 0.1, 9)
    ctx = half(scmd, [120], pos, params=scmd.sc_params(**p), mass=inputs.masses(120, 107.87))
    E, F = scmd.md_energy_forces(ctx)
    check(F, E[0], scmd.md_get_density(ctx), pos, oracle.params(**p))


def test_agrees_with_ordered_pairs(scmd):
    pos = inputs.jitter(inputs.fcc_sphere(700), 0.15, 3)
    a = half(scmd, [700], pos)
    b = scmd.md_create(scmd.config(precision=FP64, path=scmd.MD_PATH_ALLPAIRS), [700], pos, None, inputs.masses(700))
    Ea, Fa = scmd.md_energy_forces(a)
    Eb, Fb = scmd.md_energy_forces(b)
    assert np.linalg.norm(Fa - Fb) / np.linalg.norm(Fb) <= 1e-13
    assert abs(Ea[0] - Eb[0]) <= 1e-13 * abs(Eb[0])


def test_trajectories_match_oracle(scmd):
    # NVE, a Langevin ramp and Berendsen, as the FP64 trajectory tests of the ordered-pair path
    pos = inputs.mackay_icosahedron(3, 2.49)
    vel = inputs.maxwell_boltzmann(pos, inputs.masses(147), 1500.0, seed=1)
    ctx = half(scmd, [147], pos, vel, graph_chunk=32)
    scmd.md_step(ctx, 100, 1.0)
    p, v, _ = scmd.md_get_state(ctx)
    ob = oracle.Batch([147], pos, vel, inputs.masses(147))
    ob.run(100, 1.0)
    assert np.max(np.abs(p - ob.pos)) <= 1e-9 and np.max(np.abs(v - ob.vel)) <= 1e-10

    sizes = [55, 80]
    pos = np.concatenate([inputs.fcc_sphere(55), inputs.fcc_sphere(80) + 30.0])
    vel = np.concatenate([inputs.maxwell_boltzmann(pos[:55], inputs.masses(55), 1200.0, seed=3),
                          inputs.maxwell_boltzmann(pos[55:], inputs.masses(80), 1200.0, seed=4)])
    ctx = half(scmd, sizes, pos, vel, graph_chunk=16)
    scmd.md_step(ctx, 40, 2.0, scmd.thermostat(scmd.MD_LANGEVIN, 1200.0, 900.0, gamma_per_ps=5.0, seed=99))
    p, _, _ = scmd.md_get_state(ctx)
    ob = oracle.Batch(sizes, pos, vel, inputs.masses(135))
    ob.run(40, 2.0, oracle.thermostat(oracle.LANGEVIN, 1200.0, 900.0, gamma_ps=5.0, seed=99))
    assert np.max(np.abs(p - ob.pos)) <= 1e-8

    pos = inputs.fcc_sphere(79)
    vel = inputs.maxwell_boltzmann(pos, inputs.masses(79), 600.0, seed=5)
    ctx = half(scmd, [79], pos, vel, graph_chunk=10)
    scmd.md_step(ctx, 30, 1.0, scmd.thermostat(scmd.MD_BERENDSEN, 900.0, 700.0, tau_ps=0.05))
    p, _, _ = scmd.md_get_state(ctx)
    ob = oracle.Batch([79], pos, vel, inputs.masses(79))
    ob.run(30, 1.0, oracle.thermostat(oracle.BERENDSEN, 900.0, 700.0, tau_ps=0.05))
    assert np.max(np.abs(p - ob.pos)) <= 1e-9


def test_observables_and_resume_bitwise(scmd):
    pos = inputs.fcc_sphere(200)
    m = inputs.masses(200)
    vel = inputs.maxwell_boltzmann(pos, m, 1500.0, seed=6)
    ctx = half(scmd, [200], pos, vel, obs_every=10, graph_chunk=25)
    o0 = scmd.md_observables(ctx)[0]
    ref = oracle.observables(pos, vel, m)
    assert o0["epot"] == pytest.approx(ref["epot"], rel=1e-13)
    assert o0["ekin"] == pytest.approx(ref["ekin"], rel=1e-13)
    th = scmd.thermostat(scmd.MD_LANGEVIN, 1500.0, 1500.0, gamma_per_ps=1.0, seed=7)
    a = half(scmd, [200], pos, vel, graph_chunk=25)
    scmd.md_step(a, 100, 2.0, th)
    pa, va, _ = scmd.md_get_state(a)
    b = half(scmd, [200], pos, vel, graph_chunk=25)
    scmd.md_step(b, 60, 2.0, th)
    pb, vb, sb = scmd.md_get_state(b)
    c = half(scmd, [200], pos, vel, graph_chunk=25)
    scmd.md_set_state(c, pb, vb, sb)
    scmd.md_step(c, 40, 2.0, th)
    pc, vc, sc = scmd.md_get_state(c)
    assert sc == 100 and np.array_equal(pa, pc) and np.array_equal(va, vc)
    # history of an NVE run: energies match the oracle at the end
    scmd.md_step(ctx, 50, 1.0)
    hist = scmd.md_obs_history(ctx)
    p, v, _ = scmd.md_get_state(ctx)
    assert hist[-1][0]["epot"] == pytest.approx(oracle.observables(p, v, m)["epot"], rel=1e-12)


def test_automatic_choice(scmd):
    def path(prec, n, p=None):
        pos = inputs.fcc_sphere(n)
        cfg = scmd.config(precision=prec) if p is None else scmd.config(precision=prec, path=p)
        return scmd.md_get_path(scmd.md_create(cfg, [n], pos, None, inputs.masses(n)))
    assert path(FP64, 2000) == scmd.MD_PATH_ALLPAIRS_HALF
    assert path(FP64, 1000) == scmd.MD_PATH_ALLPAIRS
    assert path(FP64, 2000, scmd.MD_PATH_ALLPAIRS) == scmd.MD_PATH_ALLPAIRS
    assert path(MIXED, 2000) == scmd.MD_PATH_ALLPAIRS
    # many small clusters: enough work units, but the ordered-pair kernels suit them better
    pos = np.concatenate([inputs.mackay_icosahedron(3, 2.49)] * 64)
    ctx = scmd.md_create(scmd.config(precision=FP64), [147] * 64, pos, None, inputs.masses(len(pos)))
    assert scmd.md_get_path(ctx) == scmd.MD_PATH_ALLPAIRS
    with pytest.raises(scmd.ScmdError) as e:
        path(MIXED, 100, scmd.MD_PATH_ALLPAIRS_HALF)
    assert e.value.status == scmd.MD_ERR_INVALID
