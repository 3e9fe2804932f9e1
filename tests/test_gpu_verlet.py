"""GPU parity of the neighbour-list path (strict cutoff, lists of rcut + 1 A rebuilt after 0.5 A of
motion; per-atom lists in FP64, lists of atom quads in MIXED) against the FP64 oracle with the same
cutoff. The FP64 forces do not depend on when the lists were built, so a resumed run matches an
uninterrupted one bit for bit; MIXED sums in list order, so there it agrees to rounding, and repeated
runs are bitwise identical.

Inputs and tolerances as for the cell-list path (fcc spheres with 0.03 A of disorder, whose pair
distances keep at least 0.02 A away from rcut = 8.8 A; e_F <= 1e-12 / 1e-5 for FP64 / MIXED).
"""
import numpy as np
import pytest

import oracle
from paper_1210_3559_gb300 import inputs

from test_gpu_parity import FP64, MIXED, TOL, check_cluster, make, rel_force_err
from test_gpu_cells import RC, lattice

pytestmark = pytest.mark.gpu

VERLET, CELLS = 3, 2


@pytest.fixture(scope="module")
def scmd():
    from paper_1210_3559_gb300 import build, scmd as s
    build.build()
    return s


@pytest.mark.parametrize("prec", [FP64, MIXED])
@pytest.mark.parametrize("n", [700, 6000])
def test_verlet_energy_forces_density(scmd, prec, n):
    pos = lattice(n, 31)
    ctx = make(scmd, [n], pos, prec=prec, rcut=RC, path=VERLET)
    assert scmd.md_get_path(ctx) == VERLET
    E, F = scmd.md_energy_forces(ctx)
    check_cluster(F, E[0], scmd.md_get_density(ctx), pos, prec, rcut=RC)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_verlet_full_size_parity(scmd, prec):
    pos = lattice(50000, 32)
    ctx = make(scmd, [50000], pos, prec=prec, rcut=RC, path=VERLET)
    E, F = scmd.md_energy_forces(ctx)
    check_cluster(F, E[0], scmd.md_get_density(ctx), pos, prec, rcut=RC)
    _, _, tested = scmd.md_time_passes(ctx, 3)
    if prec == FP64:  # list entries: ~ (9.8 / 8.8)^3 x the pairs inside rcut
        assert 224 * 50000 < tested < 600 * 50000
    else:  # 4 pairs per listed atom: ~2.2 x the pairs inside rcut (~500 per atom)
        assert 224 * 50000 < tested < 700 * 50000


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_verlet_batch_far_atoms(scmd, prec):
    big = lattice(400, 33)
    big[5] = big[5] + np.array([60.0, 0.0, 0.0])
    parts = [np.zeros((1, 3)), np.array([[0.0, 0.0, 0.0], [2.6, 0.1, 0.0]]), inputs.fcc_sphere(13), big]
    sizes = [len(p) for p in parts]
    pos = np.concatenate([p + 40.0 * b for b, p in enumerate(parts)])
    ctx = make(scmd, sizes, pos, prec=prec, rcut=RC, path=VERLET)
    E, F = scmd.md_energy_forces(ctx)
    rho = scmd.md_get_density(ctx)
    off = np.concatenate([[0], np.cumsum(sizes)])
    for b in range(len(sizes)):
        s, e = off[b], off[b + 1]
        check_cluster(F[s:e], E[b], rho[s:e], pos[s:e], prec, rcut=RC)


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-8), (MIXED, 5e-4)])
def test_verlet_langevin_trajectory(scmd, prec, tol):
    sizes = [147, 300]
    pos = np.concatenate([inputs.mackay_icosahedron(3, 2.49), inputs.fcc_sphere(300) + 50.0])
    m = inputs.masses(447)
    vel = np.concatenate([inputs.maxwell_boltzmann(pos[:147], m[:147], 1400.0, seed=3),
                          inputs.maxwell_boltzmann(pos[147:], m[147:], 1400.0, seed=4)])
    th = scmd.thermostat(scmd.MD_LANGEVIN, 1400.0, 1000.0, gamma_per_ps=5.0, seed=17)
    ctx = make(scmd, sizes, pos, vel, prec=prec, rcut=RC, path=VERLET, graph_chunk=16)
    scmd.md_step(ctx, 40, 2.0, th)
    p, _, _ = scmd.md_get_state(ctx)
    ob = oracle.Batch(sizes, pos, vel, m, oracle.params(rcut=RC))
    ob.run(40, 2.0, oracle.thermostat(oracle.LANGEVIN, 1400.0, 1000.0, gamma_ps=5.0, seed=17))
    assert np.max(np.abs(p - ob.pos)) <= tol


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_verlet_berendsen_trajectory_and_observables(scmd, prec):
    pos = inputs.fcc_sphere(300)
    m = inputs.masses(300)
    vel = inputs.maxwell_boltzmann(pos, m, 600.0, seed=5)
    th = scmd.thermostat(scmd.MD_BERENDSEN, 900.0, 700.0, tau_ps=0.05)
    ctx = make(scmd, [300], pos, vel, prec=prec, rcut=RC, path=VERLET, graph_chunk=10, obs_every=5)
    scmd.md_step(ctx, 30, 1.0, th)
    p, v, _ = scmd.md_get_state(ctx)
    ob = oracle.Batch([300], pos, vel, m, oracle.params(rcut=RC))
    ob.run(30, 1.0, oracle.thermostat(oracle.BERENDSEN, 900.0, 700.0, tau_ps=0.05))
    assert np.max(np.abs(p - ob.pos)) <= (1e-9 if prec == FP64 else 2e-4)
    hist = scmd.md_obs_history(ctx)
    ref = oracle.observables(p, v, m, oracle.params(rcut=RC))
    assert hist[-1][0]["epot"] == pytest.approx(ref["epot"], rel=1e-12 if prec == FP64 else 1e-6)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_verlet_lists_follow_large_motion(scmd, prec):
    """A hot liquid moves far beyond the skin within the run: the lists must be rebuilt (many
    times) for the forces of the final state to match the oracle. In a liquid, a few pairs lie within
    the FP32 rounding of rcut, where MIXED may decide the cutoff differently from the oracle; each
    such pair moves e_F by about (its pair force at rcut, ~2e-4 eV/A) / |F| ~ 1e-5, hence 5e-5."""
    pos = inputs.fcc_sphere(2000)
    vel = inputs.maxwell_boltzmann(pos, inputs.masses(2000), 3000.0, seed=12)
    th = scmd.thermostat(scmd.MD_LANGEVIN, 3000.0, 3000.0, gamma_per_ps=1.0, seed=5)
    ctx = make(scmd, [2000], pos, vel, prec=prec, rcut=RC, path=VERLET, graph_chunk=64)
    scmd.md_step(ctx, 1000, 2.0, th)
    p, _, _ = scmd.md_get_state(ctx)
    assert np.max(np.linalg.norm(p - pos, axis=1)) > 5.0  # far more than the 0.5 A rebuild trigger
    F = scmd.md_get_forces(ctx)  # the forces the integrator used at the final positions
    _, Fr, _, _ = oracle.energy_forces(p, oracle.params(rcut=RC))
    assert rel_force_err(F, Fr) <= (1e-11 if prec == FP64 else 5e-5)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_verlet_checkpoint_resume(scmd, prec):
    """The resumed context builds its lists at step 60; the uninterrupted one built them elsewhere.
    FP64: bit for bit. MIXED: to rounding (the quads and their order depend on the build), while a
    repeat of the same run is bit for bit."""
    pos = inputs.fcc_sphere(600)
    vel = inputs.maxwell_boltzmann(pos, inputs.masses(600), 1500.0, seed=6)
    th = scmd.thermostat(scmd.MD_LANGEVIN, 1500.0, 1500.0, gamma_per_ps=1.0, seed=7)
    kw = dict(prec=prec, rcut=RC, path=VERLET, graph_chunk=25)
    a = make(scmd, [600], pos, vel, **kw)
    scmd.md_step(a, 100, 2.0, th)
    pa, va, sa = scmd.md_get_state(a)
    b = make(scmd, [600], pos, vel, **kw)
    scmd.md_step(b, 60, 2.0, th)
    pb, vb, sb = scmd.md_get_state(b)
    c = make(scmd, [600], pos, vel, **kw)
    scmd.md_set_state(c, pb, vb, sb)
    scmd.md_step(c, 40, 2.0, th)
    pc, vc, sc = scmd.md_get_state(c)
    assert sa == sc == 100
    if prec == FP64:
        assert np.array_equal(pa, pc) and np.array_equal(va, vc)
    else:
        assert np.max(np.abs(pa - pc)) <= 1e-4
        d = make(scmd, [600], pos, vel, **kw)
        scmd.md_step(d, 100, 2.0, th)
        pd, vd, _ = scmd.md_get_state(d)
        assert np.array_equal(pa, pd) and np.array_equal(va, vd)


def test_verlet_matches_cells_bitwise_free(scmd):
    """Same input, both cutoff paths, MIXED: the same pairs, different coordinate frames (offsets from
    quad reference points against offsets from cell centres): agreement at the MIXED tolerance."""
    pos = lattice(3000, 34)
    a = make(scmd, [3000], pos, prec=MIXED, rcut=RC, path=VERLET)
    b = make(scmd, [3000], pos, prec=MIXED, rcut=RC, path=CELLS)
    Ea, Fa = scmd.md_energy_forces(a)
    Eb, Fb = scmd.md_energy_forces(b)
    assert rel_force_err(Fa, Fb) <= TOL[MIXED]["eF"]
    assert abs(Ea[0] - Eb[0]) <= TOL[MIXED]["E"] * abs(Eb[0])


def test_verlet_list_overflow_is_reported(scmd):
    """A dense simple-cubic blob (spacing 1.6 A): each cell holds fewer than its 256 atoms, but the
    atom at the centre, listed first, has ~960 higher-indexed partners within rcut + skin, more than
    a list holds (512). The overflow is detected on the device and reported; nothing is written out
    of bounds (a full list drops the extra entries), and the GPU stays usable."""
    g = (np.arange(12) - 5.5) * 1.6
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    blob = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    blob = blob[np.argsort(np.linalg.norm(blob, axis=1), kind="stable")]  # the centre atoms first
    with pytest.raises(scmd.ScmdError) as e:
        make(scmd, [len(blob)], blob, prec=FP64, rcut=RC, path=VERLET)
    assert e.value.status == scmd.MD_ERR_STATE
    assert "neighbour list" in scmd.md_last_error()
    pos = lattice(700, 36)
    ctx = make(scmd, [700], pos, prec=FP64, rcut=RC, path=VERLET)
    E, F = scmd.md_energy_forces(ctx)
    check_cluster(F, E[0], scmd.md_get_density(ctx), pos, FP64, rcut=RC)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_verlet_chunking_does_not_change_the_trajectory(scmd, prec):
    """Graph chunks of 7 and of 60 steps give the same trajectory bit for bit. In MIXED the position
    kernel runs only at a chunk's first step (the force pass that moves the atoms writes their offsets
    within a chunk), so this checks that both routes write the same offsets and displacement record."""
    pos = inputs.fcc_sphere(900)
    vel = inputs.maxwell_boltzmann(pos, inputs.masses(900), 2500.0, seed=13)
    th = scmd.thermostat(scmd.MD_LANGEVIN, 2500.0, 2500.0, gamma_per_ps=1.0, seed=14)
    out = []
    for chunk in (7, 60):
        ctx = make(scmd, [900], pos, vel, prec=prec, rcut=RC, path=VERLET, graph_chunk=chunk)
        scmd.md_step(ctx, 120, 2.0, th)
        out.append(scmd.md_get_state(ctx)[:2])
    assert np.array_equal(out[0][0], out[1][0]) and np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_verlet_many_clusters(scmd, prec):
    """30 clusters of 1 to 500 atoms in one context on the lists: every cluster against the oracle."""
    rng = np.random.default_rng(15)
    sizes = [int(x) for x in rng.integers(1, 501, 30)]
    parts = [inputs.jitter(inputs.fcc_sphere(n), 0.03, 40 + b) if n > 1 else np.zeros((1, 3))
             for b, n in enumerate(sizes)]
    pos = np.concatenate([p + 70.0 * b for b, p in enumerate(parts)])
    ctx = make(scmd, sizes, pos, prec=prec, rcut=RC, path=VERLET)
    E, F = scmd.md_energy_forces(ctx)
    rho = scmd.md_get_density(ctx)
    off = np.concatenate([[0], np.cumsum(sizes)])
    for b in range(len(sizes)):
        s, e = off[b], off[b + 1]
        check_cluster(F[s:e], E[b], rho[s:e], pos[s:e], prec, rcut=RC)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_verlet_isolated_small_groups(scmd, prec):
    """A sphere with a dimer, a trimer and a tetramer detached from it (more than rcut + skin from every
    other atom): such a group can fill one quad of one cell with nothing else in reach, an empty list,
    whose pairs (the quad's own) must still be summed."""
    core = inputs.jitter(inputs.fcc_sphere(300), 0.05, 50)
    core -= core.mean(axis=0)
    groups = [np.array([[0.0, 0.0, 0.0], [2.45, 0.0, 0.0]]),
              np.array([[0.0, 0.0, 0.0], [2.5, 0.0, 0.0], [1.25, 2.1, 0.0]]),
              np.array([[0.0, 0.0, 0.0], [2.5, 0.0, 0.0], [1.25, 2.16, 0.0], [1.25, 0.72, 2.04]])]
    spots = [np.array([23.0, 3.0, -4.0]), np.array([-4.0, -24.0, 2.0]), np.array([2.0, 5.0, 25.0])]
    pos = np.concatenate([core] + [g + s for g, s in zip(groups, spots)])
    d = np.linalg.norm(pos[:, None] - pos[None], axis=-1)
    lab = np.repeat(np.arange(4), [300, 2, 3, 4])
    assert d[lab[:, None] != lab[None]].min() > RC + 1.5  # detached beyond the list reach
    ctx = make(scmd, [len(pos)], pos, prec=prec, rcut=RC, path=VERLET)
    E, F = scmd.md_energy_forces(ctx)
    check_cluster(F, E[0], scmd.md_get_density(ctx), pos, prec, rcut=RC)
    for k in range(1, 4):  # each group's own forces, not only the sum over the cluster
        _, Fr, _, _ = oracle.energy_forces(pos[lab == k], oracle.params(rcut=RC))
        assert np.abs(F[lab == k] - Fr).max() <= 1e-4 * np.abs(Fr).max()
