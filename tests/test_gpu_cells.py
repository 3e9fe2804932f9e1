"""GPU parity of the cell-list path (strict cutoff r < rcut) against the FP64 oracle with the same cutoff.

Inputs: fcc spheres with 0.03 A of Gaussian jitter. Their pair distances keep away from
rcut = 8.8 A (it falls between the fcc shells at 8.62 and 8.97 A; the margin is asserted), so the
cutoff decision of MIXED mode, taken in FP32 on coordinates that are off by ~1e-6 A, is the same as
the oracle's FP64 one and the comparison is element by element. Tolerances are those of the
all-pairs tests (e_F <= 1e-12 / 1e-5, E 1e-13 / 1e-6, rho 1e-13 / 2e-5 for FP64 / MIXED).
"""
import numpy as np
import pytest

import oracle
from paper_1210_3559_gb300 import inputs

from test_gpu_parity import FP64, MIXED, TOL, check_cluster, make, rel_force_err

pytestmark = pytest.mark.gpu

RC = 8.8
CELLS, ALLPAIRS, AUTO = 2, 1, 0


@pytest.fixture(scope="module")
def scmd():
    from paper_1210_3559_gb300 import build, scmd as s
    build.build()
    return s


def cutoff_margin(pos, rc=RC):
    """Smallest |r_ij - rc| over all pairs (FP64)."""
    spatial = pytest.importorskip("scipy.spatial")
    tree = spatial.cKDTree(pos)
    pairs = tree.query_pairs(rc + 0.1, output_type="ndarray")
    if len(pairs) == 0:
        return np.inf
    d = np.linalg.norm(pos[pairs[:, 0]] - pos[pairs[:, 1]], axis=1)
    return float(np.abs(d - rc).min())


def lattice(n, seed):
    pos = inputs.jitter(inputs.fcc_sphere(n), 0.03, seed)
    assert cutoff_margin(pos) > 0.02
    return pos


# ------------------------------------------------------------ static parity
@pytest.mark.parametrize("prec", [FP64, MIXED])
@pytest.mark.parametrize("n", [700, 6000])
def test_cells_energy_forces_density(scmd, prec, n):
    pos = lattice(n, 21)
    ctx = make(scmd, [n], pos, prec=prec, rcut=RC, path=CELLS)
    E, F = scmd.md_energy_forces(ctx)
    check_cluster(F, E[0], scmd.md_get_density(ctx), pos, prec, rcut=RC)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_cells_agree_with_all_pairs_cutoff(scmd, prec):
    pos = lattice(3000, 22)
    a = make(scmd, [3000], pos, prec=prec, rcut=RC, path=CELLS)
    b = make(scmd, [3000], pos, prec=prec, rcut=RC, path=ALLPAIRS)
    Ea, Fa = scmd.md_energy_forces(a)
    Eb, Fb = scmd.md_energy_forces(b)
    assert rel_force_err(Fa, Fb) <= TOL[prec]["eF"]
    assert abs(Ea[0] - Eb[0]) <= TOL[prec]["E"] * abs(Eb[0])
    ra, rb = scmd.md_get_density(a), scmd.md_get_density(b)
    assert np.all(np.abs(ra - rb) <= TOL[prec]["rho"] * rb)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_cells_far_atoms_tiny_clusters_batch(scmd, prec):
    """Atoms far outside a cluster's grid are clamped into its border cells: a lone atom, and a
    dimer 300 A out whose two atoms interact, keep exact forces; clusters of 1, 2 and 13 atoms.
    In MIXED the dimer's offsets from its (border) cell centre are ~260 A, where FP32 carries
    ~1.5e-5 A of rounding, so its forces are checked to 1e-3 relative; every other atom is compared
    element by element at the usual tolerances."""
    big = lattice(400, 23)
    big[5] = big[5] + np.array([60.0, 0.0, 0.0])
    big[6] = np.array([300.0, 10.0, -5.0])
    big[7] = np.array([303.1, 10.0, -5.0])
    parts = [np.zeros((1, 3)), np.array([[0.0, 0.0, 0.0], [2.6, 0.1, 0.0]]), inputs.fcc_sphere(13), big]
    sizes = [len(p) for p in parts]
    pos = np.concatenate([p + 40.0 * b for b, p in enumerate(parts)])
    ctx = make(scmd, sizes, pos, prec=prec, rcut=RC, path=CELLS)
    E, F = scmd.md_energy_forces(ctx)
    rho = scmd.md_get_density(ctx)
    off = np.concatenate([[0], np.cumsum(sizes)])
    for b in range(3):
        s, e = off[b], off[b + 1]
        check_cluster(F[s:e], E[b], rho[s:e], pos[s:e], prec, rcut=RC)
    s, e = off[3], off[4]
    Er, Fr, _, rr = oracle.energy_forces(pos[s:e], oracle.params(rcut=RC))
    assert np.abs(F[s + 7]).max() > 0.1  # the far dimer does interact
    assert np.all(F[s + 5] == 0) and rho[s + 5] == 0  # the lone far atom does not
    if prec == FP64:
        check_cluster(F[s:e], E[3], rho[s:e], pos[s:e], prec, rcut=RC)
    else:
        core = np.ones(e - s, bool)
        core[[6, 7]] = False
        assert rel_force_err(F[s:e][core], Fr[core]) <= TOL[MIXED]["eF"]
        assert np.all(np.abs(rho[s:e][core] - rr[core]) <= TOL[MIXED]["rho"] * np.maximum(rr[core], 1e-300))
        assert rel_force_err(F[s + 6:s + 8], Fr[6:8]) <= 1e-3
        assert np.all(np.abs(rho[s + 6:s + 8] - rr[6:8]) <= 1e-3 * rr[6:8])
        assert abs(E[3] - Er) <= TOL[MIXED]["E"] * abs(Er)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_cells_full_size_parity(scmd, prec):
    """Ni~50000 with rcut = 8.8 A on the cell list (the automatic choice at this size is the
    neighbour lists, tested with them): every atom against the oracle."""
    pos = lattice(50000, 24)
    vel = inputs.maxwell_boltzmann(pos, inputs.masses(50000), 300.0, seed=3)
    ctx = make(scmd, [50000], pos, vel, prec=prec, rcut=RC, path=AUTO)
    assert scmd.md_get_path(ctx) == 3
    # cell build (MIXED 1: binning, FP64 3), list build (MIXED 3, FP64 4), passes (MIXED 2, FP64 compaction + 2 + 2 gathers),
    # and in FP64 the position kernel (MIXED: once per chunk)
    assert scmd.md_launch_counts(ctx)[0] == (6 if prec == MIXED else 13)
    ctx = make(scmd, [50000], pos, vel, prec=prec, rcut=RC, path=CELLS)
    assert scmd.md_get_path(ctx) == CELLS
    assert scmd.md_launch_counts(ctx)[0] == 5  # clear, bin, sort, density, force
    E, F = scmd.md_energy_forces(ctx)
    check_cluster(F, E[0], scmd.md_get_density(ctx), pos, prec, rcut=RC)
    ms_d, ms_f, pairs = scmd.md_time_passes(ctx, 5)
    assert ms_d > 0 and ms_f > 0
    # pairs tested: more than the ~224 neighbours inside rcut per atom, far fewer than all pairs
    assert 224 * 50000 < pairs < 0.05 * 50000 * 49999


def test_cells_mixed_thermal_disorder_full_size(scmd):
    """Ni~50000 with 0.1 A of disorder (force magnitudes of a crystal at a few hundred K), MIXED.
    Some pair distances now lie within the FP32 rounding of rcut, where FP32 and FP64 may decide the
    cutoff differently; both decisions are valid. A flipped pair moves rho_i and rho_j by at most
    (a / rcut)^m and the forces and energy by far less than their tolerances, so: e_F and E are
    compared as usual, rho element by element on every atom that is not the end of such a pair, and
    on those ends within the tolerance plus their count of ambiguous pairs times (a / rcut)^m."""
    spatial = pytest.importorskip("scipy.spatial")
    pos = inputs.jitter(inputs.fcc_sphere(50000), 0.1, 25)
    ctx = make(scmd, [50000], pos, prec=MIXED, rcut=RC, path=CELLS)
    E, F = scmd.md_energy_forces(ctx)
    rho = scmd.md_get_density(ctx)
    Er, Fr, _, rhor = oracle.energy_forces(pos, oracle.params(rcut=RC))
    assert rel_force_err(F, Fr) <= TOL[MIXED]["eF"]
    assert abs(E[0] - Er) <= TOL[MIXED]["E"] * abs(Er)
    pairs = spatial.cKDTree(pos).query_pairs(RC + 1e-3, output_type="ndarray")
    r = np.linalg.norm(pos[pairs[:, 0]] - pos[pairs[:, 1]], axis=1)
    amb = pairs[np.abs(r - RC) < 1e-4]
    n_amb = np.bincount(amb.ravel(), minlength=len(pos))
    bound = TOL[MIXED]["rho"] * rhor + n_amb * 1.01 * (3.52 / (RC - 1e-4)) ** 6
    assert np.all(np.abs(rho - rhor) <= bound)
    clean = n_amb == 0
    assert clean.sum() > 0.95 * len(pos)
    assert np.all(np.abs(rho[clean] - rhor[clean]) <= TOL[MIXED]["rho"] * rhor[clean])


# ----------------------------------------------------------------- dynamics
@pytest.mark.parametrize("prec,tol", [(FP64, 1e-8), (MIXED, 5e-4)])
def test_cells_langevin_ramp_trajectory(scmd, prec, tol):
    sizes = [147, 300]
    pos = np.concatenate([inputs.mackay_icosahedron(3, 2.49), inputs.fcc_sphere(300) + 50.0])
    m = inputs.masses(447)
    vel = np.concatenate([inputs.maxwell_boltzmann(pos[:147], m[:147], 1400.0, seed=3),
                          inputs.maxwell_boltzmann(pos[147:], m[147:], 1400.0, seed=4)])
    th = scmd.thermostat(scmd.MD_LANGEVIN, 1400.0, 1000.0, gamma_per_ps=5.0, seed=17)
    ctx = make(scmd, sizes, pos, vel, prec=prec, rcut=RC, path=CELLS, graph_chunk=16)
    scmd.md_step(ctx, 40, 2.0, th)
    p, _, _ = scmd.md_get_state(ctx)
    ob = oracle.Batch(sizes, pos, vel, m, oracle.params(rcut=RC))
    ob.run(40, 2.0, oracle.thermostat(oracle.LANGEVIN, 1400.0, 1000.0, gamma_ps=5.0, seed=17))
    assert np.max(np.abs(p - ob.pos)) <= tol


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-8), (MIXED, 5e-4)])
def test_cells_nve_trajectory(scmd, prec, tol):
    pos = inputs.fcc_sphere(500)
    m = inputs.masses(500)
    vel = inputs.maxwell_boltzmann(pos, m, 1500.0, seed=8)
    ctx = make(scmd, [500], pos, vel, prec=prec, rcut=RC, path=CELLS, graph_chunk=32)
    scmd.md_step(ctx, 100, 1.0)
    p, v, _ = scmd.md_get_state(ctx)
    ob = oracle.Batch([500], pos, vel, m, oracle.params(rcut=RC))
    ob.run(100, 1.0)
    assert np.max(np.abs(p - ob.pos)) <= tol
    assert np.max(np.abs(v - ob.vel)) <= tol * 0.1


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_cells_berendsen_trajectory_and_observables(scmd, prec):
    pos = inputs.fcc_sphere(300)
    m = inputs.masses(300)
    vel = inputs.maxwell_boltzmann(pos, m, 600.0, seed=5)
    th = scmd.thermostat(scmd.MD_BERENDSEN, 900.0, 700.0, tau_ps=0.05)
    ctx = make(scmd, [300], pos, vel, prec=prec, rcut=RC, path=CELLS, graph_chunk=10, obs_every=5)
    scmd.md_step(ctx, 30, 1.0, th)
    p, v, _ = scmd.md_get_state(ctx)
    ob = oracle.Batch([300], pos, vel, m, oracle.params(rcut=RC))
    ob.run(30, 1.0, oracle.thermostat(oracle.BERENDSEN, 900.0, 700.0, tau_ps=0.05))
    assert np.max(np.abs(p - ob.pos)) <= (1e-9 if prec == FP64 else 2e-4)
    hist = scmd.md_obs_history(ctx)
    assert [h[0]["step"] for h in hist] == [5, 10, 15, 20, 25, 30]
    ref = oracle.observables(p, v, m, oracle.params(rcut=RC))
    rel = 1e-12 if prec == FP64 else 1e-6
    assert hist[-1][0]["epot"] == pytest.approx(ref["epot"], rel=rel)
    assert hist[-1][0]["ekin"] == pytest.approx(ref["ekin"], rel=1e-12)
    assert np.allclose(hist[-1][0]["angmom"], ref["angmom"], rtol=1e-9, atol=1e-9)


def test_cells_observables_history_langevin(scmd):
    pos = inputs.fcc_sphere(400)
    m = inputs.masses(400)
    vel = inputs.maxwell_boltzmann(pos, m, 1200.0, seed=9)
    ctx = make(scmd, [400], pos, vel, prec=FP64, rcut=RC, path=CELLS, graph_chunk=16, obs_every=8)
    o0 = scmd.md_observables(ctx)[0]
    ref0 = oracle.observables(pos, vel, m, oracle.params(rcut=RC))
    assert o0["epot"] == pytest.approx(ref0["epot"], rel=1e-13)
    assert o0["ekin"] == pytest.approx(ref0["ekin"], rel=1e-13)
    th = scmd.thermostat(scmd.MD_LANGEVIN, 1200.0, 1200.0, gamma_per_ps=2.0, seed=4)
    scmd.md_step(ctx, 48, 1.0, th)
    hist = scmd.md_obs_history(ctx)
    assert [h[0]["step"] for h in hist] == list(range(8, 49, 8))
    p, v, _ = scmd.md_get_state(ctx)
    ref = oracle.observables(p, v, m, oracle.params(rcut=RC))
    for key in ("epot", "ekin", "etot", "T"):
        assert hist[-1][0][key] == pytest.approx(ref[key], rel=1e-12)
    assert np.allclose(hist[-1][0]["com"], ref["com"], atol=1e-10)
    assert np.allclose(hist[-1][0]["mom"], ref["mom"], atol=1e-12)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_cells_checkpoint_resume_is_bitwise(scmd, prec):
    pos = inputs.fcc_sphere(600)
    vel = inputs.maxwell_boltzmann(pos, inputs.masses(600), 1500.0, seed=6)
    th = scmd.thermostat(scmd.MD_LANGEVIN, 1500.0, 1500.0, gamma_per_ps=1.0, seed=7)
    kw = dict(prec=prec, rcut=RC, path=CELLS, graph_chunk=25)
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
    assert np.array_equal(pa, pc) and np.array_equal(va, vc)


def test_cells_runs_are_deterministic(scmd):
    """Cell slots are taken with atomics; the per-cell sort makes every sum order, and so the
    trajectory, identical from run to run."""
    pos = inputs.fcc_sphere(2000)
    vel = inputs.maxwell_boltzmann(pos, inputs.masses(2000), 2500.0, seed=10)
    th = scmd.thermostat(scmd.MD_LANGEVIN, 2500.0, 2500.0, gamma_per_ps=1.0, seed=3)
    out = []
    for _ in range(2):
        ctx = make(scmd, [2000], pos, vel, prec=MIXED, rcut=RC, path=CELLS, graph_chunk=50)
        scmd.md_step(ctx, 100, 2.0, th)
        out.append(scmd.md_get_state(ctx)[0])
    assert np.array_equal(out[0], out[1])


# ------------------------------------------------------------------- errors
def test_cells_overflow_is_reported(scmd):
    """600 atoms 20 A apart on a line far outside the grid: more than 256 of them clamp into one
    border cell. The overflow is detected on the device and reported; nothing is written out of
    bounds (a full cell drops the extra slots)."""
    core = inputs.fcc_sphere(400)
    line = np.stack([1000.0 + 20.0 * np.arange(600), np.zeros(600), np.zeros(600)], axis=1)
    pos = np.concatenate([core, line])
    with pytest.raises(scmd.ScmdError) as e:
        make(scmd, [1000], pos, prec=MIXED, rcut=RC, path=CELLS)
    assert e.value.status == scmd.MD_ERR_STATE
    # the GPU stays usable
    ctx = make(scmd, [400], core, prec=MIXED, rcut=RC, path=CELLS)
    E, F = scmd.md_energy_forces(ctx)
    assert np.isfinite(E).all() and np.isfinite(F).all()


def test_cells_invalid_configurations(scmd):
    pos = inputs.fcc_sphere(55)
    with pytest.raises(scmd.ScmdError) as e:
        make(scmd, [55], pos, rcut=0.0, path=CELLS)
    assert e.value.status == scmd.MD_ERR_INVALID
    big = inputs.fcc_sphere(2000)
    with pytest.raises(scmd.ScmdError) as e:  # cells of side >= 20 A would hold > 256 of its atoms
        make(scmd, [2000], big, rcut=20.0, path=CELLS)
    assert e.value.status == scmd.MD_ERR_INVALID
    tiny = make(scmd, [55], pos, rcut=20.0, path=CELLS)  # a cluster of fewer atoms than a cell holds
    assert scmd.md_get_path(tiny) == CELLS
    ctx = make(scmd, [55], pos, rcut=20.0, path=ALLPAIRS)  # the all-pairs path takes any cutoff
    assert scmd.md_get_path(ctx) == ALLPAIRS and scmd.md_launch_counts(ctx)[0] == 2
    small = make(scmd, [55], pos, rcut=8.8)  # automatic choice: a small cluster keeps all pairs
    assert scmd.md_get_path(small) == ALLPAIRS
