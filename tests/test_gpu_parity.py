"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances (forces use e_F = ||F_gpu - F_ref||_2 / ||F_ref||_2 over all atoms of a
cluster, since a per-atom relative error is undefined where |F_i| ~ 0):
  FP64 mode  : e_F <= 1e-12, |dE|/|E| <= 1e-13, rho relative <= 1e-13
  MIXED mode : e_F <= 1e-5 (the stated bound for mixed-precision forces),
               |dE|/|E| <= 1e-6, rho relative <= 2e-5.
The MIXED rho and energy bounds follow from the arithmetic: pair coordinates are
FP32 offsets from a per-cluster origin at the centre of mass, so for clusters of
radius R <= 32 A each coordinate is off by at most ulp(32)/2 = 1.9e-6 A, a pair
distance by at most 2 sqrt(3) of that, and a term r^-6 by 6 * 6.6e-6 / r with
r >= 2.0 A -> 2e-5 relative in the worst case (typical errors are 10-50x smaller);
FP32 arithmetic adds ~1e-7.
Integer work (Philox words) must be bit-exact.
"""
import os

import numpy as np
import pytest

import oracle
from paper_1210_3559_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
TOL = {0: dict(eF=1e-12, E=1e-13, rho=1e-13), 1: dict(eF=1e-5, E=1e-6, rho=2e-5)}
FP64, MIXED = 0, 1


@pytest.fixture(scope="module")
def scmd():
    from paper_1210_3559_gb300 import build, scmd as s
    build.build()
    return s


def make(scmd, sizes, pos, vel=None, prec=MIXED, rcut=0.0, **cfg):
    mass = inputs.masses(int(np.sum(sizes)))
    return scmd.md_create(scmd.config(precision=prec, **cfg), sizes, pos, vel, mass, scmd.sc_params(rcut=rcut))


def rel_force_err(F, Fr):
    n = np.linalg.norm(Fr)
    return np.linalg.norm(F - Fr) / (n if n > 0 else 1.0)


def check_cluster(F, E, rho, pos, prec, rcut=0.0, shift=False):
    p = oracle.params(rcut=rcut, shift=shift)
    Er, Fr, _, rhor = oracle.energy_forces(pos, p)
    tol = TOL[prec]
    if np.linalg.norm(Fr) > 0:
        assert rel_force_err(F, Fr) <= tol["eF"], rel_force_err(F, Fr)
    else:
        assert np.abs(F).max() <= 1e-12
    if Er != 0:
        assert abs(E - Er) / abs(Er) <= tol["E"], (E, Er)
    else:
        assert abs(E) <= 1e-12
    nz = rhor > 0
    assert np.all(np.abs(rho[nz] - rhor[nz]) <= tol["rho"] * rhor[nz])
    assert np.all(rho[~nz] == 0)


# ----------------------------------------------------------- Philox / normals
def test_philox_kernel_known_answers_and_oracle_bit_exact(scmd):
    rows = []
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        rows.append([int(x, 16) for x in line.split()])
    rows = np.array(rows, dtype=np.uint64).astype(np.uint32)
    out = scmd.md_philox4x32_10(rows[:, :6])
    assert np.array_equal(out, rows[:, 6:])
    rng = np.random.Generator(np.random.PCG64(1))
    w = rng.integers(0, 2 ** 32, size=(500, 6), dtype=np.uint64).astype(np.uint32)
    out = scmd.md_philox4x32_10(w)
    ref = np.array([oracle.philox4x32_10(r[:4], r[4:]) for r in w])
    assert np.array_equal(out, ref)


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-13), (MIXED, 2e-5)])
def test_langevin_normals_match_oracle(scmd, prec, tol):
    for (seed, cl, step) in [(0, 0, 0), (12345, 3, 77), (2 ** 40 + 5, 511, 2 ** 33 + 9)]:
        z = scmd.md_langevin_normals(seed, cl, step, 300, prec)
        zr = np.array([oracle.langevin_normals(seed, cl, step, a) for a in range(300)])
        assert np.max(np.abs(z - zr)) <= tol * max(1.0, np.abs(zr).max())


# ------------------------------------------------------- energy, forces, rho
CASES = [
    ("dimer", lambda: np.array([[0, 0, 0], [2.3, 0.4, -0.1]], float)),
    ("trimer", lambda: np.array([[0, 0, 0], [2.4, 0, 0], [1.1, 2.1, 0.3]], float)),
    ("fcc13", lambda: inputs.jitter(inputs.fcc_sphere(13), 0.1, 1)),
    ("fcc55", lambda: inputs.jitter(inputs.fcc_sphere(55), 0.1, 2)),
    ("mackay147", lambda: inputs.mackay_icosahedron(3, 2.49)),
    ("fcc97", lambda: inputs.jitter(inputs.fcc_sphere(97), 0.2, 3)),
    ("fcc301", lambda: inputs.jitter(inputs.fcc_sphere(301), 0.15, 4)),
    ("fcc1000", lambda: inputs.jitter(inputs.fcc_sphere(1000), 0.15, 5)),
]


@pytest.mark.parametrize("prec", [FP64, MIXED])
@pytest.mark.parametrize("name,gen", CASES, ids=[c[0] for c in CASES])
def test_single_cluster_energy_forces_density(scmd, prec, name, gen):
    pos = gen()
    # a random rigid motion and permutation: the GPU sees a different frame and order
    R = inputs.random_rotation(len(pos))
    pos = pos @ R.T + np.array([3.7, -1.2, 40.0])
    perm = np.random.Generator(np.random.PCG64(len(pos))).permutation(len(pos))
    pos = pos[perm]
    ctx = make(scmd, [len(pos)], pos, prec=prec)
    E, F = scmd.md_energy_forces(ctx)
    rho = scmd.md_get_density(ctx)
    check_cluster(F, E[0], rho, pos, prec)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_every_launch_shape_agrees_with_oracle(scmd, prec):
    pos = inputs.jitter(inputs.fcc_sphere(333), 0.15, 6)
    Er, Fr, _, rhor = oracle.energy_forces(pos)
    ctx = make(scmd, [333], pos, prec=prec)
    for ipt in (1, 2, 4):  # 4 i-atoms per thread: the density pass only, with >= 4 warps
        for warps in (w for w in (2, 4, 8, 16) if w >= ipt):
            for cl in (1, 2, 3, 4, 5, 6, 7, 8):
                scmd.md_set_launch(ctx, 0, ipt, warps, cl)
                scmd.md_set_launch(ctx, 1, min(ipt, 2), warps, cl)
                E, F = scmd.md_energy_forces(ctx)
                rho = scmd.md_get_density(ctx)
                assert rel_force_err(F, Fr) <= TOL[prec]["eF"], (ipt, warps, cl)
                assert abs(E[0] - Er) / abs(Er) <= TOL[prec]["E"], (ipt, warps, cl)
                assert np.all(np.abs(rho - rhor) <= TOL[prec]["rho"] * rhor)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_batched_uneven_clusters(scmd, prec):
    sizes = [1, 2, 55, 64, 65, 200, 513, 31, 33]
    parts = [inputs.jitter(inputs.fcc_sphere(n), 0.1, 10 + k) + 25.0 * k for k, n in enumerate(sizes)]
    pos = np.concatenate(parts)
    ctx = make(scmd, sizes, pos, prec=prec)
    E, F = scmd.md_energy_forces(ctx)
    rho = scmd.md_get_density(ctx)
    off = np.concatenate([[0], np.cumsum(sizes)])
    for b, n in enumerate(sizes):
        s, e = off[b], off[b + 1]
        check_cluster(F[s:e], E[b], rho[s:e], pos[s:e], prec)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_four_atoms_per_thread_density_on_uneven_batches(scmd, prec):
    """Density blocks of 128 atoms reach past a cluster's 64-atom padded segment (sizes 130, 513, the last
    cluster); those i-atoms must neither change the results nor overwrite a neighbour's observables."""
    sizes = [130, 1, 55, 513, 200, 33, 130]
    parts = [inputs.jitter(inputs.fcc_sphere(n), 0.1, 40 + k) + 25.0 * k for k, n in enumerate(sizes)]
    pos = np.concatenate(parts)
    m = inputs.masses(len(pos))
    vel = np.concatenate([inputs.maxwell_boltzmann(p, inputs.masses(len(p)), 900.0, seed=k) if len(p) > 1
                          else np.zeros((1, 3)) for k, p in enumerate(parts)])
    ctx = make(scmd, sizes, pos, vel, prec=prec, path=scmd.MD_PATH_ALLPAIRS)
    ref = make(scmd, sizes, pos, vel, prec=prec, path=scmd.MD_PATH_ALLPAIRS)
    for warps, cl in ((4, 1), (4, 3), (16, 5)):
        scmd.md_set_launch(ctx, 0, 4, warps, cl)
        E, F = scmd.md_energy_forces(ctx)
        rho = scmd.md_get_density(ctx)
        off = np.concatenate([[0], np.cumsum(sizes)])
        for b in range(len(sizes)):
            a, e = off[b], off[b + 1]
            check_cluster(F[a:e], E[b], rho[a:e], pos[a:e], prec)
        obs, obs_ref = scmd.md_observables(ctx), scmd.md_observables(ref)
        for o, r in zip(obs, obs_ref):
            assert o["epot"] == pytest.approx(r["epot"], rel=TOL[prec]["E"], abs=1e-12)
            assert o["ekin"] == r["ekin"]


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_cutoff_all_pairs_matches_oracle_cutoff(scmd, prec):
    pos = inputs.jitter(inputs.fcc_sphere(400), 0.1, 8)
    ctx = make(scmd, [400], pos, prec=prec, rcut=8.8)
    E, F = scmd.md_energy_forces(ctx)
    rho = scmd.md_get_density(ctx)
    check_cluster(F, E[0], rho, pos, prec, rcut=8.8)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_general_exponents(scmd, prec):
    # another member of the Sutton-Chen family (n=12, m=6, e.g. Ag) uses the runtime-exponent path
    pos = inputs.jitter(inputs.fcc_sphere(120, a=4.09), 0.1, 9)
    p = dict(eps=2.5415e-3, c=144.41, a=4.09, n=12, m=6)
    ctx = scmd.md_create(scmd.config(precision=prec), [120], pos, None, inputs.masses(120, 107.87),
                         scmd.sc_params(**p))
    E, F = scmd.md_energy_forces(ctx)
    Er, Fr, _, _ = oracle.energy_forces(pos, oracle.params(**p))
    assert rel_force_err(F, Fr) <= TOL[prec]["eF"]
    assert abs(E[0] - Er) / abs(Er) <= TOL[prec]["E"]


def test_bench_workload_full_size_parity(scmd):
    """Ni~2000 at the launch shapes the benchmark uses (autotuned), every atom compared."""
    pos = inputs.fcc_sphere(2000)
    vel = inputs.maxwell_boltzmann(pos, inputs.masses(2000), 2000.0, seed=2, dof="3N")
    ctx = make(scmd, [2000], inputs.jitter(pos, 0.2, 2), vel, prec=MIXED, tune=1)
    _, _, step = scmd.md_get_state(ctx)
    p_now, _, _ = scmd.md_get_state(ctx)
    E, F = scmd.md_energy_forces(ctx)
    rho = scmd.md_get_density(ctx)
    check_cluster(F, E[0], rho, p_now, MIXED)


# ---------------------------------------------------------------- dynamics
def oracle_batch(sizes, pos, vel):
    return oracle.Batch(sizes, pos, vel, inputs.masses(int(np.sum(sizes))))


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-9), (MIXED, 2e-4)])
def test_nve_trajectory_short_horizon(scmd, prec, tol):
    pos = inputs.mackay_icosahedron(3, 2.49)
    vel = inputs.maxwell_boltzmann(pos, inputs.masses(147), 1500.0, seed=1)
    ctx = make(scmd, [147], pos, vel, prec=prec, graph_chunk=32)
    scmd.md_step(ctx, 100, 1.0)
    p, v, step = scmd.md_get_state(ctx)
    assert step == 100
    ob = oracle_batch([147], pos, vel)
    ob.run(100, 1.0)
    assert np.max(np.abs(p - ob.pos)) <= tol
    assert np.max(np.abs(v - ob.vel)) <= tol * 0.1


@pytest.mark.parametrize("prec,tol", [(FP64, 1e-8), (MIXED, 5e-4)])
def test_langevin_ramp_trajectory_short_horizon(scmd, prec, tol):
    sizes = [55, 80]
    pos = np.concatenate([inputs.fcc_sphere(55), inputs.fcc_sphere(80) + 30.0])
    vel = np.concatenate([inputs.maxwell_boltzmann(pos[:55], inputs.masses(55), 1200.0, seed=3),
                          inputs.maxwell_boltzmann(pos[55:], inputs.masses(80), 1200.0, seed=4)])
    th = scmd.thermostat(scmd.MD_LANGEVIN, 1200.0, 900.0, gamma_per_ps=5.0, seed=99)
    ctx = make(scmd, sizes, pos, vel, prec=prec, graph_chunk=16)
    scmd.md_step(ctx, 40, 2.0, th)
    p, v, _ = scmd.md_get_state(ctx)
    ob = oracle_batch(sizes, pos, vel)
    ob.run(40, 2.0, oracle.thermostat(oracle.LANGEVIN, 1200.0, 900.0, gamma_ps=5.0, seed=99))
    assert np.max(np.abs(p - ob.pos)) <= tol


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_berendsen_trajectory_short_horizon(scmd, prec):
    pos = inputs.fcc_sphere(79)
    vel = inputs.maxwell_boltzmann(pos, inputs.masses(79), 600.0, seed=5)
    th = scmd.thermostat(scmd.MD_BERENDSEN, 900.0, 700.0, tau_ps=0.05)
    ctx = make(scmd, [79], pos, vel, prec=prec, graph_chunk=10)
    scmd.md_step(ctx, 30, 1.0, th)
    p, v, _ = scmd.md_get_state(ctx)
    ob = oracle_batch([79], pos, vel)
    ob.run(30, 1.0, oracle.thermostat(oracle.BERENDSEN, 900.0, 700.0, tau_ps=0.05))
    tol = 1e-9 if prec == FP64 else 2e-4
    assert np.max(np.abs(p - ob.pos)) <= tol


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_trajectory_within_oracle_sensitivity_bound(scmd, prec):
    """The GPU trajectory stays within the divergence that the dynamics itself produces from an error
    of the precision's size. The oracle is run twice, once with one coordinate moved by d0 = 1e-10 A;
    its separation d(t) gives the growth of small errors. The GPU run may then deviate from the oracle
    by at most 100 d(t) e0 / d0, with e0 = 1e-15 R for FP64 (R = the cluster radius) and 1e-6 A for
    MIXED (its FP32 pair coordinates)."""
    pos = inputs.mackay_icosahedron(3, 2.49)
    m = inputs.masses(147)
    vel = inputs.maxwell_boltzmann(pos, m, 1500.0, seed=1)
    checkpoints = [250, 500, 1000, 2000]
    a = oracle_batch([147], pos, vel)
    pert = pos.copy()
    d0 = 1e-10
    pert[17, 0] += d0
    b = oracle_batch([147], pert, vel)
    ctx = make(scmd, [147], pos, vel, prec=prec, graph_chunk=250)
    e0 = 1e-15 * np.linalg.norm(pos, axis=1).max() if prec == FP64 else 1e-6
    done = 0
    for t in checkpoints:
        a.run(t - done, 1.0)
        b.run(t - done, 1.0)
        scmd.md_step(ctx, t - done, 1.0)
        done = t
        growth = max(np.max(np.abs(b.pos - a.pos)), d0) / d0
        p, _, _ = scmd.md_get_state(ctx)
        dev = np.max(np.abs(p - a.pos))
        assert dev <= 100 * growth * e0, (t, dev, growth)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_checkpoint_resume_is_bitwise(scmd, prec):
    pos = inputs.fcc_sphere(200)
    vel = inputs.maxwell_boltzmann(pos, inputs.masses(200), 1500.0, seed=6)
    th = scmd.thermostat(scmd.MD_LANGEVIN, 1500.0, 1500.0, gamma_per_ps=1.0, seed=7)
    a = make(scmd, [200], pos, vel, prec=prec, graph_chunk=25)
    scmd.md_step(a, 100, 2.0, th)
    pa, va, sa = scmd.md_get_state(a)
    b = make(scmd, [200], pos, vel, prec=prec, graph_chunk=25)
    scmd.md_step(b, 60, 2.0, th)
    pb, vb, sb = scmd.md_get_state(b)
    c = make(scmd, [200], pos, vel, prec=prec, graph_chunk=25)
    scmd.md_set_state(c, pb, vb, sb)
    scmd.md_step(c, 40, 2.0, th)
    pc, vc, sc = scmd.md_get_state(c)
    assert sa == sc == 100
    assert np.array_equal(pa, pc) and np.array_equal(va, vc)


def test_recenter_keeps_forces(scmd):
    pos = inputs.jitter(inputs.fcc_sphere(300), 0.1, 12)
    ctx = make(scmd, [300], pos, prec=MIXED)
    _, F0 = scmd.md_energy_forces(ctx)
    far = pos + np.array([500.0, -300.0, 250.0])  # same cluster, far from the creation origin
    scmd.md_set_state(ctx, far, np.zeros_like(far), 0)
    scmd.md_recenter(ctx)
    _, F1 = scmd.md_energy_forces(ctx)
    assert rel_force_err(F1, F0) <= 1e-6


def test_observables_and_history(scmd):
    pos = inputs.mackay_icosahedron(3, 2.49)
    m = inputs.masses(147)
    vel = inputs.maxwell_boltzmann(pos, m, 1500.0, seed=1)
    ctx = make(scmd, [147], pos, vel, prec=FP64, obs_every=10, graph_chunk=50)
    o0 = scmd.md_observables(ctx)[0]
    ref = oracle.observables(pos, vel, m)
    assert o0["epot"] == pytest.approx(ref["epot"], rel=1e-13)
    assert o0["ekin"] == pytest.approx(ref["ekin"], rel=1e-13)
    assert np.allclose(o0["com"], ref["com"], atol=1e-12)
    assert np.allclose(o0["angmom"], ref["angmom"], atol=1e-9)
    scmd.md_step(ctx, 200, 1.0)
    hist = scmd.md_obs_history(ctx)
    assert [h[0]["step"] for h in hist] == list(range(10, 201, 10))
    E = np.array([h[0]["etot"] for h in hist])
    assert np.max(np.abs(E - o0["etot"])) / 147 < 1e-4  # NVE: no drift beyond 1e-4 eV/atom
    p, v, _ = scmd.md_get_state(ctx)
    last = oracle.observables(p, v, m)
    assert hist[-1][0]["epot"] == pytest.approx(last["epot"], rel=1e-12)
    assert hist[-1][0]["time_fs"] == pytest.approx(200.0)


def test_nonfinite_detected_without_trap(scmd):
    """A run that blows up is reported as MD_ERR_NONFINITE; the GPU and the context stay usable."""
    pos = inputs.fcc_sphere(13)
    ctx = make(scmd, [13], pos, prec=MIXED)
    # an absurd bath temperature gives velocities ~1e148 A/fs: FP32 coordinates overflow
    th = scmd.thermostat(scmd.MD_LANGEVIN, 1e300, 1e300, gamma_per_ps=10.0, seed=1)
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_step(ctx, 3, 1.0, th)
    assert e.value.status == scmd.MD_ERR_NONFINITE
    # two atoms 1e-4 A apart: FP32 forces overflow at evaluation time
    bad = pos.copy()
    bad[1] = bad[0] + np.array([1e-4, 0, 0])
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_set_state(ctx, bad, np.zeros((13, 3)), 0)
    assert e.value.status == scmd.MD_ERR_NONFINITE
    # restore a sane state and continue on the same context
    scmd.md_set_state(ctx, pos, np.zeros((13, 3)), 0)
    scmd.md_step(ctx, 5, 1.0)
    E, F = scmd.md_energy_forces(ctx)
    assert np.isfinite(E).all() and np.isfinite(F).all()


def test_invalid_arguments(scmd):
    ctx = make(scmd, [13], inputs.fcc_sphere(13))
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_step(ctx, 10, -1.0)
    assert e.value.status == scmd.MD_ERR_INVALID
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_step(ctx, 10, 1.0, scmd.thermostat(scmd.MD_BERENDSEN, 300.0, tau_ps=0.0001))
    assert e.value.status == scmd.MD_ERR_INVALID
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_set_launch(ctx, 0, 3, 4, 1)
    assert e.value.status == scmd.MD_ERR_INVALID
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_set_launch(ctx, 1, 4, 4, 1)  # four i-atoms per thread: the density pass only
    assert e.value.status == scmd.MD_ERR_INVALID
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_set_launch(ctx, 0, 4, 2, 1)  # ... and with at least one thread per i-atom
    assert e.value.status == scmd.MD_ERR_INVALID
    bad = inputs.fcc_sphere(13)
    bad[3, 1] = np.inf
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_set_state(ctx, bad, np.zeros((13, 3)), 0)
    assert e.value.status == scmd.MD_ERR_INVALID
