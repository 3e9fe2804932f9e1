"""GPU parity of the structural observables (Sec. III) against the FP64 oracle: the central-atom
pair-distance histogram and the common-neighbour classes bit for bit (integers decided by FP64
distances evaluated the same way on both sides), the mean squared displacement to 1e-12.

Inputs: unevenly sized clusters in one context (a lone atom, a dimer, Ni13, a Mackay Ni147, jittered
fcc spheres, an hcp block), before and after Langevin MD, and a 50000-atom fcc sphere. The core
selection compares a distance with r_core through the centre of mass, whose rounding differs between
a tree and a sequential sum; the tests check that no atom lies within 1e-9 A of r_core."""
import numpy as np
import pytest

import oracle
from paper_1210_3559_gb300 import inputs

from test_gpu_parity import FP64, MIXED, make
from test_oracle_structure import hcp_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def scmd():
    from paper_1210_3559_gb300 import build, scmd as s
    build.build()
    return s


def batch():
    parts = [np.zeros((1, 3)), np.array([[0.0, 0.0, 0.0], [2.6, 0.1, 0.0]]), inputs.fcc_sphere(13),
             inputs.mackay_icosahedron(3, 2.49), inputs.jitter(inputs.fcc_sphere(600), 0.05, 1),
             inputs.jitter(inputs.fcc_sphere(2000), 0.1, 2), hcp_block(10, 10, 8)]
    sizes = [len(p) for p in parts]
    pos = np.concatenate([p + 80.0 * b for b, p in enumerate(parts)])
    return sizes, pos


def ranges(sizes):
    off = np.concatenate([[0], np.cumsum(sizes)])
    return [(int(off[b]), int(off[b + 1])) for b in range(len(sizes))]


def core_margin(pos, mass, r_core):
    r = np.linalg.norm(pos - oracle.com(pos, mass), axis=1)
    return np.min(np.abs(r - r_core))


def check_rdf(scmd, ctx, sizes, pos, mass, r_core, width, nbins):
    counts, nc = scmd.md_rdf(ctx, r_core, width, nbins)
    for b, (s, e) in enumerate(ranges(sizes)):
        assert core_margin(pos[s:e], mass[s:e], r_core) > 1e-9
        ref, nref = oracle.rdf(pos[s:e], mass[s:e], r_core, width, nbins)
        assert nc[b] == nref
        assert np.array_equal(counts[b], ref), b


def check_cna(scmd, ctx, sizes, pos):
    counts, cls, capped = scmd.md_cna(ctx, 3.0, per_atom=True)
    assert not capped.any()
    for b, (s, e) in enumerate(ranges(sizes)):
        ref, _ = oracle.cna(pos[s:e], 3.0)
        assert np.array_equal(cls[s:e], ref), b
        assert np.array_equal(counts[b], np.bincount(ref, minlength=4)), b
    return counts


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_rdf_and_cna_parity_batch(scmd, prec):
    sizes, pos = batch()
    mass = inputs.masses(len(pos))
    ctx = make(scmd, sizes, pos, prec=prec)
    check_rdf(scmd, ctx, sizes, pos, mass, 4.0, 0.1, 200)
    counts = check_cna(scmd, ctx, sizes, pos)
    assert counts[3][3] == 1 and counts[6][2] > 0  # the icosahedron's centre, hcp atoms
    # after Langevin MD at 1200 K: the same checks on the evolved state
    vel = np.concatenate([inputs.maxwell_boltzmann(pos[s:e], mass[s:e], 1200.0, seed=10 + b)
                          for b, (s, e) in enumerate(ranges(sizes))])
    ctx = make(scmd, sizes, pos, vel, prec=prec, graph_chunk=50)
    scmd.md_step(ctx, 200, 2.0, scmd.thermostat(scmd.MD_LANGEVIN, 1200.0, 1200.0, gamma_per_ps=1.0, seed=3))
    p, _, _ = scmd.md_get_state(ctx)
    check_rdf(scmd, ctx, sizes, p, mass, 4.0, 0.1, 200)
    check_rdf(scmd, ctx, sizes, p, mass, 6.0, 0.37, 41)  # the last bin ends at 15.17 A: a cut histogram
    check_cna(scmd, ctx, sizes, p)


def test_rdf_and_cna_full_size(scmd):
    pos = inputs.jitter(inputs.fcc_sphere(50000), 0.05, 7)
    mass = inputs.masses(50000)
    ctx = make(scmd, [50000], pos, prec=MIXED, rcut=8.8)
    check_rdf(scmd, ctx, [50000], pos, mass, 5.0, 0.05, 2000)
    counts = check_cna(scmd, ctx, [50000], pos)
    assert counts[0][1] > 40000  # a jittered fcc sphere: fcc but for the surface


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_msd_parity(scmd, prec):
    sizes, pos = batch()
    mass = inputs.masses(len(pos))
    vel = np.concatenate([inputs.maxwell_boltzmann(pos[s:e], mass[s:e], 1500.0, seed=20 + b)
                          for b, (s, e) in enumerate(ranges(sizes))])
    ctx = make(scmd, sizes, pos, vel, prec=prec, graph_chunk=50)
    th = scmd.thermostat(scmd.MD_LANGEVIN, 1500.0, 1500.0, gamma_per_ps=1.0, seed=4)
    scmd.md_step(ctx, 50, 2.0, th)
    ref, _, _ = scmd.md_get_state(ctx)
    for r_core in (0.0, 6.0):
        for b, (s, e) in enumerate(ranges(sizes)):
            if r_core > 0:
                assert core_margin(ref[s:e], mass[s:e], r_core) > 1e-9
        scmd.md_msd_reference(ctx, r_core)
        v0, _ = scmd.md_msd(ctx)
        assert np.all(v0 == 0.0)
        scmd.md_step(ctx, 100, 2.0, th)
        p, _, _ = scmd.md_get_state(ctx)
        v, n = scmd.md_msd(ctx)
        for b, (s, e) in enumerate(ranges(sizes)):
            vr, nr = oracle.msd(p[s:e], ref[s:e], mass[s:e], r_core)
            assert n[b] == nr
            assert v[b] == pytest.approx(vr, rel=1e-12, abs=1e-24), b
        ref = p


def test_structure_argument_checks(scmd):
    pos = inputs.fcc_sphere(55)
    ctx = make(scmd, [55], pos)
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_msd(ctx)
    assert e.value.status == scmd.MD_ERR_STATE
    for args in ((3.0, 0.1, 0), (3.0, 0.1, 8193), (3.0, 0.0, 10), (-1.0, 0.1, 10)):
        with pytest.raises(scmd.ScmdError) as e:
            scmd.md_rdf(ctx, *args)
        assert e.value.status == scmd.MD_ERR_INVALID
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_cna(ctx, 0.0)
    assert e.value.status == scmd.MD_ERR_INVALID
    counts, nc = scmd.md_rdf(ctx, 0.0, 0.1, 10)  # an empty core
    assert nc[0] == 0 and not counts.any()
