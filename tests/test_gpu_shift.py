"""GPU parity of the shifted cutoff form (every pair term inside rcut less its value at rcut) on the
cell-list and neighbour-list paths against the oracle's shifted form, the paths that reject it, and
the energy conservation it buys: in NVE, the truncated energy jumps whenever a pair crosses rcut and
the shifted one does not, so over the same run its energy wanders far less.

Inputs as for the cutoff paths: fcc spheres with 0.03 A of disorder (pair distances at least 0.02 A
from rcut = 8.8 A), tolerances as for the other paths."""
import numpy as np
import pytest

from paper_1210_3559_gb300 import inputs

from test_gpu_parity import FP64, MIXED, check_cluster, make
from test_gpu_cells import RC, lattice

pytestmark = pytest.mark.gpu

AUTO, ALLPAIRS, CELLS, VERLET = 0, 1, 2, 3


@pytest.fixture(scope="module")
def scmd():
    from paper_1210_3559_gb300 import build, scmd as s
    build.build()
    return s


def make_shift(scmd, sizes, pos, vel=None, prec=MIXED, path=AUTO, **cfg):
    mass = inputs.masses(int(np.sum(sizes)))
    return scmd.md_create(scmd.config(precision=prec, path=path, **cfg), sizes, pos, vel, mass,
                          scmd.sc_params(rcut=RC, shift=True))


@pytest.mark.parametrize("path", [CELLS, VERLET])
@pytest.mark.parametrize("prec", [FP64, MIXED])
@pytest.mark.parametrize("n", [700, 6000])
def test_shifted_energy_forces_density(scmd, path, prec, n):
    pos = lattice(n, 41)
    ctx = make_shift(scmd, [n], pos, prec=prec, path=path)
    assert scmd.md_get_path(ctx) == path
    E, F = scmd.md_energy_forces(ctx)
    check_cluster(F, E[0], scmd.md_get_density(ctx), pos, prec, rcut=RC, shift=True)


@pytest.mark.parametrize("prec", [FP64, MIXED])
def test_shifted_batch_and_automatic_path(scmd, prec):
    """Unevenly sized clusters (a lone atom, a dimer beyond and one inside rcut, Ni13, Ni300) on the
    automatic path, which takes the neighbour lists for any size when the cutoff is shifted."""
    parts = [np.zeros((1, 3)), np.array([[0.0, 0.0, 0.0], [9.0, 0.0, 0.0]]),
             np.array([[0.0, 0.0, 0.0], [8.0, 0.5, 0.0]]), inputs.fcc_sphere(13), lattice(300, 42)]
    sizes = [len(p) for p in parts]
    pos = np.concatenate([p + 60.0 * b for b, p in enumerate(parts)])
    ctx = make_shift(scmd, sizes, pos, prec=prec)
    assert scmd.md_get_path(ctx) == VERLET
    E, F = scmd.md_energy_forces(ctx)
    rho = scmd.md_get_density(ctx)
    off = np.concatenate([[0], np.cumsum(sizes)])
    for b in range(len(sizes)):
        s, e = off[b], off[b + 1]
        check_cluster(F[s:e], E[b], rho[s:e], pos[s:e], prec, rcut=RC, shift=True)


def test_shifted_cutoff_rejected_where_not_supported(scmd):
    pos = inputs.fcc_sphere(55)
    m = inputs.masses(55)
    for params, path in ((scmd.sc_params(rcut=RC, shift=True), ALLPAIRS),
                         (scmd.sc_params(rcut=0.0, shift=True), AUTO)):
        with pytest.raises(scmd.ScmdError) as e:
            scmd.md_create(scmd.config(path=path), [55], pos, None, m, params)
        assert e.value.status == scmd.MD_ERR_INVALID


@pytest.mark.parametrize("path", [CELLS, VERLET])
def test_shifted_cutoff_conserves_energy_better_in_nve(scmd, path):
    """Ni~2000 melted at 2000 K, then 4000 NVE steps of 2 fs in FP64 with each cutoff form. The
    spread of E_tot about its linear trend is set by the truncation jumps in the plain form."""
    pos = inputs.fcc_sphere(2000)
    m = inputs.masses(2000)
    vel = inputs.maxwell_boltzmann(pos, m, 2000.0, seed=8)
    spread = {}
    for shift in (False, True):
        ctx = scmd.md_create(scmd.config(precision=FP64, path=path, obs_every=20, obs_capacity=400,
                                         graph_chunk=200), [2000], pos, vel, m,
                             scmd.sc_params(rcut=RC, shift=shift))
        scmd.md_step(ctx, 2000, 2.0, scmd.thermostat(scmd.MD_LANGEVIN, 2000.0, 2000.0, gamma_per_ps=5.0, seed=2))
        scmd.md_clear_history(ctx)
        scmd.md_step(ctx, 4000, 2.0)
        e = np.array([h[0]["etot"] for h in scmd.md_obs_history(ctx)])
        t = np.arange(len(e))
        resid = e - np.polyval(np.polyfit(t, e, 1), t)
        spread[shift] = float(np.std(resid))
    assert spread[True] < 0.5 * spread[False], spread
