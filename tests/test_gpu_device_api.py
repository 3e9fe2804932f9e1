"""Contexts made from, and state exchanged with, caller-owned device memory (PyTorch CUDA tensors):
md_create_device, md_get_state_device, md_set_state_device, md_energy_forces_device. The results must
equal those of the host entry points bit for bit (the same values reach the same kernels) and the oracle
within the usual tolerances (e_F <= 1e-5 / 1e-12, |dE|/|E| <= 1e-6 / 1e-13 for MIXED / FP64)."""
import numpy as np
import pytest

import oracle
from paper_1210_3559_gb300 import inputs

pytestmark = pytest.mark.gpu
FP64, MIXED = 0, 1
TOL = {FP64: (1e-12, 1e-13), MIXED: (1e-5, 1e-6)}


@pytest.fixture(scope="module")
def env():
    torch = pytest.importorskip("torch")
    from paper_1210_3559_gb300 import build, scmd
    build.build()
    return torch, scmd


def _tensors(torch, pos, vel, mass):
    f = dict(dtype=torch.float64, device="cuda")
    return torch.tensor(pos, **f), None if vel is None else torch.tensor(vel, **f), torch.tensor(mass, **f)


@pytest.mark.parametrize("prec", [FP64, MIXED], ids=["fp64", "mixed"])
def test_create_device_equals_create_and_oracle(env, prec):
    torch, scmd = env
    sizes = [300, 55, 1000]
    pos = np.concatenate([inputs.jitter(inputs.fcc_sphere(n), 0.15, 20 + k) + 30.0 * k for k, n in enumerate(sizes)])
    mass = inputs.masses(len(pos))
    vel = np.concatenate([inputs.maxwell_boltzmann(pos[a:b], mass[a:b], 1200.0, seed=k)
                          for k, (a, b) in enumerate([(0, 300), (300, 355), (355, 1355)])])
    stream = torch.cuda.current_stream().cuda_stream
    cfg = scmd.config(precision=prec, graph_chunk=20, stream=stream)
    tp, tv, tm = _tensors(torch, pos, vel, mass)
    torch.cuda.synchronize()
    cd = scmd.md_create_device(cfg, sizes, tp, tv, tm)
    ch = scmd.md_create(scmd.config(precision=prec, graph_chunk=20), sizes, pos, vel, mass)
    Ed, Fd = scmd.md_energy_forces(cd)
    Eh, Fh = scmd.md_energy_forces(ch)
    assert np.array_equal(Ed, Eh) and np.array_equal(Fd, Fh)
    off = np.concatenate([[0], np.cumsum(sizes)])
    for b in range(len(sizes)):
        Er, Fr, _, _ = oracle.energy_forces(pos[off[b]:off[b + 1]])
        seg = Fd[off[b]:off[b + 1]]
        assert np.linalg.norm(seg - Fr) / np.linalg.norm(Fr) <= TOL[prec][0]
        assert abs(Ed[b] - Er) / abs(Er) <= TOL[prec][1]
    # the caller's tensors are untouched and still owned by the caller
    assert np.array_equal(tp.cpu().numpy(), pos) and np.array_equal(tm.cpu().numpy(), mass)
    th = scmd.thermostat(scmd.MD_LANGEVIN, 1200.0, 1000.0, gamma_per_ps=2.0, seed=5)
    scmd.md_step(cd, 50, 2.0, th)
    scmd.md_step(ch, 50, 2.0, th)
    pd, vd, sd = scmd.md_get_state(cd)
    ph, vh, sh = scmd.md_get_state(ch)
    assert sd == sh == 50 and np.array_equal(pd, ph) and np.array_equal(vd, vh)
    scmd.md_destroy(cd)
    scmd.md_destroy(ch)
    del tp, tv, tm


@pytest.mark.parametrize("prec", [FP64, MIXED], ids=["fp64", "mixed"])
def test_device_state_round_trip_and_resume(env, prec):
    torch, scmd = env
    pos = inputs.fcc_sphere(500)
    mass = inputs.masses(500)
    vel = inputs.maxwell_boltzmann(pos, mass, 1500.0, seed=8)
    th = scmd.thermostat(scmd.MD_LANGEVIN, 1500.0, 1500.0, gamma_per_ps=1.0, seed=9)
    a = scmd.md_create(scmd.config(precision=prec, graph_chunk=25), [500], pos, vel, mass)
    scmd.md_step(a, 100, 2.0, th)
    pa, va, _ = scmd.md_get_state(a)
    b = scmd.md_create(scmd.config(precision=prec, graph_chunk=25), [500], pos, vel, mass)
    scmd.md_step(b, 60, 2.0, th)
    tpos = torch.zeros((500, 3), dtype=torch.float64, device="cuda")
    tvel = torch.zeros((500, 3), dtype=torch.float64, device="cuda")
    step = scmd.md_get_state_device(b, tpos, tvel)
    ph, vh, sh = scmd.md_get_state(b)
    assert step == sh == 60
    assert np.array_equal(tpos.cpu().numpy(), ph) and np.array_equal(tvel.cpu().numpy(), vh)
    c = scmd.md_create(scmd.config(precision=prec, graph_chunk=25), [500], pos, vel, mass)
    scmd.md_set_state_device(c, tpos, tvel, step)
    scmd.md_step(c, 40, 2.0, th)
    pc, vc, sc = scmd.md_get_state(c)
    assert sc == 100 and np.array_equal(pc, pa) and np.array_equal(vc, va)
    # positions only: velocities untouched by a NULL destination
    only = torch.zeros((500, 3), dtype=torch.float64, device="cuda")
    scmd.md_get_state_device(c, only, None)
    assert np.array_equal(only.cpu().numpy(), pc)


def test_device_inputs_are_validated_on_the_gpu(env):
    torch, scmd = env
    pos = inputs.fcc_sphere(64)
    mass = inputs.masses(64)
    bad = pos.copy()
    bad[7, 2] = np.nan
    tp, _, tm = _tensors(torch, bad, None, mass)
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_create_device(scmd.config(), [64], tp, None, tm)
    assert e.value.status == scmd.MD_ERR_INVALID
    tp, _, tm = _tensors(torch, pos, None, np.where(np.arange(64) == 5, -1.0, mass))
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_create_device(scmd.config(), [64], tp, None, tm)
    assert e.value.status == scmd.MD_ERR_INVALID
    # a rejected md_set_state_device leaves the context as it was
    tp, _, tm = _tensors(torch, pos, None, mass)
    ctx = scmd.md_create_device(scmd.config(), [64], tp, None, tm)
    E0, F0 = scmd.md_energy_forces(ctx)
    tb = torch.tensor(bad, dtype=torch.float64, device="cuda")
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_set_state_device(ctx, tb, torch.zeros_like(tb), 3)
    assert e.value.status == scmd.MD_ERR_INVALID
    E1, F1 = scmd.md_energy_forces(ctx)
    assert np.array_equal(E0, E1) and np.array_equal(F0, F1) and scmd.md_get_state(ctx)[2] == 0


def test_create_device_on_the_cell_path(env):
    torch, scmd = env
    pos = inputs.jitter(inputs.fcc_sphere(700), 0.03, 3)
    mass = inputs.masses(700)
    prm = scmd.sc_params(rcut=8.8)
    tp, _, tm = _tensors(torch, pos, None, mass)
    cd = scmd.md_create_device(scmd.config(path=scmd.MD_PATH_CELLS), [700], tp, None, tm, prm)
    ch = scmd.md_create(scmd.config(path=scmd.MD_PATH_CELLS), [700], pos, None, mass, prm)
    assert scmd.md_get_path(cd) == scmd.MD_PATH_CELLS
    Ed, Fd = scmd.md_energy_forces(cd)
    Eh, Fh = scmd.md_energy_forces(ch)
    assert np.array_equal(Ed, Eh) and np.array_equal(Fd, Fh)


def test_fp32_peak_is_measured(env):
    _, scmd = env
    meas, derived = scmd.md_fp32_peak(5)
    assert 0.5 * derived < meas < 1.1 * derived, (meas, derived)


@pytest.mark.parametrize("prec", [FP64, MIXED], ids=["fp64", "mixed"])
def test_energy_forces_into_device_arrays(env, prec):
    torch, scmd = env
    sizes = [700, 55]
    pos = np.concatenate([inputs.jitter(inputs.fcc_sphere(700), 0.15, 31), inputs.fcc_sphere(55) + 40.0])
    ctx = scmd.md_create(scmd.config(precision=prec), sizes, pos, None, inputs.masses(755))
    E, F = scmd.md_energy_forces(ctx)
    tE = torch.full((2,), float("nan"), dtype=torch.float64, device="cuda")
    tF = torch.full((755, 3), float("nan"), dtype=torch.float64, device="cuda")
    scmd.md_energy_forces_device(ctx, tE, tF)
    assert np.array_equal(tE.cpu().numpy(), E) and np.array_equal(tF.cpu().numpy(), F)
    only = torch.zeros((2,), dtype=torch.float64, device="cuda")
    scmd.md_energy_forces_device(ctx, only, None)
    assert np.array_equal(only.cpu().numpy(), E)
