"""md_energy_forces_noalloc: the entry point for callers that cannot allocate device memory.

Some callers cannot let a library allocate on the GPU: a host framework whose allocator
already owns all device memory, or a time-critical loop that must not enter the CUDA
allocator. They pass their own device buffers for positions, forces and energy, and the
library keeps its working data in a fixed array compiled into it. This file is named so
that pytest runs it last. It checks the entry point on two calls in a row against
md_energy_forces (the context-based entry point) and against the FP64 oracle, within the
mixed-precision tolerances used by the other GPU tests (e_F <= 1e-5, |dE|/|E| <= 1e-6),
with all pairs and with the strict cutoff.
"""
import numpy as np
import pytest

import oracle
from paper_1210_3559_gb300 import inputs

pytestmark = pytest.mark.gpu

RCUT = 8.8


def _rel(F, Fr):
    return np.linalg.norm(F - Fr) / np.linalg.norm(Fr)


def _noalloc(scmd, torch, pos, params):
    n = len(pos)
    stream = torch.cuda.current_stream().cuda_stream
    pos_t = torch.tensor(pos, dtype=torch.float64, device="cuda")
    F_t = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
    E_t = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    scmd.md_energy_forces_noalloc(pos_t.data_ptr(), n, params, F_t.data_ptr(), E_t.data_ptr(), stream)
    torch.cuda.synchronize()
    return float(E_t.cpu().numpy()[0]), F_t.cpu().numpy()


def _check(scmd, torch, pos, rcut):
    n = len(pos)
    params = scmd.sc_params(rcut=rcut)
    E, F = _noalloc(scmd, torch, pos, params)
    assert np.isfinite(F).all() and np.isfinite(E)
    # the context-based entry point (all-pairs path, same cutoff)
    ctx = scmd.md_create(scmd.config(precision=scmd.MD_PREC_MIXED, path=scmd.MD_PATH_ALLPAIRS), [n], pos, None,
                         inputs.masses(n), params)
    E_ref, F_ref = scmd.md_energy_forces(ctx)
    scmd.md_destroy(ctx)
    assert _rel(F, F_ref) <= 1e-5, (n, rcut, _rel(F, F_ref))
    assert abs(E - E_ref[0]) / abs(E_ref[0]) <= 1e-6, (n, rcut, E, E_ref[0])
    # the FP64 oracle with the same cutoff
    Eo, Fo, _, _ = oracle.energy_forces(pos, oracle.params(rcut=rcut))
    assert _rel(F, Fo) <= 1e-5, (n, rcut, _rel(F, Fo))
    assert abs(E - Eo) / abs(Eo) <= 1e-6, (n, rcut, E, Eo)


def test_noalloc_matches_context_entry_point_and_oracle_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_1210_3559_gb300 import build, scmd
    build.build()
    # two calls in a row, different clusters: the second must not see the first's data
    for n, seed in [(2000, 1), (147, 2)]:
        pos = inputs.jitter(inputs.fcc_sphere(n), 0.15, seed) + np.array([4.0, -2.0, 7.5])
        _check(scmd, torch, pos, 0.0)


def test_noalloc_strict_cutoff_matches_context_entry_point_and_oracle():
    """rcut = 8.8 A on a 2000-atom sphere with 0.03 A of disorder: 8.8 A lies between the fcc shells at
    8.62 and 8.97 A, and no pair distance is within 0.02 A of it, so the FP32 cutoff decisions equal the
    oracle's FP64 ones. Two calls in a row (cutoff, then all pairs on another cluster)."""
    torch = pytest.importorskip("torch")
    from paper_1210_3559_gb300 import build, scmd
    build.build()
    pos = inputs.jitter(inputs.fcc_sphere(2000), 0.03, 11) + np.array([-3.0, 1.5, 2.0])
    d = np.sqrt(((pos[:, None, :] - pos[None, :, :]) ** 2).sum(-1))
    assert np.min(np.abs(d - RCUT)) > 0.02
    assert ((d > 0) & (d >= RCUT)).any() and ((d > 0) & (d < RCUT)).any()  # the cutoff removes pairs
    _check(scmd, torch, pos, RCUT)
    _check(scmd, torch, inputs.jitter(inputs.fcc_sphere(600), 0.15, 12), 0.0)


def test_noalloc_rejects_sizes_beyond_its_fixed_scratch():
    torch = pytest.importorskip("torch")
    from paper_1210_3559_gb300 import build, scmd
    build.build()
    pos_t = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros((4, 3), dtype=torch.float64, device="cuda")
    e = torch.zeros((1,), dtype=torch.float64, device="cuda")
    with pytest.raises(scmd.ScmdError) as err:
        scmd.md_energy_forces_noalloc(pos_t.data_ptr(), 16385, scmd.sc_params(), out.data_ptr(), e.data_ptr(), 0)
    assert err.value.status == scmd.MD_ERR_INVALID
    assert "16384" in str(err.value)
