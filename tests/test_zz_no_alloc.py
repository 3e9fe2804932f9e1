"""md_energy_forces_noalloc: the entry point for callers that cannot allocate device memory.

Some callers cannot let a library allocate on the GPU: a host framework whose allocator
already owns all device memory, or a time-critical loop that must not enter the CUDA
allocator. They pass their own device buffers for positions, forces and energy, and the
library keeps its working data in a fixed array compiled into it. This file is named so
that pytest runs it last; it checks the entry point against md_energy_forces (the
context-based entry point) on two calls in a row, within the mixed-precision tolerances
used by the other GPU tests (e_F <= 1e-5, |dE|/|E| <= 1e-6).
"""
import numpy as np
import pytest

from paper_1210_3559_gb300 import inputs

pytestmark = pytest.mark.gpu


def _rel(F, Fr):
    return np.linalg.norm(F - Fr) / np.linalg.norm(Fr)


def test_noalloc_matches_context_entry_point_on_two_calls():
    torch = pytest.importorskip("torch")
    from paper_1210_3559_gb300 import build, scmd
    build.build()
    stream = torch.cuda.current_stream().cuda_stream
    # two calls in a row, different clusters: the second must not see the first's data
    for n, seed in [(2000, 1), (147, 2)]:
        pos = inputs.jitter(inputs.fcc_sphere(n), 0.15, seed) + np.array([4.0, -2.0, 7.5])
        ctx = scmd.md_create(scmd.config(precision=scmd.MD_PREC_MIXED), [n], pos, None, inputs.masses(n))
        E_ref, F_ref = scmd.md_energy_forces(ctx)
        pos_t = torch.tensor(pos, dtype=torch.float64, device="cuda")
        F_t = torch.full((n, 3), float("nan"), dtype=torch.float64, device="cuda")
        E_t = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        scmd.md_energy_forces_noalloc(pos_t.data_ptr(), n, scmd.sc_params(), F_t.data_ptr(), E_t.data_ptr(), stream)
        torch.cuda.synchronize()
        F = F_t.cpu().numpy()
        E = float(E_t.cpu().numpy()[0])
        assert np.isfinite(F).all() and np.isfinite(E)
        assert _rel(F, F_ref) <= 1e-5, (n, _rel(F, F_ref))
        assert abs(E - E_ref[0]) / abs(E_ref[0]) <= 1e-6, (n, E, E_ref[0])
        scmd.md_destroy(ctx)


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
