"""CPU-side checks of the C-ABI library: it builds, loads and exports every declared entry point."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "scmd.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(md_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1210_3559_gb300 import build, scmd
    build.build()
    return scmd.lib()


def test_header_declares_the_boundary_calls():
    names = declared_functions()
    for required in ["md_create", "md_energy_forces", "md_step", "md_observables", "md_get_state",
                     "md_set_state", "md_last_error", "md_destroy"]:
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1210_3559_gb300 import scmd
    assert sorted(scmd.exported_symbols()) == declared_functions()
    for name in declared_functions():
        assert callable(getattr(scmd, name)), name


def test_abi_version_and_argument_errors_without_gpu(lib):
    from paper_1210_3559_gb300 import scmd
    assert lib.md_abi_version() == 2
    # invalid arguments are rejected before any device call
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_create(scmd.config(), [0], [[0.0, 0.0, 0.0]] * 0, None, [])
    assert e.value.status == scmd.MD_ERR_INVALID
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_create(scmd.config(), [1], [[float("nan"), 0.0, 0.0]], None, [58.6934])
    assert e.value.status == scmd.MD_ERR_INVALID
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_create(scmd.config(), [1], [[0.0, 0.0, 0.0]], None, [-1.0])
    assert e.value.status == scmd.MD_ERR_INVALID
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_create(scmd.config(precision=7), [1], [[0.0, 0.0, 0.0]], None, [1.0])
    assert e.value.status == scmd.MD_ERR_INVALID


def test_no_gpu_fails_loudly(lib):
    """Without a GPU the library reports MD_ERR_CUDA; it never falls back to the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1210_3559_gb300 import scmd
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_create(scmd.config(), [2], [[0.0, 0.0, 0.0], [2.5, 0.0, 0.0]], None, [58.6934, 58.6934])
    assert e.value.status == scmd.MD_ERR_CUDA


def test_degenerate_and_invalid_configurations_without_gpu(lib):
    """Rejected before any device call: no cluster at all, an unknown precision or path, the cell path
    without a cutoff, a negative cutoff."""
    import numpy as np
    from paper_1210_3559_gb300 import scmd
    one = np.zeros((1, 3))
    cases = [
        (scmd.config(), [], np.zeros((0, 3)), [], scmd.sc_params()),
        (scmd.config(precision=7), [1], one, [58.6934], scmd.sc_params()),
        (scmd.config(path=9), [1], one, [58.6934], scmd.sc_params()),
        (scmd.config(path=scmd.MD_PATH_CELLS), [1], one, [58.6934], scmd.sc_params(rcut=0.0)),
        (scmd.config(), [1], one, [58.6934], scmd.sc_params(rcut=-1.0)),
        (scmd.config(precision=scmd.MD_PREC_MIXED, path=scmd.MD_PATH_ALLPAIRS_HALF), [1], one, [58.6934],
         scmd.sc_params()),
    ]
    for cfg, sizes, pos, mass, prm in cases:
        with pytest.raises(scmd.ScmdError) as e:
            scmd.md_create(cfg, sizes, pos, None, mass, prm)
        assert e.value.status == scmd.MD_ERR_INVALID, (sizes, cfg.precision, cfg.path)
        assert scmd.md_last_error() != ""


def test_device_entry_points_reject_bad_arguments_without_gpu(lib):
    """md_create_device and md_fp32_peak check their arguments before any device call."""
    from paper_1210_3559_gb300 import scmd
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_create_device(scmd.config(), [4], None, None, None)
    assert e.value.status == scmd.MD_ERR_INVALID
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_create_device(scmd.config(), [0], 1, None, 1)
    assert e.value.status == scmd.MD_ERR_INVALID
    with pytest.raises(scmd.ScmdError) as e:
        scmd.md_fp32_peak(0)
    assert e.value.status == scmd.MD_ERR_INVALID
