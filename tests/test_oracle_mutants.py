"""The oracle's pins catch plausible mistakes in it.

Each mutant below is the oracle's C source with one plausible slip planted in it: a dropped
factor, a flipped sign, a wrong exponent, a transposed operand, a one-sided embedding term. The
mutant is compiled on its own (CPU only) and run against pins that come from outside the
oracle: the closed-form dimer of Eq. 1 and Eq. 2, central finite differences of its own energy,
and the vanishing net force and torque of pairwise central forces. Every mutant must fail at
least one pin, and the unmodified source must pass all of them, so a mistake of these kinds
cannot hide in the oracle the CUDA path is checked against.
"""
import ctypes
import os
import shutil
import subprocess

import numpy as np
import pytest

import oracle
from paper_1210_3559_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "sc_oracle.c")
EPS, C, A, NN, MM = 1.5707e-2, 39.432, 3.52, 9, 6

# (name, text in sc_oracle.c, replacement); each text occurs exactly once in the source
MUTANTS = [
    ("pair energy without the factor 1/2",
     "e_pair += 0.5 * p->eps * pair_i[i];", "e_pair += p->eps * pair_i[i];"),
    ("embedding energy with the wrong sign",
     "e_emb += -p->eps * p->c * sqrt(rho[i]);", "e_emb += p->eps * p->c * sqrt(rho[i]);"),
    ("embedding energy linear in rho",
     "e_emb += -p->eps * p->c * sqrt(rho[i]);", "e_emb += -p->eps * p->c * rho[i];"),
    ("density summed with the repulsive exponent",
     "acc += term(r, p->m, p);", "acc += term(r, p->n, p);"),
    ("force with g_i counted twice instead of g_i + g_j",
     "kemb * (g[i] + g[j])", "kemb * (2.0 * g[i])"),
    ("force embedding prefactor without m/2",
     "const double kemb = 0.5 * p->c * (double)p->m;", "const double kemb = p->c;"),
    ("force divided by r instead of r^2",
     "kemb * (g[i] + g[j]) * pow(s, p->m)) / (r * r);", "kemb * (g[i] + g[j]) * pow(s, p->m)) / r;"),
    ("x displacement transposed (r_j - r_i)",
     "d[0] = pos[3 * i + 0] - pos[3 * j + 0];", "d[0] = pos[3 * j + 0] - pos[3 * i + 0];"),
    ("repulsive force term without the exponent n",
     "((double)p->n * pow(s, p->n) -", "(pow(s, p->n) -"),
]


def _compile(src_text, out_dir, name):
    src = os.path.join(out_dir, name + ".c")
    lib = os.path.join(out_dir, name + ".so")
    with open(src, "w") as f:
        f.write(src_text)
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", src, "-o", lib, "-lm"],
                   check=True)
    L = ctypes.CDLL(lib)
    dp = ctypes.POINTER(ctypes.c_double)
    L.orc_energy_forces.argtypes = [ctypes.c_int, dp, ctypes.POINTER(oracle.Params), dp, dp, dp]
    L.orc_energy_forces.restype = ctypes.c_double
    return L


def _energy_forces(L, pos):
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    F = np.zeros_like(pos)
    p = oracle.params()
    dp = ctypes.POINTER(ctypes.c_double)
    U = L.orc_energy_forces(len(pos), pos.ctypes.data_as(dp), ctypes.byref(p), F.ctypes.data_as(dp), None, None)
    return U, F


def pin_dimer(L):
    """U(r) = eps [s^n - 2 c s^(m/2)], F = -dU/dr along the axis (two atoms: rho = s^m each)."""
    for r in (2.041345, 2.49, 3.1):
        s = A / r
        U_ref = EPS * (s ** NN - 2.0 * C * s ** (MM / 2))
        dUdr = EPS * (-NN * s ** NN + C * MM * s ** (MM / 2)) / r
        U, F = _energy_forces(L, [[0, 0, 0], [r, 0, 0]])
        if not (abs(U - U_ref) <= 1e-12 * abs(U_ref) and abs(F[0, 0] - dUdr) <= 1e-10 * max(abs(dUdr), 1e-3)):
            return False
    return True


def pin_finite_differences(L, h=1e-5):
    pos = inputs.jitter(inputs.fcc_sphere(13), 0.15, 2)
    _, F = _energy_forces(L, pos)
    Fn = np.zeros_like(pos)
    for i in range(len(pos)):
        for c in range(3):
            xp = pos.copy(); xp[i, c] += h
            xm = pos.copy(); xm[i, c] -= h
            Fn[i, c] = -(_energy_forces(L, xp)[0] - _energy_forces(L, xm)[0]) / (2 * h)
    return np.linalg.norm(F - Fn) / np.linalg.norm(Fn) < 1e-8


def pin_net_force_and_torque(L):
    pos = inputs.jitter(inputs.fcc_sphere(38), 0.15, 3)
    _, F = _energy_forces(L, pos)
    scale = np.abs(F).sum()
    return (np.abs(F.sum(0)).max() < 1e-12 * scale and
            np.abs(np.cross(pos, F).sum(0)).max() < 1e-12 * scale * np.abs(pos).max())


PINS = [pin_dimer, pin_finite_differences, pin_net_force_and_torque]


@pytest.fixture(scope="module")
def source():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    with open(SRC) as f:
        return f.read()


def test_unmodified_oracle_passes_every_pin(source, tmp_path):
    L = _compile(source, str(tmp_path), "control")
    assert all(pin(L) for pin in PINS)


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_planted_mistake_fails_a_pin(source, tmp_path, name, old, new):
    assert source.count(old) == 1, f"mutation site not unique or missing: {old!r}"
    L = _compile(source.replace(old, new), str(tmp_path), "mutant")
    failed = [pin.__name__ for pin in PINS if not pin(L)]
    assert failed, f"no pin catches the mutant '{name}'"
