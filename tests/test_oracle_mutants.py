"""The oracle's pins catch plausible mistakes in it.

Each mutant below is the oracle's C source with one plausible slip planted in it. The energy and
force mutants (a dropped factor, a flipped sign, a wrong exponent, a transposed operand, a one-sided
embedding term) are compiled on their own (CPU only) and run against the closed-form dimer of Eq. 1
and Eq. 2, central finite differences of the mutant's own energy, and the vanishing net force and
torque of pairwise central forces. The dynamics mutants (a wrong kick or drift, Langevin friction or
noise variance, ramp, Berendsen factor, kinetic energy, Philox rounds, Box-Muller, the observables'
centre of mass, angular momentum and temperature) are run through the pin tests of test_oracle.py
themselves: the observables of a spinning dimer, the harmonic period of the dimer, the dt^2 energy
fluctuation, the exact variance recursion of free atoms under the Langevin ramp, the closed-form
Berendsen relaxation, the published Philox known-answer vectors and the normals' moments and
layout. The cutoff mutants (inclusive, ignored, shifted with the wrong exponent or sign) run through
its cutoff and shifted-cutoff pins. The structure mutants (neighbour cutoff, bond counting, the longest bond chain, the hcp rule,
self pairs in the pair-distance histogram, the displacement's centre-of-mass correction and average)
run through the pin tests of test_oracle_structure.py. Every mutant must fail at least one pin, and
the unmodified sources must pass all of them, so a mistake of these kinds cannot hide in the oracle
the CUDA path is checked against.
"""
import ctypes
import os
import shutil
import subprocess
import sys

import numpy as np
import pytest

import oracle
from paper_1210_3559_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "sc_oracle.c")
STRUCT_SRC = os.path.join(os.path.dirname(oracle.__file__), "structure_oracle.c")
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


# ------------------------------------------------------------------- dynamics
# (name, text in sc_oracle.c, replacement); each text occurs exactly once in the source
DYN_MUTANTS = [
    ("first half kick over the full step",
     "vel[3 * i + c] += h * forces[3 * i + c] * conv / mass[i];\n        if (th->kind == 1) {",
     "vel[3 * i + c] += dt * forces[3 * i + c] * conv / mass[i];\n        if (th->kind == 1) {"),
    ("NVE drift over half the step",
     "pos[3 * i + c] += dt * vel[3 * i + c];", "pos[3 * i + c] += h * vel[3 * i + c];"),
    ("second half kick with the unit conversion inverted",
     "vel[3 * i + c] += h * forces[3 * i + c] * conv / mass[i];\n        if (th->kind == 2",
     "vel[3 * i + c] += h * forces[3 * i + c] / conv / mass[i];\n        if (th->kind == 2"),
    ("Langevin friction over half the step",
     "double c1 = exp(-th->gamma_ps * 1.0e-3 * dt);", "double c1 = exp(-th->gamma_ps * 1.0e-3 * h);"),
    ("Langevin noise variance without 1 - c1^2",
     "sqrt((1.0 - c1 * c1) * ORC_KB_EV_PER_K * T_target * conv / mass[i])",
     "sqrt(ORC_KB_EV_PER_K * T_target * conv / mass[i])"),
    ("Langevin noise at the ramp's start temperature",
     "sqrt((1.0 - c1 * c1) * ORC_KB_EV_PER_K * T_target * conv / mass[i])",
     "sqrt((1.0 - c1 * c1) * ORC_KB_EV_PER_K * th->T0 * conv / mass[i])"),
    ("ramp one step ahead",
     "(th->T1 - th->T0) * (double)k / (double)nsteps", "(th->T1 - th->T0) * (double)(k + 1) / (double)nsteps"),
    ("Berendsen factor without the square root",
     "? sqrt(1.0 + (dt / (th->tau_ps * 1.0e3)) * (T_target / T_inst - 1.0))",
     "? (1.0 + (dt / (th->tau_ps * 1.0e3)) * (T_target / T_inst - 1.0))"),
    ("kinetic energy without 1/2",
     "ke += 0.5 * mass[i] *", "ke += mass[i] *"),
    ("Philox key schedule without the second Weyl increment",
     "if (round > 0) { k0 += W0; k1 += W1; }", "if (round > 0) { k0 += W0; }"),
    ("Philox multipliers swapped",
     "const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;", "const uint32_t M0 = 0xCD9E8D57u, M1 = 0xD2511F53u;"),
    ("Box-Muller radius without the factor 2",
     "double r1 = sqrt(-2.0 * log(u01(w[0])));", "double r1 = sqrt(-log(u01(w[0])));"),
    ("second normal from the other radius",
     "z[1] = r1 * sin(two_pi * u01(w[1]));", "z[1] = r2 * sin(two_pi * u01(w[1]));"),
    ("angular momentum about the origin",
     "double r[3] = {pos[3 * i] - o->com[0], pos[3 * i + 1] - o->com[1], pos[3 * i + 2] - o->com[2]};",
     "double r[3] = {pos[3 * i], pos[3 * i + 1], pos[3 * i + 2]};"),
    ("centre of mass unweighted", "o->com[k] += mass[i] * pos[3 * i + k];", "o->com[k] += pos[3 * i + k];"),
    ("angular momentum z with the cross product reversed",
     "o->angmom[2] += mass[i] * (r[0] * v[1] - r[1] * v[0]);", "o->angmom[2] += mass[i] * (r[1] * v[0] - r[0] * v[1]);"),
    ("temperature from 3N - 6 degrees of freedom",
     "o->T = N > 0 ? 2.0 * o->ekin / (3.0 * N * ORC_KB_EV_PER_K) : 0.0;",
     "o->T = N > 2 ? 2.0 * o->ekin / ((3.0 * N - 6.0) * ORC_KB_EV_PER_K) : 0.0;"),
]


def _dyn_pins():
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import test_oracle as T

    def philox_kat():
        for ctr, key, expect in T.kat_vectors():
            T.test_philox_known_answer_vectors(ctr, key, expect)

    # cheapest first; the Ornstein-Uhlenbeck test (12 s) is left out, the others cover its terms
    return [T.test_observables_of_a_spinning_dimer_closed_forms, philox_kat,
            T.test_box_muller_normals_moments_and_counter_layout,
            T.test_berendsen_free_atoms_follow_closed_form_relaxation,
            T.test_dimer_small_oscillation_period_matches_harmonic_closed_form,
            T.test_nve_energy_fluctuation_scales_as_dt_squared_and_conserves_momenta,
            T.test_langevin_ramp_follows_variance_recursion]


def _use_oracle_library(monkeypatch, src_text, out_dir, name, structure_text=None):
    """Build the oracle from src_text and structure_text (the unchanged sources where None) and make the
    oracle module load it."""
    srcs = []
    for text, base in ((src_text, SRC), (structure_text, STRUCT_SRC)):
        if text is None:
            with open(base) as f:
                text = f.read()
        path = os.path.join(out_dir, name + "_" + os.path.basename(base))
        with open(path, "w") as f:
            f.write(text)
        srcs.append(path)
    lib = os.path.join(out_dir, name + ".so")
    subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", *srcs,
                    "-o", lib, "-lm"], check=True)
    monkeypatch.setattr(oracle, "_lib", None)
    monkeypatch.setattr(oracle, "build", lambda force=False: lib)


def _first_failing_pin(pins):
    for pin in pins:
        try:
            pin()
        except Exception:  # an assertion, or a non-finite value the pin cannot digest
            return pin.__name__
    return None


def test_unmodified_oracle_passes_every_dynamics_pin(source, tmp_path, monkeypatch):
    _use_oracle_library(monkeypatch, source, str(tmp_path), "control_dyn")
    assert _first_failing_pin(_dyn_pins()) is None


@pytest.mark.parametrize("name,old,new", DYN_MUTANTS, ids=[m[0] for m in DYN_MUTANTS])
def test_planted_dynamics_mistake_fails_a_pin(source, tmp_path, monkeypatch, name, old, new):
    assert source.count(old) == 1, f"mutation site not unique or missing: {old!r}"
    _use_oracle_library(monkeypatch, source.replace(old, new), str(tmp_path), "mutant_dyn")
    assert _first_failing_pin(_dyn_pins()) is not None, f"no pin catches the mutant '{name}'"


# ---------------------------------------------------------- structural observables
# (name, text in structure_oracle.c, replacement); each text occurs exactly once in the source
STRUCT_MUTANTS = [
    ("neighbour cutoff compared with r^2 unsquared",
     "const double rn2 = r_nb * r_nb;", "const double rn2 = r_nb;"),
    ("bonds among the common neighbours counted twice",
     "for (int y = x + 1; y < k; ++y)", "for (int y = 0; y < k; ++y)"),
    ("longest bond chain replaced by a flag",
     "per_set[find_root(parent, bond_a[e])] += 1;", "per_set[find_root(parent, bond_a[e])] = 1;"),
    ("hcp required to be 12 x 422",
     "else if (n421 == 6 && n422 == 6)", "else if (n422 == 12)"),
    ("pair-distance histogram counts an atom with itself",
     "            if (j == c) continue;\n            const double r = sqrt(r2_of(pos, c, j));",
     "            const double r = sqrt(r2_of(pos, c, j));"),
    ("displacement without removing the centre-of-mass motion",
     "const double d = (pos[3 * i + q] - X[q]) - (ref[3 * i + q] - X0[q]);",
     "const double d = pos[3 * i + q] - ref[3 * i + q];"),
    ("displacement averaged over all atoms instead of the selection",
     "return n > 0 ? s / n : 0.0;", "return n > 0 ? s / N : 0.0;"),
]


def _struct_pins():
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import test_oracle_structure as S
    return [S.test_cna_signatures_fcc_hcp_icosahedron, S.test_cna_classes_of_ideal_structures,
            S.test_cna_invariances, S.test_rdf_of_the_centre_atom_is_the_fcc_shell_count,
            S.test_rdf_counts_every_core_pair_once, S.test_msd_closed_forms]


@pytest.fixture(scope="module")
def structure_source():
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    with open(STRUCT_SRC) as f:
        return f.read()


def test_unmodified_structure_oracle_passes_every_pin(structure_source, tmp_path, monkeypatch):
    _use_oracle_library(monkeypatch, None, str(tmp_path), "control_struct", structure_source)
    assert _first_failing_pin(_struct_pins()) is None


@pytest.mark.parametrize("name,old,new", STRUCT_MUTANTS, ids=[m[0] for m in STRUCT_MUTANTS])
def test_planted_structure_mistake_fails_a_pin(structure_source, tmp_path, monkeypatch, name, old, new):
    assert structure_source.count(old) == 1, f"mutation site not unique or missing: {old!r}"
    _use_oracle_library(monkeypatch, None, str(tmp_path), "mutant_struct", structure_source.replace(old, new))
    assert _first_failing_pin(_struct_pins()) is not None, f"no pin catches the mutant '{name}'"


# ------------------------------------------------------------------- cutoff forms
# (name, text in sc_oracle.c, replacement); each text occurs exactly once in the source
CUTOFF_MUTANTS = [
    ("cutoff inclusive (r <= rc)", "return !(p->rcut > 0.0) || r < p->rcut;", "return !(p->rcut > 0.0) || r <= p->rcut;"),
    ("cutoff ignored", "return !(p->rcut > 0.0) || r < p->rcut;", "return 1;"),
    ("every term shifted with the repulsive exponent",
     "t - pow(p->a / p->rcut, k)", "t - pow(p->a / p->rcut, p->n)"),
    ("shift added instead of subtracted", "t - pow(p->a / p->rcut, k)", "t + pow(p->a / p->rcut, k)"),
]


def _cutoff_pins():
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import test_oracle as T

    def shifted_dimer():
        for r in (2.3, 2.6, 4.0, 8.0):
            T.test_shifted_dimer_closed_form(r)

    return [T.test_cutoff_pairs_beyond_range_vanish_and_isolated_atom_is_zero, shifted_dimer,
            T.test_forces_with_cutoff_match_central_differences, T.test_shifted_forces_match_central_differences,
            T.test_shifted_energy_is_continuous_at_the_cutoff]


def test_unmodified_oracle_passes_every_cutoff_pin(source, tmp_path, monkeypatch):
    _use_oracle_library(monkeypatch, source, str(tmp_path), "control_cut")
    assert _first_failing_pin(_cutoff_pins()) is None


@pytest.mark.parametrize("name,old,new", CUTOFF_MUTANTS, ids=[m[0] for m in CUTOFF_MUTANTS])
def test_planted_cutoff_mistake_fails_a_pin(source, tmp_path, monkeypatch, name, old, new):
    assert source.count(old) == 1, f"mutation site not unique or missing: {old!r}"
    _use_oracle_library(monkeypatch, source.replace(old, new), str(tmp_path), "mutant_cut")
    assert _first_failing_pin(_cutoff_pins()) is not None, f"no pin catches the mutant '{name}'"


# ------------------------------------------------------------- many-body embedding
# Three coordinated edits make the embedding pairwise while rho stays right: every pair adds
# -2 c (a/r)^(m/2) to the pair sum, the sqrt-of-density term is dropped, and the force is the matching
# pairwise one. Energy and force stay consistent, rho_i = sum (a/r)^m is untouched and the dimer is
# unchanged (one pair: sqrt of the sum equals the sum of the sqrt), so only a closed form with several
# neighbours per atom tells this from the paper's sqrt of the summed density (Eq. 1).
PAIRWISE_EMBEDDING = [
    ("acc += term(r, p->n, p);\n            }\n            pair_i[i] = acc;",
     "acc += term(r, p->n, p) - 2.0 * p->c * sqrt(term(r, p->m, p));\n            }\n            pair_i[i] = acc;"),
    ("e_emb += -p->eps * p->c * sqrt(rho[i]);", "e_emb += 0.0;"),
    ("kemb * (g[i] + g[j]) * pow(s, p->m)) / (r * r);", "kemb * 2.0 * pow(s, 0.5 * p->m)) / (r * r);"),
]


def test_pairwise_embedding_is_caught_only_by_the_many_neighbour_closed_forms(source, tmp_path, monkeypatch):
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import test_oracle as T
    text = source
    for old, new in PAIRWISE_EMBEDDING:
        assert text.count(old) == 1, f"mutation site not unique or missing: {old!r}"
        text = text.replace(old, new)
    _use_oracle_library(monkeypatch, text, str(tmp_path), "mutant_pairwise")

    def dimer():
        for r in (1.9, 2.041345, 2.3, 2.49, 3.1):
            T.test_dimer_energy_and_force_closed_form(r)

    def finite_differences():
        for n, seed in ((3, 1), (13, 2)):
            T.test_forces_match_central_differences(n, seed)

    def trimer_tetramer():
        for r in (2.3, 2.49, 3.0, 4.5):
            T.test_trimer_and_tetramer_closed_forms(r)

    assert _first_failing_pin([dimer, finite_differences, T.test_net_force_and_torque_vanish]) is None
    assert _first_failing_pin([trimer_tetramer]) == "trimer_tetramer"


# ---------------------------------------------------------------- Langevin splitting
_AOA = """                    pos[3 * i + c] += h * vel[3 * i + c];
                    vel[3 * i + c] = c1 * vel[3 * i + c] + sigma * z[c];
                    pos[3 * i + c] += h * vel[3 * i + c];"""
_O_AT_END = """        if (th->kind == 1) {
            double c1 = exp(-th->gamma_ps * 1.0e-3 * dt);
            for (int i = 0; i < N; ++i) {
                double z[3];
                orc_langevin_normals(th->seed, cluster, step0 + k, (uint32_t)i, z);
                double sigma = sqrt((1.0 - c1 * c1) * ORC_KB_EV_PER_K * T_target * conv / mass[i]);
                for (int c = 0; c < 3; ++c) vel[3 * i + c] = c1 * vel[3 * i + c] + sigma * z[c];
            }
        }
        if (th->kind == 2 && N > 0) {"""
# other orderings of the same sub-steps (each keeps the free-atom Ornstein-Uhlenbeck statistics exact)
SPLITTING_MUTANTS = [
    ("full drift, then friction (B A O B)",
     [(_AOA, """                    pos[3 * i + c] += dt * vel[3 * i + c];
                    vel[3 * i + c] = c1 * vel[3 * i + c] + sigma * z[c];""")]),
    ("velocity Verlet, then friction (B A B O)",
     [(_AOA, "                    pos[3 * i + c] += dt * vel[3 * i + c];"),
      ("        if (th->kind == 2 && N > 0) {", _O_AT_END)]),
]


_BER_BLOCK = """        if (th->kind == 2 && N > 0) {
            double T_inst = 2.0 * kinetic(N, vel, mass) / (3.0 * N * ORC_KB_EV_PER_K);
            double lambda = T_inst > 0.0
                                ? sqrt(1.0 + (dt / (th->tau_ps * 1.0e3)) * (T_target / T_inst - 1.0))
                                : 1.0;
            for (int i = 0; i < 3 * N; ++i) vel[i] *= lambda;
        }
"""
_SECOND_KICK = """        orc_energy_forces(N, pos, p, forces, NULL, NULL);
        for (int i = 0; i < N; ++i)
            for (int c = 0; c < 3; ++c) vel[3 * i + c] += h * forces[3 * i + c] * conv / mass[i];
"""


def test_berendsen_rescale_before_the_second_kick_fails_the_tau_equal_dt_pin(source, tmp_path, monkeypatch):
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import test_oracle as T
    old = _SECOND_KICK + _BER_BLOCK
    assert source.count(old) == 1, "mutation site not unique or missing"
    _use_oracle_library(monkeypatch, source.replace(old, _BER_BLOCK + _SECOND_KICK), str(tmp_path), "mutant_ber")
    # free atoms feel no kick, so the closed-form relaxation cannot tell the order apart
    assert _first_failing_pin([T.test_berendsen_free_atoms_follow_closed_form_relaxation]) is None
    assert _first_failing_pin([T.test_berendsen_with_tau_equal_to_dt_lands_on_the_ramp_target_every_step]) is not None


@pytest.mark.parametrize("name,subs", SPLITTING_MUTANTS, ids=[m[0] for m in SPLITTING_MUTANTS])
def test_other_langevin_splittings_fail_the_harmonic_sampling_pin(source, tmp_path, monkeypatch, name, subs):
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    import test_oracle as T
    text = source
    for old, new in subs:
        assert text.count(old) == 1, f"mutation site not unique or missing: {old!r}"
        text = text.replace(old, new)
    _use_oracle_library(monkeypatch, text, str(tmp_path), "mutant_split")
    # with U = 0 the kicks vanish and one friction step per step remains: the free-atom pin cannot tell
    assert _first_failing_pin([T.test_langevin_ramp_follows_variance_recursion]) is None
    assert _first_failing_pin([T.test_langevin_baoab_samples_harmonic_configurations_exactly]) is not None
