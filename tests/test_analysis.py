"""Host analysis helpers pinned to textbook structures and synthetic traces (no GPU).

Common-neighbour signatures (Honeycutt and Andersen 1987): every nearest-neighbour pair of a perfect
FCC lattice is 421; an HCP atom has six 421 (in-plane) and six 422 (out-of-plane) pairs; the centre of
a Mackay icosahedron has twelve 555 pairs.
"""
import numpy as np
import pytest

from paper_1210_3559_gb300 import analysis, inputs

pytest.importorskip("scipy.spatial")


def hcp_ball(n_target=1500, d=2.489):
    """Ideal HCP (c/a = sqrt(8/3)) points, the n_target closest to an atom at the origin."""
    c = d * np.sqrt(8.0 / 3.0)
    pts = []
    for k in range(-10, 11):
        off = np.array([d / 2, d / (2 * np.sqrt(3)), 0.0]) if k % 2 else np.zeros(3)
        for i in range(-12, 13):
            for j in range(-12, 13):
                pts.append(np.array([i * d + j * d / 2, j * d * np.sqrt(3) / 2, k * c / 2]) + off)
    pts = np.array(pts)
    return pts[np.argsort(np.einsum("ij,ij->i", pts, pts), kind="stable")[:n_target]]


def test_fcc_signatures_and_interior_fraction():
    pos = inputs.fcc_sphere(2000)
    r_cut = 0.5 * (1 / np.sqrt(2) + 1) * 3.52
    nbrs = analysis.neighbour_lists(pos, r_cut)
    assert len(nbrs[0]) == 12  # the centre atom
    assert all(analysis.cna_signature(nbrs, 0, int(j)) == (4, 2, 1) for j in nbrs[0])
    kind = analysis.classify(pos)
    r = np.linalg.norm(pos, axis=1)
    assert np.all(kind[r < r.max() - 6.0] == 1)  # two full shells inside the surface: FCC
    assert np.all(kind[r > r.max() - 1.0] == 0)  # surface atoms lack neighbours
    f = analysis.crystalline_fraction(pos)
    assert f["hcp"] == 0 and 0.4 < f["fcc"] == f["crystalline"] < 1


def test_hcp_signatures():
    pos = hcp_ball()
    nbrs = analysis.neighbour_lists(pos, 0.5 * (1 / np.sqrt(2) + 1) * 3.52)
    sig = sorted(analysis.cna_signature(nbrs, 0, int(j)) for j in nbrs[0])
    assert sig == [(4, 2, 1)] * 6 + [(4, 2, 2)] * 6
    kind = analysis.classify(pos)
    r = np.linalg.norm(pos, axis=1)
    assert np.all(kind[r < r.max() - 6.0] == 2)


def test_icosahedral_centre_is_not_crystalline():
    pos = inputs.mackay_icosahedron(3, 2.49)
    nbrs = analysis.neighbour_lists(pos, 3.0)
    assert len(nbrs[0]) == 12
    assert all(analysis.cna_signature(nbrs, 0, int(j)) == (5, 5, 5) for j in nbrs[0])
    assert analysis.classify(pos)[0] == 0


def test_disordered_structure_is_not_crystalline():
    pos = inputs.jitter(inputs.fcc_sphere(1000), 0.6, 3)  # rms displacement ~40 % of the bond
    assert analysis.crystalline_fraction(pos)["crystalline"] < 0.01
    rng = np.random.default_rng(1)  # uniform points at the same density: no order at all
    R = 3.52 * (3 * 1000 / (16 * np.pi)) ** (1 / 3)
    gas = rng.uniform(-R, R, (4000, 3))
    gas = gas[np.linalg.norm(gas, axis=1) < R][:1000]
    assert analysis.crystalline_fraction(gas)["crystalline"] == 0


def test_solidification_time_on_synthetic_traces():
    rng = np.random.default_rng(0)
    t = np.arange(400.0)  # ps
    e = -4.0 + 0.002 * rng.standard_normal(len(t))
    fall = (t >= 150) & (t < 190)
    e[fall] -= 0.06 * (t[fall] - 150) / 40
    e[t >= 190] -= 0.06
    tn = analysis.solidification_time(e)
    assert tn is not None and 146 <= tn <= 152
    # the thermalisation after a quench (energy relaxing within a few ps) is not a solidification
    relax = -4.0 + 0.15 * np.exp(-t / 2.0) + 0.002 * rng.standard_normal(len(t))
    assert analysis.solidification_time(relax) is None
    # a small cluster's large fluctuations (0.02 eV per sample) are not either, but its real fall is
    noisy = -4.0 + 0.02 * rng.standard_normal(len(t))
    assert analysis.solidification_time(noisy) is None
    noisy[t >= 200] -= 0.08
    tn3 = analysis.solidification_time(noisy)
    assert tn3 is not None and 185 <= tn3 <= 201
    # a dip that recovers within one window is not a solidification
    dip = -4.0 + 0.002 * rng.standard_normal(len(t))
    dip[(t >= 200) & (t < 212)] -= 0.05
    assert analysis.solidification_time(dip) is None
    flat = -4.0 + 0.002 * rng.standard_normal(len(t))
    assert analysis.solidification_time(flat) is None  # censored
    # a time step of 0.5 ps gives the same time in ps
    e2 = np.repeat(e, 2)
    tn2 = analysis.solidification_time(e2, dt_ps=0.5)
    assert abs(tn2 - tn) <= 1.0


def test_energy_drift_recovers_a_linear_trend():
    t = np.linspace(0.0, 2.0e4, 201)  # fs
    n = 100
    e = n * (-4.0 + 0.05 * t * 1e-6)  # 0.05 eV / atom / ns
    d = analysis.energy_drift(t, e, n)
    assert d["slope_eV_per_atom_per_ns"] == pytest.approx(0.05, rel=1e-9)
    assert d["max_abs_dE_eV_per_atom"] == pytest.approx(0.05 * 0.02, rel=1e-9)
    assert d["rms_eV_per_atom"] < 1e-12


def test_cycle_transition_temperatures_on_synthetic_curves():
    """The heating-cooling analysis finds the steepest rise and fall of E(T) (a latent-heat step on
    a linear heat-capacity background, with noise)."""
    from paper_1210_3559_gb300 import cycle
    rng = np.random.default_rng(4)
    T_up = np.arange(400.0, 1400.0, 1.0)
    e_up = -4.4 + 2.6e-4 * (T_up - 400) + 0.06 / (1 + np.exp(-(T_up - 1180.0) / 4.0)) + 3e-4 * rng.standard_normal(len(T_up))
    T_dn = T_up[::-1]
    e_dn = -4.4 + 2.6e-4 * (T_dn - 400) + 0.06 / (1 + np.exp(-(T_dn - 790.0) / 4.0)) + 3e-4 * rng.standard_normal(len(T_dn))
    assert abs(cycle._steepest(T_up, e_up) - 1180.0) <= 5.0
    assert abs(cycle._steepest(T_dn, e_dn) - 790.0) <= 5.0
