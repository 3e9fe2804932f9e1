"""Host-side analysis of what the library returns (snapshots and observable histories).

None of this is on the GPU path; it reads the positions and energy traces of finished runs:
  * common-neighbour analysis (Honeycutt and Andersen, J. Phys. Chem. 91, 4950 (1987)) and the
    crystalline (FCC + HCP) fraction of a cluster, the structural signal of solidification that the
    paper reads off energies, radial distribution functions and diffusion (Sec. III);
  * the solidification time of a cluster from its total energy per atom against time: the moment
    at which the energy starts to fall rapidly (Sec. III D), made operational as stated below;
  * the drift of the total energy of an NVE run.
"""
from __future__ import annotations

import numpy as np


# ------------------------------------------------------------ common neighbours
def neighbour_lists(pos: np.ndarray, r_cut: float) -> list[np.ndarray]:
    """Indices of the atoms within r_cut of each atom (itself excluded), ascending."""
    from scipy.spatial import cKDTree
    tree = cKDTree(pos)
    lists = tree.query_ball_point(pos, r_cut)
    return [np.array(sorted(j for j in lst if j != i), dtype=np.int64) for i, lst in enumerate(lists)]


def _longest_chain(nodes: np.ndarray, bonds: list[tuple[int, int]]) -> int:
    """Bonds in the largest connected group of bonds among the common neighbours."""
    parent = {int(k): int(k) for k in nodes}

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    for a, b in bonds:
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[ra] = rb
    count: dict[int, int] = {}
    for a, _ in bonds:
        r = find(a)
        count[r] = count.get(r, 0) + 1
    return max(count.values()) if count else 0


def cna_signature(nbrs: list[np.ndarray], i: int, j: int, sets: list[set] | None = None) -> tuple[int, int, int]:
    """(common neighbours, bonds among them, bonds in their longest chain) of the bonded pair i-j."""
    common = np.intersect1d(nbrs[i], nbrs[j], assume_unique=True)
    bonds = []
    for x in range(len(common)):
        a = int(common[x])
        sa = sets[a] if sets is not None else set(nbrs[a].tolist())
        bonds.extend((a, int(b)) for b in common[x + 1:] if int(b) in sa)
    return len(common), len(bonds), _longest_chain(common, bonds)


def classify(pos: np.ndarray, a: float = 3.52) -> np.ndarray:
    """Per-atom structure: 1 = FCC (12 neighbours, all pairs 421), 2 = HCP (12 neighbours, six
    421 and six 422), 0 = other. Neighbour cutoff halfway between the first and second FCC shells,
    (1/sqrt(2) + 1) a / 2 (3.00 A for Ni)."""
    r_cut = 0.5 * (1.0 / np.sqrt(2.0) + 1.0) * a
    nbrs = neighbour_lists(np.asarray(pos, dtype=np.float64), r_cut)
    sets = [set(x.tolist()) for x in nbrs]
    out = np.zeros(len(pos), dtype=np.int8)
    for i, ni in enumerate(nbrs):
        if len(ni) != 12:
            continue
        n421 = n422 = 0
        for j in ni:
            s = cna_signature(nbrs, i, int(j), sets)
            if s == (4, 2, 1):
                n421 += 1
            elif s == (4, 2, 2):
                n422 += 1
            else:
                break
        if n421 == 12:
            out[i] = 1
        elif n421 == 6 and n422 == 6:
            out[i] = 2
    return out


def crystalline_fraction(pos: np.ndarray, a: float = 3.52) -> dict:
    kind = classify(pos, a)
    n = max(len(kind), 1)
    return {"fcc": float(np.sum(kind == 1) / n), "hcp": float(np.sum(kind == 2) / n),
            "crystalline": float(np.sum(kind > 0) / n)}


# -------------------------------------------------------- solidification time
def solidification_time(e_per_atom: np.ndarray, dt_ps: float = 1.0, ref_ps: float = 20.0,
                        window_ps: float = 10.0, drop_eV: float = 0.02, skip_ps: float = 10.0,
                        n_sigma: float = 4.0, persist_ps: float = 30.0) -> float | None:
    """Time (ps from the first sample) at which the energy per atom starts its fall, or None if it
    never falls (right-censored).

    The first skip_ps are left out (the liquid thermalising at the bath temperature after the
    quench) and the liquid reference is the mean over the next ref_ps. The fall is detected where
    the trailing window_ps running mean first lies below the reference by the larger of drop_eV
    (about a third of the latent heat per atom of a 2000-atom Ni cluster) and n_sigma standard
    deviations of that running mean over the reference span (small clusters fluctuate more), and
    stays below for persist_ps (a freezing cluster does not melt back at these temperatures). It is
    dated at the last sample before that point still within one standard deviation of the liquid
    reference."""
    e = np.asarray(e_per_atom, dtype=np.float64)
    skip = int(round(skip_ps / dt_ps))
    n_ref = max(2, int(round(ref_ps / dt_ps)))
    w = max(1, int(round(window_ps / dt_ps)))
    if len(e) < skip + n_ref + w:
        return None
    ref_span = e[skip:skip + n_ref]
    ref, sigma = ref_span.mean(), ref_span.std()
    run = np.convolve(e, np.ones(w) / w, mode="valid")  # run[k] = mean of e[k : k + w]
    ref_run = run[skip:skip + n_ref - w + 1]
    thresh = ref - max(drop_eV, n_sigma * (ref_run.std() if len(ref_run) > 1 else 0.0))
    below = run < thresh
    hold = max(1, int(round(persist_ps / dt_ps)))
    for k in range(skip + n_ref - w + 1, len(run) - hold):
        if below[k] and below[k:k + hold + 1].all():
            j = k + w - 1  # last sample of the first window below the threshold
            while j > skip and e[j] < ref - sigma:
                j -= 1
            return j * dt_ps
    return None


# ------------------------------------------------------------------ NVE drift
def energy_drift(t_fs: np.ndarray, e_tot_eV: np.ndarray, n_atoms: int) -> dict:
    """Least-squares slope of E_tot / N against time (eV per atom per ns), the largest deviation
    from the first sample and the RMS fluctuation about the fitted line (eV per atom)."""
    t = np.asarray(t_fs, dtype=np.float64) * 1e-6  # ns
    e = np.asarray(e_tot_eV, dtype=np.float64) / n_atoms
    if len(t) < 2:
        return {"slope_eV_per_atom_per_ns": None, "max_abs_dE_eV_per_atom": None, "rms_eV_per_atom": None}
    slope, icpt = np.polyfit(t, e, 1)
    return {"slope_eV_per_atom_per_ns": float(slope), "max_abs_dE_eV_per_atom": float(np.max(np.abs(e - e[0]))),
            "rms_eV_per_atom": float(np.sqrt(np.mean((e - (slope * t + icpt)) ** 2)))}
