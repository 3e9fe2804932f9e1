"""Seeded synthetic inputs: cluster geometries, masses and initial velocities.

This module holds input preparation only: lattice and icosahedron site lists,
Maxwell-Boltzmann velocity draws, and the Ni parameter set printed in the paper
(Sec. II A). It contains none of the potential, force or integrator arithmetic.
Both the CUDA library's tests and the oracle's tests build their inputs here.

Recipes:
  * ``fcc_sphere(N)``: the N sites of the FCC lattice (lattice constant a, sites
    (a/2)(i, j, k) with i + j + k even, one atom at the origin) nearest to the
    origin; ties in |r|^2 are broken by (i, j, k) in lexicographic order, so the
    count is exact for any N.
  * ``mackay_icosahedron(shells, d_nn)``: centre atom plus shells k = 1..shells of
    10k^2 + 2 atoms each; the spacing between neighbouring sites along a shell
    edge is d_nn, so the vertex radius of shell k is k * d_nn * 0.9510565...
  * ``maxwell_boltzmann``: Gaussian velocities (numpy PCG64 with the given seed),
    centre-of-mass velocity removed, rigid rotation removed (omega = I^-1 L), then
    rescaled so that 2 E_kin / (dof k_B) equals the target temperature.
"""
from __future__ import annotations

import itertools

import numpy as np

# Ni parameters of the Sutton-Chen potential as printed in the paper (Sec. II A).
NI_SC = dict(eps=1.5707e-2, c=39.432, a=3.52, n=9, m=6)
# Standard atomic weight of nickel, amu.
NI_MASS_AMU = 58.6934
# Unit conversions used only to draw velocities at a temperature:
# k_B in eV/K (exact, SI 2019); 1 eV/amu in (Angstrom/fs)^2 (e and u, CODATA).
_KB = 8.617333262e-5
_EV_PER_AMU_IN_A2_FS2 = 1.602176634e-19 / 1.66053906660e-27 * 1.0e-10


def fcc_sphere(n_atoms: int, a: float = 3.52) -> np.ndarray:
    """Exactly ``n_atoms`` FCC sites nearest the origin (deterministic order), shape (N, 3)."""
    n_atoms = int(n_atoms)
    if n_atoms <= 0:
        return np.zeros((0, 3))
    # radius estimate from the FCC number density 4 / a^3, plus a margin of two cells
    r_est = a * (3.0 * n_atoms / (16.0 * np.pi)) ** (1.0 / 3.0) + 2.0 * a
    K = int(np.ceil(2.0 * r_est / a)) + 1
    rng = np.arange(-K, K + 1)
    i, j, k = np.meshgrid(rng, rng, rng, indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    keep = (i + j + k) % 2 == 0
    i, j, k = i[keep], j[keep], k[keep]
    r2 = i * i + j * j + k * k
    order = np.lexsort((k, j, i, r2))  # primary key r2, then i, j, k
    sel = order[:n_atoms]
    if r2[sel[-1]] * (a / 2.0) ** 2 >= (K * a / 2.0) ** 2:
        raise RuntimeError("fcc_sphere: enumeration box too small")
    return (a / 2.0) * np.stack([i[sel], j[sel], k[sel]], axis=1).astype(np.float64)


def _icosahedron_vertices() -> np.ndarray:
    phi = (1.0 + 5.0 ** 0.5) / 2.0
    v = []
    for s1 in (-1.0, 1.0):
        for s2 in (-1.0, 1.0):
            v += [(0.0, s1, s2 * phi), (s1, s2 * phi, 0.0), (s2 * phi, 0.0, s1)]
    return np.array(v) / 2.0  # edge length 1


def mackay_icosahedron(shells: int = 3, d_nn: float = 2.49) -> np.ndarray:
    """Mackay icosahedron with ``shells`` closed shells (1 + sum 10k^2 + 2 atoms)."""
    V = _icosahedron_vertices()
    d = np.linalg.norm(V[:, None, :] - V[None, :, :], axis=-1)
    faces = [f for f in itertools.combinations(range(12), 3)
             if abs(d[f[0], f[1]] - 1) < 1e-9 and abs(d[f[1], f[2]] - 1) < 1e-9 and abs(d[f[0], f[2]] - 1) < 1e-9]
    assert len(faces) == 20
    pts = [np.zeros(3)]
    for k in range(1, shells + 1):
        seen = {}
        for (p, q, r) in faces:
            A, B, C = V[p] * k, V[q] * k, V[r] * k
            for u in range(k + 1):
                for w in range(k + 1 - u):
                    x = A + (u / k) * (B - A) + (w / k) * (C - A)
                    key = tuple(np.round(x, 9))
                    seen.setdefault(key, x)
        shell = sorted(seen.values(), key=lambda x: tuple(np.round(x, 9)))
        assert len(shell) == 10 * k * k + 2
        pts += shell
    return np.array(pts) * d_nn


def masses(n_atoms: int, mass_amu: float = NI_MASS_AMU) -> np.ndarray:
    return np.full(int(n_atoms), float(mass_amu))


def maxwell_boltzmann(pos: np.ndarray, mass: np.ndarray, T_K: float, seed: int,
                      dof: str = "3N-6") -> np.ndarray:
    """Velocities (Angstrom/fs) at temperature T_K with zero momentum and angular momentum."""
    pos = np.asarray(pos, dtype=np.float64)
    mass = np.asarray(mass, dtype=np.float64)
    N = len(pos)
    if N == 0:
        return np.zeros((0, 3))
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    sigma = np.sqrt(_KB * T_K * _EV_PER_AMU_IN_A2_FS2 / mass)
    v = rng.standard_normal((N, 3)) * sigma[:, None]
    M = mass.sum()
    v -= (mass[:, None] * v).sum(0) / M
    if N >= 3:
        com = (mass[:, None] * pos).sum(0) / M
        r = pos - com
        L = (mass[:, None] * np.cross(r, v)).sum(0)
        I = (mass[:, None, None] * ((r * r).sum(1)[:, None, None] * np.eye(3) - r[:, :, None] * r[:, None, :])).sum(0)
        if abs(np.linalg.det(I)) > 1e-12 * max(1.0, np.trace(I)) ** 3:
            omega = np.linalg.solve(I, L)
            v -= np.cross(omega, r)
    ndof = {"3N": 3 * N, "3N-3": 3 * N - 3, "3N-6": 3 * N - 6}[dof] if N > 2 else 3 * N
    ke = 0.5 * (mass[:, None] * v * v).sum() / _EV_PER_AMU_IN_A2_FS2
    if ke > 0 and ndof > 0 and T_K > 0:
        v *= np.sqrt(0.5 * ndof * _KB * T_K / ke)
    elif T_K == 0:
        v[:] = 0.0
    return v


def batched_sizes(n_clusters: int = 512, lo: int = 55, hi: int = 2000, seed: int = 5) -> np.ndarray:
    """Cluster sizes uniform on {lo..hi} from a seeded PCG64 stream."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    return rng.integers(lo, hi + 1, size=int(n_clusters)).astype(np.int32)


def random_rotation(seed: int) -> np.ndarray:
    """A seeded uniformly random proper rotation matrix (QR of a Gaussian matrix)."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def jitter(pos: np.ndarray, amplitude: float, seed: int) -> np.ndarray:
    """Positions displaced by independent uniform noise in [-amplitude, amplitude]."""
    rng = np.random.Generator(np.random.PCG64(int(seed)))
    return np.asarray(pos, dtype=np.float64) + rng.uniform(-amplitude, amplitude, size=np.shape(pos))
