"""FP64 CPU oracle for Sutton-Chen Ni cluster MD (ctypes wrapper around sc_oracle.c).

TEST INFRASTRUCTURE. Only the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package. The product library
(``paper_1210_3559_gb300``) never imports it and has no CPU fallback to it.

Every function follows the plain definitions of the paper (Eq. 1 energy, Eq. 2
density, the derivative of Eq. 1 for forces, velocity Verlet with a Langevin
thermostat, Sec. II "Computational approach"); see the C source for each.
The structural observables of Sec. III (central-atom pair distances, mean squared
displacement, common-neighbour analysis) are in structure_oracle.c.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRCS = [os.path.join(_HERE, "sc_oracle.c"), os.path.join(_HERE, "structure_oracle.c")]
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the C sources with gcc (-O2, IEEE double evaluated as written, OpenMP) into oracle/_build."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(os.path.getmtime(f) for f in _SRCS):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", *_SRCS, "-o", tmp,
               "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


class Params(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("c", ctypes.c_double), ("a", ctypes.c_double),
                ("n", ctypes.c_int), ("m", ctypes.c_int), ("rcut", ctypes.c_double), ("shift", ctypes.c_int),
                ("reserved", ctypes.c_int)]


class Thermostat(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("T0", ctypes.c_double), ("T1", ctypes.c_double),
                ("gamma_ps", ctypes.c_double), ("tau_ps", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class Obs(ctypes.Structure):
    _fields_ = [("epot", ctypes.c_double), ("ekin", ctypes.c_double), ("etot", ctypes.c_double),
                ("T", ctypes.c_double), ("com", ctypes.c_double * 3), ("mom", ctypes.c_double * 3),
                ("angmom", ctypes.c_double * 3)]


NVE, LANGEVIN, BERENDSEN = 0, 1, 2
_DP = ctypes.POINTER(ctypes.c_double)


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            lib.orc_num_threads.argtypes = [ctypes.c_int]
            lib.orc_num_threads.restype = ctypes.c_int
            lib.orc_unit_ev_per_amu_a2_fs2.restype = ctypes.c_double
            lib.orc_unit_kb.restype = ctypes.c_double
            lib.orc_density.argtypes = [ctypes.c_int, _DP, ctypes.POINTER(Params), _DP]
            lib.orc_energy_forces.argtypes = [ctypes.c_int, _DP, ctypes.POINTER(Params), _DP, _DP, _DP]
            lib.orc_energy_forces.restype = ctypes.c_double
            lib.orc_atom_energies.argtypes = [ctypes.c_int, _DP, ctypes.POINTER(Params), _DP]
            u32p = ctypes.POINTER(ctypes.c_uint32)
            lib.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            lib.orc_langevin_normals.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int64,
                                                 ctypes.c_uint32, _DP]
            lib.orc_observables.argtypes = [ctypes.c_int, _DP, _DP, _DP, ctypes.POINTER(Params),
                                            ctypes.POINTER(Obs)]
            lib.orc_md_batch.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int32), _DP, _DP, _DP,
                                         _DP, ctypes.POINTER(Params), ctypes.c_int64, ctypes.c_int64,
                                         ctypes.c_double, ctypes.POINTER(Thermostat)]
            i32p = ctypes.POINTER(ctypes.c_int32)
            lib.ors_com.argtypes = [ctypes.c_int, _DP, _DP, _DP]
            lib.ors_rdf.argtypes = [ctypes.c_int, _DP, _DP, ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                    ctypes.POINTER(ctypes.c_int64), i32p]
            lib.ors_msd.argtypes = [ctypes.c_int, _DP, _DP, _DP, ctypes.c_double, i32p]
            lib.ors_msd.restype = ctypes.c_double
            lib.ors_cna_signature.argtypes = [ctypes.c_int, _DP, ctypes.c_double, ctypes.c_int, ctypes.c_int,
                                              i32p]
            lib.ors_cna.argtypes = [ctypes.c_int, _DP, ctypes.c_double, i32p, i32p]
            _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(_DP)


def _pos(pos) -> np.ndarray:
    pos = np.ascontiguousarray(pos, dtype=np.float64)
    if pos.ndim != 2 or pos.shape[1] != 3:
        raise ValueError("positions must have shape (N, 3)")
    return pos


def params(eps=1.5707e-2, c=39.432, a=3.52, n=9, m=6, rcut=0.0, shift=False) -> Params:
    """Sutton-Chen parameters; defaults are the paper's Ni set (Sec. II A). With rcut > 0 the pair
    terms are truncated at rcut, or with shift=True also shifted by their value at rcut."""
    return Params(float(eps), float(c), float(a), int(n), int(m), float(rcut), 1 if shift else 0, 0)


def num_threads(n: int = 0) -> int:
    """Set (n > 0) and return the OpenMP thread count the oracle uses."""
    return _load().orc_num_threads(int(n))


def ev_per_amu_a2_fs2() -> float:
    return _load().orc_unit_ev_per_amu_a2_fs2()


def kb() -> float:
    return _load().orc_unit_kb()


def density(pos, p: Params | None = None) -> np.ndarray:
    """rho_i = sum_{j != i} (a/r_ij)^m (Eq. 2)."""
    p = p or params()
    pos = _pos(pos)
    rho = np.zeros(len(pos))
    _load().orc_density(len(pos), _dp(pos), ctypes.byref(p), _dp(rho))
    return rho


def energy_forces(pos, p: Params | None = None):
    """Return (U, F[N,3], (E_pair, E_emb), rho) for one cluster (Eq. 1, Eq. 2, -dU/dr)."""
    p = p or params()
    pos = _pos(pos)
    F = np.zeros_like(pos)
    et = np.zeros(2)
    rho = np.zeros(len(pos))
    U = _load().orc_energy_forces(len(pos), _dp(pos), ctypes.byref(p), _dp(F), _dp(et), _dp(rho))
    return U, F, (et[0], et[1]), rho


def energy(pos, p: Params | None = None) -> float:
    p = p or params()
    pos = _pos(pos)
    return _load().orc_energy_forces(len(pos), _dp(pos), ctypes.byref(p), None, None, None)


def atom_energies(pos, p: Params | None = None) -> np.ndarray:
    """Per-atom summand of Eq. 1: eps [1/2 sum_j (a/r_ij)^n - c sqrt(rho_i)]."""
    p = p or params()
    pos = _pos(pos)
    e = np.zeros(len(pos))
    _load().orc_atom_energies(len(pos), _dp(pos), ctypes.byref(p), _dp(e))
    return e


def philox4x32_10(ctr, key) -> np.ndarray:
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    _load().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def langevin_normals(seed: int, cluster: int, step: int, atom: int) -> np.ndarray:
    z = np.zeros(3)
    _load().orc_langevin_normals(int(seed), int(cluster), int(step), int(atom), _dp(z))
    return z


def observables(pos, vel, mass, p: Params | None = None) -> dict:
    p = p or params()
    pos = _pos(pos)
    vel = _pos(vel)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    o = Obs()
    _load().orc_observables(len(pos), _dp(pos), _dp(vel), _dp(mass), ctypes.byref(p), ctypes.byref(o))
    return dict(epot=o.epot, ekin=o.ekin, etot=o.etot, T=o.T, com=np.array(o.com[:]),
                mom=np.array(o.mom[:]), angmom=np.array(o.angmom[:]))


# ---------------------------------------------------------------- structure (Sec. III)
CNA_OTHER, CNA_FCC, CNA_HCP, CNA_ICO = 0, 1, 2, 3


def _i32p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))


def com(pos, mass) -> np.ndarray:
    """Centre of mass sum m x / sum m."""
    pos = _pos(pos)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    X = np.zeros(3)
    _load().ors_com(len(pos), _dp(pos), _dp(mass), _dp(X))
    return X


def rdf(pos, mass, r_core: float, bin_A: float, nbins: int):
    """(counts[nbins], n_core): pair distances from the atoms within r_core of the centre of mass to
    every other atom, histogrammed in bins of bin_A."""
    pos = _pos(pos)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    counts = np.zeros(int(nbins), dtype=np.int64)
    nc = np.zeros(1, dtype=np.int32)
    _load().ors_rdf(len(pos), _dp(pos), _dp(mass), float(r_core), float(bin_A), int(nbins),
                    counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _i32p(nc))
    return counts, int(nc[0])


def msd(pos, ref, mass, r_core: float = 0.0):
    """(MSD in A^2, atoms averaged): displacement from ref with the centre-of-mass motion removed, over
    the atoms within r_core of the reference centre of mass (all atoms if r_core <= 0)."""
    pos = _pos(pos)
    ref = _pos(ref)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    n = np.zeros(1, dtype=np.int32)
    v = _load().ors_msd(len(pos), _dp(pos), _dp(ref), _dp(mass), float(r_core), _i32p(n))
    return v, int(n[0])


def cna_signature(pos, i: int, j: int, r_nb: float = 3.0):
    """Common-neighbour signature (k, b, l) of the pair i-j."""
    pos = _pos(pos)
    out = np.zeros(3, dtype=np.int32)
    _load().ors_cna_signature(len(pos), _dp(pos), float(r_nb), int(i), int(j), _i32p(out))
    return tuple(int(x) for x in out)


def cna(pos, r_nb: float = 3.0):
    """(class[N], neighbours[N]): CNA_FCC / CNA_HCP / CNA_ICO / CNA_OTHER per atom."""
    pos = _pos(pos)
    cls = np.zeros(len(pos), dtype=np.int32)
    nnb = np.zeros(len(pos), dtype=np.int32)
    _load().ors_cna(len(pos), _dp(pos), float(r_nb), _i32p(cls), _i32p(nnb))
    return cls, nnb


def thermostat(kind=NVE, T0=0.0, T1=None, gamma_ps=1.0, tau_ps=0.1, seed=0) -> Thermostat:
    return Thermostat(int(kind), float(T0), float(T0 if T1 is None else T1), float(gamma_ps),
                      float(tau_ps), int(seed))


class Batch:
    """Independent clusters stored back to back; state advanced in place by run()."""

    def __init__(self, sizes, pos, vel, mass, p: Params | None = None):
        self.sizes = np.ascontiguousarray(sizes, dtype=np.int32)
        self.pos = _pos(pos).copy()
        self.vel = _pos(vel).copy()
        self.mass = np.ascontiguousarray(mass, dtype=np.float64).copy()
        if self.sizes.sum() != len(self.pos) or len(self.vel) != len(self.pos) or len(self.mass) != len(self.pos):
            raise ValueError("sizes, positions, velocities and masses disagree")
        self.p = p or params()
        self.step = 0
        self.forces = np.zeros_like(self.pos)
        for s, e in self.ranges():
            if e > s:
                _, F, _, _ = energy_forces(self.pos[s:e], self.p)
                self.forces[s:e] = F

    def ranges(self):
        off = np.concatenate([[0], np.cumsum(self.sizes)])
        return [(int(off[b]), int(off[b + 1])) for b in range(len(self.sizes))]

    def run(self, nsteps: int, dt_fs: float, th: Thermostat | None = None):
        th = th or thermostat()
        _load().orc_md_batch(len(self.sizes), self.sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                             _dp(self.pos), _dp(self.vel), _dp(self.forces), _dp(self.mass),
                             ctypes.byref(self.p), int(self.step), int(nsteps), float(dt_fs),
                             ctypes.byref(th))
        self.step += int(nsteps)

    def observables(self):
        return [observables(self.pos[s:e], self.vel[s:e], self.mass[s:e], self.p) for s, e in self.ranges()]
