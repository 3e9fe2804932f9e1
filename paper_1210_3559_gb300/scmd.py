"""Python binding of libscmd (include/scmd.h): same entry-point names, ctypes marshalling only.

Every computation runs in the CUDA library; this module converts numpy arrays
to the C ABI's host pointers and status codes to exceptions. There is no CPU
fallback: if libscmd.so has not been built, or no sm_103a GPU is present, the
calls raise.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libscmd.so")

MD_OK, MD_ERR_INVALID, MD_ERR_CUDA, MD_ERR_OOM, MD_ERR_NONFINITE, MD_ERR_TIMEOUT, MD_ERR_STATE = range(7)
MD_PREC_FP64, MD_PREC_MIXED = 0, 1
MD_PATH_AUTO, MD_PATH_ALLPAIRS, MD_PATH_CELLS, MD_PATH_VERLET, MD_PATH_ALLPAIRS_HALF = 0, 1, 2, 3, 4
MD_NVE, MD_LANGEVIN, MD_BERENDSEN = 0, 1, 2
_STATUS = {0: "MD_OK", 1: "MD_ERR_INVALID", 2: "MD_ERR_CUDA", 3: "MD_ERR_OOM", 4: "MD_ERR_NONFINITE",
           5: "MD_ERR_TIMEOUT", 6: "MD_ERR_STATE"}


class md_sc_params(ctypes.Structure):
    _fields_ = [("eps_eV", ctypes.c_double), ("c", ctypes.c_double), ("a_A", ctypes.c_double),
                ("n", ctypes.c_int32), ("m", ctypes.c_int32), ("rcut_A", ctypes.c_double),
                ("cutoff_shift", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class md_config(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int32), ("path", ctypes.c_int32), ("obs_every", ctypes.c_int32),
                ("graph_chunk", ctypes.c_int32), ("tune", ctypes.c_int32), ("obs_capacity", ctypes.c_int32),
                ("tune_cache", ctypes.c_char_p), ("stream", ctypes.c_uint64)]


class md_thermostat(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("reserved", ctypes.c_int32), ("T0_K", ctypes.c_double),
                ("T1_K", ctypes.c_double), ("gamma_per_ps", ctypes.c_double), ("tau_ps", ctypes.c_double),
                ("seed", ctypes.c_uint64)]


class md_obs(ctypes.Structure):
    _fields_ = [("epot_eV", ctypes.c_double), ("ekin_eV", ctypes.c_double), ("etot_eV", ctypes.c_double),
                ("T_K", ctypes.c_double), ("com_A", ctypes.c_double * 3), ("mom", ctypes.c_double * 3),
                ("angmom", ctypes.c_double * 3), ("step", ctypes.c_int64), ("time_fs", ctypes.c_double),
                ("status", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class ScmdError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{_STATUS.get(status, status)}: {message}")
        self.status = status


_lock = threading.Lock()
_lib = None
_DP = ctypes.POINTER(ctypes.c_double)
_VP = ctypes.c_void_p


def lib() -> ctypes.CDLL:
    """Load libscmd.so (built by paper_1210_3559_gb300.build); raises if it is missing."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(f"libscmd.so not built ({LIB_PATH}); run paper_1210_3559_gb300/build.py")
            L = ctypes.CDLL(LIB_PATH)
            i32, i64, u32, u64 = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32, ctypes.c_uint64
            P = ctypes.POINTER
            sig = {
                "md_abi_version": ([], i32),
                "md_create": ([P(md_config), i32, P(i32), _DP, _DP, _DP, P(md_sc_params), P(_VP)], i32),
                "md_energy_forces": ([_VP, _DP, _DP], i32),
                "md_get_density": ([_VP, _DP], i32),
                "md_step": ([_VP, i64, ctypes.c_double, P(md_thermostat)], i32),
                "md_observables": ([_VP, P(md_obs)], i32),
                "md_obs_history": ([_VP, P(md_obs), i32, P(i32)], i32),
                "md_clear_history": ([_VP], i32),
                "md_create_device": ([P(md_config), i32, P(i32), _VP, _VP, _VP, P(md_sc_params), P(_VP)], i32),
                "md_get_state": ([_VP, _DP, _DP, P(i64)], i32),
                "md_get_state_device": ([_VP, _VP, _VP, P(i64)], i32),
                "md_energy_forces_device": ([_VP, _VP, _VP], i32),
                "md_set_state_device": ([_VP, _VP, _VP, i64], i32),
                "md_fp32_peak": ([i32, _DP, _DP], i32),
                "md_set_state": ([_VP, _DP, _DP, i64], i32),
                "md_get_forces": ([_VP, _DP], i32),
                "md_recenter": ([_VP], i32),
                "md_get_launch": ([_VP, i32, P(i32), P(i32), P(i32)], i32),
                "md_set_launch": ([_VP, i32, i32, i32, i32], i32),
                "md_autotune": ([_VP, i32], i32),
                "md_time_passes": ([_VP, i32, _DP, _DP, _DP], i32),
                "md_launch_counts": ([_VP, P(i32), P(i32)], i32),
                "md_get_path": ([_VP, P(i32)], i32),
                "md_last_error": ([_VP], ctypes.c_char_p),
                "md_destroy": ([_VP], None),
                "md_philox4x32_10": ([P(u32), P(u32), i32], i32),
                "md_langevin_normals": ([u64, u32, i64, i32, i32, _DP], i32),
                "md_energy_forces_noalloc": ([_VP, i32, P(md_sc_params), _VP, _VP, u64], i32),
                "md_rdf": ([_VP, ctypes.c_double, ctypes.c_double, i32, P(i64), P(i32)], i32),
                "md_msd_reference": ([_VP, ctypes.c_double], i32),
                "md_msd": ([_VP, _DP, P(i32)], i32),
                "md_cna": ([_VP, ctypes.c_double, P(i32), P(ctypes.c_int8), P(i32)], i32),
            }
            for name, (args, res) in sig.items():
                f = getattr(L, name)
                f.argtypes = args
                f.restype = res
            _lib = L
    return _lib


def exported_symbols():
    return ["md_abi_version", "md_create", "md_energy_forces", "md_get_density", "md_step", "md_observables",
            "md_obs_history", "md_clear_history", "md_get_state", "md_set_state", "md_get_forces", "md_recenter",
            "md_get_launch", "md_set_launch", "md_autotune", "md_time_passes", "md_launch_counts", "md_get_path",
            "md_last_error", "md_destroy", "md_philox4x32_10", "md_langevin_normals",
            "md_energy_forces_noalloc", "md_rdf", "md_msd_reference", "md_msd", "md_cna", "md_create_device",
            "md_get_state_device", "md_set_state_device", "md_fp32_peak", "md_energy_forces_device"]


def md_abi_version() -> int:
    return int(lib().md_abi_version())


def md_last_error(ctx=None) -> str:
    s = lib().md_last_error(_h(ctx))
    return s.decode() if s else ""


def _check(status: int, ctx=None):
    if status != MD_OK:
        raise ScmdError(status, md_last_error(ctx))


def _arr(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim == 1 and a.size % 3 == 0:
        a = a.reshape(-1, 3)
    if n is not None and a.shape != (n, 3):
        raise ValueError(f"expected shape ({n}, 3), got {a.shape}")
    return a


def sc_params(eps=1.5707e-2, c=39.432, a=3.52, n=9, m=6, rcut=0.0, shift=False) -> md_sc_params:
    """Sutton-Chen parameters; defaults are the paper's Ni set (Sec. II A). rcut > 0 truncates the
    pair terms at rcut; shift=True also shifts them by their value there (continuous energy)."""
    return md_sc_params(float(eps), float(c), float(a), int(n), int(m), float(rcut), 1 if shift else 0, 0)


def config(precision=MD_PREC_MIXED, path=MD_PATH_AUTO, obs_every=0, graph_chunk=0, tune=0, obs_capacity=0,
           tune_cache=None, stream=0) -> md_config:
    return md_config(int(precision), int(path), int(obs_every), int(graph_chunk), int(tune), int(obs_capacity),
                     tune_cache.encode() if tune_cache else None, int(stream))


def thermostat(kind=MD_NVE, T0=0.0, T1=None, gamma_per_ps=1.0, tau_ps=0.1, seed=0) -> md_thermostat:
    return md_thermostat(int(kind), 0, float(T0), float(T0 if T1 is None else T1), float(gamma_per_ps),
                         float(tau_ps), int(seed))


class Context:
    """Owner of one md_ctx*: holds the cluster sizes so results come back with their shapes."""

    def __init__(self, handle, sizes):
        self.handle = handle
        self.sizes = np.asarray(sizes, dtype=np.int32)
        self.ntot = int(self.sizes.sum())
        self.n_clusters = len(self.sizes)

    def __del__(self):
        try:
            md_destroy(self)
        except Exception:
            pass


def _h(ctx):
    return ctx.handle if isinstance(ctx, Context) else ctx


def md_create(cfg: md_config, sizes, pos, vel, mass, params: md_sc_params | None = None) -> Context:
    sizes = np.ascontiguousarray(sizes, dtype=np.int32)
    ntot = int(sizes.sum())
    pos = _arr(pos, ntot)
    vel = None if vel is None else _arr(vel, ntot)
    mass = np.ascontiguousarray(mass, dtype=np.float64)
    if mass.shape != (ntot,):
        raise ValueError("mass must have shape (Ntot,)")
    params = params or sc_params()
    out = _VP()
    st = lib().md_create(ctypes.byref(cfg), len(sizes), sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                         pos.ctypes.data_as(_DP), None if vel is None else vel.ctypes.data_as(_DP),
                         mass.ctypes.data_as(_DP), ctypes.byref(params), ctypes.byref(out))
    _check(st)
    return Context(out.value, sizes)


def _dptr(x) -> int:
    """Device address of a CUDA tensor (anything with data_ptr()) or a raw integer address; None -> 0."""
    if x is None:
        return 0
    return int(x.data_ptr()) if hasattr(x, "data_ptr") else int(x)


def md_create_device(cfg: md_config, sizes, pos_dev, vel_dev, mass_dev, params: md_sc_params | None = None) -> Context:
    """md_create from caller-owned device arrays: pos_dev/vel_dev [Ntot][3] float64, mass_dev [Ntot]
    float64 (CUDA tensors or raw device addresses; vel_dev may be None). The caller keeps ownership."""
    sizes = np.ascontiguousarray(sizes, dtype=np.int32)
    params = params or sc_params()
    out = _VP()
    st = lib().md_create_device(ctypes.byref(cfg), len(sizes), sizes.ctypes.data_as(ctypes.POINTER(ctypes.c_int32)),
                                _dptr(pos_dev) or None, _dptr(vel_dev) or None, _dptr(mass_dev) or None,
                                ctypes.byref(params), ctypes.byref(out))
    _check(st)
    return Context(out.value, sizes)


def md_get_state_device(ctx: Context, pos_dev, vel_dev) -> int:
    """Copy positions and/or velocities into caller-owned device arrays [Ntot][3] float64 (either may
    be None); returns the step counter."""
    step = ctypes.c_int64(0)
    _check(lib().md_get_state_device(ctx.handle, _dptr(pos_dev) or None, _dptr(vel_dev) or None, ctypes.byref(step)),
           ctx.handle)
    return step.value


def md_energy_forces_device(ctx: Context, epot_dev, forces_dev):
    """Energies [n_clusters] and forces [Ntot][3] (float64) into caller-owned device arrays (either may be None)."""
    _check(lib().md_energy_forces_device(ctx.handle, _dptr(epot_dev) or None, _dptr(forces_dev) or None), ctx.handle)


def md_set_state_device(ctx: Context, pos_dev, vel_dev, step: int):
    _check(lib().md_set_state_device(ctx.handle, _dptr(pos_dev) or None, _dptr(vel_dev) or None, int(step)),
           ctx.handle)


def md_fp32_peak(reps: int = 20):
    """Measured FP32 lane-operation rate of the device (FFMA chains on every SM) and its clock-derived
    ceiling: returns (measured, derived) in lane-ops/s."""
    meas = ctypes.c_double(0.0)
    derived = ctypes.c_double(0.0)
    _check(lib().md_fp32_peak(int(reps), ctypes.byref(meas), ctypes.byref(derived)))
    return meas.value, derived.value


def md_destroy(ctx: Context):
    if ctx.handle:
        lib().md_destroy(ctx.handle)
        ctx.handle = None


def md_energy_forces(ctx: Context, forces: bool = True):
    e = np.zeros(ctx.n_clusters)
    F = np.zeros((ctx.ntot, 3)) if forces else None
    _check(lib().md_energy_forces(ctx.handle, e.ctypes.data_as(_DP), F.ctypes.data_as(_DP) if forces else None),
           ctx.handle)
    return e, F


def md_get_density(ctx: Context) -> np.ndarray:
    rho = np.zeros(ctx.ntot)
    _check(lib().md_get_density(ctx.handle, rho.ctypes.data_as(_DP)), ctx.handle)
    return rho


def md_get_forces(ctx: Context) -> np.ndarray:
    F = np.zeros((ctx.ntot, 3))
    _check(lib().md_get_forces(ctx.handle, F.ctypes.data_as(_DP)), ctx.handle)
    return F


def md_step(ctx: Context, nsteps: int, dt_fs: float, th: md_thermostat | None = None):
    _check(lib().md_step(ctx.handle, int(nsteps), float(dt_fs), ctypes.byref(th) if th is not None else None),
           ctx.handle)


def _obs_dict(o: md_obs) -> dict:
    return dict(epot=o.epot_eV, ekin=o.ekin_eV, etot=o.etot_eV, T=o.T_K, com=np.array(o.com_A[:]),
                mom=np.array(o.mom[:]), angmom=np.array(o.angmom[:]), step=o.step, time_fs=o.time_fs,
                status=o.status)


def md_observables(ctx: Context) -> list:
    arr = (md_obs * ctx.n_clusters)()
    _check(lib().md_observables(ctx.handle, arr), ctx.handle)
    return [_obs_dict(o) for o in arr]


def md_obs_history(ctx: Context, max_samples: int = 1 << 20) -> list:
    """List of samples, each a list (one dict per cluster)."""
    n = ctypes.c_int32(0)
    cap = max(0, int(max_samples))
    arr = (md_obs * (max(1, cap) * ctx.n_clusters))()
    _check(lib().md_obs_history(ctx.handle, arr, cap, ctypes.byref(n)), ctx.handle)
    B = ctx.n_clusters
    return [[_obs_dict(arr[s * B + b]) for b in range(B)] for s in range(n.value)]


def md_clear_history(ctx: Context):
    _check(lib().md_clear_history(ctx.handle), ctx.handle)


def md_get_state(ctx: Context):
    pos = np.zeros((ctx.ntot, 3))
    vel = np.zeros((ctx.ntot, 3))
    step = ctypes.c_int64(0)
    _check(lib().md_get_state(ctx.handle, pos.ctypes.data_as(_DP), vel.ctypes.data_as(_DP), ctypes.byref(step)),
           ctx.handle)
    return pos, vel, step.value


def md_set_state(ctx: Context, pos, vel, step: int):
    pos = _arr(pos, ctx.ntot)
    vel = _arr(vel, ctx.ntot)
    _check(lib().md_set_state(ctx.handle, pos.ctypes.data_as(_DP), vel.ctypes.data_as(_DP), int(step)), ctx.handle)


def md_recenter(ctx: Context):
    _check(lib().md_recenter(ctx.handle), ctx.handle)


def md_get_launch(ctx: Context, which: int):
    v = [ctypes.c_int32() for _ in range(3)]
    _check(lib().md_get_launch(ctx.handle, int(which), *[ctypes.byref(x) for x in v]), ctx.handle)
    return tuple(x.value for x in v)


def md_set_launch(ctx: Context, which: int, ipt: int, warps: int, cluster: int):
    _check(lib().md_set_launch(ctx.handle, int(which), int(ipt), int(warps), int(cluster)), ctx.handle)


def md_autotune(ctx: Context, reps: int = 10):
    _check(lib().md_autotune(ctx.handle, int(reps)), ctx.handle)


def md_time_passes(ctx: Context, reps: int = 20):
    d, f, p = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
    _check(lib().md_time_passes(ctx.handle, int(reps), ctypes.byref(d), ctypes.byref(f), ctypes.byref(p)),
           ctx.handle)
    return d.value, f.value, p.value


def md_launch_counts(ctx: Context):
    a, b = ctypes.c_int32(), ctypes.c_int32()
    _check(lib().md_launch_counts(ctx.handle, ctypes.byref(a), ctypes.byref(b)), ctx.handle)
    return a.value, b.value


def md_get_path(ctx: Context) -> int:
    p = ctypes.c_int32()
    _check(lib().md_get_path(ctx.handle, ctypes.byref(p)), ctx.handle)
    return p.value


CNA_OTHER, CNA_FCC, CNA_HCP, CNA_ICO = 0, 1, 2, 3


def md_rdf(ctx: Context, r_core_A: float, bin_A: float, nbins: int):
    """(counts[B][nbins] int64, n_core[B]): pair distances from each cluster's central atoms."""
    counts = np.zeros((ctx.n_clusters, int(nbins)), dtype=np.int64)
    nc = np.zeros(ctx.n_clusters, dtype=np.int32)
    _check(lib().md_rdf(ctx.handle, float(r_core_A), float(bin_A), int(nbins),
                        counts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)),
                        nc.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))), ctx.handle)
    return counts, nc


def md_msd_reference(ctx: Context, r_core_A: float = 0.0):
    _check(lib().md_msd_reference(ctx.handle, float(r_core_A)), ctx.handle)


def md_msd(ctx: Context):
    """(msd[B] in A^2, atoms averaged[B]) since md_msd_reference, centre-of-mass motion removed."""
    v = np.zeros(ctx.n_clusters)
    n = np.zeros(ctx.n_clusters, dtype=np.int32)
    _check(lib().md_msd(ctx.handle, v.ctypes.data_as(_DP), n.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))),
           ctx.handle)
    return v, n


def md_cna(ctx: Context, r_nb_A: float = 3.0, per_atom: bool = False):
    """counts[B][4] (other, fcc, hcp, icosahedral); with per_atom also (class[Ntot] int8, capped[B])."""
    counts = np.zeros((ctx.n_clusters, 4), dtype=np.int32)
    capped = np.zeros(ctx.n_clusters, dtype=np.int32)
    cls = np.zeros(ctx.ntot, dtype=np.int8) if per_atom else None
    I32 = ctypes.POINTER(ctypes.c_int32)
    _check(lib().md_cna(ctx.handle, float(r_nb_A), counts.ctypes.data_as(I32),
                        cls.ctypes.data_as(ctypes.POINTER(ctypes.c_int8)) if per_atom else None,
                        capped.ctypes.data_as(I32)), ctx.handle)
    return (counts, cls, capped) if per_atom else counts


def md_philox4x32_10(words) -> np.ndarray:
    """words: array (count, 6) of (ctr0..ctr3, key0, key1) -> (count, 4) outputs from the GPU kernel."""
    w = np.ascontiguousarray(words, dtype=np.uint32).reshape(-1, 6)
    out = np.zeros((len(w), 4), dtype=np.uint32)
    P = ctypes.POINTER(ctypes.c_uint32)
    _check(lib().md_philox4x32_10(w.ctypes.data_as(P), out.ctypes.data_as(P), len(w)))
    return out


def md_langevin_normals(seed: int, cluster: int, step: int, n_atoms: int, precision: int = MD_PREC_MIXED):
    out = np.zeros((int(n_atoms), 3))
    _check(lib().md_langevin_normals(int(seed), int(cluster), int(step), int(n_atoms), int(precision),
                                     out.ctypes.data_as(_DP)))
    return out


def md_energy_forces_noalloc(pos_ptr: int, n_atoms: int, params: md_sc_params | None, forces_ptr: int,
                             epot_ptr: int, stream: int = 0):
    """Energy and forces of one cluster from caller-owned device buffers (raw device addresses),
    for callers that cannot allocate device memory; the library allocates nothing either.
    Queued on `stream`: synchronise it before reading the outputs."""
    params = params or sc_params()
    _check(lib().md_energy_forces_noalloc(int(pos_ptr), int(n_atoms), ctypes.byref(params), int(forces_ptr),
                                          int(epot_ptr), int(stream)))
