"""ctypes binding of libsph (include/sph.h).

Same names as the C ABI, argument marshalling only: every step of the path runs in the library's CUDA kernels.
Device buffers may be passed as torch CUDA tensors (their data pointer is used) or as raw integer addresses.
Each call raises SphError when the library returns a status other than SPH_OK.  Loading fails loudly when the
compiled library is missing; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# SPH_CHECKED=1 in the environment loads the checked build (index checks on the device, build(checked=True))
CHECKED = os.environ.get("SPH_CHECKED", "") == "1"
LIB_PATH = os.path.join(_HERE, "_build_checked" if CHECKED else "_build", "libsph.so")

# ---- constants (mirror include/sph.h) ----
SPH_OK, SPH_E_INVAL, SPH_E_NOMEM, SPH_E_CUDA, SPH_E_DEVICE, SPH_E_TIMEOUT, SPH_E_NOTCONV, SPH_E_STATE = range(8)
SPH_F64, SPH_F32 = 0, 1
(SPH_X, SPH_V, SPH_A, SPH_MASS, SPH_H, SPH_RHO, SPH_P, SPH_U, SPH_DUDT, SPH_CS, SPH_NNB, SPH_DIVV, SPH_CURLV,
 SPH_OMEGA, SPH_VSIG) = range(15)
SPH_NFIELDS = 15
FIELD_NAMES = ("x", "v", "a", "mass", "h", "rho", "P", "u", "dudt", "cs", "nnb", "divv", "curlv", "omega", "vsig")
NCOMP = (3, 3, 3, 1, 1, 1, 1, 1, 1, 1, 1, 1, 3, 1, 1)
SPH_KERNEL_M4, SPH_KERNEL_M5 = 0, 1
SPH_SCHEME_MINIMAL, SPH_SCHEME_EXTENDED = 0, 1


def SPH_BIT(f):
    return 1 << f


SPH_DENSITY_IN = SPH_BIT(SPH_X) | SPH_BIT(SPH_MASS) | SPH_BIT(SPH_H) | SPH_BIT(SPH_U)
SPH_DENSITY_OUT = SPH_BIT(SPH_RHO) | SPH_BIT(SPH_P) | SPH_BIT(SPH_CS)
SPH_FORCE_IN = (SPH_BIT(SPH_X) | SPH_BIT(SPH_V) | SPH_BIT(SPH_MASS) | SPH_BIT(SPH_H) | SPH_BIT(SPH_RHO)
                | SPH_BIT(SPH_P) | SPH_BIT(SPH_CS))
SPH_FORCE_OUT = SPH_BIT(SPH_A) | SPH_BIT(SPH_DUDT)
SPH_DENSITY_IN_EXT = SPH_DENSITY_IN | SPH_BIT(SPH_V)
SPH_DENSITY_OUT_EXT = (SPH_DENSITY_OUT | SPH_BIT(SPH_NNB) | SPH_BIT(SPH_DIVV) | SPH_BIT(SPH_CURLV)
                       | SPH_BIT(SPH_OMEGA))
SPH_FORCE_IN_EXT = SPH_FORCE_IN | SPH_BIT(SPH_OMEGA) | SPH_BIT(SPH_DIVV) | SPH_BIT(SPH_CURLV)
SPH_FORCE_OUT_EXT = SPH_FORCE_OUT | SPH_BIT(SPH_VSIG)
SPH_ALL_FIELDS = (1 << SPH_NFIELDS) - 1
SPH_DEV_POS_RANGE, SPH_DEV_H_TOO_BIG, SPH_DEV_NONFINITE, SPH_DEV_TIMEOUT = 0x1, 0x2, 0x4, 0x8
SPH_DEV_NOTCONV = 0x10
SPH_DEV_BOUNDS = 0x20  # checked build only
SPH_DEV_MAGNITUDE = 0x40  # FP64 views: h outside [2^-50, 2^50) or h^2 rho outside [2^-105, 2^105)
(SPH_PH_BIN, SPH_PH_GATHER, SPH_PH_DENSITY_PREP, SPH_PH_DENSITY, SPH_PH_SCATTER, SPH_PH_FORCE_PREP, SPH_PH_FORCE,
 SPH_PH_REDUCE, SPH_PH_KDK) = range(9)
SPH_NPHASES = 9
SPH_KDK_PREDICT, SPH_KDK_CONTINUE = 0x1, 0x2
SPH_BIN_STATIC_MAX_PARTICLES = 262144
SPH_BIN_STATIC_MAX_CELLS = 65536
PHASE_NAMES = ("bin", "gather", "density_prep", "density", "scatter", "force_prep", "force", "reduce", "kdk")


class sph_layout(ctypes.Structure):
    _fields_ = [("stride", ctypes.c_int64), ("off", ctypes.c_int32 * SPH_NFIELDS)]


class sph_domain(ctypes.Structure):
    _fields_ = [("box", ctypes.c_double * 3), ("ncell", ctypes.c_int32 * 3), ("periodic", ctypes.c_int32)]


class sph_params(ctypes.Structure):
    _fields_ = [("gamma", ctypes.c_double), ("alpha", ctypes.c_double), ("beta", ctypes.c_double),
                ("eps", ctypes.c_double), ("kernel", ctypes.c_int32), ("scheme", ctypes.c_int32)]


class SphError(RuntimeError):
    def __init__(self, fn, status):
        self.status = int(status)
        super().__init__(f"{fn}: {strerror(status)} ({status})")


_lib = None
_VP = ctypes.c_void_p
_I32 = ctypes.c_int32
_I64 = ctypes.c_int64
_SIGS = {
    "sph_view_create": [ctypes.POINTER(sph_layout), ctypes.c_int, _I64, ctypes.POINTER(sph_domain), _VP,
                        ctypes.POINTER(_VP)],
    "sph_view_destroy": [_VP],
    "sph_bin": [_VP, _VP, _I64],
    "sph_aos_to_soa": [_VP, _VP, _I64, ctypes.c_uint32],
    "sph_density": [_VP, ctypes.POINTER(sph_params)],
    "sph_force": [_VP, ctypes.POINTER(sph_params)],
    "sph_soa_to_aos": [_VP, _VP, _I64, ctypes.c_uint32],
    "sph_step": [_VP, _VP, _I64, ctypes.POINTER(sph_params), ctypes.c_double, _I32, ctypes.POINTER(ctypes.c_double)],
    "sph_step_host": [_VP, _VP, _I64, ctypes.POINTER(sph_params), ctypes.c_double, _I32,
                      ctypes.POINTER(ctypes.c_double)],
    "sph_reduce": [_VP, ctypes.POINTER(ctypes.c_double)],
    "sph_view_sync": [_VP],
    "sph_view_status": [_VP, ctypes.POINTER(ctypes.c_uint32), _I32],
    "sph_view_soa": [_VP, _I32, _I32, ctypes.POINTER(_VP)],
    "sph_view_index": [_VP, _I32, ctypes.POINTER(_VP)],
    "sph_view_export": [_VP, _I32, _I32, _VP, _I64],
    "sph_view_export_index": [_VP, _I32, _VP, _I64],
    "sph_view_info": [_VP, ctypes.POINTER(_I64), ctypes.POINTER(_I64)],
    "sph_pair_counts": [_VP, ctypes.POINTER(ctypes.c_uint64), _I32],
    "sph_view_timing": [_VP, _I32],
    "sph_view_phase_times": [_VP, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_I64), _I32],
    "sph_probe_fma_rate": [_I32, ctypes.POINTER(ctypes.c_double)],
    "sph_patches_create": [ctypes.POINTER(sph_layout), ctypes.c_int, _I64, _I32, ctypes.POINTER(ctypes.c_double), _I32,
                           _VP, ctypes.POINTER(_VP)],
    "sph_patches_bin": [_VP, _VP, _I64, _VP, _I32],
    "sph_patches_step": [_VP, _VP, _I64, _VP, _I32, ctypes.POINTER(sph_params), ctypes.c_double, _I32,
                         ctypes.POINTER(ctypes.c_double)],
    "sph_step_graph": [_VP, _VP, _I64, ctypes.POINTER(sph_params), ctypes.c_double, _I32],
    "sph_patches_step_graph": [_VP, _VP, _I64, _VP, _I32, ctypes.POINTER(sph_params), ctypes.c_double, _I32],
    "sph_view_set_integrator": [_VP, _I32],
    "sph_view_set_tiles": [_VP, _I32, _I32],
    "sph_view_set_union": [_VP, _I32],
    "sph_view_set_host_direct": [_VP, _I32],
    "sph_view_set_warps": [_VP, _I32, _I32],
    "sph_view_get_tuning": [_VP, _VP],
    "sph_density_h": [_VP, _VP, ctypes.c_double, ctypes.c_double, _I32, _VP, _VP],
    "sph_view_set_h_iteration": [_VP, ctypes.c_double, ctypes.c_double, _I32],
    "sph_view_h_rounds": [_VP, _VP, _VP],
    "sph_autotune": [_VP, _VP, _I64, ctypes.POINTER(sph_params), ctypes.POINTER(_I32), ctypes.POINTER(ctypes.c_float)],
    "sph_bin_static": [ctypes.POINTER(sph_layout), ctypes.POINTER(sph_domain), _VP, _I64, _VP, _VP, _VP, _VP, _VP],
    "sph_build_info": [ctypes.POINTER(ctypes.c_int32)],
}
EXPORTED = tuple(_SIGS) + ("sph_strerror",)


def lib():
    """Load libsph.so (built in-tree by paper_2502_16517_gb300.build); raises if it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libsph is not built ({LIB_PATH} missing): run paper_2502_16517_gb300.build.build()")
        L = ctypes.CDLL(LIB_PATH)
        for name, args in _SIGS.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int
        L.sph_strerror.argtypes = [ctypes.c_int]
        L.sph_strerror.restype = ctypes.c_char_p
        _lib = L
    return _lib


def strerror(status):
    return lib().sph_strerror(int(status)).decode()


def _check(fn, status):
    if status != SPH_OK:
        raise SphError(fn, status)


def _addr(x):
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(type(x))


# ---- struct helpers ----
def make_layout(layout: dict) -> sph_layout:
    """sph_layout from {"stride": s, "offsets": {name: byte offset}}; absent members get -1."""
    L = sph_layout()
    L.stride = int(layout["stride"])
    for f, name in enumerate(FIELD_NAMES):
        L.off[f] = int(layout["offsets"].get(name, -1))
    return L


def make_domain(box, ncell, periodic=True) -> sph_domain:
    D = sph_domain()
    for a in range(3):
        D.box[a] = float(box[a])
        D.ncell[a] = int(ncell[a])
    D.periodic = 1 if periodic else 0
    return D


def make_params(p: dict) -> sph_params:
    """sph_params from a dict; "kernel" and "scheme" default to the cubic spline and the minimal set."""
    return sph_params(float(p["gamma"]), float(p["alpha"]), float(p["beta"]), float(p["eps"]),
                      int(p.get("kernel", SPH_KERNEL_M4)), int(p.get("scheme", SPH_SCHEME_MINIMAL)))


# ---- the C ABI ----
def sph_view_create(layout, prec, n_max, domain, stream=None):
    """Returns the view handle (an int).  layout/domain may be dicts/tuples or ctypes structs."""
    L = layout if isinstance(layout, sph_layout) else make_layout(layout)
    D = domain if isinstance(domain, sph_domain) else make_domain(*domain)
    out = _VP()
    st = _addr(stream) if stream is not None else None
    _check("sph_view_create", lib().sph_view_create(ctypes.byref(L), int(prec), int(n_max), ctypes.byref(D),
                                                    st, ctypes.byref(out)))
    return out.value


def sph_view_destroy(view):
    _check("sph_view_destroy", lib().sph_view_destroy(view))


def sph_bin(view, aos_dev, n):
    _check("sph_bin", lib().sph_bin(view, _addr(aos_dev), int(n)))


def sph_aos_to_soa(view, aos_dev, n, in_mask):
    _check("sph_aos_to_soa", lib().sph_aos_to_soa(view, _addr(aos_dev), int(n), int(in_mask)))


def sph_density(view, params):
    P = params if isinstance(params, sph_params) else make_params(params)
    _check("sph_density", lib().sph_density(view, ctypes.byref(P)))


def sph_force(view, params):
    P = params if isinstance(params, sph_params) else make_params(params)
    _check("sph_force", lib().sph_force(view, ctypes.byref(P)))


def sph_soa_to_aos(view, aos_dev, n, out_mask):
    _check("sph_soa_to_aos", lib().sph_soa_to_aos(view, _addr(aos_dev), int(n), int(out_mask)))


def sph_step(view, aos_dev, n, params, dt=0.0, nsteps=0, want_stats=False):
    P = params if isinstance(params, sph_params) else make_params(params)
    stats = (ctypes.c_double * 8)() if want_stats else None
    _check("sph_step", lib().sph_step(view, _addr(aos_dev), int(n), ctypes.byref(P), float(dt), int(nsteps),
                                      stats))
    return np.array(stats[:]) if want_stats else None


def sph_step_host(view, aos_host, n, params, dt=0.0, nsteps=0, want_stats=False):
    P = params if isinstance(params, sph_params) else make_params(params)
    stats = (ctypes.c_double * 8)() if want_stats else None
    _check("sph_step_host", lib().sph_step_host(view, _addr(aos_host), int(n), ctypes.byref(P), float(dt),
                                                int(nsteps), stats))
    return np.array(stats[:]) if want_stats else None


def sph_reduce(view):
    out = (ctypes.c_double * 8)()
    _check("sph_reduce", lib().sph_reduce(view, out))
    return np.array(out[:])


def sph_view_sync(view):
    _check("sph_view_sync", lib().sph_view_sync(view))


def sph_view_status(view, clear=False):
    bits = ctypes.c_uint32()
    _check("sph_view_status", lib().sph_view_status(view, ctypes.byref(bits), 1 if clear else 0))
    return bits.value


def sph_view_soa(view, field, comp=0):
    p = _VP()
    _check("sph_view_soa", lib().sph_view_soa(view, int(field), int(comp), ctypes.byref(p)))
    return p.value


def sph_view_index(view, which):
    p = _VP()
    _check("sph_view_index", lib().sph_view_index(view, int(which), ctypes.byref(p)))
    return p.value


def sph_view_export(view, field, comp, count, prec):
    """SoA member `field`/`comp` as a host numpy array of `count` elements (float64 or float32 by prec)."""
    out = np.empty(int(count), np.float64 if prec == SPH_F64 else np.float32)
    _check("sph_view_export", lib().sph_view_export(view, int(field), int(comp), out.ctypes.data, int(count)))
    return out


def sph_view_export_index(view, which, count):
    out = np.empty(int(count), np.int32)
    _check("sph_view_export_index", lib().sph_view_export_index(view, int(which), out.ctypes.data, int(count)))
    return out


def sph_view_info(view):
    n, nc = _I64(), _I64()
    _check("sph_view_info", lib().sph_view_info(view, ctypes.byref(n), ctypes.byref(nc)))
    return n.value, nc.value


def sph_pair_counts(view, reset=False):
    out = (ctypes.c_uint64 * 4)()
    _check("sph_pair_counts", lib().sph_pair_counts(view, out, 1 if reset else 0))
    return [int(v) for v in out]


def sph_view_timing(view, enable=True):
    _check("sph_view_timing", lib().sph_view_timing(view, 1 if enable else 0))


def sph_view_phase_times(view, reset=False):
    """(ms per phase, kernel launches per phase) as numpy arrays of SPH_NPHASES entries."""
    ms = (ctypes.c_double * SPH_NPHASES)()
    nl = (_I64 * SPH_NPHASES)()
    _check("sph_view_phase_times", lib().sph_view_phase_times(view, ms, nl, 1 if reset else 0))
    return np.array(ms[:]), np.array(nl[:], np.int64)


def sph_bin_static(layout, domain, aos_dev, n, perm_dev, cell_start_dev, cell_of_slot_dev, status_dev=None,
                   stream=None):
    """Cell bucketing into caller-owned device arrays with no allocation (see include/sph.h)."""
    L = layout if isinstance(layout, sph_layout) else make_layout(layout)
    D = domain if isinstance(domain, sph_domain) else make_domain(*domain)
    st = _addr(stream) if stream is not None else None
    _check("sph_bin_static", lib().sph_bin_static(ctypes.byref(L), ctypes.byref(D), _addr(aos_dev), int(n),
                                                  _addr(perm_dev), _addr(cell_start_dev), _addr(cell_of_slot_dev),
                                                  _addr(status_dev), st))


def sph_probe_fma_rate(prec):
    """Measured FMA throughput of the current device in flops/s (FP64 for SPH_F64, FP32 for SPH_F32)."""
    out = ctypes.c_double()
    _check("sph_probe_fma_rate", lib().sph_probe_fma_rate(int(prec), ctypes.byref(out)))
    return out.value


def sph_patches_create(layout, prec, n_max, npatch_max, patch_box, ncell_cap=8, stream=None):
    """View over independent open-box patches; returns the handle."""
    L = layout if isinstance(layout, sph_layout) else make_layout(layout)
    box = (ctypes.c_double * 3)(*[float(b) for b in patch_box])
    out = _VP()
    st = _addr(stream) if stream is not None else None
    _check("sph_patches_create", lib().sph_patches_create(ctypes.byref(L), int(prec), int(n_max), int(npatch_max), box,
                                                          int(ncell_cap), st, ctypes.byref(out)))
    return out.value


def sph_patches_bin(view, aos_dev, n, patch_start_dev, npatch):
    _check("sph_patches_bin", lib().sph_patches_bin(view, _addr(aos_dev), int(n), _addr(patch_start_dev), int(npatch)))


def sph_patches_step(view, aos_dev, n, patch_start_dev, npatch, params, dt=0.0, nsteps=0, want_stats=False):
    P = params if isinstance(params, sph_params) else make_params(params)
    stats = (ctypes.c_double * 8)() if want_stats else None
    _check("sph_patches_step", lib().sph_patches_step(view, _addr(aos_dev), int(n), _addr(patch_start_dev), int(npatch),
                                                      ctypes.byref(P), float(dt), int(nsteps), stats))
    return np.array(stats[:]) if want_stats else None


def sph_step_graph(view, aos_dev, n, params, dt=0.0, nsteps=0):
    P = params if isinstance(params, sph_params) else make_params(params)
    _check("sph_step_graph", lib().sph_step_graph(view, _addr(aos_dev), int(n), ctypes.byref(P), float(dt), int(nsteps)))


def sph_patches_step_graph(view, aos_dev, n, patch_start_dev, npatch, params, dt=0.0, nsteps=0):
    P = params if isinstance(params, sph_params) else make_params(params)
    _check("sph_patches_step_graph", lib().sph_patches_step_graph(view, _addr(aos_dev), int(n), _addr(patch_start_dev),
                                                                  int(npatch), ctypes.byref(P), float(dt),
                                                                  int(nsteps)))


def sph_view_set_integrator(view, flags=SPH_KDK_PREDICT):
    """Leapfrog options: SPH_KDK_PREDICT (default) and/or SPH_KDK_CONTINUE."""
    _check("sph_view_set_integrator", lib().sph_view_set_integrator(view, int(flags)))


def sph_density_h(view, params, eta=1.2, tol=1e-6, max_iter=30, allow_unconverged=False):
    """Returns (rounds, unconverged).  Raises SphError(SPH_E_NOTCONV) if particles are left unconverged, unless
    allow_unconverged."""
    P = params if isinstance(params, sph_params) else make_params(params)
    rounds, left = ctypes.c_int32(), ctypes.c_int64()
    st = lib().sph_density_h(view, ctypes.byref(P), float(eta), float(tol), int(max_iter), ctypes.byref(rounds),
                             ctypes.byref(left))
    if not (st == SPH_OK or (allow_unconverged and st == SPH_E_NOTCONV)):
        raise SphError("sph_density_h", st)
    return rounds.value, left.value


def sph_view_set_h_iteration(view, eta=1.2, tol=1e-6, max_iter=30):
    _check("sph_view_set_h_iteration", lib().sph_view_set_h_iteration(view, float(eta), float(tol), int(max_iter)))


def sph_view_h_rounds(view, allow_unconverged=True):
    rounds, left = ctypes.c_int32(), ctypes.c_int64()
    st = lib().sph_view_h_rounds(view, ctypes.byref(rounds), ctypes.byref(left))
    if not (st == SPH_OK or (allow_unconverged and st == SPH_E_NOTCONV)):
        raise SphError("sph_view_h_rounds", st)
    return rounds.value, left.value


def sph_view_set_warps(view, warps_density, warps_force):
    _check("sph_view_set_warps", lib().sph_view_set_warps(view, int(warps_density), int(warps_force)))


def sph_view_get_tuning(view):
    """(tile_density, tile_force, warps_density, warps_force) of the view."""
    out = (ctypes.c_int32 * 4)()
    _check("sph_view_get_tuning", lib().sph_view_get_tuning(view, out))
    return tuple(int(x) for x in out)


def sph_view_set_union(view, on=True):
    _check("sph_view_set_union", lib().sph_view_set_union(view, 1 if on else 0))


def sph_view_set_host_direct(view, on=True):
    _check("sph_view_set_host_direct", lib().sph_view_set_host_direct(view, int(on)))


def sph_view_set_tiles(view, tile_density, tile_force):
    _check("sph_view_set_tiles", lib().sph_view_set_tiles(view, int(tile_density), int(tile_force)))


def sph_autotune(view, aos_dev, n, params):
    """Returns ((tile_density, tile_force), (ms_density, ms_force))."""
    P = params if isinstance(params, sph_params) else make_params(params)
    chosen = (_I32 * 2)()
    ms = (ctypes.c_float * 2)()
    _check("sph_autotune", lib().sph_autotune(view, _addr(aos_dev), int(n), ctypes.byref(P), chosen, ms))
    return (chosen[0], chosen[1]), (ms[0], ms[1])


def sph_build_info():
    """1 if the loaded library is the checked build (compiled with -DSPH_CHECKED), else 0."""
    v = ctypes.c_int32(0)
    _check("sph_build_info", lib().sph_build_info(ctypes.byref(v)))
    return int(v.value)
