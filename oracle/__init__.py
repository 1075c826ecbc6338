"""FP64 CPU oracle for the SPH view path: test infrastructure only.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg may import this package.  The
CUDA library and its Python binding never import it, and it imports nothing from them.  It wraps the plain C
restatement in ``sph_oracle.c`` (brute-force all-pairs sums, no cell list) with ctypes and composes its pieces
into whole passes.

Each function names the passage of the paper (arXiv 2502.16517) it follows.  Where the paper fixes no formula,
the C file names the textbook form that is used.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sph_oracle.c")
_LIB_PATH = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

_D = ctypes.POINTER(ctypes.c_double)
_F = ctypes.POINTER(ctypes.c_float)
_I32 = ctypes.POINTER(ctypes.c_int32)
_I64 = ctypes.POINTER(ctypes.c_int64)
_U8 = ctypes.POINTER(ctypes.c_uint8)


def build(force: bool = False) -> str:
    """Compile sph_oracle.c into a shared library (gcc, no FP contraction, so every op rounds as written)."""
    os.makedirs(os.path.dirname(_LIB_PATH), exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                        "-o", tmp, _SRC, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            lib = ctypes.CDLL(path)
            i64, i32, dbl, vp = ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_void_p
            sig = {
                "or_w": (dbl, [dbl, dbl]),
                "or_dwdr": (dbl, [dbl, dbl]),
                "or_w_array": (None, [i64, _D, _D, _D]),
                "or_dwdr_array": (None, [i64, _D, _D, _D]),
                "or_density": (None, [i64, _D, _D, _D, _D, ctypes.c_int, i64, _I64, _D]),
                "or_eos": (None, [i64, _D, _D, dbl, _D, _D]),
                "or_force": (None, [i64, _D, _D, _D, _D, _D, _D, _D, _D, ctypes.c_int, dbl, dbl, dbl, i64,
                                    _I64, _D, _D]),
                "or_neighbours": (i64, [i64, _D, _D, _D, ctypes.c_int, i64, dbl, i64, _I64]),
                "or_bin": (i64, [i64, _D, _D, _I32, _I32, _I32, _I32, _I32]),
                "or_bin_patches": (i64, [i64, _D, _D, _I64, i32, _D, i32, _I32, _I32, _I32, _I32, _I32, _I32]),
                "or_gather_pos_f32_patches": (None, [_U8, i64, i64, _I32, i64, _I32, _I32, _I32, i32, _D, _F]),
                "or_gather_f64": (None, [_U8, i64, i64, _I32, i64, ctypes.c_int, _D]),
                "or_gather_f32": (None, [_U8, i64, i64, _I32, i64, ctypes.c_int, _F]),
                "or_gather_pos_f32": (None, [_U8, i64, i64, _I32, i64, _I32, _D, _I32, _F]),
                "or_scatter_f64": (None, [_U8, i64, i64, _I32, i64, ctypes.c_int, _D]),
                "or_scatter_f32": (None, [_U8, i64, i64, _I32, i64, ctypes.c_int, _F]),
                "or_scatter_pos_f32": (None, [_U8, i64, i64, _I32, i64, _I32, _D, _I32, _F]),
                "or_reduce": (None, [i64, _D, _D, _D, _D, _D, _D]),
                "or_kick": (None, [i64, dbl, _D, _D, _D, _D]),
                "or_drift": (None, [i64, dbl, _D, _D, ctypes.c_int, _D]),
                "or_drift_walls": (None, [i64, dbl, _D, _D, _D]),
                "or_h_iterate": (i64, [i64, _D, _D, _D, _D, ctypes.c_int, dbl, dbl, i32, _D, _I32]),
                "or_kappa": (dbl, [ctypes.c_int]),
                "or_kw": (dbl, [ctypes.c_int, dbl, dbl]),
                "or_kdwdr": (dbl, [ctypes.c_int, dbl, dbl]),
                "or_kdwdh": (dbl, [ctypes.c_int, dbl, dbl]),
                "or_kernel_array": (None, [ctypes.c_int, ctypes.c_int, i64, _D, _D, _D]),
                "or_density_ext": (None, [ctypes.c_int, i64, _D, _D, _D, _D, _D, ctypes.c_int, i64, _I64, _D, _D,
                                          _D, _D, _D]),
                "or_force_ext": (None, [ctypes.c_int, ctypes.c_int, ctypes.c_int, i64, _D, _D, _D, _D, _D, _D,
                                        _D, _D, _D, _D, _D, ctypes.c_int, dbl, dbl, dbl, i64, _I64, _D, _D, _D]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a, ptype):
    return a.ctypes.data_as(ptype)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ----------------------------------------------------------------------------------------------------------
# Kernel (cubic spline, support 2h).
# ----------------------------------------------------------------------------------------------------------
def w(r, h):
    """W(r, h) of the 3D cubic spline, elementwise."""
    r, h = np.broadcast_arrays(np.asarray(r, np.float64), np.asarray(h, np.float64))
    r, h = _c(r, np.float64).ravel(), _c(h, np.float64).ravel()
    out = np.empty_like(r)
    _load().or_w_array(r.size, _p(r, _D), _p(h, _D), _p(out, _D))
    return out


def dwdr(r, h):
    """dW/dr of the 3D cubic spline, elementwise."""
    r, h = np.broadcast_arrays(np.asarray(r, np.float64), np.asarray(h, np.float64))
    r, h = _c(r, np.float64).ravel(), _c(h, np.float64).ravel()
    out = np.empty_like(r)
    _load().or_dwdr_array(r.size, _p(r, _D), _p(h, _D), _p(out, _D))
    return out


# ----------------------------------------------------------------------------------------------------------
# Pair sums (Section 2.1 steps 1-2, predicate of Listing 1 as a branch, all pairs).
# ----------------------------------------------------------------------------------------------------------
def density(x, m, h, box, periodic=True, targets=None):
    """rho_i for the target particles (all particles if targets is None), brute force over all j."""
    x, m, h = _c(x, np.float64), _c(m, np.float64), _c(h, np.float64)
    box = _c(box, np.float64)
    n = m.size
    tg = np.arange(n, dtype=np.int64) if targets is None else _c(targets, np.int64)
    out = np.empty(tg.size, np.float64)
    _load().or_density(n, _p(x, _D), _p(m, _D), _p(h, _D), _p(box, _D), int(bool(periodic)), tg.size,
                       _p(tg, _I64), _p(out, _D))
    return out


def eos(rho, u, gamma):
    """Ideal-gas P and c_s."""
    rho, u = _c(rho, np.float64), _c(u, np.float64)
    P = np.empty_like(rho)
    cs = np.empty_like(rho)
    _load().or_eos(rho.size, _p(rho, _D), _p(u, _D), float(gamma), _p(P, _D), _p(cs, _D))
    return P, cs


def force(x, v, m, h, rho, P, cs, box, periodic=True, alpha=1.0, beta=2.0, eps=0.01, targets=None):
    """(a_i, du_i/dt) for the target particles, brute force over all j."""
    x, v = _c(x, np.float64), _c(v, np.float64)
    m, h, rho, P, cs = (_c(q, np.float64) for q in (m, h, rho, P, cs))
    box = _c(box, np.float64)
    n = m.size
    tg = np.arange(n, dtype=np.int64) if targets is None else _c(targets, np.int64)
    a = np.empty((tg.size, 3), np.float64)
    du = np.empty(tg.size, np.float64)
    _load().or_force(n, _p(x, _D), _p(v, _D), _p(m, _D), _p(h, _D), _p(rho, _D), _p(P, _D), _p(cs, _D),
                     _p(box, _D), int(bool(periodic)), float(alpha), float(beta), float(eps), tg.size,
                     _p(tg, _I64), _p(a, _D), _p(du, _D))
    return a, du


# ----------------------------------------------------------------------------------------------------------
# Kernel families (M4 cubic, M5 quartic: the paper's kernel, Section 2.1) and the fuller density / force views
# (Section 2.1, Table 1).
# ----------------------------------------------------------------------------------------------------------
KERNEL_M4, KERNEL_M5 = 0, 1
SCHEME_MINIMAL, SCHEME_EXTENDED = 0, 1


def kappa(kern):
    """Support radius in units of h: 2 (M4), 5/2 (M5)."""
    return float(_load().or_kappa(int(kern)))


def kernel(kern, which, r, h):
    """W (which 0), dW/dr (1) or dW/dh (2) of kernel family `kern`, elementwise."""
    r, h = np.broadcast_arrays(np.asarray(r, np.float64), np.asarray(h, np.float64))
    r, h = _c(r, np.float64).ravel(), _c(h, np.float64).ravel()
    out = np.empty_like(r)
    _load().or_kernel_array(int(kern), int(which), r.size, _p(r, _D), _p(h, _D), _p(out, _D))
    return out


def density_ext(kern, x, v, m, h, box, periodic=True, targets=None):
    """The fuller density view of the targets: dict rho, omega, nnb, divv, curlv ([nt, 3])."""
    x, v, m, h = (_c(q, np.float64) for q in (x, v, m, h))
    box = _c(box, np.float64)
    n = m.size
    tg = np.arange(n, dtype=np.int64) if targets is None else _c(targets, np.int64)
    rho, om, nnb, dv = (np.empty(tg.size, np.float64) for _ in range(4))
    curl = np.empty((tg.size, 3), np.float64)
    _load().or_density_ext(int(kern), n, _p(x, _D), _p(v, _D), _p(m, _D), _p(h, _D), _p(box, _D),
                           int(bool(periodic)), tg.size, _p(tg, _I64), _p(rho, _D), _p(om, _D), _p(nnb, _D),
                           _p(dv, _D), _p(curl, _D))
    return {"rho": rho, "omega": om, "nnb": nnb, "divv": dv, "curlv": curl}


def force_ext(kern, use_gradh, use_balsara, x, v, m, h, rho, P, cs, omega, divv, curlv, box, periodic=True,
              alpha=1.0, beta=2.0, eps=0.01, targets=None):
    """(a_i, du_i/dt, vsig_i) of the fuller force view for the targets, brute force over all j."""
    x, v, curlv = _c(x, np.float64), _c(v, np.float64), _c(curlv, np.float64)
    m, h, rho, P, cs, omega, divv = (_c(q, np.float64) for q in (m, h, rho, P, cs, omega, divv))
    box = _c(box, np.float64)
    n = m.size
    tg = np.arange(n, dtype=np.int64) if targets is None else _c(targets, np.int64)
    a = np.empty((tg.size, 3), np.float64)
    du = np.empty(tg.size, np.float64)
    vs = np.empty(tg.size, np.float64)
    _load().or_force_ext(int(kern), int(bool(use_gradh)), int(bool(use_balsara)), n, _p(x, _D), _p(v, _D),
                         _p(m, _D), _p(h, _D), _p(rho, _D), _p(P, _D), _p(cs, _D), _p(omega, _D), _p(divv, _D),
                         _p(curlv, _D), _p(box, _D), int(bool(periodic)), float(alpha), float(beta), float(eps),
                         tg.size, _p(tg, _I64), _p(a, _D), _p(du, _D), _p(vs, _D))
    return a, du, vs


def neighbours(x, h, box, i, periodic=True, rad_factor=2.0):
    """All j (including i) with |r_ij| < rad_factor * max(h_i, h_j)."""
    x, h, box = _c(x, np.float64), _c(h, np.float64), _c(box, np.float64)
    n = h.size
    cap = 4096
    while True:
        out = np.empty(cap, np.int64)
        cnt = _load().or_neighbours(n, _p(x, _D), _p(h, _D), _p(box, _D), int(bool(periodic)), int(i),
                                     float(rad_factor), cap, _p(out, _I64))
        if cnt <= cap:
            return out[:cnt].copy()
        cap = int(cnt)


# ----------------------------------------------------------------------------------------------------------
# Cell bucketing and view conversions (Sections 2.1-2.2, 4.2).
# ----------------------------------------------------------------------------------------------------------
def bin_cells(x, box, ncell):
    """Stable counting sort into cells: returns (cell_of, cell_start, perm, cell_of_slot, n_out_of_box)."""
    x, box = _c(x, np.float64), _c(box, np.float64)
    nc = _c(ncell, np.int32)
    n = x.shape[0]
    ncells = int(nc[0]) * int(nc[1]) * int(nc[2])
    cell_of = np.empty(n, np.int32)
    cell_start = np.empty(ncells + 1, np.int32)
    perm = np.empty(n, np.int32)
    cos = np.empty(n, np.int32)
    bad = _load().or_bin(n, _p(x, _D), _p(box, _D), _p(nc, _I32), _p(cell_of, _I32), _p(cell_start, _I32),
                         _p(perm, _I32), _p(cos, _I32))
    return cell_of, cell_start, perm, cos, int(bad)


def bin_patches(x, h, patch_start, box, ncap):
    """Per-patch grids (edge >= 2 h_max of the patch, at most ncap per axis) and the stable counting sort over the
    concatenated patch cells: returns dict patch_n [npatch, 3], patch_cell_base, cell_of, cell_start, perm,
    cell_of_slot."""
    x, h, box = _c(x, np.float64), _c(h, np.float64), _c(box, np.float64)
    ps = _c(patch_start, np.int64)
    npatch = ps.size - 1
    n = h.size
    patch_n = np.empty(3 * npatch, np.int32)
    pcb = np.empty(npatch + 1, np.int32)
    cell_of = np.empty(n, np.int32)
    cap = npatch * int(ncap) ** 3
    cell_start = np.empty(cap + 1, np.int32)
    perm = np.empty(n, np.int32)
    cos = np.empty(n, np.int32)
    nc = _load().or_bin_patches(n, _p(x, _D), _p(h, _D), _p(ps, _I64), npatch, _p(box, _D), int(ncap),
                                _p(patch_n, _I32), _p(pcb, _I32), _p(cell_of, _I32), _p(cell_start, _I32),
                                _p(perm, _I32), _p(cos, _I32))
    return {"patch_n": patch_n.reshape(npatch, 3), "patch_cell_base": pcb, "cell_of": cell_of,
            "cell_start": cell_start[:nc + 1].copy(), "perm": perm, "cell_of_slot": cos, "ncells": int(nc)}


def gather_pos_f32_patches(aos, stride, perm, off, cell_of_slot, patch_cell_base, patch_n, box):
    """FP32 patch-local positions relative to the slot's cell origin, array [3, n]."""
    aos = _c(aos, np.uint8)
    perm, cos = _c(perm, np.int32), _c(cell_of_slot, np.int32)
    pcb, pn = _c(patch_cell_base, np.int32), _c(patch_n, np.int32).ravel()
    box = _c(box, np.float64)
    n = perm.size
    out = np.empty((3, n), np.float32)
    _load().or_gather_pos_f32_patches(_p(aos, _U8), int(stride), n, _p(perm, _I32), int(off), _p(cos, _I32),
                                      _p(pcb, _I32), _p(pn, _I32), pcb.size - 1, _p(box, _D), _p(out, _F))
    return out


def step_patches(aos, layout, patch_start, box, params, patches=None):
    """Expected rho, P, c_s, a, du/dt of every record of the listed patches (all if None): each patch is an open
    box whose particles interact only with each other; brute force within the patch."""
    f = unpack(aos, layout)
    ps = np.asarray(patch_start, np.int64)
    n = f["h"].size
    out = {k: np.full(n, np.nan) for k in ("rho", "P", "cs", "dudt")}
    out["a"] = np.full((n, 3), np.nan)
    for p in (range(ps.size - 1) if patches is None else patches):
        s, e = int(ps[p]), int(ps[p + 1])
        if e == s:
            continue
        x, v, m, h, u = f["x"][s:e], f["v"][s:e], f["mass"][s:e], f["h"][s:e], f["u"][s:e]
        rho = density(x, m, h, box, periodic=False)
        P, cs = eos(rho, u, params["gamma"])
        a, du = force(x, v, m, h, rho, P, cs, box, False, params["alpha"], params["beta"], params["eps"])
        out["rho"][s:e], out["P"][s:e], out["cs"][s:e], out["a"][s:e], out["dudt"][s:e] = rho, P, cs, a, du
    return out


def gather(aos, stride, perm, off, ncomp, dtype=np.float64):
    """Narrow + AoS->SoA (Eq. 3-5): array [ncomp, n] of the field at byte `off` of each record perm[s]."""
    aos = _c(aos, np.uint8)
    perm = _c(perm, np.int32)
    n = perm.size
    if dtype == np.float64:
        out = np.empty((ncomp, n), np.float64)
        _load().or_gather_f64(_p(aos, _U8), int(stride), n, _p(perm, _I32), int(off), int(ncomp), _p(out, _D))
    else:
        out = np.empty((ncomp, n), np.float32)
        _load().or_gather_f32(_p(aos, _U8), int(stride), n, _p(perm, _I32), int(off), int(ncomp), _p(out, _F))
    return out


def gather_pos_f32(aos, stride, perm, off, cell_of_slot, box, ncell):
    """FP32 cell-relative positions: (float)(x - k * (box / ncell)) per axis, array [3, n]."""
    aos = _c(aos, np.uint8)
    perm = _c(perm, np.int32)
    cos = _c(cell_of_slot, np.int32)
    box = _c(box, np.float64)
    nc = _c(ncell, np.int32)
    n = perm.size
    out = np.empty((3, n), np.float32)
    _load().or_gather_pos_f32(_p(aos, _U8), int(stride), n, _p(perm, _I32), int(off), _p(cos, _I32),
                              _p(box, _D), _p(nc, _I32), _p(out, _F))
    return out


def scatter(aos, stride, perm, off, values):
    """SoA->AoS + widen (Eq. 5), in place on a writable uint8 [n, stride] array; values is [ncomp, n]."""
    assert aos.dtype == np.uint8 and aos.flags.c_contiguous
    perm = _c(perm, np.int32)
    n = perm.size
    vals = np.ascontiguousarray(values)
    ncomp = vals.shape[0]
    if vals.dtype == np.float64:
        _load().or_scatter_f64(_p(aos, _U8), int(stride), n, _p(perm, _I32), int(off), ncomp, _p(vals, _D))
    elif vals.dtype == np.float32:
        _load().or_scatter_f32(_p(aos, _U8), int(stride), n, _p(perm, _I32), int(off), ncomp, _p(vals, _F))
    else:
        raise TypeError(vals.dtype)
    return aos


def scatter_pos_f32(aos, stride, perm, off, cell_of_slot, box, ncell, rel):
    """Widen FP32 cell-relative positions [3, n] back into the records' x member (in place)."""
    assert aos.dtype == np.uint8 and aos.flags.c_contiguous
    perm = _c(perm, np.int32)
    cos = _c(cell_of_slot, np.int32)
    box = _c(box, np.float64)
    nc = _c(ncell, np.int32)
    rel = _c(rel, np.float32)
    _load().or_scatter_pos_f32(_p(aos, _U8), int(stride), perm.size, _p(perm, _I32), int(off), _p(cos, _I32),
                               _p(box, _D), _p(nc, _I32), _p(rel, _F))
    return aos


def reduce_sums(m, v, a, u, dudt):
    """[sum m v (3), sum m a (3), sum m (v^2/2 + u), sum m (v.a + du/dt)] in FP64."""
    m, v, a, u, dudt = (_c(q, np.float64) for q in (m, v, a, u, dudt))
    out = np.empty(8, np.float64)
    _load().or_reduce(m.size, _p(m, _D), _p(v, _D), _p(a, _D), _p(u, _D), _p(dudt, _D), _p(out, _D))
    return out


def h_iterate(x, m, h, box, periodic=True, eta=1.2, tol=1e-6, max_iter=30):
    """Smoothing-length iteration: returns (h, rho, rounds run, particles not converged)."""
    x, m, box = _c(x, np.float64), _c(m, np.float64), _c(box, np.float64)
    h = np.array(h, np.float64, copy=True, order="C")
    n = m.size
    rho = np.empty(n, np.float64)
    it = np.zeros(1, np.int32)
    left = _load().or_h_iterate(n, _p(x, _D), _p(m, _D), _p(h, _D), _p(box, _D), int(bool(periodic)), float(eta),
                                float(tol), int(max_iter), _p(rho, _D), _p(it, _I32))
    return h, rho, int(it[0]), int(left)


def kick(dtk, a, dudt, v, u):
    """v += a dtk, u += du/dt dtk, in place on copies; returns (v, u)."""
    a, dudt = _c(a, np.float64), _c(dudt, np.float64)
    v, u = np.array(v, np.float64, copy=True, order="C"), np.array(u, np.float64, copy=True, order="C")
    _load().or_kick(u.size, float(dtk), _p(a, _D), _p(dudt, _D), _p(v, _D), _p(u, _D))
    return v, u


def drift(dt, v, x, box, periodic=True):
    """x += v dt, wrapped into the periodic box; returns the new x."""
    v, box = _c(v, np.float64), _c(box, np.float64)
    x = np.array(x, np.float64, copy=True, order="C")
    _load().or_drift(x.shape[0], float(dt), _p(v, _D), _p(box, _D), int(bool(periodic)), _p(x, _D))
    return x


def drift_walls(dt, v, x, box):
    """x += v dt in the open box [0, box] with reflecting walls; returns the new (x, v)."""
    box = _c(box, np.float64)
    x = np.array(x, np.float64, copy=True, order="C")
    v = np.array(v, np.float64, copy=True, order="C")
    _load().or_drift_walls(x.shape[0], float(dt), _p(v, _D), _p(box, _D), _p(x, _D))
    return x, v


# ----------------------------------------------------------------------------------------------------------
# Whole passes on AoS bytes (the composition f = W o C o f^ o C o N of Eq. 5, evaluated by the definition).
# ----------------------------------------------------------------------------------------------------------
VECTOR_FIELDS = ("x", "v", "a", "curlv")


def unpack(aos, layout):
    """All physics fields of an AoS buffer in record order: dict name -> array ([n,3] for vectors)."""
    aos = _c(aos, np.uint8)
    stride = int(layout["stride"])
    n = aos.size // stride
    ident = np.arange(n, dtype=np.int32)
    out = {}
    for name, off in layout["offsets"].items():
        nc = 3 if name in VECTOR_FIELDS else 1
        g = gather(aos, stride, ident, off, nc)
        out[name] = g.T.copy() if nc == 3 else g[0].copy()
    return out


def density_pass(aos, layout, box, gamma, periodic=True, targets=None):
    """rho, P, c_s of the target records (all if None) from the AoS state."""
    f = unpack(aos, layout)
    rho = density(f["x"], f["mass"], f["h"], box, periodic, targets)
    u = f["u"] if targets is None else f["u"][np.asarray(targets)]
    P, cs = eos(rho, u, gamma)
    return rho, P, cs


def density_h_pass(aos, layout, box, params, eta=1.2, tol=1e-6, max_iter=30, periodic=True):
    """Expected results of the smoothing-length iteration on the AoS state: dict h, rho, P, cs, iters, left."""
    f = unpack(aos, layout)
    h, rho, it, left = h_iterate(f["x"], f["mass"], f["h"], box, periodic, eta, tol, max_iter)
    P, cs = eos(rho, f["u"], params["gamma"])
    return {"h": h, "rho": rho, "P": P, "cs": cs, "iters": it, "left": left}


def step_all(aos, layout, box, params, periodic=True):
    """Expected results of one density + force pass over every record: dict rho, P, cs, a, dudt."""
    f = unpack(aos, layout)
    rho = density(f["x"], f["mass"], f["h"], box, periodic)
    P, cs = eos(rho, f["u"], params["gamma"])
    a, du = force(f["x"], f["v"], f["mass"], f["h"], rho, P, cs, box, periodic, params["alpha"],
                  params["beta"], params["eps"])
    return {"rho": rho, "P": P, "cs": cs, "a": a, "dudt": du}


def step_sampled(aos, layout, box, params, targets, periodic=True):
    """Expected rho, P, c_s, a, du/dt of sampled records of a large state, one by one.

    The force of i needs rho, P, c_s of every j within 2 max(h_i, h_j); those densities are computed here by
    brute force too, so no value comes from anywhere but this oracle."""
    f = unpack(aos, layout)
    x, h = f["x"], f["h"]
    targets = np.asarray(targets, np.int64)
    need = set(int(t) for t in targets)
    for t in targets:
        need.update(int(j) for j in neighbours(x, h, box, int(t), periodic, 2.0))
    need = np.array(sorted(need), np.int64)
    n = h.size
    rho = np.full(n, np.nan)
    rho[need] = density(x, f["mass"], h, box, periodic, need)
    P = np.full(n, np.nan)
    cs = np.full(n, np.nan)
    P[need], cs[need] = eos(rho[need], f["u"][need], params["gamma"])
    a, du = force(x, f["v"], f["mass"], h, rho, P, cs, box, periodic, params["alpha"], params["beta"],
                  params["eps"], targets)
    return {"rho": rho[targets], "P": P[targets], "cs": cs[targets], "a": a, "dudt": du}


def _scheme_of(params):
    return int(params.get("kernel", KERNEL_M4)), int(params.get("scheme", SCHEME_MINIMAL))


def step_all_ext(aos, layout, box, params, periodic=True):
    """Expected results of one density + force pass with the kernel family and scheme of `params` ("kernel",
    "scheme"): dict rho, P, cs, a, dudt, and for the extended scheme also nnb, divv, curlv, omega, vsig."""
    kern, scheme = _scheme_of(params)
    f = unpack(aos, layout)
    d = density_ext(kern, f["x"], f["v"], f["mass"], f["h"], box, periodic)
    P, cs = eos(d["rho"], f["u"], params["gamma"])
    ext = scheme == SCHEME_EXTENDED
    a, du, vs = force_ext(kern, ext, ext, f["x"], f["v"], f["mass"], f["h"], d["rho"], P, cs, d["omega"],
                          d["divv"], d["curlv"], box, periodic, params["alpha"], params["beta"], params["eps"])
    out = {"rho": d["rho"], "P": P, "cs": cs, "a": a, "dudt": du}
    if ext:
        out.update(nnb=d["nnb"], divv=d["divv"], curlv=d["curlv"], omega=d["omega"], vsig=vs)
    return out


def step_sampled_ext(aos, layout, box, params, targets, periodic=True):
    """step_all_ext for sampled records of a large state, one by one: the force of i needs the density-view
    outputs of every j within kappa max(h_i, h_j), computed here by brute force as well."""
    kern, scheme = _scheme_of(params)
    f = unpack(aos, layout)
    x, h = f["x"], f["h"]
    targets = np.asarray(targets, np.int64)
    need = set(int(t) for t in targets)
    for t in targets:
        need.update(int(j) for j in neighbours(x, h, box, int(t), periodic, kappa(kern)))
    need = np.array(sorted(need), np.int64)
    n = h.size
    d = density_ext(kern, x, f["v"], f["mass"], h, box, periodic, need)
    full = {k: np.full((n, 3) if k == "curlv" else n, np.nan) for k in d}
    for k, val in d.items():
        full[k][need] = val
    P = np.full(n, np.nan)
    cs = np.full(n, np.nan)
    P[need], cs[need] = eos(full["rho"][need], f["u"][need], params["gamma"])
    ext = scheme == SCHEME_EXTENDED
    a, du, vs = force_ext(kern, ext, ext, x, f["v"], f["mass"], h, full["rho"], P, cs, full["omega"], full["divv"],
                          full["curlv"], box, periodic, params["alpha"], params["beta"], params["eps"], targets)
    out = {"rho": full["rho"][targets], "P": P[targets], "cs": cs[targets], "a": a, "dudt": du}
    if ext:
        out.update(nnb=full["nnb"][targets], divv=full["divv"][targets], curlv=full["curlv"][targets],
                   omega=full["omega"][targets], vsig=vs)
    return out


# ----------------------------------------------------------------------------------------------------------
# Leapfrog kick-drift-kick runs (Section 2.1 steps 1-5), composed from the pieces above.
# ----------------------------------------------------------------------------------------------------------
def _forces(x, v, u, m, h, box, periodic, params):
    """Density, EOS and force of every particle of one domain at (x, v, u)."""
    rho = density(x, m, h, box, periodic)
    P, cs = eos(rho, u, params["gamma"])
    a, du = force(x, v, m, h, rho, P, cs, box, periodic, params["alpha"], params["beta"], params["eps"])
    return rho, P, cs, a, du


def kdk_run(fields, box, params, dt, nsteps, periodic=True, predict=True, from_records=False, patch_start=None):
    """nsteps leapfrog steps from the state `fields` (dict x, v, u, mass, h and, with from_records, a and dudt).

    Step order (Section 2.1): kick v, u by dt/2 with the current a, du/dt; drift x by dt (periodic wrap, or the
    reflecting walls of an open box, which also turn the velocity); density, EOS and force at the new positions;
    kick the half-step v, u by dt/2 with the new a, du/dt.  With predict, the density and force see predicted
    values v_half + a dt/2 and u_half + du/dt dt/2 (the old a, du/dt), and the second kick, which starts again
    from the half-step values, replaces them: the "predicted values" the paper's second kick resets (Section
    2.2).  Without it they see the half-step values.  Unless from_records, one density + force pass first gives
    the initial a, du/dt (from_records: the state's own a and dudt, as left by an earlier run).  patch_start:
    independent open patches (records patch_start[p] .. patch_start[p+1]-1, no pair across patches, walls at
    0 and box).  Returns dict x, v, u, rho, P, cs, a, dudt of the final state."""
    x = np.array(fields["x"], np.float64)
    v = np.array(fields["v"], np.float64)
    u = np.array(fields["u"], np.float64)
    m, h = np.asarray(fields["mass"], np.float64), np.asarray(fields["h"], np.float64)
    n = u.size
    segs = [(0, n)] if patch_start is None else [(int(patch_start[p]), int(patch_start[p + 1]))
                                                 for p in range(len(patch_start) - 1)]
    per = bool(periodic) and patch_start is None

    def all_forces(x, v, u):
        out = [np.zeros(n), np.zeros(n), np.zeros(n), np.zeros((n, 3)), np.zeros(n)]
        for s, e in segs:
            if e > s:
                for dst, val in zip(out, _forces(x[s:e], v[s:e], u[s:e], m[s:e], h[s:e], box, per, params)):
                    dst[s:e] = val
        return out

    if from_records:
        a, du = np.array(fields["a"], np.float64), np.array(fields["dudt"], np.float64)
        rho, P, cs = (np.array(fields[k], np.float64) for k in ("rho", "P", "cs"))
    else:
        rho, P, cs, a, du = all_forces(x, v, u)
    for _ in range(nsteps):
        vh, uh = kick(0.5 * dt, a, du, v, u)
        if per:
            x = drift(dt, vh, x, box, True)
        else:
            x, vh = drift_walls(dt, vh, x, box)
        vp, up = kick(0.5 * dt, a, du, vh, uh) if predict else (vh, uh)
        rho, P, cs, a, du = all_forces(x, vp, up)
        v, u = kick(0.5 * dt, a, du, vh, uh)
    return {"x": x, "v": v, "u": u, "rho": rho, "P": P, "cs": cs, "a": a, "dudt": du}


def energy(m, v, u):
    """Total energy sum m (|v|^2 / 2 + u) in FP64 (slot 6 of reduce_sums)."""
    m, v, u = np.asarray(m, np.float64), np.asarray(v, np.float64), np.asarray(u, np.float64)
    return float(reduce_sums(m, v, np.zeros_like(v), u, np.zeros_like(u))[6])


def _split_targets(fn, targets, threads):
    """fn(chunk) over contiguous chunks of `targets` on `threads` host threads (the C loops release the GIL);
    results concatenated in target order, each value the one a single call gives."""
    import concurrent.futures as cf
    targets = np.asarray(targets, np.int64)
    chunks = [c for c in np.array_split(targets, max(1, min(4 * threads, targets.size))) if c.size]
    if threads <= 1 or len(chunks) <= 1:
        return fn(targets)
    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        parts = list(ex.map(fn, chunks))
    if isinstance(parts[0], tuple):
        return tuple(np.concatenate([p[k] for p in parts]) for k in range(len(parts[0])))
    return np.concatenate(parts)


def cube_sample(fields, box, params, centre, half, halo, threads=1):
    """The pass restricted to a cube of a periodic state: the force (a, du/dt) of every particle within `half` of
    `centre` (per axis, minimum image) and the density, P and c_s of every particle within half + halo (all that
    force needs when halo >= 2 h_max), brute force against all particles, on `threads` host threads.
    Returns dict block, halo (particle indices), rho, P, cs (of the halo), a, dudt (of the block)."""
    x, m, h = fields["x"], fields["mass"], fields["h"]
    n = m.size
    d = x - np.asarray(centre, np.float64)
    d -= box * np.round(d / box)
    blk = np.nonzero(np.all(np.abs(d) <= half, axis=1))[0]
    hal = np.nonzero(np.all(np.abs(d) <= half + halo, axis=1))[0]
    rho = np.full(n, np.nan)
    rho[hal] = _split_targets(lambda t: density(x, m, h, box, True, t), hal, threads)
    P = np.full(n, np.nan)
    cs = np.full(n, np.nan)
    P[hal], cs[hal] = eos(rho[hal], fields["u"][hal], params["gamma"])
    a, du = _split_targets(lambda t: force(x, fields["v"], m, h, rho, P, cs, box, True, params["alpha"],
                                           params["beta"], params["eps"], t), blk, threads)
    return {"block": blk, "halo": hal, "rho": rho[hal], "P": P[hal], "cs": cs[hal], "a": a, "dudt": du}
