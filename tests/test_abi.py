"""CPU-only checks of the C ABI: the library builds and loads, exports every symbol include/sph.h declares, and
rejects bad arguments on the host before touching the GPU."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sph():
    from paper_2502_16517_gb300 import build as b
    b.build()
    from paper_2502_16517_gb300 import sph as s
    s.lib()
    return s


def _declared():
    with open(os.path.join(ROOT, "include", "sph.h")) as fh:
        txt = fh.read()
    return sorted(set(re.findall(r"^SPH_API\s+[\w\s\*]+?\b(sph_\w+)\s*\(", txt, flags=re.M)))


def test_every_declared_symbol_is_exported(sph):
    names = _declared()
    assert len(names) >= 19
    L = sph.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing
    assert sorted(sph.EXPORTED) == names


def test_header_constants_match_binding(sph):
    with open(os.path.join(ROOT, "include", "sph.h")) as fh:
        txt = fh.read()
    enum = dict(re.findall(r"\b(SPH_[A-Z0-9_]+)\s*=\s*(\d+)", txt))
    for k, v in enum.items():
        assert getattr(sph, k) == int(v), k
    for k, v in re.findall(r"#define (SPH_DEV_\w+) (0x[0-9a-f]+)u", txt):
        assert getattr(sph, k) == int(v, 16)


def test_strerror(sph):
    for s in range(8):
        assert sph.strerror(s)
    assert sph.strerror(99) == "unknown status"


def _create(sph, lay, prec=0, n_max=10, box=(1, 1, 1), ncell=(4, 4, 4), periodic=True):
    L = sph.make_layout(lay) if isinstance(lay, dict) else lay
    D = sph.make_domain(box, ncell, periodic)
    out = ctypes.c_void_p()
    st = sph.lib().sph_view_create(ctypes.byref(L), prec, n_max, ctypes.byref(D), None, ctypes.byref(out))
    if out.value:
        sph.lib().sph_view_destroy(out.value)
    return st


def _lay():
    return {"stride": 160, "offsets": {"x": 0, "v": 24, "a": 48, "mass": 72, "h": 80, "rho": 88, "P": 96, "u": 104,
                                       "dudt": 112, "cs": 120}}


@pytest.mark.parametrize("bad", [
    {"stride": 100},                       # not a multiple of 8
    {"stride": 0},
    {"x": 4},                              # misaligned member
    {"v": 16},                             # overlaps x
    {"cs": 160},                           # outside the record
    {"x": -8},
])
def test_create_rejects_bad_layout(sph, bad):
    lay = _lay()
    if "stride" in bad:
        lay["stride"] = bad["stride"]
    else:
        lay["offsets"].update(bad)
    assert _create(sph, lay) == sph.SPH_E_INVAL


@pytest.mark.parametrize("kw", [
    {"ncell": (2, 4, 4)},                  # periodic needs >= 3 cells per axis
    {"ncell": (0, 4, 4), "periodic": False},
    {"box": (1, -1, 1)},
    {"box": (1, float("nan"), 1)},
    {"n_max": -1},
    {"n_max": 1 << 31},
    {"prec": 7},
    {"ncell": (1024, 1024, 1024)},         # more than 2^27 cells
])
def test_create_rejects_bad_domain_and_sizes(sph, kw):
    assert _create(sph, _lay(), **kw) == sph.SPH_E_INVAL


def test_create_null_out_and_null_view_calls(sph):
    L = sph.make_layout(_lay())
    D = sph.make_domain((1, 1, 1), (4, 4, 4))
    assert sph.lib().sph_view_create(ctypes.byref(L), 0, 1, ctypes.byref(D), None, None) == sph.SPH_E_INVAL
    lib = sph.lib()
    assert lib.sph_bin(None, None, 0) == sph.SPH_E_INVAL
    assert lib.sph_view_sync(None) == sph.SPH_E_INVAL
    assert lib.sph_density(None, None) == sph.SPH_E_INVAL
    assert lib.sph_view_set_union(None, 1) == sph.SPH_E_INVAL
    assert lib.sph_view_set_host_direct(None, 1) == sph.SPH_E_INVAL
    assert lib.sph_view_set_warps(None, 4, 4) == sph.SPH_E_INVAL
    assert lib.sph_view_get_tuning(None, None) == sph.SPH_E_INVAL
    assert lib.sph_view_destroy(None) == sph.SPH_OK


def test_create_accepts_open_small_grid_layout_validation_only(sph):
    # open boxes may have fewer than 3 cells per axis: validation passes; creation then needs a device, so only
    # the host-side checks are exercised here (no GPU in this process means the allocation reports an error).
    st = _create(sph, _lay(), ncell=(1, 2, 1), periodic=False)
    assert st in (sph.SPH_OK, sph.SPH_E_NOMEM, sph.SPH_E_CUDA)


@pytest.mark.parametrize("kw", [{"npatch_max": 0}, {"ncell_cap": 0}, {"ncell_cap": 65}, {"box": (3, 0, 3)},
                                {"npatch_max": 1 << 20, "ncell_cap": 64}])
def test_patches_create_rejects_bad_arguments(sph, kw):
    args = {"npatch_max": 4, "ncell_cap": 8, "box": (3, 3, 3)}
    args.update(kw)
    L = sph.make_layout(_lay())
    box = (ctypes.c_double * 3)(*args["box"])
    out = ctypes.c_void_p()
    st = sph.lib().sph_patches_create(ctypes.byref(L), 0, 100, args["npatch_max"], box, args["ncell_cap"], None,
                                      ctypes.byref(out))
    assert st == sph.SPH_E_INVAL and not out.value


@pytest.mark.parametrize("ncell", [(1 << 22, 1 << 21, 1 << 21),   # product wraps to 0 in 64-bit arithmetic
                                   (65537, 1, 1),                   # one axis beyond the capacity
                                   (300, 300, 1)])                  # 90,000 cells > SPH_BIN_STATIC_MAX_CELLS
def test_static_bin_rejects_large_grids_on_the_host(sph, ncell):
    # rejected before any device work, so the (never dereferenced) device pointers may be placeholders
    fake = 1 << 20
    st = sph.lib().sph_bin_static(ctypes.byref(sph.make_layout(_lay())),
                                  ctypes.byref(sph.make_domain((1, 1, 1), ncell, False)), fake, 8, fake, fake, fake,
                                  None, None)
    assert st == sph.SPH_E_INVAL
