"""GPU parity of the cell bucketing and the view conversions against the oracle: bit-exact (index and byte work,
FP64 copies, FP32 round-to-nearest casts)."""
import numpy as np
import pytest

import helpers as H
from paper_2502_16517_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

MASKS = {"dens_in": ("x", "mass", "h", "u"), "force_in": ("x", "v", "mass", "h", "rho", "P", "cs"),
         "all": wl.FIELDS}


@pytest.fixture(scope="module")
def sph():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_16517_gb300 import build as b
    b.build()
    from paper_2502_16517_gb300 import sph as s
    return s


def _mask(sph, names):
    m = 0
    for nm in names:
        m |= 1 << wl.FIELDS.index(nm)
    return m


def _cases():
    return {
        "tiny": (wl.tiny(), None),
        "ragged": (wl.jittered_lattice(11, jitter=0.45, vel_sigma=0.2, seed=3), None),   # 1331: 6 tiles, tail
        "one_cell": (None, "one_cell"),
        "single": (None, "single"),
    }


def _special(kind):
    rng = np.random.default_rng(1)
    if kind == "one_cell":
        n = 700
        x = 0.34 + rng.uniform(0, 0.3, size=(n, 3))      # all inside cell (1,1,1) of a 3^3 grid
    else:
        n = 1
        x = np.array([[0.5, 0.25, 0.75]])
    return {"x": x, "v": rng.normal(size=(n, 3)), "mass": np.full(n, 1.0 / n), "h": np.full(n, 0.1),
            "u": np.ones(n), "box": np.ones(3)}


@pytest.mark.parametrize("case", ["tiny", "ragged", "one_cell", "single"])
@pytest.mark.parametrize("layout_kind", ["default", "shuffled"])
def test_bin_matches_oracle(sph, oracle, case, layout_kind):
    f, special = _cases()[case]
    if special:
        f = _special(special)
    lay = wl.default_layout() if layout_kind == "default" else wl.shuffled_layout(seed=12)
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
    n = aos_h.shape[0]
    ncell = np.array([3, 3, 3], np.int32) if special else wl.ncell_for(f["box"], f["h"].max())
    x = oracle.unpack(aos_h, lay)["x"]
    cell_of, start, perm, cos, bad = oracle.bin_cells(x, f["box"], ncell)
    aos = H.to_dev(aos_h)
    v = H.new_view(lay, sph.SPH_F64, n, f["box"], ncell)
    try:
        sph.sph_bin(v, aos, n)
        sph.sph_view_sync(v)
        g_perm = sph.sph_view_export_index(v, 0, n)
        g_start = sph.sph_view_export_index(v, 1, int(np.prod(ncell)) + 1)
        g_cos = sph.sph_view_export_index(v, 2, n)
    finally:
        sph.sph_view_destroy(v)
    np.testing.assert_array_equal(g_perm, perm)
    np.testing.assert_array_equal(g_start, start)
    np.testing.assert_array_equal(g_cos, cos)


@pytest.mark.parametrize("ncell", [(64, 64, 64), (256, 256, 256), (512, 512, 511)],
                         ids=["64^3", "256^3", "near_2^27"])
def test_bin_large_grids(sph, oracle, ncell):
    """Sparse particles on large grids: the multi-CTA cell scan over 64 to 32,704 blocks, up to 133,955,584
    cells (just under the 2^27 limit), bit-exact against the oracle's counting sort."""
    rng = np.random.default_rng(7)
    n = 20011
    f = {"x": rng.uniform(0, 1, size=(n, 3)), "v": np.zeros((n, 3)), "mass": np.full(n, 1.0 / n),
         "h": np.full(n, 1e-4), "u": np.ones(n), "box": np.ones(3)}
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
    nc = np.asarray(ncell, np.int32)
    x = oracle.unpack(aos_h, lay)["x"]
    cell_of, start, perm, cos, bad = oracle.bin_cells(x, f["box"], nc)
    assert bad == 0
    aos = H.to_dev(aos_h)
    v = H.new_view(lay, sph.SPH_F64, n, f["box"], nc)
    try:
        sph.sph_bin(v, aos, n)
        sph.sph_view_sync(v)
        g_perm = sph.sph_view_export_index(v, 0, n)
        g_start = sph.sph_view_export_index(v, 1, int(np.prod(nc.astype(np.int64))) + 1)
        g_cos = sph.sph_view_export_index(v, 2, n)
    finally:
        sph.sph_view_destroy(v)
    np.testing.assert_array_equal(g_perm, perm)
    np.testing.assert_array_equal(g_start, start)
    np.testing.assert_array_equal(g_cos, cos)


def test_bin_empty_input(sph):
    lay = wl.default_layout()
    aos = H.to_dev(np.zeros((4, lay["stride"]), np.uint8))
    v = H.new_view(lay, sph.SPH_F64, 4, np.ones(3), (4, 4, 4))
    try:
        sph.sph_bin(v, aos, 0)
        sph.sph_view_sync(v)
        start = sph.sph_view_export_index(v, 1, 65)
        assert np.all(start == 0)
        # an empty pass is legal end to end
        sph.sph_step(v, aos, 0, wl.SPH_PARAMS)
        sph.sph_view_sync(v)
    finally:
        sph.sph_view_destroy(v)


def _layouts():
    d = wl.default_layout()
    s = wl.shuffled_layout(seed=21)
    s8 = wl.shuffled_layout(seed=5, stride=200)          # stride not a multiple of 16: 8-byte path
    return {"default": d, "shuffled": s, "stride200": s8}


@pytest.mark.parametrize("layout_kind", ["default", "shuffled", "stride200", "misaligned"])
@pytest.mark.parametrize("mask_kind", ["dens_in", "force_in", "all"])
@pytest.mark.parametrize("prec", [0, 1])
def test_gather_is_bitexact(sph, oracle, layout_kind, mask_kind, prec):
    lays = _layouts()
    lay = lays["default" if layout_kind == "misaligned" else layout_kind]
    f = wl.jittered_lattice(11, jitter=0.45, vel_sigma=0.2, seed=4)
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
    n = aos_h.shape[0]
    ncell = wl.ncell_for(f["box"], f["h"].max())
    import torch
    if layout_kind == "misaligned":
        # records start 8 bytes into a buffer: 16-byte loads are not legal, the 8-byte path must serve
        raw = torch.zeros(n * lay["stride"] + 16, dtype=torch.uint8, device=H.device())
        raw[8:8 + n * lay["stride"]] = torch.from_numpy(aos_h.reshape(-1)).to(H.device())
        aos = raw[8:]
        assert aos.data_ptr() % 16 == 8
    else:
        aos = H.to_dev(aos_h)
    names = MASKS[mask_kind]
    x = oracle.unpack(aos_h, lay)["x"]
    _, _, perm, cos, _ = oracle.bin_cells(x, f["box"], ncell)
    v = H.new_view(lay, prec, n, f["box"], ncell)
    try:
        sph.sph_bin(v, aos, n)
        sph.sph_aos_to_soa(v, aos, n, _mask(sph, names))
        sph.sph_view_sync(v)
        for nm in names:
            fidx = wl.FIELDS.index(nm)
            nc = wl.NCOMP[nm]
            off = lay["offsets"][nm]
            if prec == 0:
                ref = oracle.gather(aos_h, lay["stride"], perm, off, nc)
            elif nm == "x":
                ref = oracle.gather_pos_f32(aos_h, lay["stride"], perm, off, cos, f["box"], ncell)
            else:
                ref = oracle.gather(aos_h, lay["stride"], perm, off, nc, np.float32)
            for c in range(nc):
                got = sph.sph_view_export(v, fidx, c, n, prec)
                assert np.array_equal(got.view(np.uint8), ref[c].view(np.uint8)), (nm, c)
    finally:
        sph.sph_view_destroy(v)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("layout_kind", ["default", "shuffled", "stride200"])
def test_scatter_writes_only_its_members(sph, oracle, prec, layout_kind):
    lay = _layouts()[layout_kind]
    f = wl.jittered_lattice(10, jitter=0.45, vel_sigma=0.2, seed=8)
    src_h, _ = wl.pack_aos(f, lay, order="shuffled", seed=1)
    n = src_h.shape[0]
    dst_h = np.random.default_rng(77).integers(0, 256, size=src_h.shape, dtype=np.uint8)
    ncell = wl.ncell_for(f["box"], f["h"].max())
    names = ("x", "v", "mass", "cs")
    src, dst = H.to_dev(src_h), H.to_dev(dst_h)
    v = H.new_view(lay, prec, n, f["box"], ncell)
    try:
        sph.sph_bin(v, src, n)
        sph.sph_aos_to_soa(v, src, n, _mask(sph, wl.FIELDS))
        sph.sph_soa_to_aos(v, dst, n, _mask(sph, names))
        sph.sph_view_sync(v)
        out = dst.cpu().numpy()
    finally:
        sph.sph_view_destroy(v)
    wm = H.written_mask(lay, names)
    assert np.array_equal(out[:, ~wm], dst_h[:, ~wm])
    if prec == 0:
        assert np.array_equal(out[:, wm], src_h[:, wm])
    else:
        # FP32 views widen exactly: the written bytes are the oracle's f32 gather scattered back
        x = oracle.unpack(src_h, lay)["x"]
        _, _, perm, cos, _ = oracle.bin_cells(x, f["box"], ncell)
        ref = dst_h.copy()
        for nm in names:
            off = lay["offsets"][nm]
            if nm == "x":
                rel = oracle.gather_pos_f32(src_h, lay["stride"], perm, off, cos, f["box"], ncell)
                oracle.scatter_pos_f32(ref, lay["stride"], perm, off, cos, f["box"], ncell, rel)
            else:
                vals = oracle.gather(src_h, lay["stride"], perm, off, wl.NCOMP[nm], np.float32)
                oracle.scatter(ref, lay["stride"], perm, off, vals)
        assert np.array_equal(out, ref)


def test_round_trip_all_members_is_byte_identical(sph):
    lay = wl.shuffled_layout(seed=3)
    f = wl.jittered_lattice(12, jitter=0.45, vel_sigma=0.2, seed=9)
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
    n = aos_h.shape[0]
    aos = H.to_dev(aos_h)
    ncell = wl.ncell_for(f["box"], f["h"].max())
    v = H.new_view(lay, sph.SPH_F64, n, f["box"], ncell)
    try:
        sph.sph_bin(v, aos, n)
        allm = _mask(sph, wl.FIELDS)
        sph.sph_aos_to_soa(v, aos, n, allm)
        sph.sph_soa_to_aos(v, aos, n, allm)
        sph.sph_view_sync(v)
        assert np.array_equal(aos.cpu().numpy(), aos_h)
    finally:
        sph.sph_view_destroy(v)
