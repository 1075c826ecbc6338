"""The bin and the first gather of a pass run as one record pass plus a permutation (the staged gather), with the
leapfrog's first kick and drift and the predicted v, u folded in.  Index and byte work, so bit-exact against the
oracle: the slot order (perm, cell_start, cell_of_slot) and every staged SoA member after sph_step, in both
precisions, on grid and patch views, on a layout the record pass takes and on one it leaves to the separate
kernels (200-byte records)."""
import numpy as np
import pytest

import helpers as H
from paper_2502_16517_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

UNION = ("x", "mass", "h", "u", "v")


@pytest.fixture(scope="module")
def sph():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_16517_gb300 import build as b
    b.build()
    from paper_2502_16517_gb300 import sph as s
    return s


def _export(sph, v, n, prec):
    out = {}
    for name in UNION:
        f = wl.FIELDS.index(name)
        nc = wl.NCOMP[name]
        out[name] = np.stack([sph.sph_view_export(v, f, c, n, prec) for c in range(nc)])
    return out


def _expected_soa(oracle, aos_h, lay, perm, cos, prec, pos_f32):
    """The oracle's gather of the union members from records aos_h in slot order perm."""
    exp = {}
    for name in UNION:
        off, nc = lay["offsets"][name], wl.NCOMP[name]
        if name == "x" and prec == 1:
            exp[name] = pos_f32(off)
        else:
            exp[name] = oracle.gather(aos_h, lay["stride"], perm, off, nc, np.float64 if prec == 0 else np.float32)
    return exp


def _assert_bits(got, exp):
    for name in UNION:
        g, e = np.ascontiguousarray(got[name]), np.ascontiguousarray(exp[name])
        assert g.dtype == e.dtype and np.array_equal(g.view(np.uint8), e.view(np.uint8)), name


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("layout_kind", ["default", "shuffled", "stride200"])
def test_pass_gather_grid_bitexact(sph, oracle, prec, layout_kind):
    f = wl.jittered_lattice(13, jitter=0.3, vel_sigma=0.2, seed=9)             # 2197 particles: ragged tiles
    lay = {"default": wl.default_layout(), "shuffled": wl.shuffled_layout(seed=12),
           "stride200": wl.shuffled_layout(seed=5, stride=200)}[layout_kind]
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
    n = aos_h.shape[0]
    ncell = wl.ncell_for(f["box"], f["h"].max())
    aos = H.to_dev(aos_h)
    v = H.new_view(lay, prec, n, f["box"], ncell)
    try:
        sph.sph_step(v, aos, n, wl.SPH_PARAMS)
        sph.sph_view_sync(v)
        perm = sph.sph_view_export_index(v, 0, n)
        start = sph.sph_view_export_index(v, 1, int(np.prod(ncell)) + 1)
        cos = sph.sph_view_export_index(v, 2, n)
        got = _export(sph, v, n, prec)
    finally:
        sph.sph_view_destroy(v)
    x = oracle.unpack(aos_h, lay)["x"]
    _, o_start, o_perm, o_cos, _ = oracle.bin_cells(x, f["box"], ncell)
    np.testing.assert_array_equal(perm, o_perm)
    np.testing.assert_array_equal(start, o_start)
    np.testing.assert_array_equal(cos, o_cos)
    exp = _expected_soa(oracle, aos_h, lay, o_perm, o_cos, prec,
                        lambda off: oracle.gather_pos_f32(aos_h, lay["stride"], o_perm, off, o_cos, f["box"], ncell))
    _assert_bits(got, exp)


@pytest.mark.parametrize("prec", [0, 1])
def test_step_staged_kick_drift_and_prediction_bitexact(sph, oracle, prec):
    """One leapfrog step: the records after it hold the oracle's kicked and drifted x (and the second kick's v, u),
    and the view holds x and the predicted v_half + a dt/2, u_half + du/dt dt/2 of the pass, bit for bit (FP32
    views: their round-to-nearest casts)."""
    f = wl.jittered_lattice(12, jitter=0.2, vel_sigma=0.4, seed=10)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
    n = aos_h.shape[0]
    ncell = wl.ncell_for(f["box"], f["h"].max())
    p = wl.SPH_PARAMS
    dt = 3e-3
    aos = H.to_dev(aos_h)
    v = H.new_view(lay, prec, n, f["box"], ncell)
    try:
        sph.sph_step(v, aos, n, p)                                   # a, du/dt of the initial state
        mid = aos.cpu().numpy()
        sph.sph_view_set_integrator(v, sph.SPH_KDK_PREDICT | sph.SPH_KDK_CONTINUE)
        sph.sph_step(v, aos, n, p, dt=dt, nsteps=1)
        sph.sph_view_sync(v)
        perm = sph.sph_view_export_index(v, 0, n)
        cos = sph.sph_view_export_index(v, 2, n)
        got = _export(sph, v, n, prec)
        out = aos.cpu().numpy()
    finally:
        sph.sph_view_destroy(v)
    st = oracle.unpack(mid, lay)
    vh, uh = oracle.kick(0.5 * dt, st["a"], st["dudt"], st["v"], st["u"])
    x1 = oracle.drift(dt, vh, st["x"], f["box"], True)
    vp, up = oracle.kick(0.5 * dt, st["a"], st["dudt"], vh, uh)
    # the records after the drift, with the predicted v, u in place of the stored ones, gathered by the oracle
    rec = mid.copy()
    for name, val in (("x", x1), ("v", vp), ("u", up)):
        off = lay["offsets"][name]
        vals = np.ascontiguousarray(np.atleast_2d(val.T if val.ndim == 2 else val[None, :]))
        oracle.scatter(rec, lay["stride"], np.arange(n, dtype=np.int32), off, vals)
    _, _, o_perm, o_cos, _ = oracle.bin_cells(x1, f["box"], ncell)
    np.testing.assert_array_equal(perm, o_perm)
    np.testing.assert_array_equal(cos, o_cos)
    exp = _expected_soa(oracle, rec, lay, o_perm, o_cos, prec,
                        lambda off: oracle.gather_pos_f32(rec, lay["stride"], o_perm, off, o_cos, f["box"], ncell))
    _assert_bits(got, exp)
    # the records: x drifted, v and u after the second kick (half-step values + new a, du/dt times dt/2)
    fin = oracle.unpack(out, lay)
    np.testing.assert_array_equal(fin["x"], x1)
    v2, u2 = oracle.kick(0.5 * dt, fin["a"], fin["dudt"], vh, uh)
    np.testing.assert_array_equal(fin["v"], v2)
    np.testing.assert_array_equal(fin["u"], u2)


@pytest.mark.parametrize("prec", [0, 1])
def test_patches_pass_gather_bitexact(sph, oracle, prec):
    import torch
    fp = wl.patches(11, lam_lo=8, lam_hi=200, seed=14, vel_sigma=0.2)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(fp, lay, order="shuffled", segments=fp["patch_start"])
    n = aos_h.shape[0]
    ps = fp["patch_start"]
    npatch = len(ps) - 1
    aos = H.to_dev(aos_h)
    ps_dev = torch.tensor(ps, dtype=torch.int64, device=H.device())
    v = sph.sph_patches_create(lay, prec, n, npatch, fp["box"], 8, H.stream())
    try:
        sph.sph_patches_step(v, aos, n, ps_dev, npatch, wl.SPH_PARAMS)
        sph.sph_view_sync(v)
        perm = sph.sph_view_export_index(v, 0, n)
        cos = sph.sph_view_export_index(v, 2, n)
        got = _export(sph, v, n, prec)
    finally:
        sph.sph_view_destroy(v)
    st = oracle.unpack(aos_h, lay)
    r = oracle.bin_patches(st["x"], st["h"], ps, fp["box"], 8)
    np.testing.assert_array_equal(perm, r["perm"])
    np.testing.assert_array_equal(cos, r["cell_of_slot"])
    exp = _expected_soa(oracle, aos_h, lay, r["perm"], r["cell_of_slot"], prec,
                        lambda off: oracle.gather_pos_f32_patches(aos_h, lay["stride"], r["perm"], off,
                                                                  r["cell_of_slot"], r["patch_cell_base"],
                                                                  r["patch_n"], fp["box"]))
    _assert_bits(got, exp)
