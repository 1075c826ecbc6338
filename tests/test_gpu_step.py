"""GPU checks of the whole-pass entry points, the FP64 reductions, the leapfrog steps and the error paths of the
C ABI (host validation, call-order state, device status bits set by host-made bad inputs)."""
import numpy as np
import pytest

import helpers as H
from paper_2502_16517_gb300 import workloads as wl

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sph():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_16517_gb300 import build as b
    b.build()
    from paper_2502_16517_gb300 import sph as s
    return s


def _tiny_aos(order="shuffled"):
    f = wl.jittered_lattice(16, jitter=0.1, vel_sigma=0.1)
    lay = wl.default_layout()
    aos_h, where = wl.pack_aos(f, lay, order=order)
    return f, lay, aos_h, wl.ncell_for(f["box"], f["h"].max())


@pytest.mark.parametrize("prec", [0, 1])
def test_step_equals_separate_calls_and_is_deterministic(sph, prec):
    f, lay, aos_h, ncell = _tiny_aos()
    a1, _ = H.run_step(aos_h, lay, f["box"], ncell, prec, separate_calls=True)
    a2, _ = H.run_step(aos_h, lay, f["box"], ncell, prec, separate_calls=False)
    a3, _ = H.run_step(aos_h, lay, f["box"], ncell, prec, separate_calls=False)
    assert np.array_equal(a1, a2)
    assert np.array_equal(a2, a3)


@pytest.mark.parametrize("prec", [0, 1])
def test_step_host_equals_step(sph, prec):
    import torch
    f, lay, aos_h, ncell = _tiny_aos()
    n = aos_h.shape[0]
    ref, _ = H.run_step(aos_h, lay, f["box"], ncell, prec, separate_calls=False)
    host = torch.from_numpy(aos_h.copy()).pin_memory()
    v = H.new_view(lay, prec, n, f["box"], ncell)
    try:
        stats = sph.sph_step_host(v, host, n, wl.SPH_PARAMS, want_stats=True)
    finally:
        sph.sph_view_destroy(v)
    assert np.array_equal(host.numpy(), ref)
    assert stats.shape == (8,)


@pytest.mark.parametrize("prec", [0, 1])
def test_step_host_in_place_equals_staged(sph, prec):
    """sph_step_host with the records read and written in place across the host link gives the bytes of the
    staged-copy mode, for one pass and for leapfrog steps; pageable memory is refused before any launch."""
    import torch
    f, lay, aos_h, ncell = _tiny_aos()
    n = aos_h.shape[0]
    out = {}
    for direct in (False, True):
        for nsteps in (0, 2):
            host = torch.from_numpy(aos_h.copy()).pin_memory()
            v = H.new_view(lay, prec, n, f["box"], ncell)
            try:
                sph.sph_view_set_host_direct(v, direct)
                sph.sph_step_host(v, host, n, wl.SPH_PARAMS, dt=1e-3 if nsteps else 0.0, nsteps=nsteps)
            finally:
                sph.sph_view_destroy(v)
            out[direct, nsteps] = host.numpy().copy()
    assert np.array_equal(out[True, 0], out[False, 0])
    assert np.array_equal(out[True, 2], out[False, 2])
    assert not np.array_equal(out[True, 0], aos_h)
    pageable = aos_h.copy()
    v = H.new_view(lay, prec, n, f["box"], ncell)
    try:
        sph.sph_view_set_host_direct(v, True)
        with pytest.raises(sph.SphError) as e:
            sph.sph_step_host(v, pageable, n, wl.SPH_PARAMS)
        assert e.value.status == sph.SPH_E_INVAL
        with pytest.raises(sph.SphError) as e:
            sph.sph_view_set_host_direct(v, 2)
        assert e.value.status == sph.SPH_E_INVAL
    finally:
        sph.sph_view_destroy(v)
    assert np.array_equal(pageable, aos_h)


@pytest.mark.parametrize("prec", [0, 1])
def test_step_host_in_place_replays(sph, prec):
    """Repeated in-place sph_step_host calls with the same records and arguments replay the step as a captured
    graph: three leapfrog calls in a row leave the bytes the staged-copy mode leaves."""
    import torch
    f, lay, aos_h, ncell = _tiny_aos()
    n = aos_h.shape[0]
    out = {}
    for direct in (False, True):
        host = torch.from_numpy(aos_h.copy()).pin_memory()
        v = H.new_view(lay, prec, n, f["box"], ncell)
        try:
            sph.sph_view_set_host_direct(v, direct)
            for _ in range(3):
                sph.sph_step_host(v, host, n, wl.SPH_PARAMS, dt=1e-3, nsteps=1)
        finally:
            sph.sph_view_destroy(v)
        out[direct] = host.numpy().copy()
    assert np.array_equal(out[True], out[False])
    assert not np.array_equal(out[True], aos_h)


@pytest.mark.parametrize("prec", [0, 1])
def test_reduce_matches_oracle_sums(sph, oracle, prec):
    """The FP64 sums run over the view's values: FP64 views hold the records' values, FP32 views their
    round-to-nearest casts (numpy's float32 cast), so the oracle sums those."""
    f, lay, aos_h, ncell = _tiny_aos()
    out, info = H.run_step(aos_h, lay, f["box"], ncell, prec)
    g = oracle.unpack(out, lay)
    if prec == 1:
        g = {k: v.astype(np.float32).astype(np.float64) for k, v in g.items()}
    ref = oracle.reduce_sums(g["mass"], g["v"], g["a"], g["u"], g["dudt"])
    red = info["reduce"]
    m = g["mass"]
    scale = np.array([np.sum(m[:, None] * np.abs(g["v"]))] * 3 + [np.sum(m[:, None] * np.abs(g["a"]))] * 3
                     + [abs(ref[6]), np.sum(m * (np.abs((g["v"] * g["a"]).sum(1)) + np.abs(g["dudt"])))])
    assert np.all(np.abs(red - ref) <= 1e-12 * scale)


def test_call_order_and_argument_errors(sph):
    f, lay, aos_h, ncell = _tiny_aos()
    n = aos_h.shape[0]
    aos = H.to_dev(aos_h)
    v = H.new_view(lay, sph.SPH_F64, n, f["box"], ncell)
    try:
        with pytest.raises(sph.SphError) as e:
            sph.sph_aos_to_soa(v, aos, n, sph.SPH_DENSITY_IN)     # before any bin
        assert e.value.status == sph.SPH_E_STATE
        with pytest.raises(sph.SphError) as e:
            sph.sph_bin(v, aos, n + 1)                            # n > n_max
        assert e.value.status == sph.SPH_E_INVAL
        sph.sph_bin(v, aos, n)
        with pytest.raises(sph.SphError) as e:
            sph.sph_density(v, wl.SPH_PARAMS)                     # density view not gathered
        assert e.value.status == sph.SPH_E_STATE
        with pytest.raises(sph.SphError) as e:
            sph.sph_aos_to_soa(v, aos, n - 1, sph.SPH_DENSITY_IN)  # n differs from the binned n
        assert e.value.status == sph.SPH_E_INVAL
        with pytest.raises(sph.SphError) as e:
            sph.sph_aos_to_soa(v, aos, n, 1 << 12)                # not a member bit
        assert e.value.status == sph.SPH_E_INVAL
        sph.sph_aos_to_soa(v, aos, n, sph.SPH_DENSITY_IN)
        with pytest.raises(sph.SphError) as e:
            sph.sph_soa_to_aos(v, aos, n, sph.SPH_DENSITY_OUT)    # not computed yet
        assert e.value.status == sph.SPH_E_STATE
        with pytest.raises(sph.SphError) as e:
            sph.sph_force(v, wl.SPH_PARAMS)
        assert e.value.status == sph.SPH_E_STATE
        for eps in (-0.01, float("nan"), float("inf")):           # the softening must be finite and >= 0
            with pytest.raises(sph.SphError) as e:
                sph.sph_density(v, dict(wl.SPH_PARAMS, eps=eps))
            assert e.value.status == sph.SPH_E_INVAL
        sph.sph_density(v, wl.SPH_PARAMS)
        sph.sph_soa_to_aos(v, aos, n, sph.SPH_DENSITY_OUT)
        sph.sph_bin(v, aos, n)                                     # re-binning invalidates the view
        with pytest.raises(sph.SphError) as e:
            sph.sph_soa_to_aos(v, aos, n, sph.SPH_DENSITY_OUT)
        assert e.value.status == sph.SPH_E_STATE
        sph.sph_view_sync(v)
    finally:
        sph.sph_view_destroy(v)


def test_layout_without_force_members_rejects_force(sph):
    f, lay, aos_h, ncell = _tiny_aos()
    small = {"stride": lay["stride"], "offsets": {k: lay["offsets"][k] for k in ("x", "mass", "h", "u", "rho", "P", "cs")}}
    n = aos_h.shape[0]
    aos = H.to_dev(aos_h)
    v = H.new_view(small, sph.SPH_F64, n, f["box"], ncell)
    try:
        sph.sph_bin(v, aos, n)
        sph.sph_aos_to_soa(v, aos, n, sph.SPH_DENSITY_IN)
        sph.sph_density(v, wl.SPH_PARAMS)
        with pytest.raises(sph.SphError) as e:
            sph.sph_aos_to_soa(v, aos, n, sph.SPH_FORCE_IN)        # v absent from this layout
        assert e.value.status == sph.SPH_E_INVAL
    finally:
        sph.sph_view_destroy(v)


def test_device_status_position_outside_box(sph):
    f, lay, aos_h, ncell = _tiny_aos()
    bad = aos_h.copy()
    o = lay["offsets"]["x"]
    bad[5, o:o + 8] = np.array([1.5]).view(np.uint8)              # outside [0, 1]
    bad[9, o + 8:o + 16] = np.array([np.nan]).view(np.uint8)
    n = bad.shape[0]
    aos = H.to_dev(bad)
    v = H.new_view(lay, sph.SPH_F64, n, f["box"], ncell)
    try:
        sph.sph_bin(v, aos, n)
        with pytest.raises(sph.SphError) as e:
            sph.sph_view_sync(v)
        assert e.value.status == sph.SPH_E_DEVICE
        assert sph.sph_view_status(v, clear=True) & sph.SPH_DEV_POS_RANGE
        assert sph.sph_view_status(v) == 0
        sph.sph_view_sync(v)
    finally:
        sph.sph_view_destroy(v)


def test_device_status_h_too_big(sph):
    f, lay, aos_h, ncell = _tiny_aos()
    bad = aos_h.copy()
    o = lay["offsets"]["h"]
    bad[17, o:o + 8] = np.array([0.2]).view(np.uint8)             # 2h = 0.4 > cell edge 1/6
    n = bad.shape[0]
    aos = H.to_dev(bad)
    v = H.new_view(lay, sph.SPH_F64, n, f["box"], ncell)
    try:
        sph.sph_step(v, aos, n, wl.SPH_PARAMS)
        with pytest.raises(sph.SphError) as e:
            sph.sph_view_sync(v)
        assert e.value.status == sph.SPH_E_DEVICE
        assert sph.sph_view_status(v, clear=True) & sph.SPH_DEV_H_TOO_BIG
    finally:
        sph.sph_view_destroy(v)


@pytest.mark.parametrize("prec", [0, 1])
def test_kick_drift_kick_steps(sph, oracle, prec):
    """Three leapfrog steps (kick dt/2, drift + wrap, rebin, density, force, kick dt/2) against the oracle's
    composition of the same steps."""
    f = wl.jittered_lattice(12, jitter=0.1, vel_sigma=0.2, seed=3)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay)
    n = aos_h.shape[0]
    ncell = wl.ncell_for(f["box"], f["h"].max())
    dt, nsteps = 2e-3, 3
    aos = H.to_dev(aos_h)
    v = H.new_view(lay, prec, n, f["box"], ncell)
    try:
        sph.sph_step(v, aos, n, wl.SPH_PARAMS, dt=dt, nsteps=nsteps)
        sph.sph_view_sync(v)
        out = aos.cpu().numpy()
    finally:
        sph.sph_view_destroy(v)
    # oracle: initial pass, then per step kick / drift / pass with the predicted values / kick
    p = wl.SPH_PARAMS
    ref = oracle.kdk_run(oracle.unpack(aos_h, lay), f["box"], p, dt, nsteps)
    x, vel, u, rho, a = ref["x"], ref["v"], ref["u"], ref["rho"], ref["a"]
    got = oracle.unpack(out, lay)
    tol = 1e-10 if prec == 0 else 1e-4
    assert H.normwise(got["x"], x) <= tol
    assert H.normwise(got["v"], vel) <= tol
    assert H.rel_max(got["u"], u) <= tol
    assert H.rel_max(got["rho"], rho) <= tol
    assert H.normwise(got["a"], a) <= tol
