"""GPU parity of the leapfrog steps (Section 2.1 steps 3-5) against the oracle's runs (oracle.kdk_run).

Batched form: independent open patches with reflecting walls, several steps in one graph launch and, with
SPH_KDK_CONTINUE, one step per graph launch continuing from the records.  Grid form: an open (non-periodic) box,
whose walls reflect as well.  Both integrators: the predicted values the second kick resets (the default) and
the half-step values.  Multi-step bars: 1e-10 (FP64) and 1e-3 (FP32) normwise, as for the large run: round-off
differences grow through the steps (and in FP32 the pair loops' 2e-5 per pass), so the single-pass bars do not
apply."""
import numpy as np
import pytest

import helpers as H
from paper_2502_16517_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL_RUN = {0: 1e-10, 1: 1e-3}


@pytest.fixture(scope="module")
def sph():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_16517_gb300 import build as b
    b.build()
    from paper_2502_16517_gb300 import sph as s
    return s


@pytest.fixture
def side_stream():
    import torch
    s = torch.cuda.Stream(device=H.device())
    with torch.cuda.stream(s):
        yield s


def _patch_input(npatch=12, seed=11, vel=0.3):
    f = wl.patches(npatch, lam_lo=8, lam_hi=40, seed=seed, vel_sigma=vel)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled", segments=f["patch_start"])
    return f, lay, aos_h


def _cfl_dt(oracle, f, params, patch_start=None, periodic=True, courant=0.3):
    r0 = oracle.kdk_run(f, f["box"], params, 0.0, 0, periodic=periodic, patch_start=patch_start)
    return courant * f["h"].min() / np.max(r0["cs"] + np.linalg.norm(f["v"], axis=1))


def _compare(got, ref, prec, box):
    tol = TOL_RUN[prec]
    d = got["x"] - ref["x"]
    assert np.max(np.abs(d)) <= tol * np.max(box), "x"
    assert H.normwise(got["v"], ref["v"]) <= tol, "v"
    for k in ("u", "rho", "P", "cs"):
        assert H.rel_max(got[k], ref[k]) <= tol, k
    assert H.normwise(got["a"], ref["a"]) <= tol, "a"
    assert H.normwise(got["dudt"], ref["dudt"]) <= tol, "dudt"


def _fields_of(oracle, aos_h, lay, where):
    """The particle-ordered fields of records `aos_h` (particle k lives in record where[k])."""
    st = oracle.unpack(aos_h, lay)
    return {k: val[where] for k, val in st.items()}


@pytest.mark.parametrize("prec,predict", [(0, True), (1, True), (0, False)])
def test_patches_kdk_steps_in_one_graph(sph, oracle, side_stream, prec, predict):
    import torch
    f, lay, aos_h = _patch_input()
    _, where = wl.pack_aos(f, lay, order="shuffled", segments=f["patch_start"])
    ps = f["patch_start"]
    n, npatch = aos_h.shape[0], len(ps) - 1
    p = wl.SPH_PARAMS
    dt = _cfl_dt(oracle, f, p, patch_start=ps)
    nsteps = 4
    aos = H.to_dev(aos_h)
    ps_dev = torch.tensor(ps, dtype=torch.int64, device=H.device())
    v = sph.sph_patches_create(lay, prec, n, npatch, f["box"], 8, side_stream.cuda_stream)
    try:
        sph.sph_view_set_integrator(v, sph.SPH_KDK_PREDICT if predict else 0)
        sph.sph_patches_step_graph(v, aos, n, ps_dev, npatch, p, dt=dt, nsteps=nsteps)   # runs, then captures
        sph.sph_view_sync(v)
        first = aos.cpu().numpy()
        aos.copy_(H.to_dev(aos_h))
        sph.sph_patches_step_graph(v, aos, n, ps_dev, npatch, p, dt=dt, nsteps=nsteps)   # replays
        sph.sph_view_sync(v)
        out = aos.cpu().numpy()
        _, launches = sph.sph_view_phase_times(v)
    finally:
        sph.sph_view_destroy(v)
    assert np.array_equal(first, out)                     # the replay repeats the captured run bit for bit
    ref = oracle.kdk_run(f, f["box"], p, dt, nsteps, predict=predict, patch_start=ps)
    got = _fields_of(oracle, out, lay, where)
    _compare(got, ref, prec, f["box"])
    assert got["x"].min() >= 0.0 and got["x"].max() <= 3.0
    assert np.sum(np.sign(got["v"]) != np.sign(f["v"])) > 0        # some particle met a wall
    # the kicks and drifts run inside the bin and scatter kernels of each step's pass: one bin per pass
    assert launches[sph.SPH_PH_BIN] > 0 and np.max(np.abs(got["x"] - f["x"])) > 0.0
    # members outside the leapfrog's and the loops' sets are untouched
    wm = H.written_mask(lay, ("x", "v", "u", "rho", "P", "cs", "a", "dudt"))
    assert np.array_equal(out[:, ~wm], aos_h[:, ~wm])


@pytest.mark.parametrize("prec", [0, 1])
def test_patches_kdk_continues_one_step_per_launch(sph, oracle, side_stream, prec):
    """An initial pass, then SPH_KDK_CONTINUE: every graph launch is one kick-drift-kick step from the records'
    a and du/dt; three launches equal the oracle's three-step run."""
    import torch
    f, lay, aos_h = _patch_input(npatch=9, seed=12)
    _, where = wl.pack_aos(f, lay, order="shuffled", segments=f["patch_start"])
    ps = f["patch_start"]
    n, npatch = aos_h.shape[0], len(ps) - 1
    p = wl.SPH_PARAMS
    dt = _cfl_dt(oracle, f, p, patch_start=ps)
    aos = H.to_dev(aos_h)
    ps_dev = torch.tensor(ps, dtype=torch.int64, device=H.device())
    v = sph.sph_patches_create(lay, prec, n, npatch, f["box"], 8, side_stream.cuda_stream)
    try:
        sph.sph_patches_step(v, aos, n, ps_dev, npatch, p)                 # a, du/dt of the initial state
        sph.sph_view_set_integrator(v, sph.SPH_KDK_PREDICT | sph.SPH_KDK_CONTINUE)
        for _ in range(3):
            sph.sph_patches_step_graph(v, aos, n, ps_dev, npatch, p, dt=dt, nsteps=1)
        stats = sph.sph_patches_step(v, aos, n, ps_dev, npatch, p, dt=dt, nsteps=1, want_stats=True)
        sph.sph_view_sync(v)
        out = aos.cpu().numpy()
    finally:
        sph.sph_view_destroy(v)
    ref = oracle.kdk_run(f, f["box"], p, dt, 4, patch_start=ps)
    got = _fields_of(oracle, out, lay, where)
    _compare(got, ref, prec, f["box"])
    # the sums of the final state (v, u re-read from the kicked records)
    m = got["mass"]
    exp = oracle.reduce_sums(m, ref["v"], ref["a"], ref["u"], ref["dudt"])
    scale = np.abs(oracle.reduce_sums(m, np.abs(ref["v"]), np.abs(ref["a"]), np.abs(ref["u"]), np.abs(ref["dudt"])))
    assert np.all(np.abs(stats - exp) <= TOL_RUN[prec] * np.maximum(scale, 1e-300))


@pytest.mark.parametrize("prec,predict", [(0, True), (1, False)])
def test_open_box_grid_reflects_at_walls(sph, oracle, side_stream, prec, predict):
    """A single open (non-periodic) grid: its walls reflect as the patches' do."""
    f = wl.jittered_lattice(12, jitter=0.2, vel_sigma=0.5, seed=13)
    lay = wl.default_layout()
    aos_h, where = wl.pack_aos(f, lay, order="shuffled")
    n = aos_h.shape[0]
    ncell = wl.ncell_for(f["box"], f["h"].max())
    p = wl.SPH_PARAMS
    dt = _cfl_dt(oracle, f, p, periodic=False)
    aos = H.to_dev(aos_h)
    v = sph.sph_view_create(lay, prec, n, (f["box"], ncell, False), side_stream.cuda_stream)
    try:
        sph.sph_view_set_integrator(v, sph.SPH_KDK_PREDICT if predict else 0)
        sph.sph_step_graph(v, aos, n, p, dt=dt, nsteps=5)
        sph.sph_view_sync(v)
        out = aos.cpu().numpy()
    finally:
        sph.sph_view_destroy(v)
    ref = oracle.kdk_run(f, f["box"], p, dt, 5, periodic=False, predict=predict)
    got = _fields_of(oracle, out, lay, where)
    _compare(got, ref, prec, f["box"])
    assert got["x"].min() >= 0.0 and got["x"].max() <= 1.0


def test_integrator_flags_are_checked(sph):
    lay = wl.default_layout()
    v = H.new_view(lay, 0, 16, np.ones(3), (4, 4, 4))
    try:
        with pytest.raises(sph.SphError):
            sph.sph_view_set_integrator(v, 4)
        sph.sph_view_set_integrator(v, sph.SPH_KDK_CONTINUE)
        sph.sph_view_set_integrator(v, 0)
    finally:
        sph.sph_view_destroy(v)
