"""The large-run form: clustered particles, ten leapfrog kick-drift-kick steps with per-step conversion and
re-binning, each ten-step run one CUDA graph launch.

Parity: a 4096-particle clustered set through the same ten steps against the oracle's composition of the steps
(FP64 within 1e-10 normwise after ten steps: round-off grows through the steps, so the single-pass 1e-12 bar is
not kept; FP32 within 1e-3).  Full size (2,097,152 particles): properties that hold at any size -- momentum
conserved, the semi-discrete energy rate zero, the integrator's energy drift first order in dt -- and the FP32
path stays close to the FP64 path."""
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


@pytest.fixture
def side_stream():
    import torch
    s = torch.cuda.Stream(device=H.device())
    with torch.cuda.stream(s):
        yield s


def cfl_dt(out, lay, courant=0.3):
    """dt = courant * min h / max(c_s + |v|), in FP64 from the records after the initial pass."""
    import oracle
    st = oracle.unpack(out, lay)
    return courant * st["h"].min() / np.max(st["cs"] + np.linalg.norm(st["v"], axis=1))


@pytest.mark.parametrize("prec,predict", [(0, True), (1, True), (0, False), (1, False)])
def test_ten_kdk_steps_small_clustered_parity(sph, oracle, side_stream, prec, predict):
    f = wl.clustered(4096, sigma=0.05, peak=4.0, n_side_equiv=16, seed=8)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay)
    n = aos_h.shape[0]
    ncell = wl.ncell_for(f["box"], f["h"].max())
    p = wl.SPH_PARAMS
    first = oracle.step_all(aos_h, lay, f["box"], p)
    dt = 0.3 * f["h"].min() / np.max(first["cs"])
    aos = H.to_dev(aos_h)
    v = sph.sph_view_create(lay, prec, n, (f["box"], ncell, True), side_stream.cuda_stream)
    try:
        sph.sph_view_set_integrator(v, sph.SPH_KDK_PREDICT if predict else 0)
        sph.sph_step_graph(v, aos, n, p, dt=dt, nsteps=10)
        sph.sph_view_sync(v)
        out = aos.cpu().numpy()
    finally:
        sph.sph_view_destroy(v)
    ref = oracle.kdk_run(oracle.unpack(aos_h, lay), f["box"], p, dt, 10, predict=predict)
    got = oracle.unpack(out, lay)
    tol = 1e-10 if prec == 0 else 1e-3
    d = got["x"] - ref["x"]
    d -= np.round(d)                              # periodic distance
    assert np.max(np.abs(d)) / f["h"][0] <= tol * 10
    assert H.normwise(got["v"], ref["v"]) <= tol
    assert H.rel_max(got["u"], ref["u"]) <= tol
    assert H.rel_max(got["rho"], ref["rho"]) <= tol
    assert H.normwise(got["a"], ref["a"]) <= tol


def _large_run(sph, aos_h, lay, box, ncell, prec, stream, dt=None, nsteps=10, predict=True):
    """Initial pass, then nsteps KDK steps as one graph launch, then one more pass so that the force sees the
    final velocities.  Returns (stats after the initial pass, stats after the final pass, final records, dt)."""
    n = aos_h.shape[0]
    p = wl.SPH_PARAMS
    aos = H.to_dev(aos_h)
    v = sph.sph_view_create(lay, prec, n, (box, ncell, True), stream.cuda_stream)
    try:
        sph.sph_view_set_integrator(v, sph.SPH_KDK_PREDICT if predict else 0)
        s0 = sph.sph_step(v, aos, n, p, want_stats=True)          # initial pass: rho, P, c_s, a, du/dt
        if dt is None:
            dt = cfl_dt(aos.cpu().numpy(), lay)
        sph.sph_step_graph(v, aos, n, p, dt=dt, nsteps=nsteps)
        s1 = sph.sph_step(v, aos, n, p, want_stats=True)          # a, du/dt at the final x, v, u
        out = aos.cpu().numpy()
    finally:
        sph.sph_view_destroy(v)
    return s0, s1, out, dt


def test_large_run_full_size_properties(sph, oracle, side_stream):
    """Full size, 2,097,152 particles, FP64 and FP32.

    - Momentum: zero initially (v = 0) and conserved exactly by the pairwise-antisymmetric force (FP64).
    - Energy rate: the semi-discrete equations conserve sum m (|v|^2/2 + u) exactly, so sum m (v.a + du/dt)
      vanishes up to round-off when a and du/dt are evaluated with the same v (the final pass).
    - Energy drift: with the half-step values in the force (SPH_KDK_PREDICT off) the leapfrog's energy error is
      first order in dt, so the ten-step drift halves when dt halves (twenty steps of dt/2).  With the predicted
      values (the default) it is second order; at this dt the ten-step drift is not yet in its asymptotic regime
      (the oracle's small clustered runs show it), so only its size is checked: far below the first-order drift.
    - The FP32 path follows the FP64 path over the ten steps."""
    f = wl.large()
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay, canary=False)
    n = aos_h.shape[0]
    ncell = wl.ncell_for(f["box"], f["h"].max())
    assert n == 2097152 and tuple(ncell) == (53, 53, 53)
    s0, s1, out64, dt = _large_run(sph, aos_h, lay, f["box"], ncell, 0, side_stream)
    st64 = oracle.unpack(out64, lay)
    m = st64["mass"]
    assert np.all(np.abs(s1[0:3]) <= 1e-12 * np.sum(m[:, None] * np.abs(st64["v"])))
    scale = np.sum(m * (np.abs(np.sum(st64["v"] * st64["a"], axis=1)) + np.abs(st64["dudt"])))
    assert scale > 0 and abs(s1[7]) <= 1e-10 * scale
    drift_pred = (s1[6] - s0[6]) / s0[6]
    p0, p1, _, _ = _large_run(sph, aos_h, lay, f["box"], ncell, 0, side_stream, dt=dt, predict=False)
    drift1 = (p1[6] - p0[6]) / p0[6]
    h0, h1, _, _ = _large_run(sph, aos_h, lay, f["box"], ncell, 0, side_stream, dt=0.5 * dt, nsteps=20,
                              predict=False)
    drift2 = (h1[6] - h0[6]) / h0[6]
    assert 0 < drift1 < 0.1 and 1.6 < drift1 / drift2 < 2.5
    assert abs(drift_pred) < 0.1 * drift1
    t0, t1, out32, _ = _large_run(sph, aos_h, lay, f["box"], ncell, 1, side_stream, dt=dt)
    st32 = oracle.unpack(out32, lay)
    assert abs(t1[7]) <= 1e-4 * scale
    d = st32["x"] - st64["x"]
    d -= np.round(d)
    assert np.max(np.abs(d)) / f["h"][0] < 1e-3
    assert H.rel_max(st32["rho"], st64["rho"]) < 1e-3
    assert abs((t1[6] - t0[6]) / t0[6] - drift_pred) < 1e-3 * drift1
    assert np.all(np.isfinite(st64["a"])) and np.all(np.isfinite(st32["a"]))


@pytest.fixture(scope="module")
def large_sample(oracle):
    """The large input, 12 sampled particles (3 at the centres of overdensities, 9 at random) and their oracle
    values, computed once for both precisions."""
    f = wl.large()
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled", canary=False)
    n = aos_h.shape[0]
    st = oracle.unpack(aos_h, lay)
    dense = []
    for c in f["centres"][:3]:
        d = st["x"] - c
        d -= np.round(d)
        dense.append(int(np.argmin(np.sum(d * d, axis=1))))
    rng = np.random.default_rng(21)
    targets = np.unique(np.concatenate([dense, rng.choice(n, size=9, replace=False)]))
    ref = oracle.step_sampled(aos_h, lay, f["box"], wl.SPH_PARAMS, targets)
    return f, lay, aos_h, targets, ref


@pytest.mark.parametrize("prec", [0, 1])
def test_large_initial_pass_sampled(sph, oracle, large_sample, prec):
    """Full size (2,097,152 clustered particles, 53^3 cells), one pass in the launch configuration the benchmark
    uses; the sampled particles checked one by one against the brute-force oracle."""
    f, lay, aos_h, targets, ref = large_sample
    ncell = wl.ncell_for(f["box"], f["h"].max())
    out, info = H.run_step(aos_h, lay, f["box"], ncell, prec, separate_calls=False)
    got_all = oracle.unpack(out, lay)
    got = {k: got_all[k][targets] for k in ("rho", "P", "cs", "a", "dudt")}
    tol = H.TOL[prec]
    for k in ("rho", "P", "cs"):
        assert H.rel_max(got[k], ref[k]) <= tol, k
    assert H.normwise(got["a"], ref["a"]) <= tol
    assert H.normwise(got["dudt"], ref["dudt"]) <= tol
    assert np.max(got["rho"]) > 2.0 * np.median(got_all["rho"])   # the sample reaches into an overdensity
