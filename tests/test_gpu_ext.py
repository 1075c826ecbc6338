"""GPU parity of the kernel families and the fuller views against the brute-force FP64 oracle.

Every (kernel, scheme) pair other than (cubic, minimal) runs the generic FP64 loop bodies: the quartic spline
M5 (the paper's kernel, support 5h/2) with the minimal equations, and both kernels with the fuller density view
(neighbour count, div v, curl v, Omega) and force view (grad-h terms, Balsara switch, signal velocity), on the
paper's 272-byte record.  Bars (FP64 path): 1e-12; relative per particle for rho, P, c_s, Omega and the signal
velocity; normwise (max|err| / max|ref|) for a, du/dt, div v and curl v, sums that nearly cancel; the neighbour
count exactly.  FP32 views and patch views reject these schemes, and so does a layout without the fuller views'
members.
"""
import numpy as np
import pytest

import helpers as H
from paper_2502_16517_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

COMBOS = [(1, 0), (0, 1), (1, 1)]  # (kernel, scheme): M5 minimal, M4 extended, M5 extended
TOL = 1e-12


@pytest.fixture(scope="module")
def sph():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_16517_gb300 import build as b
    b.build()
    from paper_2502_16517_gb300 import sph as s
    return s


def _params(kern, scheme):
    return dict(wl.SPH_PARAMS, kernel=kern, scheme=scheme)


def _written(scheme):
    names = ["rho", "P", "cs", "a", "dudt"]
    if scheme == 1:
        names += ["nnb", "divv", "curlv", "omega", "vsig"]
    return names


def _run(sph, aos_h, lay, box, ncell, params, periodic=True, separate_calls=False):
    n = aos_h.shape[0]
    aos = H.to_dev(aos_h)
    v = H.new_view(lay, sph.SPH_F64, n, box, ncell, periodic)
    try:
        if separate_calls:
            ext = params.get("scheme", 0) == 1
            sph.sph_bin(v, aos, n)
            sph.sph_aos_to_soa(v, aos, n, sph.SPH_DENSITY_IN_EXT if ext else sph.SPH_DENSITY_IN)
            sph.sph_density(v, params)
            sph.sph_soa_to_aos(v, aos, n, sph.SPH_DENSITY_OUT_EXT if ext else sph.SPH_DENSITY_OUT)
            sph.sph_aos_to_soa(v, aos, n, sph.SPH_FORCE_IN_EXT if ext else sph.SPH_FORCE_IN)
            sph.sph_force(v, params)
            sph.sph_soa_to_aos(v, aos, n, sph.SPH_FORCE_OUT_EXT if ext else sph.SPH_FORCE_OUT)
        else:
            sph.sph_step(v, aos, n, params)
        sph.sph_view_sync(v)
        counts = sph.sph_pair_counts(v)
        out = aos.cpu().numpy()
    finally:
        sph.sph_view_destroy(v)
    return out, counts


def _rel_or_exact(got, ref):
    """Relative error where the reference is nonzero; where it is zero (a particle without force neighbours has
    signal velocity 0) the result must be zero too."""
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    z = ref == 0
    assert np.all(got[z] == 0)
    return H.rel_max(got[~z], ref[~z])


def _compare(got, ref, scheme, label):
    errs = {k: H.rel_max(got[k], ref[k]) for k in ("rho", "P", "cs")}
    errs.update(a=H.normwise(got["a"], ref["a"]), dudt=H.normwise(got["dudt"], ref["dudt"]))
    if scheme == 1:
        errs.update(omega=H.rel_max(got["omega"], ref["omega"]), vsig=_rel_or_exact(got["vsig"], ref["vsig"]),
                    divv=H.normwise(got["divv"], ref["divv"]), curlv=H.normwise(got["curlv"], ref["curlv"]))
        assert np.array_equal(got["nnb"], ref["nnb"]), f"{label}: neighbour counts differ"
    bad = {k: v for k, v in errs.items() if not (v <= TOL)}
    assert not bad, f"{label} errors above {TOL}: {bad} (all: {errs})"
    return errs


def _check(sph, oracle, f, kern, scheme, periodic=True, separate_calls=False, label=""):
    lay = wl.extended_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
    ncell = wl.ncell_for(f["box"], f["h"].max(), oracle.kappa(kern))
    params = _params(kern, scheme)
    out, counts = _run(sph, aos_h, lay, f["box"], ncell, params, periodic, separate_calls)
    got = oracle.unpack(out, lay)
    ref = oracle.step_all_ext(aos_h, lay, f["box"], params, periodic)
    _compare(got, ref, scheme, label)
    wm = H.written_mask(lay, _written(scheme))
    assert np.array_equal(out[:, ~wm], aos_h[:, ~wm]), "bytes outside the written members changed"
    return got, ref, counts


@pytest.mark.parametrize("kern,scheme", COMBOS)
def test_tiny_lattice_with_velocities(sph, oracle, kern, scheme):
    f = wl.jittered_lattice(16, jitter=0.1, vel_sigma=0.1)
    got, ref, counts = _check(sph, oracle, f, kern, scheme, label=f"tiny k{kern} s{scheme}")
    # density pairs: every j within kappa h_i, the particle itself included
    kap = oracle.kappa(kern)
    n_dens = sum(oracle.neighbours(f["x"], f["h"], f["box"], i, True, kap).size for i in range(len(f["h"])))
    assert counts[1] == n_dens and counts[2] == n_dens - len(f["h"])


@pytest.mark.parametrize("kern,scheme", COMBOS)
def test_random_unequal_h_open_box_separate_calls(sph, oracle, kern, scheme):
    # h between 0.08 and 0.12 for 2317 random particles: every particle has neighbours inside its own support.
    # (Without any, the grad-h term Omega = 1 + h/(3 rho) drho/dh is 0 up to rounding: the self term alone gives
    # drho/dh = -3 rho / h.  The fuller force then divides by a rounding residue.)
    rng = np.random.default_rng(11 + kern + 2 * scheme)
    n = 2317
    f = {"x": rng.uniform(0, 1, size=(n, 3)), "v": rng.normal(0, 0.3, size=(n, 3)),
         "mass": rng.uniform(0.5, 1.5, n) / n, "h": rng.uniform(0.08, 0.12, n), "u": rng.uniform(0.5, 1.5, n),
         "box": np.ones(3)}
    got, ref, _ = _check(sph, oracle, f, kern, scheme, periodic=False, separate_calls=True,
                         label=f"random k{kern} s{scheme}")
    if scheme == 1:
        assert ref["nnb"].min() >= 3


def test_extended_m5_full_size_sampled(sph, oracle):
    """The plain 262,144-particle workload on the 272-byte record, quartic kernel and fuller views, in one
    sph_step; sampled particles (every corner of the box and random ones) against the oracle one by one."""
    f = wl.plain()
    lay = wl.extended_layout()
    aos_h, where = wl.pack_aos(f, lay, order="shuffled")
    params = _params(1, 1)
    ncell = wl.ncell_for(f["box"], f["h"].max(), oracle.kappa(1))
    out, _ = _run(sph, aos_h, lay, f["box"], ncell, params)
    got = oracle.unpack(out, lay)
    rng = np.random.default_rng(7)
    n = aos_h.shape[0]
    targets = np.unique(np.concatenate([[0, n - 1], rng.integers(0, n, 22)]))
    ref = oracle.step_sampled_ext(aos_h, lay, f["box"], params, targets)
    sub = {k: np.asarray(v)[targets] for k, v in got.items()}
    _compare(sub, ref, 1, "plain M5 extended (sampled)")


def test_rejections(sph, oracle):
    f = wl.tiny()
    box, n = f["box"], len(f["h"])
    ncell = wl.ncell_for(box, f["h"].max(), 2.5)
    # FP32 view
    lay = wl.extended_layout()
    aos_h, _ = wl.pack_aos(f, lay)
    aos = H.to_dev(aos_h)
    for prec, params in ((1, _params(1, 0)), (1, _params(0, 1))):
        v = H.new_view(lay, prec, n, box, ncell)
        try:
            with pytest.raises(sph.SphError) as e:
                sph.sph_step(v, aos, n, params)
            assert e.value.status == sph.SPH_E_INVAL
        finally:
            sph.sph_view_destroy(v)
    # a layout without the fuller views' members
    lay0 = wl.default_layout()
    aos0 = H.to_dev(wl.pack_aos(f, lay0)[0])
    v = H.new_view(lay0, 0, n, box, ncell)
    try:
        with pytest.raises(sph.SphError) as e:
            sph.sph_step(v, aos0, n, _params(0, 1))
        assert e.value.status == sph.SPH_E_INVAL
        # unknown kernel / scheme values
        for bad in (_params(2, 0), _params(0, 2)):
            with pytest.raises(sph.SphError) as e:
                sph.sph_step(v, aos0, n, bad)
            assert e.value.status == sph.SPH_E_INVAL
        sph.sph_step(v, aos0, n, _params(1, 0))  # the quartic kernel needs no extra member
        sph.sph_view_sync(v)
    finally:
        sph.sph_view_destroy(v)
    # patch view
    fp = wl.patches(8, seed=3)
    lay = wl.extended_layout()
    aosp_h, _ = wl.pack_aos(fp, lay, segments=fp["patch_start"])
    import torch
    aosp = H.to_dev(aosp_h)
    ps = torch.tensor(fp["patch_start"], dtype=torch.int64, device=H.device())
    v = sph.sph_patches_create(lay, 0, aosp_h.shape[0], 8, fp["box"], 8, H.stream())
    try:
        with pytest.raises(sph.SphError) as e:
            sph.sph_patches_step(v, aosp, aosp_h.shape[0], ps, 8, _params(1, 1))
        assert e.value.status == sph.SPH_E_INVAL
    finally:
        sph.sph_view_destroy(v)


def test_m5_cells_narrower_than_the_support_are_flagged(sph, oracle):
    """Cells sized for the cubic spline (2h) are too narrow for the quartic's 5h/2: the density flags it."""
    f = wl.tiny()
    lay = wl.extended_layout()
    aos = H.to_dev(wl.pack_aos(f, lay)[0])
    n = len(f["h"])
    v = H.new_view(lay, 0, n, f["box"], wl.ncell_for(f["box"], f["h"].max(), 2.0))
    try:
        sph.sph_step(v, aos, n, _params(1, 0))
        with pytest.raises(sph.SphError) as e:
            sph.sph_view_sync(v)
        assert e.value.status == sph.SPH_E_DEVICE
        assert sph.sph_view_status(v, clear=True) & sph.SPH_DEV_H_TOO_BIG
    finally:
        sph.sph_view_destroy(v)


def test_extended_m5_kick_drift_kick_and_graph_replay(sph, oracle):
    """Three leapfrog steps (with the predicted values, the default) with the quartic kernel and the fuller views
    against the oracle's composition of the same steps; then the same call through a captured graph, twice, gives
    the same bytes."""
    f = wl.jittered_lattice(12, jitter=0.1, vel_sigma=0.2, seed=3)
    lay = wl.extended_layout()
    aos_h, _ = wl.pack_aos(f, lay)
    n = aos_h.shape[0]
    ncell = wl.ncell_for(f["box"], f["h"].max(), 2.5)
    params = _params(1, 1)
    dt, nsteps = 2e-3, 3
    import torch
    outs = []
    side = torch.cuda.Stream(device=H.device())  # a graph is captured on a stream other than the legacy default
    with torch.cuda.stream(side):
        for graph in (False, True, True):
            aos = H.to_dev(aos_h)
            v = sph.sph_view_create(lay, sph.SPH_F64, n, (f["box"], ncell, True), side.cuda_stream)
            try:
                if graph:
                    sph.sph_step_graph(v, aos, n, params, dt=dt, nsteps=nsteps)   # runs, then captures
                    aos.copy_(H.to_dev(aos_h))
                    sph.sph_step_graph(v, aos, n, params, dt=dt, nsteps=nsteps)   # replays
                else:
                    sph.sph_step(v, aos, n, params, dt=dt, nsteps=nsteps)
                sph.sph_view_sync(v)
                outs.append(aos.cpu().numpy())
            finally:
                sph.sph_view_destroy(v)
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
    st = oracle.unpack(aos_h, lay)
    x, vel, u = st["x"], st["v"], st["u"]

    def forces(x, vel, u):
        d = oracle.density_ext(1, x, vel, st["mass"], st["h"], f["box"])
        P, cs = oracle.eos(d["rho"], u, params["gamma"])
        a, du, vs = oracle.force_ext(1, True, True, x, vel, st["mass"], st["h"], d["rho"], P, cs, d["omega"],
                                     d["divv"], d["curlv"], f["box"], True, params["alpha"], params["beta"],
                                     params["eps"])
        return d, a, du, vs
    d, a, du, vs = forces(x, vel, u)
    for _ in range(nsteps):
        vh, uh = oracle.kick(0.5 * dt, a, du, vel, u)
        x = oracle.drift(dt, vh, x, f["box"])
        vp, up = oracle.kick(0.5 * dt, a, du, vh, uh)      # the predicted values the loops see
        d, a, du, vs = forces(x, vp, up)
        vel, u = oracle.kick(0.5 * dt, a, du, vh, uh)
    got = oracle.unpack(outs[0], lay)
    tol = 1e-10
    assert H.normwise(got["x"], x) <= tol
    assert H.normwise(got["v"], vel) <= tol
    assert H.rel_max(got["u"], u) <= tol
    assert H.rel_max(got["rho"], d["rho"]) <= tol
    assert H.rel_max(got["omega"], d["omega"]) <= tol
    assert H.normwise(got["divv"], d["divv"]) <= tol and H.normwise(got["curlv"], d["curlv"]) <= tol
    assert H.normwise(got["a"], a) <= tol
    assert _rel_or_exact(got["vsig"], vs) <= tol
