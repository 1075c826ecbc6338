"""GPU parity of the density and force loops against the brute-force FP64 oracle.

Bars (written here, applied per field): FP64 path <= 1e-12, FP32 path <= 2e-5; relative error per particle for
rho, P, c_s (all positive, far from zero), normwise error max|err| / max|ref| for a and du/dt (sums that nearly
cancel make per-particle relative error meaningless).  Inputs span several tiles and ragged tails, and the
degenerate cases of the method: empty cells, one particle, all particles in one cell, a pair exactly at 2h,
particles on cell faces, coincident particles, periodic wrap and open boxes, unequal smoothing lengths."""
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


def _check(oracle, f, prec, periodic=True, ncell=None, order="shuffled", layout=None, label="",
           separate_calls=True, params=None):
    lay = layout or wl.default_layout()
    params = params or wl.SPH_PARAMS
    aos_h, _ = wl.pack_aos(f, lay, order=order)
    ncell = wl.ncell_for(f["box"], f["h"].max()) if ncell is None else np.asarray(ncell, np.int32)
    out, info = H.run_step(aos_h, lay, f["box"], ncell, prec, periodic, params=params,
                           separate_calls=separate_calls)
    got = oracle.unpack(out, lay)
    ref = oracle.step_all(aos_h, lay, f["box"], params, periodic)
    errs = H.compare_fields(got, ref, prec, label)
    wm = H.written_mask(lay, ("rho", "P", "cs", "a", "dudt"))
    assert np.array_equal(out[:, ~wm], aos_h[:, ~wm]), "bytes outside the written members changed"
    return got, ref, info, errs


@pytest.mark.parametrize("prec", [0, 1])
def test_tiny_config(sph, oracle, prec):
    """4096 particles, 16^3 jittered lattice, h = 1.2 s, 6^3 cells (the small configuration)."""
    got, ref, info, errs = _check(oracle, wl.tiny(), prec, label="tiny")
    # pair counts: density pairs (self included) and ordered force pairs, against the oracle's neighbour lists
    f = wl.tiny()
    n_dens = sum(oracle.neighbours(f["x"], f["h"], f["box"], i).size for i in range(0, 4096, 1))
    c = info["counts"]
    assert c[1] == n_dens and c[2] == n_dens - 4096
    assert c[0] == c[3] and c[0] >= c[1]


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("seed", [1, 2])
def test_random_ragged_unequal_h(sph, oracle, prec, seed):
    """Uniform random particles, h varying by 2x, N not a multiple of any tile: several tiles + ragged tail."""
    rng = np.random.default_rng(seed)
    n = 2000 + 317 * seed
    f = {"x": rng.uniform(0, 1, size=(n, 3)), "v": rng.normal(0, 0.3, size=(n, 3)),
         "mass": rng.uniform(0.5, 1.5, size=n) / n, "h": rng.uniform(0.04, 0.08, size=n),
         "u": rng.uniform(0.5, 1.5, size=n), "box": np.ones(3)}
    _check(oracle, f, prec, label=f"random{seed}")


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("visc", [{"eps": 0.0}, {"eps": 0.3, "alpha": 0.5, "beta": 1.0}], ids=["eps0", "eps0.3"])
def test_viscosity_parameters(sph, oracle, prec, visc):
    """No softening (eps = 0: D1 = r^2, the FP64 force's unsoftened variant) and a strong one with other alpha
    and beta, on random particles with unequal h, approaching and receding pairs, and no coincident pair (with
    eps = 0 the viscosity of a coincident pair is 0/0)."""
    rng = np.random.default_rng(11)
    n = 2100
    f = {"x": rng.uniform(0, 1, size=(n, 3)), "v": rng.normal(0, 0.5, size=(n, 3)),
         "mass": rng.uniform(0.5, 1.5, size=n) / n, "h": rng.uniform(0.04, 0.08, size=n),
         "u": rng.uniform(0.5, 1.5, size=n), "box": np.ones(3)}
    _check(oracle, f, prec, label=f"visc{visc['eps']}", params=dict(wl.SPH_PARAMS, **visc))


@pytest.mark.parametrize("seed", [3, 4])
def test_receding_estimate_of_the_wrong_sign_matches_oracle(sph, oracle, seed):
    """The FP64 force sorts its pairs by an FP32 estimate of v_ij . r_ij and evaluates the pairs estimated receding
    without the viscosity, except where the FP64 v_ij . r_ij is negative after all.  Here every velocity is
    1000 + eps_i along x (eps_i < 2e-5, below FP32 resolution at 1000) plus small y, z parts, so the estimate sees
    only the y, z parts and gets the sign wrong for many pairs; their viscosity must still be there, to the FP64
    bar.  (Without any viscosity the oracle's a and du/dt of this input change by 3.6e-5 normwise.)"""
    f = wl.jittered_lattice(14, jitter=0.3, seed=seed)
    rng = np.random.default_rng(100 + seed)
    n = f["x"].shape[0]
    v = np.empty((n, 3))
    v[:, 0] = 1000.0 + rng.uniform(0.0, 2e-5, size=n)
    v[:, 1:] = rng.uniform(-2e-5, 2e-5, size=(n, 2))
    f["v"] = v
    # the input does what it is for: many neighbour pairs whose FP32-rounded velocities give v.r > 0 while the
    # FP64 v.r is negative
    vf = v.astype(np.float32).astype(np.float64)
    box = f["box"]
    wrong = 0
    for i in range(0, n, 7):
        d = f["x"][i] - f["x"]
        d -= box * np.round(d / box)
        near = np.einsum("ij,ij->i", d, d) < (2 * f["h"][i]) ** 2
        near[i] = False
        exact = np.einsum("ij,ij->i", v[i] - v[near], d[near])
        est = np.einsum("ij,ij->i", vf[i] - vf[near], d[near])
        wrong += int(np.count_nonzero((est > 0) & (exact < 0)))
    assert wrong > 1000, wrong
    _check(oracle, f, 0, label=f"receding estimate, seed {seed}")


@pytest.mark.parametrize("prec", [0, 1])
def test_open_box(sph, oracle, prec):
    rng = np.random.default_rng(3)
    n = 1500
    f = {"x": rng.uniform(0, 1, size=(n, 3)), "v": rng.normal(0, 0.3, size=(n, 3)), "mass": np.full(n, 1.0 / n),
         "h": np.full(n, 0.07), "u": np.ones(n), "box": np.ones(3)}
    _check(oracle, f, prec, periodic=False, label="open")


@pytest.mark.parametrize("prec", [0, 1])
def test_clustered_with_empty_cells(sph, oracle, prec):
    f = wl.clustered(4096, sigma=0.03, peak=40.0, seed=5, vel_sigma=0.1)
    f["h"] = np.full(4096, 0.05)
    _check(oracle, f, prec, label="clustered")


@pytest.mark.parametrize("prec", [0, 1])
def test_all_particles_in_one_cell_multiple_tiles(sph, oracle, prec):
    """1300 particles inside one cell of a 3^3 grid: the local set exceeds one local block (128) and the
    active set exceeds one staged tile."""
    rng = np.random.default_rng(4)
    n = 1300
    f = {"x": 0.34 + rng.uniform(0, 0.3, size=(n, 3)), "v": rng.normal(0, 0.1, size=(n, 3)),
         "mass": np.full(n, 1.0 / n), "h": np.full(n, 0.15), "u": np.ones(n), "box": np.ones(3)}
    _check(oracle, f, prec, ncell=(3, 3, 3), label="one_cell")


@pytest.mark.parametrize("prec", [0, 1])
def test_degenerate_geometry(sph, oracle, prec):
    """A pair exactly 2h apart, particles exactly on cell faces, a coincident pair, wrap across the box edge,
    an isolated particle."""
    h = 0.05
    x = np.array([
        [0.30, 0.50, 0.50], [0.40, 0.50, 0.50],          # exactly 2h apart along x
        [0.25, 0.25, 0.25], [0.26, 0.25, 0.25],          # on cell faces (edge 0.125)
        [0.70, 0.70, 0.70], [0.70, 0.70, 0.70],          # coincident
        [0.01, 0.90, 0.10], [0.97, 0.90, 0.10],          # across the periodic face x = 0
        [0.10, 0.10, 0.80],                              # alone
        [0.50, 0.125, 0.875],
    ])
    n = x.shape[0]
    f = {"x": x, "v": np.random.default_rng(0).normal(0, 0.5, size=(n, 3)), "mass": np.full(n, 0.01),
         "h": np.full(n, h), "u": np.ones(n), "box": np.ones(3)}
    _check(oracle, f, prec, ncell=(8, 8, 8), label="degenerate")


@pytest.mark.parametrize("prec", [0, 1])
def test_single_particle(sph, oracle, prec):
    f = {"x": np.array([[0.3, 0.6, 0.9]]), "v": np.zeros((1, 3)), "mass": np.array([0.5]), "h": np.array([0.1]),
         "u": np.array([2.0]), "box": np.ones(3)}
    _check(oracle, f, prec, ncell=(4, 4, 4), label="single")


@pytest.mark.parametrize("prec", [0, 1])
def test_uniform_lattice(sph, oracle, prec):
    """Unjittered lattice: every density equals the lattice shell sum; the force vanishes by symmetry, so a is
    checked against the unit of one pressure term, P / (rho h), not against the oracle's round-off noise."""
    f = wl.jittered_lattice(16, jitter=0.0)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay)
    ncell = wl.ncell_for(f["box"], f["h"].max())
    out, info = H.run_step(aos_h, lay, f["box"], ncell, prec)
    got = oracle.unpack(out, lay)
    ref = oracle.step_all(aos_h, lay, f["box"], wl.SPH_PARAMS)
    tol = H.TOL[prec]
    assert H.rel_max(got["rho"], ref["rho"]) <= tol
    assert H.rel_max(got["P"], ref["P"]) <= tol
    assert H.rel_max(got["cs"], ref["cs"]) <= tol
    if prec == 0:
        assert np.max(np.abs(got["rho"] - ref["rho"][0])) <= 1e-14
    unit = ref["P"][0] / (ref["rho"][0] * f["h"][0])
    assert np.max(np.abs(got["a"])) <= tol * unit
    assert np.max(np.abs(got["dudt"])) == 0.0     # v = 0


@pytest.mark.parametrize("layout_kind", ["shuffled", "stride200"])
def test_other_layouts(sph, oracle, layout_kind):
    lay = wl.shuffled_layout(seed=21) if layout_kind == "shuffled" else wl.shuffled_layout(seed=5, stride=200)
    _check(oracle, wl.jittered_lattice(12, jitter=0.2, vel_sigma=0.1, seed=6), 0, layout=lay, label=layout_kind)


@pytest.mark.parametrize("prec", [0, 1])
def test_conservation_on_gpu_output(sph, oracle, prec):
    """Sum m a = 0 and sum m (v.a + du/dt) = 0 up to round-off of the path's precision."""
    f = wl.jittered_lattice(14, jitter=0.3, vel_sigma=0.3, seed=7)
    got, ref, info, errs = _check(oracle, f, prec, label="conservation")
    m = f["mass"]
    mom = np.abs((m[:, None] * got["a"]).sum(0)).max() / (m[:, None] * np.abs(got["a"])).sum()
    tol = 1e-13 if prec == 0 else 1e-5
    assert mom < tol
    red = info["reduce"]
    scale = np.sum(m[:, None] * np.abs(got["a"]))
    assert np.all(np.abs(red[3:6]) < tol * scale)


@pytest.mark.parametrize("prec", [0, 1])
def test_full_size_plain_sampled(sph, oracle, prec):
    """262,144 particles (64^3 jittered lattice, v ~ N(0, 0.1)), one pass in the launch configuration the
    benchmark times; 24 sampled particles checked one by one against the oracle."""
    f = wl.plain()
    lay = wl.default_layout()
    aos_h, where = wl.pack_aos(f, lay, order="shuffled")
    ncell = wl.ncell_for(f["box"], f["h"].max())
    out, info = H.run_step(aos_h, lay, f["box"], ncell, prec, separate_calls=False)
    rng = np.random.default_rng(11)
    targets = np.sort(rng.choice(aos_h.shape[0], size=24, replace=False))
    ref = oracle.step_sampled(aos_h, lay, f["box"], wl.SPH_PARAMS, targets)
    got_all = oracle.unpack(out, lay)
    got = {k: got_all[k][targets] for k in ("rho", "P", "cs", "a", "dudt")}
    tol = H.TOL[prec]
    assert H.rel_max(got["rho"], ref["rho"]) <= tol
    assert H.rel_max(got["P"], ref["P"]) <= tol
    assert H.rel_max(got["cs"], ref["cs"]) <= tol
    # normwise over the sample, scaled by the sample's largest reference magnitude
    assert H.normwise(got["a"], ref["a"]) <= tol
    assert H.normwise(got["dudt"], ref["dudt"]) <= tol
    # properties at full size: every density positive and finite, momentum conserved
    assert np.all(np.isfinite(got_all["rho"])) and np.all(got_all["rho"] > 0)
    c = info["counts"]
    assert 50 * 262144 < c[1] < 65 * 262144
