"""GPU parity of the batched form (independent open-box patches) against the oracle.

Binning and FP32 conversions bit-exact; density and force within 1e-12 (FP64) / 2e-5 (FP32) of the brute-force
per-patch oracle, with the same per-field error definitions as test_gpu_pairs.  Cases: uneven Poisson
occupancy, an empty patch, a one-particle patch, a patch whose grid is capped, positions on box faces, and the
full 4096-patch workload checked on sampled patches."""
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


def _run(sph, aos_h, lay, ps, box, prec, ncap=8, separate=False, stats=False):
    import torch
    n = aos_h.shape[0]
    npatch = len(ps) - 1
    aos = H.to_dev(aos_h)
    ps_dev = torch.tensor(np.asarray(ps, np.int64), device=H.device())
    v = sph.sph_patches_create(lay, prec, max(n, 1), npatch, box, ncap, H.stream())
    try:
        if separate:
            sph.sph_patches_bin(v, aos, n, ps_dev, npatch)
            sph.sph_aos_to_soa(v, aos, n, sph.SPH_DENSITY_IN)
            sph.sph_density(v, wl.SPH_PARAMS)
            sph.sph_soa_to_aos(v, aos, n, sph.SPH_DENSITY_OUT)
            sph.sph_aos_to_soa(v, aos, n, sph.SPH_FORCE_IN)
            sph.sph_force(v, wl.SPH_PARAMS)
            sph.sph_soa_to_aos(v, aos, n, sph.SPH_FORCE_OUT)
        else:
            sph.sph_patches_step(v, aos, n, ps_dev, npatch, wl.SPH_PARAMS)
        sph.sph_view_sync(v)
        info = {"perm": sph.sph_view_export_index(v, 0, n), "cos": sph.sph_view_export_index(v, 2, n),
                "counts": sph.sph_pair_counts(v), "view": None}
        if stats:
            info["reduce"] = sph.sph_reduce(v)
        start_cap = npatch * ncap ** 3 + 1
        info["cell_start"] = sph.sph_view_export_index(v, 1, start_cap)
        out = aos.cpu().numpy()
    finally:
        sph.sph_view_destroy(v)
    return out, info


def _patch_input(npatch, lam_lo, lam_hi, seed, vel=0.2):
    f = wl.patches(npatch, lam_lo=lam_lo, lam_hi=lam_hi, seed=seed, vel_sigma=vel)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled", segments=f["patch_start"])
    return f, lay, aos_h


@pytest.mark.parametrize("ncap", [8, 3])
def test_patch_bin_matches_oracle(sph, oracle, ncap):
    f, lay, aos_h = _patch_input(10, 8, 120, seed=2)
    out, info = _run(sph, aos_h, lay, f["patch_start"], f["box"], 0, ncap=ncap)
    st = oracle.unpack(aos_h, lay)
    r = oracle.bin_patches(st["x"], st["h"], f["patch_start"], f["box"], ncap)
    np.testing.assert_array_equal(info["perm"], r["perm"])
    np.testing.assert_array_equal(info["cos"], r["cell_of_slot"])
    np.testing.assert_array_equal(info["cell_start"][:r["ncells"] + 1], r["cell_start"])


def test_patch_gather_fp32_positions_bitexact(sph, oracle):
    import torch
    f, lay, aos_h = _patch_input(7, 8, 200, seed=5)
    n = aos_h.shape[0]
    aos = H.to_dev(aos_h)
    ps_dev = torch.tensor(f["patch_start"], device=H.device())
    v = sph.sph_patches_create(lay, sph.SPH_F32, n, 7, f["box"], 8, H.stream())
    try:
        sph.sph_patches_bin(v, aos, n, ps_dev, 7)
        sph.sph_aos_to_soa(v, aos, n, sph.SPH_DENSITY_IN)
        sph.sph_view_sync(v)
        got = np.stack([sph.sph_view_export(v, sph.SPH_X, c, n, 1) for c in range(3)])
    finally:
        sph.sph_view_destroy(v)
    st = oracle.unpack(aos_h, lay)
    r = oracle.bin_patches(st["x"], st["h"], f["patch_start"], f["box"], 8)
    ref = oracle.gather_pos_f32_patches(aos_h, lay["stride"], r["perm"], lay["offsets"]["x"], r["cell_of_slot"],
                                        r["patch_cell_base"], r["patch_n"], f["box"])
    assert np.array_equal(got.view(np.uint32), ref.view(np.uint32))


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("separate", [False, True])
def test_patch_pass_matches_oracle(sph, oracle, prec, separate):
    f, lay, aos_h = _patch_input(16, 8, 150, seed=7)
    out, info = _run(sph, aos_h, lay, f["patch_start"], f["box"], prec, separate=separate)
    got = oracle.unpack(out, lay)
    ref = oracle.step_patches(aos_h, lay, f["patch_start"], f["box"], wl.SPH_PARAMS)
    H.compare_fields(got, ref, prec, f"patches prec={prec}")
    wm = H.written_mask(lay, ("rho", "P", "cs", "a", "dudt"))
    assert np.array_equal(out[:, ~wm], aos_h[:, ~wm])
    # pair counts: density pairs (self included) against the per-patch neighbour lists
    ps = f["patch_start"]
    st = oracle.unpack(aos_h, lay)
    nd = 0
    for p in range(len(ps) - 1):
        s, e = ps[p], ps[p + 1]
        for i in range(e - s):
            nd += oracle.neighbours(st["x"][s:e], st["h"][s:e], f["box"], i, periodic=False).size
    assert info["counts"][1] == nd


@pytest.mark.parametrize("prec", [0, 1])
def test_patch_degenerate_cases(sph, oracle, prec):
    """Empty patch, one-particle patch, all particles in one cell of a capped grid, positions on the box faces."""
    rng = np.random.default_rng(9)
    xs, hs = [], []
    sizes = []
    # patch 0: ordinary
    xs.append(rng.uniform(0, 3, size=(200, 3)))
    hs.append(np.full(200, 0.3))
    # patch 1: empty
    xs.append(np.zeros((0, 3)))
    hs.append(np.zeros(0))
    # patch 2: one particle
    xs.append(np.array([[1.0, 2.0, 0.5]]))
    hs.append(np.array([0.4]))
    # patch 3: tiny h (grid capped at ncap) and everything in one corner cell
    xs.append(rng.uniform(0, 0.2, size=(150, 3)))
    hs.append(np.full(150, 0.01))
    # patch 4: positions on the faces 0 and 3 and on interior cell faces
    xs.append(np.array([[0.0, 0.0, 0.0], [3.0, 3.0, 3.0], [1.5, 1.5, 1.5], [1.0, 0.0, 3.0], [2.0, 2.0, 1.0]]))
    hs.append(np.full(5, 0.5))
    for x in xs:
        sizes.append(len(x))
    x = np.concatenate(xs)
    n = len(x)
    f = {"x": x, "v": rng.normal(0, 0.3, size=(n, 3)), "mass": np.full(n, 0.01), "h": np.concatenate(hs),
         "u": np.ones(n)}
    ps = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled", segments=ps)
    box = np.full(3, 3.0)
    out, info = _run(sph, aos_h, lay, ps, box, prec, ncap=4)
    got = oracle.unpack(out, lay)
    ref = oracle.step_patches(aos_h, lay, ps, box, wl.SPH_PARAMS)
    H.compare_fields(got, ref, prec, "degenerate patches")


def test_sph_bin_and_patches_bin_reject_the_wrong_view(sph):
    import torch
    f, lay, aos_h = _patch_input(2, 8, 20, seed=1)
    n = aos_h.shape[0]
    aos = H.to_dev(aos_h)
    ps_dev = torch.tensor(f["patch_start"], device=H.device())
    v = sph.sph_patches_create(lay, 0, n, 2, f["box"], 8, H.stream())
    try:
        with pytest.raises(sph.SphError) as e:
            sph.sph_bin(v, aos, n)
        assert e.value.status == sph.SPH_E_INVAL
        with pytest.raises(sph.SphError) as e:
            sph.sph_patches_bin(v, aos, n, ps_dev, 3)            # more patches than the view holds
        assert e.value.status == sph.SPH_E_INVAL
    finally:
        sph.sph_view_destroy(v)
    u = H.new_view(lay, 0, n, np.ones(3), (3, 3, 3))
    try:
        with pytest.raises(sph.SphError) as e:
            sph.sph_patches_bin(u, aos, n, ps_dev, 2)
        assert e.value.status == sph.SPH_E_INVAL
    finally:
        sph.sph_view_destroy(u)


@pytest.mark.parametrize("prec", [1, 0])
def test_full_batched_workload_sampled_patches(sph, oracle, prec):
    """4096 patches, Poisson(lambda ~ U(8, 256)) per cell (~14.6 M particles), one pass in the launch
    configuration the benchmark times; four patches checked record by record against the oracle."""
    f = wl.patches(4096, seed=wl.SEED)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled", segments=f["patch_start"], canary=False)
    ps = f["patch_start"]
    out, info = _run(sph, aos_h, lay, ps, f["box"], prec)
    lam = f["lam"]
    sample = [int(np.argmin(lam)), int(np.argmax(lam)), 1000, 3000]
    ref = oracle.step_patches(aos_h, lay, ps, f["box"], wl.SPH_PARAMS, patches=sample)
    got = oracle.unpack(out, lay)
    idx = np.concatenate([np.arange(ps[p], ps[p + 1]) for p in sample])
    sub = lambda d: {k: d[k][idx] for k in ("rho", "P", "cs", "a", "dudt")}
    H.compare_fields(sub(got), sub(ref), prec, "batched sample")
    assert np.all(np.isfinite(got["rho"])) and np.all(got["rho"] > 0)
