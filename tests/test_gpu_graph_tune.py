"""Graph-captured steps and the tile autotuner.

A replayed CUDA graph must produce exactly what the same step produces without a graph (the launch sequence is
identical, so the results are bitwise equal); the autotuner must pick tiles from its candidate list and leave
results within the path's tolerance of the default tiles (a different tile size changes only the summation
order across tiles)."""
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


def _tiny():
    f = wl.jittered_lattice(16, jitter=0.1, vel_sigma=0.1)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay)
    return f, lay, aos_h, wl.ncell_for(f["box"], f["h"].max())


@pytest.mark.parametrize("prec", [0, 1])
def test_graph_replay_equals_plain_step(sph, side_stream, prec):
    f, lay, aos_h, ncell = _tiny()
    n = aos_h.shape[0]
    ref, _ = H.run_step(aos_h, lay, f["box"], ncell, prec, separate_calls=False)
    aos = H.to_dev(aos_h)
    v = sph.sph_view_create(lay, prec, n, (f["box"], ncell, True), side_stream.cuda_stream)
    try:
        for _ in range(3):                      # capture on the first call, replay on the next two
            sph.sph_step_graph(v, aos, n, wl.SPH_PARAMS)
        sph.sph_view_sync(v)
        _, launches = sph.sph_view_phase_times(v)
        out = aos.cpu().numpy()
    finally:
        sph.sph_view_destroy(v)
    assert np.array_equal(out, ref)
    assert launches.sum() > 0                   # replays count their kernels too


def test_graph_kdk_replays_advance_the_state(sph, side_stream):
    f = wl.jittered_lattice(10, jitter=0.1, vel_sigma=0.2, seed=3)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay)
    n = aos_h.shape[0]
    ncell = wl.ncell_for(f["box"], f["h"].max())
    a1, a2 = H.to_dev(aos_h), H.to_dev(aos_h)
    v1 = sph.sph_view_create(lay, 0, n, (f["box"], ncell, True), side_stream.cuda_stream)
    v2 = sph.sph_view_create(lay, 0, n, (f["box"], ncell, True), side_stream.cuda_stream)
    try:
        for _ in range(3):
            sph.sph_step(v1, a1, n, wl.SPH_PARAMS, dt=1e-3, nsteps=2)
            sph.sph_step_graph(v2, a2, n, wl.SPH_PARAMS, dt=1e-3, nsteps=2)
        sph.sph_view_sync(v1)
        sph.sph_view_sync(v2)
        assert np.array_equal(a1.cpu().numpy(), a2.cpu().numpy())
        assert not np.array_equal(a1.cpu().numpy(), aos_h)
    finally:
        sph.sph_view_destroy(v1)
        sph.sph_view_destroy(v2)


def test_graph_needs_a_capturable_stream(sph):
    f, lay, aos_h, ncell = _tiny()
    n = aos_h.shape[0]
    aos = H.to_dev(aos_h)
    v = sph.sph_view_create(lay, 0, n, (f["box"], ncell, True), None)   # legacy default stream
    try:
        with pytest.raises(sph.SphError) as e:
            sph.sph_step_graph(v, aos, n, wl.SPH_PARAMS)
        assert e.value.status == sph.SPH_E_INVAL
    finally:
        sph.sph_view_destroy(v)


@pytest.mark.parametrize("prec", [0, 1])
def test_patches_graph_replay_equals_plain_step(sph, side_stream, prec):
    import torch
    fp = wl.patches(12, lam_lo=8, lam_hi=100, seed=4, vel_sigma=0.2)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(fp, lay, segments=fp["patch_start"])
    n = aos_h.shape[0]
    ps = torch.tensor(fp["patch_start"], device=H.device())
    outs = []
    for graph in (False, True):
        aos = H.to_dev(aos_h)
        v = sph.sph_patches_create(lay, prec, n, 12, fp["box"], 8, side_stream.cuda_stream)
        try:
            for _ in range(3):
                if graph:
                    sph.sph_patches_step_graph(v, aos, n, ps, 12, wl.SPH_PARAMS)
                else:
                    sph.sph_patches_step(v, aos, n, ps, 12, wl.SPH_PARAMS)
            sph.sph_view_sync(v)
            outs.append(aos.cpu().numpy())
        finally:
            sph.sph_view_destroy(v)
    assert np.array_equal(outs[0], outs[1])


@pytest.mark.parametrize("prec", [0, 1])
def test_autotune_picks_candidates_and_keeps_results(sph, oracle, side_stream, prec):
    f = wl.jittered_lattice(24, jitter=0.1, vel_sigma=0.1, seed=5)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay)
    n = aos_h.shape[0]
    ncell = wl.ncell_for(f["box"], f["h"].max())
    aos = H.to_dev(aos_h)
    v = sph.sph_view_create(lay, prec, n, (f["box"], ncell, True), side_stream.cuda_stream)
    try:
        (td, tf), (md, mf) = sph.sph_autotune(v, aos, n, wl.SPH_PARAMS)
        tuned_first = aos.cpu().numpy()
        sph.sph_step(v, aos, n, wl.SPH_PARAMS)
        sph.sph_view_sync(v)
        tuned = aos.cpu().numpy()
    finally:
        sph.sph_view_destroy(v)
    cands = {0: ([256, 384, 448, 512, 768, 1024, 1536], [128, 192, 256, 384, 448, 512, 768]),
             1: ([256, 512, 1024, 2048, 4096], [256, 384, 512, 1024, 2048])}[prec]
    assert td in cands[0] and tf in cands[1] and md > 0 and mf > 0
    ref = oracle.step_all(aos_h, lay, f["box"], wl.SPH_PARAMS)
    for out in (tuned_first, tuned):
        H.compare_fields(oracle.unpack(out, lay), ref, prec, "autotuned")


def test_set_tiles_validates(sph):
    f, lay, aos_h, ncell = _tiny()
    v = H.new_view(lay, 0, aos_h.shape[0], f["box"], ncell)
    try:
        sph.sph_view_set_tiles(v, 512, 256)
        for bad in ((100, 256), (512, 4160), (-64, 0)):
            with pytest.raises(sph.SphError) as e:
                sph.sph_view_set_tiles(v, *bad)
            assert e.value.status == sph.SPH_E_INVAL
    finally:
        sph.sph_view_destroy(v)


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("kdk", [False, True])
def test_union_view_equals_per_loop_views(sph, side_stream, prec, kdk):
    """One view for both loops (the force reads the density view's members and outputs in SoA, one scatter at the
    end) leaves exactly the records that a view per loop, converted forth and back around each, leaves."""
    f = wl.jittered_lattice(12, jitter=0.1, vel_sigma=0.2, seed=6)
    lay = wl.shuffled_layout(seed=5, stride=200)
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
    n = aos_h.shape[0]
    ncell = wl.ncell_for(f["box"], f["h"].max())
    outs, launches = [], []
    for union in (True, False):
        aos = H.to_dev(aos_h)
        v = sph.sph_view_create(lay, prec, n, (f["box"], ncell, True), side_stream.cuda_stream)
        try:
            if not union:
                sph.sph_view_set_union(v, False)
            if kdk:
                sph.sph_step(v, aos, n, wl.SPH_PARAMS, dt=1e-3, nsteps=2)
            else:
                sph.sph_step(v, aos, n, wl.SPH_PARAMS)
            sph.sph_view_sync(v)
            _, nl = sph.sph_view_phase_times(v)
            outs.append(aos.cpu().numpy())
            launches.append(nl)
        finally:
            sph.sph_view_destroy(v)
    assert np.array_equal(outs[0], outs[1])
    gi, si = sph.PHASE_NAMES.index("gather"), sph.PHASE_NAMES.index("scatter")
    # one gather and one scatter per pass instead of two of each
    assert launches[0][gi] < launches[1][gi] and launches[0][si] < launches[1][si]


def test_set_union_validates(sph):
    f, lay, aos_h, ncell = _tiny()
    v = H.new_view(lay, 0, aos_h.shape[0], f["box"], ncell)
    try:
        for bad in (2, -1):
            assert sph.lib().sph_view_set_union(v, bad) == sph.SPH_E_INVAL
        assert sph.lib().sph_view_set_union(v, 0) == sph.SPH_OK
    finally:
        sph.sph_view_destroy(v)


@pytest.mark.parametrize("prec", [0, 1])
def test_warps_per_cell(sph, oracle, side_stream, prec):
    """8 warps per cell: FP64 results bit-identical to 4 warps (each local particle keeps one warp and the same
    queue order); FP32 within its bar of the oracle (the lanes split each particle's candidates differently)."""
    f = wl.jittered_lattice(20, jitter=0.1, vel_sigma=0.1, seed=9)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay)
    n = aos_h.shape[0]
    ncell = wl.ncell_for(f["box"], f["h"].max())
    outs = []
    for warps in (4, 8):
        aos = H.to_dev(aos_h)
        v = sph.sph_view_create(lay, prec, n, (f["box"], ncell, True), side_stream.cuda_stream)
        try:
            sph.sph_view_set_warps(v, warps, warps)
            sph.sph_step(v, aos, n, wl.SPH_PARAMS)
            sph.sph_view_sync(v)
            assert sph.sph_view_get_tuning(v)[2:] == (warps, warps)
            outs.append(aos.cpu().numpy())
        finally:
            sph.sph_view_destroy(v)
    if prec == 0:
        assert np.array_equal(outs[0], outs[1])
    ref = oracle.step_all(aos_h, lay, f["box"], wl.SPH_PARAMS)
    H.compare_fields(oracle.unpack(outs[1], lay), ref, prec, "8 warps")


@pytest.mark.parametrize("prec", [0, 1])
def test_warps_per_cell_patches(sph, oracle, side_stream, prec):
    import torch
    fp = wl.patches(12, lam_lo=8, lam_hi=150, seed=11, vel_sigma=0.2)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(fp, lay, order="shuffled", segments=fp["patch_start"])
    n = aos_h.shape[0]
    ps = torch.tensor(fp["patch_start"], device=H.device())
    aos = H.to_dev(aos_h)
    v = sph.sph_patches_create(lay, prec, n, 12, fp["box"], 8, side_stream.cuda_stream)
    try:
        sph.sph_view_set_warps(v, 8, 8)
        sph.sph_patches_step(v, aos, n, ps, 12, wl.SPH_PARAMS)
        sph.sph_view_sync(v)
        out = aos.cpu().numpy()
    finally:
        sph.sph_view_destroy(v)
    ref = oracle.step_patches(aos_h, lay, fp["patch_start"], fp["box"], wl.SPH_PARAMS)
    H.compare_fields(oracle.unpack(out, lay), ref, prec, "patches, 8 warps")


def test_set_warps_validates(sph):
    f, lay, aos_h, ncell = _tiny()
    v = H.new_view(lay, 0, aos_h.shape[0], f["box"], ncell)
    try:
        for bad in ((2, 4), (4, 16), (-4, 4)):
            with pytest.raises(sph.SphError) as e:
                sph.sph_view_set_warps(v, *bad)
            assert e.value.status == sph.SPH_E_INVAL
        assert sph.sph_view_get_tuning(v) == (0, 0, 4, 8)    # FP64 view: the force loop defaults to 8 warps
    finally:
        sph.sph_view_destroy(v)
