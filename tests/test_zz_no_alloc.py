"""sph_bin_static: cell bucketing for callers that may not allocate device memory (inside an allocator
callback, under a framework that owns all device memory, or in a loop with a no-allocation rule).

It keeps its intermediate arrays in one fixed device array inside the library instead of a view.  Its outputs
must be identical to sph_bin's (index work, so bit-exact), call after call.  The calls below run back to back
on different inputs, so a call that left stale scratch behind would corrupt the next one.  This file is named to
be collected last, so a failure here cannot hide failures of the other tests.
"""
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


def _inputs():
    a = wl.jittered_lattice(16, jitter=0.1, vel_sigma=0.1)                      # 4096 particles, 6^3 cells
    rng = np.random.default_rng(31)
    n = 3001
    b = {"x": rng.uniform(0, 1, size=(n, 3)), "v": np.zeros((n, 3)), "mass": np.full(n, 1.0 / n),
         "h": np.full(n, 0.04), "u": np.ones(n), "box": np.ones(3)}                # 3001 particles, 12^3 cells
    return [(a, wl.ncell_for(a["box"], a["h"].max())), (b, np.array([12, 12, 12], np.int32))]


def _view_bin(sph, aos, lay, f, ncell, n):
    v = H.new_view(lay, sph.SPH_F64, n, f["box"], ncell)
    try:
        sph.sph_bin(v, aos, n)
        sph.sph_view_sync(v)
        return (sph.sph_view_export_index(v, 0, n), sph.sph_view_export_index(v, 1, int(np.prod(ncell)) + 1),
                sph.sph_view_export_index(v, 2, n))
    finally:
        sph.sph_view_destroy(v)


def test_static_bin_matches_view_bin_on_consecutive_calls(sph):
    import torch
    dev = H.device()
    lay = wl.default_layout()
    for f, ncell in _inputs():
        aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
        n = aos_h.shape[0]
        aos = H.to_dev(aos_h)
        ref = _view_bin(sph, aos, lay, f, ncell, n)
        ncells = int(np.prod(ncell))
        perm = torch.full((n,), -1, dtype=torch.int32, device=dev)
        start = torch.full((ncells + 1,), -1, dtype=torch.int32, device=dev)
        cos = torch.full((n,), -1, dtype=torch.int32, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        sph.sph_bin_static(lay, (f["box"], ncell, True), aos, n, perm, start, cos, status, H.stream())
        torch.cuda.synchronize(dev)
        np.testing.assert_array_equal(perm.cpu().numpy(), ref[0])
        np.testing.assert_array_equal(start.cpu().numpy(), ref[1])
        np.testing.assert_array_equal(cos.cpu().numpy(), ref[2])
        assert int(status.item()) == 0


def test_static_bin_rejects_sizes_beyond_capacity(sph):
    import torch
    lay = wl.default_layout()
    dev = H.device()
    aos = torch.zeros((8, lay["stride"]), dtype=torch.uint8, device=dev)
    out = torch.zeros(8, dtype=torch.int32, device=dev)
    with pytest.raises(sph.SphError) as e:
        sph.sph_bin_static(lay, (np.ones(3), (64, 64, 64), True), aos, 8, out, out, out, None, H.stream())
    assert e.value.status == sph.SPH_E_INVAL                      # 262,144 cells > SPH_BIN_STATIC_MAX_CELLS
    with pytest.raises(sph.SphError) as e:
        sph.sph_bin_static(lay, (np.ones(3), (4, 4, 4), True), aos, sph.SPH_BIN_STATIC_MAX_PARTICLES + 1,
                           out, out, out, None, H.stream())
    assert e.value.status == sph.SPH_E_INVAL
