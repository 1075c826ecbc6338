"""sph_bin_static: cell bucketing for callers that may not allocate device memory (inside an allocator
callback, under a framework that owns all device memory, or in a loop with a no-allocation rule).

It keeps its intermediate arrays in one fixed device array inside the library instead of a view.  Its outputs
must equal the oracle's stable counting sort and sph_bin's (index work, so bit-exact), call after call.  The
calls below run back to back on different inputs: a larger grid first, then a smaller one, then the larger one
again, so that leftovers of a larger call in the shared array would show in the next.  One input has more cells
than one scan block covers, so the multi-block scan and its scratch in the fixed array run too.  This file is
named to be collected last, so a failure here cannot hide failures of the other tests.
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


def _uniform(n, seed, h):
    rng = np.random.default_rng(seed)
    return {"x": rng.uniform(0, 1, size=(n, 3)), "v": np.zeros((n, 3)), "mass": np.full(n, 1.0 / max(n, 1)),
            "h": np.full(n, h), "u": np.ones(n), "box": np.ones(3)}


def _inputs():
    """(fields, ncell): 40^3 = 64,000 cells (more than one scan block), 6^3 cells, 12^3 cells."""
    big = (_uniform(5000, 41, 0.0124), np.array([40, 40, 40], np.int32))
    a = wl.jittered_lattice(16, jitter=0.1, vel_sigma=0.1)                      # 4096 particles, 6^3 cells
    lat = (a, wl.ncell_for(a["box"], a["h"].max()))
    mid = (_uniform(3001, 31, 0.04), np.array([12, 12, 12], np.int32))
    return [big, lat, mid, big]


def _view_bin(sph, aos, lay, f, ncell, n):
    v = H.new_view(lay, sph.SPH_F64, max(n, 1), f["box"], ncell)
    try:
        sph.sph_bin(v, aos, n)
        sph.sph_view_sync(v)
        return (sph.sph_view_export_index(v, 0, n), sph.sph_view_export_index(v, 1, int(np.prod(ncell)) + 1),
                sph.sph_view_export_index(v, 2, n))
    finally:
        sph.sph_view_destroy(v)


def _static_bin(sph, lay, f, ncell, aos, n, with_status):
    import torch
    dev = H.device()
    ncells = int(np.prod(ncell))
    perm = torch.full((max(n, 1),), -1, dtype=torch.int32, device=dev)
    start = torch.full((ncells + 1,), -1, dtype=torch.int32, device=dev)
    cos = torch.full((max(n, 1),), -1, dtype=torch.int32, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev) if with_status else None
    sph.sph_bin_static(lay, (f["box"], ncell, True), aos, n, perm, start, cos, status, H.stream())
    torch.cuda.synchronize(dev)
    st = int(status.item()) if with_status else 0
    return perm.cpu().numpy()[:n], start.cpu().numpy(), cos.cpu().numpy()[:n], st


def test_static_bin_matches_oracle_and_view_bin_on_consecutive_calls(sph, oracle):
    lay = wl.default_layout()
    for k, (f, ncell) in enumerate(_inputs()):
        aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
        n = aos_h.shape[0]
        rec = oracle.unpack(aos_h, lay)
        _, o_start, o_perm, o_cos, bad = oracle.bin_cells(rec["x"], f["box"], ncell)
        assert bad == 0
        aos = H.to_dev(aos_h)
        ref = _view_bin(sph, aos, lay, f, ncell, n)
        # every other call leaves the status word to the library (status_dev = NULL)
        perm, start, cos, st = _static_bin(sph, lay, f, ncell, aos, n, with_status=(k % 2 == 0))
        for got, o, r, name in ((perm, o_perm, ref[0], "perm"), (start, o_start, ref[1], "cell_start"),
                                (cos, o_cos, ref[2], "cell_of_slot")):
            np.testing.assert_array_equal(got, o, err_msg=f"input {k}: {name} vs oracle")
            np.testing.assert_array_equal(got, r, err_msg=f"input {k}: {name} vs sph_bin")
        assert st == 0


def test_static_bin_no_particles(sph, oracle):
    import torch
    lay = wl.default_layout()
    ncell = np.array([5, 5, 5], np.int32)
    f = _uniform(0, 1, 0.1)
    _, o_start, _, _, _ = oracle.bin_cells(np.zeros((0, 3)), f["box"], ncell)
    # once with placeholder arrays, once with NULL per-particle arrays (allowed when n = 0)
    aos = torch.zeros((1, lay["stride"]), dtype=torch.uint8, device=H.device())
    perm, start, cos, st = _static_bin(sph, lay, f, ncell, aos, 0, with_status=True)
    np.testing.assert_array_equal(start, o_start)
    assert st == 0 and perm.size == 0 and cos.size == 0
    start = torch.full((126,), -1, dtype=torch.int32, device=H.device())
    sph.sph_bin_static(lay, (f["box"], ncell, True), None, 0, None, start, None, None, H.stream())
    torch.cuda.synchronize(H.device())
    np.testing.assert_array_equal(start.cpu().numpy(), o_start)


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
