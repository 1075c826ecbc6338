"""The checked build (compiled with -DSPH_CHECKED, paper_2502_16517_gb300/_build_checked/libsph.so): every index the
kernels read from device data (a cell's slot range, a neighbour cell and its slot range, a work-list entry, a
placement slot, a permutation entry) is range-checked on the device, and a failed check sets SPH_DEV_BOUNDS in
the view's status word instead of accessing out of range.  It stands in for a memory checker where none can run.

A process loads one build, so the checks run in a child process with SPH_CHECKED=1:
  - the parity suites of the pair loops, the conversions, the batched form and the leapfrog, against the checked
    library: an out-of-range index anywhere would surface as SPH_E_DEVICE at the tests' sync;
  - a host-made bad index (one cell_start entry overwritten past the particle count after binning), which the
    checked build must report as SPH_DEV_BOUNDS.  That test refuses to run unless the loaded library says it is
    the checked build, so the default build never sees the bad index."""
import os
import subprocess
import sys

import numpy as np
import pytest

import helpers as H
from paper_2502_16517_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
IN_CHILD = os.environ.get("SPH_CHECKED", "") == "1"
SUITES = ["tests/test_gpu_pairs.py", "tests/test_gpu_convert.py", "tests/test_gpu_staged.py",
          "tests/test_gpu_patches.py", "tests/test_gpu_kdk.py"]


@pytest.mark.skipif(IN_CHILD, reason="the child process runs the suites themselves")
def test_checked_build_passes_the_parity_suites():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_16517_gb300 import build as b
    b.build(checked=True)
    env = dict(os.environ, SPH_CHECKED="1")
    cmd = [sys.executable, "-m", "pytest", "-x", "-q", "-rp", "-p", "no:cacheprovider", "-m", "gpu"] + SUITES + [
        "tests/test_gpu_checked.py::test_checked_build_reports_a_bad_cell_start"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=1500)
    tail = (r.stdout + r.stderr)[-3000:]
    assert r.returncode == 0, tail
    for prec in (0, 1):  # the bad-index test ran (it skips outside the checked build)
        assert f"PASSED tests/test_gpu_checked.py::test_checked_build_reports_a_bad_cell_start[{prec}]" in r.stdout, tail


@pytest.mark.skipif(not IN_CHILD, reason="runs in the checked build's child process only")
@pytest.mark.parametrize("prec", [0, 1])
def test_checked_build_reports_a_bad_cell_start(prec):
    import torch
    from paper_2502_16517_gb300 import sph
    assert sph.sph_build_info() == 1, "not the checked build: the bad index must not reach the default build"
    f = wl.jittered_lattice(12, jitter=0.2, seed=4)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
    n = aos_h.shape[0]
    ncell = wl.ncell_for(f["box"], f["h"].max())
    aos = H.to_dev(aos_h)
    v = H.new_view(lay, prec, n, f["box"], ncell)
    try:
        sph.sph_bin(v, aos, n)
        sph.sph_aos_to_soa(v, aos, n, sph.SPH_DENSITY_IN)
        sph.sph_view_sync(v)
        assert sph.sph_view_status(v) == 0
        ptr = sph.sph_view_index(v, 1)  # cell_start, int32, ncells + 1 entries

        class _Ref:  # a view of the device array for torch (CUDA array interface)
            __cuda_array_interface__ = {"shape": (int(np.prod(ncell)) + 1,), "typestr": "<i4", "data": (ptr, False),
                                        "version": 3}

        cell_start = torch.as_tensor(_Ref(), device=H.device())
        cell_start[5] = n + 1000  # past the particle count: cells 4 and 5 get impossible slot ranges
        torch.cuda.synchronize()
        sph.sph_density(v, wl.SPH_PARAMS)
        with pytest.raises(sph.SphError) as e:
            sph.sph_view_sync(v)
        assert e.value.status == sph.SPH_E_DEVICE
        bits = sph.sph_view_status(v, clear=True)
        assert bits & sph.SPH_DEV_BOUNDS, bits
        assert not bits & sph.SPH_DEV_POS_RANGE, bits
    finally:
        sph.sph_view_destroy(v)
