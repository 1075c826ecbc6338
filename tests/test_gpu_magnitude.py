"""Units far from 1.  The FP64 pair loops refine FP32-seeded reciprocals and square roots of r^2 and of
(r^2 + eps hbar^2)(rho_i + rho_j), so they need 2^-50 <= h < 2^50 and 2^-105 <= h^2 rho < 2^105 (those inputs then
stay in the float range); the set-up kernels flag a particle outside these bounds with SPH_DEV_MAGNITUDE.

One workload is scaled in length: x, the box, h and v by s, the masses by s^3, so rho is unchanged.  Well inside
the bounds (s = 2^40 and 2^-40: h near 2^37 and 2^-43) the FP64 step still meets the oracle bar; beyond them
(s = 2^56 and 2^-56) the FP64 view reports the flag.  Only arithmetic sees the scaled values: every index the
kernels form comes from the binning, which the scaling leaves alone."""
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


def _scaled(s):
    f = wl.jittered_lattice(12, jitter=0.2, vel_sigma=0.3, seed=21)
    g = dict(f)
    for k in ("x", "box", "h", "v"):
        g[k] = f[k] * s
    g["mass"] = f["mass"] * s ** 3
    return g


@pytest.mark.parametrize("s", [2.0 ** 40, 2.0 ** -40])
def test_fp64_step_at_far_scales_matches_oracle(sph, oracle, s):
    f = _scaled(s)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
    ncell = wl.ncell_for(f["box"], f["h"].max())
    out, info = H.run_step(aos_h, lay, f["box"], ncell, 0, separate_calls=False)   # syncs: no status bit set
    got = oracle.unpack(out, lay)
    ref = oracle.step_all(aos_h, lay, f["box"], wl.SPH_PARAMS)
    h2rho = f["h"] ** 2 * ref["rho"]
    assert 2.0 ** -50 <= f["h"].min() and f["h"].max() < 2.0 ** 50
    assert 2.0 ** -105 <= h2rho.min() and h2rho.max() < 2.0 ** 105
    H.compare_fields(got, ref, 0, f"scale {s:g}")


@pytest.mark.parametrize("s", [2.0 ** 56, 2.0 ** -56])
def test_fp64_view_flags_smoothing_lengths_outside_the_bounds(sph, s):
    f = _scaled(s)
    assert not (2.0 ** -50 <= f["h"].min() and f["h"].max() < 2.0 ** 50)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
    n = aos_h.shape[0]
    ncell = wl.ncell_for(f["box"], f["h"].max())
    aos = H.to_dev(aos_h)
    v = H.new_view(lay, sph.SPH_F64, n, f["box"], ncell)
    try:
        sph.sph_step(v, aos, n, wl.SPH_PARAMS)
        with pytest.raises(sph.SphError) as e:
            sph.sph_view_sync(v)
        assert e.value.status == sph.SPH_E_DEVICE
        bits = sph.sph_view_status(v, clear=True)
        assert bits & sph.SPH_DEV_MAGNITUDE, bits
        assert not bits & sph.SPH_DEV_POS_RANGE, bits
    finally:
        sph.sph_view_destroy(v)
