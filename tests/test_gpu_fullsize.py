"""Full-size parity of the plain 262,144-particle workload in the launch configuration the benchmark times (the
autotuner's tiles and warps per cell, one view for both loops, sph_step), element by element against the oracle
on two 12^3-spacing cubes: the benchmark's own sample cube (1,728 force targets, their 2h halo's densities) and a
cube around the box corner, whose particles reach their neighbours across all three periodic faces.

Bars per field, as everywhere: rho, P, c_s relative per particle; a and du/dt normwise (max |err| / max |ref| over
the cube); 1e-12 for FP64, 2e-5 for FP32."""
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


def _cores():
    import os
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


@pytest.fixture(scope="module")
def plain_cubes(oracle):
    f = wl.plain()
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
    st = oracle.unpack(aos_h, lay)
    s = 1.0 / 64
    halo = 2.0 * float(f["h"].max()) * (1 + 1e-9)
    centres = {"bench": np.random.default_rng(0).uniform(0.2, 0.8, size=3),   # the benchmark's sample cube
               "corner": np.zeros(3)}                                         # straddles every periodic face
    cubes = {k: oracle.cube_sample(st, f["box"], wl.SPH_PARAMS, c, 0.5 * 12 * s, halo, threads=_cores())
             for k, c in centres.items()}
    return f, lay, aos_h, cubes


def _bench_step(sph, aos_h, lay, box, ncell, prec, tmp_path):
    """One sph_step exactly as the benchmark's timed step runs it (fresh autotuner cache)."""
    import torch
    from paper_2502_16517_gb300 import autotune
    n = aos_h.shape[0]
    aos = H.to_dev(aos_h)
    v = H.new_view(lay, prec, n, box, ncell)
    try:
        key = autotune.cache_key(torch.cuda.get_device_name(H.device()), prec, "grid", n / float(np.prod(ncell)))
        tiles = autotune.tuned_tiles(v, aos, n, wl.SPH_PARAMS, key, str(tmp_path / "tiles.json"))
        sph.sph_step(v, aos, n, wl.SPH_PARAMS)
        sph.sph_view_sync(v)
        out = aos.cpu().numpy()
    finally:
        sph.sph_view_destroy(v)
    return out, tiles


@pytest.mark.parametrize("prec", [0, 1])
def test_plain_full_size_cubes_match_oracle(sph, oracle, plain_cubes, prec, tmp_path):
    f, lay, aos_h, cubes = plain_cubes
    ncell = wl.ncell_for(f["box"], f["h"].max())
    assert aos_h.shape[0] == 262144 and tuple(ncell) == (26, 26, 26)
    out, tiles = _bench_step(sph, aos_h, lay, f["box"], ncell, prec, tmp_path)
    got = oracle.unpack(out, lay)
    tol = H.TOL[prec]
    for name, c in cubes.items():
        assert c["block"].size > 1500 and c["halo"].size > c["block"].size
        errs = {k: H.rel_max(got[k][c["halo"]], c[k]) for k in ("rho", "P", "cs")}
        errs.update({k: H.normwise(got[k][c["block"]], c[k]) for k in ("a", "dudt")})
        bad = {k: e for k, e in errs.items() if not e <= tol}
        assert not bad, f"{name} cube, prec {prec}, tiles {tiles}: {errs}"
