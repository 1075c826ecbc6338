"""Shared helpers for the tests: run the CUDA path through the C ABI and compare with the oracle."""
import numpy as np

from paper_2502_16517_gb300 import workloads as wl

TOL = {0: 1e-12, 1: 2e-5}  # FP64 path, FP32 path: relative error bars against the FP64 oracle


def device():
    import torch
    return torch.device("cuda:0")


def stream():
    import torch
    return torch.cuda.current_stream(device()).cuda_stream


def to_dev(aos_h):
    import torch
    return torch.from_numpy(np.ascontiguousarray(aos_h)).to(device())


def new_view(lay, prec, n_max, box, ncell, periodic=True):
    from paper_2502_16517_gb300 import sph
    return sph.sph_view_create(lay, prec, n_max, (box, ncell, periodic), stream())


def run_step(aos_h, lay, box, ncell, prec, periodic=True, params=None, separate_calls=True):
    """One pass (bin, gather, density, scatter, gather, force, scatter) on the GPU; returns (aos_out, info)."""
    from paper_2502_16517_gb300 import sph
    params = params or wl.SPH_PARAMS
    n = aos_h.shape[0]
    aos = to_dev(aos_h)
    v = new_view(lay, prec, max(n, 1), box, ncell, periodic)
    try:
        if separate_calls:
            sph.sph_bin(v, aos, n)
            sph.sph_aos_to_soa(v, aos, n, sph.SPH_DENSITY_IN)
            sph.sph_density(v, params)
            sph.sph_soa_to_aos(v, aos, n, sph.SPH_DENSITY_OUT)
            sph.sph_aos_to_soa(v, aos, n, sph.SPH_FORCE_IN)
            sph.sph_force(v, params)
            sph.sph_soa_to_aos(v, aos, n, sph.SPH_FORCE_OUT)
        else:
            sph.sph_step(v, aos, n, params)
        sph.sph_view_sync(v)
        info = {
            "perm": sph.sph_view_export_index(v, 0, n),
            "counts": sph.sph_pair_counts(v),
            "reduce": sph.sph_reduce(v) if n else None,
        }
        out = aos.cpu().numpy()
    finally:
        sph.sph_view_destroy(v)
    return out, info


def rel_max(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    return float(np.max(np.abs(got - ref) / np.abs(ref))) if ref.size else 0.0


def normwise(got, ref):
    got, ref = np.asarray(got, np.float64), np.asarray(ref, np.float64)
    if ref.size == 0:
        return 0.0
    scale = np.max(np.abs(ref))
    return float(np.max(np.abs(got - ref)) / scale) if scale > 0 else float(np.max(np.abs(got)))


def compare_fields(got, ref, prec, label=""):
    """Per-field errors (relative for rho, P, cs; normwise for a and du/dt) against the stated bar."""
    tol = TOL[prec]
    errs = {
        "rho": rel_max(got["rho"], ref["rho"]),
        "P": rel_max(got["P"], ref["P"]),
        "cs": rel_max(got["cs"], ref["cs"]),
        "a": normwise(got["a"], ref["a"]),
        "dudt": normwise(got["dudt"], ref["dudt"]),
    }
    bad = {k: v for k, v in errs.items() if not (v <= tol)}
    assert not bad, f"{label} errors above {tol}: {bad} (all: {errs})"
    return errs


def written_mask(lay, names):
    m = np.zeros(lay["stride"], bool)
    for nm in names:
        o = lay["offsets"][nm]
        m[o:o + 8 * wl.NCOMP[nm]] = True
    return m
