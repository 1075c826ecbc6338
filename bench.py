#!/usr/bin/env python3
"""Benchmark of the SPH view path on GB300: pair interactions per second including the AoS<->SoA view conversions.

Workload (the plain FP64 configuration): 262,144 particles on a 64^3 lattice jittered by U(-0.1, 0.1) * spacing,
v ~ N(0, 0.1), equal mass, cubic spline with h = 1.2 spacing, 26^3 periodic cells of edge >= 2h, ideal gas
gamma = 5/3, u = 1, in 160-byte AoS records stored in a seeded random order (heap-scattered records).  One step =
sph_step: bin, gather the density view, density loop, scatter rho/P/c_s, gather the force view, force loop,
scatter a/du/dt.  value = (density pairs incl. self + ordered force pairs) per step / device time per step.
The AoS (42 MB) fits in the 129 MB L2, so a 256 MB buffer is written between timed steps (outside the events).

Also reported: the FP32 form on the same input (forms.f32), the end-to-end figure through sph_step_host with
pinned host records (copies inside the timed region), per-phase device times, conversion bandwidth, the
roofline of the dominant kernel, SM clocks sampled during the timed region, and the FP64 CPU oracle timed on a
bounded sample of the same workload (cpu_baseline).  --impl reference times that oracle alone.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "pair interactions/sec incl. AoS<->SoA conversion, FP32 vs FP64; conversion HBM GB/s"
UNIT = "pair interactions/s"
WORKLOAD = ("plain FP64 method: 262,144 particles, jittered 64^3 lattice, v ~ N(0,0.1), cubic spline h=1.2 s, "
            "26^3 periodic cells, 160 B AoS records in scattered order, one density + force pass with view "
            "conversion in and out")

# Algorithmic FP64/FP32 flops per in-support pair, counted from the pair terms of the loop bodies (one kernel
# piece per pair, the viscosity block for half of the pairs): density 17, force 64.
FLOPS_DENSITY_PAIR = 17
FLOPS_FORCE_PAIR = 64
# ALU peaks derived from unit counts and clocks: FP32 = 152 SMs x 128 lanes x 2 flops x 2.07 GHz;
# FP64 = the GB300's nominal 1.25 TFLOP/s.
PEAK_FP32_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
PEAK_FP64_TFLOPS = 1.25


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return {}


# ----------------------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------------------------------
class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        # the raw samples (the line carries their summary): SPH_BENCH_CLOCKS_DIR, else the temp directory
        import tempfile
        out_dir = os.environ.get("SPH_BENCH_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(out_dir, f"clocks_bench_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.QUERY}",
                                          "--format=csv,noheader,nounits", "-lms", "50"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return None
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    mx.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------------------------------------
# the GPU arm
# ----------------------------------------------------------------------------------------------------------
def _inputs():
    from paper_2502_16517_gb300 import workloads as wl
    f = wl.plain()
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled")
    ncell = wl.ncell_for(f["box"], f["h"].max())
    return f, lay, aos_h, ncell


def run_form(prec, steps, warmup, dev, aos_h, lay, box, ncell, clocks_gpu=None, tune_cache=None, union=True,
             params=None, tune_form="grid", flush_l2=True, keep_out=False):
    import torch
    from paper_2502_16517_gb300 import autotune, sph
    from paper_2502_16517_gb300 import workloads as wl
    params = params or wl.SPH_PARAMS
    n = aos_h.shape[0]
    aos = torch.from_numpy(aos_h).to(dev)
    stream = torch.cuda.current_stream(dev)
    view = sph.sph_view_create(lay, prec, n, (box, ncell, True), stream.cuda_stream)
    if not union:
        sph.sph_view_set_union(view, False)
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)  # 256 MB > 129 MB L2
    tiles = None
    try:
        if tune_cache:
            key = autotune.cache_key(torch.cuda.get_device_name(dev), prec, tune_form, n / float(np.prod(ncell)))
            tiles = autotune.tuned_tiles(view, aos, n, params, key, tune_cache)
        for _ in range(max(warmup, 0)):
            if flush_l2:
                flush.zero_()
            sph.sph_step(view, aos, n, params)
        sph.sph_view_sync(view)
        sph.sph_pair_counts(view, reset=True)
        sph.sph_view_timing(view, True)
        sph.sph_view_phase_times(view, reset=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        sampler = ClockSampler(clocks_gpu) if clocks_gpu is not None else None
        if torch.distributed.is_initialized():
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        if sampler:
            sampler.__enter__()
        try:
            for k in range(steps):
                if flush_l2:
                    flush.zero_()
                ev[k][0].record(stream)
                sph.sph_step(view, aos, n, params)
                ev[k][1].record(stream)
            torch.cuda.synchronize(dev)
        finally:
            if sampler:
                sampler.__exit__(None, None, None)
        wall = time.perf_counter() - t0
        if torch.distributed.is_initialized():
            torch.distributed.barrier()
        sph.sph_view_sync(view)
        step_ms = [a.elapsed_time(b) for a, b in ev]
        counts = sph.sph_pair_counts(view)
        phase_ms, launches = sph.sph_view_phase_times(view)
        sph.sph_view_timing(view, False)
        out = aos.cpu().numpy() if keep_out else None      # the records after the last timed step
    finally:
        sph.sph_view_destroy(view)
    return {
        "step_ms": step_ms, "wall_s": wall, "counts": counts, "phase_ms": phase_ms, "launches": launches,
        "clocks": sampler.summary() if sampler else None, "tiles": tiles, "union": union, "out": out,
    }


EXT_PARAMS_NOTE = ("quartic spline M5 (support 5h/2, the paper's kernel) with the fuller views: the density also "
                   "writes the neighbour count, div v, curl v and Omega; the force uses grad-h terms and the Balsara "
                   "switch and writes the signal velocity")


def presorted_aos(aos_h, lay, box, ncell, dev):
    """The plain records rearranged in cell order (the paper's continuous AoS, Section 6): the path's own binning of
    the scattered records gives the slot -> record permutation, and record perm[s] moves to position s.  Host
    preparation outside every timed region."""
    import torch
    from paper_2502_16517_gb300 import sph
    n = aos_h.shape[0]
    stream = torch.cuda.current_stream(dev)
    aos = torch.from_numpy(aos_h).to(dev)
    view = sph.sph_view_create(lay, 0, n, (box, ncell, True), stream.cuda_stream)
    try:
        sph.sph_bin(view, aos, n)
        perm = sph.sph_view_export_index(view, 0, n)
    finally:
        sph.sph_view_destroy(view)
    return np.ascontiguousarray(aos_h[perm])


def extended_inputs():
    """The plain 262,144-particle input on the paper's 272-byte record with the fuller views' members, cells of
    edge >= 5h/2 for the quartic spline."""
    from paper_2502_16517_gb300 import workloads as wl
    f = wl.plain()
    lay = wl.extended_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled", canary=False)
    return lay, aos_h, wl.ncell_for(f["box"], f["h"].max(), 2.5)


def batched_inputs(npatch=4096):
    """The batched workload: 4096 independent 3x3x3-cell patches, Poisson(lambda ~ U(8, 256)) particles per cell,
    v ~ N(0, 0.1) as in the plain workload (records grouped by patch, scattered inside each patch).  Profiling
    runs may take fewer patches of the same distribution."""
    from paper_2502_16517_gb300 import workloads as wl
    fp = wl.patches(npatch, seed=wl.SEED, vel_sigma=0.1)
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(fp, lay, order="shuffled", segments=fp["patch_start"], canary=False)
    return fp, lay, aos_h


def large_inputs():
    """The large-run workload: 2,097,152 clustered particles (8 Gaussian overdensities, sigma 0.05, peak 4x),
    h = 1.2/128, 53^3 periodic cells, v = 0, u = 1."""
    from paper_2502_16517_gb300 import workloads as wl
    f = wl.large()
    lay = wl.default_layout()
    aos_h, _ = wl.pack_aos(f, lay, order="shuffled", canary=False)
    return f, lay, aos_h, wl.ncell_for(f["box"], f["h"].max())


def run_large(prec, reps, dev, f, lay, aos_h, ncell, dt=None, nsteps=10, tune_cache=None):
    """Ten kick-drift-kick steps (initial pass + per step: kick, drift, re-bin, gather, density, scatter, gather,
    force, scatter, kick) as ONE CUDA graph launch per run; each timed run starts from the same initial records
    (restored outside the timed region).  dt = 0.3 min h / max(c_s + |v|) from the initial pass, in FP64."""
    import torch
    from paper_2502_16517_gb300 import autotune, sph
    from paper_2502_16517_gb300 import workloads as wl
    n = aos_h.shape[0]
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        aos0 = torch.from_numpy(aos_h).to(dev)
        aos = aos0.clone()
        view = sph.sph_view_create(lay, prec, n, (f["box"], ncell, True), stream.cuda_stream)
        try:
            stats0 = sph.sph_step(view, aos, n, wl.SPH_PARAMS, want_stats=True)
            if dt is None:
                rec = aos.cpu().numpy()
                hv = rec[:, 80:88].copy().view(np.float64)[:, 0]
                cs = rec[:, 120:128].copy().view(np.float64)[:, 0]
                vv = rec[:, 24:48].copy().view(np.float64)
                dt = 0.3 * hv.min() / np.max(cs + np.linalg.norm(vv, axis=1))
            tiles = None
            if tune_cache:
                key = autotune.cache_key(torch.cuda.get_device_name(dev), prec, "grid", n / float(np.prod(ncell)))
                tiles = autotune.tuned_tiles(view, aos, n, wl.SPH_PARAMS, key, tune_cache)
            aos.copy_(aos0)
            sph.sph_step_graph(view, aos, n, wl.SPH_PARAMS, dt=dt, nsteps=nsteps)  # capture (and one run)
            sph.sph_view_sync(view)
            sph.sph_pair_counts(view, reset=True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
            stats1 = None
            barrier()
            torch.cuda.synchronize(dev)
            for k in range(reps):
                aos.copy_(aos0)
                ev[k][0].record(stream)
                sph.sph_step_graph(view, aos, n, wl.SPH_PARAMS, dt=dt, nsteps=nsteps)
                ev[k][1].record(stream)
            torch.cuda.synchronize(dev)
            counts = sph.sph_pair_counts(view, reset=True)
            out = aos.cpu().numpy()
            stats1 = sph.sph_step(view, aos, n, wl.SPH_PARAMS, want_stats=True)   # sums of the final records
            # the same run with the half-step values in the force (first-order energy error), for comparison
            aos.copy_(aos0)
            sph.sph_view_set_integrator(view, 0)
            sph.sph_step(view, aos, n, wl.SPH_PARAMS, dt=dt, nsteps=nsteps)
            stats_plain = sph.sph_step(view, aos, n, wl.SPH_PARAMS, want_stats=True)
        finally:
            sph.sph_view_destroy(view)
    ms = float(np.sum([a.elapsed_time(b) for a, b in ev]))
    pairs_run = (counts[1] + counts[2]) / reps
    return {"value": pairs_run * reps / (ms / 1e3), "ms_per_run": ms / reps, "pairs_per_run": pairs_run,
            "steps_per_run": nsteps, "passes_per_run": nsteps + 1, "dt": dt, "particles": int(n),
            "energy_rel_drift": float((stats1[6] - stats0[6]) / stats0[6]),
            "energy_rel_drift_half_step_values": float((stats_plain[6] - stats0[6]) / stats0[6]),
            "integrator": "leapfrog KDK, the force after each drift sees the predicted v, u (second kick resets them)",
            "momentum_abs": [float(x) for x in stats1[0:3]], "tiles": tiles, "dtype": "f64" if prec == 0 else "f32",
            "graph": "one CUDA graph launch per ten-step run"}, out


def cfl_dt(rec, lay, courant=0.3):
    """dt = courant * min h / max(c_s + |v|), in FP64 from records after a pass (host copy)."""
    o = lay["offsets"]
    hv = rec[:, o["h"]:o["h"] + 8].copy().view(np.float64)[:, 0]
    cs = rec[:, o["cs"]:o["cs"] + 8].copy().view(np.float64)[:, 0]
    vv = rec[:, o["v"]:o["v"] + 24].copy().view(np.float64)
    return float(courant * hv.min() / np.max(cs + np.linalg.norm(vv, axis=1)))


def run_batched(prec, steps, warmup, dev, fp, lay, aos_h, tune_cache=None, ncap=8):
    """One leapfrog step over all patches per graph launch: kick + drift (reflecting patch walls), bin, work list,
    gather (with the predicted v, u), density, force, scatter, kick.  An initial pass (outside the timed region)
    gives a, du/dt; then SPH_KDK_CONTINUE makes every launch exactly one step of one continuing run.  dt is the
    CFL step of the initial state.  Per-phase times from one extra un-captured step with event timing."""
    import torch
    from paper_2502_16517_gb300 import autotune, sph
    from paper_2502_16517_gb300 import workloads as wl
    n = aos_h.shape[0]
    npatch = len(fp["patch_start"]) - 1
    stream = torch.cuda.Stream(device=dev)
    with torch.cuda.stream(stream):
        aos = torch.from_numpy(aos_h).to(dev)
        ps = torch.tensor(fp["patch_start"], dtype=torch.int64, device=dev)
        view = sph.sph_patches_create(lay, prec, n, npatch, fp["box"], ncap, stream.cuda_stream)
        try:
            sph.sph_patches_bin(view, aos, n, ps, npatch)
            tiles = None
            if tune_cache:
                key = autotune.cache_key(torch.cuda.get_device_name(dev), prec, "patches", float(fp["lam"].mean()))
                tiles = autotune.tuned_tiles(view, aos, n, wl.SPH_PARAMS, key, tune_cache)
            e0 = sph.sph_patches_step(view, aos, n, ps, npatch, wl.SPH_PARAMS, want_stats=True)
            dt = cfl_dt(aos.cpu().numpy(), lay)
            sph.sph_view_set_integrator(view, sph.SPH_KDK_PREDICT | sph.SPH_KDK_CONTINUE)
            for _ in range(max(warmup, 1)):
                sph.sph_patches_step_graph(view, aos, n, ps, npatch, wl.SPH_PARAMS, dt=dt, nsteps=1)
            sph.sph_view_sync(view)
            sph.sph_pair_counts(view, reset=True)
            sph.sph_view_phase_times(view, reset=True)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
            barrier()
            torch.cuda.synchronize(dev)
            for k in range(steps):
                ev[k][0].record(stream)
                sph.sph_patches_step_graph(view, aos, n, ps, npatch, wl.SPH_PARAMS, dt=dt, nsteps=1)
                ev[k][1].record(stream)
            torch.cuda.synchronize(dev)
            sph.sph_view_sync(view)
            step_ms = [a.elapsed_time(b) for a, b in ev]
            counts = sph.sph_pair_counts(view, reset=True)
            _, launches = sph.sph_view_phase_times(view, reset=True)
            # phase breakdown (outside the timed region): one more step, un-captured, with event timing
            sph.sph_view_timing(view, True)
            e1 = sph.sph_patches_step(view, aos, n, ps, npatch, wl.SPH_PARAMS, dt=dt, nsteps=1, want_stats=True)
            phase_ms, _ = sph.sph_view_phase_times(view, reset=True)
            sph.sph_view_timing(view, False)
            sph.sph_view_sync(view)
            x = aos.cpu().numpy()[:, lay["offsets"]["x"]:lay["offsets"]["x"] + 24].copy().view(np.float64)
        finally:
            sph.sph_view_destroy(view)
    ms = float(np.sum(step_ms))
    pairs_step = (counts[1] + counts[2]) / steps
    nrun = max(warmup, 1) + steps + 1
    return {"value": pairs_step * steps / (ms / 1e3), "ms_per_step": ms / steps, "pairs_per_step": pairs_step,
            "particles": int(n), "patches": int(npatch), "dt": dt, "steps_run": nrun,
            "energy_rel_change": float((e1[6] - e0[6]) / e0[6]),
            "positions_inside_patch_boxes": bool(np.all((x >= 0.0) & (x <= 3.0))),
            "phases_ms": {nm: float(phase_ms[i]) for i, nm in enumerate(sph.PHASE_NAMES)},
            "gpu_launches": int(launches.sum()), "tiles": tiles, "dtype": "f64" if prec == 0 else "f32",
            "graph": ("one CUDA graph launch per leapfrog step: kick + drift, bin, work list, gather, density, "
                      "force, scatter, kick"),
            "kdk": "fused: the first kick and the drift run in the bin kernel, the second kick in the scatter kernel"}


def run_e2e(prec, steps, warmup, dev, aos_h, lay, box, ncell, direct=False):
    """sph_step_host on pinned host records, every step: staged (H2D copy of the records, the pass, D2H copy of the
    records) or in place (direct: the bin and gather kernels read the view members from the host records, the
    scatter writes the written members back, across the host link)."""
    import torch
    from paper_2502_16517_gb300 import sph
    from paper_2502_16517_gb300 import workloads as wl
    n = aos_h.shape[0]
    host = torch.from_numpy(aos_h.copy()).pin_memory()
    stream = torch.cuda.current_stream(dev)
    view = sph.sph_view_create(lay, prec, n, (box, ncell, True), stream.cuda_stream)
    try:
        sph.sph_view_set_host_direct(view, direct)
        for _ in range(max(warmup, 1)):
            sph.sph_step_host(view, host, n, wl.SPH_PARAMS)
        sph.sph_pair_counts(view, reset=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(steps):
            sph.sph_step_host(view, host, n, wl.SPH_PARAMS)
        torch.cuda.synchronize(dev)
        wall = time.perf_counter() - t0
        counts = sph.sph_pair_counts(view)
    finally:
        sph.sph_view_destroy(view)
    pairs = (counts[1] + counts[2])
    if direct:
        # algorithmic member bytes across the link: x for binning, the union view {x, v, m, h, u} for the gather;
        # {rho, P, cs, a, du/dt} written back
        h2d, d2h = n * (3 + 9) * 8, n * 7 * 8
    else:
        h2d = d2h = n * lay["stride"]
    return {"value": pairs / wall, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
            "ms_per_step": wall * 1e3 / steps, "mode": "in place" if direct else "staged copies"}


def conversion_bytes(prec, n, union=True):
    """Algorithmic bytes of the view conversions of one pass (read + written, incl. the 4-byte perm read; FP32
    positions also read the 4-byte cell of the slot).  Union view: one gather of {x,m,h,u,v}, one scatter of
    {rho,P,cs,a,dudt}; per-loop views: gather {x,m,h,u} and {x,v,m,h,rho,P,cs}, scatter {rho,P,cs} and {a,dudt}."""
    e = 8 if prec == 0 else 4
    pos_extra = 0 if prec == 0 else 4
    if union:
        return n * (9 * 8 + 9 * e + 4 + pos_extra), n * (7 * 8 + 7 * e + 4)
    gather_d = n * (6 * 8 + 6 * e + 4 + pos_extra)
    gather_f = n * (11 * 8 + 11 * e + 4 + pos_extra)
    scatter_d = n * (3 * 8 + 3 * e + 4)
    scatter_f = n * (4 * 8 + 4 * e + 4)
    return gather_d + gather_f, scatter_d + scatter_f


def summarize_form(prec, r, n, steps, world):
    from paper_2502_16517_gb300 import sph
    ms = float(np.sum(r["step_ms"]))
    pairs_step = (r["counts"][1] + r["counts"][2]) / steps
    value = world * pairs_step * steps / (ms / 1e3)
    ph = {name: float(r["phase_ms"][i]) / steps for i, name in enumerate(sph.PHASE_NAMES)}
    nl = {name: int(r["launches"][i]) for i, name in enumerate(sph.PHASE_NAMES)}
    g_bytes, s_bytes = conversion_bytes(prec, n, r.get("union", True))
    # the bin and the gather run as one record pass plus a permutation (phases bin and gather together give the
    # SoA view in slot order)
    bg_ms = ph["bin"] + ph["gather"]
    conv = {
        "bin_and_gather_GBps": g_bytes / (bg_ms * 1e-3) / 1e9 if bg_ms > 0 else None,
        "scatter_GBps": s_bytes / (ph["scatter"] * 1e-3) / 1e9 if ph["scatter"] > 0 else None,
        "gather_bytes_per_step": g_bytes, "scatter_bytes_per_step": s_bytes,
        "bytes": "algorithmic: view members read from the records and written to the SoA (and back), plus perm",
    }
    # the paper's normalisation: cost per particle update of each loop, and of the whole step
    upd = {"density_ns": ph["density"] * 1e6 / n, "force_ns": ph["force"] * 1e6 / n,
           "step_ns": ms / steps * 1e6 / n, "particle_updates_per_s": world * 2.0 * n * steps / (ms / 1e3)}
    return {"value": value, "ms_per_step": ms / steps, "ms_per_step_median": float(np.median(r["step_ms"])),
            "ms_per_step_best": float(np.min(r["step_ms"])), "pairs_per_step": pairs_step,
            "density_pairs_per_step": r["counts"][1] / steps, "force_pairs_per_step": r["counts"][2] / steps,
            "candidates_per_step": (r["counts"][0] + r["counts"][3]) / steps, "phases_ms_per_step": ph,
            "launches": nl, "conversion": conv, "per_particle_update": upd}


def max_over_ranks(vals, device=None):
    """Element-wise max of vals over all ranks of the default process group (the values unchanged when there is
    none): the timing of a replica run is its slowest rank."""
    import torch
    if not (torch.distributed.is_available() and torch.distributed.is_initialized()):
        return [float(v) for v in vals]
    t = torch.tensor([float(v) for v in vals], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def barrier():
    import torch
    if torch.distributed.is_available() and torch.distributed.is_initialized():
        torch.distributed.barrier()


def whole_job_rate(units_per_rank, world, seconds):
    """Units all ranks processed per second: every replica processes units_per_rank in at most `seconds`."""
    return world * float(units_per_rank) / float(seconds)


def profiled_traffic(kernel, root=None):
    """DRAM bytes per launch of `kernel` from a committed ncu summary under profiles/ (its 'traffic:' line), if
    the kernel's source file still has the hash the counters were taken on; else (None, reason).  root: the
    directory holding profiles/ and the sources (default: this file's)."""
    import glob
    import hashlib
    here = root or os.path.dirname(os.path.abspath(__file__))
    for path in sorted(glob.glob(os.path.join(here, "profiles", "*.md"))):
        with open(path) as fh:
            for line in fh:
                if not line.startswith("traffic: "):
                    continue
                kv = dict(tok.split("=", 1) for tok in line.split()[1:] if "=" in tok)
                if kv.get("kernel") != kernel:
                    continue
                src = os.path.join(here, kv.get("source", ""))
                if not os.path.isfile(src):
                    return None, f"{os.path.basename(path)}: source file missing"
                with open(src, "rb") as fs:
                    sha = hashlib.sha256(fs.read()).hexdigest()
                if sha != kv.get("sha256"):
                    return None, f"{os.path.basename(path)}: kernel source changed since the capture"
                return int(kv["bytes_per_launch"]), os.path.relpath(path, here)
    return None, "no ncu capture of this kernel under profiles/"


def roofline_of(prec, s, steps, peaks, measured=None):
    """Dominant kernel = the phase with the largest device time (the force pair kernel)."""
    ph = s["phases_ms_per_step"]
    dom = max(("density", "force"), key=lambda k: ph[k])
    pairs = s["force_pairs_per_step"] if dom == "force" else s["density_pairs_per_step"]
    flops = pairs * (FLOPS_FORCE_PAIR if dom == "force" else FLOPS_DENSITY_PAIR)
    dur = ph[dom] * 1e-3  # one launch of the pair kernel per step
    achieved = flops / dur / 1e12
    peak = PEAK_FP64_TFLOPS if prec == 0 else PEAK_FP32_TFLOPS
    # (the FP64 force body is instantiated per softening: eps > 0 here)
    kernel = (("k_cell_pairs<ForceF64<true>>" if dom == "force" else "k_cell_pairs<DensF64>") if prec == 0 else
              f"k_cell_lanes<{'Force' if dom == 'force' else 'Dens'}F32>")
    traffic, traffic_src = profiled_traffic(kernel)
    return {"kernel": kernel,
            "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic, "traffic_unit": "bytes per launch (dram read + write, ncu)",
            "traffic_source": traffic_src,
            "peak_source": ("derived: GB300 nominal FP64 1.25 TFLOP/s" if prec == 0 else
                            "derived: 152 SMs x 128 FP32 lanes x 2 x 2.07 GHz"),
            "algorithmic_flops_per_launch": flops, "flops_per_pair": FLOPS_FORCE_PAIR if dom == "force" else
            FLOPS_DENSITY_PAIR, "launch_ms": ph[dom],
            "measured_fma_peak_tflops": measured, "frac_of_measured_fma_peak": (achieved / measured) if measured else None}


# ----------------------------------------------------------------------------------------------------------
# the oracle on a bounded sample (CPU baseline and the reference arm)
# ----------------------------------------------------------------------------------------------------------
def host_cores():
    """Host cores this process may run on."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(aos_h, lay, f, block_cells, seed=0, threads=1):
    """Time the FP64 oracle on a compact sample: the force of every particle in a cube of block_cells^3 lattice
    spacings, and the density of every particle within 2 h_max of that cube (all the force needs), with the
    targets split over `threads` host threads.  Work and pairs are those of the same pass restricted to the sample.
    Returns (pairs, seconds, description, values) with values = the oracle's rho, P, c_s of the halo and
    a, du/dt of the cube, by record."""
    import oracle
    p = {"gamma": 5.0 / 3.0, "alpha": 1.0, "beta": 2.0, "eps": 0.01}
    n = aos_h.shape[0]
    box = f["box"]
    s = 1.0 / round(n ** (1 / 3))
    hmax = float(f["h"].max())
    rng = np.random.default_rng(seed)
    c = rng.uniform(0.2, 0.8, size=3)
    t0 = time.perf_counter()
    st = oracle.unpack(aos_h, lay)
    values = oracle.cube_sample(st, box, p, c, 0.5 * block_cells * s, 2.0 * hmax * (1 + 1e-9), threads)
    secs = time.perf_counter() - t0
    # in-support pairs of the sample (counted outside the timed region)
    x, halo, blk = st["x"], values["halo"], values["block"]
    dens_pairs = sum(oracle.neighbours(x, st["h"], box, int(i)).size for i in halo)
    force_pairs = sum(oracle.neighbours(x, st["h"], box, int(i)).size - 1 for i in blk)
    desc = (f"brute-force FP64 oracle on {threads} host thread(s): density of {halo.size} and force of {blk.size} "
            f"particles (a {block_cells}^3-spacing cube plus its 2h halo) of the 262,144-particle workload, each "
            f"against all {n} particles")
    return dens_pairs + force_pairs, secs, desc, values


def cpu_baseline(aos_h, lay, f, block_cells):
    cores = host_cores()
    pairs, secs, desc, values = oracle_sample(aos_h, lay, f, block_cells, threads=cores)
    return {"value": pairs / secs, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc,
            "seconds": secs}, values


def error_vs_oracle(out_records, lay, values):
    """Per-field error of the GPU's records against the oracle's sample values: rho, P, c_s as the largest
    relative error over the halo, a and du/dt normwise (max |err| / max |ref|) over the cube."""
    import oracle
    got = oracle.unpack(out_records, lay)
    h, b = values["halo"], values["block"]
    err = {k: float(np.max(np.abs(got[k][h] - values[k]) / np.abs(values[k]))) for k in ("rho", "P", "cs")}
    for k in ("a", "dudt"):
        ref = values[k]
        err[k] = float(np.max(np.abs(got[k][b] - ref)) / np.max(np.abs(ref)))
    err["particles"] = {"rho_P_cs": int(h.size), "a_dudt": int(b.size)}
    return err


def reference_arm(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    f, lay, aos_h, ncell = _inputs()
    block = args.ref_block
    cores = host_cores()
    for _ in range(args.warmup):
        oracle_sample(aos_h, lay, f, block, seed=1, threads=cores)
    tot_pairs, tot_s = 0, 0.0
    for k in range(args.steps):
        pairs, secs, desc, _ = oracle_sample(aos_h, lay, f, block, seed=2 + k, threads=cores)
        tot_pairs += pairs
        tot_s += secs
    value = tot_pairs / tot_s
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": tot_s * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "particles": int(aos_h.shape[0]),
                       "step": "one bounded sample of the pass (see cpu_baseline.sample)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-block", type=int, default=12, help="oracle sample cube (lattice spacings) for cpu_baseline")
    ap.add_argument("--ref-block", type=int, default=8, help="oracle sample cube per step of --impl reference")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end measurement")
    ap.add_argument("--no-tune", action="store_true", help="keep the default tiles (no autotuning)")
    ap.add_argument("--no-batched", dest="batched", action="store_false", help="skip the batched (patches) forms")
    ap.add_argument("--no-large", dest="large", action="store_false", help="skip the large ten-step run forms")
    ap.add_argument("--only", choices=["f64", "f32", "batched_f32", "batched_f64", "extended_m5"], default=None,
                    help="run one form only (profiling runs); the JSON line then carries that form's numbers")
    ap.add_argument("--patches", type=int, default=4096,
                    help="patches of the batched form with --only batched_* (profiling runs on a smaller case)")
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2502_16517_gb300 import build as b
    b.build()
    f, lay, aos_h, ncell = _inputs()
    n = aos_h.shape[0]
    steps, warmup = args.steps, max(args.warmup, 3)
    gpu_index = int(os.environ.get("CUDA_VISIBLE_DEVICES", str(local)).split(",")[local]) if \
        os.environ.get("CUDA_VISIBLE_DEVICES") else local

    import tempfile
    tune_cache = os.path.join(tempfile.mkdtemp(prefix="sph_tiles_"), "tiles.json") if not args.no_tune else None
    if args.only in ("batched_f32", "batched_f64"):
        # profiling runs of one batched form: its graph-captured steps only
        fp, lay_b, aos_b = batched_inputs(args.patches)
        b = run_batched(0 if args.only == "batched_f64" else 1, steps, warmup, dev, fp, lay_b, aos_b,
                        tune_cache=tune_cache)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": b["value"] * world, "unit": UNIT, "n_gpus": world,
                              "steps": steps, "warmup": warmup, "ms_per_step": b["ms_per_step"],
                              "higher_is_better": True, "form": args.only, "details": b}))
        return 0
    if args.only == "extended_m5":
        # profiling runs of the quartic kernel with the fuller views: that form only
        lay_e, aos_e, ncell_e = extended_inputs()
        from paper_2502_16517_gb300 import workloads as wl
        ext = run_form(0, steps, warmup, dev, aos_e, lay_e, f["box"], ncell_e, tune_cache=tune_cache,
                       params=dict(wl.SPH_PARAMS, kernel=1, scheme=1), tune_form="grid_m5_extended")
        se = summarize_form(0, ext, n, steps, world)
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": se["value"], "unit": UNIT, "n_gpus": world,
                              "steps": steps, "warmup": warmup, "ms_per_step": se["ms_per_step"],
                              "higher_is_better": True, "form": args.only,
                              "phases_ms_per_step": se["phases_ms_per_step"], "tiles": ext["tiles"]}))
        return 0
    forms = ["f64", "f32"] if args.only is None else [args.only]
    runs = {}
    sampler = ClockSampler(gpu_index)
    sampler.__enter__()
    try:
        for k, form in enumerate(forms):
            runs[form] = run_form(0 if form == "f64" else 1, steps, warmup, dev, aos_h, lay, f["box"], ncell,
                                  tune_cache=tune_cache, keep_out=True)
        per_loop = None
        ext = None
        warm = None
        presorted = {}
        if args.only is None:
            # the paper's conversion pattern: one view per loop, converted forth and back around each
            per_loop = run_form(0, steps, warmup, dev, aos_h, lay, f["box"], ncell, tune_cache=tune_cache,
                                union=False)
            # the paper's kernel and fuller views on its 272-byte record
            from paper_2502_16517_gb300 import workloads as wl
            lay_e, aos_e, ncell_e = extended_inputs()
            ext = run_form(0, steps, warmup, dev, aos_e, lay_e, f["box"], ncell_e, tune_cache=tune_cache,
                           params=dict(wl.SPH_PARAMS, kernel=1, scheme=1), tune_form="grid_m5_extended")
            ext["cells"] = int(np.prod(ncell_e))
            del aos_e
            # the same pass with L2 left warm between steps (the 42 MB of records stay in the 129 MB L2)
            warm = run_form(0, steps, warmup, dev, aos_h, lay, f["box"], ncell, tune_cache=tune_cache,
                            flush_l2=False)
            # the paper's continuous AoS: the same records stored in cell order
            aos_s = presorted_aos(aos_h, lay, f["box"], ncell, dev)
            for fm in ("f64", "f32"):
                presorted[fm] = run_form(0 if fm == "f64" else 1, steps, warmup, dev, aos_s, lay, f["box"], ncell,
                                         tune_cache=tune_cache)
            del aos_s
        batched = {}
        if args.batched and args.only is None:
            fp, lay_b, aos_b = batched_inputs()
            for form in ("f32", "f64"):
                batched[form] = run_batched(0 if form == "f64" else 1, max(steps // 3, 3), 2, dev, fp, lay_b, aos_b,
                                            tune_cache=tune_cache)
            del aos_b
        large = {}
        if args.large and args.only is None:
            fl, lay_l, aos_l, ncell_l = large_inputs()
            large["f64"], out64 = run_large(0, 3, dev, fl, lay_l, aos_l, ncell_l, tune_cache=tune_cache)
            large["f32"], out32 = run_large(1, 3, dev, fl, lay_l, aos_l, ncell_l, dt=large["f64"]["dt"],
                                            tune_cache=tune_cache)
            x64 = out64[:, 0:24].copy().view(np.float64)
            x32 = out32[:, 0:24].copy().view(np.float64)
            d = x32 - x64
            d -= np.round(d)
            rho64 = out64[:, 88:96].copy().view(np.float64)[:, 0]
            rho32 = out32[:, 88:96].copy().view(np.float64)[:, 0]
            large["f32"]["vs_f64_after_10_steps"] = {
                "max_position_diff_over_h": float(np.max(np.abs(d)) / fl["h"][0]),
                "max_rel_density_diff": float(np.max(np.abs(rho32 - rho64) / rho64))}
            del aos_l, out64, out32
    finally:
        sampler.__exit__(None, None, None)
    clocks = sampler.summary()
    # max over ranks of the summed step times; the batched / large forms' times likewise
    tot = max_over_ranks([float(np.sum(runs[fm]["step_ms"])) for fm in forms], dev)
    summ = {}
    for k, fm in enumerate(forms):
        local = list(runs[fm]["step_ms"])
        runs[fm]["step_ms"] = [tot[k] / steps] * steps
        summ[fm] = summarize_form(0 if fm == "f64" else 1, runs[fm], n, steps, world)
        # this rank's own per-step event times: median and best beside the max-over-ranks mean
        summ[fm]["ms_per_step_median"] = float(np.median(local))
        summ[fm]["ms_per_step_best"] = float(np.min(local))
    for r in [per_loop, ext, warm] + list(presorted.values()):
        if r is not None:
            t = max_over_ranks([float(np.sum(r["step_ms"]))], dev)[0]
            r["step_ms"] = [t / steps] * steps
    for b in batched.values():
        b["ms_per_step"] = max_over_ranks([b["ms_per_step"]], dev)[0]
        b["value"] = whole_job_rate(b["pairs_per_step"], world, b["ms_per_step"] * 1e-3)
    for b in large.values():
        b["ms_per_run"] = max_over_ranks([b["ms_per_run"]], dev)[0]
        b["value"] = whole_job_rate(b["pairs_per_run"], world, b["ms_per_run"] * 1e-3)
    main_form = forms[0]
    s64, r64 = summ[main_form], runs[main_form]
    s32 = summ.get("f32") if main_form == "f64" else None
    e2e = None
    if not args.no_e2e:
        # both ways to reach host records; the line's e2e is the faster, the other is reported beside it
        modes = []
        for direct in (False, True):
            r = run_e2e(0 if main_form == "f64" else 1, max(steps // 2, 3), 2, dev, aos_h, lay, f["box"], ncell,
                        direct=direct)
            pairs_step = r["value"] * r["ms_per_step"] * 1e-3
            r["ms_per_step"] = max_over_ranks([r["ms_per_step"]], dev)[0]
            r["value"] = whole_job_rate(pairs_step, world, r["ms_per_step"] * 1e-3)
            modes.append(r)
        modes.sort(key=lambda r: -r["value"])
        e2e = dict(modes[0])
        e2e["other_mode"] = modes[1]
    peaks = measured_peaks()
    from paper_2502_16517_gb300 import sph as _sph
    fma_peak = {"f64": _sph.sph_probe_fma_rate(_sph.SPH_F64) / 1e12, "f32": _sph.sph_probe_fma_rate(_sph.SPH_F32) / 1e12}
    if rank != 0:
        torch.distributed.destroy_process_group()
        return 0
    cpu = None
    errors = {}
    if world == 1 and not args.no_cpu_baseline:
        cpu, oracle_values = cpu_baseline(aos_h, lay, f, args.cpu_block)
        # the same oracle values, compared with the records of each timed form's last step
        for fm in forms:
            errors[fm] = error_vs_oracle(runs[fm]["out"], lay, oracle_values)
            errors[fm]["bar"] = 1e-12 if fm == "f64" else 2e-5
    hbm = peaks.get("hbm_gbs")
    conv = dict(s64["conversion"])
    if hbm:
        conv["hbm_peak_GBps"] = hbm
        conv["bin_and_gather_frac"] = conv["bin_and_gather_GBps"] / hbm if conv["bin_and_gather_GBps"] else None
        conv["scatter_frac"] = conv["scatter_GBps"] / hbm if conv["scatter_GBps"] else None
    prec_main = 0 if main_form == "f64" else 1
    line = {
        "metric": METRIC, "value": s64["value"], "unit": UNIT, "n_gpus": world, "steps": steps, "warmup": warmup,
        "ms_per_step": s64["ms_per_step"], "ms_per_step_median": s64["ms_per_step_median"],
        "ms_per_step_best": s64["ms_per_step_best"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": main_form, "data": "synthetic",
        "config": {"workload": WORKLOAD, "particles": n, "cells": int(np.prod(ncell)), "record_bytes": lay["stride"],
                   "l2": "256 MB buffer written between timed steps (outside the step events)",
                   "step": ("sph_step with one view for both loops: bin + one gather of {x,m,h,u,v} + density + "
                            "force + one scatter of {rho,P,cs,a,dudt}"),
                   "pairs": "density pairs incl. self + ordered force pairs, counted on the device",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": roofline_of(prec_main, s64, steps, peaks, fma_peak[main_form]),
        "error_vs_oracle": errors.get(main_form),
        "measured_fma_peak_tflops": fma_peak,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "gpu_launches": int(sum(s64["launches"].values())),
        "clocks": clocks,
        "tiles": r64["tiles"],
        "phases_ms_per_step": s64["phases_ms_per_step"],
        "pairs_per_step": s64["pairs_per_step"],
        "candidates_per_step": s64["candidates_per_step"],
        "per_particle_update": s64["per_particle_update"],
        "conversion": conv,
        "forms": {},
        "wall_s_timed_bracket": r64["wall_s"],
    }
    if s32 is not None:
        line["forms"]["f32"] = {
            "workload": "FP32 precision form: the same 262,144-particle input, FP32 views, Kahan sums",
            "value": s32["value"], "ms_per_step": s32["ms_per_step"], "dtype": "f32",
            "speedup_vs_f64": s32["value"] / s64["value"], "phases_ms_per_step": s32["phases_ms_per_step"],
            "roofline": roofline_of(1, s32, steps, peaks, fma_peak["f32"]), "conversion": s32["conversion"],
            "gpu_launches": int(sum(s32["launches"].values())), "tiles": runs["f32"]["tiles"],
            "per_particle_update": s32["per_particle_update"], "error_vs_oracle": errors.get("f32")}
    if per_loop is not None:
        per_loop["step_ms"] = list(per_loop["step_ms"])
        sp = summarize_form(0, per_loop, n, steps, world)
        line["forms"]["f64_per_loop_views"] = {
            "workload": ("the plain FP64 input, one view per loop converted forth and back around each: bin + "
                         "gather {x,m,h,u} + density + scatter {rho,P,cs} + gather {x,v,m,h,rho,P,cs} + force + "
                         "scatter {a,dudt}"),
            "value": sp["value"], "ms_per_step": sp["ms_per_step"], "dtype": "f64",
            "phases_ms_per_step": sp["phases_ms_per_step"], "conversion": sp["conversion"],
            "gpu_launches": int(sum(sp["launches"].values()))}
    if ext is not None:
        ext["step_ms"] = list(ext["step_ms"])
        se = summarize_form(0, ext, n, steps, world)
        line["forms"]["extended_m5_f64"] = {
            "workload": ("the plain 262,144-particle input on the paper's 272-byte record, " + EXT_PARAMS_NOTE +
                         f"; {ext['cells']} periodic cells (edge >= 5h/2)"),
            "value": se["value"], "ms_per_step": se["ms_per_step"], "dtype": "f64",
            "pairs_per_step": (ext["counts"][1] + ext["counts"][2]) / steps,
            "phases_ms_per_step": se["phases_ms_per_step"], "gpu_launches": int(sum(se["launches"].values())),
            "tiles": ext["tiles"]}
    if warm is not None:
        warm["step_ms"] = list(warm["step_ms"])
        sw = summarize_form(0, warm, n, steps, world)
        line["forms"]["f64_l2_warm"] = {
            "workload": "the plain FP64 form with no L2 flush between steps (records and views stay L2-resident)",
            "value": sw["value"], "ms_per_step": sw["ms_per_step"], "dtype": "f64",
            "phases_ms_per_step": sw["phases_ms_per_step"], "conversion": sw["conversion"],
            "gpu_launches": int(sum(sw["launches"].values()))}
    for fm, r in presorted.items():
        r["step_ms"] = list(r["step_ms"])
        sp = summarize_form(0 if fm == "f64" else 1, r, n, steps, world)
        ref = summ.get(fm)
        line["forms"][f"{fm}_presorted_aos"] = {
            "workload": ("the plain input with its records stored in cell order (continuous AoS) instead of "
                         "scattered; otherwise as the " + ("FP64" if fm == "f64" else "FP32") + " form"),
            "value": sp["value"], "ms_per_step": sp["ms_per_step"], "dtype": fm,
            "vs_scattered": sp["value"] / ref["value"] if ref else None,
            "phases_ms_per_step": sp["phases_ms_per_step"], "conversion": sp["conversion"],
            "gpu_launches": int(sum(sp["launches"].values()))}
    for form, b in large.items():
        b = dict(b)
        b["workload"] = ("large run: 2,097,152 particles, 8 Gaussian overdensities (sigma 0.05, 4x) on a uniform "
                         "background, 53^3 periodic cells, 10 KDK steps with per-step conversion and re-binning")
        line["forms"][f"large_{form}"] = b
    for form, b in batched.items():
        b = dict(b)
        b["workload"] = ("batched form: 4096 independent 3x3x3-cell patches (reflecting walls), Poisson(lambda ~ "
                         f"U(8,256)) per cell, v ~ N(0,0.1), {b['particles']} particles, one leapfrog step per "
                         "graph launch, inputs larger than L2 (no flush)")
        b["speedup_vs_plain_f64"] = b["value"] / s64["value"]
        line["forms"][f"batched_{form}"] = b
    print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
