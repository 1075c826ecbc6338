"""Seeded synthetic particle sets and their AoS records.

This module only makes inputs: positions, velocities, masses, smoothing lengths and internal energies, written
into wide particle records.  It holds none of the SPH view path's arithmetic (no binning, no conversion, no
kernel, no pair sum).  The tests hand the same buffers to the CUDA library and to the CPU oracle.

The record is the 160-byte particle struct
    double x[3], v[3], a[3], mass, h, rho, P, u, dudt, cs;  int64 id;  int32 cell, flags;  16 reserved bytes
(the members fill 144 bytes; the struct is padded to 160).  The paper's own struct is 272 bytes (Section 2.2);
the library never assumes this layout, it takes a stride and per-field byte offsets.

Workloads (all in the periodic unit box, seed 2502 unless stated):
  * jittered_lattice: n_side^3 particles on a lattice, jittered by U(-j, j) * spacing per axis, equal mass
    1/N, h = 1.2 * spacing, u = 1, v ~ N(0, sigma) per component (sigma = 0 gives v = 0);
  * clustered: N particles drawn iid from a density with 8 Gaussian overdensities (sigma 0.05, peak 4x the
    background) on a uniform background, h from the mean spacing;
  * patches: independent 3x3x3-cell patches, Poisson(lambda) particles per cell with lambda ~ U(8, 256) per
    patch, uniform positions inside each cell.
"""
from __future__ import annotations

import numpy as np

SEED = 2502

# Field order of the layout's offset table: the same order as the library's field bits.
FIELDS = ("x", "v", "a", "mass", "h", "rho", "P", "u", "dudt", "cs")
# the members of the fuller density / force views (neighbour count, div v, curl v, Omega, signal velocity)
EXT_FIELDS = ("nnb", "divv", "curlv", "omega", "vsig")
ALL_FIELDS = FIELDS + EXT_FIELDS
NCOMP = {"x": 3, "v": 3, "a": 3, "mass": 1, "h": 1, "rho": 1, "P": 1, "u": 1, "dudt": 1, "cs": 1,
         "nnb": 1, "divv": 1, "curlv": 3, "omega": 1, "vsig": 1}

RECORD_STRIDE = 160
RECORD_OFFSETS = {"x": 0, "v": 24, "a": 48, "mass": 72, "h": 80, "rho": 88, "P": 96, "u": 104, "dudt": 112,
                  "cs": 120}
ID_OFFSET, CELL_OFFSET, FLAGS_OFFSET = 128, 136, 140


def default_layout():
    return {"stride": RECORD_STRIDE, "offsets": dict(RECORD_OFFSETS)}


# The paper's default particle footprint, 272 bytes (Section 2.2): the 160-byte record above (members, id, cell,
# flags, padding) followed by the fuller views' members and more administrative bytes.
EXT_RECORD_STRIDE = 272
EXT_RECORD_OFFSETS = dict(RECORD_OFFSETS, nnb=160, divv=168, curlv=176, omega=200, vsig=208)


def extended_layout():
    return {"stride": EXT_RECORD_STRIDE, "offsets": dict(EXT_RECORD_OFFSETS)}


def shuffled_layout(seed=7, stride=None):
    """A different legal record: the fields in a random order at 8-byte granularity, with admin bytes between
    them, so no test passes only because of the default layout."""
    rng = np.random.default_rng(seed)
    names = list(FIELDS)
    rng.shuffle(names)
    off = 8 * int(rng.integers(0, 3))
    offsets = {}
    for nm in names:
        offsets[nm] = off
        off += 8 * NCOMP[nm] + 8 * int(rng.integers(0, 2))
    min_stride = off + 16
    if stride is None:
        stride = ((min_stride + 15) // 16) * 16 + 16 * int(rng.integers(0, 2))
    assert stride >= min_stride
    return {"stride": int(stride), "offsets": offsets}


def _wrap_unit(x, box):
    x = x - box * np.floor(x / box)
    return np.where(x >= box, 0.0, x)


def jittered_lattice(n_side, jitter=0.1, vel_sigma=0.0, hfac=1.2, u0=1.0, box=1.0, seed=SEED):
    """Fields of an n_side^3 jittered lattice in a periodic cube of edge `box`."""
    rng = np.random.default_rng(seed)
    n = n_side ** 3
    s = box / n_side
    idx = np.indices((n_side, n_side, n_side)).reshape(3, -1).T[:, ::-1].astype(np.float64)
    x = (idx + 0.5) * s
    if jitter:
        x = x + rng.uniform(-jitter, jitter, size=(n, 3)) * s
    x = _wrap_unit(x, box)
    v = rng.normal(0.0, vel_sigma, size=(n, 3)) if vel_sigma else np.zeros((n, 3))
    return {
        "x": x,
        "v": v,
        "mass": np.full(n, box ** 3 / n),
        "h": np.full(n, hfac * s),
        "u": np.full(n, float(u0)),
        "box": np.array([box, box, box], np.float64),
    }


def clustered(n, nclusters=8, sigma=0.05, peak=4.0, hfac=1.2, n_side_equiv=None, u0=1.0, vel_sigma=0.0,
              seed=SEED):
    """N particles iid from rho(x) ~ 1 + (peak - 1) sum_k exp(-|x - c_k|^2 / (2 sigma^2)) (periodic image of the
    nearest centre), drawn by mixture sampling: background uniform, clusters Gaussian, wrapped."""
    rng = np.random.default_rng(seed)
    centres = rng.uniform(0.0, 1.0, size=(nclusters, 3))
    w_cluster = (peak - 1.0) * (2.0 * np.pi * sigma ** 2) ** 1.5
    p_bg = 1.0 / (1.0 + nclusters * w_cluster)
    is_bg = rng.uniform(size=n) < p_bg
    k = rng.integers(0, nclusters, size=n)
    x = np.where(is_bg[:, None], rng.uniform(0.0, 1.0, size=(n, 3)),
                 centres[k] + rng.normal(0.0, sigma, size=(n, 3)))
    x = _wrap_unit(x, 1.0)
    if n_side_equiv is None:
        n_side_equiv = round(n ** (1.0 / 3.0))
    v = rng.normal(0.0, vel_sigma, size=(n, 3)) if vel_sigma else np.zeros((n, 3))
    return {
        "x": x,
        "v": v,
        "mass": np.full(n, 1.0 / n),
        "h": np.full(n, hfac / n_side_equiv),
        "u": np.full(n, float(u0)),
        "box": np.array([1.0, 1.0, 1.0]),
        "centres": centres,
    }


def patches(npatch, lam_lo=8.0, lam_hi=256.0, hfac=1.2, hmax=0.5, u0=1.0, vel_sigma=0.0, seed=SEED):
    """Independent 3x3x3 patches of unit cells with Poisson occupancy.

    Patch p occupies its own [0,3)^3 (coordinates are patch-local).  Occupancy per cell ~ Poisson(lambda_p),
    lambda_p ~ U(lam_lo, lam_hi); particles uniform in their cell; m = 1/lambda_p; h = min(1.2 lambda^(-1/3),
    hmax).  Returns fields in patch-major order plus patch_start (npatch + 1 offsets) and lam (npatch)."""
    rng = np.random.default_rng(seed)
    lam = rng.uniform(lam_lo, lam_hi, size=npatch)
    counts = rng.poisson(np.repeat(lam, 27)).reshape(npatch, 27)
    per_patch = counts.sum(axis=1)
    patch_start = np.zeros(npatch + 1, np.int64)
    np.cumsum(per_patch, out=patch_start[1:])
    n = int(patch_start[-1])
    cell_local = np.repeat(np.tile(np.arange(27), npatch), counts.ravel())
    ck = np.stack([cell_local % 3, (cell_local // 3) % 3, cell_local // 9], axis=1).astype(np.float64)
    x = ck + rng.uniform(0.0, 1.0, size=(n, 3))
    pid = np.repeat(np.arange(npatch), per_patch)
    lam_p = lam[pid]
    v = rng.normal(0.0, vel_sigma, size=(n, 3)) if vel_sigma else np.zeros((n, 3))
    return {
        "x": x,
        "v": v,
        "mass": 1.0 / lam_p,
        "h": np.minimum(hfac * lam_p ** (-1.0 / 3.0), hmax),
        "u": np.full(n, float(u0)),
        "box": np.array([3.0, 3.0, 3.0]),
        "patch_start": patch_start,
        "lam": lam,
    }


def pack_aos(fields, layout=None, order="shuffled", seed=SEED + 1, canary=True, segments=None):
    """Write the fields into records: a uint8 array [n, stride].

    order: "shuffled" puts particle k at a seeded random record (heap-scattered AoS, the paper's pointer-indexed
    storage), "given" keeps particle k at record k.  With segments (ascending offsets, e.g. patch_start) the
    shuffle stays inside each segment, so every patch keeps a contiguous range of records.
    Returns (aos, where) with where[k] = record of particle k.
    Bytes outside the given fields (a, rho, P, dudt, cs, admin fields, padding) are random canary bytes when
    canary is set, else zero; the id field (when inside the default layout) holds the particle index."""
    layout = layout or default_layout()
    stride = int(layout["stride"])
    offs = layout["offsets"]
    n = fields["mass"].shape[0]
    rng = np.random.default_rng(seed)
    if canary:
        aos = rng.integers(0, 256, size=(n, stride), dtype=np.uint8)
    else:
        aos = np.zeros((n, stride), np.uint8)
    if order != "shuffled":
        where = np.arange(n)
    elif segments is None:
        where = rng.permutation(n)
    else:
        seg = np.asarray(segments, np.int64)
        where = np.arange(n)
        for a, b in zip(seg[:-1], seg[1:]):
            where[a:b] = a + rng.permutation(int(b - a))
    rec = np.empty_like(aos)
    rec[:] = aos
    for name in ALL_FIELDS:
        if name not in fields or name not in offs:
            continue
        val = np.ascontiguousarray(np.asarray(fields[name], np.float64).reshape(n, NCOMP[name]))
        o = int(offs[name])
        rec[:, o:o + 8 * NCOMP[name]] = val.view(np.uint8).reshape(n, 8 * NCOMP[name])
    if all(layout["offsets"].get(k) == o for k, o in RECORD_OFFSETS.items()) and stride >= ID_OFFSET + 8:
        rec[:, ID_OFFSET:ID_OFFSET + 8] = np.arange(n, dtype=np.int64).view(np.uint8).reshape(n, 8)
    aos[where] = rec
    return aos, where


def particle_values(values, where):
    """Reorder per-record values (record order) into particle order using `where` from pack_aos."""
    return np.asarray(values)[where]


def tiny(seed=SEED):
    """4096 particles on a 16^3 lattice jittered by U(-0.1, 0.1) * spacing, v = 0, h = 1.2 s."""
    return jittered_lattice(16, jitter=0.1, vel_sigma=0.0, seed=seed)


def plain(seed=SEED):
    """262,144 particles on a 64^3 lattice jittered by U(-0.1, 0.1) * spacing, v ~ N(0, 0.1), h = 1.2 s."""
    return jittered_lattice(64, jitter=0.1, vel_sigma=0.1, seed=seed)


def large(n_side=128, seed=SEED):
    """2,097,152 particles (n_side = 128) drawn iid from a uniform background plus 8 Gaussian overdensities
    (sigma 0.05, peak 4x the background), periodic unit box, m = 1/N, h = 1.2 / n_side for every particle, u = 1,
    v = 0.  The lattice size only sets N and the background spacing."""
    return clustered(n_side ** 3, nclusters=8, sigma=0.05, peak=4.0, hfac=1.2, n_side_equiv=n_side, seed=seed)


def ncell_for(box, hmax, kappa=2.0):
    """Largest cell count per axis with cell edge >= kappa h_max, the kernel's support (2 for the cubic spline,
    5/2 for the quartic), and at least 3 for the periodic stencil."""
    box = np.asarray(box, np.float64)
    nc = np.floor(box / (kappa * hmax)).astype(np.int64)
    return np.maximum(nc, 3).astype(np.int32)


SPH_PARAMS = {"gamma": 5.0 / 3.0, "alpha": 1.0, "beta": 2.0, "eps": 0.01}
