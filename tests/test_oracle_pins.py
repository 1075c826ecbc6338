"""Pins of the FP64 oracle against facts that do not come from the oracle itself.

Each test names what fixes the expected value: a closed form of the cubic spline, a hand-derived two-particle
case, a lattice shell sum, a conservation law of the symmetrised SPH equations, or a library routine that
computes the same special case.  Chosen so that a dropped term, a wrong sign, a swapped h_i/h_j or a transposed
operand in the oracle fails at least one of them.
"""
import math
import os

import numpy as np
import pytest

from paper_2502_16517_gb300 import workloads as wl

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
PI = math.pi


# --------------------------------------------------------------------------------------------------------
# Kernel (cubic spline, Monaghan & Lattanzio 1985)
# --------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("h", [0.01875, 0.075, 0.3, 1.0])
def test_kernel_unit_integral(oracle, h):
    # int_0^{2h} W(r, h) 4 pi r^2 dr = 1 (normalisation of a 3D kernel).  On [0,h] and [h,2h] the integrand is
    # a polynomial of degree 5, so 4-point Gauss-Legendre (exact to degree 7) gives the integral to round-off.
    t, wt = np.polynomial.legendre.leggauss(4)
    total = 0.0
    for lo, hi in ((0.0, h), (h, 2 * h)):
        r = 0.5 * (hi - lo) * t + 0.5 * (hi + lo)
        total += 0.5 * (hi - lo) * np.sum(wt * oracle.w(r, np.full(r.size, h)) * 4 * PI * r * r)
    assert abs(total - 1.0) < 1e-13


def test_kernel_closed_values(oracle):
    h = 0.2
    # f(0) = 1, f(1) = 1/4, f(2) = 0; f'(1) = -3/4 (from both pieces); f'(0) = 0.
    w = oracle.w(np.array([0.0, h, 2 * h, 3 * h]), np.full(4, h))
    assert w[0] == pytest.approx(1.0 / (PI * h ** 3), rel=1e-15)
    assert w[1] == pytest.approx(0.25 / (PI * h ** 3), rel=1e-15)
    assert w[2] == 0.0 and w[3] == 0.0
    dw = oracle.dwdr(np.array([0.0, h, 2 * h]), np.full(3, h))
    assert dw[0] == 0.0
    assert dw[1] == pytest.approx(-0.75 / (PI * h ** 4), rel=1e-15)
    assert dw[2] == 0.0
    # hand values at q = 0.8 and q = 1.2 (one per piece): f = 0.424, 0.128; f' = -0.96, -0.48
    q = np.array([0.8, 1.2])
    w = oracle.w(q * h, np.full(2, h)) * PI * h ** 3
    dw = oracle.dwdr(q * h, np.full(2, h)) * PI * h ** 4
    np.testing.assert_allclose(w, [0.424, 0.128], rtol=1e-14)
    np.testing.assert_allclose(dw, [-0.96, -0.48], rtol=1e-14)


def test_kernel_derivative_matches_finite_difference(oracle):
    h = 0.3
    r = np.linspace(0.01, 0.59, 97)
    eps = 1e-6
    fd = (oracle.w(r + eps, np.full_like(r, h)) - oracle.w(r - eps, np.full_like(r, h))) / (2 * eps)
    dw = oracle.dwdr(r, np.full_like(r, h))
    scale = np.abs(dw).max()
    assert np.max(np.abs(fd - dw)) < 1e-6 * scale


def test_kernel_is_c2(oracle):
    # The cubic spline is twice continuously differentiable: W, W' and W'' match across q = 1 and q = 2.
    h = 1.0
    for q0 in (1.0, 2.0):
        e = 1e-7
        lo, hi = np.array([q0 - e]), np.array([q0 + e])
        hh = np.array([h])
        assert abs(oracle.w(lo, hh)[0] - oracle.w(hi, hh)[0]) < 1e-6
        assert abs(oracle.dwdr(lo, hh)[0] - oracle.dwdr(hi, hh)[0]) < 1e-6
        d = 1e-4
        second_lo = (oracle.dwdr(lo, hh)[0] - oracle.dwdr(lo - d, hh)[0]) / d
        second_hi = (oracle.dwdr(hi + d, hh)[0] - oracle.dwdr(hi, hh)[0]) / d
        assert abs(second_lo - second_hi) < 1e-3


# --------------------------------------------------------------------------------------------------------
# Density
# --------------------------------------------------------------------------------------------------------
def _golden_lattice():
    with open(os.path.join(GOLDEN, "lattice_density.txt")) as fh:
        for line in fh:
            if line.startswith("rho "):
                return float(line.split()[1])
    raise AssertionError("no rho line")


@pytest.mark.parametrize("n_side", [16, 24])
def test_lattice_density_matches_shell_sum(oracle, n_side):
    f = wl.jittered_lattice(n_side, jitter=0.0)
    rho = oracle.density(f["x"], f["mass"], f["h"], f["box"])
    ref = _golden_lattice()
    assert np.max(np.abs(rho - ref)) < 1e-13
    # Riemann sum of a unit-integral kernel: close to the mean density 1
    assert abs(ref - 1.0) < 1e-3


def test_density_translation_and_axis_permutation_invariance(oracle):
    f = wl.jittered_lattice(10, jitter=0.3, seed=11)
    rho = oracle.density(f["x"], f["mass"], f["h"], f["box"])
    shifted = np.mod(f["x"] + np.array([0.31, -0.17, 0.443]), 1.0)
    rho_s = oracle.density(shifted, f["mass"], f["h"], f["box"])
    np.testing.assert_allclose(rho_s, rho, rtol=1e-12)
    rho_p = oracle.density(f["x"][:, [2, 0, 1]], f["mass"], f["h"], f["box"])
    np.testing.assert_allclose(rho_p, rho, rtol=1e-13)


def test_density_self_term_and_isolated_particle(oracle):
    # One particle alone: rho = m W(0, h) = m / (pi h^3).
    x = np.array([[0.5, 0.5, 0.5]])
    rho = oracle.density(x, np.array([2.0]), np.array([0.1]), np.ones(3))
    assert rho[0] == pytest.approx(2.0 / (PI * 1e-3), rel=1e-15)


def test_density_periodic_wrap_pair(oracle):
    # Two particles 0.12 apart across the periodic face x = 0 / x = 1, h = 0.1 (q = 1.2): f(1.2) = 0.128.
    x = np.array([[0.05, 0.5, 0.5], [0.93, 0.5, 0.5]])
    rho = oracle.density(x, np.ones(2), np.full(2, 0.1), np.ones(3))
    np.testing.assert_allclose(rho, (1.0 + 0.128) / (PI * 1e-3), rtol=1e-12)
    # non-periodic: they do not see each other
    rho_o = oracle.density(x, np.ones(2), np.full(2, 0.1), np.ones(3), periodic=False)
    np.testing.assert_allclose(rho_o, 1.0 / (PI * 1e-3), rtol=1e-15)


# --------------------------------------------------------------------------------------------------------
# Two-particle closed forms for the force (derived by hand from f(q) values above)
# --------------------------------------------------------------------------------------------------------
def _two(oracle, x, v, h, gamma=5.0 / 3.0, u=1.0, alpha=1.0, beta=2.0, eps=0.01):
    m = np.ones(2)
    rho = oracle.density(x, m, h, np.ones(3))
    P, cs = oracle.eos(rho, np.full(2, u), gamma)
    a, du = oracle.force(x, v, m, h, rho, P, cs, np.ones(3), True, alpha, beta, eps)
    return rho, P, cs, a, du


def test_two_particles_equal_h_pressure_only(oracle):
    # d = h = 0.1 (q = 1): rho = 1.25 / (pi h^3); a_0x = -2 A 0.75/(pi h^4) with A = (gamma-1)/rho
    #   = -1.2 (gamma - 1) u / h = -8 for gamma = 5/3, u = 1; repulsive, equal and opposite; du/dt = 0 at v = 0.
    x = np.array([[0.5, 0.5, 0.5], [0.6, 0.5, 0.5]])
    rho, P, cs, a, du = _two(oracle, x, np.zeros((2, 3)), np.full(2, 0.1))
    np.testing.assert_allclose(rho, 1.25 / (PI * 1e-3), rtol=1e-14)
    np.testing.assert_allclose(cs, math.sqrt(10.0 / 9.0), rtol=1e-14)
    np.testing.assert_allclose(a[:, 0], [-8.0, 8.0], rtol=1e-12)
    assert np.all(np.abs(a[:, 1:]) < 1e-12)
    np.testing.assert_allclose(du, 0.0, atol=1e-12)


def test_two_particles_equal_h_approaching_viscosity(oracle):
    # Same pair, v_0 = +w, v_1 = -w along x (approaching), w = 0.5: v_ij . r_ij = -2 w h < 0,
    # mu = -2w/(1+eps), Pi = (c |mu| + 2 mu^2)/rho.  With K = c/(1+eps) * 2w + 2 (2w)^2/(1+eps)^2 (here 2w = 1):
    #   a_0x = -8 - 6 K,  du_0/dt = 4 + 3 K (pressure work 0.8 w/h plus viscous heating).
    x = np.array([[0.5, 0.5, 0.5], [0.6, 0.5, 0.5]])
    v = np.array([[0.5, 0, 0], [-0.5, 0, 0]], np.float64)
    rho, P, cs, a, du = _two(oracle, x, v, np.full(2, 0.1))
    c = math.sqrt(10.0 / 9.0)
    K = c / 1.01 + 2.0 / 1.01 ** 2
    np.testing.assert_allclose(a[:, 0], [-8.0 - 6.0 * K, 8.0 + 6.0 * K], rtol=1e-12)
    np.testing.assert_allclose(du, [4.0 + 3.0 * K] * 2, rtol=1e-12)
    # receding pair: no viscosity, du/dt = -0.8 w / h each
    rho, P, cs, a, du = _two(oracle, x, -v, np.full(2, 0.1))
    np.testing.assert_allclose(a[:, 0], [-8.0, 8.0], rtol=1e-12)
    np.testing.assert_allclose(du, [-4.0, -4.0], rtol=1e-12)


@pytest.mark.parametrize("alpha,beta,eps", [(1.0, 2.0, 0.0), (0.5, 1.0, 0.3), (0.0, 3.0, 0.05)])
def test_two_particles_viscosity_parameters(oracle, alpha, beta, eps):
    # The approaching pair above for other Monaghan constants: mu = -2w/(1 + eps) with 2w = 1 (eps softens
    # hbar^2 against r^2 = h^2), Pi = (alpha c |mu| + beta mu^2)/rho, so K = alpha c/(1 + eps) + beta/(1 + eps)^2
    # and again a_0x = -8 - 6 K, du_0/dt = 4 + 3 K.  Separates eps, alpha and beta (a swapped or misplaced
    # constant changes K).
    x = np.array([[0.5, 0.5, 0.5], [0.6, 0.5, 0.5]])
    v = np.array([[0.5, 0, 0], [-0.5, 0, 0]], np.float64)
    rho, P, cs, a, du = _two(oracle, x, v, np.full(2, 0.1), alpha=alpha, beta=beta, eps=eps)
    c = math.sqrt(10.0 / 9.0)
    K = alpha * c / (1.0 + eps) + beta / (1.0 + eps) ** 2
    np.testing.assert_allclose(a[:, 0], [-8.0 - 6.0 * K, 8.0 + 6.0 * K], rtol=1e-12)
    np.testing.assert_allclose(du, [4.0 + 3.0 * K] * 2, rtol=1e-12)


def test_two_particles_unequal_h(oracle):
    # h_0 = 0.1, h_1 = 0.15, d = 0.12: q_0 = 1.2 (outer piece), q_1 = 0.8 (inner piece).
    # rho_0 = (1 + 0.128)/(pi h_0^3), rho_1 = (1 + 0.424)/(pi h_1^3);  A_k = (2/3)/rho_k;
    # a_0x = -(2/3) [0.48/(1.128 h_0) + 0.96/(1.424 h_1)],  a_1x = -a_0x.
    h = np.array([0.1, 0.15])
    x = np.array([[0.4, 0.5, 0.5], [0.52, 0.5, 0.5]])
    rho, P, cs, a, du = _two(oracle, x, np.zeros((2, 3)), h)
    np.testing.assert_allclose(rho, [1.128 / (PI * 0.1 ** 3), 1.424 / (PI * 0.15 ** 3)], rtol=1e-13)
    a0 = -(2.0 / 3.0) * (0.48 / (1.128 * 0.1) + 0.96 / (1.424 * 0.15))
    np.testing.assert_allclose(a[:, 0], [a0, -a0], rtol=1e-12)


# --------------------------------------------------------------------------------------------------------
# Conservation laws of the symmetrised equations (pin the pairing of every term)
# --------------------------------------------------------------------------------------------------------
def _random_state(oracle, n=400, seed=5):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0, 1, size=(n, 3))
    v = rng.normal(0, 0.3, size=(n, 3))
    m = rng.uniform(0.5, 1.5, size=n) / n
    h = rng.uniform(0.06, 0.1, size=n)
    u = rng.uniform(0.5, 1.5, size=n)
    box = np.ones(3)
    rho = oracle.density(x, m, h, box)
    P, cs = oracle.eos(rho, u, 5.0 / 3.0)
    a, du = oracle.force(x, v, m, h, rho, P, cs, box)
    return x, v, m, h, u, rho, P, cs, a, du


def test_momentum_conserved(oracle):
    x, v, m, h, u, rho, P, cs, a, du = _random_state(oracle)
    tot = (m[:, None] * a).sum(axis=0)
    scale = (m[:, None] * np.abs(a)).sum()
    assert np.all(np.abs(tot) < 1e-13 * scale)


def test_energy_conserved(oracle):
    x, v, m, h, u, rho, P, cs, a, du = _random_state(oracle)
    rate = m * ((v * a).sum(axis=1) + du)
    scale = (m * (np.abs((v * a).sum(axis=1)) + np.abs(du))).sum()
    assert abs(rate.sum()) < 1e-13 * scale


def test_galilean_invariance(oracle):
    x, v, m, h, u, rho, P, cs, a, du = _random_state(oracle, n=200)
    a2, du2 = oracle.force(x, v + np.array([3.0, -1.0, 0.5]), m, h, rho, P, cs, np.ones(3))
    np.testing.assert_allclose(a2, a, rtol=1e-10, atol=1e-10 * np.abs(a).max())
    np.testing.assert_allclose(du2, du, rtol=1e-10, atol=1e-10 * np.abs(du).max())


def test_uniform_lattice_force_vanishes(oracle):
    f = wl.jittered_lattice(10, jitter=0.0)
    rho = oracle.density(f["x"], f["mass"], f["h"], f["box"])
    P, cs = oracle.eos(rho, f["u"], 5.0 / 3.0)
    a, du = oracle.force(f["x"], f["v"], f["mass"], f["h"], rho, P, cs, f["box"])
    # a single pair term is of order m A |grad W| r ~ 1e-1; the lattice sum cancels to round-off
    assert np.abs(a).max() < 1e-10
    assert np.abs(du).max() == 0.0


# --------------------------------------------------------------------------------------------------------
# Binning and conversions
# --------------------------------------------------------------------------------------------------------
def test_bin_is_stable_cell_major_and_contains_positions(oracle):
    f = wl.jittered_lattice(12, jitter=0.4, seed=3)
    rng = np.random.default_rng(0)
    x = f["x"][rng.permutation(f["x"].shape[0])]
    box = f["box"]
    nc = np.array([5, 4, 7], np.int32)
    cell_of, start, perm, cos, bad = oracle.bin_cells(x, box, nc)
    n = x.shape[0]
    assert bad == 0
    assert np.array_equal(np.sort(perm), np.arange(n))
    assert start[0] == 0 and start[-1] == n and np.all(np.diff(start) >= 0)
    assert np.array_equal(np.bincount(cell_of, minlength=int(nc.prod())), np.diff(start))
    for c in range(int(nc.prod())):
        seg = perm[start[c]:start[c + 1]]
        assert np.all(np.diff(seg) > 0)            # stable: ascending particle index inside a cell
        assert np.all(cell_of[seg] == c) and np.all(cos[start[c]:start[c + 1]] == c)
        k = np.array([c % nc[0], (c // nc[0]) % nc[1], c // (nc[0] * nc[1])])
        edge = box / nc
        assert np.all(x[seg] >= k * edge - 1e-15) and np.all(x[seg] < (k + 1) * edge + 1e-15)


def test_bin_clamps_and_counts_out_of_box(oracle):
    x = np.array([[1.0, 0.5, 0.5], [-0.1, 0.5, 0.5], [0.5, np.nan, 0.5], [0.2, 0.2, 0.2]])
    cell_of, start, perm, cos, bad = oracle.bin_cells(x, np.ones(3), np.array([4, 4, 4], np.int32))
    assert bad == 2                    # x = 1.0 is inside [0, box]; -0.1 and NaN are not
    assert cell_of[0] % 4 == 3         # x == box clamps into the last cell
    assert cell_of[1] % 4 == 0


@pytest.mark.parametrize("layout_kind", ["default", "shuffled"])
def test_gather_scatter_round_trip_is_byte_identical(oracle, layout_kind):
    lay = wl.default_layout() if layout_kind == "default" else wl.shuffled_layout(seed=4)
    f = wl.jittered_lattice(8, jitter=0.2, vel_sigma=0.1)
    aos, where = wl.pack_aos(f, lay, order="shuffled")
    n = aos.shape[0]
    perm = np.random.default_rng(9).permutation(n).astype(np.int32)
    out = aos.copy()
    for name, off in lay["offsets"].items():
        nc = wl.NCOMP[name]
        g = oracle.gather(aos, lay["stride"], perm, off, nc)
        oracle.scatter(out, lay["stride"], perm, off, g)
    assert np.array_equal(out, aos)


def test_scatter_touches_only_the_written_field(oracle):
    lay = wl.default_layout()
    f = wl.jittered_lattice(6, jitter=0.2)
    aos, _ = wl.pack_aos(f, lay)
    n = aos.shape[0]
    perm = np.arange(n, dtype=np.int32)[::-1].copy()
    out = aos.copy()
    oracle.scatter(out, lay["stride"], perm, lay["offsets"]["rho"], np.full((1, n), 7.5))
    changed = np.any(out != aos, axis=0)
    o = lay["offsets"]["rho"]
    assert not changed[:o].any() and not changed[o + 8:].any()
    assert np.all(out[:, o:o + 8].copy().view(np.float64)[:, 0] == 7.5)


def test_gather_values_and_fp32_rounding(oracle):
    lay = wl.default_layout()
    f = wl.jittered_lattice(6, jitter=0.2, vel_sigma=0.3)
    aos, where = wl.pack_aos(f, lay)
    n = aos.shape[0]
    perm = np.arange(n, dtype=np.int32)
    g = oracle.gather(aos, lay["stride"], perm, lay["offsets"]["v"], 3)
    inv = np.empty(n, np.int64)
    inv[where] = np.arange(n)
    np.testing.assert_array_equal(g.T, f["v"][inv])
    g32 = oracle.gather(aos, lay["stride"], perm, lay["offsets"]["v"], 3, np.float32)
    np.testing.assert_array_equal(g32, g.astype(np.float32))      # numpy's cast is IEEE round-to-nearest


def test_fp32_positions_are_cell_relative(oracle):
    lay = wl.default_layout()
    f = wl.jittered_lattice(10, jitter=0.4, seed=8)
    aos, _ = wl.pack_aos(f, lay)
    nc = np.array([3, 5, 4], np.int32)
    x = oracle.unpack(aos, lay)["x"]
    cell_of, start, perm, cos, _ = oracle.bin_cells(x, f["box"], nc)
    rel = oracle.gather_pos_f32(aos, lay["stride"], perm, lay["offsets"]["x"], cos, f["box"], nc)
    edge = f["box"] / nc
    k = np.stack([cos % nc[0], (cos // nc[0]) % nc[1], cos // (nc[0] * nc[1])], axis=0)
    assert np.all(rel >= 0) and np.all(rel <= edge[:, None].astype(np.float32))
    back = rel.astype(np.float64) + k * edge[:, None]
    np.testing.assert_allclose(back.T, x[perm], atol=1e-7)


def test_reduce_hand_computed_three_particles(oracle):
    """All eight sums of a three-particle state worked out by hand (every product and sum exact in binary):
      sum m v        = (2 - 2 + 1, -4 + 0 + 1, 6 + 1 + 0)                     = (1, -3, 7)
      sum m a        = (1 + 1 - 2, 2 - 2 + 3, -2 + 0 + 0.5)                   = (0, 3, -1.5)
      sum m (v^2/2 + u)   = 2 (7 + 1.5) + 0.5 (10 + 3) + 1 (1 + 0)           = 24.5
      sum m (v.a + du/dt) = 2 (-4.5 + 0.25) + 0.5 (-8 - 1) + 1 (1 + 2)      = -10
    The eight values differ from each other, so a slot written with another's quantity, a dropped 1/2, a missing
    u or du/dt, or a wrong component pairing in v.a changes at least one of them."""
    m = np.array([2.0, 0.5, 1.0])
    v = np.array([[1.0, -2.0, 3.0], [-4.0, 0.0, 2.0], [1.0, 1.0, 0.0]])
    a = np.array([[0.5, 1.0, -1.0], [2.0, -4.0, 0.0], [-2.0, 3.0, 0.5]])
    u = np.array([1.5, 3.0, 0.0])
    du = np.array([0.25, -1.0, 2.0])
    out = oracle.reduce_sums(m, v, a, u, du)
    np.testing.assert_array_equal(out, [1.0, -3.0, 7.0, 0.0, 3.0, -1.5, 24.5, -10.0])
    # the empty sum
    np.testing.assert_array_equal(oracle.reduce_sums(np.zeros(0), np.zeros((0, 3)), np.zeros((0, 3)), np.zeros(0),
                                                     np.zeros(0)), np.zeros(8))


def test_reduce_of_oracle_forces_conserves_momentum_and_energy(oracle):
    """On a random state whose a and du/dt come from the (separately pinned) force, the momentum change
    sum m a (slots 3-5) and the energy change sum m (v.a + du/dt) (slot 7) vanish to round-off: the pair terms
    are antisymmetric, and a pair's energy terms cancel.  The momentum slots 0-2 and the energy slot 6 are
    non-zero on that state."""
    f = wl.jittered_lattice(8, jitter=0.3, vel_sigma=0.3, seed=5)
    p = wl.SPH_PARAMS
    rho = oracle.density(f["x"], f["mass"], f["h"], f["box"])
    P, cs = oracle.eos(rho, f["u"], p["gamma"])
    a, du = oracle.force(f["x"], f["v"], f["mass"], f["h"], rho, P, cs, f["box"], True, p["alpha"], p["beta"],
                         p["eps"])
    out = oracle.reduce_sums(f["mass"], f["v"], a, f["u"], du)
    scale_a = np.sum(f["mass"] * np.linalg.norm(a, axis=1))
    scale_e = np.sum(f["mass"] * (np.abs(np.sum(f["v"] * a, axis=1)) + np.abs(du)))
    assert np.all(np.abs(out[3:6]) <= 1e-13 * scale_a)
    assert abs(out[7]) <= 1e-13 * scale_e
    assert np.all(np.abs(out[0:3]) > 1e-6) and out[6] > 0.0


def test_kick_drift_closed_form(oracle):
    v = np.array([[1.0, -2.0, 0.5]])
    a = np.array([[0.5, 0.25, -1.0]])
    v2, u2 = oracle.kick(0.5, a, np.array([2.0]), v, np.array([1.0]))
    np.testing.assert_array_equal(v2, [[1.25, -1.875, 0.0]])
    np.testing.assert_array_equal(u2, [2.0])
    x2 = oracle.drift(0.25, np.array([[1.0, -2.0, 0.0]]), np.array([[0.875, 0.25, 0.5]]), np.ones(3))
    np.testing.assert_allclose(x2, [[0.125, 0.75, 0.5]], atol=1e-15)


def test_lattice_neighbour_count_is_57(oracle):
    # |k| < 2.4 spacing holds for exactly 57 lattice vectors (shells 0..5: 1+6+12+8+6+24), self included.
    f = wl.jittered_lattice(12, jitter=0.0)
    for i in (0, 77, 1000):
        nb = oracle.neighbours(f["x"], f["h"], f["box"], i)
        assert nb.size == 57 and i in nb


def test_scatter_f32_widens_exactly(oracle):
    lay = wl.default_layout()
    f = wl.jittered_lattice(4, jitter=0.2)
    aos, _ = wl.pack_aos(f, lay)
    n = aos.shape[0]
    vals = np.random.default_rng(2).normal(size=(3, n)).astype(np.float32)
    perm = np.arange(n, dtype=np.int32)
    oracle.scatter(aos, lay["stride"], perm, lay["offsets"]["a"], vals)
    back = oracle.gather(aos, lay["stride"], perm, lay["offsets"]["a"], 3)
    np.testing.assert_array_equal(back, vals.astype(np.float64))


def test_sampled_pass_equals_full_pass(oracle):
    f = wl.jittered_lattice(8, jitter=0.1, vel_sigma=0.1)
    lay = wl.default_layout()
    aos, _ = wl.pack_aos(f, lay)
    full = oracle.step_all(aos, lay, f["box"], wl.SPH_PARAMS)
    tg = np.array([0, 5, 100, 511])
    smp = oracle.step_sampled(aos, lay, f["box"], wl.SPH_PARAMS, tg)
    for k in ("rho", "P", "cs", "a", "dudt"):
        np.testing.assert_array_equal(smp[k], full[k][tg])


def test_fp32_position_round_trip_within_float_rounding(oracle):
    lay = wl.default_layout()
    f = wl.jittered_lattice(9, jitter=0.45, seed=13)
    aos, _ = wl.pack_aos(f, lay)
    nc = np.array([4, 3, 5], np.int32)
    x = oracle.unpack(aos, lay)["x"]
    _, _, perm, cos, _ = oracle.bin_cells(x, f["box"], nc)
    rel = oracle.gather_pos_f32(aos, lay["stride"], perm, lay["offsets"]["x"], cos, f["box"], nc)
    out = aos.copy()
    oracle.scatter_pos_f32(out, lay["stride"], perm, lay["offsets"]["x"], cos, f["box"], nc, rel)
    back = oracle.unpack(out, lay)["x"]
    edge = f["box"] / nc
    # |rel| <= edge, so the float rounding error is at most half an ulp of the edge (2^-24 relative)
    assert np.all(np.abs(back - x) <= edge * 2.0 ** -24 + 1e-17)
    changed = np.any(out != aos, axis=0)
    o = lay["offsets"]["x"]
    assert not changed[:o].any() and not changed[o + 24:].any()


# --------------------------------------------------------------------------------------------------------
# Patches (independent open boxes)
# --------------------------------------------------------------------------------------------------------
def test_patch_grids_respect_interaction_radius(oracle):
    f = wl.patches(12, lam_lo=8, lam_hi=80, seed=3)
    r = oracle.bin_patches(f["x"], f["h"], f["patch_start"], f["box"], 8)
    ps = f["patch_start"]
    for p in range(12):
        hm = f["h"][ps[p]:ps[p + 1]].max()
        for d in range(3):
            nn = r["patch_n"][p, d]
            edge = f["box"][d] / nn
            assert edge >= 2 * hm                       # every pair within 2h lies in neighbouring cells
            assert nn == 8 or nn + 1 > f["box"][d] / (2 * hm)   # and the grid is the finest that allows it
    # stable cell-major order; every slot's cell contains its position
    n = f["h"].size
    assert np.array_equal(np.sort(r["perm"]), np.arange(n))
    for c in range(r["ncells"]):
        seg = r["perm"][r["cell_start"][c]:r["cell_start"][c + 1]]
        assert np.all(np.diff(seg) > 0)
        assert np.all(r["cell_of"][seg] == c)
    # cells never mix patches
    patch_of = np.searchsorted(ps, np.arange(n), side="right") - 1
    patch_of_cell = np.searchsorted(r["patch_cell_base"], r["cell_of"], side="right") - 1
    assert np.array_equal(patch_of, patch_of_cell)


def test_patches_do_not_interact(oracle):
    # two copies of one patch side by side give identical results; a patch with one particle gives m W(0, h)
    rng = np.random.default_rng(4)
    k = 300
    x = rng.uniform(0, 3, size=(k, 3))
    fields = {"x": np.concatenate([x, x, [[1.5, 1.5, 1.5]]]), "v": rng.normal(0, 0.2, size=(2 * k + 1, 3)),
              "mass": np.full(2 * k + 1, 0.01), "h": np.full(2 * k + 1, 0.3), "u": np.ones(2 * k + 1)}
    fields["v"][k:2 * k] = fields["v"][:k]
    lay = wl.default_layout()
    aos, _ = wl.pack_aos(fields, lay, order="given")
    ps = np.array([0, k, 2 * k, 2 * k + 1])
    out = oracle.step_patches(aos, lay, ps, np.full(3, 3.0), wl.SPH_PARAMS)
    for key in ("rho", "P", "cs", "dudt"):
        np.testing.assert_array_equal(out[key][:k], out[key][k:2 * k])
    np.testing.assert_array_equal(out["a"][:k], out["a"][k:2 * k])
    assert out["rho"][-1] == pytest.approx(0.01 / (PI * 0.3 ** 3), rel=1e-15)
    assert np.all(out["a"][-1] == 0.0)


def test_patch_fp32_positions_round_trip(oracle):
    f = wl.patches(5, lam_lo=10, lam_hi=40, seed=6)
    lay = wl.default_layout()
    aos, _ = wl.pack_aos(f, lay, order="given")
    r = oracle.bin_patches(f["x"], f["h"], f["patch_start"], f["box"], 8)
    rel = oracle.gather_pos_f32_patches(aos, lay["stride"], r["perm"], lay["offsets"]["x"], r["cell_of_slot"],
                                        r["patch_cell_base"], r["patch_n"], f["box"])
    x = f["x"][r["perm"]]
    patch_of_cell = np.searchsorted(r["patch_cell_base"], r["cell_of_slot"], side="right") - 1
    edge = f["box"][None, :] / r["patch_n"][patch_of_cell]
    assert np.all(rel.T >= 0) and np.all(rel.T <= edge.astype(np.float32))
    local = r["cell_of_slot"] - r["patch_cell_base"][patch_of_cell]
    nn = r["patch_n"][patch_of_cell]
    k = np.stack([local % nn[:, 0], (local // nn[:, 0]) % nn[:, 1], local // (nn[:, 0] * nn[:, 1])], axis=1)
    back = k * edge + rel.T.astype(np.float64)
    assert np.all(np.abs(back - x) <= edge * 2.0 ** -24 + 1e-16)


# ---- smoothing-length iteration (Section 2.1, step 1) ----
def test_h_iteration_isolated_particles_closed_form(oracle):
    """A particle with no neighbour has rho = m W(0, h) = m / (pi h^3), so every round multiplies h by
    eta pi^(1/3) exactly and the iteration never terminates."""
    x = np.array([[1.0, 1.0, 1.0], [20.0, 1.0, 1.0], [1.0, 40.0, 60.0]])
    m = np.array([1.0, 2.0, 0.5])
    h0 = np.array([0.1, 0.2, 0.05])
    eta = 1.2
    h, rho, it, left = oracle.h_iterate(x, m, h0, np.full(3, 100.0), periodic=False, eta=eta, tol=1e-6, max_iter=3)
    g = eta * np.pi ** (1.0 / 3.0)
    np.testing.assert_allclose(h, h0 * g ** 3, rtol=1e-13)
    np.testing.assert_allclose(rho, m / (np.pi * h ** 3), rtol=1e-13)
    assert it == 3 and left == 3


def test_h_iteration_scale_invariance(oracle):
    """x -> 2x, box -> 2 box, h -> 2h, m -> 8m leaves every density unchanged, so the iteration must return 2h
    after the same number of rounds: this fixes the exponent 1/3 and the m / rho ratio of the update."""
    f = wl.clustered(400, sigma=0.08, peak=4.0, n_side_equiv=8, seed=4)
    h1, rho1, it1, left1 = oracle.h_iterate(f["x"], f["mass"], f["h"], f["box"], eta=1.2, tol=1e-6, max_iter=30)
    h2, rho2, it2, left2 = oracle.h_iterate(2 * f["x"], 8 * f["mass"], 2 * f["h"], 2 * f["box"], eta=1.2,
                                            tol=1e-6, max_iter=30)
    assert it1 == it2 and left1 == left2 == 0
    np.testing.assert_allclose(h2, 2 * h1, rtol=1e-13)
    np.testing.assert_allclose(rho2, rho1, rtol=1e-12)


def test_h_iteration_perfect_lattice_fixed_point(oracle):
    """On a perfect periodic lattice every particle sees the same neighbourhood, so all converge to one h; that h
    solves h = eta (m / rho(h))^(1/3) to within the termination tolerance, and sits near eta s (the update is
    exact at uniform density)."""
    ns = 8
    s = 1.0 / ns
    idx = np.indices((ns, ns, ns)).reshape(3, -1).T.astype(np.float64)
    x = (idx + 0.5) * s
    n = ns ** 3
    m = np.full(n, 1.0 / n)
    tol = 1e-8
    h, rho, it, left = oracle.h_iterate(x, m, np.full(n, 1.05 * s), np.ones(3), eta=1.2, tol=tol, max_iter=50)
    assert left == 0 and 1 < it < 50
    assert np.ptp(h) <= 1e-12 * h[0]
    assert 1.1 < h[0] / s < 1.3
    resid = 1.2 * np.cbrt(m / rho) - h
    assert np.max(np.abs(resid)) <= 2 * tol * h[0]


def test_h_iteration_stops_at_max_iter(oracle):
    f = wl.tiny()
    h, rho, it, left = oracle.h_iterate(f["x"], f["mass"], f["h"], f["box"], max_iter=1)
    assert it == 1 and 0 < left <= len(h)
    h_full, _, it_full, left_full = oracle.h_iterate(f["x"], f["mass"], f["h"], f["box"], max_iter=30)
    assert left_full == 0 and it_full > 1
