"""Pins of the oracle's kernel families and fuller density / force views against facts that do not come from
the oracle's pair loops: closed values of the quartic spline M5, quadrature of its normalisation, finite
differences, lattice sums over integer offsets (the exact value of an SPH estimate on a uniform lattice),
hand-derived two-particle cases, and the conservation laws of the symmetrised equations.  Chosen so that a
dropped term, a wrong sign, a swapped i/j or a wrong power of h fails one of them.
"""
import itertools
import math

import numpy as np
import pytest

PI = math.pi
M4, M5 = 0, 1


def _gauss(f, edges, npts=4):
    t, wt = np.polynomial.legendre.leggauss(npts)
    total = 0.0
    for lo, hi in zip(edges[:-1], edges[1:]):
        r = 0.5 * (hi - lo) * t + 0.5 * (hi + lo)
        total += 0.5 * (hi - lo) * np.sum(wt * f(r))
    return total


# --------------------------------------------------------------------------------------------------------
# Kernel families
# --------------------------------------------------------------------------------------------------------
@pytest.mark.parametrize("h", [0.02, 0.3, 1.0])
def test_m5_unit_integral_and_zero_h_derivative_integral(oracle, h):
    # int W dV = 1 for every h; hence int dW/dh dV = 0.  The integrands are polynomials of degree <= 6 on
    # [0, h/2], [h/2, 3h/2], [3h/2, 5h/2], so 4-point Gauss-Legendre is exact to round-off.
    edges = [0.0, 0.5 * h, 1.5 * h, 2.5 * h]
    hh = lambda r: np.full(r.size, h)
    total = _gauss(lambda r: oracle.kernel(M5, 0, r, hh(r)) * 4 * PI * r * r, edges)
    assert abs(total - 1.0) < 1e-13
    dh = _gauss(lambda r: oracle.kernel(M5, 2, r, hh(r)) * 4 * PI * r * r, edges)
    assert abs(dh) < 1e-12 / h


def test_m4_dwdh_integral_vanishes(oracle):
    h = 0.4
    dh = _gauss(lambda r: oracle.kernel(M4, 2, r, np.full(r.size, h)) * 4 * PI * r * r, [0.0, h, 2 * h])
    assert abs(dh) < 1e-12


def test_m5_closed_values(oracle):
    # f(q) = (5/2 - q)^4 - 5 (3/2 - q)^4 + 10 (1/2 - q)^4 (each term only while positive), sigma = 1/(20 pi):
    # f(0) = 14.375, f(1/2) = 11, f(1) = 4.75, f(3/2) = 1, f(5/2) = 0; f'(0) = 0, f'(1/2) = -12, f'(1) = -11,
    # f'(3/2) = -4, f'(5/2) = 0.
    h = 0.25
    q = np.array([0.0, 0.5, 1.0, 1.5, 2.5, 3.0])
    f = oracle.kernel(M5, 0, q * h, np.full(q.size, h)) * 20 * PI * h ** 3
    fp = oracle.kernel(M5, 1, q * h, np.full(q.size, h)) * 20 * PI * h ** 4
    np.testing.assert_allclose(f, [14.375, 11.0, 4.75, 1.0, 0.0, 0.0], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(fp, [0.0, -12.0, -11.0, -4.0, 0.0, 0.0], rtol=1e-14, atol=1e-13)
    assert oracle.kappa(M5) == 2.5 and oracle.kappa(M4) == 2.0


def test_m4_family_form_equals_the_piecewise_cubic(oracle):
    h = 0.3
    r = np.linspace(0.0, 0.7, 301)
    hh = np.full(r.size, h)
    np.testing.assert_allclose(oracle.kernel(M4, 0, r, hh), oracle.w(r, hh), rtol=1e-14, atol=1e-16)
    np.testing.assert_allclose(oracle.kernel(M4, 1, r, hh), oracle.dwdr(r, hh), rtol=1e-13, atol=1e-15)


@pytest.mark.parametrize("kern", [M4, M5])
def test_kernel_family_derivatives_match_finite_differences(oracle, kern):
    h = 0.3
    kap = oracle.kappa(kern)
    r = np.linspace(0.013, kap * h - 0.013, 113)
    hh = np.full(r.size, h)
    e = 1e-6
    fd_r = (oracle.kernel(kern, 0, r + e, hh) - oracle.kernel(kern, 0, r - e, hh)) / (2 * e)
    dwdr = oracle.kernel(kern, 1, r, hh)
    assert np.max(np.abs(fd_r - dwdr)) < 1e-6 * np.abs(dwdr).max()
    fd_h = (oracle.kernel(kern, 0, r, hh + e) - oracle.kernel(kern, 0, r, hh - e)) / (2 * e)
    dwdh = oracle.kernel(kern, 2, r, hh)
    assert np.max(np.abs(fd_h - dwdh)) < 1e-6 * np.abs(dwdh).max()


def test_m5_is_smooth_across_its_knots(oracle):
    # M5 is a quartic spline: W, W' and W'' are continuous at q = 1/2, 3/2, 5/2.
    h = np.array([1.0])
    for q0 in (0.5, 1.5, 2.5):
        e = 1e-7
        lo, hi = np.array([q0 - e]), np.array([q0 + e])
        assert abs(oracle.kernel(M5, 0, lo, h)[0] - oracle.kernel(M5, 0, hi, h)[0]) < 1e-6
        assert abs(oracle.kernel(M5, 1, lo, h)[0] - oracle.kernel(M5, 1, hi, h)[0]) < 1e-6
        d = 1e-4
        s_lo = (oracle.kernel(M5, 1, lo, h)[0] - oracle.kernel(M5, 1, lo - d, h)[0]) / d
        s_hi = (oracle.kernel(M5, 1, hi + d, h)[0] - oracle.kernel(M5, 1, hi, h)[0]) / d
        assert abs(s_lo - s_hi) < 1e-3


# --------------------------------------------------------------------------------------------------------
# Fuller density view on a uniform lattice: exact lattice sums over integer offsets
# --------------------------------------------------------------------------------------------------------
def _offsets(kern, s, h, kap):
    rng = int(math.ceil(kap * h / s)) + 1
    ks = np.array(list(itertools.product(range(-rng, rng + 1), repeat=3)), np.float64) * s
    r = np.sqrt((ks ** 2).sum(1))
    keep = r < kap * h
    return ks[keep], r[keep]


@pytest.mark.parametrize("kern", [M4, M5])
def test_lattice_velocity_estimates_and_omega_equal_their_lattice_sums(oracle, kern):
    # Interior particle of an open cubic lattice (spacing s, h = 1.23 s, so that no lattice distance lies on the
    # support radius) with v = c x + w x x.  With the offset
    # sums S0 = sum W(r_k), S2 = sum r_k^2 G(r_k) (G = W'/r) and Sh = sum dW/dh(r_k):
    #   rho = m S0,  div v = -c S2 / S0,  curl v = -(2/3) (S2 / S0) w,  Omega = 1 + h Sh / (3 S0),
    # exactly, because the lattice is symmetric under axis swaps and reflections.  In the continuum limit
    # -S2/S0 -> 3, so div v ~ 3c and curl v ~ 2w.
    n_side, s = 13, 1.0 / 13
    h = 1.23 * s
    kap = oracle.kappa(kern)
    g = (np.arange(n_side) + 0.5) * s
    x = np.array(list(itertools.product(g, g, g)))
    c, w = 0.7, np.array([0.3, -0.2, 0.5])
    v = c * x + np.cross(w, x)
    m = np.full(len(x), 1.0 / len(x))
    hv = np.full(len(x), h)
    centre = len(x) // 2
    assert np.allclose(x[centre], 0.5)
    d = oracle.density_ext(kern, x, v, m, hv, np.ones(3), periodic=False, targets=[centre])
    ks, r = _offsets(kern, s, h, kap)
    hr = np.full(r.size, h)
    S0 = oracle.kernel(kern, 0, r, hr).sum()
    nz = r > 0
    G = oracle.kernel(kern, 1, r[nz], hr[nz]) / r[nz]
    S2 = (r[nz] ** 2 * G).sum()
    Sh = oracle.kernel(kern, 2, r, hr).sum()
    assert d["rho"][0] == pytest.approx(m[0] * S0, rel=1e-13)
    assert d["divv"][0] == pytest.approx(-c * S2 / S0, rel=1e-12)
    np.testing.assert_allclose(d["curlv"][0], -(2.0 / 3.0) * (S2 / S0) * w, rtol=1e-11, atol=1e-14)
    assert d["omega"][0] == pytest.approx(1.0 + h * Sh / (3 * S0), rel=1e-13)
    assert d["nnb"][0] == np.count_nonzero(nz)
    assert d["divv"][0] == pytest.approx(3 * c, rel=0.03)
    np.testing.assert_allclose(d["curlv"][0], 2 * w, rtol=0.03)


def test_lattice_neighbour_counts(oracle):
    # h = 1.23 s: the lattice points with |k| < 2.46 (M4: |k|^2 <= 6) and |k| < 3.075 (M5: |k|^2 <= 9), self
    # excluded.  Shell sizes of |k|^2 = 1, 2, 3, 4, 5, 6, 8, 9 on the cubic lattice: 6, 12, 8, 6, 24, 24, 12, 30
    # (none at 7).
    expect = {M4: 6 + 12 + 8 + 6 + 24 + 24, M5: 6 + 12 + 8 + 6 + 24 + 24 + 12 + 30}
    n_side, s = 10, 0.1
    g = (np.arange(n_side) + 0.5) * s
    x = np.array(list(itertools.product(g, g, g)))
    for kern in (M4, M5):
        d = oracle.density_ext(kern, x, np.zeros_like(x), np.full(len(x), 1e-3), np.full(len(x), 1.23 * s),
                               np.ones(3), periodic=True, targets=[0, 123, 999])
        assert np.all(d["nnb"] == expect[kern])


def test_two_particle_divergence_and_curl_by_hand(oracle):
    # i at the origin moving with v_i, j at (d, 0, 0) at rest; x_ij = (-d, 0, 0), grad_i W = G x_ij, G = W'(d)/d.
    for kern in (M4, M5):
        h, d, mm = 0.2, 0.23, 0.5
        x = np.array([[0.3, 0.3, 0.3], [0.3 + d, 0.3, 0.3]])
        hv = np.full(2, h)
        G = oracle.kernel(kern, 1, np.array([d]), np.array([h]))[0] / d
        rho_i = mm * (oracle.kernel(kern, 0, np.array([0.0]), np.array([h]))[0] +
                      oracle.kernel(kern, 0, np.array([d]), np.array([h]))[0])
        u = 0.9
        v = np.array([[u, 0.0, 0.0], [0.0, 0.0, 0.0]])
        out = oracle.density_ext(kern, x, v, np.full(2, mm), hv, np.ones(3), periodic=False, targets=[0])
        assert out["divv"][0] == pytest.approx(mm * u * G * d / rho_i, rel=1e-14)  # -(1/rho) m (u)(G)(-d)
        np.testing.assert_allclose(out["curlv"][0], 0.0, atol=1e-30)
        v = np.array([[0.0, u, 0.0], [0.0, 0.0, 0.0]])
        out = oracle.density_ext(kern, x, v, np.full(2, mm), hv, np.ones(3), periodic=False, targets=[0])
        np.testing.assert_allclose(out["curlv"][0], [0.0, 0.0, mm * u * G * d / rho_i], rtol=1e-14, atol=1e-30)
        assert out["divv"][0] == 0.0
        assert out["nnb"][0] == 1.0


# --------------------------------------------------------------------------------------------------------
# Fuller force view
# --------------------------------------------------------------------------------------------------------
def _random_state(seed, n=60, kern=M4):
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.2, 0.8, (n, 3))
    v = rng.normal(0, 0.3, (n, 3))
    m = rng.uniform(0.5, 1.5, n) / n
    h = rng.uniform(0.08, 0.14, n)
    rho = rng.uniform(0.8, 1.2, n)
    P = rng.uniform(0.5, 1.0, n)
    cs = rng.uniform(0.9, 1.3, n)
    om = rng.uniform(0.7, 1.3, n)
    dv = rng.normal(0, 1.0, n)
    cv = rng.normal(0, 1.0, (n, 3))
    return x, v, m, h, rho, P, cs, om, dv, cv


def test_force_ext_with_switches_off_is_the_minimal_force(oracle):
    x, v, m, h, rho, P, cs, om, dv, cv = _random_state(3)
    a, du, _ = oracle.force_ext(M4, False, False, x, v, m, h, rho, P, cs, om, dv, cv, np.ones(3), False)
    a0, du0 = oracle.force(x, v, m, h, rho, P, cs, np.ones(3), False)
    # the same sums; the kernel family writes the cubic spline as truncated powers, which rounds differently
    np.testing.assert_allclose(a, a0, rtol=1e-12, atol=1e-12 * np.abs(a0).max())
    np.testing.assert_allclose(du, du0, rtol=1e-12, atol=1e-12 * np.abs(du0).max())


@pytest.mark.parametrize("kern", [M4, M5])
@pytest.mark.parametrize("switches", [(False, False), (True, False), (False, True), (True, True)])
def test_force_ext_conserves_momentum_and_energy(oracle, kern, switches):
    x, v, m, h, rho, P, cs, om, dv, cv = _random_state(5, kern=kern)
    a, du, _ = oracle.force_ext(kern, *switches, x, v, m, h, rho, P, cs, om, dv, cv, np.ones(3), False)
    ma = m[:, None] * a
    assert np.all(np.abs(ma.sum(0)) < 1e-13 * np.abs(ma).sum(0))
    pw = m * ((v * a).sum(1) + du)
    assert abs(pw.sum()) < 1e-13 * np.abs(pw).sum()


def test_gradh_terms_two_particles_by_hand(oracle):
    # alpha = beta = 0: a_i = -m_j (P_i / (Om_i rho_i^2) G_i + P_j / (Om_j rho_j^2) G_j) x_ij, with G_k = W'(r, h_k) / r
    # and unequal h, Omega, rho, P on the two sides (a swapped i/j fails).
    for kern in (M4, M5):
        x = np.array([[0.4, 0.4, 0.4], [0.47, 0.43, 0.41]])
        v = np.zeros((2, 3))
        m = np.array([0.3, 0.7])
        h = np.array([0.06, 0.045])
        rho, P, cs = np.array([1.1, 0.8]), np.array([0.6, 0.9]), np.array([1.0, 1.2])
        om, dv, cv = np.array([0.85, 1.2]), np.zeros(2), np.zeros((2, 3))
        a, du, _ = oracle.force_ext(kern, True, False, x, v, m, h, rho, P, cs, om, dv, cv, np.ones(3), False,
                                    alpha=0.0, beta=0.0)
        xij = x[0] - x[1]
        r = np.sqrt((xij ** 2).sum())
        Gi = oracle.kernel(kern, 1, np.array([r]), h[:1])[0] / r
        Gj = oracle.kernel(kern, 1, np.array([r]), h[1:])[0] / r
        expect = -m[1] * (P[0] / (om[0] * rho[0] ** 2) * Gi + P[1] / (om[1] * rho[1] ** 2) * Gj) * xij
        np.testing.assert_allclose(a[0], expect, rtol=1e-14)
        assert du[0] == 0.0


def test_balsara_scales_the_viscosity_by_the_pair_mean(oracle):
    x = np.array([[0.4, 0.4, 0.4], [0.46, 0.42, 0.4]])
    v = np.array([[0.5, 0.1, 0.0], [-0.3, 0.0, 0.2]])  # approaching: v_ij . r_ij < 0
    m = np.array([0.3, 0.7])
    h = np.array([0.05, 0.04])
    rho, P, cs = np.array([1.1, 0.8]), np.array([0.6, 0.9]), np.array([1.0, 1.2])
    om = np.ones(2)
    dv = np.array([-2.0, 0.7])
    cv = np.array([[0.5, -1.0, 0.3], [0.0, 0.4, 0.0]])
    args = (x, v, m, h, rho, P, cs, om, dv, cv, np.ones(3), False)
    a_off, du_off, _ = oracle.force_ext(M5, False, False, *args)
    a_on, du_on, _ = oracle.force_ext(M5, False, True, *args)
    a_nv, du_nv, _ = oracle.force_ext(M5, False, False, *args, alpha=0.0, beta=0.0)
    B = np.abs(dv) / (np.abs(dv) + np.sqrt((cv ** 2).sum(1)) + 1e-4 * cs / h)
    fac = 0.5 * (B[0] + B[1])
    assert 0.1 < fac < 0.9
    np.testing.assert_allclose(a_on[0] - a_nv[0], fac * (a_off[0] - a_nv[0]), rtol=1e-12)
    assert du_on[0] - du_nv[0] == pytest.approx(fac * (du_off[0] - du_nv[0]), rel=1e-12)


def test_signal_velocity_two_particles_by_hand(oracle):
    x = np.array([[0.4, 0.4, 0.4], [0.45, 0.4, 0.4]])
    m, h = np.array([0.3, 0.7]), np.array([0.05, 0.04])
    rho, P, cs = np.array([1.1, 0.8]), np.array([0.6, 0.9]), np.array([1.0, 1.2])
    z = (np.ones(2), np.zeros(2), np.zeros((2, 3)))
    # approaching along x: w = v_ij . r_ij / r = (0.5 - (-0.25)) * (-0.05) / 0.05 = -0.75
    v = np.array([[0.5, 0.0, 0.0], [-0.25, 0.0, 0.0]])
    _, _, vs = oracle.force_ext(M5, False, False, x, v, m, h, rho, P, cs, *z, np.ones(3), False)
    assert vs[0] == pytest.approx(1.0 + 1.2 + 3 * 0.75, rel=1e-15)
    # receding: no -3w term
    _, _, vs = oracle.force_ext(M5, False, False, x, -v, m, h, rho, P, cs, *z, np.ones(3), False)
    assert vs[0] == pytest.approx(2.2, rel=1e-15)
    # no neighbour within kappa max(h): 0
    _, _, vs = oracle.force_ext(M4, False, False, x, v, m, np.array([0.02, 0.02]), rho, P, cs, *z, np.ones(3),
                                False)
    assert vs[0] == 0.0


@pytest.mark.parametrize("kern", [M4, M5])
def test_extended_pass_on_a_lattice_at_rest(oracle, kern):
    # Periodic uniform lattice at rest: every velocity estimate and every force vanish, Omega is the lattice
    # sum of the previous test, and vsig = 2 c exactly (equal sound speeds, no approach).
    from paper_2502_16517_gb300 import workloads as wl
    n_side = 8
    s = 1.0 / n_side
    g = (np.arange(n_side) + 0.5) * s
    x = np.array(list(itertools.product(g, g, g)))
    f = {"x": x, "v": np.zeros_like(x), "mass": np.full(len(x), s ** 3), "h": np.full(len(x), 1.2 * s),
         "u": np.ones(len(x)), "a": np.zeros_like(x), "rho": np.zeros(len(x)), "P": np.zeros(len(x)),
         "dudt": np.zeros(len(x)), "cs": np.zeros(len(x))}
    lay = wl.default_layout()
    aos, _ = wl.pack_aos(f, lay, order="given", canary=False)
    params = dict(wl.SPH_PARAMS, kernel=kern, scheme=1)
    out = oracle.step_all_ext(aos, lay, np.ones(3), params)
    assert np.max(np.abs(out["a"])) < 1e-10
    assert np.max(np.abs(out["divv"])) < 1e-12 and np.max(np.abs(out["curlv"])) < 1e-12
    np.testing.assert_array_equal(out["vsig"], 2 * out["cs"])
    assert np.ptp(out["omega"]) < 1e-14 and np.all(out["omega"] > 0)
