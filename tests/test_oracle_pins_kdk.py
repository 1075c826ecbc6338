"""Pins of the oracle's leapfrog runs (Section 2.1 steps 3-5) against facts fixed by the mathematics: closed-form
reflections at the walls of an open box, the order of the energy error in dt (first order when the force sees the
half-step velocity, second order when it sees the predicted values the second kick resets, Section 2.2), exact
continuation of a run from its own records, and isolated particles moving on straight lines."""
import numpy as np
import pytest

from paper_2502_16517_gb300 import workloads as wl


def test_drift_walls_closed_form(oracle):
    box = np.array([1.0, 2.0, 4.0])
    x = np.array([[0.875, 0.25, 2.0], [0.125, 1.5, 3.5], [0.5, 1.0, 0.5]])
    v = np.array([[0.5, -2.0, 1.0], [-1.0, 2.0, 4.0], [8.0, -12.0, 0.0]])
    x2, v2 = oracle.drift_walls(0.25, v, x, box)
    # row 0: 1.0 (on the wall, kept), -0.25 -> 0.25 (v flips), 2.25;  row 1: -0.125 -> 0.125, 2.0 -> kept on
    # the wall, 4.5 -> 3.5 (v flips); row 2: 2.5 -> 2 - 2.5 = -0.5 -> clamped to 0, -2.0 -> 2.0 (flip), 0.5
    np.testing.assert_array_equal(x2, [[1.0, 0.25, 2.25], [0.125, 2.0, 3.5], [0.0, 2.0, 0.5]])
    np.testing.assert_array_equal(v2, [[0.5, 2.0, 1.0], [1.0, 2.0, -4.0], [-8.0, 12.0, 0.0]])


def test_isolated_particles_move_on_straight_lines(oracle):
    """Particles farther apart than their supports feel no force: a, du/dt stay 0, u is unchanged, and positions
    advance by v dt per step, mirrored at the walls (with and without prediction, in patches)."""
    x = np.array([[0.5, 0.5, 0.5], [2.5, 2.5, 2.5], [1.0, 1.0, 1.0]])
    v = np.array([[0.25, 0.0, -0.5], [0.0, 0.5, 0.0], [1.0, 0.0, 0.0]])
    f = {"x": x, "v": v, "u": np.array([1.0, 2.0, 3.0]), "mass": np.ones(3), "h": np.full(3, 0.1)}
    box = np.array([3.0, 3.0, 3.0])
    for predict in (False, True):
        r = oracle.kdk_run(f, box, wl.SPH_PARAMS, 0.5, 4, periodic=False, predict=predict,
                           patch_start=np.array([0, 2, 3]))
        np.testing.assert_array_equal(r["a"], 0.0)
        np.testing.assert_array_equal(r["dudt"], 0.0)
        np.testing.assert_array_equal(r["u"], f["u"])
        # 2 time units: particle 0 moves (0.5, 0, -1) -> z = -0.5 mirrored to 0.5; particle 1 moves 1 in y ->
        # 3.5 mirrored to 2.5; particle 2 moves 2 in x -> 3.0, on the wall
        np.testing.assert_array_equal(r["x"], [[1.0, 0.5, 0.5], [2.5, 2.5, 2.5], [3.0, 1.0, 1.0]])
        np.testing.assert_array_equal(r["v"], [[0.25, 0.0, 0.5], [0.0, -0.5, 0.0], [1.0, 0.0, 0.0]])


def _energy_errors(oracle, f, params, T, ks, predict, patch_start=None, periodic=True):
    E0 = oracle.energy(f["mass"], f["v"], f["u"])
    out = []
    for k in ks:
        r = oracle.kdk_run(f, f["box"], params, T / k, k, periodic=periodic, predict=predict,
                           patch_start=patch_start)
        out.append((oracle.energy(f["mass"], r["v"], r["u"]) - E0) / E0)
    return np.array(out)


def test_energy_error_order_periodic(oracle):
    """The semi-discrete equations conserve sum m (|v|^2/2 + u); the leapfrog's energy error over a fixed time
    halves with dt when the force sees the half-step velocity and internal energy (first order), and falls by
    four when it sees the predicted values (second order).  A prediction with the wrong sign, or a velocity left
    at its half-step value, does not give the second order."""
    p = wl.SPH_PARAMS
    f = wl.jittered_lattice(8, jitter=0.2, vel_sigma=0.3, seed=3)
    r0 = oracle.kdk_run(f, f["box"], p, 0.0, 0)
    dt0 = 0.3 * f["h"].min() / np.max(r0["cs"] + np.linalg.norm(f["v"], axis=1))
    ks = (20, 40, 80)
    plain = _energy_errors(oracle, f, p, 5 * dt0, ks, predict=False)
    pred = _energy_errors(oracle, f, p, 5 * dt0, ks, predict=True)
    assert np.all(plain > 0)
    assert 1.9 < plain[0] / plain[1] < 2.1 and 1.9 < plain[1] / plain[2] < 2.1
    assert 3.4 < pred[0] / pred[1] < 4.6 and 3.6 < pred[1] / pred[2] < 4.4
    assert np.all(np.abs(pred) < 0.1 * plain)


def test_trajectory_error_order_periodic(oracle):
    """Self-convergence of the final state over a fixed time with k, 2k and 4k steps: successive differences
    shrink by 4 (second order) for x, v and u with the predicted values, by 2 without.  Unlike the energy, whose
    order a pressure from the half-step u does not spoil (P enters a and du/dt consistently), the trajectory needs
    both v and u predicted: leaving u at its half-step value brings its order down to about 2."""
    p = wl.SPH_PARAMS
    f = wl.jittered_lattice(8, jitter=0.2, vel_sigma=0.3, seed=3)
    r0 = oracle.kdk_run(f, f["box"], p, 0.0, 0)
    dt0 = 0.3 * f["h"].min() / np.max(r0["cs"] + np.linalg.norm(f["v"], axis=1))
    for predict, lo, hi in ((True, 3.4, 4.6), (False, 1.8, 2.2)):
        rs = [oracle.kdk_run(f, f["box"], p, 5 * dt0 / k, k, predict=predict) for k in (20, 40, 80)]
        for key in ("x", "v", "u"):
            d0 = np.max(np.abs(rs[0][key] - rs[1][key]))
            d1 = np.max(np.abs(rs[1][key] - rs[2][key]))
            assert lo < d0 / d1 < hi, (predict, key, d0 / d1)


def test_energy_error_order_open_patches(oracle):
    """The same in independent open patches with reflecting walls: the walls turn velocities without changing
    |v|, so the energy error keeps its order; every position stays inside its patch box."""
    p = wl.SPH_PARAMS
    fp = wl.patches(3, lam_lo=8, lam_hi=16, vel_sigma=0.3, seed=7)
    ps = fp["patch_start"]
    r0 = oracle.kdk_run(fp, fp["box"], p, 0.0, 0, patch_start=ps)
    dt0 = 0.3 * fp["h"].min() / np.max(r0["cs"] + np.linalg.norm(fp["v"], axis=1))
    ks = (40, 80, 160)
    plain = _energy_errors(oracle, fp, p, 20 * dt0, ks, predict=False, patch_start=ps)
    pred = _energy_errors(oracle, fp, p, 20 * dt0, ks, predict=True, patch_start=ps)
    assert 1.8 < plain[0] / plain[1] < 2.4 and 1.8 < plain[1] / plain[2] < 2.4
    assert pred[0] / pred[1] > 3.5 and pred[1] / pred[2] > 3.5
    r = oracle.kdk_run(fp, fp["box"], p, 20 * dt0 / 40, 40, patch_start=ps)
    assert r["x"].min() >= 0.0 and r["x"].max() <= 3.0
    assert np.sum(np.sign(r["v"]) != np.sign(fp["v"])) > 100          # the walls were hit


@pytest.mark.parametrize("predict", [False, True])
def test_run_continues_exactly_from_its_records(oracle, predict):
    """Three steps equal two steps followed by one step that starts from the records' a and du/dt."""
    p = wl.SPH_PARAMS
    f = wl.jittered_lattice(6, jitter=0.2, vel_sigma=0.3, seed=4)
    dt = 2e-3
    full = oracle.kdk_run(f, f["box"], p, dt, 3, predict=predict)
    part = oracle.kdk_run(f, f["box"], p, dt, 2, predict=predict)
    part.update(mass=f["mass"], h=f["h"])
    rest = oracle.kdk_run(part, f["box"], p, dt, 1, predict=predict, from_records=True)
    for k in ("x", "v", "u", "rho", "P", "cs", "a", "dudt"):
        np.testing.assert_array_equal(rest[k], full[k], err_msg=k)
