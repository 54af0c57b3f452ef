"""Pins for the oracle's sediment refraction model (Sec. III-B: a refraction
model in the propagation time for imaging below the seabed): a flat
interface with water above and sediment (sound speed c_s) below; a leg from a
sensor in the water to a point below crosses where the travel time is
stationary (Fermat)."""
import numpy as np
import pytest

import oracle

C = 1500.0
SIG = oracle.Signal(fc=100e3, fs=40e3, c=C, t0=0.0, n_samples=1024)


def _leg_by_minimiser(x, s, zint, cs):
    """Water-metre length of the leg by a bounded scalar minimiser of the
    travel time over the crossing point's horizontal distance (scipy)."""
    from scipy.optimize import minimize_scalar
    a, b = zint - s[2], x[2] - zint
    rho = np.hypot(x[0] - s[0], x[1] - s[1])
    n = C / cs
    L = lambda xi: np.hypot(xi, a) + n * np.hypot(rho - xi, b)
    r = minimize_scalar(L, bounds=(0.0, rho), method="bounded", options={"xatol": 1e-13, "maxiter": 2000})
    return min(L(r.x), L(0.0), L(rho))


def test_equal_speeds_and_points_above_are_straight():
    t, r = np.array([0.0, 0.0, -2.0]), np.array([0.1, 0.05, -2.0])
    for x in (np.array([0.4, 1.5, 0.3]), np.array([-0.2, 0.8, -0.1])):
        straight = oracle.delay(x, t, r, None, C)[0]
        with oracle.medium(0.0, C):
            assert abs(oracle.delay(x, t, r, None, C)[0] - straight) < 1e-15
    with oracle.medium(0.0, 1700.0):
        x = np.array([0.4, 1.5, -0.05])                 # above the interface: water only
        assert oracle.delay(x, t, r, None, C)[0] == (np.linalg.norm(x - t) + np.linalg.norm(x - r)) / C


def test_vertical_leg_closed_form():
    s = np.array([0.3, -0.2, -2.0])
    x = np.array([0.3, -0.2, 0.45])
    with oracle.medium(0.0, 1750.0):
        tau = oracle.delay(x, s, s, None, C)[0]
    assert abs(tau - 2 * (2.0 + (C / 1750.0) * 0.45) / C) < 1e-16


@pytest.mark.parametrize("cs", [1600.0, 1750.0, 1400.0])
def test_refracted_leg_is_the_travel_time_minimum(cs):
    rng = np.random.default_rng(int(cs))
    with oracle.medium(0.1, cs):
        for _ in range(25):
            s = np.array([rng.uniform(-1, 1), rng.uniform(-1, 1), rng.uniform(-3, -1)])
            x = np.array([rng.uniform(-2, 2), rng.uniform(-2, 2), 0.1 + rng.uniform(0.01, 1.0)])
            tau = oracle.delay(x, s, s, None, C)[0]
            L = _leg_by_minimiser(x, s, 0.1, cs)
            assert abs(0.5 * tau * C - L) <= 1e-12 * L
            # and it is shorter (in time) than the straight path through the interface
            assert 0.5 * tau * C <= np.linalg.norm(x - s) * max(1.0, C / cs) + 1e-12


def test_point_below_the_interface_focuses_only_with_the_model():
    """Echoes of a buried point simulated with refraction focus to I = A P C at
    that voxel when imaged with refraction (32-tap truth interpolator, ideal
    pulse); imaging with straight paths loses coherence."""
    P, C_ = 16, 4
    lat = np.arange(4) * 0.3 - 0.45
    pos = np.array([[x, y, -2.0] for y in lat for x in lat])
    rxl = np.array([[dx, dy, 0.0] for dy in (-0.02, 0.02) for dx in (-0.02, 0.02)])
    tx, rx = oracle.sensor_positions(pos, np.zeros((P, 3)), np.zeros(3), rxl)
    A = 0.7 * np.exp(-0.4j)
    scat = np.array([[0.05, -0.1, 0.35, A.real, A.imag]])
    with oracle.medium(0.0, 1700.0):
        echo = oracle.simulate_points(tx, rx, SIG, 20e3, 0.0, scat)
        I_r = oracle.backproject(tx, rx, SIG, echo, 32, 10.0, scat[:, :3])[0]
    assert abs(I_r - A * P * C_) <= 1e-4 * abs(A) * P * C_
    I_s = oracle.backproject(tx, rx, SIG, echo, 32, 10.0, scat[:, :3])[0]
    assert abs(I_s) < 0.5 * abs(A) * P * C_


def test_adjoint_and_gradient_with_refraction():
    P, C_ = 4, 2
    rng = np.random.default_rng(7)
    pos = np.stack([rng.uniform(-0.5, 0.5, P), rng.uniform(-0.5, 0.5, P), np.full(P, -2.0)], 1)
    rxl = np.array([[-0.02, 0.0, 0.0], [0.02, 0.0, 0.0]])
    att = rng.uniform(-0.05, 0.05, (P, 3))
    pix = oracle.grid_points(-0.2, -0.2, -0.1, 0.06, 0.06, 0.07, 6, 5, 4)   # layers above and below z = 0
    e = rng.normal(size=(P, C_, SIG.n_samples)) + 1j * rng.normal(size=(P, C_, SIG.n_samples))
    img = rng.normal(size=pix.shape[0]) + 1j * rng.normal(size=pix.shape[0])
    with oracle.medium(0.0, 1650.0):
        tx, rx = oracle.sensor_positions(pos, att, np.zeros(3), rxl)
        Be = oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix)
        BhI = oracle.backproject_adjoint(tx, rx, SIG, img, 8, 4.0, pix)
        lhs, rhs = np.vdot(Be, img), np.vdot(e, BhI)
        assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
        off = rng.normal(0, 0.002, size=(P, 3))

        def S(o):
            t, r = oracle.sensor_positions(pos, att, np.zeros(3), rxl, o)
            return oracle.sharpness(oracle.backproject(t, r, SIG, e, 8, 4.0, pix))[0]

        t, r = oracle.sensor_positions(pos, att, np.zeros(3), rxl, off)
        _, g = oracle.sharpness(oracle.backproject(t, r, SIG, e, 8, 4.0, pix), want_grad=True)
        grad = oracle.vjp_offsets(t, r, SIG, e, 8, 4.0, pix, g)
        h = 1e-7
        fd = np.zeros((P, 3))
        for i in range(P):
            for a in range(3):
                op, om = off.copy(), off.copy()
                op[i, a] += h
                om[i, a] -= h
                fd[i, a] = (S(op) - S(om)) / (2 * h)
    assert oracle.rel_l2(grad, fd) < 1e-6
