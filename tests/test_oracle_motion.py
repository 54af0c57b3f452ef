"""Pins for the oracle's continuous-motion delay (Sec. II-D: transmission is
instantaneous and the platform keeps moving during reception): the receiver
at time t after transmission is at r + v t, and the two-way delay tau solves
c tau = |x - t_x| + |x - r - v tau|."""
import numpy as np
import pytest

import oracle
from oracle import brute

SIG = oracle.Signal(fc=100e3, fs=40e3, c=1500.0, t0=0.025, n_samples=512)


def _scene(P=5, C=2, seed=0):
    rng = np.random.default_rng(seed)
    pos = np.stack([np.arange(P) * 0.1, rng.normal(0, 0.02, P), -10.0 + rng.normal(0, 0.02, P)], 1)
    att = rng.uniform(-0.05, 0.05, size=(P, 3))
    txl = np.array([0.01, -0.02, 0.03])
    rxl = np.stack([(np.arange(C) - 0.5 * (C - 1)) * 0.025, np.full(C, 0.01), np.zeros(C)], 1)
    vel = np.stack([np.full(P, 1.95), rng.normal(0, 0.1, P), rng.normal(0, 0.1, P)], 1)
    return pos, att, txl, rxl, vel


def _echo(P, C, seed):
    rng = np.random.default_rng(seed)
    return rng.normal(size=(P, C, SIG.n_samples)) + 1j * rng.normal(size=(P, C, SIG.n_samples))


def test_zero_velocity_is_stop_and_hop():
    x, t, r = np.array([1.0, 16.0, 0.2]), np.array([0.0, 0.0, -10.0]), np.array([0.05, 0.01, -10.0])
    tau0, k0 = oracle.delay(x, t, r, None, SIG.c)
    assert tau0 == (np.linalg.norm(x - t) + np.linalg.norm(x - r)) / SIG.c and k0 == 1.0
    tau1, k1 = oracle.delay(x, t, r, np.zeros(3), SIG.c)
    assert tau1 == tau0 and k1 == 1.0


@pytest.mark.parametrize("v", [[1.95, 0.0, 0.0], [1.5, -0.8, 0.3], [-2.5, 1.0, -1.0], [40.0, 10.0, 0.0]])
def test_delay_is_the_root_brent(v):
    """The fixed point against Brent's root of the defining equation."""
    rng = np.random.default_rng(1)
    v = np.array(v)
    for _ in range(20):
        x = np.array([rng.uniform(-20, 20), rng.uniform(5, 60), rng.uniform(-1, 1)])
        t = np.array([0.0, 0.0, -10.0]) + rng.normal(0, 0.1, 3)
        r = t + rng.normal(0, 0.3, 3)
        tau, _ = oracle.delay(x, t, r, v, SIG.c)
        ref = brute.moving_receiver_tau(t[None], r[None, None], v[None], SIG.c, x[None])[0, 0, 0]
        assert abs(tau - ref) <= 4e-15 * ref
        assert abs(SIG.c * tau - np.linalg.norm(x - t) - np.linalg.norm(x - r - v * tau)) < 1e-12


def test_delay_gradient_factor_central_differences():
    """dtau/d(dp) = -(u_T + u_R) kappa / c, u_R at reception; dp shifts both
    sensors (central differences of the root)."""
    rng = np.random.default_rng(2)
    v = np.array([1.95, 0.3, -0.2])
    for _ in range(10):
        x = np.array([rng.uniform(-20, 20), rng.uniform(5, 60), 0.0])
        t = np.array([0.0, 0.0, -10.0])
        r = t + np.array([0.3, 0.0, 0.0])
        tau, kappa = oracle.delay(x, t, r, v, SIG.c)
        ut = (x - t) / np.linalg.norm(x - t)
        w = x - r - v * tau
        ur = w / np.linalg.norm(w)
        an = -(ut + ur) * kappa / SIG.c
        h = 1e-4
        fd = np.array([(oracle.delay(x, t + h * e, r + h * e, v, SIG.c)[0]
                        - oracle.delay(x, t - h * e, r - h * e, v, SIG.c)[0]) / (2 * h) for e in np.eye(3)])
        assert np.abs(fd - an).max() <= 1e-9 * np.abs(an).max()
        assert abs(kappa - SIG.c / (SIG.c + ur @ v)) < 1e-15


def test_backproject_with_motion_matches_brute_force():
    P, C = 4, 2
    pos, att, txl, rxl, vel = _scene(P, C, seed=3)
    tx, rx = oracle.sensor_positions(pos, att, txl, rxl)
    e = _echo(P, C, 4)
    pix = oracle.grid_points(0.0, 16.0, 0.0, 0.05, 0.04, 0.0, 6, 5, 1)
    a = oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix, vel=vel)
    tau = brute.moving_receiver_tau(tx, rx, vel, SIG.c, pix)
    b = brute.backproject(tx, rx, SIG.fc, SIG.fs, SIG.c, SIG.t0, e, 8, 4.0, pix, tau=tau)
    assert oracle.rel_l2(a, b) < 1e-10
    # and the motion matters at this speed
    assert oracle.rel_l2(oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix), b) > 0.1


def test_point_scatterer_focuses_only_with_the_motion_model():
    """Echoes simulated with a moving receiver (ideal compressed pulse
    sinc(B t)) focus to I = A P C at the scatterer when imaged with the same
    model (32-tap truth interpolator: the only error is the interpolator's);
    stop-and-hop imaging of the same echo loses coherence."""
    P, C = 32, 4
    pos = np.stack([np.arange(P) * 0.1 - 1.6, np.zeros(P), np.full(P, -10.0)], 1)
    att = np.zeros((P, 3))
    rxl = np.stack([(np.arange(C) - 1.5) * 0.025, np.zeros(C), np.zeros(C)], 1)
    vel = np.tile([1.95, 0.0, 0.0], (P, 1))
    tx, rx = oracle.sensor_positions(pos, att, np.zeros(3), rxl)
    A = 0.8 * np.exp(0.7j)
    scat = np.array([[0.0, 20.0, 0.0, A.real, A.imag]])
    sig = oracle.Signal(fc=100e3, fs=40e3, c=1500.0, t0=0.02, n_samples=1024)
    echo = oracle.simulate_points(tx, rx, sig, 20e3, 0.0, scat, vel=vel)
    pix = scat[:, :3]
    I_m = oracle.backproject(tx, rx, sig, echo, 32, 10.0, pix, vel=vel)[0]
    assert abs(abs(I_m) - abs(A) * P * C) <= 1e-4 * abs(A) * P * C
    assert abs(np.angle(I_m / A)) < 1e-4
    I_s = oracle.backproject(tx, rx, sig, echo, 32, 10.0, pix)[0]
    assert abs(I_s) < 0.9 * abs(A) * P * C


def test_adjoint_and_gradient_with_motion():
    P, C = 5, 2
    pos, att, txl, rxl, vel = _scene(P, C, seed=5)
    tx, rx = oracle.sensor_positions(pos, att, txl, rxl)
    e = _echo(P, C, 6)
    pix = oracle.grid_points(0.0, 16.0, 0.0, 0.06, 0.05, 0.0, 8, 6, 1)
    rng = np.random.default_rng(7)
    img = rng.normal(size=pix.shape[0]) + 1j * rng.normal(size=pix.shape[0])
    Be = oracle.backproject(tx, rx, SIG, e, 8, 4.0, pix, vel=vel)
    BhI = oracle.backproject_adjoint(tx, rx, SIG, img, 8, 4.0, pix, vel=vel)
    lhs, rhs = np.vdot(Be, img), np.vdot(e, BhI)
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    off = rng.normal(0, 0.002, size=(P, 3))

    def S(o):
        t, r = oracle.sensor_positions(pos, att, txl, rxl, o)
        return oracle.sharpness(oracle.backproject(t, r, SIG, e, 8, 4.0, pix, vel=vel))[0]

    t, r = oracle.sensor_positions(pos, att, txl, rxl, off)
    _, g = oracle.sharpness(oracle.backproject(t, r, SIG, e, 8, 4.0, pix, vel=vel), want_grad=True)
    grad = oracle.vjp_offsets(t, r, SIG, e, 8, 4.0, pix, g, vel=vel)
    h = 1e-7
    fd = np.zeros((P, 3))
    for i in range(P):
        for a in range(3):
            op, om = off.copy(), off.copy()
            op[i, a] += h
            om[i, a] -= h
            fd[i, a] = (S(op) - S(om)) / (2 * h)
    assert oracle.rel_l2(grad, fd) < 1e-6
