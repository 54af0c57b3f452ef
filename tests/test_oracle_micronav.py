"""Pins for the DPC micronavigation oracle (Sec. II-D, Eqs. 3-8).

The residual of Eq. 4 is pinned to the echo simulator (which is pinned to
the exact moving-receiver delay elsewhere): the arrival time of a seafloor
point's echo in two consecutive pings differs by the delay that makes g
vanish.  The time-delay estimator is pinned on pure shifts of a real
band-limited signal (whose correlation phase is exactly -2 pi fc delay);
the solver on exact delays (recovers the truth), outliers (Huber) and the
limits of the regularisers."""
import numpy as np
import pytest

import oracle
from oracle import micronav as mn

import _dpc

C_SOUND, FC, FS = 1500.0, 100e3, 40e3


def _sensors(pl, vy, vz):
    """Transmitters, receivers at the ping times, and velocities for the simulator."""
    p = mn.positions(pl, vy, vz)
    tx, rx = oracle.sensor_positions(p, pl.att, pl.tx_lever, pl.rx_lever)
    vel = np.stack([pl.vx, vy, vz], 1)
    return tx, rx, vel


def test_kinematics():
    pl = _dpc.platform(P=5)
    vy, vz = _dpc.true_velocities(5)
    p = mn.positions(pl, vy, vz)
    assert np.allclose(p[0], pl.p0)
    for i in range(4):
        assert np.allclose(p[i + 1] - p[i], np.array([pl.vx[i], vy[i], vz[i]]) * pl.dt[i], atol=1e-15)
    tx, rx = mn.sensors_at(pl, vy, vz, 3, 0.02)
    txs, rxs = oracle.sensor_positions(p, pl.att, pl.tx_lever, pl.rx_lever)
    assert np.allclose(tx, txs[3], atol=1e-14)
    assert np.allclose(rx, rxs[3] + 0.02 * np.array([pl.vx[3], vy[3], vz[3]]), atol=1e-14)


def test_footprint_geometry():
    pl = _dpc.platform(P=4)
    vy, vz = _dpc.true_velocities(4)
    meas = _dpc.measurements(pl, 5, 0.03, 0.05, 2)
    ps = mn.footprints(pl, vy, vz, meas, C_SOUND)
    p = mn.positions(pl, vy, vz)
    for m in range(meas.ping.size):
        i, ch = meas.ping[m], meas.chan[m]
        R = oracle.attitude_matrix(*pl.att[i])
        pc = p[i] + 0.5 * (R @ pl.tx_lever + R @ pl.rx_lever[ch + 2])
        assert ps[m, 2] == 0.0
        assert abs(np.linalg.norm(ps[m] - pc) - 0.5 * C_SOUND * meas.t[m]) < 1e-9
        heading = np.array([np.cos(pl.att[i, 2]), np.sin(pl.att[i, 2]), 0.0])
        assert abs(np.dot(ps[m] - pc, heading)) < 1e-9          # abeam
        assert np.cross(heading, ps[m] - pc)[2] > 0              # starboard (NED: +z down)


def test_residual_matches_simulated_arrival_times():
    """One seafloor point: the peak of the matched-filtered echo of receiver
    c + s in ping i and of receiver c in ping i + 1 arrive the model delay
    apart (to the model's own approximation: both receivers at one time)."""
    P, C, s = 3, 6, 2
    pl = _dpc.platform(P=P, C=C, shift=s)
    vy, vz = _dpc.true_velocities(P, amp_y=0.2, amp_z=0.15)
    t_k = 0.035
    meas = _dpc.measurements(pl, 1, t_k, t_k, s)
    ps = mn.footprints(pl, vy, vz, meas, C_SOUND)
    delays = mn.model_delays(pl, vy, vz, meas, ps, C_SOUND)
    tx, rx, vel = _sensors(pl, vy, vz)
    sig = oracle.Signal(FC, FS * 16, C_SOUND, t_k - 0.0015, 2048)   # 640 kHz sampling: sharp peaks
    for m in range(meas.ping.size):
        i, ch = int(meas.ping[m]), int(meas.chan[m])
        scat = np.array([[*ps[m], 1.0, 0.0]])
        e = oracle.simulate_points(tx, rx, sig, 20e3, 0.0, scat, vel=vel)
        arr = []
        for (pi, ci) in ((i, ch + s), (i + 1, ch)):
            row = np.abs(e[pi, ci])
            k = int(np.argmax(row))
            assert 0 < k < row.size - 1
            ym, y0, yp = row[k - 1], row[k], row[k + 1]
            arr.append(sig.t0 + (k + 0.5 * (ym - yp) / (ym - 2 * y0 + yp)) / sig.fs)
        # sinc-pulse peak by parabola: accurate to a small fraction of the 1.6 us sample
        assert abs((arr[1] - arr[0]) - delays[m]) < 3e-8
    assert np.abs(delays).min() > 1e-6                       # sway and heave matter here (80x the tolerance)


def test_delay_estimator_on_pure_shifts():
    from paper_2101_05888_gb300 import synth
    rng = np.random.default_rng(1)
    base = synth.bandlimited_noise((1, 4096), 0.25, 1.0, 7)[0].real     # real: Hermitian spectrum
    N = base.size
    f = np.fft.fftfreq(N)
    for delay_samples in (0.0, 0.37, -2.81, 5.5, -0.05):
        delay = delay_samples / FS
        e1 = base.astype(np.complex128)
        e2 = np.fft.ifft(np.fft.fft(base) * np.exp(-2j * np.pi * f * delay_samples)) * np.exp(-2j * np.pi * FC * delay)
        coarse, fine, rho = mn.estimate_delay(e1, e2, 2000, 256, 8, FS, FC)
        assert abs(coarse - delay) < 0.08 / FS                # parabola on |R|: a small fraction of a sample
        assert abs(mn.unwrap(fine, delay, FC) - delay) < 1e-10
        assert abs(mn.unwrap(fine, coarse, FC) - delay) < 1e-10   # the coarse delay suffices to unwrap
        assert rho > 0.85                                     # integer peak lag of a fractional shift
    # the window limits the lags: a shift beyond them is not found
    e2 = np.roll(base, 12).astype(np.complex128)
    coarse, _, _ = mn.estimate_delay(base, e2, 2000, 256, 8, FS, FC)
    assert abs(coarse * FS) <= 8


def test_unwrap():
    fine = np.array([1e-6, -4e-6, 4.9e-6])
    ref = np.array([3.1e-5, -2.2e-5, 0.0])
    u = mn.unwrap(fine, ref, FC)
    assert np.all(np.abs(u - ref) <= 0.5 / FC + 1e-18)
    k = (u - fine) * FC
    assert np.allclose(k, np.round(k), atol=1e-9)


def _problem(P=14, C=8, s=2, K=5, seed=4):
    pl = _dpc.platform(P=P, C=C, shift=s)
    vy, vz = _dpc.true_velocities(P, seed=seed)
    meas = _dpc.measurements(pl, K, 0.03, 0.06, s)
    prior_vy, prior_vz = np.zeros(P), np.zeros(P)
    ps = mn.footprints(pl, prior_vy, prior_vz, meas, C_SOUND)
    meas.delay = mn.model_delays(pl, vy, vz, meas, ps, C_SOUND)
    z_dvl = mn.heave_positions(pl, vz)
    return pl, vy, vz, meas, ps, z_dvl


def test_solver_recovers_truth_from_exact_delays():
    pl, vy, vz, meas, ps, z_dvl = _problem()
    P = pl.P
    assert np.all(np.abs(mn.dpc_residuals(pl, vy, vz, meas, ps, C_SOUND)) < 1e-12)
    sy, sz, loss = mn.solve(pl, np.zeros(P), np.zeros(P), meas, ps, C_SOUND, z_dvl, 1e-10, 1e-10)
    # of ~3e-2 m/s; the tiny regularisers (the truth is not smooth) leave ~1e-7
    assert np.abs(sy - vy).max() < 3e-7 and np.abs(sz - vz).max() < 3e-7
    assert loss < 1e-12                     # the smoothness term of the non-smooth truth


def test_huber_resists_outliers():
    pl, vy, vz, meas, ps, z_dvl = _problem(seed=8)
    P = pl.P
    rng = np.random.default_rng(2)
    bad = rng.choice(meas.delay.size, meas.delay.size // 25, replace=False)
    meas.delay = meas.delay + rng.normal(0, 2e-8, meas.delay.size)
    meas.delay[bad] += rng.choice([-1, 1], bad.size) * 5e-6          # 7.5 mm of path: outliers
    ly, lz, _ = mn.solve(pl, np.zeros(P), np.zeros(P), meas, ps, C_SOUND, z_dvl, 1e-6, 1e-4)
    hy, hz, _ = mn.solve(pl, np.zeros(P), np.zeros(P), meas, ps, C_SOUND, z_dvl, 1e-6, 1e-4, huber=1e-4)
    err_ls = np.hypot(ly - vy, lz - vz).max()
    err_h = np.hypot(hy - vy, hz - vz).max()
    assert err_h < 0.2 * err_ls
    # the Huber solution is a stationary point of its loss (scipy's robust trust region)
    f0 = mn.total_loss(pl, hy, hz, meas, ps, C_SOUND, z_dvl, 1e-6, 1e-4, huber=1e-4)
    for k in (0, 5, P + 3):
        x = np.concatenate([hy, hz])
        for h in (1e-7, -1e-7):
            x2 = x.copy()
            x2[k] += h
            assert mn.total_loss(pl, x2[:P], x2[P:], meas, ps, C_SOUND, z_dvl, 1e-6, 1e-4, huber=1e-4) >= f0 - 1e-13


def test_regulariser_limits():
    pl, vy, vz, meas, ps, z_dvl = _problem(P=10, K=3)
    P = pl.P
    # no DPC information, strong DVL: the heave positions follow the DVL
    meas.weight[:] = 0.0
    z_target = z_dvl + np.linspace(0, 0.05, P)
    sy, sz, _ = mn.solve(pl, np.zeros(P), np.zeros(P), meas, ps, C_SOUND, z_target, 1e-12, 1.0)
    assert np.abs(mn.heave_positions(pl, sz) - z_target).max() < 1e-9
    # very strong smoothing: velocities along a straight line in the ping index
    meas.weight[:] = 1.0
    sy, sz, _ = mn.solve(pl, np.zeros(P), np.zeros(P), meas, ps, C_SOUND, z_dvl, 1e8, 1e-6)
    assert np.abs(mn.smooth_residuals(sy)).max() < 1e-7 and np.abs(mn.smooth_residuals(sz)).max() < 1e-7
