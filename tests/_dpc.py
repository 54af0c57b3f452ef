"""Seeded DPC micronavigation scenes for the tests: a stripmap platform with
sinusoidal sway and heave velocities, a receive array whose phase centres
overlap from ping to ping, and a seafloor field of point scatterers (inputs
only; the kinematics and the residuals come from ``oracle.micronav``)."""
import numpy as np

from oracle import micronav as mn


def platform(P=12, C=8, pitch=0.05, shift=2, speed=1.0, altitude=10.0, yaw=0.02, seed=3):
    """Array advances shift half-pitches per ping: speed * dt = shift * pitch / 2."""
    rng = np.random.default_rng(seed)
    dt = np.full(P - 1, shift * 0.5 * pitch / speed)
    att = np.zeros((P, 3))
    att[:, 0] = rng.normal(0.0, 0.002, P)            # roll
    att[:, 1] = rng.normal(0.0, 0.002, P)            # pitch
    att[:, 2] = yaw + np.cumsum(rng.normal(0.0, 1e-4, P))
    rx = np.stack([(np.arange(C) - 0.5 * (C - 1)) * pitch, np.zeros(C), np.zeros(C)], 1)
    pl = mn.Platform(p0=np.array([0.0, 0.0, -altitude]), vx=np.full(P, speed), att=att, dt=dt,
                     tx_lever=np.array([0.0, 0.0, 0.0]), rx_lever=rx, side=1)
    return pl


def true_velocities(P, seed=4, amp_y=0.03, amp_z=0.02):
    """Sway / heave velocities [m/s]: a slow sinusoid plus a little jitter."""
    rng = np.random.default_rng(seed)
    i = np.arange(P)
    ph = rng.uniform(0, 2 * np.pi, 2)
    vy = amp_y * np.sin(2 * np.pi * i / 9.0 + ph[0]) + rng.normal(0, 0.002, P)
    vz = amp_z * np.sin(2 * np.pi * i / 13.0 + ph[1]) + rng.normal(0, 0.002, P)
    return vy, vz


def measurements(pl, K, t_lo, t_hi, shift, delays=None, weight=None):
    """Dense (pair, receiver, window) layout: window centre times evenly in [t_lo, t_hi]."""
    P, C = pl.P, pl.rx_lever.shape[0]
    nc = C - shift
    t = np.linspace(t_lo, t_hi, K)
    ping = np.repeat(np.arange(P - 1), nc * K)
    chan = np.tile(np.repeat(np.arange(nc), K), P - 1)
    tt = np.tile(t, (P - 1) * nc)
    M = ping.size
    return mn.Measurements(ping=ping, chan=chan, t=tt,
                           delay=np.zeros(M) if delays is None else np.asarray(delays, float),
                           weight=np.ones(M) if weight is None else np.asarray(weight, float), shift=shift)


def seafloor_points(n, x_lo, x_hi, y_lo, y_hi, seed=5):
    """Point scatterers (x, y, 0, Re A, Im A) uniform on the patch, complex Gaussian A."""
    rng = np.random.default_rng(seed)
    A = (rng.normal(size=n) + 1j * rng.normal(size=n)) / np.sqrt(2)
    return np.stack([rng.uniform(x_lo, x_hi, n), rng.uniform(y_lo, y_hi, n), np.zeros(n), A.real, A.imag], 1)
