"""Independent NumPy brute force of the backprojection sum, for tiny grids.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).  Written separately from
``oracle.c`` so that each checks the other: the attitude matrix is built as a
product of textbook single-axis rotations instead of the entries printed in
Eq. 2, the Bessel function comes from ``scipy.special.i0`` instead of a series,
and the sum is a broadcast over (pixel, ping, channel, tap).

Paper: arXiv 2101.05888.  Sec. II-A (per-pixel inversion of Eq. 1), Eq. 2.
"""
from __future__ import annotations

import numpy as np
from scipy.special import i0 as scipy_i0


def rot_x(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[1.0, 0.0, 0.0], [0.0, c, -s], [0.0, s, c]])


def rot_y(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def rot_z(a):
    c, s = np.cos(a), np.sin(a)
    return np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])


def attitude_matrix(roll, pitch, yaw):
    """Rz(yaw) Ry(pitch) Rx(roll): body -> NED."""
    return rot_z(yaw) @ rot_y(pitch) @ rot_x(roll)


def sensor_positions(pos, att, tx_lever, rx_lever, offsets=None):
    pos = np.asarray(pos, dtype=np.float64)
    P = pos.shape[0]
    base = pos + (0.0 if offsets is None else np.asarray(offsets, dtype=np.float64))
    Rs = np.stack([attitude_matrix(*att[i]) for i in range(P)])           # [P,3,3]
    tx = base + np.einsum("pab,b->pa", Rs, np.asarray(tx_lever, dtype=np.float64))
    rx = base[:, None, :] + np.einsum("pab,cb->pca", Rs, np.asarray(rx_lever, dtype=np.float64))
    return tx, rx


def kaiser_sinc(d, taps, beta):
    """Un-normalised Kaiser-windowed sinc v(d) (support |d| < taps/2)."""
    h = taps / 2.0
    arg = np.clip(1.0 - (d / h) ** 2, 0.0, None)
    win = scipy_i0(beta * np.sqrt(arg)) / scipy_i0(beta)
    return np.where(np.abs(d) < h, np.sinc(d) * win, 0.0)


def weights(f, taps, beta):
    """Normalised weights for fractions f [...]; returns [..., taps]."""
    k = np.arange(taps) - taps // 2 + 1
    v = kaiser_sinc(np.asarray(f)[..., None] - k, taps, beta)
    return v / v.sum(axis=-1, keepdims=True)


def beam_mask(att, tx, rx, pix, beam_width, side):
    """[n,P,C] boolean: both the transmitter and the receiver see the pixel,
    i.e. the azimuth arctan2(b_x, side b_y) of the body-frame vector lies
    within +-beam_width/2 (and in front of the side axis)."""
    Rs = np.stack([attitude_matrix(*a) for a in att])                         # [P,3,3]
    def sees(sensor):                                                           # sensor [P,(C,)3]
        v = pix[:, None, None, :] - (sensor[None, :, None, :] if sensor.ndim == 2 else sensor[None])
        b = np.einsum("pji,npcj->npci", Rs, v)                                 # R^T v
        az = np.arctan2(b[..., 0], side * b[..., 1])
        return (side * b[..., 1] > 0) & (np.abs(az) <= 0.5 * beam_width)
    return sees(tx) & sees(rx)


def stop_and_hop_tau(tx, rx, c, pix):
    """[n,P,C] two-way delays with one position per ping for TX and RX."""
    pix = np.asarray(pix, dtype=np.float64)
    rt = np.linalg.norm(pix[:, None, :] - tx[None, :, :], axis=-1)                 # [n,P]
    rr = np.linalg.norm(pix[:, None, None, :] - rx[None, :, :, :], axis=-1)        # [n,P,C]
    return (rt[:, :, None] + rr) / c


def terms(tx, rx, fc, fs, c, t0, echo, taps, beta, pix, tau=None):
    """Every term of the sum: [n,P,C] complex.  tau [n,P,C] overrides the
    stop-and-hop delays (e.g. delays found by a root finder)."""
    P, C, Ns = echo.shape
    if tau is None:
        tau = stop_and_hop_tau(tx, rx, c, pix)
    u = (tau - t0) * fs
    j0 = np.floor(u)
    f = u - j0
    k = np.arange(taps) - taps // 2 + 1
    j = j0[..., None].astype(np.int64) + k                                          # [n,P,C,T]
    valid = (j >= 0) & (j < Ns)
    jc = np.clip(j, 0, Ns - 1)
    ii = np.arange(P)[None, :, None, None]
    cc = np.arange(C)[None, None, :, None]
    samples = np.where(valid, echo[ii, cc, jc], 0.0)
    s = (weights(f, taps, beta) * samples).sum(-1)
    return s * np.exp(2j * np.pi * fc * tau)


def backproject(tx, rx, fc, fs, c, t0, echo, taps, beta, pix, mask=None, tau=None):
    """Direct broadcast evaluation; pix [n,3], echo [P,C,Ns]; optional mask
    [n,P,C] of the terms that count and delays tau [n,P,C]; returns [n]."""
    t = terms(tx, rx, fc, fs, c, t0, echo, taps, beta, pix, tau=tau)
    if mask is not None:
        t = np.where(mask, t, 0.0)
    return t.sum(axis=(1, 2))


def moving_receiver_tau(tx, rx, vel, c, pix):
    """[n,P,C] delays with the receiver moving at vel [P,3] during reception:
    the root of c tau - |x - t| - |x - r - v tau| on a bracket, by Brent's
    method (scipy), term by term (tiny grids only)."""
    from scipy.optimize import brentq
    pix = np.asarray(pix, dtype=np.float64)
    n, P, C = pix.shape[0], tx.shape[0], rx.shape[1]
    out = np.zeros((n, P, C))
    for a in range(n):
        for i in range(P):
            rt = np.linalg.norm(pix[a] - tx[i])
            for ch in range(C):
                f = lambda t: c * t - rt - np.linalg.norm(pix[a] - rx[i, ch] - vel[i] * t)
                t0 = (rt + np.linalg.norm(pix[a] - rx[i, ch])) / c
                out[a, i, ch] = brentq(f, 0.5 * t0, 2.0 * t0, xtol=1e-18, rtol=8.9e-16, maxiter=200)
    return out
