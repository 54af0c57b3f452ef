"""Shared helpers for the GPU parity tests: build the same seeded scene for
the library and for the oracle (inputs only; no arithmetic of the method)."""
import numpy as np

import oracle
import paper_2101_05888_gb300 as sas
from paper_2101_05888_gb300 import synth


def oracle_signal(w):
    return oracle.Signal(synth.FC, synth.FS, synth.C_SOUND, w.t0, w.n_samples)


def lib_signal(w):
    return sas.make_signal(synth.FC, synth.FS, synth.C_SOUND, w.t0, w.n_samples)


def oracle_positions(nav, true=False, offsets=None):
    pos = nav["true_pos"] if true else nav["pos"]
    return oracle.sensor_positions(pos, nav["att"], nav["tx_lever"], nav["rx_lever"], offsets)


def point_echo(w, nav, scat, snr_db=20.0, noise=True, half_width=0):
    """Matched-filtered LFM echo of the scatterers from the true track plus
    band-limited noise at the stated SNR; complex128 [P,C,Ns]."""
    tx, rx = oracle_positions(nav, true=True)
    echo = oracle.simulate_points(tx, rx, oracle_signal(w), synth.BANDWIDTH, synth.PULSE_T, scat,
                                  half_width=half_width)
    if noise:
        echo += synth.bandlimited_noise(echo.shape, synth.NU_BAND, synth.snr_noise_power(scat, snr_db),
                                        w.seed + 77)
    return echo


def grid_pixels(g):
    return oracle.grid_points(g.x0, g.y0, g.z0, g.dx, g.dy, g.dz, g.nx, g.ny, g.nz)


def index_pixels(g, idx):
    return oracle.grid_index_points(g.x0, g.y0, g.z0, g.dx, g.dy, g.dz, idx)


def image_at(img, idx):
    """Values of a [nz][ny][nx] image (numpy) at indices idx [n,3] = (ix, iy, iz)."""
    idx = np.asarray(idx)
    return img[idx[:, 2], idx[:, 1], idx[:, 0]]


def in_band(echo, nu_b=0.25):
    """The part of echo rows (last axis) inside |nu| <= nu_b cycles/sample:
    FFT, zero the rest, inverse FFT (complex128)."""
    E = np.fft.fft(np.asarray(echo, dtype=np.complex128), axis=-1)
    nu = np.fft.fftfreq(E.shape[-1])
    E[..., np.abs(nu) > nu_b] = 0.0
    return np.fft.ifft(E, axis=-1)

