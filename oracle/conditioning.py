"""FP64 NumPy oracle for the data conditioning of Sec. II-E and for matched
filtering: spectral whitening (Eq. 9), time-varying gain (Eq. 10), dynamic
range compression (Eqs. 11-12), and range compression of raw linear-FM
echoes by correlation with the transmitted replica.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``): plain definitions with
NumPy's FFT, median and correlation as the library steps; no blocking or
reordering.  Readings where the paper is silent (all recorded in the
repository's design notes):

* Eq. 9 and Eq. 10 give gains in units of inverse power; they are applied
  as power gains, i.e. the complex samples are multiplied by sqrt(G).
* h in Eq. 9 scales G so that its largest value is 1 (the smallest
  attenuation is 0 dB).
* P-hat(f) in Eq. 9 is the mean of |FFT(e)|^2 over all rows of the batch;
  the mean in both equations is over frequency / time.
* Medians are taken of FP32 powers (re*re + im*im with two roundings to
  FP32, no fused multiply-add) and FP32 magnitudes (correctly rounded
  square root), since the selection of an element is decided by the FP32
  values; for an even count the median is the FP64 mean of the two middle
  values.
* Eq. 11: I is the magnitude |I| normalised by its maximum (FP32 division);
  Eq. 12 uses the median of that normalised image.  Where Eq. 12 has no
  value (median 1: every pixel at the maximum; median 0) the limits are
  taken: the identity map, and 1 for every non-zero pixel.  Eq. 10 with a
  zero denominator (alpha = 0 and a silent median) applies no correction.
* The replica of a pulse of length T and bandwidth B is the complex
  baseband up-chirp p(t) = exp(j pi (B/T) (t - T/2)^2) sampled at t = l/fs,
  l = 0 .. round(T fs) - 1; the matched filter output is
  y[k] = sum_l e[k + l] conj(p[l]) / sum_l |p[l]|^2 (samples past the row
  read zero), which peaks at the sample of the echo's delay.
"""
from __future__ import annotations

import numpy as np

import oracle


def power_f32(e) -> np.ndarray:
    """|e|^2 rounded as FP32 arithmetic does it: re*re, im*im, sum."""
    e = np.asarray(e, dtype=np.complex64)
    re, im = e.real.astype(np.float32), e.imag.astype(np.float32)
    return (re * re + im * im).astype(np.float32)


def magnitude_f32(e) -> np.ndarray:
    return np.sqrt(power_f32(e)).astype(np.float32)


def median_of(values, axis=None) -> np.ndarray:
    """Median with the even-count rule above (FP64 mean of the middle two)."""
    v = np.sort(np.asarray(values), axis=axis)
    if axis is None:
        v = v.reshape(-1)
        n = v.size
        lo, hi = v[(n - 1) // 2], v[n // 2]
        return 0.5 * (np.float64(lo) + np.float64(hi))
    n = v.shape[axis]
    lo = np.take(v, (n - 1) // 2, axis=axis).astype(np.float64)
    hi = np.take(v, n // 2, axis=axis).astype(np.float64)
    return 0.5 * (lo + hi)


def whiten(e, gamma: float):
    """Eq. 9 on a batch e [rows, N] (complex): returns (whitened e, G_h)."""
    S = np.fft.fft(np.asarray(e, dtype=np.complex128), axis=-1)
    P = np.mean(np.abs(S) ** 2, axis=0)
    G = 1.0 / (gamma * np.mean(P) + P)
    Gh = G / np.max(G)
    return np.fft.ifft(S * np.sqrt(Gh), axis=-1), Gh


def tvg(e, alpha: float):
    """Eq. 10 on a batch e [rows, N]: returns (e sqrt(G), G, P_med)."""
    e = np.asarray(e)
    Pmed = median_of(power_f32(e), axis=0)
    den = alpha * np.mean(Pmed) + Pmed
    # a silent median with alpha = 0 leaves Eq. 10 without a value: no correction
    G = np.where(den > 0, 1.0 / np.where(den > 0, den, 1.0), 1.0)
    return e.astype(np.complex128) * np.sqrt(G), G, Pmed


def drc(img, b: float):
    """Eqs. 11-12 on a complex image: returns (I_DRC, q, median of I_n)."""
    m = magnitude_f32(img).reshape(-1)
    In = (m / np.max(m)).astype(np.float32)
    med = median_of(In)
    In64 = In.astype(np.float64)
    if med >= 1.0:            # every pixel at the maximum: Eq. 12 is 0/0, the identity map
        q = 1.0
        out = In64
    elif med <= 0.0:          # the median pixel is dark: q -> infinity, every lit pixel to 1
        q = np.inf
        out = (In64 > 0).astype(np.float64)
    else:
        q = (b - b * med) / (med - b * med)
        out = q * In64 / ((q - 1.0) * In64 + 1.0)
    return out.reshape(np.shape(img)), q, med


def lfm_replica(B: float, T: float, fs: float) -> np.ndarray:
    L = int(round(T * fs))
    t = np.arange(L) / fs
    return np.exp(1j * np.pi * (B / T) * (t - 0.5 * T) ** 2)


def matched_filter(raw, replica) -> np.ndarray:
    """Correlation of every row of raw [rows, N] with the replica."""
    raw = np.atleast_2d(np.asarray(raw, dtype=np.complex128))
    p = np.asarray(replica, dtype=np.complex128)
    L = p.size
    N = raw.shape[-1]
    out = np.zeros_like(raw)
    pad = np.concatenate([raw, np.zeros((raw.shape[0], L), dtype=np.complex128)], axis=1)
    for r in range(raw.shape[0]):
        # y[k] = sum_l pad[k + l] conj(p[l]);  np.correlate(a, v)[k] = sum_l a[k + l] conj(v[l])
        out[r] = np.correlate(pad[r], p, mode="valid")[:N]
    return out / np.sum(np.abs(p) ** 2)


def simulate_raw_points(tx, rx, sig, B: float, T: float, scat) -> np.ndarray:
    """Raw (uncompressed) baseband echoes of point scatterers, stop-and-hop:
    e[i][c][n] = sum_s A_s p(t_n - tau) exp(-j 2 pi fc tau), t_n = t0 + n/fs,
    p(t) = exp(j pi (B/T) (t - T/2)^2) on 0 <= t < T."""
    tx, rx = np.asarray(tx, float), np.asarray(rx, float)
    P, C = tx.shape[0], rx.shape[1]
    out = np.zeros((P, C, sig.n_samples), dtype=np.complex128)
    tn = sig.t0 + np.arange(sig.n_samples) / sig.fs
    for s in np.asarray(scat, float).reshape(-1, 5):
        A = s[3] + 1j * s[4]
        for i in range(P):
            for c in range(C):
                tau, _ = oracle.delay(s[:3], tx[i], rx[i, c], None, sig.c)
                dt = tn - tau
                inside = (dt >= 0) & (dt < T)
                out[i, c] += np.where(inside, A * np.exp(1j * np.pi * (B / T) * (dt - 0.5 * T) ** 2), 0.0) \
                    * np.exp(-2j * np.pi * sig.fc * tau)
    return out
