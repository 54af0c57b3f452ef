"""Pins for the conditioning oracle (Sec. II-E, Eqs. 9-12) and the matched
filter, against closed forms that follow from the equations themselves."""
import numpy as np
import pytest

import oracle
from oracle import conditioning as cond

FS = 40e3


def _colored_rows(rows, n, seed):
    """Complex Gaussian rows through a fixed 5-tap FIR: a non-flat spectrum."""
    rng = np.random.default_rng(seed)
    w = rng.normal(size=(rows, n + 4)) + 1j * rng.normal(size=(rows, n + 4))
    h = np.array([1.0, 0.7 - 0.2j, 0.3, -0.1j, 0.05])
    return np.stack([np.convolve(r, h, mode="valid") for r in w])


def test_matched_filter_on_grid_point_is_the_discrete_autocorrelation():
    """An echo of A p(t - tau) with tau on a sample: y[k0 + n] = A (1/L)
    sum_{l < L - |n|} p[l + |n|] conj(p[l]) (conj for n < 0), a geometric
    series with ratio exp(j 2 pi (B/T) |n| / fs^2) times exp(j pi (B/T) (n/fs)^2
    - j pi (B/T) |n| T / fs)."""
    B, T = 20e3, 5e-3
    p = cond.lfm_replica(B, T, FS)
    L = p.size
    N, k0 = 1024, 300
    A = 0.6 - 0.3j
    raw = np.zeros(N, dtype=np.complex128)
    raw[k0:k0 + L] = A * p
    y = cond.matched_filter(raw[None], p)[0]
    kk = B / T
    for n in range(-L + 1, L):
        m = abs(n)
        r = np.exp(2j * np.pi * kk * m / FS ** 2)
        geo = L - m if abs(r - 1) < 1e-15 else (r ** (L - m) - 1) / (r - 1)
        val = A * np.exp(1j * np.pi * kk * ((m / FS) ** 2 - m * T / FS)) * geo / L
        if n < 0:
            val = A * np.conj(val / A)
        assert abs(y[k0 + n] - val) < 1e-12
    assert abs(y[k0] - A) < 1e-12
    assert np.abs(y[:k0 - L]).max() == 0 and np.abs(y[k0 + L:]).max() == 0


def test_matched_filter_of_raw_echo_compresses_the_pulse():
    """Raw LFM echoes of points (on-sample delays) compress to |A| peaks at the
    delay samples, with the carrier phase exp(-j 2 pi fc tau)."""
    sig = oracle.Signal(100e3, FS, 1500.0, 0.02, 1024)
    B, T = 20e3, 5e-3
    tx = np.array([[0.0, 0.0, -10.0]])
    rx = np.array([[[0.0, 0.0, -10.0]]])
    # a point whose two-way delay falls on sample 400
    tau = sig.t0 + 400 / sig.fs
    r = 0.5 * tau * sig.c
    y0 = np.sqrt(r ** 2 - 100.0)
    scat = np.array([[0.0, y0, 0.0, 0.8, 0.2]])
    assert abs(oracle.delay(scat[0, :3], tx[0], rx[0, 0], None, sig.c)[0] - tau) < 1e-15
    raw = cond.simulate_raw_points(tx, rx, sig, B, T, scat)
    y = cond.matched_filter(raw.reshape(1, -1), cond.lfm_replica(B, T, sig.fs))[0]
    assert int(np.argmax(np.abs(y))) == 400
    A = 0.8 + 0.2j
    assert abs(y[400] - A * np.exp(-2j * np.pi * sig.fc * tau)) < 1e-9


def test_whitening_flattens_and_normalises():
    """gamma = 0: G_h = min P / P, so the batch's mean power spectrum after
    whitening is exactly min P at every frequency (flat); max G_h = 1 (0 dB);
    a large gamma leaves the rows nearly unchanged."""
    e = _colored_rows(40, 256, 1)
    out, Gh = cond.whiten(e, 0.0)
    P_in = np.mean(np.abs(np.fft.fft(e, axis=-1)) ** 2, axis=0)
    P_out = np.mean(np.abs(np.fft.fft(out, axis=-1)) ** 2, axis=0)
    assert np.max(Gh) == 1.0
    assert np.abs(P_out / P_in.min() - 1.0).max() < 1e-12
    assert np.std(P_in) / np.mean(P_in) > 0.3          # the input was far from flat
    out_big, Gh_big = cond.whiten(e, 1e9)
    assert oracle.rel_l2(out_big, e) < 1e-6 and np.min(Gh_big) > 1 - 1e-6


def test_tvg_equalises_median_power():
    """alpha = 0: every sample time's median output power is exactly 1; the
    median rule matches numpy's median; the gain follows the envelope."""
    rng = np.random.default_rng(2)
    rows, n = 41, 300
    env = np.exp(-np.linspace(0, 4, n))                 # spreading/absorption-like decay
    e = ((rng.normal(size=(rows, n)) + 1j * rng.normal(size=(rows, n))) * env).astype(np.complex64)
    out, G, Pmed = cond.tvg(e, 0.0)
    assert np.array_equal(Pmed, np.median(cond.power_f32(e).astype(np.float64), axis=0))   # odd count
    med_out = np.median(np.abs(out) ** 2, axis=0)
    assert np.abs(med_out - 1.0).max() < 1e-6
    out_a, G_a, _ = cond.tvg(e, 0.5)
    assert np.all(G_a < G)
    assert np.corrcoef(np.log(G), np.log(env))[0, 1] < -0.99     # the gain undoes the decay
    # even count: FP64 mean of the two middle FP32 values
    v = np.array([3.0, 1.0, 4.0, 2.0], dtype=np.float32)
    assert cond.median_of(v) == 2.5


def test_drc_median_maps_to_brightness():
    """Eq. 12 makes Eq. 11 send the median normalised pixel to b; the map is
    monotone, sends 0 to 0 and the brightest pixel to 1."""
    rng = np.random.default_rng(3)
    img = (rng.standard_exponential((63, 63)) ** 3 * np.exp(1j * rng.uniform(0, 6.28, (63, 63)))).astype(np.complex64)
    for b in (0.2, 0.35, 0.6):
        out, q, med = cond.drc(img, b)
        assert abs(q * med / ((q - 1) * med + 1) - b) < 1e-12
        m = cond.magnitude_f32(img).reshape(-1)
        order = np.argsort(m, kind="stable")
        o = out.reshape(-1)[order]
        assert np.all(np.diff(o) >= 0)
        assert abs(o[-1] - 1.0) < 1e-12 and o[0] >= 0.0
        assert m.size % 2 == 1 and abs(o[(m.size - 1) // 2] - b) < 1e-12     # the median pixel


def test_drc_degenerate_medians_take_the_limits():
    """Median 1 (one pixel, or all pixels equal): the identity; median 0
    (most pixels dark): every lit pixel maps to 1, as q -> infinity in
    Eq. 11."""
    out, q, med = cond.drc(np.array([[0.3 - 0.4j]], dtype=np.complex64), 0.4)
    assert med == 1.0 and q == 1.0 and out[0, 0] == 1.0
    img = np.array([0, 0, 0, 0.5, 2.0], dtype=np.complex64)
    out, q, med = cond.drc(img, 0.4)
    assert med == 0.0 and np.isinf(q) and list(out) == [0, 0, 0, 1, 1]
    # the limit agrees with Eq. 11 at a large finite q
    In = np.array([0.25, 1.0])
    qq = 1e12
    assert np.allclose(qq * In / ((qq - 1) * In + 1), 1.0)


def test_tvg_silent_median_leaves_samples():
    e = np.zeros((3, 4), dtype=np.complex64)
    e[0, 1] = 1.0 + 1.0j
    e[:, 2:] = 1.0
    out, G, Pmed = cond.tvg(e, 0.0)
    assert Pmed[0] == 0 and Pmed[1] == 0 and G[0] == 1.0 and G[1] == 1.0
    assert np.array_equal(out[:, :2], e[:, :2].astype(np.complex128))
    assert np.allclose(np.abs(out[:, 2:]) ** 2, 1.0)


def _colored(rows, n, seed):
    rng = np.random.default_rng(seed)
    w = rng.normal(size=(rows, n + 4)) + 1j * rng.normal(size=(rows, n + 4))
    h = np.array([1.0, 0.7 - 0.2j, 0.3, -0.1j, 0.05])
    return np.stack([np.convolve(r, h, mode="valid") for r in w]).astype(np.complex64)


@pytest.mark.parametrize("rows,n,gamma", [(40, 256, 0.0), (64, 1024, 0.1), (9, 16384, 0.05), (7, 2048, 0.1),
                                          (3, 4096, 0.0), (5, 8192, 0.2), (17, 512, 0.3)])
def test_whitening_gain_tolerance_holds_for_an_independent_fp32_fft(rows, n, gamma):
    """The GPU whitening tests bound the gain error by
    max(1e-6, 2^-23 sqrt(log2 n kappa)), kappa = mean P / (gamma mean P + min P):
    the rounding of FP32 spectra amplified by the conditioning of Eq. 9.  An
    independent single-precision FFT (scipy.fft on complex64) meets that
    bound on the same inputs, so the bound asks no more than FP32 arithmetic
    can give."""
    sfft = pytest.importorskip("scipy.fft")
    e = _colored(rows, n, n + rows)
    _, Gh = cond.whiten(e, gamma)
    S = sfft.fft(e, axis=-1)
    assert S.dtype == np.complex64
    P = np.mean(np.abs(S.astype(np.complex128)) ** 2, axis=0)
    G = 1.0 / (gamma * P.mean() + P)
    gain = np.sqrt(G / G.max()).astype(np.float32)
    kappa = np.mean(1.0 / Gh) / (1.0 + gamma)
    tol = max(1e-6, 2.0 ** -23 * np.sqrt(np.log2(n) * kappa))
    assert np.abs(gain - np.sqrt(Gh)).max() < tol
