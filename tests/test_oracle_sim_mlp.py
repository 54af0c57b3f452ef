"""Pins for the test-input simulator and the FP64 learned-interpolator maths."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp
from paper_2101_05888_gb300 import synth


def test_lfm_compressed_pulse_against_numerical_correlation():
    """Matched-filter output of a sampled LFM (rectangular envelope) against the
    closed form (1-|t|/T) sinc(B t (1-|t|/T)), normalised to a unit peak."""
    B, T = 20e3, 1e-3
    F = 32 * B
    n = int(round(T * F))
    t = (np.arange(n) - 0.5 * (n - 1)) / F
    s = np.exp(1j * np.pi * (B / T) * t ** 2)
    corr = np.correlate(s, s, mode="full") / n          # sum_n s[n+l] conj(s[n])
    lags = (np.arange(corr.size) - (n - 1)) / F
    sel = np.abs(lags) < 4.0 / B
    ref = np.array([oracle.lfm_compressed_pulse(x, B, T) for x in lags[sel]])
    assert np.max(np.abs(corr[sel] - ref)) < 3e-3
    assert abs(oracle.lfm_compressed_pulse(0.0, B, T) - 1.0) == 0.0
    assert oracle.lfm_compressed_pulse(1.5 * T, B, T) == 0.0


def test_simulated_point_has_unit_peak_on_grid():
    """A point whose two-way delay falls exactly on sample n gives
    e[n] = A exp(-j 2 pi fc tau) there and zeros at the other samples for the
    ideal pulse at 2x oversampling (sinc(B t) vanishes at t = 2m/fs)."""
    sig = oracle.Signal(100e3, 40e3, 1500.0, 0.0, 256)
    n0 = 100
    tau = n0 / sig.fs
    r = tau * sig.c / 2
    tx = np.array([[0.0, 0.0, 0.0]])
    rx = np.array([[[0.0, 0.0, 0.0]]])
    A = 0.6 - 0.3j
    e = oracle.simulate_points(tx, rx, sig, 20e3, 0.0, [[0.0, r, 0.0, A.real, A.imag]])[0, 0]
    assert abs(e[n0] - A * np.exp(-2j * np.pi * sig.fc * tau)) < 1e-12
    assert np.max(np.abs(e[n0 + 2::2])) < 1e-12


def test_mlp_gradient_central_difference():
    rng = np.random.default_rng(1)
    theta = rng.normal(0, 0.3, mlp.N_PARAMS)
    f = rng.random(17)
    s = rng.normal(size=(17, 8)) + 1j * rng.normal(size=(17, 8))
    y = rng.normal(size=17) + 1j * rng.normal(size=17)
    L, g = mlp.loss_and_grad(theta, f, s, y)
    h = 1e-6
    idx = rng.choice(mlp.N_PARAMS, 60, replace=False)
    for i in idx:
        tp, tm = theta.copy(), theta.copy()
        tp[i] += h
        tm[i] -= h
        fd = (mlp.loss_and_grad(tp, f, s, y)[0] - mlp.loss_and_grad(tm, f, s, y)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(abs(fd), 1e-3)


def test_gelu_closed_form_values():
    assert mlp.gelu(np.array(0.0)) == 0.0
    assert abs(mlp.gelu(np.array(1.0)) - 0.5 * (1 + math.erf(1 / math.sqrt(2)))) < 1e-16
    assert abs(mlp.gelu(np.array(-10.0))) < 1e-20
    z = np.linspace(-3, 3, 11)
    h = 1e-6
    assert np.allclose(mlp.gelu_grad(z), (mlp.gelu(z + h) - mlp.gelu(z - h)) / (2 * h), atol=1e-9)


def test_adam_first_step_is_signed_lr():
    """With bias correction the first Adam step moves each parameter by lr in
    the direction opposite its gradient (|g| >> eps)."""
    th = np.zeros(5)
    g = np.array([1.0, -2.0, 3.0, -0.5, 0.25])
    th1, m, v = mlp.adam_step(th, g, np.zeros(5), np.zeros(5), 1, 0.01)
    assert np.allclose(th1, -0.01 * np.sign(g), atol=1e-9)


def test_ls_optimal_fir_properties():
    nu_b = synth.NU_BAND
    h0, e0 = mlp.ls_optimal_fir(0.0, nu_b)
    assert np.allclose(h0, np.eye(8)[3], atol=1e-12) and abs(e0) < 1e-12
    for f in np.linspace(0.05, 0.95, 10):
        h, e = mlp.ls_optimal_fir(f, nu_b)
        assert e >= -1e-15
        for beta in (4.0, 6.0):
            wk = oracle.kaiser_sinc_weights(f, 8, beta)
            assert mlp.fir_mse(wk, f, nu_b) >= e - 1e-15
        assert abs(mlp.fir_mse(h, f, nu_b) - e) < 1e-12


def test_fir_mse_against_monte_carlo():
    """fir_mse against a Monte-Carlo estimate on band-limited noise, with the
    exact fractional value from an FFT phase ramp (exact for periodic
    band-limited sequences)."""
    nu_b = synth.NU_BAND
    n = 4096
    x = synth.bandlimited_noise((8, n), nu_b, 1.0, 5)
    f = 0.37
    nu = np.fft.fftfreq(n)
    xf = np.fft.ifft(np.fft.fft(x, axis=-1) * np.exp(2j * np.pi * nu * f), axis=-1)
    k = np.arange(8) - 3
    for h in (oracle.kaiser_sinc_weights(f, 8, 4.0), mlp.ls_optimal_fir(f, nu_b)[0]):
        est = np.zeros_like(x)
        for m, kk in enumerate(k):
            est += h[m] * np.roll(x, -kk, axis=-1)
        mc = np.mean(np.abs(est - xf) ** 2)
        an = mlp.fir_mse(h, f, nu_b)
        assert abs(mc - an) <= 0.1 * an + 1e-9


def test_interp_taps_prior_plus_network():
    """With a zero network the learned interpolator's taps are its prior, the
    normalised Kaiser-sinc (unit sum at every fraction); without a prior they
    are the network's output alone."""
    import oracle
    f = np.linspace(0.0, 0.999, 37)
    zero = np.zeros(mlp.N_PARAMS)
    t = mlp.interp_taps(zero, f, 4.0)
    assert np.allclose(t.sum(axis=1), 1.0, atol=1e-13)
    assert np.allclose(t[5], oracle.kaiser_sinc_weights(f[5], 8, 4.0), atol=1e-15)
    theta = np.random.default_rng(3).normal(0.0, 0.1, mlp.N_PARAMS)
    assert np.allclose(mlp.interp_taps(theta, f, -1.0), mlp.forward(theta, f)[0])
    assert np.allclose(mlp.interp_taps(theta, f, 6.0) - mlp.interp_taps(zero, f, 6.0), mlp.forward(theta, f)[0])
