"""Pins for the oracle's Kaiser-windowed-sinc interpolator."""
import numpy as np
import pytest
from scipy.special import i0, i1

import oracle
from oracle import brute


@pytest.mark.parametrize("x", [0.0, 1e-3, 0.5, 1.0, 2.5, 4.0, 8.0, 10.0, 20.0])
def test_bessel_series_against_scipy(x):
    assert abs(oracle.bessel_i0(x) - i0(x)) <= 1e-14 * i0(x)
    if x > 0:
        assert abs(oracle.bessel_i1_over_x(x) - i1(x) / x) <= 1e-14 * (i1(x) / x)
    else:
        assert oracle.bessel_i1_over_x(0.0) == 0.5


@pytest.mark.parametrize("taps,beta", [(8, 4.0), (8, 6.0), (32, 10.0)])
def test_integer_position_is_identity(taps, beta):
    w = oracle.kaiser_sinc_weights(0.0, taps, beta)
    e = np.zeros(taps)
    e[taps // 2 - 1] = 1.0     # tap offset k = 0
    assert np.max(np.abs(w - e)) < 1e-15   # sin(pi k) rounds to ~1e-17, not 0


@pytest.mark.parametrize("taps,beta", [(8, 4.0), (32, 10.0)])
def test_unit_sum_symmetry_continuity(taps, beta):
    for f in np.linspace(0, 1, 37)[:-1]:
        w = oracle.kaiser_sinc_weights(f, taps, beta)
        assert abs(w.sum() - 1.0) < 1e-14
        # mirror: w_m(f) = w_{N-1-m}(1-f) (with the tap set re-centred)
        if f > 0:
            wm = oracle.kaiser_sinc_weights(1.0 - f, taps, beta)
            assert np.allclose(w, wm[::-1], atol=1e-14)
    # f -> 1 equals f = 0 with the taps shifted by one sample
    w1 = oracle.kaiser_sinc_weights(1.0 - 1e-13, taps, beta)
    w0 = oracle.kaiser_sinc_weights(0.0, taps, beta)
    assert np.allclose(w1[1:], w0[:-1], atol=1e-11) and abs(w1[0]) < 1e-11


@pytest.mark.parametrize("taps,beta", [(8, 4.0), (32, 10.0)])
def test_weights_match_scipy_restatement(taps, beta):
    f = np.linspace(0, 1, 101)[:-1]
    wb = brute.weights(f, taps, beta)
    for i, ff in enumerate(f):
        assert np.allclose(oracle.kaiser_sinc_weights(ff, taps, beta), wb[i], atol=1e-14)


@pytest.mark.parametrize("taps,beta", [(8, 4.0), (32, 10.0)])
def test_weight_derivative_central_difference(taps, beta):
    h = 1e-6
    for f in np.linspace(0.01, 0.99, 23):
        _, dw = oracle.kaiser_sinc_weights(f, taps, beta, deriv=True)
        fd = (oracle.kaiser_sinc_weights(f + h, taps, beta) - oracle.kaiser_sinc_weights(f - h, taps, beta)) / (2 * h)
        assert np.allclose(dw, fd, atol=2e-8)


def _tone_error(taps, beta, nu_max=0.25):
    k = oracle.tap_offsets(taps)
    err = 0.0
    for nu in np.linspace(-nu_max, nu_max, 41):
        for f in np.linspace(0, 1, 33)[:-1]:
            w = oracle.kaiser_sinc_weights(f, taps, beta)
            err = max(err, abs(np.dot(w, np.exp(2j * np.pi * nu * k)) - np.exp(2j * np.pi * nu * f)))
    return err


def test_truth_interpolator_tone_error():
    """The 32-tap reference interpolator (beta = 10) reproduces any complex tone
    inside the echo band (|nu| <= B/(2 fs) = 0.25, i.e. 2x oversampled) to 1e-5."""
    assert _tone_error(32, 10.0) < 1e-5


def test_hot_path_interpolator_tone_error():
    """8 taps, beta = 4: worst tone error about 1e-2 inside the band."""
    e = _tone_error(8, 4.0)
    assert 5e-3 < e < 1.2e-2
