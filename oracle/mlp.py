"""FP64 restatement of the learned fractional-delay interpolator.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper has no learned component; the interpolator network is an addition
whose shape is fixed by the workload definition: an MLP 1 -> 64 -> 64 -> 8 with
GELU activations and FP16-stored weights, mapping the fractional sample
position f in [0, 1) to the 8 taps applied at offsets k = -3 .. 4 from floor(u)
(the same slot the Kaiser-sinc weights fill in the backprojection sum of
Sec. II-A).

Network (all maths here in FP64, weights as given, usually FP16-rounded):
    x  = 2 f - 1
    a1 = gelu(W1 x + b1)            W1 [64,1], b1 [64]
    a2 = gelu(W2 a1 + b2)           W2 [64,64] ([out][in]), b2 [64]
    t  = W3 a2 + b3                 W3 [8,64], b3 [8]
    gelu(z) = z/2 (1 + erf(z / sqrt 2))   (exact erf form)
Flat parameter vector order: W1, b1, W2, b2, W3, b3 (4808 values).

Loss on a batch of windows s_b [8] (complex) with targets y_b:
    L = (1/B) sum_b | sum_m t_m(f_b) s_b,m - y_b |^2
Optimiser: Adam (Kingma & Ba, 2015) with bias correction.

Interpolator taps with a prior (``interp_taps``): the normalised 8-tap
Kaiser-windowed sinc at beta_p plus the network's output t, the network
trained on residual targets y_b - sum_m k_m(f_b) s_b,m (k the prior's taps),
so that L above is the squared error of prior + network; without a prior
(beta_p < 0) the taps are t.

Also: the least-squares-optimal 8-tap FIR for a wide-sense-stationary signal
with flat spectrum on |nu| <= nu_b (cycles/sample), autocorrelation
r(tau) = sinc(2 nu_b tau), from the normal equations R h = p.
"""
from __future__ import annotations

import math

import numpy as np

try:
    from scipy.special import erf as _erf
except Exception:  # pragma: no cover - scipy is present on both machines
    _erf = np.vectorize(math.erf)

H = 64
TAPS = 8
SHAPES = [("W1", (H, 1)), ("b1", (H,)), ("W2", (H, H)), ("b2", (H,)), ("W3", (TAPS, H)),
          ("b3", (TAPS,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    theta = np.asarray(theta, dtype=np.float64).reshape(-1)
    assert theta.size == N_PARAMS
    out, o = {}, 0
    for name, shp in SHAPES:
        n = int(np.prod(shp))
        out[name] = theta[o:o + n].reshape(shp)
        o += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=np.float64).reshape(-1) for name, _ in SHAPES])


def gelu(z):
    return 0.5 * z * (1.0 + _erf(z / math.sqrt(2.0)))


def gelu_grad(z):
    return 0.5 * (1.0 + _erf(z / math.sqrt(2.0))) + z * np.exp(-0.5 * z * z) / math.sqrt(2.0 * math.pi)


def forward(theta, f):
    """Taps t [n, 8] for fractions f [n]; also returns the activations."""
    p = unpack(theta)
    x = 2.0 * np.asarray(f, dtype=np.float64).reshape(-1, 1) - 1.0
    z1 = x @ p["W1"].T + p["b1"]
    a1 = gelu(z1)
    z2 = a1 @ p["W2"].T + p["b2"]
    a2 = gelu(z2)
    t = a2 @ p["W3"].T + p["b3"]
    return t, (x, z1, a1, z2, a2)


def interp_taps(theta, f, prior_beta: float):
    """Taps [n, 8] of the learned interpolator at fractions f [n]: the
    prior's Kaiser-sinc taps (FP64, none if prior_beta < 0) plus the network's."""
    t, _ = forward(theta, f)
    if prior_beta >= 0:
        import oracle
        t = t + np.stack([oracle.kaiser_sinc_weights(float(x), TAPS, prior_beta)
                          for x in np.asarray(f, dtype=np.float64).reshape(-1)])
    return t


def loss_and_grad(theta, f, windows, targets):
    """Mean squared complex error and its gradient w.r.t. the flat parameters."""
    p = unpack(theta)
    t, (x, z1, a1, z2, a2) = forward(theta, f)
    s = np.asarray(windows, dtype=np.complex128).reshape(-1, TAPS)
    y = np.asarray(targets, dtype=np.complex128).reshape(-1)
    B = s.shape[0]
    r = (t * s).sum(axis=1) - y
    L = float(np.mean(np.abs(r) ** 2))
    dt = (2.0 / B) * np.real(np.conj(r)[:, None] * s)               # [B,8]
    g = {}
    g["W3"] = dt.T @ a2
    g["b3"] = dt.sum(0)
    dz2 = (dt @ p["W3"]) * gelu_grad(z2)
    g["W2"] = dz2.T @ a1
    g["b2"] = dz2.sum(0)
    dz1 = (dz2 @ p["W2"]) * gelu_grad(z1)
    g["W1"] = dz1.T @ x
    g["b1"] = dz1.sum(0)
    return L, pack(g)


def adam_step(theta, grad, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (step counts from 1); returns new (theta, m, v)."""
    m = beta1 * m + (1.0 - beta1) * grad
    v = beta2 * v + (1.0 - beta2) * grad * grad
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v


def flat_band_autocorr(tau, nu_b):
    return np.sinc(2.0 * nu_b * np.asarray(tau, dtype=np.float64))


def fir_mse(h, f, nu_b, taps=TAPS):
    """Expected squared error of FIR taps h [taps] interpolating at fraction f a
    unit-power signal with flat spectrum on |nu| <= nu_b."""
    k = np.arange(taps) - taps // 2 + 1
    R = flat_band_autocorr(k[:, None] - k[None, :], nu_b)
    p = flat_band_autocorr(f - k, nu_b)
    h = np.asarray(h, dtype=np.float64)
    return float(1.0 - 2.0 * h @ p + h @ R @ h)


def ls_optimal_fir(f, nu_b, taps=TAPS):
    """Least-squares-optimal taps and their mean-square error at fraction f."""
    k = np.arange(taps) - taps // 2 + 1
    R = flat_band_autocorr(k[:, None] - k[None, :], nu_b)
    p = flat_band_autocorr(f - k, nu_b)
    h = np.linalg.solve(R, p)
    return h, float(1.0 - p @ h)
