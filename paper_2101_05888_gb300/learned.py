"""Learned fractional-delay interpolator: training driver and tabulation.

The network (MLP 1 -> 64 -> 64 -> 8, GELU, FP16-stored weights) maps the
fractional sample position f to a correction of the 8 taps the backprojector
applies at offsets -3 .. 4 from floor(u): the interpolator is the plain 8-tap
Kaiser-sinc (beta = PRIOR_BETA, the hot path's default) plus the network's
output.  It is trained, with the library's own forward, backward and Adam
kernels, to reproduce the 32-tap Kaiser-windowed-sinc interpolation of echo
windows produced by the library's own echo simulator (the targets are the
residual of that interpolation over the prior's), then tabulated (prior +
network) at table_n + 1 fractions and handed to the backprojection kernels
through the interpolator table slot (SAS_INTERP_TABLE).  The plain
Kaiser-sinc stays available as the fallback, and the 32-tap Kaiser-sinc is the
reference its error is measured against.

Learning the correction rather than the taps themselves keeps the network's
outputs small, so the FP16 rounding of its weights and its fitting error cost
little in absolute terms: on a flat band at a quarter of the sample rate the
learned taps come within a small factor of the least-squares-optimal 8-tap
filter, where a network that outputs the taps directly stays an order of
magnitude above the best Kaiser window.

The host only schedules kernels and draws seeded random numbers.
"""
from __future__ import annotations

import math

import numpy as np
import torch

import paper_2101_05888_gb300 as sas
from paper_2101_05888_gb300 import synth

N_PARAMS = sas.SAS_MLP_NPARAMS
H = 64
PRIOR_BETA = 4.0       # the prior: the plain 8-tap Kaiser-sinc of the hot path
TRAIN_STEPS = 10000


def init_params(seed: int = 0, residual: bool = True) -> torch.Tensor:
    """Seeded initial FP32 master parameters on the device.  First-layer
    biases spread the GELU knees over x in [-1, 1]; the output starts near
    zero (a correction of the prior), or, without a prior, at linear
    interpolation at f = 1/2."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0.0, 3.0, (H, 1))
    b1 = rng.uniform(-3.0, 3.0, H)
    W2 = rng.normal(0.0, 1.0 / math.sqrt(H), (H, H))
    b2 = rng.normal(0.0, 0.1, H)
    W3 = rng.normal(0.0, (0.001 if residual else 0.1) / math.sqrt(H), (8, H))
    b3 = np.zeros(8)
    if not residual:
        b3[3] = b3[4] = 0.5
    theta = np.concatenate([W1.reshape(-1), b1, W2.reshape(-1), b2, W3.reshape(-1), b3]).astype(np.float32)
    assert theta.size == N_PARAMS
    return torch.from_numpy(theta).cuda()


def training_echo(w, n_scatterers: int = 4000, seed: int = 0, snr_db: float = 20.0) -> torch.Tensor:
    """Echoes of a random scene in the given workload's geometry, from the
    library's simulator: point scatterers with complex Gaussian amplitudes over
    the grid's patch (a speckle-like field), matched-filtered LFM pulses, plus
    band-limited noise.  Returns device complex64 [P*C, Ns]."""
    rng = np.random.default_rng(seed)
    g = w.grid
    xs = rng.uniform(g.x0, g.x0 + g.nx * g.dx, n_scatterers)
    ys = rng.uniform(g.y0, g.y0 + g.ny * g.dy, n_scatterers)
    amp = (rng.standard_normal(n_scatterers) + 1j * rng.standard_normal(n_scatterers)) / math.sqrt(2.0)
    scat = np.stack([xs, ys, np.zeros(n_scatterers), amp.real, amp.imag], 1)
    nav = synth.nav(w, seed_offset=seed + 1)
    geom = sas.Geometry(nav["true_pos"], nav["att"], nav["tx_lever"], nav["rx_lever"],
                        sas.make_signal(synth.FC, synth.FS, synth.C_SOUND, w.t0, w.n_samples))
    echo = torch.zeros((w.n_pings * w.n_rx, w.n_samples), dtype=torch.complex64, device="cuda")
    sas.sas_simulate_points(geom.h, torch.from_numpy(scat).cuda(), n_scatterers, synth.BANDWIDTH, synth.PULSE_T,
                            256, echo)
    torch.cuda.synchronize()
    geom.close()
    p = float(torch.mean(echo.abs() ** 2).item())
    noise = synth.bandlimited_noise((w.n_pings * w.n_rx, w.n_samples), synth.NU_BAND,
                                    p / 10.0 ** (snr_db / 10.0), seed + 2)
    return echo + torch.from_numpy(noise.astype(np.complex64)).cuda()


def training_set(echo: torch.Tensor, n: int, seed: int = 0, target_beta: float = 10.0, margin: int = 24,
                 prior_beta: float = PRIOR_BETA):
    """n (fraction, 8-sample window, 32-tap target less the prior's 8-tap
    interpolation) draws from the echo rows."""
    rows, Ns = echo.shape
    frac, row, pos = synth.training_draws(n, rows, margin, Ns - margin, seed)
    d_frac = torch.from_numpy(frac.astype(np.float32)).cuda()
    d_row = torch.from_numpy(row.astype(np.int32)).cuda()
    d_pos = torch.from_numpy(pos.astype(np.int32)).cuda()
    win = torch.empty((n, 8), dtype=torch.complex64, device="cuda")
    tgt = torch.empty((n,), dtype=torch.complex64, device="cuda")
    sas.sas_mlp_make_windows(echo.contiguous(), rows, Ns, d_frac, d_row, d_pos, n, target_beta, prior_beta, win,
                             tgt)
    return d_frac, win, tgt


def train(frac, win, tgt, steps: int = TRAIN_STEPS, batch: int = 8192, lr: float = 3e-3, lr_final: float = 3e-5,
          seed: int = 0, theta=None):
    """Adam on mean squared interpolation error; cosine learning-rate decay.
    Returns (theta, loss history)."""
    n = frac.numel()
    theta = init_params(seed) if theta is None else theta.clone()
    m = torch.zeros_like(theta)
    v = torch.zeros_like(theta)
    grad = torch.empty_like(theta)
    loss = torch.empty(1, dtype=torch.float32, device="cuda")
    work = torch.empty(sas.sas_mlp_workspace_bytes(batch), dtype=torch.uint8, device="cuda")
    hist = []
    nb = max(1, n // batch)
    for k in range(steps):
        b = k % nb
        sl = slice(b * batch, (b + 1) * batch)
        sas.sas_mlp_loss_grad(theta, frac[sl], win[sl], tgt[sl], batch, loss, grad, work)
        a = lr_final + 0.5 * (lr - lr_final) * (1.0 + math.cos(math.pi * k / max(1, steps - 1)))
        sas.sas_mlp_adam(theta, grad, m, v, k + 1, a)
        if k % 50 == 0 or k == steps - 1:
            hist.append(float(loss.item()))
    return theta, hist


def tabulate(theta: torch.Tensor, table_n: int = 4096, prior_beta: float = PRIOR_BETA) -> torch.Tensor:
    table = torch.empty((table_n + 1, 8), dtype=torch.float32, device="cuda")
    sas.sas_interp_tabulate_mlp(theta, table_n, prior_beta, table)
    return table


def trained_table(table_n: int = 4096, n_windows: int = 1_000_000, steps: int = TRAIN_STEPS, seed: int = 7):
    """The learned-interpolator workload's network, trained from scratch:
    simulator echoes in the small-2D geometry (4000-point speckle-like scene,
    20 dB band-limited noise), n_windows training windows, steps Adam steps;
    returns (table, loss history)."""
    echo = training_echo(synth.workload("small_2d", seed=4321), seed=seed)
    frac, win, tgt = training_set(echo, n_windows, seed=seed + 1)
    theta, hist = train(frac, win, tgt, steps=steps)
    return tabulate(theta, table_n), hist


def interp_from_table(table: torch.Tensor) -> sas.sas_interp:
    return sas.table_interp(table, table.shape[0] - 1)
