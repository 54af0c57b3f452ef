"""GPU parity of continuous receiver motion during reception (Sec. II-D: the
platform keeps moving while the echo comes in; the two-way delay solves
c tau = |x - x_TX| + |x - x_RX - v tau|).  The kernels solve the fixed point
in FP64 at each tile centre and correct each pixel to first order in the
receiver's displacement (about a millimetre); the oracle solves every term
to convergence in FP64."""
import numpy as np
import pytest

import oracle
import paper_2101_05888_gb300 as sas
from paper_2101_05888_gb300 import synth

from _scene import grid_pixels, in_band, lib_signal, oracle_positions, oracle_signal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BETA = 4.0


def _stripmap(nx=200, ny=100, P=64, C=4, x0=2.0, y0=40.0):
    # 1.95 m/s along-track plus sway/heave rates; pixels 40 m out on the seabed
    g = synth.Grid(x0, y0, 0.0, 0.02, 0.02, 0.0, nx, ny, 1)
    w = synth.workload("stripmap_2d", grid=g, n_pings=P, n_rx=C, n_samples=4096, t0=0.05)
    nav = synth.nav(w)
    assert np.abs(nav["vel"][:, 0] - 1.95).max() == 0.0
    return w, nav


def test_forward_2d_with_motion_matches_oracle():
    w, nav = _stripmap()
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=51)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.set_velocity(nav["vel"])
    geom.upload_echo(echo)
    img = geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA)).cpu().numpy()
    geom.sync_status()
    tx, rx = oracle_positions(nav)
    pix = grid_pixels(w.grid)
    ref = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, pix, vel=nav["vel"]).reshape(img.shape)
    assert oracle.rel_l2(img, ref) < 1e-4
    # the model matters: stop-and-hop differs by far more than the tolerance
    sh = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, pix[:3000])
    assert oracle.rel_l2(ref.reshape(-1)[:3000], sh) > 0.1
    # and switching the velocity off returns to stop-and-hop
    geom.set_velocity(None)
    img0 = geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA)).cpu().numpy().reshape(-1)
    assert oracle.rel_l2(img0[:3000], sh) < 1e-4
    geom.close()


def test_forward_3d_with_motion_and_16bit():
    g = synth.Grid(0.5, 2.0, 0.0, 0.05, 0.05, 0.05, 40, 30, 10)
    w = synth.workload("volume_3d", grid=g, n_pings=16, n_rx=4, n_samples=2048, lattice=4, lattice_pitch=1.0,
                       echo_dtype="c64")
    nav = synth.nav(w)
    vel = np.tile([0.6, -0.4, 0.15], (w.n_pings, 1))       # surface craft drifting during reception
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=52)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.set_velocity(vel)
    geom.upload_echo(echo)
    img = geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA)).cpu().numpy()
    tx, rx = oracle_positions(nav)
    ref = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, grid_pixels(w.grid),
                             vel=vel).reshape(img.shape)
    assert oracle.rel_l2(img, ref) < 1e-4
    geom.upload_echo(echo, sas.SAS_ECHO_C32_F16)
    img16 = geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA)).cpu().numpy()
    geom.sync_status()
    assert oracle.rel_l2(img16, ref) < 3e-3
    geom.close()


def test_adjoint_and_offset_gradient_with_motion():
    w, nav = _stripmap(nx=96, ny=64, P=32, C=2)
    g = w.grid
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.set_velocity(nav["vel"])
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=53)
    geom.upload_echo(echo)
    G = synth.random_image((1, g.ny, g.nx), seed=54).astype(np.complex64)
    eadj = torch.empty((w.n_pings, w.n_rx, w.n_samples), dtype=torch.complex64, device="cuda")
    grad = torch.empty((w.n_pings, 3), dtype=torch.float64, device="cuda")
    img = geom.backproject(sas.grid_from(g), sas.kaiser(BETA)).cpu().numpy()
    sas.sas_backproject_adjoint(geom.h, sas.grid_from(g), sas.kaiser(BETA), torch.from_numpy(G).cuda(), eadj, grad)
    geom.sync_status()
    Be, Gv = img.reshape(-1).astype(np.complex128), G.reshape(-1).astype(np.complex128)
    lhs = np.vdot(Be, Gv)
    rhs = np.vdot(echo.reshape(-1).astype(np.complex128), eadj.cpu().numpy().reshape(-1).astype(np.complex128))
    # scale of a random inner product: see test_gpu_dot_product
    assert abs(lhs - rhs) <= 2e-5 * np.linalg.norm(Be) * np.linalg.norm(Gv) / np.sqrt(Gv.size)
    tx, rx = oracle_positions(nav)
    pix = grid_pixels(g)
    ref_adj = oracle.backproject_adjoint(tx, rx, oracle_signal(w), G.reshape(-1), 8, BETA, pix, vel=nav["vel"])
    got_adj = eadj.cpu().numpy()
    # in band at the FP32 tolerance; the full band carries the Farrow form's weight error
    assert oracle.rel_l2(in_band(got_adj), in_band(ref_adj)) < 1e-4
    assert oracle.rel_l2(got_adj, ref_adj) < 1e-3
    ref_grad = oracle.vjp_offsets(tx, rx, oracle_signal(w), echo, 8, BETA, pix, G.reshape(-1), vel=nav["vel"])
    assert oracle.rel_l2(grad.cpu().numpy(), ref_grad) < 1e-3
    geom.close()


def test_simulator_with_motion_matches_oracle():
    w = synth.scaled(synth.workload("small_2d"), n_pings=8, n_rx=3, n_samples=1024)
    nav = synth.nav(w)
    scat = synth.scatterers(w)
    geom = sas.Geometry(nav["true_pos"], nav["att"], nav["tx_lever"], nav["rx_lever"], lib_signal(w))
    geom.set_velocity(nav["vel"])
    echo = torch.zeros((w.n_pings, w.n_rx, w.n_samples), dtype=torch.complex64, device="cuda")
    sas.sas_simulate_points(geom.h, torch.from_numpy(scat).cuda(), len(scat), synth.BANDWIDTH, synth.PULSE_T, 0, echo)
    geom.sync_status()
    tx, rx = oracle_positions(nav, true=True)
    ref = oracle.simulate_points(tx, rx, oracle_signal(w), synth.BANDWIDTH, synth.PULSE_T, scat, vel=nav["vel"])
    assert oracle.rel_l2(echo.cpu().numpy(), ref) < 2e-5
    geom.close()


def test_motion_with_beam_matches_oracle():
    """Beam tests keep the ping-time sensor positions; delays use the motion."""
    w, nav = _stripmap(nx=300, ny=80, P=100, C=4, x0=4.0)
    width = np.deg2rad(20.0)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=55)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.set_velocity(nav["vel"])
    geom.set_beam(width, 1)
    geom.upload_echo(echo)
    img = geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA)).cpu().numpy().reshape(-1)
    geom.sync_status()
    tx, rx = oracle_positions(nav)
    sure, amb = oracle.backproject_beam_split(tx, rx, oracle_signal(w), echo, 8, BETA, grid_pixels(w.grid),
                                              nav["att"], width, 1, eps=2e-6, vel=nav["vel"])
    clean = amb == 0.0
    assert clean.mean() > 0.98
    assert oracle.rel_l2(img[clean], sure[clean]) < 1e-4
    scale = np.sqrt(np.mean(np.abs(sure) ** 2))
    assert np.all(np.abs(img[~clean] - sure[~clean]) <= amb[~clean] + 1e-4 * scale)
    geom.close()
