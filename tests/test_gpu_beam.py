"""GPU parity of the beam field of view (Sec. II-C: pixels outside the
transmit or receive beam are not integrated; blocks of pixels that no beam
can see are culled).  The GPU culls (ping, channel, tile) blocks with a
conservative corner test and tests pixels on beam edges in FP32; the oracle
applies the per-pixel definition in FP64.  A term whose decision lies within
a relative 2e-6 of a beam edge can go either way in FP32, so the oracle
splits the image into the sure terms and the magnitudes of those ambiguous
ones: pixels without ambiguous terms are compared element by element, the
others must lie within their ambiguous mass.  The adjoint and gradient tests
give the pixels with ambiguous terms zero weight, which removes those terms
from both sides.  Grids are chosen so that many tiles are culled, many are
fully inside and many straddle a beam edge."""
import numpy as np
import pytest

import oracle
import paper_2101_05888_gb300 as sas
from paper_2101_05888_gb300 import synth

from _scene import grid_pixels, in_band, lib_signal, oracle_positions, oracle_signal

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

BETA = 4.0
EPS = 2e-6          # relative decision margin; the FP32 beam test errs by about 1e-7


def _stripmap(nx, ny, x0, y0, P, C):
    # track 0 .. 0.1 P m along x at 10 m altitude; pixels on the seabed at 40 m range
    g = synth.Grid(x0, y0, 0.0, 0.03, 0.03, 0.0, nx, ny, 1)
    w = synth.workload("stripmap_2d", grid=g, n_pings=P, n_rx=C, n_samples=4096, t0=0.05)
    return w, synth.nav(w)


def _check_split(got, sure, amb):
    """Clean pixels within 1e-4 (rel. L2), the rest within their ambiguous mass."""
    got, sure, amb = got.reshape(-1), sure.reshape(-1), amb.reshape(-1)
    clean = amb == 0.0
    assert clean.mean() > 0.98
    assert oracle.rel_l2(got[clean], sure[clean]) < 1e-4
    scale = np.sqrt(np.mean(np.abs(sure) ** 2))
    assert np.all(np.abs(got[~clean] - sure[~clean]) <= amb[~clean] + 1e-4 * scale)


@pytest.mark.parametrize("side", [1, -1])
def test_beam_forward_2d_matches_oracle(side):
    # track 0 .. 12 m, grid 4 .. 16 m along-track at 40 .. 43.6 m range: a 20
    # degree beam covers about +-7 m, so each ping culls, fully sees and cuts
    # through tiles; side -1 mirrors the grid to port
    y0 = 40.0 if side == 1 else -43.6
    w, nav = _stripmap(400, 120, 4.0, y0, 120, 4)
    width = np.deg2rad(20.0)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=41)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.set_beam(width, side)
    geom.upload_echo(echo)
    geom.cull_stats(reset=True)
    img = geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA))
    cand, computed, edge = geom.cull_stats()
    geom.sync_status()
    tiles = -(-w.grid.nx // 56) * -(-w.grid.ny // 32)
    assert cand == tiles * w.n_pings * w.n_rx
    assert 0 < edge < computed < cand                 # some culled, some on an edge
    tx, rx = oracle_positions(nav)
    pix = grid_pixels(w.grid)
    sure, amb = oracle.backproject_beam_split(tx, rx, oracle_signal(w), echo, 8, BETA, pix, nav["att"], width,
                                              side, eps=EPS)
    _check_split(img.cpu().numpy(), sure, amb)
    # the beam matters here: the unmasked image is different
    full = oracle.backproject(tx, rx, oracle_signal(w), echo, 8, BETA, pix[:2000])
    assert oracle.rel_l2(sure[:2000], full) > 0.1
    geom.close()


def test_beam_forward_3d_and_16bit():
    g = synth.Grid(0.5, 2.0, 0.0, 0.05, 0.05, 0.05, 60, 40, 12)
    w = synth.workload("volume_3d", grid=g, n_pings=16, n_rx=4, n_samples=2048, lattice=4, lattice_pitch=1.0,
                       echo_dtype="c64")
    nav = synth.nav(w)
    width = np.deg2rad(35.0)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=42)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.set_beam(width, 1)
    geom.upload_echo(echo)
    img = geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA)).cpu().numpy()
    tx, rx = oracle_positions(nav)
    sure, amb = oracle.backproject_beam_split(tx, rx, oracle_signal(w), echo, 8, BETA, grid_pixels(w.grid),
                                              nav["att"], width, 1, eps=EPS)
    _check_split(img, sure, amb)
    geom.upload_echo(echo, sas.SAS_ECHO_C32_F16)
    img16 = geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA)).cpu().numpy().reshape(-1)
    geom.sync_status()
    clean = amb == 0.0
    assert oracle.rel_l2(img16[clean], sure[clean]) < 3e-3
    geom.close()


def test_beam_off_counts_every_block():
    w, nav = _stripmap(120, 40, 4.0, 40.0, 16, 4)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.upload_echo(synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=45))
    geom.cull_stats(reset=True)
    geom.backproject(sas.grid_from(w.grid), sas.kaiser(BETA))
    cand, computed, edge = geom.cull_stats()
    tiles = -(-w.grid.nx // 56) * -(-w.grid.ny // 32)
    assert cand == computed == tiles * w.n_pings * w.n_rx and edge == 0
    geom.close()


def test_beam_adjoint_and_offset_gradient():
    # track 0 .. 4 m, grid 8 .. 12.8 m: the beam edge (about +-8.9 m at 40 m)
    # sweeps across the grid
    w, nav = _stripmap(160, 60, 8.0, 40.0, 40, 2)
    g = w.grid
    width = np.deg2rad(25.0)
    geom = sas.Geometry.from_nav(nav, lib_signal(w))
    geom.set_beam(width, 1)
    echo = synth.random_echo(w.n_pings, w.n_rx, w.n_samples, seed=43)
    geom.upload_echo(echo)
    tx, rx = oracle_positions(nav)
    pix = grid_pixels(g)
    _, amb = oracle.backproject_beam_split(tx, rx, oracle_signal(w), echo, 8, BETA, pix, nav["att"], width, 1,
                                           eps=EPS)
    G = synth.random_image((1, g.ny, g.nx), seed=44).astype(np.complex64)
    Gm = np.where(amb.reshape(G.shape) > 0, 0, G).astype(np.complex64)   # no weight on ambiguous pixels
    eadj = torch.empty((w.n_pings, w.n_rx, w.n_samples), dtype=torch.complex64, device="cuda")
    grad = torch.empty((w.n_pings, 3), dtype=torch.float64, device="cuda")
    img = geom.backproject(sas.grid_from(g), sas.kaiser(BETA)).cpu().numpy()
    # dot test with the full G: forward and adjoint take the same FP32 decisions
    # (one term decided differently would move <B e, G> by about 1; FP32
    # rounding moves it by ~1e-6 of a random inner product's size
    # |B e| |G| / sqrt(n))
    sas.sas_backproject_adjoint(geom.h, sas.grid_from(g), sas.kaiser(BETA), torch.from_numpy(G).cuda(), eadj, None)
    Be, Gv = img.reshape(-1).astype(np.complex128), G.reshape(-1).astype(np.complex128)
    lhs = np.vdot(Be, Gv)
    rhs = np.vdot(echo.reshape(-1).astype(np.complex128), eadj.cpu().numpy().reshape(-1).astype(np.complex128))
    assert abs(lhs - rhs) <= 2e-5 * np.linalg.norm(Be) * np.linalg.norm(Gv) / np.sqrt(Gv.size)
    # against the oracle with ambiguous pixels weighted zero
    sas.sas_backproject_adjoint(geom.h, sas.grid_from(g), sas.kaiser(BETA), torch.from_numpy(Gm).cuda(), eadj,
                                grad)
    geom.sync_status()
    kw = dict(att=nav["att"], beam_width=width, side=1)
    ref_adj = oracle.backproject_adjoint(tx, rx, oracle_signal(w), Gm.reshape(-1), 8, BETA, pix, **kw)
    got_adj = eadj.cpu().numpy()
    # in band at the FP32 tolerance; the full band carries the Farrow form's weight error
    assert oracle.rel_l2(in_band(got_adj), in_band(ref_adj)) < 1e-4
    assert oracle.rel_l2(got_adj, ref_adj) < 1e-3
    ref_grad = oracle.vjp_offsets(tx, rx, oracle_signal(w), echo, 8, BETA, pix, Gm.reshape(-1), **kw)
    assert oracle.rel_l2(grad.cpu().numpy(), ref_grad) < 1e-3
    geom.close()
