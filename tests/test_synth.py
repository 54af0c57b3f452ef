"""The seeded synthetic inputs that stand in for the paper's data (its
stripmap survey, sub-bottom volume and timing set are not available): the
workload shapes, the determinism of every generator in its seed, the
band limit and power of the echo rows, and the platform-motion recipe."""
import numpy as np
import pytest

from paper_2101_05888_gb300 import synth


@pytest.mark.parametrize("name,shape,grid,pixel", [
    ("stripmap_2d", (2048, 32, 16384), (4096, 4096, 1), 0.015),
    ("volume_3d", (1024, 64, 8192), (1024, 1024, 128), 0.02),
    ("small_2d", (128, 4, 2048), (256, 256, 1), 0.02),
    ("autofocus_2d", (1024, 16, 8192), (2048, 2048, 1), 0.015),
])
def test_workload_shapes(name, shape, grid, pixel):
    w = synth.workload(name)
    assert (w.n_pings, w.n_rx, w.n_samples) == shape
    assert (w.grid.nx, w.grid.ny, w.grid.nz) == grid and w.grid.dx == pixel
    assert w.updates == w.grid.nx * w.grid.ny * w.grid.nz * w.n_pings * w.n_rx


def test_random_echo_is_seeded_band_limited_and_unit_power():
    a = synth.random_echo(3, 4, 1024, seed=7)
    assert a.shape == (3, 4, 1024) and a.dtype == np.complex64
    assert np.array_equal(a, synth.random_echo(3, 4, 1024, seed=7))
    assert not np.array_equal(a, synth.random_echo(3, 4, 1024, seed=8))
    spec = np.abs(np.fft.fft(a.astype(np.complex128), axis=-1)) ** 2
    nu = np.fft.fftfreq(1024)
    outside = spec[..., np.abs(nu) > synth.NU_BAND].sum() / spec.sum()
    assert outside < 1e-12                          # circular shift and phase keep the band limit
    assert abs(np.mean(np.abs(a) ** 2) - 1.0) < 0.1


def test_stripmap_motion_recipe():
    w = synth.workload("stripmap_2d")
    nav = synth.nav(w)
    pos, vel, att = nav["pos"], nav["vel"], nav["att"]
    assert np.array_equal(pos, synth.nav(w)["pos"])                      # seeded
    assert np.abs(pos[:, 1]).max() <= 0.05 + 1e-12                       # sway +-5 cm
    assert np.abs(pos[:, 2] + w.altitude).max() <= 0.05 + 1e-12          # heave +-5 cm
    assert np.abs(pos[:, 1]).max() > 0.04 and np.abs(pos[:, 2] + w.altitude).max() > 0.04
    assert np.allclose(np.diff(pos[:, 0]), w.ping_spacing)
    # the stated velocities are the sinusoids' rates: central differences over
    # periods of at least 20 pings agree to sin(w)/w >= 0.98
    pps = w.speed / w.ping_spacing
    for ax in (1, 2):
        fd = (pos[2:, ax] - pos[:-2, ax]) / 2.0 * pps
        assert np.abs(fd - vel[1:-1, ax]).max() <= 0.02 * np.abs(vel[:, ax]).max()
    assert np.allclose(vel[:, 0], w.speed)
    # yaw: a random walk of 0.01 deg steps
    steps = np.diff(att[:, 2])
    assert abs(np.std(steps) / np.deg2rad(0.01) - 1.0) < 0.1
    assert np.all(att[:, :2] == 0.0)
